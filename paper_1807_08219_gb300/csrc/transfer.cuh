// transfer.cuh -- node binning, spreading S* and interpolation S
// (Sec. "Interpolation Scheme"; Algorithm steps 2 and 4), and the FP64
// conservation sums.
//
// Binning. Every node is assigned the cell c = floor(x n/L) of its box. For
// both kernels and all three MAC lattices its stencil lies inside cells
// c-2 .. c+2 per axis. Boxes are cut into tiles (edge t, the last tile per
// axis t..t+4 cells, never fewer than 5), so the stencil meets at most two
// tiles per axis. The binning writes
//   cand lists: for every tile, the nodes whose stencil meets it (spread);
//   own lists:  for every tile, the nodes whose cell lies in it (interp).
// Spreading is owner-computes: the CTA that owns a tile accumulates every
// contribution that lands in it and writes each touched value once, so no
// global atomics are needed and no value is written by two CTAs.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace ifem {

struct TileInfo {
    int box;
    int start[3];
    int edge[3];
};

__device__ inline int box_of_tile(const DevGrid &g, long long tile)
{
    int lo = 0, hi = g.n_boxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (g.boxes[mid].tile_base <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ inline TileInfo decode_tile(const DevGrid &g, long long tile)
{
    TileInfo ti;
    ti.box = box_of_tile(g, tile);
    const BoxDev &B = g.boxes[ti.box];
    long long local = tile - B.tile_base;
    int j[3] = {(int)(local % B.T), (int)((local / B.T) % B.T), (int)(local / ((long long)B.T * B.T))};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ti.start[a] = tile_start(j[a], B.t);
        ti.edge[a] = tile_edge(j[a], B.t, B.T, B.n);
    }
    return ti;
}

__device__ __forceinline__ float mac_off(int d, int a) { return a == d ? 0.f : 0.5f; }

// ---------------------------------------------------------------- binning
// Cell of a node from its coordinates xa (all finite: true, else the cell is
// zero from the first non-finite axis on); s receives the lattice coordinates.
template <typename real>
__device__ inline bool node_cell_xyz(const InstDev &I, const BoxDev &B, const real xa[3], int c[3], real s[3])
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ok = ok && isfinite(xa[a]);
        int I0;
        s[a] = LatCoord<real>::get(I, B, a, xa[a], real(0), I0);
        if constexpr (std::is_same<real, float>::value) {
            // 32-bit integer arithmetic while the cell is within 2^30 of the
            // particle's origin cell (every node near its box): with 64-bit
            // arithmetic for the cell and the own-list key the FP64 pipe was
            // 40 % busy in the binning pass
            const float fl = floorf(s[a]);
            if (fabsf(fl) < 1073741824.f && I0 > -1073741824 && I0 < 1073741824) {
                const int ci = I0 + (int)fl;
                int cw;
                if (ci >= 0 && ci < 2 * B.n) {
                    cw = ci >= B.n ? ci - B.n : ci;
                } else {
                    cw = ci % B.n;
                    cw += cw < 0 ? B.n : 0;
                }
                c[a] = ok ? cw : 0;
                continue;
            }
        }
        long long ci = (long long)I0 + (long long)floor(s[a]);
        int cw;
        if (ci >= 0 && ci < 2LL * B.n)
            cw = ci >= B.n ? (int)ci - B.n : (int)ci;
        else
            cw = wrapi(ci, B.n);
        c[a] = ok ? cw : 0;
    }
    return ok;
}

template <typename real>
__device__ inline bool node_cell(const InstDev &I, const BoxDev &B, const real *x, long long N, int node,
                                 int c[3])
{
    const real xa[3] = {x[node], x[N + node], x[2 * N + node]};
    real s[3];
    return node_cell_xyz<real>(I, B, xa, c, s);
}

// Own-list key of a cell: (tile, 4^3 sub-block of the tile). Nodes come out
// of the binning grouped by position, which keeps the gathers of
// neighbouring lanes on shared cache lines.
// 32-bit: the workspace holds fewer than 2^31 - 1 keys (n_tiles * kOwnSub3,
// checked when it is set up). r receives the cell within its tile.
__device__ __forceinline__ int own_key(const BoxDev &B, const int c[3], int r[3])
{
    int o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = tile_of(c[a], B.t, B.T);
        r[a] = c[a] - tile_start(o[a], B.t);
    }
    return ((int)B.tile_base + (o[2] * B.T + o[1]) * B.T + o[0]) * kOwnSub3 +
           ((r[2] >> 2) * kOwnSub + (r[1] >> 2)) * kOwnSub + (r[0] >> 2);
}

// Warp-aggregated list append: lanes with the same tile share one global
// atomic (count pass: the count; fill pass: the slot range). Every lane of
// the warp must call this (invalid lanes pass valid = false).
template <bool FILL>
__device__ __forceinline__ int agg_append(int *count, int *cursor, int *list, long long tile, bool valid,
                                           int node)
{
    const unsigned key = valid ? (unsigned)tile : 0xffffffffu;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (!valid)
        return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    if (!FILL) {
        if (lane == leader)
            atomicAdd(&count[tile], __popc(grp));
        return -1;
    }
    int base = 0;
    if (lane == leader)
        base = atomicAdd(&cursor[tile], __popc(grp));
    base = __shfl_sync(grp, base, leader);
    const int slot = base + __popc(grp & ((1u << lane) - 1u));
    list[slot] = node;
    return slot;
}

// One-pass own-list binning (FP32 halo path): per node its rank within its
// own-list key (the old value of the key's count, one atomic per group of
// lanes with the same key) and its record -- fractional lattice coordinates
// and cell within the tile, 8-bit x | y << 8 | z << 16 -- kept by node for
// own_scatter_kernel; the leader of each group also marks the key's tile as
// owning nodes. Nodes that are not finite or not in the box get the key -1
// and are counted in ST_DOMAIN. kBinPer nodes per thread, node
// (blockIdx.x * kBinPer + j) * blockDim.x + threadIdx.x of instance
// blockIdx.y, each phase's loads, atomics and stores issued for all of them
// before their results are used: with one node per thread the pass is a
// chain of dependent latencies.
constexpr int kBinPer = 4;
static __global__ void __launch_bounds__(256) own_count_kernel(DevBatch b, DevGrid g, DevWork w, const float *__restrict__ x)
{
    const InstDev I = b.inst[blockIdx.y];
    const BoxDev B = g.boxes[I.box];
    const long long N = b.N;
    const int lane = threadIdx.x & 31;
    int node[kBinPer];
    bool in[kBinPer];
    float xa[kBinPer][3];
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
        const int k = (blockIdx.x * kBinPer + j) * blockDim.x + threadIdx.x;
        in[j] = k < I.n_nodes;
        node[j] = I.node_off + (in[j] ? k : 0);
        xa[j][0] = xa[j][1] = xa[j][2] = 0.f;
        if (in[j]) {
            xa[j][0] = x[node[j]];
            xa[j][1] = x[N + node[j]];
            xa[j][2] = x[2 * N + node[j]];
        }
    }
    bool ok[kBinPer];
    int key[kBinPer];
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
        int c[3] = {0, 0, 0};
        float sl[3];
        ok[j] = in[j] && node_cell_xyz<float>(I, B, xa[j], c, sl);
        if (in[j] && !ok[j])
            status_add(w.status, ST_DOMAIN, 1);
        int r[3];
        key[j] = own_key(B, c, r);
        if (ok[j]) {
            const unsigned pk = (unsigned)r[0] | ((unsigned)r[1] << 8) | ((unsigned)r[2] << 16);
            w.node_rec[node[j]] = make_float4(sl[0] - floorf(sl[0]), sl[1] - floorf(sl[1]), sl[2] - floorf(sl[2]),
                                              __uint_as_float(pk));
        }
    }
    // every lane takes part in the votes and shuffles (invalid lanes form
    // their own group under the key 0xffffffff, which no valid key reaches)
    unsigned grp[kBinPer];
    int base[kBinPer];
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
        grp[j] = __match_any_sync(0xffffffffu, ok[j] ? (unsigned)key[j] : 0xffffffffu);
        base[j] = 0;
        if (ok[j] && lane == __ffs(grp[j]) - 1) {
            base[j] = atomicAdd(&w.own_count[key[j]], __popc(grp[j]));
            w.own_flag[key[j] / kOwnSub3] = 1;
        }
    }
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
        const int rank = __shfl_sync(0xffffffffu, base[j], __ffs(grp[j]) - 1) + __popc(grp[j] & ((1u << lane) - 1u));
        if (in[j])
            w.node_key[node[j]] = make_int2(ok[j] ? key[j] : -1, rank);
    }
}

// FILL = false: count candidate / own pairs per tile; FILL = true: write them
// (paths with candidate lists; the FP32 halo path bins with own_count_kernel
// and own_scatter_kernel). Block size must be a multiple of 32 (every lane
// reaches the warp votes).
template <typename real, bool FILL>
__global__ void bin_kernel(DevBatch b, DevGrid g, DevWork w, const real *__restrict__ x)
{
    const InstDev I = b.inst[blockIdx.y];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = k < I.n_nodes;
    const BoxDev B = g.boxes[I.box];
    const int node = I.node_off + (in ? k : 0);
    int c[3] = {0, 0, 0};
    bool ok = false;
    if (in) {
        ok = node_cell<real>(I, B, x, b.N, node, c);
        if (!FILL && !ok)
            status_add(w.status, ST_DOMAIN, 1);
    }
    int tl[3][2], nt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int lo = c[a] - 2, hi = c[a] + 2;
        lo += lo < 0 ? B.n : 0;
        hi -= hi >= B.n ? B.n : 0;
        tl[a][0] = tile_of(lo, B.t, B.T);
        tl[a][1] = tile_of(hi, B.t, B.T);
        nt[a] = tl[a][0] == tl[a][1] ? 1 : 2;
    }
    int r[3];
    agg_append<FILL>(w.own_count, w.own_cursor, w.own_nodes, own_key(B, c, r), ok, node);
#pragma unroll
    for (int slot = 0; slot < 8; ++slot) {
        const int ix = slot & 1, iy = (slot >> 1) & 1, iz = slot >> 2;
        const bool valid = ok && ix < nt[0] && iy < nt[1] && iz < nt[2];
        if (!__any_sync(0xffffffffu, valid))
            continue;   // most nodes meet one or two tiles: skip empty slots warp-wide
        const long long tile = B.tile_base + ((long long)tl[2][iz] * B.T + tl[1][iy]) * B.T + tl[0][ix];
        agg_append<FILL>(w.cand_count, w.cand_cursor, w.cand_nodes, tile, valid, node);
    }
}

// Exclusive scan of the per-tile counts (two lists at once): block-local
// scan, whose last block to finish scans the block sums -> add + cursors +
// active lists (scan_finish_kernel; in the FP32 halo path
// own_scatter_kernel adds the block offsets itself).

__device__ inline int block_exclusive_scan(int v, int *sh, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        sh[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? sh[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o)
                si += t;
        }
        if (lane < nw)
            sh[lane] = si - s;
        if (lane == nw - 1)
            sh[32] = si;
    }
    __syncthreads();
    int r = sh[wid] + incl - v;
    total = sh[32];
    __syncthreads();
    return r;
}

static __global__ void scan_local_kernel(long long n1, long long n2, const int *__restrict__ c1,
                                         const int *__restrict__ c2, int *__restrict__ o1, int *__restrict__ o2,
                                         int *__restrict__ bsum, int *__restrict__ ticket, int *__restrict__ totals)
{
    __shared__ int sh[33];
    __shared__ int last;
    long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanPer;
    int v1[kScanPer], v2[kScanPer], s1 = 0, s2 = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        long long i = base + q;
        v1[q] = i < n1 ? c1[i] : 0;
        v2[q] = i < n2 ? c2[i] : 0;
        s1 += v1[q];
        s2 += v2[q];
    }
    int t1, t2;
    int e1 = block_exclusive_scan(s1, sh, t1);
    int e2 = block_exclusive_scan(s2, sh, t2);
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        long long i = base + q;
        if (i < n1)
            o1[i] = e1;
        if (i < n2)
            o2[i] = e2;
        e1 += v1[q];
        e2 += v2[q];
    }
    // block sums out, then a ticket: the block that takes the last one sees
    // every block's sum (fence before the ticket, L2 loads after it)
    if (threadIdx.x == 0) {
        bsum[2 * blockIdx.x] = t1;
        bsum[2 * blockIdx.x + 1] = t2;
        __threadfence();
        last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last)
        return;
    __threadfence();
    const int nb = (int)gridDim.x;
    int run1 = 0, run2 = 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        const int u1 = i < nb ? __ldcg(&bsum[2 * i]) : 0, u2 = i < nb ? __ldcg(&bsum[2 * i + 1]) : 0;
        int w1, w2;
        const int x1 = block_exclusive_scan(u1, sh, w1);
        const int x2 = block_exclusive_scan(u2, sh, w2);
        if (i < nb) {
            bsum[2 * i] = x1 + run1;
            bsum[2 * i + 1] = x2 + run2;
        }
        run1 += w1;
        run2 += w2;
    }
    if (threadIdx.x == 0) {
        totals[0] = run1;
        totals[1] = run2;
    }
}

// n1 tiles (candidate lists), n2 own sub-blocks. Adds the block offsets,
// sets the fill cursors, writes the terminal offsets and the list of tiles
// with candidates (order irrelevant: tiles are processed independently).
static __global__ void scan_finish_kernel(long long n1, long long n2, DevWork w)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = n1 > n2 ? n1 : n2;
    if (i > n)
        return;
    const int blk = (int)(i / kScanBlock);
    if (i == n1)
        w.cand_off[n1] = w.counters[4];
    if (i == n2)
        w.own_off[n2] = w.counters[5];
    if (i < n2) {
        const int o2 = w.own_off[i] + w.scan_blocks[2 * blk + 1];
        w.own_off[i] = o2;
        w.own_cursor[i] = o2;
    }
    int c1 = 0;
    if (i < n1) {
        c1 = w.cand_count[i];
        const int o1 = w.cand_off[i] + w.scan_blocks[2 * blk];
        w.cand_off[i] = o1;
        w.cand_cursor[i] = o1;
    }
    const unsigned act = __activemask();
    const unsigned m1 = __ballot_sync(act, c1 > 0);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    int b1 = 0;
    if (lane == leader && m1)
        b1 = atomicAdd(&w.counters[0], __popc(m1));
    b1 = __shfl_sync(act, b1, leader);
    if (c1 > 0)
        w.active[b1 + __popc(m1 & ((1u << lane) - 1u))] = (int)i;
}

// Deterministic mode: sort each tile's candidate list by node id (bitonic
// sort in shared memory). Lists longer than kSortCap are flagged.
constexpr int kSortCap = 4096;
static __global__ void sort_segments_kernel(DevWork w)
{
    __shared__ int key[kSortCap];
    const int n_active = w.counters[0];
    for (int it = blockIdx.x; it < n_active; it += gridDim.x) {
        const int tile = w.active[it];
        const int beg = w.cand_off[tile], len = w.cand_off[tile + 1] - beg;
        if (len > kSortCap) {
            if (threadIdx.x == 0)
                status_add(w.status, ST_CAPACITY, 1);
            continue;
        }
        int P = 1;
        while (P < len)
            P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x)
            key[i] = i < len ? w.cand_nodes[beg + i] : 0x7fffffff;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    int l = i ^ j;
                    if (l > i) {
                        int a = key[i], bb = key[l];
                        bool up = (i & k) == 0;
                        if ((a > bb) == up) {
                            key[i] = bb;
                            key[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x)
            w.cand_nodes[beg + i] = key[i];
        __syncthreads();
    }
}

// --------------------------------------------------------- stencil per axis
// Peskin: i0 = floor(s) - 1 (relative to I0), phi[m] = phi4(s - (i0 + m)).
template <typename real>
__device__ __forceinline__ long long peskin_axis(real s, real ph[4])
{
    long long i0 = (long long)floor(s) - 1;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        ph[m] = phi4<real>(s - (real)(i0 + m));
    return i0;
}

// FP64 Peskin stencils of every node on the three lattices (thread per
// (node, lattice)), computed once after binning: the deterministic spread
// stages its candidates from this table instead of re-evaluating them for
// every tile a node reaches, and the step's interpolation reads it too. The
// values are those of peskin_axis<double> on the same coordinates (same
// expressions, same compilation), bit for bit. Non-finite nodes are never
// binned and their entries are left unwritten.
static __global__ void det_weights_kernel(DevBatch b, DevGrid g, DetW *__restrict__ wt, const double *__restrict__ x)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = b.N;
    if (t >= 3 * N)
        return;
    const long long node = t / 3;
    const int d = (int)(t - 3 * node);
    const InstDev I = b.inst[b.node_inst[node]];
    const BoxDev B = g.boxes[I.box];
    double xl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        xl[a] = x[a * N + node];
    if (!(isfinite(xl[0]) && isfinite(xl[1]) && isfinite(xl[2])))
        return;
    DetW &W = wt[node];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int I0;
        const double sa = LatCoord<double>::get(I, B, a, xl[a], (double)mac_off(d, a), I0);
        double ph[4];
        W.base[d][a] = wrapi(peskin_axis<double>(sa, ph), B.n);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            W.ph[d][a][m] = ph[m];
    }
    if (d == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int I0;
            const double sc = LatCoord<double>::get(I, B, a, xl[a], 0.0, I0);
            W.lo[a] = wrapi((long long)floor(sc) - 2, B.n);
        }
    }
}

// Per-thread partial sums as unevaluated float pairs (hi + lo, Knuth's
// TwoSum and the FMA product error): about 44 significant bits, at FP32
// speed; the FP64 pipe of this GPU is far narrower than its FP32 pipe.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_add(DF &x, float v)
{
    const float s = x.hi + v;
    const float bv = s - x.hi;
    const float e = (x.hi - (s - bv)) + (v - bv);
    const float t = x.lo + e;
    x.hi = s + t;
    x.lo = t - (x.hi - s);
}
// x += y for two float pairs, with both the high and the low sums made exact
// by TwoSum before renormalising (relative error a few 2^-48).
__device__ __forceinline__ void df_add_df(DF &x, DF y)
{
    const float s = x.hi + y.hi;
    const float bs = s - x.hi;
    float e = (x.hi - (s - bs)) + (y.hi - bs);
    const float t = x.lo + y.lo;
    const float bt = t - x.lo;
    const float f = (x.lo - (t - bt)) + (y.lo - bt);
    e += t;
    const float h = s + e;
    e = (e - (h - s)) + f;
    x.hi = h + e;
    x.lo = e - (x.hi - h);
}
__device__ __forceinline__ void df_add_prod(DF &x, float a, float b)
{
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    df_add(x, p);
    x.lo += pe;
}

// ---------------------------------------------------- spread, FP32 fast
// One CTA per active tile, tiles taken from a global counter. Contributions
// are accumulated in shared memory as fixed-point integers (Acc = int or
// long long) with native integer atomics: integer addition is associative,
// so the accumulated tile is independent of the order in which threads add
// (the FP32 result is reproducible run to run). Per tile and lattice the
// scale is a power of two chosen from a bound on the largest possible sum,
// |f_J| <= wmax * sum_k |g_k| over the tile's candidates, so no sum can
// overflow. Work units are (candidate node, lattice) pairs. Flush: one
// read-modify-write per non-zero owned value, rows of x in lanes.
template <typename Acc>
struct FixedPoint;
template <>
struct FixedPoint<int> {
    static constexpr float kRange = 1073741824.0f;  // 2^30
    __device__ static __forceinline__ int conv(float v) { return __float2int_rn(v); }
};
template <>
struct FixedPoint<long long> {
    static constexpr float kRange = 1152921504606846976.0f;  // 2^60
    __device__ static __forceinline__ long long conv(float v) { return __float2ll_rn(v); }
};

// The four Peskin weights of one axis share one square root: with
// r = s - floor(s) in [0, 1) and q = sqrt(1 + 4r - 4r^2),
//   phi(1 + r) = (3 - 2r - q)/8, phi(r) = (3 - 2r + q)/8,
//   phi(1 - r) = (1 + 2r + q)/8, phi(2 - r) = (1 + 2r - q)/8
// (the radicands of both branches of phi reduce to the same 1 + 4r - 4r^2,
// which lies in [1, 2], so sqrt(t) = t * rsqrt(t) needs no special cases).
// Used by the FP32 kernels; the FP64 kernels evaluate phi point by point.
__device__ __forceinline__ void peskin_frac(float r, float ph[4])
{
    const float t = 1.f + 4.f * r - 4.f * r * r;   // in [1, 2] for r in [0, 1)
    const float q = t * rsqrtf(t);
    ph[0] = (3.f - 2.f * r - q) * 0.125f;
    ph[1] = (3.f - 2.f * r + q) * 0.125f;
    ph[2] = (1.f + 2.f * r + q) * 0.125f;
    ph[3] = (1.f + 2.f * r - q) * 0.125f;
}
__device__ __forceinline__ int peskin_axis_fast(float s, float ph[4])
{
    const float fl = floorf(s);
    peskin_frac(s - fl, ph);
    return (int)fl - 1;
}

__device__ __forceinline__ void acc_add(int *p, int v) { atomicAdd(p, v); }

// Fire-and-forget adds performed at L2 (no value returned, so the SM does not
// wait for the line): the tile flush adds its sums to the grid this way.
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_global(p)), "f"(a),
                 "f"(b), "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void red_add(float *p, float a)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(a) : "memory");
}

// Shared-memory pitches of a tile accumulator: odd row and plane pitches
// spread the atomics of neighbouring nodes over the 32 banks.
__host__ __device__ inline int acc_px(int ex) { return ex | 1; }
__host__ __device__ inline int acc_pp(int ey, int px) { return (ey * px) | 1; }
__host__ __device__ inline int acc_stride(int ex, int ey, int ez) { return ez * acc_pp(ey, acc_px(ex)); }
// two's-complement addition through the unsigned 64-bit atomic
__device__ __forceinline__ void acc_add(long long *p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

// n-periodic wrap of an index that is normally already in (-n, 2n)
__device__ __forceinline__ int wrap_near(int v, int n)
{
    if (v < 0)
        v += n;
    else if (v >= n)
        v -= n;
    if ((unsigned)v >= (unsigned)n)
        v = wrapi(v, n);
    return v;
}

template <int KER, typename Acc>
__global__ void __launch_bounds__(256) spread_fast_kernel(DevBatch b, DevGrid g, DevWork w,
                                                          const float *__restrict__ x,
                                                          const float *__restrict__ F, float *__restrict__ f,
                                                          int density, float support)
{
    extern __shared__ __align__(16) unsigned char spread_smem[];
    Acc *acc = reinterpret_cast<Acc *>(spread_smem);
    __shared__ float s_part[3][8];
    __shared__ float s_scale[3];
    __shared__ double s_red[3][8];
    __shared__ int s_tile;
    __shared__ TileInfo s_ti;
    __shared__ BoxDev s_B;
    const long long N = b.N;
    const int n_active = w.counters[0];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status_add(w.status, ST_PAIRS, (unsigned long long)w.cand_off[g.n_tiles]);
        status_add(w.status, ST_ACTIVE, (unsigned long long)n_active);
    }
    // accumulators start at zero; the flush of every tile clears what it read
    {
        const int E = g.max_edge;
        for (int i = threadIdx.x; i < 3 * acc_stride(E, E, E); i += blockDim.x)
            acc[i] = 0;
    }
    for (;;) {
        if (threadIdx.x == 0) {
            int it = atomicAdd(&w.counters[2], 1);
            s_tile = it < n_active ? w.active[it] : -1;
            if (it < n_active) {
                s_ti = decode_tile(g, s_tile);
                s_B = g.boxes[s_ti.box];
            }
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0)
            break;
        const int ex = s_ti.edge[0], ey = s_ti.edge[1], ez = s_ti.edge[2];
        const int sx = s_ti.start[0], sy = s_ti.start[1], sz = s_ti.start[2];
        const int px = acc_px(ex), pp = acc_pp(ey, px);
        const int vol = ez * pp;   // per-lattice stride of the padded accumulator
        const int n = s_B.n;
        const float sd = density ? s_B.scale_f : 1.f;
        const double h3 = 1.0 / s_B.scale;
        const int beg = w.cand_off[tile], end = w.cand_off[tile + 1];
        // bound on |sum| per lattice: wmax * sum_k |F_k,d| * sd
        float gs0 = 0.f, gs1 = 0.f, gs2 = 0.f;
        for (int q = beg + threadIdx.x; q < end; q += blockDim.x) {
            const int node = w.cand_nodes[q];
            gs0 += fabsf(F[node]);
            gs1 += fabsf(F[N + node]);
            gs2 += fabsf(F[2 * N + node]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gs0 += __shfl_down_sync(0xffffffffu, gs0, o);
            gs1 += __shfl_down_sync(0xffffffffu, gs1, o);
            gs2 += __shfl_down_sync(0xffffffffu, gs2, o);
        }
        if (lane == 0) {
            s_part[0][wid] = gs0;
            s_part[1][wid] = gs1;
            s_part[2][wid] = gs2;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            float tot = 0.f;
            for (int q = 0; q < nw; ++q)
                tot += s_part[threadIdx.x][q];
            // |phi| <= 1/8 (Peskin: (1/2)^3); MLS weights are non-negative, sum to 1
            // and stay below 1/2 in practice; the bound sums over every candidate
            // of the tile, far above what any single value receives
            const float wmax = KER == 0 ? 0.125f : 0.5f;
            float bound = tot * sd * wmax * 1.0001f;
            float sc = 1.f;
            if (bound > 0.f && isfinite(bound)) {
                int e = (int)floorf(log2f(FixedPoint<Acc>::kRange / bound));
                e = e > 120 ? 120 : (e < -120 ? -120 : e);
                sc = exp2f((float)e);
            }
            s_scale[threadIdx.x] = sc;
        }
        __syncthreads();
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            Acc *accd = acc + d * vol;
            const float gsc = sd * s_scale[d];
            for (int q = beg + threadIdx.x; q < end; q += blockDim.x) {
                const int node = w.cand_nodes[q];
                const InstDev &I = b.inst[b.node_inst[node]];
                const float gq = F[d * N + node] * gsc;
                if constexpr (KER == 0) {
                    float ph[3][4];
                    int l[3][4];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int I0 = I.I0[a];
                        const float s = (I.f0[a] - (a == d ? 0.f : 0.5f)) + x[a * N + node] * s_B.inv_h_f;
                        const int base = wrap_near(I0 + peskin_axis_fast(s, ph[a]), n);
                        const int st = a == 0 ? sx : (a == 1 ? sy : sz);
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            int idx = base + m;
                            idx -= idx >= n ? n : 0;
                            l[a][m] = idx - st;
                        }
                    }
                    // validity bit masks; every slot runs, the atomic is predicated
                    // (no divergent branches around the 64 slots)
                    unsigned okx = 0, oky = 0, okz = 0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        okx |= (unsigned)((unsigned)l[0][m] < (unsigned)ex) << m;
                        oky |= (unsigned)((unsigned)l[1][m] < (unsigned)ey) << m;
                        okz |= (unsigned)((unsigned)l[2][m] < (unsigned)ez) << m;
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float wz = ph[2][c] * gq;
#pragma unroll
                        for (int bb = 0; bb < 4; ++bb) {
                            const float wyz = ph[1][bb] * wz;
                            const unsigned rowok = (okz >> c) & (oky >> bb) & 1u;
                            const int row = l[2][c] * pp + l[1][bb] * px;
#pragma unroll
                            for (int a = 0; a < 4; ++a) {
                                const Acc qv = FixedPoint<Acc>::conv(ph[0][a] * wyz);
                                if (rowok & (okx >> a))
                                    acc_add(accd + row + l[0][a], qv);
                            }
                        }
                    }
                } else {
                    float s[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        s[a] = (I.f0[a] - (a == d ? 0.f : 0.5f)) + x[a * N + node] * s_B.inv_h_f;
                    int base[3];
                    float wt[27];
                    if (!mls_weights<float>(s, support, base, wt)) {
                        status_add(w.status, ST_DOMAIN, 1);
                        continue;
                    }
                    int l[3][3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int bw = wrap_near(I.I0[a] + base[a], n);
                        const int st = a == 0 ? sx : (a == 1 ? sy : sz);
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            int idx = bw + m;
                            idx -= idx >= n ? n : 0;
                            l[a][m] = idx - st;
                        }
                    }
                    int J = 0;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb)
#pragma unroll
                            for (int a = 0; a < 3; ++a, ++J)
                                if ((unsigned)l[2][c] < (unsigned)ez && (unsigned)l[1][bb] < (unsigned)ey &&
                                    (unsigned)l[0][a] < (unsigned)ex)
                                    acc_add(accd + l[2][c] * pp + l[1][bb] * px + l[0][a],
                                            FixedPoint<Acc>::conv(wt[J] * gq));
                }
            }
        }
        __syncthreads();
        // flush: per lattice, every row (z, y) of the tile, x in quads when the
        // rows are 16-byte aligned; non-zero sums are added to the grid with
        // L2 reductions (each value belongs to this tile only) and cleared
        const long long n3 = (long long)n * n * n;
        unsigned touched = 0;
        // quads need 16-byte aligned rows: box field base, n, tile start and
        // edge all multiples of 4 floats
        const bool vec = ((sx | n | ex) & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(f + s_B.grid_off)) & 15) == 0;
        const int nq = vec ? (ex >> 2) : ex;
        const int items = ey * ez * nq;
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            const float inv = 1.f / s_scale[d];
            DF part{0.f, 0.f};
            float *fd = f + s_B.grid_off + d * n3;
            Acc *ad = acc + d * vol;
            for (int item = threadIdx.x; item < items; item += blockDim.x) {
                const int r = item / nq, qx = item - r * nq;
                const int lz = r / ey, ly = r - lz * ey;
                Acc *src = ad + lz * pp + ly * px;
                float *dst = fd + ((long long)(sz + lz) * n + (sy + ly)) * n + sx;
                if (vec) {
                    const int x0 = qx << 2;
                    const Acc q0 = src[x0], q1 = src[x0 + 1], q2 = src[x0 + 2], q3 = src[x0 + 3];
                    if ((q0 | q1 | q2 | q3) != 0) {
                        src[x0] = 0;
                        src[x0 + 1] = 0;
                        src[x0 + 2] = 0;
                        src[x0 + 3] = 0;
                        const float v0 = (float)q0 * inv, v1 = (float)q1 * inv, v2 = (float)q2 * inv,
                                    v3 = (float)q3 * inv;
                        red_add_v4(dst + x0, v0, v1, v2, v3);
                        df_add(part, v0);
                        df_add(part, v1);
                        df_add(part, v2);
                        df_add(part, v3);
                        touched += (q0 != 0) + (q1 != 0) + (q2 != 0) + (q3 != 0);
                    }
                } else {
                    const Acc q = src[qx];
                    if (q != 0) {
                        src[qx] = 0;
                        const float v = (float)q * inv;
                        red_add(dst + qx, v);
                        df_add(part, v);
                        ++touched;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float hi = __shfl_down_sync(0xffffffffu, part.hi, o);
                const float lo = __shfl_down_sync(0xffffffffu, part.lo, o);
                df_add(part, hi);
                part.lo += lo;
            }
            if (lane == 0)
                s_red[d][wid] = (double)part.hi + (double)part.lo;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            touched += __shfl_down_sync(0xffffffffu, touched, o);
        if (lane == 0)
            status_add(w.status, ST_TOUCHED, touched);
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = 0.0;
            for (int q = 0; q < nw; ++q)
                v += s_red[threadIdx.x][q];
            w.red_tile[3LL * tile + threadIdx.x] = v * h3;
        }
        // the next iteration's barrier orders these reads before s_red is rewritten
    }
}

// ------------------------------------------- spread, FP32, halo scatter
// IFEM_SCATTER_ATOMIC, Peskin kernel. Work item = (tile, lattice) taken from
// a global counter over every tile. Each node is visited only by the tile
// that holds its cell (no candidate lists): the CTA accumulates the 64
// contributions of each own node into a buffer covering the tile plus a
// halo of 4 cells in x (keeps 16-byte quads aligned) and 2 cells in y and z,
// so every stencil point of every node lands in the buffer. Accumulation is
// int32 fixed point with shared-memory atomics (scale from the bound
// sum_k |g_k| / 8 over the tile's own nodes); the flush adds every non-zero
// value to the grid with L2 reductions, where neighbouring tiles' halos
// combine atomically (summation order of a value across tiles is not fixed).
// ST_TOUCHED counts the non-zero sums inside the tile itself.
// INTERP = true fuses the interpolation S of the same step: each (node,
// lattice) unit also gathers u at the 64 stencil points with the unscaled
// weights it has just computed, v_d = sum phi u_d (Algorithm step 4).
// AB2 = true (with INTERP) also takes the position update of Eq.
// Bashforth_eqn from the velocity it has just gathered, out of place:
// xn_d = x_d + dt (3/2 v_d - 1/2 vp_d), rounded as in ab2_kernel.
constexpr int kHaloX = 4, kHaloYZ = 2;

// Buffer pitches: the row pitch is 8 mod 16 and the plane pitch 4 mod 8, so
// the 4 x 4 x 4 cells around a group of neighbouring nodes fall on all 32
// banks, two cells per bank; both stay multiples of 4 for 16-byte rows.
__host__ __device__ inline int halo_px(int bx) { return bx + (24 - bx % 16) % 16; }
__host__ __device__ inline int halo_pp(int by, int px) { return by * px + 4; }
__host__ __device__ inline int halo_ints(int E)
{
    const int px = halo_px(E + 2 * kHaloX);
    return halo_pp(E + 2 * kHaloYZ, px) * (E + 2 * kHaloYZ);
}

// FP32 halo path, after the scan: every binned node goes to its slot (the
// scanned offset of its key plus its rank from own_count_kernel) with its
// record, kBinPer nodes per thread as in own_count_kernel (loads first, then
// the offsets, then the stores); the tile boundaries of the own lists are
// finalised (own_off[t * kOwnSub3] = local offset + block offset, the total
// at t = n_tiles: the only entries the halo kernels read); the per-tile FP64
// sums of the spread are cleared for every tile (the transfer writes them
// for the listed tiles only) and the tiles that own nodes are listed,
// counters[3] of them. The fused transfer kernels take their (tile,
// lattice) items from that list, so no CTA walks empty tiles; it keeps
// roughly the tile order (in order within each warp's append), so items
// running at the same time are spatial neighbours whose velocity rows and
// grid lines share L2 (listing the largest tiles first measured slower).
// With the forces F given, the placement also sums |F_d| over each tile's
// own nodes into tile_fsum (zeroed with the counts): the fused transfer's
// fixed-point scale of item (tile, d) comes from that sum instead of a pass
// over the item's forces. Lanes of a warp hold consecutive nodes, so the
// tiles come in runs: a segmented shuffle scan sums each run and its last
// lane adds it with one atomic per lattice (the order of those atomics is
// not fixed; the transfer's bound allows for it).
// Grid: as own_count_kernel along x and y, at least n_tiles + 1 threads in all.
static __global__ void __launch_bounds__(256) own_scatter_kernel(DevBatch b, DevWork w, long long n_tiles,
                                                                 const float *__restrict__ F)
{
    const InstDev I = b.inst[blockIdx.y];
    const long long N = b.N;
    const int lane = threadIdx.x & 31;
    int node[kBinPer];
    int2 kr[kBinPer];
    float4 rec[kBinPer];
    float fa[kBinPer][3];
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
        const int k = (blockIdx.x * kBinPer + j) * blockDim.x + threadIdx.x;
        node[j] = I.node_off + k;
        kr[j] = make_int2(-1, 0);
        fa[j][0] = fa[j][1] = fa[j][2] = 0.f;
        if (k < I.n_nodes) {
            kr[j] = w.node_key[node[j]];
            rec[j] = w.node_rec[node[j]];
            if (F) {
                fa[j][0] = fabsf(F[node[j]]);
                fa[j][1] = fabsf(F[N + node[j]]);
                fa[j][2] = fabsf(F[2 * N + node[j]]);
            }
        }
    }
    if (F) {   // the same for every thread of the grid
#pragma unroll
        for (int j = 0; j < kBinPer; ++j) {
            const int tile = kr[j].x >= 0 ? kr[j].x / kOwnSub3 : -1;
            const int prev = __shfl_up_sync(0xffffffffu, tile, 1);
            const int next = __shfl_down_sync(0xffffffffu, tile, 1);
            const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != tile);
            // first lane of this lane's run
            const int seg = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float t = __shfl_up_sync(0xffffffffu, fa[j][d], o);
                    if (lane - o >= seg)
                        fa[j][d] += t;
                }
            }
            if (tile >= 0 && (lane == 31 || next != tile)) {
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    atomicAdd(&w.tile_fsum[3LL * tile + d], fa[j][d]);
            }
        }
    }
    int off[kBinPer];
#pragma unroll
    for (int j = 0; j < kBinPer; ++j)
        off[j] = kr[j].x >= 0 ? w.own_cursor[kr[j].x] + w.scan_blocks[2 * (kr[j].x / kScanBlock) + 1] : 0;
#pragma unroll
    for (int j = 0; j < kBinPer; ++j) {
        if (kr[j].x >= 0) {
            const int slot = off[j] + kr[j].y;
            w.own_nodes[slot] = node[j];
            w.own_rec[slot] = rec[j];
        }
    }
    const long long nthr = (long long)gridDim.x * gridDim.y * blockDim.x;
    const long long tid = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    for (long long t0 = tid - lane; t0 <= n_tiles; t0 += nthr) {   // warp-uniform bounds
        const long long t = t0 + lane;
        bool has = false;
        if (t < n_tiles) {
            const long long i = t * kOwnSub3;
            w.own_off[i] = w.own_cursor[i] + w.scan_blocks[2 * (i / kScanBlock) + 1];
            has = w.own_flag[t] != 0;
            w.red_tile[3 * t] = 0.0;
            w.red_tile[3 * t + 1] = 0.0;
            w.red_tile[3 * t + 2] = 0.0;
        } else if (t == n_tiles) {
            w.own_off[t * kOwnSub3] = w.counters[5];
        }
        const unsigned m = __ballot_sync(0xffffffffu, has);
        int base = 0;
        if (lane == 0 && m)
            base = atomicAdd(&w.counters[3], __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (has)
            w.own_tiles[base + __popc(m & ((1u << lane) - 1u))] = (int)t;
    }
}

// red.shared.add without a compiler memory clobber: for accumulators that
// no thread reads before the next barrier (the caller places a compiler
// fence before it).
__device__ __forceinline__ void red_shared_add_nc(unsigned a, int v)
{
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v));
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Next (tile, lattice) item of the fused transfer kernels (thread 0): items
// are the three lattices of each listed tile, in list order (lattice < 0,
// work counter counters[2]), or lattice d of each listed tile (work
// counters[1], [6], [7] for d = 0, 1, 2), so that one launch per lattice
// completes row d of v at its end.
__device__ __forceinline__ void staged_next(const DevGrid &g, const DevWork &w, int lattice, int &item,
                                            TileInfo &ti, BoxDev &B)
{
    const int n_tiles = w.counters[3];
    int tile = -1, d = 0;
    if (lattice < 0) {
        const int it = atomicAdd(&w.counters[2], 1);
        if (it < 3 * n_tiles) {
            const int q = it / 3;
            tile = w.own_tiles[q];
            d = it - 3 * q;
        }
    } else {
        const int it = atomicAdd(&w.counters[lattice == 0 ? 1 : (lattice == 1 ? 6 : 7)], 1);
        if (it < n_tiles) {
            tile = w.own_tiles[it];
            d = lattice;
        }
    }
    item = -1;
    if (tile >= 0) {
        item = 3 * tile + d;
        ti = decode_tile(g, tile);
        B = g.boxes[ti.box];
    }
}

__device__ __forceinline__ void cp_async8(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(__cvta_generic_to_global(src))
                 : "memory");
}

// Periodic wrap of a box coordinate in [-n, 2n): the boxes of a grid have
// at least 8 cells and the halos at most 4, so one correction suffices.
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Shared buffers of the fused transfer kernel. A, the spread accumulator,
// covers the tile plus the halo of spread_halo_kernel (4 cells in x, so
// that the flush adds 16-byte quads, and 2 in y and z). U, the staged
// velocities, covers exactly the cells the stencils read, 2 cells on every
// side of the tile: rows of ex + 4 values from x = sx - 2, plane pitch 12
// floats above the plane size. U starts 8 bytes past a 16-byte boundary, so
// that the values of x = sx .. sx + ex - 1 fill 16-byte quads. Both rounded
// to 16 bytes; the pair fits three CTAs per SM for 16-cell tiles.
constexpr int kStagedThreads = 128;
__host__ __device__ inline int pair_buf_bytes(int E) { return ((halo_ints(E) * 4 + 15) / 16) * 16; }
__host__ __device__ inline int pair_u_px(int ex) { return ex + 4; }
__host__ __device__ inline int pair_u_pp(int ey, int pxu) { return pxu * (ey + 4) + 12; }
__host__ __device__ inline int pair_u_bytes(int E)
{
    return ((8 + 4 * pair_u_pp(E, pair_u_px(E)) * (E + 4) + 15) / 16) * 16;
}
__host__ __device__ inline int pair_smem_bytes(int E) { return pair_u_bytes(E) + pair_buf_bytes(E); }

// One (tile, lattice) item of the fused transfer kernel, in registers.
struct PairItem {
    int item, tile, d;
    int sx, sy, sz, ex, ey, ez;
    int n, bx, by, bz, px, pp;
    int pxu, ppu;   // pitches of the U box
    long long grid_off;
    float sd;
    double box_scale;
};
__device__ __forceinline__ PairItem pair_item(int item, const TileInfo &ti, const BoxDev &B, int density)
{
    PairItem it;
    it.item = item;
    it.tile = item / 3;
    it.d = item - 3 * it.tile;
    it.sx = ti.start[0];
    it.sy = ti.start[1];
    it.sz = ti.start[2];
    it.ex = ti.edge[0];
    it.ey = ti.edge[1];
    it.ez = ti.edge[2];
    it.n = B.n;
    it.bx = it.ex + 2 * kHaloX;
    it.by = it.ey + 2 * kHaloYZ;
    it.bz = it.ez + 2 * kHaloYZ;
    it.px = halo_px(it.bx);
    it.pp = halo_pp(it.by, it.px);
    it.pxu = pair_u_px(it.ex);
    it.ppu = pair_u_pp(it.ey, it.pxu);
    it.grid_off = B.grid_off;
    it.sd = density ? B.scale_f : 1.f;
    it.box_scale = B.scale;
    return it;
}

// Rows of a (tile + halo) box walked by the warps of a CTA: a lane takes x
// unit qx = lq (+ multiples of nql) of every row it visits; rows advance by
// a fixed (y, z) step, so no index is divided in the loop. fn(lz, ly, gz, gy, qx)
// receives the row's box coordinates and its wrapped grid coordinates.
// a / b for 0 <= a < 2^21 and b >= 1, exactly, through a float reciprocal:
// (a + 1/2) / b lies at least 1/(2b) from the nearest integer, while the
// rounding of the reciprocal and the product moves it by at most about
// (a/b) 2^-22 < 1/(2b).
__device__ __forceinline__ int small_div(int a, int b) { return (int)(((float)a + 0.5f) * __frcp_rn((float)b)); }

// Columns of a (tile + halo) box walked by the threads of a CTA: a column is
// one x unit (quad or value) qx of one y row ly; each thread takes one column
// and steps through the z planes (several planes at a time when the CTA has
// threads for more than one plane's columns), so the loop carries only a
// plane index. fn(lz, ly, gz, gy, qx) receives the box coordinates and the
// wrapped grid coordinates. Boxes with more columns than threads take the
// generic walk (one division per value).
template <typename Fn>
__device__ __forceinline__ void box_cols(const PairItem &it, int bz, int by, int nq, Fn fn)
{
    const int C = by * nq, T = blockDim.x, t = threadIdx.x;
    if (C <= T) {
        const int P = small_div(T, C);
        const int pz = small_div(t, C);
        if (pz >= P)
            return;
        const int c = t - pz * C;
        const int ly = small_div(c, nq), qx = c - ly * nq;
        const int gy = wrap1(it.sy - kHaloYZ + ly, it.n);
        int gz = wrap1(it.sz - kHaloYZ + pz, it.n);
        for (int lz = pz; lz < bz; lz += P) {
            fn(lz, ly, gz, gy, qx);
            gz += P;
            gz -= gz >= it.n ? it.n : 0;
        }
    } else {
        for (int q = t; q < C * bz; q += T) {
            const int lz = small_div(q, C), c = q - lz * C;
            const int ly = small_div(c, nq), qx = c - ly * nq;
            fn(lz, ly, wrap1(it.sz - kHaloYZ + lz, it.n), wrap1(it.sy - kHaloYZ + ly, it.n), qx);
        }
    }
}

// The same over a box of bz x by rows starting 2 cells below the tile in y
// and z (the A box and the U box both do).
template <typename Fn>
__device__ __forceinline__ void box_rows(const PairItem &it, int bz, int by, int nq, int lane, int wid, int nw,
                                         Fn fn)
{
    const int nql = nq <= 32 ? nq : 32;
    const int rpw = small_div(32, nql);
    const int lr = small_div(lane, nql), lq = lane - lr * nql;
    if (lr >= rpw)
        return;
    const int rstep = nw * rpw;
    const int r0 = wid * rpw + lr;
    int lz = small_div(r0, by), ly = r0 - lz * by;
    const int dz = small_div(rstep, by), dy = rstep - dz * by;
    while (lz < bz) {
        const int gz = wrap1(it.sz - kHaloYZ + lz, it.n), gy = wrap1(it.sy - kHaloYZ + ly, it.n);
        for (int qx = lq; qx < nq; qx += nql)
            fn(lz, ly, gz, gy, qx);
        ly += dy;
        lz += dz;
        if (ly >= by) {
            ly -= by;
            ++lz;
        }
    }
}

template <typename Fn>
__device__ __forceinline__ void pair_rows(const PairItem &it, int nq, int lane, int wid, int nw, Fn fn)
{
    box_rows(it, it.bz, it.by, nq, lane, wid, nw, fn);
}
// Copies the velocity box of an item's lattice into the U buffer (value i
// of a row is x = sx - 2 + i, rows from y and z = tile start - 2)
// asynchronously with cp.async, waited for before the next node loop. When
// n, the tile start and edge are multiples of 4 and the lattice is 16-byte
// aligned, the ex values x = sx .. sx + ex - 1 of every row move as 16-byte
// quads and the two values at each end as 8-byte pairs (two column walks,
// so no thread branches per copy); otherwise single values.
__device__ __forceinline__ void pair_stage(const PairItem &it, const float *__restrict__ u, unsigned sU)
{
    const long long n3 = (long long)it.n * it.n * it.n;
    const float *ud = u + it.grid_off + it.d * n3;
    const bool vec = ((it.sx | it.n | it.ex) & 3) == 0 && ((reinterpret_cast<uintptr_t>(ud)) & 15) == 0;
    const int n = it.n, bzu = it.ez + 4, byu = it.ey + 4;
    if (vec) {
        box_cols(it, bzu, byu, it.ex >> 2, [&](int lz, int ly, int gz, int gy, int qx) {
            cp_async16(sU + 4u * (unsigned)(lz * it.ppu + ly * it.pxu + 2 + 4 * qx),
                       ud + (gz * n + gy) * n + it.sx + 4 * qx);
        });
        box_cols(it, bzu, byu, 2, [&](int lz, int ly, int gz, int gy, int e) {
            cp_async8(sU + 4u * (unsigned)(lz * it.ppu + ly * it.pxu + (e ? it.ex + 2 : 0)),
                      ud + (gz * n + gy) * n + wrap1(e ? it.sx + it.ex : it.sx - 2, n));
        });
    } else {
        box_cols(it, bzu, byu, it.ex + 4, [&](int lz, int ly, int gz, int gy, int qx) {
            cp_async4(sU + 4u * (unsigned)(lz * it.ppu + ly * it.pxu + qx),
                      ud + (gz * n + gy) * n + wrap1(it.sx - 2 + qx, n));
        });
    }
}

// The first own unit of this thread in an item (node id, binning record,
// F_d), loaded ahead of the item's node loop.
struct PairUnit {
    int node;
    float4 rec;
    float f;
};

// The first unit of this thread for an item's node loop; thread 0 also puts
// into s_part[0] an upper bound of sum |F_d| over the item's own nodes: the
// placement's atomic float sum, whose rounding in any order is below
// (n - 1) 2^-24 of the exact sum for n nodes, times 1.0001 + n 2^-23.
__device__ __forceinline__ PairUnit pair_first(const PairItem &it, const DevWork &w, const float *__restrict__ F,
                                               long long N, float *s_part)
{
    const int beg = w.own_off[(long long)it.tile * kOwnSub3], end = w.own_off[(long long)(it.tile + 1) * kOwnSub3];
    PairUnit u0{0, make_float4(0.f, 0.f, 0.f, 0.f), 0.f};
    const int q = beg + (int)threadIdx.x;
    if (q < end) {
        u0.node = w.own_nodes[q];
        u0.rec = w.own_rec[q];
        u0.f = F[it.d * N + u0.node];
    }
    if (threadIdx.x == 0)
        s_part[0] = w.tile_fsum[3LL * it.tile + it.d] * (1.0001f + (float)(end - beg) * 1.1920929e-7f);
    return u0;
}

// Fixed-point scale of a (tile, lattice) accumulator: the largest power of
// two that keeps wmax * sum_k |g_k| (wmax = 1/8 for Peskin, sd the density
// factor) below the int32 range, from the per-warp partial sums of |F_d|.
// Every thread computes the same value.
__device__ __forceinline__ float halo_scale(const float *s_part, int nw, float sd)
{
    float tot = 0.f;
    for (int q = 0; q < nw; ++q)
        tot += s_part[q];
    const float bound = tot * sd * 0.125f * 1.0001f;
    float scale = 1.f;
    if (bound > 0.f && isfinite(bound)) {
        int e = (int)floorf(log2f(FixedPoint<int>::kRange / bound));
        e = e > 120 ? 120 : (e < -120 ? -120 : e);
        scale = exp2f((float)e);
    }
    return scale;
}

template <bool INTERP, bool AB2 = false>
__global__ void __launch_bounds__(256, 5) spread_halo_kernel(DevBatch b, DevGrid g, DevWork w,
                                                          const float *__restrict__ x,
                                                          const float *__restrict__ F, float *__restrict__ f,
                                                          int density, const float *__restrict__ u,
                                                          float *__restrict__ v, const float *__restrict__ vp,
                                                          float *__restrict__ xn, float dt)
{
    const int lattice = -1;   // every lattice in one launch
    static_assert(INTERP || !AB2, "the position update needs the fused interpolation");
    extern __shared__ __align__(16) unsigned char halo_smem[];
    int *acc = reinterpret_cast<int *>(halo_smem);
    const unsigned sacc = smem_u32(acc);
    __shared__ float s_part[8];
    __shared__ long long s_red[8];
    // the next item, published by thread 0 in slot (k + 1) & 1 during the
    // flush of item k and read after that flush's barrier (two slots: the
    // slot of item k is rewritten only during item k + 1's flush)
    __shared__ int s_item[2];
    __shared__ TileInfo s_ti[2];
    __shared__ BoxDev s_B[2];
    const long long N = b.N;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < halo_ints(g.max_edge); i += blockDim.x)
        acc[i] = 0;
    if (threadIdx.x == 0)
        staged_next(g, w, lattice, s_item[0], s_ti[0], s_B[0]);
    __syncthreads();
    for (int slot = 0;; slot ^= 1) {
        if (s_item[slot] < 0)
            break;
        // item fields for the node loop, from the shared slot (it stays
        // valid until the next item's flush; the flush re-reads it)
        const int tile = s_item[slot] / 3, d = s_item[slot] - 3 * tile;
        const int sx = s_ti[slot].start[0], sy = s_ti[slot].start[1], sz = s_ti[slot].start[2];
        const int bx = s_ti[slot].edge[0] + 2 * kHaloX, by = s_ti[slot].edge[1] + 2 * kHaloYZ,
                  bz = s_ti[slot].edge[2] + 2 * kHaloYZ;
        const int px = halo_px(bx), pp = halo_pp(by, px);
        const int n = s_B[slot].n;
        const float sd = density ? s_B[slot].scale_f : 1.f;
        const int beg = w.own_off[(long long)tile * kOwnSub3], end = w.own_off[(long long)(tile + 1) * kOwnSub3];
        // fixed-point scale from sum |F_d| over the own nodes
        float gs = 0.f;
        for (int q = beg + threadIdx.x; q < end; q += blockDim.x)
            gs += fabsf(F[d * N + w.own_nodes[q]]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            gs += __shfl_down_sync(0xffffffffu, gs, o);
        if (lane == 0)
            s_part[wid] = gs;
        __syncthreads();
        const float gsc = sd * halo_scale(s_part, nw, sd);
        for (int q = beg + threadIdx.x; q < end; q += blockDim.x) {
            const int node = w.own_nodes[q];
            const float4 rec = w.own_rec[q];   // written by the binning
            const float gq = F[d * N + node] * gsc;
            const unsigned pk = __float_as_uint(rec.w);
            const float fr[3] = {rec.x, rec.y, rec.z};
            float ph[3][4];
            int l0[3];
            bool inside = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // lattice d sits at the cell coordinate, the other two half a
                // cell lower: s = t - 1/2 has floor(t) - 1 and fraction r + 1/2
                // below r = 1/2, so the stencil starts 2 (not 1) cells below
                const int c = (int)((pk >> (8 * a)) & 255u);   // cell within the tile
                int sh = -1;
                float r = fr[a];
                if (a != d) {
                    const bool low = r < 0.5f;
                    r = low ? r + 0.5f : r - 0.5f;
                    sh = low ? -2 : -1;
                }
                peskin_frac(r, ph[a]);
                l0[a] = c + (a == 0 ? kHaloX : kHaloYZ) + sh;
                const int lim = (a == 0 ? bx : (a == 1 ? by : bz)) - 4;
                inside = inside && (unsigned)l0[a] <= (unsigned)lim;
            }
            if (!inside) {   // a record inconsistent with this tile: never expected
                status_add(w.status, ST_DOMAIN, 1);
                continue;
            }
            const unsigned base = sacc + 4u * (unsigned)(l0[2] * pp + l0[1] * px + l0[0]);
            if constexpr (INTERP) {
                // grid indices of the stencil (the buffer origin is the tile
                // start minus the halo); per z plane the 16 gathers are issued
                // before that plane's shared-memory reductions
                const float *ud = u + s_B[slot].grid_off + (long long)d * n * n * n;
                int gx[4], gy[4], gz[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    gx[m] = wrap_near(sx - kHaloX + l0[0] + m, n);
                    gy[m] = wrap_near(sy - kHaloYZ + l0[1] + m, n);
                    gz[m] = wrap_near(sz - kHaloYZ + l0[2] + m, n);
                }
                float out = 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float uv[4][4];
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const float *row = ud + (gz[c] * n + gy[bb]) * n;
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            uv[bb][a] = __ldg(row + gx[a]);
                    }
                    const float wz = ph[2][c] * gq;
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const float wyz = ph[1][bb] * wz;
                        const unsigned row = base + 4u * (unsigned)(c * pp + bb * px);
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            red_shared_add(row + 4u * a, __float2int_rn(ph[0][a] * wyz));
                    }
                    float accz = 0.f;
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        float accy = ph[0][0] * uv[bb][0];
#pragma unroll
                        for (int a = 1; a < 4; ++a)
                            accy += ph[0][a] * uv[bb][a];
                        accz += ph[1][bb] * accy;
                    }
                    out += ph[2][c] * accz;
                }
                v[d * N + node] = out;
                if constexpr (AB2) {
                    const long long i = d * N + node;
                    xn[i] = ab2_value(x[i], out, vp[i], dt);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float wz = ph[2][c] * gq;
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const float wyz = ph[1][bb] * wz;
                        const unsigned row = base + 4u * (unsigned)(c * pp + bb * px);
#pragma unroll
                        for (int a = 0; a < 4; ++a)
                            red_shared_add(row + 4u * a, __float2int_rn(ph[0][a] * wyz));
                    }
                }
            }
        }
        __syncthreads();
        // flush: every non-zero sum is added to the grid with an L2 reduction
        // (quads of x when rows are 16-byte aligned) and cleared; meanwhile
        // thread 0 fetches the next item
        if (threadIdx.x == 0)
            staged_next(g, w, lattice, s_item[slot ^ 1], s_ti[slot ^ 1], s_B[slot ^ 1]);
        const PairItem cur = pair_item(s_item[slot], s_ti[slot], s_B[slot], density);
        const float scale = halo_scale(s_part, nw, cur.sd);   // the node loop's scale, recomputed
        {
            const long long n3 = (long long)n * n * n;
            float *fd = f + cur.grid_off + d * n3;
            const bool vec = ((sx | n | bx) & 3) == 0 && ((reinterpret_cast<uintptr_t>(fd)) & 15) == 0;
            const float inv = 1.f / scale;
            long long qsum = 0;
            unsigned touched = 0;
            if (vec) {
                pair_rows(cur, bx >> 2, lane, wid, nw, [&](int lz, int ly, int gz, int gy, int qx) {
                    int4 *sp = reinterpret_cast<int4 *>(acc + lz * pp + ly * px + 4 * qx);
                    const int4 qv = *sp;
                    if ((qv.x | qv.y | qv.z | qv.w) != 0) {
                        *sp = make_int4(0, 0, 0, 0);
                        const int x0 = 4 * qx;
                        red_add_v4(fd + (gz * n + gy) * n + wrap1(sx - kHaloX + x0, n), (float)qv.x * inv,
                                   (float)qv.y * inv, (float)qv.z * inv, (float)qv.w * inv);
                        qsum += (long long)qv.x + (long long)qv.y + (long long)qv.z + (long long)qv.w;
                        if ((unsigned)(lz - kHaloYZ) < (unsigned)cur.ez && (unsigned)(ly - kHaloYZ) < (unsigned)cur.ey &&
                            (unsigned)(x0 - kHaloX) < (unsigned)cur.ex)
                            touched += (qv.x != 0) + (qv.y != 0) + (qv.z != 0) + (qv.w != 0);
                    }
                });
            } else {
                pair_rows(cur, bx, lane, wid, nw, [&](int lz, int ly, int gz, int gy, int qx) {
                    int *sp = acc + lz * pp + ly * px + qx;
                    const int qv = *sp;
                    if (qv != 0) {
                        *sp = 0;
                        red_add(fd + (gz * n + gy) * n + wrap1(sx - kHaloX + qx, n), (float)qv * inv);
                        qsum += qv;
                        touched += (unsigned)(lz - kHaloYZ) < (unsigned)cur.ez &&
                                   (unsigned)(ly - kHaloYZ) < (unsigned)cur.ey && (unsigned)(qx - kHaloX) < (unsigned)cur.ex;
                    }
                });
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                qsum += __shfl_down_sync(0xffffffffu, qsum, o);
                touched += __shfl_down_sync(0xffffffffu, touched, o);
            }
            if (lane == 0) {
                s_red[wid] = qsum;
                if (touched)
                    status_add(w.status, ST_TOUCHED, touched);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long vsum = 0;
            for (int q = 0; q < nw; ++q)
                vsum += s_red[q];
            // exact: |vsum| < 2^53, 1/scale a power of two
            w.red_tile[3LL * tile + d] = (double)vsum * (double)(1.f / scale) / cur.box_scale;
        }
        // s_part and s_red are written again only after the next barriers
    }
}

// ---------------------------------- spread + interp, FP32, staged velocity
// IFEM_SCATTER_ATOMIC, Peskin kernel, with the interpolation of the same
// step fused (Algorithm steps 2 and 4 use the same stencil weights of the
// same positions). Work item = (tile, lattice) over the tiles with own
// nodes (own_scatter_kernel), taken from a global counter; thread 0 fetches
// the next item during the node loop. Two shared buffers per CTA: U, the
// velocity values the item's stencils read (2 cells around the tile), and A,
// the spread accumulator over the tile plus the halo of spread_halo_kernel
// (int32 fixed point, scale from the bound sum_k |g_k| / 8 over the tile's
// own nodes, from the sum of |F_d| that the binning's placement keeps per
// tile). Per item:
//   1. node loop, one (node, lattice) unit per thread: the Peskin weights
//      of the unit; interpolation from U (64 shared-memory loads at
//      immediate offsets, v_d = sum phi u_d in z-y-x order), then the 64
//      contributions added to A with shared-memory reductions;
//   2. the next item's velocity box is copied into U (cp.async), each
//      thread's first unit of it loaded and its scale bound read, while A
//      is flushed: every non-zero value is added to the
//      grid with an L2 reduction (halos of neighbouring tiles combine there)
//      and cleared.
// CTAs are small (kStagedThreads): an item has a few hundred units, and the
// last round of the node loop leaves threads idle at the barrier; with
// fewer threads per CTA that round is a smaller share of the item.
// AB2 = true also writes the position update of Eq. Bashforth_eqn from each
// interpolated velocity, out of place. lattice >= 0 restricts the launch to
// that lattice's items (see staged_next).
template <bool AB2>
__global__ void __launch_bounds__(kStagedThreads, 3) transfer_staged_kernel(DevBatch b, DevGrid g, DevWork w,
                                                                     const float *__restrict__ x,
                                                                     const float *__restrict__ F,
                                                                     float *__restrict__ f, int density,
                                                                     const float *__restrict__ u,
                                                                     float *__restrict__ v,
                                                                     const float *__restrict__ vp,
                                                                     float *__restrict__ xn, float dt,
                                                                     int lattice)
{
    extern __shared__ __align__(16) unsigned char pair_smem[];
    __shared__ float s_part[kStagedThreads / 32];
    __shared__ long long s_red[kStagedThreads / 32];
    // the next item, published by thread 0 in slot (k + 1) & 1 during the
    // node loop of item k and read after that loop's barrier (two slots: the
    // slot of item k is rewritten only during item k + 1's node loop)
    __shared__ int s_item[2];
    __shared__ TileInfo s_ti[2];
    __shared__ BoxDev s_B[2];
    const int ubytes = pair_u_bytes(g.max_edge), buf = pair_buf_bytes(g.max_edge);
    const float *U = reinterpret_cast<const float *>(pair_smem + 8);
    int *A = reinterpret_cast<int *>(pair_smem + ubytes);
    const unsigned sU = smem_u32(pair_smem) + 8u, sA = smem_u32(pair_smem) + (unsigned)ubytes;
    const long long N = b.N;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // a kernel launched after this one with programmatic serialization (the
    // next lattice of the same step, which reads nothing this one writes) may
    // start at once: the grid is sized to be resident, so its CTAs take the
    // SMs that this grid's CTAs leave when the items run out
    asm volatile("griddepcontrol.launch_dependents;");
    for (int i = threadIdx.x; i < buf / 16; i += blockDim.x)
        reinterpret_cast<int4 *>(A)[i] = make_int4(0, 0, 0, 0);
    if (threadIdx.x == 0)
        staged_next(g, w, lattice, s_item[0], s_ti[0], s_B[0]);
    __syncthreads();
    if (s_item[0] < 0)
        return;
    PairUnit u0;
    {
        const PairItem first = pair_item(s_item[0], s_ti[0], s_B[0], density);
        pair_stage(first, u, sU);
        u0 = pair_first(first, w, F, N, s_part);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int slot = 0;; slot ^= 1) {
        const PairItem cur = pair_item(s_item[slot], s_ti[slot], s_B[slot], density);
        // fixed-point scale of this item from the bound of sum |F_d|
        float scale = 1.f;
        {
            const float bound = s_part[0] * cur.sd * 0.125f;
            if (bound > 0.f && isfinite(bound)) {
                int e = (int)floorf(log2f(FixedPoint<int>::kRange / bound));
                e = e > 120 ? 120 : (e < -120 ? -120 : e);
                scale = exp2f((float)e);
            }
        }
        const float gsc = cur.sd * scale;
        if (threadIdx.x == 0)
            staged_next(g, w, lattice, s_item[slot ^ 1], s_ti[slot ^ 1], s_B[slot ^ 1]);
        const int d = cur.d;
        const int beg = w.own_off[(long long)cur.tile * kOwnSub3];
        const int end = w.own_off[(long long)(cur.tile + 1) * kOwnSub3];
        const int px = cur.px, pp = cur.pp;
        // 1. node loop: one (node, lattice) unit per thread; the first unit
        // was loaded ahead (pair_first)
        PairUnit un = u0;
        for (int q = beg + (int)threadIdx.x; q < end;) {
            const int node = un.node;
            const float4 rec = un.rec;   // written by the binning
            const float gq = un.f * gsc;
            q += blockDim.x;
            if (q < end) {
                un.node = w.own_nodes[q];
                un.rec = w.own_rec[q];
                un.f = F[d * N + un.node];
            }
            const unsigned pk = __float_as_uint(rec.w);
            const float fr[3] = {rec.x, rec.y, rec.z};
            float ph[3][4];
            int l0[3];
            bool inside = true;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                // lattice d sits at the cell coordinate, the other two half a
                // cell lower: s = t - 1/2 has floor(t) - 1 and fraction r + 1/2
                // below r = 1/2, so the stencil starts 2 (not 1) cells below
                const int c = (int)((pk >> (8 * ax)) & 255u);   // cell within the tile
                int sh = -1;
                float r = fr[ax];
                if (ax != d) {
                    const bool low = r < 0.5f;
                    r = low ? r + 0.5f : r - 0.5f;
                    sh = low ? -2 : -1;
                }
                peskin_frac(r, ph[ax]);
                l0[ax] = c + (ax == 0 ? kHaloX : kHaloYZ) + sh;
                // inside both boxes: in x within [2, ex + 2] of A (U starts
                // 2 cells later), in y and z within [0, e]
                const int lo = ax == 0 ? 2 : 0;
                const int hi = ax == 0 ? cur.ex + 2 : (ax == 1 ? cur.ey : cur.ez);
                inside = inside && (unsigned)(l0[ax] - lo) <= (unsigned)(hi - lo);
            }
            if (!inside) {   // a record inconsistent with this tile: never expected
                status_add(w.status, ST_DOMAIN, 1);
                continue;
            }
            const int off = l0[2] * pp + l0[1] * px + l0[0];
            const float *ub = U + (l0[2] * cur.ppu + l0[1] * cur.pxu + (l0[0] - 2));
            const unsigned ab = sA + 4u * (unsigned)off;
            // interpolation first (all 64 loads can be in flight), then the
            // 64 fixed-point reductions; the reductions carry no compiler
            // memory clobber, so they do not hold back the loads of the next
            // unit (the barrier after the loop orders them)
            float out = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float accz = 0.f;
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const float *row = ub + c * cur.ppu + bb * cur.pxu;
                    float accy = ph[0][0] * row[0];
#pragma unroll
                    for (int a = 1; a < 4; ++a)
                        accy += ph[0][a] * row[a];
                    accz += ph[1][bb] * accy;
                }
                out += ph[2][c] * accz;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float wz = ph[2][c] * gq;
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const float wyz = ph[1][bb] * wz;
                    const unsigned arow = ab + 4u * (unsigned)(c * pp + bb * px);
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        red_shared_add_nc(arow + 4u * a, __float2int_rn(ph[0][a] * wyz));
                }
            }
            v[d * N + node] = out;
            if constexpr (AB2) {
                const long long i = d * N + node;
                xn[i] = ab2_value(x[i], out, vp[i], dt);
            }
        }
        asm volatile("" ::: "memory");   // the reductions above stay before the barrier
        __syncthreads();   // A complete, U free, the next item published

        // 2. next item's velocities and scale bound; flush of A
        const int next = s_item[slot ^ 1];
        if (next >= 0) {
            const PairItem nxt = pair_item(next, s_ti[slot ^ 1], s_B[slot ^ 1], density);
            pair_stage(nxt, u, sU);
            u0 = pair_first(nxt, w, F, N, s_part);
        }
        {
            const long long n3 = (long long)cur.n * cur.n * cur.n;
            float *fd = f + cur.grid_off + d * n3;
            const bool vec = ((cur.sx | cur.n | cur.bx) & 3) == 0 && ((reinterpret_cast<uintptr_t>(fd)) & 15) == 0;
            const float inv = 1.f / scale;
            const int n = cur.n;
            long long qsum = 0;
            unsigned touched = 0;
            if (vec) {
                box_cols(cur, cur.bz, cur.by, cur.bx >> 2, [&](int lz, int ly, int gz, int gy, int qx) {
                    int4 *sp = reinterpret_cast<int4 *>(A + lz * pp + ly * px + 4 * qx);
                    const int4 qv = *sp;
                    if ((qv.x | qv.y | qv.z | qv.w) != 0) {
                        *sp = make_int4(0, 0, 0, 0);
                        const int x0 = 4 * qx;
                        red_add_v4(fd + (gz * n + gy) * n + wrap1(cur.sx - kHaloX + x0, n), (float)qv.x * inv,
                                   (float)qv.y * inv, (float)qv.z * inv, (float)qv.w * inv);
                        qsum += (long long)qv.x + (long long)qv.y + (long long)qv.z + (long long)qv.w;
                        if ((unsigned)(lz - kHaloYZ) < (unsigned)cur.ez && (unsigned)(ly - kHaloYZ) < (unsigned)cur.ey &&
                            (unsigned)(x0 - kHaloX) < (unsigned)cur.ex)
                            touched += (qv.x != 0) + (qv.y != 0) + (qv.z != 0) + (qv.w != 0);
                    }
                });
            } else {
                box_cols(cur, cur.bz, cur.by, cur.bx, [&](int lz, int ly, int gz, int gy, int qx) {
                    int *sp = A + lz * pp + ly * px + qx;
                    const int qv = *sp;
                    if (qv != 0) {
                        *sp = 0;
                        red_add(fd + (gz * n + gy) * n + wrap1(cur.sx - kHaloX + qx, n), (float)qv * inv);
                        qsum += qv;
                        touched += (unsigned)(lz - kHaloYZ) < (unsigned)cur.ez &&
                                   (unsigned)(ly - kHaloYZ) < (unsigned)cur.ey && (unsigned)(qx - kHaloX) < (unsigned)cur.ex;
                    }
                });
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                qsum += __shfl_down_sync(0xffffffffu, qsum, o);
                touched += __shfl_down_sync(0xffffffffu, touched, o);
            }
            if (lane == 0) {
                s_red[wid] = qsum;
                if (touched)
                    status_add(w.status, ST_TOUCHED, touched);
            }
        }
        cp_async_wait_all();
        __syncthreads();   // U holds the next box, A is clear, s_part and s_red are written
        if (threadIdx.x == 0) {
            long long vsum = 0;
            for (int q = 0; q < nw; ++q)
                vsum += s_red[q];
            // exact: |vsum| < 2^53, 1/scale a power of two
            w.red_tile[3LL * cur.tile + d] = (double)vsum * (double)(1.f / scale) / cur.box_scale;
        }
        if (next < 0)
            break;
        // s_red and s_part are written again only after the next node loop's barrier
    }
}

// ------------------------------------------------- interp, FP32 direct
// Thread per (node, lattice) unit over the nodes in tile order (spatial
// locality for the L1/L2-cached gathers): v = sum_z phi_z sum_y phi_y
// sum_x phi_x u, one square root per axis, 32-bit row offsets.
template <int KER>
__global__ void __launch_bounds__(256, 6) interp_direct_kernel(DevBatch b, DevGrid g, DevWork w,
                                                            const float *__restrict__ u,
                                                            const float *__restrict__ x, float *__restrict__ v,
                                                            float support)
{
    const int total = w.counters[5];
    const long long unit = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (unit >= 3LL * total)
        return;
    const int d = (int)(unit / total);
    const int node = w.own_nodes[unit - (long long)d * total];
    const InstDev I = b.inst[b.node_inst[node]];
    const BoxDev B = g.boxes[I.box];
    const long long N = b.N;
    const int n = B.n;
    const float *ud = u + B.grid_off + (long long)d * n * n * n;
    float out = 0.f;
    if constexpr (KER == 0) {
        float ph[3][4];
        int ix[4], iy[4], iz[4];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int I0;
            float s = LatCoord<float>::get(I, B, a, x[a * N + node], mac_off(d, a), I0);
            int base = wrap_near(I0 + peskin_axis_fast(s, ph[a]), n);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                int idx = base + m;
                idx -= idx >= n ? n : 0;
                if (a == 0) ix[m] = idx;
                else if (a == 1) iy[m] = idx;
                else iz[m] = idx;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float accz = 0.f;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                const float *row = ud + (iz[c] * n + iy[bb]) * n;
                float accy = ph[0][0] * __ldg(row + ix[0]);
#pragma unroll
                for (int a = 1; a < 4; ++a)
                    accy += ph[0][a] * __ldg(row + ix[a]);
                accz += ph[1][bb] * accy;
            }
            out += ph[2][c] * accz;
        }
    } else {
        float s[3];
        int I0[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            s[a] = LatCoord<float>::get(I, B, a, x[a * N + node], mac_off(d, a), I0[a]);
        int base[3];
        float wt[27];
        if (!mls_weights<float>(s, support, base, wt)) {
            status_add(w.status, ST_DOMAIN, 1);
        } else {
            int ix[3], iy[3], iz[3];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                ix[m] = wrap_near(I0[0] + base[0] + m, n);
                iy[m] = wrap_near(I0[1] + base[1] + m, n);
                iz[m] = wrap_near(I0[2] + base[2] + m, n);
            }
            int J = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb)
#pragma unroll
                    for (int a = 0; a < 3; ++a, ++J)
                        out += wt[J] * __ldg(ud + (iz[c] * n + iy[bb]) * n + ix[a]);
        }
    }
    v[d * N + node] = out;
}

// ---------------------------------------- spread, FP64 deterministic, MLS
// Owner-computes gather: each thread owns up to kDetCells values of the tile
// (per lattice), starts from the current grid value and adds the
// contributions of the tile's candidate nodes in ascending node order:
// f = f + w*g with the node's MLS weight w of that value, g = F*scale. This is
// the oracle's per-value summation order, so the result is bit-identical.
// (The Peskin kernel has its own warp-per-unit kernel, spread_det_warp_kernel.)
constexpr int kDetThreads = 256;
constexpr int kDetCells = 4;     // owned values per thread and lattice (1024 per chunk; 2 CTAs per SM)
constexpr int kDetChunk = 32;    // candidates staged per round

struct DetCand {
    int lo[3];            // wrapped cell c-2 (union reach of all lattices)
    int base[3][3];       // [d][a] wrapped first stencil index
    double wt[3][27];     // [d][J] MLS weights
    double g[3];
    int ok;
};

static __global__ void __launch_bounds__(kDetThreads, 2) spread_det_mls_kernel(DevBatch b, DevGrid g, DevWork w,
                                                                 const double *__restrict__ x,
                                                                 const double *__restrict__ F,
                                                                 double *__restrict__ f, int density,
                                                                 double support)
{
    __shared__ DetCand cand[kDetChunk];
    __shared__ double red_sh[3][kDetThreads / 32];
    const long long N = b.N;
    const int n_active = w.counters[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status_add(w.status, ST_PAIRS, (unsigned long long)w.cand_off[g.n_tiles]);
        status_add(w.status, ST_ACTIVE, (unsigned long long)n_active);
    }
    for (int it = blockIdx.x; it < n_active; it += gridDim.x) {
        const int tile = w.active[it];
        const TileInfo ti = decode_tile(g, tile);
        const BoxDev B = g.boxes[ti.box];
        const int ex = ti.edge[0], ey = ti.edge[1], ez = ti.edge[2];
        const int vol = ex * ey * ez;
        const long long n3 = (long long)B.n * B.n * B.n;
        double part[3] = {0.0, 0.0, 0.0};
        // owned values in chunks of kDetThreads * kDetCells; each chunk walks
        // every candidate of the tile in ascending node order
        for (int cbase = 0; cbase < vol; cbase += kDetThreads * kDetCells) {
            double accv[kDetCells][3], init[kDetCells][3];
            int cx[kDetCells], cy[kDetCells], cz[kDetCells];
#pragma unroll
            for (int q = 0; q < kDetCells; ++q) {
                int i = cbase + threadIdx.x + q * kDetThreads;
                int lx = i % ex, ly = (i / ex) % ey, lz = i / (ex * ey);
                cx[q] = ti.start[0] + lx;
                cy[q] = ti.start[1] + ly;
                cz[q] = ti.start[2] + lz;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    double v = 0.0;
                    if (i < vol)
                        v = f[B.grid_off + d * n3 + ((long long)cz[q] * B.n + cy[q]) * B.n + cx[q]];
                    accv[q][d] = v;
                    init[q][d] = v;
                }
            }
            const double scale = density ? B.scale : 1.0;
            const int beg = w.cand_off[tile], end = w.cand_off[tile + 1];
            for (int c0 = beg; c0 < end; c0 += kDetChunk) {
                const int nc = min(kDetChunk, end - c0);
                __syncthreads();
                // stage candidate data: one thread per (candidate, lattice)
                for (int t = threadIdx.x; t < nc * 3; t += blockDim.x) {
                    const int j = t / 3, d = t % 3;
                    const int node = w.cand_nodes[c0 + j];
                    DetCand &C = cand[j];
                    const InstDev I = b.inst[b.node_inst[node]];
                    double s[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        int I0;
                        s[a] = LatCoord<double>::get(I, B, a, x[a * N + node], (double)mac_off(d, a), I0);
                    }
                    if (d == 0) {
                        C.ok = 1;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            int I0;
                            double sc = LatCoord<double>::get(I, B, a, x[a * N + node], 0.0, I0);
                            C.lo[a] = wrapi((long long)floor(sc) - 2, B.n);
                        }
                    }
                    C.g[d] = F[d * N + node] * scale;
                    int base[3];
                    if (!mls_weights<double>(s, support, base, C.wt[d])) {
                        status_add(w.status, ST_DOMAIN, 1);
                        C.g[d] = 0.0;
#pragma unroll
                        for (int J = 0; J < 27; ++J)
                            C.wt[d][J] = 0.0;
                    }
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        C.base[d][a] = wrapi(base[a], B.n);
                }
                __syncthreads();
                for (int j = 0; j < nc; ++j) {
                    const DetCand &C = cand[j];
#pragma unroll
                    for (int q = 0; q < kDetCells; ++q) {
                        if (cbase + threadIdx.x + q * kDetThreads >= vol)
                            break;
                        int rx = cx[q] - C.lo[0], ry = cy[q] - C.lo[1], rz = cz[q] - C.lo[2];
                        rx += rx < 0 ? B.n : 0;
                        ry += ry < 0 ? B.n : 0;
                        rz += rz < 0 ? B.n : 0;
                        if (rx > 4 || ry > 4 || rz > 4)
                            continue;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            int mx = cx[q] - C.base[d][0], my = cy[q] - C.base[d][1], mz = cz[q] - C.base[d][2];
                            mx += mx < 0 ? B.n : 0;
                            my += my < 0 ? B.n : 0;
                            mz += mz < 0 ? B.n : 0;
                            if (mx <= 2 && my <= 2 && mz <= 2)
                                accv[q][d] = accv[q][d] + C.wt[d][(mz * 3 + my) * 3 + mx] * C.g[d];
                        }
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kDetCells; ++q) {
                int i = cbase + threadIdx.x + q * kDetThreads;
                if (i >= vol)
                    break;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    f[B.grid_off + d * n3 + ((long long)cz[q] * B.n + cy[q]) * B.n + cx[q]] = accv[q][d];
                    part[d] += accv[q][d] - init[q][d];
                }
            }
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double v = part[d];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0)
                red_sh[d][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = 0.0;
            for (int q = 0; q < kDetThreads / 32; ++q)
                v += red_sh[threadIdx.x][q];
            w.red_tile[3LL * tile + threadIdx.x] = v * (1.0 / B.scale);
        }
    }
}

// FP64 deterministic Peskin spread, one warp per (tile, lattice) unit. The
// unit's owned values sit in a shared-memory accumulator loaded from f; the
// warp walks the tile's candidates in ascending node order, spreading each
// candidate's 64 stencil points over its lanes (two points per lane, on
// distinct cells since every box has at least 8 cells per axis), with a warp
// barrier between candidates, so every value receives its terms in the
// oracle's node order, f = f + ((phi_x phi_y) phi_z) g. Every lane carries
// FP64 work on every candidate whose stencil it meets inside the tile (this
// GPU's FP64 pipe is charged per warp instruction, whatever the active
// lanes). Stencils come from the binning's table (det_weights_kernel).
constexpr int kDetWarps = 4;   // units (warps) per CTA at most
constexpr int kDetStage = 32;  // candidates staged per round
struct DetStage {
    double ph[3][4];
    double g;
    int base[3];
    int pad;
};
// Shared memory of one warp: the accumulator of the largest tile + staging.
__host__ __device__ inline size_t det_warp_bytes(int max_edge)
{
    const size_t e3 = (size_t)max_edge * max_edge * max_edge;
    return e3 * sizeof(double) + kDetStage * sizeof(DetStage);
}

static __global__ void __launch_bounds__(32 * kDetWarps) spread_det_warp_kernel(DevBatch b, DevGrid g, DevWork w,
                                                                              const double *__restrict__ F,
                                                                              double *__restrict__ f, int density)
{
    extern __shared__ __align__(16) unsigned char det_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t e3 = (size_t)g.max_edge * g.max_edge * g.max_edge;
    double *acc = reinterpret_cast<double *>(det_smem) + wid * e3;
    DetStage *st = reinterpret_cast<DetStage *>(reinterpret_cast<double *>(det_smem) + nw * e3) + wid * kDetStage;
    const long long N = b.N;
    const int n_active = w.counters[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        status_add(w.status, ST_PAIRS, (unsigned long long)w.cand_off[g.n_tiles]);
        status_add(w.status, ST_ACTIVE, (unsigned long long)n_active);
    }
    // this lane's stencil points: (a, bb, c0) and (a, bb, c0 + 2)
    const int a = lane & 3, bb = (lane >> 2) & 3, c0 = lane >> 4;
    const long long n_units = 3LL * n_active;
    for (long long unit = (long long)blockIdx.x * nw + wid; unit < n_units; unit += (long long)gridDim.x * nw) {
        const int tile = w.active[unit / 3];
        const int d = (int)(unit - 3 * (unit / 3));
        const TileInfo ti = decode_tile(g, tile);
        const BoxDev B = g.boxes[ti.box];
        const int ex = ti.edge[0], ey = ti.edge[1], ez = ti.edge[2];
        const int sx = ti.start[0], sy = ti.start[1], sz = ti.start[2];
        const int n = B.n, vol = ex * ey * ez;
        double *fd = f + B.grid_off + (long long)d * n * n * n;
        for (int i = lane; i < vol; i += 32) {
            const int lx = i % ex, ly = (i / ex) % ey, lz = i / (ex * ey);
            acc[i] = fd[((long long)(sz + lz) * n + sy + ly) * n + sx + lx];
        }
        const double scale = density ? B.scale : 1.0;
        const int beg = w.cand_off[tile], end = w.cand_off[tile + 1];
        for (int c = beg; c < end; c += kDetStage) {
            const int nc = min(kDetStage, end - c);
            __syncwarp();
            if (lane < nc) {
                const int node = w.cand_nodes[c + lane];
                const DetW &Wn = w.wtab[node];
                DetStage &S = st[lane];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    S.base[q] = Wn.base[d][q];
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        S.ph[q][m] = Wn.ph[d][q][m];
                }
                S.g = F[d * N + node] * scale;
            }
            __syncwarp();
            for (int j = 0; j < nc; ++j) {
                const DetStage &S = st[j];
                // tile-relative cell of each point (base is wrapped into [0, n))
                int lx = S.base[0] + a - sx, ly = S.base[1] + bb - sy;
                int lz0 = S.base[2] + c0 - sz, lz1 = lz0 + 2;
                lx += lx < 0 ? n : (lx >= n ? -n : 0);
                ly += ly < 0 ? n : (ly >= n ? -n : 0);
                lz0 += lz0 < 0 ? n : (lz0 >= n ? -n : 0);
                lz1 += lz1 < 0 ? n : (lz1 >= n ? -n : 0);
                if ((unsigned)lx < (unsigned)ex && (unsigned)ly < (unsigned)ey) {
                    const double t = S.ph[0][a] * S.ph[1][bb];
                    if ((unsigned)lz0 < (unsigned)ez) {
                        const int i = (lz0 * ey + ly) * ex + lx;
                        acc[i] = acc[i] + (t * S.ph[2][c0]) * S.g;
                    }
                    if ((unsigned)lz1 < (unsigned)ez) {
                        const int i = (lz1 * ey + ly) * ex + lx;
                        acc[i] = acc[i] + (t * S.ph[2][c0 + 2]) * S.g;
                    }
                }
                __syncwarp();
            }
        }
        // write back; the unit's FP64 sum of the values it added
        double part = 0.0;
        for (int i = lane; i < vol; i += 32) {
            const int lx = i % ex, ly = (i / ex) % ey, lz = i / (ex * ey);
            double *p = fd + ((long long)(sz + lz) * n + sy + ly) * n + sx + lx;
            const double old = *p;
            *p = acc[i];
            part += acc[i] - old;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0)
            w.red_tile[3LL * tile + d] = part * (1.0 / B.scale);
        __syncwarp();
    }
}

// ------------------------------------------------------------- interp
// Thread per node (in tile order for locality). DET: the oracle's order,
// acc = acc + ((phi_x*phi_y)*phi_z)*u from 0, z-outer, x-inner. Fast FP32:
// separable sum_z phi_z sum_y phi_y sum_x phi_x u.
template <typename real, bool DET, int KER>
__global__ void __launch_bounds__(256) interp_kernel(DevBatch b, DevGrid g, DevWork w,
                                                     const real *__restrict__ u, const real *__restrict__ x,
                                                     real *__restrict__ v, real support, int use_order,
                                                     int use_wtab)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // in tile order only the binned nodes are listed (non-finite ones are not)
    if (idx >= (use_order ? (long long)w.counters[5] : b.N))
        return;
    const int node = use_order ? w.own_nodes[idx] : (int)idx;
    const InstDev I = b.inst[b.node_inst[node]];
    const BoxDev B = g.boxes[I.box];
    const long long N = b.N;
    const long long n3 = (long long)B.n * B.n * B.n;
    const int n = B.n;
    real xl[3];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xl[a] = x[a * N + node];
        finite = finite && isfinite(xl[a]);
    }
    if (!finite) {
        if (!use_order)
            status_add(w.status, ST_DOMAIN, 1);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            v[d * N + node] = xl[0] + xl[1] + xl[2];
        return;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const real *ud = u + B.grid_off + d * n3;
        real out = real(0);
        if constexpr (KER == 0) {
            real ph[3][4];
            int ix[4], iy[4], iz[4];
            // with use_wtab the stencil comes from the binning's per-node table
            // (det_weights_kernel: the same values, computed once per node)
            const DetW *wt = nullptr;
            if constexpr (std::is_same<real, double>::value)
                wt = use_wtab ? &w.wtab[node] : nullptr;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                long long i0;
                if (wt) {
                    i0 = wt->base[d][a];
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        ph[a][m] = (real)wt->ph[d][a][m];
                } else {
                    int I0;
                    real s = LatCoord<real>::get(I, B, a, xl[a], (real)mac_off(d, a), I0);
                    i0 = I0 + peskin_axis<real>(s, ph[a]);
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    int wi = wrapi(i0 + m, n);
                    if (a == 0) ix[m] = wi;
                    else if (a == 1) iy[m] = wi;
                    else iz[m] = wi;
                }
            }
            if (DET) {
                real acc = real(0);
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb)
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            real wgt = (ph[0][a] * ph[1][bb]) * ph[2][c];
                            acc = acc + wgt * ud[((long long)iz[c] * n + iy[bb]) * n + ix[a]];
                        }
                out = acc;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    real accz = real(0);
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const real *row = ud + ((long long)iz[c] * n + iy[bb]) * n;
                        real accy = ph[0][0] * __ldg(row + ix[0]);
#pragma unroll
                        for (int a = 1; a < 4; ++a)
                            accy += ph[0][a] * __ldg(row + ix[a]);
                        accz += ph[1][bb] * accy;
                    }
                    out += ph[2][c] * accz;
                }
            }
        } else {
            real s[3];
            int I0[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                s[a] = LatCoord<real>::get(I, B, a, xl[a], (real)mac_off(d, a), I0[a]);
            int base[3];
            real wt[27];
            if (!mls_weights<real>(s, support, base, wt)) {
                status_add(w.status, ST_DOMAIN, 1);
                out = real(0);
            } else {
                real acc = real(0);
                int J = 0;
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
                        for (int a = 0; a < 3; ++a, ++J) {
                            long long gi = ((long long)wrapi((long long)I0[2] + base[2] + c, n) * n
                                            + wrapi((long long)I0[1] + base[1] + bb, n)) * n
                                           + wrapi((long long)I0[0] + base[0] + a, n);
                            acc = acc + wt[J] * ud[gi];
                        }
                out = acc;
            }
        }
        v[d * N + node] = out;
    }
}

// ------------------------------------------- interpolation, cell-centred
// S of a cell-centred field with ncomp components (the conformation tensor
// C_J of Sec. "Interpolation Scheme"): all components at ((i,j,k) + 1/2) h.
// Thread per (node, component), component-major (neighbouring threads are
// neighbouring nodes of one component). FP64 in the oracle's order:
// acc = acc + w * c_J from 0, z-outer, x-inner, w = (phi_x * phi_y) * phi_z;
// FP32 Peskin in separable form (x rows, then y, then z). Field layout: box b
// holds ncomp blocks of n_b^3 values from (grid_off_b / 3) * ncomp; out:
// ncomp rows of N.
template <typename real, int KER>
__global__ void __launch_bounds__(256) interp_cc_kernel(DevBatch b, DevGrid g, DevWork w,
                                                        const real *__restrict__ field, int ncomp,
                                                        const real *__restrict__ x, real *__restrict__ out,
                                                        real support)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = b.N;
    if (idx >= N * ncomp)
        return;
    const int q = (int)(idx / N);
    const long long node = idx - q * N;
    const InstDev I = b.inst[b.node_inst[node]];
    const BoxDev B = g.boxes[I.box];
    const int n = B.n;
    const long long n3 = (long long)n * n * n;
    const real *cq = field + (B.grid_off / 3) * ncomp + q * n3;
    real xl[3];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xl[a] = x[a * N + node];
        finite = finite && isfinite(xl[a]);
    }
    if (!finite) {
        if (q == 0)
            status_add(w.status, ST_DOMAIN, 1);
        out[q * N + node] = xl[0] + xl[1] + xl[2];
        return;
    }
    real acc = real(0);
    if constexpr (KER == 0 && std::is_same<real, float>::value) {
        float ph[3][4];
        int ix[4], iy[4], iz[4];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int I0;
            const float s = LatCoord<float>::get(I, B, a, xl[a], 0.5f, I0);
            const int base = wrap_near(I0 + peskin_axis_fast(s, ph[a]), n);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                int id = base + m;
                id -= id >= n ? n : 0;
                if (a == 0) ix[m] = id;
                else if (a == 1) iy[m] = id;
                else iz[m] = id;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float accz = 0.f;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                const float *row = cq + ((long long)iz[c] * n + iy[bb]) * n;
                float accy = ph[0][0] * __ldg(row + ix[0]);
#pragma unroll
                for (int a = 1; a < 4; ++a)
                    accy += ph[0][a] * __ldg(row + ix[a]);
                accz += ph[1][bb] * accy;
            }
            acc += ph[2][c] * accz;
        }
    } else if constexpr (KER == 0) {
        real ph[3][4];
        int ix[4], iy[4], iz[4];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int I0;
            real s = LatCoord<real>::get(I, B, a, xl[a], real(0.5), I0);
            long long i0 = peskin_axis<real>(s, ph[a]);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                int wi = wrapi(I0 + i0 + m, n);
                if (a == 0) ix[m] = wi;
                else if (a == 1) iy[m] = wi;
                else iz[m] = wi;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int bb = 0; bb < 4; ++bb)
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    real wgt = (ph[0][a] * ph[1][bb]) * ph[2][c];
                    acc = acc + wgt * cq[((long long)iz[c] * n + iy[bb]) * n + ix[a]];
                }
    } else {
        real s[3];
        int I0[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            s[a] = LatCoord<real>::get(I, B, a, xl[a], real(0.5), I0[a]);
        int base[3];
        real wt[27];
        if (!mls_weights<real>(s, support, base, wt)) {
            if (q == 0)
                status_add(w.status, ST_DOMAIN, 1);
            out[q * N + node] = real(0);
            return;
        }
        int J = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int bb = 0; bb < 3; ++bb)
#pragma unroll
                for (int a = 0; a < 3; ++a, ++J) {
                    long long gi = ((long long)wrapi((long long)I0[2] + base[2] + c, n) * n
                                    + wrapi((long long)I0[1] + base[1] + bb, n)) * n
                                   + wrapi((long long)I0[0] + base[0] + a, n);
                    acc = acc + wt[J] * cq[gi];
                }
    }
    out[q * N + node] = acc;
}

// ------------------------------------------------------------- reductions
// Block per instance: FP64 sums in a fixed order (per-thread strided sums,
// then a fixed shared-memory tree). Layout: 12 doubles per instance.
template <int NT>
__device__ inline double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// One launch for all conservation sums. Blocks [0, n_inst): one instance
// each -- partial sums of x, F, v and x (x) F (about the instance's local
// origin) per thread, float pairs for FP32 inputs (FP64 for FP64 inputs),
// then a fixed-order tree: FP32 partials are transposed through shared
// memory so that each warp reduces one or two quantities in float pairs and
// converts once to FP64. Torque about the centroid:
// sum (x - c) x F = sum x x F - c x sum F.
// Blocks [n_inst, n_inst + 3 n_boxes): box b, lattice d -- h^3 * sum of the
// values the last spread added, from the per-tile FP64 partials in tile order.
// parts selects what one launch writes: 1 the x/F sums (centroid, sum F,
// torque: entries 0..8), 2 sum v (entries 9..11) and the box blocks, 3 all;
// the sums of one quantity do not depend on parts.

constexpr int kReduceThreads = 256;

// Float-pair partials of one node's x, F and x (x) F terms (the x/F sums).
__device__ __forceinline__ void df_add_xF(DF q[9], const float xk[3], const float Fk[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        df_add(q[a], xk[a]);
        df_add(q[3 + a], Fk[a]);
    }
    df_add_prod(q[6], xk[1], Fk[2]);
    df_add_prod(q[6], -xk[2], Fk[1]);
    df_add_prod(q[7], xk[2], Fk[0]);
    df_add_prod(q[7], -xk[0], Fk[2]);
    df_add_prod(q[8], xk[0], Fk[1]);
    df_add_prod(q[8], -xk[1], Fk[0]);
}

// Fixed-order total of kReduceThreads float-pair partials (one warp: lane
// sums over a stride of 32, then a shuffle tree); the value is in lane 0.
__device__ __forceinline__ double df_row_total(const float2 *row, int lane)
{
    DF s{0.f, 0.f};
    for (int k = lane; k < kReduceThreads; k += 32) {
        const float2 e = row[k];
        df_add_df(s, DF{e.x, e.y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF y{__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o)};
        df_add_df(s, y);
    }
    return (double)s.hi + (double)s.lo;
}

// Entries 0..8 of a particle's sums from the totals of x, F and x (x) F:
// centroid, sum F, torque about the centroid, sum (x - c) x F = sum x x F - c x sum F.
__device__ __forceinline__ void write_xF_sums(double *o, const double *tot, int n_nodes)
{
    const double c[3] = {tot[0] / n_nodes, tot[1] / n_nodes, tot[2] / n_nodes};
    const double *S = tot + 3;
    o[0] = c[0];
    o[1] = c[1];
    o[2] = c[2];
    o[3] = S[0];
    o[4] = S[1];
    o[5] = S[2];
    o[6] = tot[6] - (c[1] * S[2] - c[2] * S[1]);
    o[7] = tot[7] - (c[2] * S[0] - c[0] * S[2]);
    o[8] = tot[8] - (c[0] * S[1] - c[1] * S[0]);
}

template <typename real>
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(DevBatch b, DevGrid g,
                                                               const double *__restrict__ red_tile,
                                                               const real *__restrict__ x,
                                                               const real *__restrict__ F,
                                                               const real *__restrict__ v, double *__restrict__ red,
                                                               int parts)
{
    __shared__ double sh[kReduceThreads];
    __shared__ double tot[12];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (blockIdx.x >= b.n_inst) {
        const int k = blockIdx.x - b.n_inst, bx = k / 3, d = k - 3 * bx;
        const BoxDev B = g.boxes[bx];
        const long long nt = (long long)B.T * B.T * B.T;
        double s = 0.0;
        for (long long t = threadIdx.x; t < nt; t += blockDim.x)
            s += red_tile[3 * (B.tile_base + t) + d];
        const double r = block_sum<kReduceThreads>(s, sh);
        if (threadIdx.x == 0) {
            double *o = red + 12LL * b.n_inst + 6LL * bx;
            o[d] = r;
            o[3 + d] = 0.0;
        }
        return;
    }
    const InstDev I = b.inst[blockIdx.x];
    const long long N = b.N;
    if constexpr (std::is_same<real, float>::value) {
        __shared__ float2 part[12][kReduceThreads];
        DF q[12];
#pragma unroll
        for (int i = 0; i < 12; ++i)
            q[i] = DF{0.f, 0.f};
        if (parts & 1) {
#pragma unroll 4
            for (int k = threadIdx.x; k < I.n_nodes; k += blockDim.x) {
                const int node = I.node_off + k;
                float xk[3], Fk[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    xk[a] = x[a * N + node];
                    Fk[a] = F ? F[a * N + node] : 0.f;
                }
                df_add_xF(q, xk, Fk);
            }
        }
        if ((parts & 2) && v) {
#pragma unroll 4
            for (int k = threadIdx.x; k < I.n_nodes; k += blockDim.x) {
                const int node = I.node_off + k;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    df_add(q[9 + a], v[a * N + node]);
            }
        }
#pragma unroll
        for (int i = 0; i < 12; ++i)
            part[i][threadIdx.x] = make_float2(q[i].hi, q[i].lo);
        __syncthreads();
        for (int i = wid; i < 12; i += nw) {
            const bool want = i < 9 ? (parts & 1) != 0 : (parts & 2) != 0;
            if (!want)
                continue;
            const double t = df_row_total(part[i], lane);
            if (lane == 0)
                tot[i] = t;
        }
    } else {
        double p[12];
#pragma unroll
        for (int i = 0; i < 12; ++i)
            p[i] = 0.0;
        for (int k = threadIdx.x; k < I.n_nodes; k += blockDim.x) {
            const int node = I.node_off + k;
            if (parts & 1) {
                double xk[3], Fk[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    xk[a] = (double)x[a * N + node];
                    Fk[a] = F ? (double)F[a * N + node] : 0.0;
                    p[a] += xk[a];
                    p[3 + a] += Fk[a];
                }
                p[6] += xk[1] * Fk[2] - xk[2] * Fk[1];
                p[7] += xk[2] * Fk[0] - xk[0] * Fk[2];
                p[8] += xk[0] * Fk[1] - xk[1] * Fk[0];
            }
            if (parts & 2) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    p[9 + a] += v ? (double)v[a * N + node] : 0.0;
            }
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            double t = p[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0)
                sh[i * 8 + wid] = t;
        }
        __syncthreads();
        if (threadIdx.x < 12) {
            double t = 0.0;
            for (int k = 0; k < nw; ++k)
                t += sh[threadIdx.x * 8 + k];
            tot[threadIdx.x] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double *o = red + 12LL * blockIdx.x;
        if (parts & 1)
            write_xF_sums(o, tot, I.n_nodes);
        if (parts & 2) {
            o[9] = tot[9];
            o[10] = tot[10];
            o[11] = tot[11];
        }
    }
}

}  // namespace ifem
