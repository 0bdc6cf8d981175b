// common.cuh -- device-side data layout and helpers shared by the libifem
// kernels (internal; not part of the C ABI).
//
// Data layout in device memory
//   node arrays   SoA: component a of node k at arr[a*N + k]
//   instances     InstDev[n_inst]: template, box, first node, first element,
//                 FP64 origin and its split origin*(n/L) = I0 + f0 (FP32 mode)
//   templates     TmplDev[n_tmpl]: element connectivity, reference data
//                 (FP64 and an FP32 copy), node->element incidence CSR
//   boxes         BoxDev[n_boxes]: cells per side, tiles, field offset
//   grid field    per box: 3 lattices of n^3 values, x fastest
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ifem {

constexpr int kMaxTileEdge = 20;   // tile edge t + 4 at most (t <= 16)
constexpr int kOwnSub = 5;         // own-list sub-blocks (4 cells) per tile axis (tile edge <= 20)
constexpr int kOwnSub3 = kOwnSub * kOwnSub * kOwnSub;
constexpr int kScanThreads = 512;  // tile-count scan: threads per block
constexpr int kScanPer = 4;        // and values per thread
constexpr int kScanBlock = kScanThreads * kScanPer;
constexpr int kCounters = 16;      // DevWork::counters entries
// FP32 fused force kernel: 7 floats of shared memory per template node
constexpr int kMaxCtaSmemBytes = 227 * 1024;   // opt-in dynamic shared memory of one CTA
constexpr int kFusedMaxSmemBytes = kMaxCtaSmemBytes;
__host__ __device__ inline size_t fused_smem_bytes(int n_nodes) { return (size_t)7 * n_nodes * sizeof(float); }
constexpr int kStatusWords = 8;
enum StatusWord {
    ST_INVERTED = 0,
    ST_DOMAIN = 1,
    ST_CAPACITY = 2,
    ST_TIMEOUT = 3,
    ST_PAIRS = 4,
    ST_ACTIVE = 5,
    ST_TOUCHED = 6,
};

struct TmplDev {
    int kind;        // 0 membrane (triangles), 1 solid (tetrahedra)
    int law;         // membrane law (0 neo-Hookean, 1 Skalak)
    int n_nodes;
    int n_elems;
    const int *elems;      // 3 or 4 node ids per element (template-local)
    const double *ref_d;   // membrane: [m00 m01 m10 m11 A0]; solid: [M (3x3 row-major), V0]
    const float *ref_f;    // FP32 copy of ref_d
    const int *inc_off;    // n_nodes + 1: incidence CSR offsets
    const int *inc_idx;    // element*4 + local vertex, ascending element id
    const int2 *ring;      // membranes: per incidence, the other two vertices (j, k) of the
                           // triangle in its orientation order starting at the vertex
    double mu, C, kb, c0, lam;
};

struct InstDev {
    int tmpl;
    int box;
    int node_off;
    int n_nodes;
    long long elem_off;    // first element of this instance in element buffers
    int n_elems;
    int pad;
    double origin[3];
    int I0[3];             // floor(origin * n/L)      (FP32 transfer)
    float f0[3];           // origin * n/L - I0        (FP32 transfer)
};

struct BoxDev {
    int n;           // cells per side
    int t;           // nominal tile edge
    int T;           // tiles per axis (last tile absorbs the remainder, edge <= t + 4)
    int pad;
    long long tile_base;
    long long grid_off;    // offset of this box's first value in a grid field
    double L;
    double inv_h;          // n / L
    double scale;          // (n/L)^3
    float inv_h_f;         // FP32 copies for the FP32 kernels (no FP64 pipe use)
    float scale_f;
};

struct DevBatch {
    int n_inst;
    int n_tmpl;
    long long N;
    int max_nodes;
    int max_elems;
    long long n_elems_total;
    int any_bending;       // some membrane template has kb != 0
    int fused_ok;          // every template fits the FP32 fused shared-memory kernel
    const InstDev *inst;
    const TmplDev *tmpl;
    const int *node_inst;
};

struct DevGrid {
    int n_boxes;
    long long n_tiles;
    int max_edge;
    const BoxDev *boxes;
};

// FP64 Peskin stencil of one node on the three MAC lattices (deterministic
// FP64 path), computed once per binning from the positions: per lattice d
// and axis a the wrapped first stencil index base[d][a] and the four weights
// ph[d][a][m]; lo[a] is the wrapped cell index c - 2, the low corner of the
// reach of all three lattices.
struct DetW {
    double ph[3][3][4];
    int base[3][3];
    int lo[3];
};
static_assert(sizeof(DetW) == 336, "DetW layout");

struct DevWork {
    int *cand_count;    // n_tiles + 1
    int *cand_off;      // n_tiles + 1
    int *cand_cursor;   // n_tiles
    int *cand_nodes;    // pair list: node id per (tile, node) candidate pair
    long long cand_cap;
    int *own_count;     // per (tile, 4^3 sub-block): n_tiles * kOwnSub3 + 1, then own_flag, tile_fsum
    int *own_flag;      // n_tiles (FP32 halo path): 1 where the tile owns a node
    float *tile_fsum;   // 3 per tile (FP32 halo path): sum of |F_d| over the tile's own nodes, from the
                        // placement when it is given the forces (the fused transfer's fixed-point scale)
    int *own_off;       // n_tiles * kOwnSub3 + 1 offsets; the FP32 halo path finalises the tile
                        // boundaries only (entries t * kOwnSub3)
    int *own_cursor;    // fill cursors; local (per scan block) offsets in the FP32 halo path
    int *own_nodes;     // N entries: nodes grouped by the tile (and sub-block) of their cell
    float4 *own_rec;    // beside own_nodes (FP32 halo path): fractional cell coordinates x, y, z of
                        // the node and, in w, its cell within the tile packed as 8-bit x | y << 8 | z << 16
    int2 *node_key;     // N entries, by node (FP32 halo path): own-list key (-1: not binned) and
                        // the node's rank among the nodes of that key
    float4 *node_rec;   // N entries, by node (FP32 halo path): the own_rec entry of the node
    int *active;        // tiles with candidate pairs
    int *own_tiles;     // tiles with own nodes (FP32 halo path), counters[3] of them
    int *counters;      // kCounters: [0] n_active, [2] work counter, [3] tiles with own nodes,
                        // [4] total pairs, [5] total own nodes, [1] [6] [7] work counters of
                        // one-lattice launches, [8] scan blocks finished
    int *scan_blocks;   // block partial sums for the tile scan
    void *elem_buf;     // per element nodal forces (12 reals per element)
    void *bend_buf;     // per node bending scratch (A, kH, n[3], lap) 6 reals
    double *red_tile;   // per active tile: 3 FP64 sums of added spread values
    DetW *wtab;         // N entries (FP64 Peskin only, else null): written by the binning
    unsigned long long *status;  // kStatusWords
};

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int wrapi(long long i, int n)
{
    long long m = i % n;
    return (int)(m < 0 ? m + n : m);
}

// Tile of a (wrapped) cell along one axis: tiles of edge t, the last one
// absorbing the remainder.
__host__ __device__ inline int tile_of(int c, int t, int T)
{
    int j = c / t;
    return j < T - 1 ? j : T - 1;
}
__host__ __device__ inline int tile_start(int j, int t) { return j * t; }
__host__ __device__ inline int tile_edge(int j, int t, int T, int n) { return j < T - 1 ? t : n - j * t; }

// Tiles per axis for a box of n cells and nominal tile edge t: every tile has
// at least 5 cells (so 5 consecutive cells meet at most 2 tiles) and at most
// t + 4.
__host__ __device__ inline int tiles_per_axis(int n, int t)
{
    int T = (n + t - 1) / t;
    int r = n - (T - 1) * t;
    if (T > 1 && r < 5)
        T -= 1;
    return T;
}

// Adams-Bashforth position update of one value (Eq. Bashforth_eqn),
// x + dt*(1.5*v - 0.5*vp) rounded operation by operation in this order (no
// contraction into FMAs), so every kernel that takes it gives the same bits.
__device__ __forceinline__ float ab2_value(float x, float v, float vp, float dt)
{
    return __fadd_rn(x, __fmul_rn(dt, __fsub_rn(__fmul_rn(1.5f, v), __fmul_rn(0.5f, vp))));
}
__device__ __forceinline__ double ab2_value(double x, double v, double vp, double dt)
{
    return __dadd_rn(x, __dmul_rn(dt, __dsub_rn(__dmul_rn(1.5, v), __dmul_rn(0.5, vp))));
}

// Reductions into shared memory addressed by 32-bit shared-window offsets
// (no generic-to-shared address check per access).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void red_shared_add(unsigned a, int v)
{
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_shared_add(unsigned a, float v)
{
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

__device__ inline void status_add(unsigned long long *st, int w, unsigned long long v)
{
    if (v)
        atomicAdd(st + w, v);
}

// 4-point discrete delta (Peskin 2002), evaluation order fixed:
//   a = |r|, q = 4a; |r| <= 1: ((3 - 2a) + sqrt((1 + q) - q*a)) * 0.125
//   1 < |r| <= 2: ((5 - 2a) - sqrt(((12a) - 7) - q*a)) * 0.125
template <typename real>
__device__ __forceinline__ real phi4(real r)
{
    real a = r < real(0) ? -r : r;
    real q = real(4) * a;
    if (a <= real(1)) {
        real t = (real(1) + q) - q * a;
        return ((real(3) - real(2) * a) + sqrt(t)) * real(0.125);
    }
    if (a <= real(2)) {
        real t = ((real(12) * a) - real(7)) - q * a;
        return ((real(5) - real(2) * a) - sqrt(t)) * real(0.125);
    }
    return real(0);
}

// MLS cubic-spline weight W(r) (Sec. "Interpolation Scheme"; first branch
// read as 2/3 - 4r^2 + 4r^3, continuous at r = 1/2).
template <typename real>
__device__ __forceinline__ real mls_w(real r)
{
    if (r <= real(0.5))
        return real(2.0 / 3.0) - real(4) * r * r + real(4) * r * r * r;
    if (r <= real(1))
        return real(4.0 / 3.0) - real(4) * r + real(4) * r * r - real(4.0 / 3.0) * r * r * r;
    return real(0);
}

// Linear MLS weights at one point: s = lattice coordinates (3), support in
// cells. base = floor(s + 1/2) - 1 (unwrapped). w[27] in z-outer, x-inner
// order. Returns false if the 4x4 moment matrix is not positive definite.
template <typename real>
__device__ inline bool mls_weights(const real s[3], real support, int base[3], real w[27])
{
    real A[10];   // packed lower triangle of the symmetric 4x4 moment matrix
#pragma unroll
    for (int i = 0; i < 10; ++i)
        A[i] = real(0);
    for (int a = 0; a < 3; ++a)
        base[a] = (int)floor(s[a] + real(0.5)) - 1;
    int J = 0;
    for (int kz = 0; kz < 3; ++kz)
        for (int jy = 0; jy < 3; ++jy)
            for (int ix = 0; ix < 3; ++ix, ++J) {
                real y0 = real(base[0] + ix) - s[0];
                real y1 = real(base[1] + jy) - s[1];
                real y2 = real(base[2] + kz) - s[2];
                real Wj = mls_w(sqrt(y0 * y0 + y1 * y1 + y2 * y2) / support);
                w[J] = Wj;
                real p[4] = {real(1), y0, y1, y2};
                int q = 0;
                for (int r = 0; r < 4; ++r)
                    for (int c = 0; c <= r; ++c, ++q)
                        A[q] += Wj * p[r] * p[c];
            }
    // Cholesky of the packed matrix, then solve A z = e1.
    real Lm[10];
    int q = 0;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c <= r; ++c, ++q) {
            real acc = A[q];
            for (int k = 0; k < c; ++k)
                acc -= Lm[r * (r + 1) / 2 + k] * Lm[c * (c + 1) / 2 + k];
            if (r == c) {
                if (!(acc > real(0)))
                    return false;
                Lm[q] = sqrt(acc);
            } else {
                Lm[q] = acc / Lm[c * (c + 1) / 2 + c];
            }
        }
    real y[4], z[4];
    for (int r = 0; r < 4; ++r) {
        real acc = r == 0 ? real(1) : real(0);
        for (int k = 0; k < r; ++k)
            acc -= Lm[r * (r + 1) / 2 + k] * y[k];
        y[r] = acc / Lm[r * (r + 1) / 2 + r];
    }
    for (int r = 3; r >= 0; --r) {
        real acc = y[r];
        for (int k = r + 1; k < 4; ++k)
            acc -= Lm[k * (k + 1) / 2 + r] * z[k];
        z[r] = acc / Lm[r * (r + 1) / 2 + r];
    }
    J = 0;
    for (int kz = 0; kz < 3; ++kz)
        for (int jy = 0; jy < 3; ++jy)
            for (int ix = 0; ix < 3; ++ix, ++J) {
                real y0 = real(base[0] + ix) - s[0];
                real y1 = real(base[1] + jy) - s[1];
                real y2 = real(base[2] + kz) - s[2];
                w[J] = w[J] * (z[0] + z[1] * y0 + z[2] * y1 + z[3] * y2);
            }
    return true;
}

// Lattice coordinate of node k along axis a for MAC component d.
//   FP64: s = (origin + x) * (n/L) - o, I0 = 0  (exact order of the oracle)
//   FP32: s = (f0 - o) + x * (n/L) relative to the integer offset I0
template <typename real>
struct LatCoord;

template <>
struct LatCoord<double> {
    __device__ static inline double get(const InstDev &I, const BoxDev &B, int a, double x, double o, int &I0)
    {
        I0 = 0;
        double p = I.origin[a] + x;
        return p * B.inv_h - o;
    }
};

template <>
struct LatCoord<float> {
    __device__ static inline float get(const InstDev &I, const BoxDev &B, int a, float x, float o, int &I0)
    {
        I0 = I.I0[a];
        return (I.f0[a] - o) + x * B.inv_h_f;
    }
};

// ------------------------------------------------------------- launchers
struct ForcesArgs {
    DevBatch b;
    DevWork w;
    const void *x;
    void *F;
    const void *wv;   // HVP direction (or null)
    int scatter;      // 0 det, 1 atomic
    int hvp;          // 1: compute Hw instead of F
    int inst0, inst_n;  // particle range [inst0, inst0 + inst_n) (inst_n = 0: all); the FP32
                        // one-CTA-per-particle kernel only (forces_ranged_ok)
    cudaStream_t stream;
};

struct TransferArgs {
    DevBatch b;
    DevGrid g;
    DevWork w;
    const void *x;
    const void *F;
    const void *u;
    void *f;
    void *v;
    int kernel;       // 0 Peskin4, 1 MLS27
    int density;
    double support;
    int n_sm;
    int acc64;        // FP32 spread: 64-bit (1) or 32-bit (0) fixed-point accumulators
    int halo;         // FP32 Peskin spread with halo scatter (IFEM_SCATTER_ATOMIC): 1; 2 with the
                      // velocity box staged in shared memory when interpolation is fused
    int binned;       // the binning of this step ran just before on the same stream (own tiles
                      // listed, work counter and per-tile sums cleared)
    int lattice;      // staged fused transfer: -1 all three lattices, else that lattice only
    int pdl;          // staged fused transfer: may start before the previous kernel in the stream ends
    int use_wtab;     // FP64 Peskin interpolation: read the stencils the binning of x tabulated
    const void *vp;   // fused position update (halo spread + interpolation only):
    void *xn;         //   xn = x + dt (3/2 v - 1/2 vp) when xn is not null
    double dt;
    cudaStream_t stream;
};

struct ReduceArgs {
    DevBatch b;
    DevGrid g;
    DevWork w;
    const void *x;
    const void *F;
    const void *v;
    double *red;
    int parts;        // 1: per-particle x/F sums; 2: per-particle sum v and the per-box sums; 3: all
    cudaStream_t stream;
};

// Defined once per precision in kernels_f32.cu / kernels_f64.cu.
cudaError_t launch_forces_f32(const ForcesArgs &a);
cudaError_t launch_forces_f64(const ForcesArgs &a);
// Binning in two parts: the clears, the count pass and the scan, then the
// placement (which also sums |F| per tile when TransferArgs::F is given).
// Only the FP32 halo path (with_cand = 0) takes them apart.
enum BinStage { BIN_COUNT = 1, BIN_PLACE = 2, BIN_ALL = 3 };
cudaError_t launch_bin_f32(const TransferArgs &a, int det_sort, int with_cand, int stages = BIN_ALL);
cudaError_t launch_bin_f64(const TransferArgs &a, int det_sort, int with_cand, int stages = BIN_ALL);
cudaError_t launch_spread_f32(const TransferArgs &a);
cudaError_t launch_spread_f64(const TransferArgs &a);
cudaError_t launch_interp_f32(const TransferArgs &a);
cudaError_t launch_interp_f64(const TransferArgs &a);
cudaError_t launch_reduce_f32(const ReduceArgs &a);
cudaError_t launch_reduce_f64(const ReduceArgs &a);

// Fluid-stress forces inside solids: F = (F +) sum of element contributions.
struct FluidArgs {
    DevBatch b;
    DevWork w;
    const void *x;
    const void *u;
    const void *C;    // 6 rows of N, or null
    double eta;
    double cp;        // eta (1 - beta) / lambda
    int add;          // 1: F = F + fluid forces
    void *F;
    cudaStream_t stream;
};
cudaError_t launch_fluid_f32(const FluidArgs &a);
cudaError_t launch_fluid_f64(const FluidArgs &a);
// Cell-centred multi-component interpolation (TransferArgs.u = field).
cudaError_t launch_interp_cc_f32(const TransferArgs &a, int ncomp);
cudaError_t launch_interp_cc_f64(const TransferArgs &a, int ncomp);

// Lagrangian update: AB2 positions, volumes, membrane volume correction.
struct LagrangeArgs {
    DevBatch b;
    void *x;
    void *x_out;      // AB2 result (null: in place)
    const void *v;
    const void *vp;
    double dt;
    const double *V0;
    double *out;      // volumes, or Lambda per instance (may be null for the correction)
    double *alpha;    // 3 doubles per node of scratch (correction)
    unsigned long long *status;
    cudaStream_t stream;
};
cudaError_t launch_ab2_f32(const LagrangeArgs &a);
cudaError_t launch_ab2_f64(const LagrangeArgs &a);
cudaError_t launch_volume_f32(const LagrangeArgs &a);
cudaError_t launch_volume_f64(const LagrangeArgs &a);
cudaError_t launch_vcorr_f32(const LagrangeArgs &a);
cudaError_t launch_vcorr_f64(const LagrangeArgs &a);
cudaError_t launch_area_normals_f32(const DevBatch &b, const void *x, void *nA, cudaStream_t s);
cudaError_t launch_area_normals_f64(const DevBatch &b, const void *x, void *nA, cudaStream_t s);

}  // namespace ifem
