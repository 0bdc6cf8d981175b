// api.cu -- the extern "C" entry points of libifem (declared in ifem.h):
// handle management, host-side argument checks, FP64 reference data of the
// templates, work-buffer sizing and the launch sequences of the coupling
// step. Host code here is compiled with -ffp-contract=off so that the FP64
// reference invariants follow the exact evaluation order written below.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ifem.h"
#include "common.cuh"

using namespace ifem;

#include "handles.h"

// ------------------------------------------------------------ helpers
static int fail(ifem_ctx ctx, int code, const std::string &msg)
{
    if (ctx)
        ctx->err = msg;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? IFEM_ERR_OOM : IFEM_ERR_CUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

template <typename T>
static cudaError_t upload(T **dst, const T *src, size_t n)
{
    *dst = nullptr;
    if (n == 0)
        return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * n);
    if (e != cudaSuccess)
        return e;
    return cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
}

static size_t real_size(ifem_ctx ctx) { return ctx->cfg.precision == IFEM_FP64 ? 8 : 4; }

// ------------------------------------------------------------ context
extern "C" int ifem_config_default(ifem_config *cfg)
{
    if (!cfg)
        return IFEM_ERR_ARG;
    cfg->precision = IFEM_FP32;
    cfg->kernel = IFEM_KERNEL_PESKIN4;
    cfg->scatter = IFEM_SCATTER_DET;
    cfg->tile = 0;
    cfg->mls_support = 0.0;
    cfg->device = 0;
    cfg->profile = 0;
    return IFEM_OK;
}

extern "C" int ifem_ctx_create(const ifem_config *cfg, ifem_ctx *out)
{
    DeviceScope ifem_device_scope_(cfg ? cfg->device : -1);
    ifem_ctx ctx = nullptr;
    if (!cfg || !out)
        return IFEM_ERR_ARG;
    *out = nullptr;
    if (cfg->precision != IFEM_FP32 && cfg->precision != IFEM_FP64)
        return IFEM_ERR_ARG;
    if (cfg->kernel != IFEM_KERNEL_PESKIN4 && cfg->kernel != IFEM_KERNEL_MLS27)
        return IFEM_ERR_ARG;
    if (cfg->scatter != IFEM_SCATTER_DET && cfg->scatter != IFEM_SCATTER_ATOMIC)
        return IFEM_ERR_ARG;
    if (cfg->tile != 0 && (cfg->tile < 6 || cfg->tile > 16))
        return IFEM_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
        return IFEM_ERR_CUDA;
    ctx = new ifem_ctx_s();
    ctx->cfg = *cfg;
    if (!(ctx->cfg.mls_support > 0.0))
        ctx->cfg.mls_support = std::sqrt(3.0);
    // default tile edge: 16 cells for the FP32 kernels (fewer (tile, node)
    // pairs), 8 for the deterministic FP64 spread (its cost grows with the
    // candidates per tile times the values per tile)
    ctx->tile = cfg->tile ? cfg->tile : (cfg->precision == IFEM_FP64 ? 8 : 16);
    // FP32 spread accumulator width (tuning knob): IFEM_SPREAD_ACC=64 selects
    // 64-bit fixed point (slower shared-memory atomics), anything else 32-bit
    if (const char *acc = std::getenv("IFEM_SPREAD_ACC"))
        ctx->acc64 = std::string(acc) == "64" ? 1 : 0;
    // fused FP32 transfer kernel (tuning knob): the velocity box of each item
    // is staged in shared memory (transfer_staged_kernel) unless
    // IFEM_TRANSFER=halo selects the kernel that gathers velocities through L1
    ctx->staged = 1;
    if (const char *tr = std::getenv("IFEM_TRANSFER"))
        ctx->staged = std::string(tr) == "halo" ? 0 : 1;
    if (cudaSetDevice(cfg->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess ||
        cudaMalloc((void **)&ctx->d_status, sizeof(unsigned long long) * kStatusWords) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(unsigned long long) * kStatusWords) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_status, sizeof(unsigned long long) * kStatusWords) != cudaSuccess) {
        if (ctx->d_status)
            cudaFree(ctx->d_status);
        delete ctx;
        return IFEM_ERR_CUDA;
    }
    for (int i = 0; i < 2; ++i)
        if (cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking) != cudaSuccess) {
            ifem_ctx_destroy(ctx);
            return IFEM_ERR_CUDA;
        }
    for (int i = 0; i < ifem_ctx_s::kForkEvents; ++i)
        if (cudaEventCreateWithFlags(&ctx->fork[i], cudaEventDisableTiming) != cudaSuccess) {
            ifem_ctx_destroy(ctx);
            return IFEM_ERR_CUDA;
        }
    if (cfg->profile) {
        ctx->ev_ok = 1;
        for (int i = 0; i < 6; ++i)
            if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess)
                ctx->ev_ok = 0;
    }
    *out = ctx;
    return IFEM_OK;
}

extern "C" int ifem_ctx_destroy(ifem_ctx ctx)
{
    IFEM_DEVICE_SCOPE(ctx);
    if (!ctx)
        return IFEM_ERR_ARG;
    for (int i = 0; i < 6; ++i)
        if (ctx->ev[i])
            cudaEventDestroy(ctx->ev[i]);
    for (int i = 0; i < ifem_ctx_s::kForkEvents; ++i)
        if (ctx->fork[i])
            cudaEventDestroy(ctx->fork[i]);
    for (int i = 0; i < 2; ++i)
        if (ctx->aux[i])
            cudaStreamDestroy(ctx->aux[i]);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    delete ctx;
    return IFEM_OK;
}

extern "C" const char *ifem_last_error(ifem_ctx ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int ifem_ctx_tile(ifem_ctx ctx) { return ctx ? ctx->tile : IFEM_ERR_ARG; }

extern "C" int ifem_stage_times(ifem_ctx ctx, double *ms)
{
    IFEM_DEVICE_SCOPE(ctx);
    if (!ctx || !ms || !ctx->ev_ok || !ctx->ev_recorded)
        return fail(ctx, IFEM_ERR_ARG, "stage_times: profiling off or no step recorded");
    CK(cudaEventSynchronize(ctx->ev[5]));
    // the step records ev1, forces, ev0, binning, ev2, spread, ev3, interp, ev4, sums, ev5
    const int from[5] = {0, 1, 2, 3, 4}, to[5] = {2, 0, 3, 4, 5};
    for (int i = 0; i < 5; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ctx->ev[from[i]], ctx->ev[to[i]]));
        ms[i] = t;
    }
    if (ctx->ev_fused) {
        ms[2] += ms[3];
        ms[3] = 0.0;
    }
    return IFEM_OK;
}

static void mark(ifem_ctx ctx, int i, void *stream)
{
    if (ctx->ev_ok)
        cudaEventRecord(ctx->ev[i], (cudaStream_t)stream);
}

extern "C" int ifem_sync_status(ifem_ctx ctx, ifem_stats *out)
{
    IFEM_DEVICE_SCOPE(ctx);
    if (!ctx)
        return IFEM_ERR_ARG;
    CK(cudaSetDevice(ctx->cfg.device));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(ctx->h_status, ctx->d_status, sizeof(unsigned long long) * kStatusWords, cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->d_status, 0, sizeof(unsigned long long) * kStatusWords));
    const unsigned long long *s = ctx->h_status;
    if (out) {
        out->inverted_elements = (int64_t)s[ST_INVERTED];
        out->domain_errors = (int64_t)s[ST_DOMAIN];
        out->capacity_errors = (int64_t)s[ST_CAPACITY];
        out->timeouts = (int64_t)s[ST_TIMEOUT];
        out->pairs = (int64_t)s[ST_PAIRS];
        out->active_tiles = (int64_t)s[ST_ACTIVE];
        out->touched_cells = (int64_t)s[ST_TOUCHED];
    }
    if (s[ST_TIMEOUT])
        return fail(ctx, IFEM_ERR_TIMEOUT, "a bounded device wait expired");
    if (s[ST_DOMAIN])
        return fail(ctx, IFEM_ERR_DOMAIN, "non-finite position or singular MLS moment matrix");
    if (s[ST_CAPACITY])
        return fail(ctx, IFEM_ERR_CAPACITY, "a per-tile list exceeded the deterministic kernels' limit");
    if (s[ST_INVERTED])
        return fail(ctx, IFEM_ERR_INVERTED, "inverted elements (J <= 0) were evaluated");
    return IFEM_OK;
}

// ------------------------------------------------------------ templates
// Membrane reference data per triangle (a, b, c), FP64, in this order:
//   E1 = Xb - Xa, E2 = Xc - Xa; l1 = sqrt((E1x^2 + E1y^2) + E1z^2); e1 = E1 / l1;
//   nr = E1 x E2; nl = sqrt((nrx^2 + nry^2) + nrz^2); nh = nr / nl; e2 = nh x e1;
//   d01 = (e1x E2x + e1y E2y) + e1z E2z; d11 = (e2x E2x + e2y E2y) + e2z E2z;
//   Dm^-1 = [1/l1, -d01/(l1*d11); 0, 1/d11]; A0 = 0.5*nl.
static void membrane_reference(int nt, const int32_t *tri, const double *X, std::vector<double> &ref)
{
    ref.assign((size_t)nt * 5, 0.0);
    for (int e = 0; e < nt; ++e) {
        const double *Xa = X + 3 * tri[3 * e], *Xb = X + 3 * tri[3 * e + 1], *Xc = X + 3 * tri[3 * e + 2];
        double E1[3], E2[3], e1[3], nr[3], nh[3], e2[3];
        for (int i = 0; i < 3; ++i) {
            E1[i] = Xb[i] - Xa[i];
            E2[i] = Xc[i] - Xa[i];
        }
        double l1 = std::sqrt((E1[0] * E1[0] + E1[1] * E1[1]) + E1[2] * E1[2]);
        for (int i = 0; i < 3; ++i)
            e1[i] = E1[i] / l1;
        nr[0] = E1[1] * E2[2] - E1[2] * E2[1];
        nr[1] = E1[2] * E2[0] - E1[0] * E2[2];
        nr[2] = E1[0] * E2[1] - E1[1] * E2[0];
        double nl = std::sqrt((nr[0] * nr[0] + nr[1] * nr[1]) + nr[2] * nr[2]);
        for (int i = 0; i < 3; ++i)
            nh[i] = nr[i] / nl;
        e2[0] = nh[1] * e1[2] - nh[2] * e1[1];
        e2[1] = nh[2] * e1[0] - nh[0] * e1[2];
        e2[2] = nh[0] * e1[1] - nh[1] * e1[0];
        double d01 = (e1[0] * E2[0] + e1[1] * E2[1]) + e1[2] * E2[2];
        double d11 = (e2[0] * E2[0] + e2[1] * E2[1]) + e2[2] * E2[2];
        double *r = ref.data() + 5 * (size_t)e;
        r[0] = 1.0 / l1;
        r[1] = -d01 / (l1 * d11);
        r[2] = 0.0;
        r[3] = 1.0 / d11;
        r[4] = 0.5 * nl;
    }
}

// Solid reference data per tet: Dm = [X1-X0, X2-X0, X3-X0] (columns),
// det by cofactors of row 0, Dm^-1 = adj(Dm)/det (rows = grad N_1..3),
// V0 = det / 6.
static bool tet_reference(int ne, const int32_t *tet, const double *X, std::vector<double> &ref)
{
    ref.assign((size_t)ne * 10, 0.0);
    for (int e = 0; e < ne; ++e) {
        const double *X0 = X + 3 * tet[4 * e];
        double M[3][3];
        for (int c = 0; c < 3; ++c) {
            const double *Xc = X + 3 * tet[4 * e + 1 + c];
            for (int i = 0; i < 3; ++i)
                M[i][c] = Xc[i] - X0[i];
        }
        double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                   - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                   + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        if (!(det > 0.0))
            return false;
        double *r = ref.data() + 10 * (size_t)e;
        r[0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
        r[1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
        r[2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
        r[3] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
        r[4] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
        r[5] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
        r[6] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
        r[7] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
        r[8] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
        r[9] = det / 6.0;
    }
    return true;
}

// Node -> (element*4 + local vertex) incidence, ascending element id.
static void incidence(int nn, int ne, int nv, const int32_t *el, std::vector<int> &off, std::vector<int> &idx)
{
    off.assign(nn + 1, 0);
    for (int e = 0; e < ne; ++e)
        for (int v = 0; v < nv; ++v)
            off[el[nv * e + v] + 1]++;
    for (int i = 0; i < nn; ++i)
        off[i + 1] += off[i];
    idx.assign(off[nn], 0);
    std::vector<int> cur(off.begin(), off.end() - 1);
    for (int e = 0; e < ne; ++e)
        for (int v = 0; v < nv; ++v)
            idx[cur[el[nv * e + v]]++] = e * 4 + v;
}

static int tmpl_upload(ifem_ctx ctx, ifem_tmpl t, int nv, const int32_t *el, const std::vector<double> &ref)
{
    std::vector<float> reff(ref.begin(), ref.end());
    std::vector<int> off, idx;
    incidence(t->n_nodes, t->n_elems, nv, el, off, idx);
    CK(upload(&t->d_elems, el, (size_t)t->n_elems * nv));
    CK(upload(&t->d_ref_d, ref.data(), ref.size()));
    CK(upload(&t->d_ref_f, reff.data(), reff.size()));
    CK(upload(&t->d_inc_off, off.data(), off.size()));
    CK(upload(&t->d_inc_idx, idx.data(), idx.size()));
    if (nv == 3) {
        // vertex one-ring: for each incidence (element e, corner c), the next two
        // corners of e in its orientation order
        std::vector<int2> ring(idx.size());
        for (size_t q = 0; q < idx.size(); ++q) {
            const int e = idx[q] >> 2, c = idx[q] & 3;
            ring[q] = make_int2(el[3 * e + (c + 1) % 3], el[3 * e + (c + 2) % 3]);
        }
        CK(upload(&t->d_ring, ring.data(), ring.size()));
    }
    return IFEM_OK;
}

static int check_elems(int nn, int ne, int nv, const int32_t *el)
{
    for (long long i = 0; i < (long long)ne * nv; ++i)
        if (el[i] < 0 || el[i] >= nn)
            return 0;
    for (int e = 0; e < ne; ++e)
        for (int a = 0; a < nv; ++a)
            for (int b = a + 1; b < nv; ++b)
                if (el[nv * e + a] == el[nv * e + b])
                    return 0;
    return 1;
}

extern "C" int ifem_tmpl_create_membrane(ifem_ctx ctx, int n_nodes, int n_tris, const int32_t *tris,
                                         const double *X_ref, int law, const ifem_membrane_params *p,
                                         ifem_tmpl *out)
{
    IFEM_DEVICE_SCOPE(ctx);
    if (!ctx || !out || !tris || !X_ref || !p || n_nodes < 3 || n_tris < 1)
        return fail(ctx, IFEM_ERR_ARG, "membrane template: null pointer or empty mesh");
    *out = nullptr;
    if (law != IFEM_LAW_NEO_HOOKE && law != IFEM_LAW_SKALAK)
        return fail(ctx, IFEM_ERR_ARG, "membrane template: unknown law");
    if (!check_elems(n_nodes, n_tris, 3, tris))
        return fail(ctx, IFEM_ERR_ARG, "membrane template: node index out of range or repeated");
    if (p->kb != 0.0) {
        // bending needs a closed 2-manifold: every edge shared by exactly two triangles
        std::map<std::pair<int, int>, int> edges;
        for (int e = 0; e < n_tris; ++e)
            for (int c = 0; c < 3; ++c) {
                int a = tris[3 * e + c], b = tris[3 * e + (c + 1) % 3];
                edges[{std::min(a, b), std::max(a, b)}]++;
            }
        for (auto &kv : edges)
            if (kv.second != 2)
                return fail(ctx, IFEM_ERR_ARG, "membrane template: bending needs a closed surface");
    }
    std::vector<double> ref;
    membrane_reference(n_tris, tris, X_ref, ref);
    for (int e = 0; e < n_tris; ++e)
        if (!(ref[5 * (size_t)e + 4] > 0.0) || !std::isfinite(ref[5 * (size_t)e + 1]))
            return fail(ctx, IFEM_ERR_ARG, "membrane template: degenerate reference triangle");
    ifem_tmpl t = new ifem_tmpl_s();
    t->ctx = ctx;
    t->kind = 0;
    t->law = law;
    t->n_nodes = n_nodes;
    t->n_elems = n_tris;
    t->mu = p->mu;
    t->C = p->C;
    t->kb = p->kb;
    t->c0 = p->c0;
    t->lam = 0.0;
    CK(cudaSetDevice(ctx->cfg.device));
    int rc = tmpl_upload(ctx, t, 3, tris, ref);
    if (rc != IFEM_OK) {
        ifem_tmpl_destroy(t);
        return rc;
    }
    *out = t;
    return IFEM_OK;
}

extern "C" int ifem_tmpl_create_solid(ifem_ctx ctx, int n_nodes, int n_tets, const int32_t *tets,
                                      const double *X_ref, const ifem_solid_params *p, ifem_tmpl *out)
{
    IFEM_DEVICE_SCOPE(ctx);
    if (!ctx || !out || !tets || !X_ref || !p || n_nodes < 4 || n_tets < 1)
        return fail(ctx, IFEM_ERR_ARG, "solid template: null pointer or empty mesh");
    *out = nullptr;
    if (!check_elems(n_nodes, n_tets, 4, tets))
        return fail(ctx, IFEM_ERR_ARG, "solid template: node index out of range or repeated");
    std::vector<double> ref;
    if (!tet_reference(n_tets, tets, X_ref, ref))
        return fail(ctx, IFEM_ERR_ARG, "solid template: a reference tet has det <= 0");
    ifem_tmpl t = new ifem_tmpl_s();
    t->ctx = ctx;
    t->kind = 1;
    t->law = 0;
    t->n_nodes = n_nodes;
    t->n_elems = n_tets;
    t->mu = p->mu;
    t->C = 0.0;
    t->kb = 0.0;
    t->c0 = 0.0;
    t->lam = p->lambda;
    CK(cudaSetDevice(ctx->cfg.device));
    int rc = tmpl_upload(ctx, t, 4, tets, ref);
    if (rc != IFEM_OK) {
        ifem_tmpl_destroy(t);
        return rc;
    }
    *out = t;
    return IFEM_OK;
}

extern "C" int ifem_tmpl_destroy(ifem_tmpl t)
{
    IFEM_DEVICE_SCOPE(t ? t->ctx : nullptr);
    if (!t)
        return IFEM_ERR_ARG;
    cudaFree(t->d_elems);
    cudaFree(t->d_ref_d);
    cudaFree(t->d_ref_f);
    cudaFree(t->d_inc_off);
    cudaFree(t->d_inc_idx);
    cudaFree(t->d_ring);
    delete t;
    return IFEM_OK;
}

// ------------------------------------------------------------ grid
extern "C" int ifem_grid_create(ifem_ctx ctx, int n_boxes, const int32_t *n, const double *L, ifem_grid *out)
{
    if (!ctx || !out || !n || !L || n_boxes < 1)
        return fail(ctx, IFEM_ERR_ARG, "grid: null pointer or no boxes");
    *out = nullptr;
    for (int b = 0; b < n_boxes; ++b)
        if (n[b] < 8 || n[b] > 1024 || !(L[b] > 0.0) || !std::isfinite(L[b]))
            return fail(ctx, IFEM_ERR_ARG, "grid: box sides must be 8..1024 cells with L > 0");
    ifem_grid g = new ifem_grid_s();
    g->ctx = ctx;
    g->n_boxes = n_boxes;
    g->n.assign(n, n + n_boxes);
    g->L.assign(L, L + n_boxes);
    g->off.resize(n_boxes);
    long long tot = 0;
    for (int b = 0; b < n_boxes; ++b) {
        g->off[b] = tot;
        tot += 3LL * n[b] * n[b] * n[b];
    }
    g->total = tot;
    *out = g;
    return IFEM_OK;
}

extern "C" int ifem_grid_destroy(ifem_grid g)
{
    if (!g)
        return IFEM_ERR_ARG;
    delete g;
    return IFEM_OK;
}

extern "C" int64_t ifem_grid_values(ifem_grid g) { return g ? g->total : -1; }
extern "C" int64_t ifem_grid_box_offset(ifem_grid g, int b)
{
    return (g && b >= 0 && b < g->n_boxes) ? g->off[b] : -1;
}

// ------------------------------------------------------------ batch
static void split_origins(ifem_batch b, ifem_grid g)
{
    for (size_t i = 0; i < b->h_inst.size(); ++i) {
        InstDev &I = b->h_inst[i];
        double inv_h = (double)g->n[I.box] / g->L[I.box];
        for (int a = 0; a < 3; ++a) {
            double s0 = I.origin[a] * inv_h;
            double fl = std::floor(s0);
            I.I0[a] = (int)((long long)fl % g->n[I.box]);
            I.f0[a] = (float)(s0 - fl);
        }
    }
}

extern "C" int ifem_batch_create(ifem_ctx ctx, int n_tmpl, const ifem_tmpl *tmpls, int n_inst,
                                 const ifem_instance_desc *inst, ifem_grid grid, ifem_batch *out)
{
    IFEM_DEVICE_SCOPE(ctx);
    if (!ctx || !out || !tmpls || n_tmpl < 1 || n_inst < 0 || (n_inst > 0 && !inst) || !grid)
        return fail(ctx, IFEM_ERR_ARG, "batch: null pointer or bad counts");
    *out = nullptr;
    if (n_inst > 65535)
        return fail(ctx, IFEM_ERR_CAPACITY, "batch: at most 65535 instances");
    for (int t = 0; t < n_tmpl; ++t)
        if (!tmpls[t] || tmpls[t]->ctx != ctx)
            return fail(ctx, IFEM_ERR_ARG, "batch: template from another context");
    ifem_batch b = new ifem_batch_s();
    b->ctx = ctx;
    b->tmpls.assign(tmpls, tmpls + n_tmpl);
    b->inst.assign(inst, inst + n_inst);
    b->grid0 = grid;
    long long N = 0, E = 0;
    std::vector<int> node_inst;
    for (int i = 0; i < n_inst; ++i) {
        const ifem_instance_desc &d = inst[i];
        if (d.tmpl < 0 || d.tmpl >= n_tmpl || d.box < 0 || d.box >= grid->n_boxes ||
            !std::isfinite(d.origin[0]) || !std::isfinite(d.origin[1]) || !std::isfinite(d.origin[2])) {
            delete b;
            return fail(ctx, IFEM_ERR_ARG, "batch: instance with bad template, box or origin");
        }
        ifem_tmpl t = tmpls[d.tmpl];
        InstDev I{};
        I.tmpl = d.tmpl;
        I.box = d.box;
        I.node_off = (int)N;
        I.n_nodes = t->n_nodes;
        I.elem_off = E;
        I.n_elems = t->n_elems;
        for (int a = 0; a < 3; ++a)
            I.origin[a] = d.origin[a];
        b->h_inst.push_back(I);
        node_inst.insert(node_inst.end(), t->n_nodes, i);
        N += t->n_nodes;
        E += t->n_elems;
        b->max_nodes = std::max(b->max_nodes, t->n_nodes);
        b->max_elems = std::max(b->max_elems, t->n_elems);
        b->max_box = std::max(b->max_box, d.box);
        if (t->kind == 0 && t->kb != 0.0)
            b->any_bending = 1;
    }
    if (N >= (1LL << 31)) {
        delete b;
        return fail(ctx, IFEM_ERR_CAPACITY, "batch: more than 2^31 - 1 nodes");
    }
    b->N = N;
    b->n_elems = E;
    b->fused_ok = fused_smem_bytes(b->max_nodes) <= (size_t)kFusedMaxSmemBytes;
    split_origins(b, grid);
    std::vector<TmplDev> td(n_tmpl);
    for (int t = 0; t < n_tmpl; ++t) {
        ifem_tmpl s = tmpls[t];
        TmplDev &d = td[t];
        d.kind = s->kind;
        d.law = s->law;
        d.n_nodes = s->n_nodes;
        d.n_elems = s->n_elems;
        d.elems = s->d_elems;
        d.ref_d = s->d_ref_d;
        d.ref_f = s->d_ref_f;
        d.inc_off = s->d_inc_off;
        d.inc_idx = s->d_inc_idx;
        d.ring = s->d_ring;
        d.mu = s->mu;
        d.C = s->C;
        d.kb = s->kb;
        d.c0 = s->c0;
        d.lam = s->lam;
    }
    cudaSetDevice(ctx->cfg.device);
    size_t rs = real_size(ctx);
    if (upload(&b->d_tmpl, td.data(), td.size()) != cudaSuccess ||
        upload(&b->d_inst, b->h_inst.data(), b->h_inst.size()) != cudaSuccess ||
        upload(&b->d_node_inst, node_inst.data(), node_inst.size()) != cudaSuccess ||
        cudaMalloc(&b->d_elem_buf, std::max<size_t>(1, (size_t)E * 12 * rs)) != cudaSuccess ||
        cudaMalloc(&b->d_bend_buf, std::max<size_t>(1, (size_t)N * 6 * rs)) != cudaSuccess) {
        ifem_batch_destroy(b);
        return fail(ctx, IFEM_ERR_OOM, "batch: device allocation failed");
    }
    *out = b;
    return IFEM_OK;
}

static void ws_free(Workspace &ws)
{
    for (void *p : ws.allocs)
        cudaFree(p);
    ws.allocs.clear();
    ws.grid = nullptr;
    ws.tile = 0;
}

extern "C" int ifem_batch_destroy(ifem_batch b)
{
    IFEM_DEVICE_SCOPE(b ? b->ctx : nullptr);
    if (!b)
        return IFEM_ERR_ARG;
    ws_free(b->ws);
    cudaFree(b->d_inst);
    cudaFree(b->d_tmpl);
    cudaFree(b->d_node_inst);
    cudaFree(b->d_elem_buf);
    cudaFree(b->d_bend_buf);
    delete b;
    return IFEM_OK;
}

extern "C" int64_t ifem_batch_nodes(ifem_batch b) { return b ? b->N : -1; }
extern "C" int ifem_batch_instances(ifem_batch b) { return b ? (int)b->inst.size() : -1; }

extern "C" int ifem_batch_set_origins(ifem_batch b, const double *origins)
{
    IFEM_DEVICE_SCOPE(b ? b->ctx : nullptr);
    if (!b || !origins)
        return IFEM_ERR_ARG;
    ifem_ctx ctx = b->ctx;
    for (size_t i = 0; i < b->h_inst.size(); ++i)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(origins[3 * i + a]))
                return fail(ctx, IFEM_ERR_ARG, "set_origins: non-finite origin");
            b->h_inst[i].origin[a] = origins[3 * i + a];
        }
    split_origins(b, b->grid0);
    CK(cudaSetDevice(ctx->cfg.device));
    if (!b->h_inst.empty())
        CK(cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(InstDev) * b->h_inst.size(), cudaMemcpyHostToDevice));
    return IFEM_OK;
}

static int use_halo(ifem_ctx ctx);

// Work buffers for (batch, grid, tile): box/tile tables, per-tile lists.
static int ws_ensure(ifem_ctx ctx, ifem_batch b, ifem_grid g, int tile)
{
    Workspace &ws = b->ws;
    if (ws.grid == g && ws.tile == tile)
        return IFEM_OK;
    ws_free(ws);
    std::vector<BoxDev> boxes(g->n_boxes);
    long long nt = 0;
    int max_edge = 0;
    for (int i = 0; i < g->n_boxes; ++i) {
        BoxDev &B = boxes[i];
        B.n = g->n[i];
        B.t = std::min(tile, B.n);
        B.T = tiles_per_axis(B.n, B.t);
        B.tile_base = nt;
        B.grid_off = g->off[i];
        B.L = g->L[i];
        B.inv_h = (double)B.n / B.L;
        B.scale = B.inv_h * B.inv_h * B.inv_h;
        B.inv_h_f = (float)B.inv_h;
        B.scale_f = (float)B.scale;
        nt += (long long)B.T * B.T * B.T;
        for (int j = 0; j < B.T; ++j)
            max_edge = std::max(max_edge, tile_edge(j, B.t, B.T, B.n));
    }
    if (max_edge > kMaxTileEdge * 2)
        return fail(ctx, IFEM_ERR_CAPACITY, "tile edge too large");
    if (nt * kOwnSub3 >= (1LL << 31) - 1)
        return fail(ctx, IFEM_ERR_CAPACITY, "too many tiles");
    auto alloc = [&](void **p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess)
            ws.allocs.push_back(*p);
        return e;
    };
    DevWork &w = ws.w;
    w = DevWork{};
    long long N = b->N;
    const long long no = nt * kOwnSub3;
    int nb = (int)((no + kScanBlock - 1) / kScanBlock);
    w.cand_cap = 8 * N;
    CK(alloc((void **)&ws.d_boxes, sizeof(BoxDev) * boxes.size()));
    CK(cudaMemcpy(ws.d_boxes, boxes.data(), sizeof(BoxDev) * boxes.size(), cudaMemcpyHostToDevice));
    CK(alloc((void **)&w.cand_count, sizeof(int) * (nt + 1)));
    CK(alloc((void **)&w.cand_off, sizeof(int) * (nt + 1)));
    CK(alloc((void **)&w.cand_cursor, sizeof(int) * (nt + 1)));
    CK(alloc((void **)&w.cand_nodes, sizeof(int) * (size_t)w.cand_cap));
    CK(alloc((void **)&w.own_count, sizeof(int) * (no + 1 + 4 * nt)));
    w.own_flag = w.own_count + no + 1;
    w.tile_fsum = reinterpret_cast<float *>(w.own_flag + nt);
    CK(alloc((void **)&w.own_off, sizeof(int) * (no + 1)));
    CK(alloc((void **)&w.own_cursor, sizeof(int) * (no + 1)));
    CK(alloc((void **)&w.own_nodes, sizeof(int) * (size_t)std::max<long long>(N, 1)));
    CK(alloc((void **)&w.own_rec, sizeof(float4) * (size_t)std::max<long long>(N, 1)));
    w.node_key = nullptr;
    w.node_rec = nullptr;
    if (use_halo(ctx)) {
        CK(alloc((void **)&w.node_key, sizeof(int2) * (size_t)std::max<long long>(N, 1)));
        CK(alloc((void **)&w.node_rec, sizeof(float4) * (size_t)std::max<long long>(N, 1)));
    }
    w.wtab = nullptr;
    if (ctx->cfg.precision == IFEM_FP64 && ctx->cfg.kernel == IFEM_KERNEL_PESKIN4)
        CK(alloc((void **)&w.wtab, sizeof(DetW) * (size_t)std::max<long long>(N, 1)));
    CK(alloc((void **)&w.active, sizeof(int) * (nt + 1)));
    CK(alloc((void **)&w.own_tiles, sizeof(int) * (nt + 1)));
    CK(alloc((void **)&w.counters, sizeof(int) * kCounters));
    CK(alloc((void **)&w.scan_blocks, sizeof(int) * 2 * (nb + 1)));
    CK(alloc((void **)&w.red_tile, sizeof(double) * 3 * (nt + 1)));
    CK(cudaMemset(w.red_tile, 0, sizeof(double) * 3 * (nt + 1)));
    w.elem_buf = b->d_elem_buf;
    w.bend_buf = b->d_bend_buf;
    w.status = ctx->d_status;
    ws.grid = g;
    ws.tile = tile;
    ws.n_tiles = nt;
    ws.max_edge = max_edge;
    return IFEM_OK;
}

static DevGrid dev_grid(ifem_batch b)
{
    DevGrid d{};
    d.n_boxes = b->ws.grid->n_boxes;
    d.n_tiles = b->ws.n_tiles;
    d.max_edge = b->ws.max_edge;
    d.boxes = b->ws.d_boxes;
    return d;
}

static int check_call(ifem_ctx ctx, ifem_batch b, ifem_grid g)
{
    if (!ctx || !b || b->ctx != ctx)
        return fail(ctx, IFEM_ERR_ARG, "null or foreign batch");
    if (g && (g->ctx != ctx || b->max_box >= g->n_boxes))
        return fail(ctx, IFEM_ERR_ARG, "grid does not match the batch");
    if (cudaSetDevice(ctx->cfg.device) != cudaSuccess)
        return fail(ctx, IFEM_ERR_CUDA, "cudaSetDevice failed");
    return IFEM_OK;
}

static int launch_rc(ifem_ctx ctx, cudaError_t e, const char *what)
{
    if (e != cudaSuccess)
        return fail(ctx, IFEM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return IFEM_OK;
}

// The FP32 Peskin spread of an IFEM_SCATTER_ATOMIC context uses the halo
// scatter (own nodes only, L2 reductions); every other configuration the
// owner-computes spread over candidate lists.
static int use_halo(ifem_ctx ctx)
{
    return ctx->cfg.precision == IFEM_FP32 && ctx->cfg.kernel == IFEM_KERNEL_PESKIN4 &&
           ctx->cfg.scatter == IFEM_SCATTER_ATOMIC;
}

static TransferArgs transfer_args(ifem_ctx ctx, ifem_batch b, const void *x, const void *F, const void *u,
                                  void *f, void *v, int flags, void *stream)
{
    TransferArgs a{};
    a.b = dev_batch(b);
    a.g = dev_grid(b);
    a.w = b->ws.w;
    a.x = x;
    a.F = F;
    a.u = u;
    a.f = f;
    a.v = v;
    a.kernel = ctx->cfg.kernel;
    a.density = (flags & IFEM_SPREAD_FORCE) ? 0 : 1;
    a.support = ctx->cfg.mls_support;
    a.n_sm = ctx->n_sm;
    a.acc64 = ctx->acc64;
    a.halo = use_halo(ctx) ? (ctx->staged ? 2 : 1) : 0;
    a.lattice = -1;
    a.stream = (cudaStream_t)stream;
    return a;
}

// Forces of particles [inst0, inst0 + inst_n) only (inst_n = 0: all), where
// forces_ranged_ok says the kernel takes a range.
static int do_forces(ifem_ctx ctx, ifem_batch b, const void *x, void *F, const void *wv, int hvp, void *stream,
                     int inst0 = 0, int inst_n = 0)
{
    ForcesArgs a{};
    a.inst0 = inst0;
    a.inst_n = inst_n;
    a.b = dev_batch(b);
    a.w.elem_buf = b->d_elem_buf;
    a.w.bend_buf = b->d_bend_buf;
    a.w.status = ctx->d_status;
    a.x = x;
    a.F = F;
    a.wv = wv;
    a.scatter = ctx->cfg.scatter;
    a.hvp = hvp;
    a.stream = (cudaStream_t)stream;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_forces_f64(a) : launch_forces_f32(a);
    return launch_rc(ctx, e, "forces");
}

// stages other than BIN_ALL: the FP32 halo path only. F (FP32 halo path):
// the placement also sums |F| per tile, which the fused transfer requires
// (every do_spread_interp follows a binning given the same forces).
static int do_bin(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, void *stream, int stages = BIN_ALL,
                  const void *F = nullptr)
{
    int rc = ws_ensure(ctx, b, g, ctx->tile);
    if (rc != IFEM_OK)
        return rc;
    TransferArgs a = transfer_args(ctx, b, x, F, nullptr, nullptr, nullptr, 0, stream);
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_bin_f64(a, 1, 1, stages)
                                                    : launch_bin_f32(a, 0, !use_halo(ctx), stages);
    return launch_rc(ctx, e, "binning");
}

static int do_spread(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *F, void *f, int flags,
                     void *stream)
{
    if (flags & IFEM_SPREAD_OVERWRITE) {
        cudaError_t e = cudaMemsetAsync(f, 0, (size_t)g->total * real_size(ctx), (cudaStream_t)stream);
        if (e != cudaSuccess)
            return launch_rc(ctx, e, "spread overwrite");
    }
    TransferArgs a = transfer_args(ctx, b, x, F, nullptr, f, nullptr, flags, stream);
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_spread_f64(a) : launch_spread_f32(a);
    return launch_rc(ctx, e, "spread");
}

// Spreading with the interpolation of the same step fused into it (the
// halo-scatter configuration only): one launch per step for both transfers.
// With xn given the launch also writes the position update from the
// velocities it gathers (xn = x + dt (3/2 v - 1/2 vp)).
static int do_spread_interp(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *F, const void *u,
                            void *f, void *v, int flags, void *stream, const void *vp = nullptr,
                            void *xn = nullptr, double dt = 0.0, int lattice = -1, int pdl = 0)
{
    if (flags & IFEM_SPREAD_OVERWRITE) {
        cudaError_t e = cudaMemsetAsync(f, 0, (size_t)g->total * real_size(ctx), (cudaStream_t)stream);
        if (e != cudaSuccess)
            return launch_rc(ctx, e, "spread overwrite");
    }
    TransferArgs a = transfer_args(ctx, b, x, F, u, f, v, flags, stream);
    a.vp = vp;
    a.xn = xn;
    a.dt = dt;
    a.binned = 1;   // every caller bins just before, on this stream or one joined to it
    a.lattice = lattice;
    a.pdl = pdl;
    return launch_rc(ctx, launch_spread_f32(a), "spread + interpolate");
}

// use_wtab: the binning of this same x ran earlier on the stream (FP64 Peskin
// stencils are read from its table instead of recomputed).
static int do_interp(ifem_ctx ctx, ifem_batch b, const void *u, const void *x, void *v, void *stream,
                     int use_wtab = 0)
{
    TransferArgs a = transfer_args(ctx, b, x, nullptr, u, nullptr, v, 0, stream);
    a.use_wtab = use_wtab;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_interp_f64(a) : launch_interp_f32(a);
    return launch_rc(ctx, e, "interpolate");
}

// Out-of-place position update xn = x + dt (3/2 v - 1/2 vp) (Eq. Bashforth_eqn).
static int do_ab2(ifem_ctx ctx, ifem_batch b, const void *x, const void *v, const void *vp, double dt, void *xn,
                  void *stream)
{
    LagrangeArgs a{};
    a.b = dev_batch(b);
    a.x = const_cast<void *>(x);
    a.x_out = xn;
    a.v = v;
    a.vp = vp;
    a.dt = dt;
    a.status = ctx->d_status;
    a.stream = (cudaStream_t)stream;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_ab2_f64(a) : launch_ab2_f32(a);
    return launch_rc(ctx, e, "position update");
}

static int do_reduce(ifem_ctx ctx, ifem_batch b, const void *x, const void *F, const void *v, double *red,
                     void *stream, int parts = 3)
{
    ReduceArgs a{};
    a.parts = parts;
    a.b = dev_batch(b);
    a.g = dev_grid(b);
    a.w = b->ws.w;
    a.x = x;
    a.F = F;
    a.v = v;
    a.red = red;
    a.stream = (cudaStream_t)stream;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_reduce_f64(a) : launch_reduce_f32(a);
    return launch_rc(ctx, e, "reduce");
}

// ------------------------------------------------------------ compute
extern "C" int ifem_compute_forces(ifem_ctx ctx, ifem_batch b, const void *x, void *F, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if ((!x || !F) && b->N > 0)
        return fail(ctx, IFEM_ERR_ARG, "compute_forces: null array");
    return do_forces(ctx, b, x, F, nullptr, 0, stream);
}

extern "C" int ifem_force_hvp(ifem_ctx ctx, ifem_batch b, const void *x, const void *w, void *Hw, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if ((!x || !w || !Hw) && b->N > 0)
        return fail(ctx, IFEM_ERR_ARG, "force_hvp: null array");
    return do_forces(ctx, b, x, Hw, w, 1, stream);
}

extern "C" int ifem_spread(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *F, void *f,
                           int flags, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, g);
    if (rc != IFEM_OK)
        return rc;
    if (!g || !f || ((!x || !F) && b->N > 0))
        return fail(ctx, IFEM_ERR_ARG, "spread: null array or grid");
    if (flags & ~(IFEM_SPREAD_FORCE | IFEM_SPREAD_OVERWRITE))
        return fail(ctx, IFEM_ERR_ARG, "spread: unknown flags");
    if ((rc = do_bin(ctx, b, g, x, stream)) != IFEM_OK)
        return rc;
    return do_spread(ctx, b, g, x, F, f, flags, stream);
}

static LagrangeArgs lagrange_args(ifem_ctx ctx, ifem_batch b, void *x, void *stream)
{
    LagrangeArgs a{};
    a.b = dev_batch(b);
    a.x = x;
    a.status = ctx->d_status;
    a.alpha = (double *)b->d_bend_buf;   // 6 reals per node: room for 3 doubles in either precision
    a.stream = (cudaStream_t)stream;
    return a;
}

extern "C" int ifem_ab2_update(ifem_ctx ctx, ifem_batch b, void *x, const void *v, const void *v_prev, double dt,
                               void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if ((!x || !v || !v_prev) && b->N > 0)
        return fail(ctx, IFEM_ERR_ARG, "ab2_update: null array");
    if (!std::isfinite(dt))
        return fail(ctx, IFEM_ERR_ARG, "ab2_update: dt must be finite");
    LagrangeArgs a = lagrange_args(ctx, b, x, stream);
    a.v = v;
    a.vp = v_prev;
    a.dt = dt;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_ab2_f64(a) : launch_ab2_f32(a);
    return launch_rc(ctx, e, "ab2_update");
}

extern "C" int ifem_volumes(ifem_ctx ctx, ifem_batch b, const void *x, double *vol, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if ((!x && b->N > 0) || (!vol && !b->inst.empty()))
        return fail(ctx, IFEM_ERR_ARG, "volumes: null array");
    LagrangeArgs a = lagrange_args(ctx, b, const_cast<void *>(x), stream);
    a.out = vol;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_volume_f64(a) : launch_volume_f32(a);
    return launch_rc(ctx, e, "volumes");
}

extern "C" int ifem_volume_correct(ifem_ctx ctx, ifem_batch b, void *x, const double *V0, double *lambda,
                                   void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if ((!x && b->N > 0) || (!V0 && !b->inst.empty()))
        return fail(ctx, IFEM_ERR_ARG, "volume_correct: null array");
    LagrangeArgs a = lagrange_args(ctx, b, x, stream);
    a.V0 = V0;
    a.out = lambda;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_vcorr_f64(a) : launch_vcorr_f32(a);
    return launch_rc(ctx, e, "volume_correct");
}

extern "C" int ifem_indicator_source(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, void *G, int flags,
                                     void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, g);
    if (rc != IFEM_OK)
        return rc;
    if (!g || !G || (!x && b->N > 0))
        return fail(ctx, IFEM_ERR_ARG, "indicator_source: null array or grid");
    if (flags & ~(IFEM_SPREAD_FORCE | IFEM_SPREAD_OVERWRITE))
        return fail(ctx, IFEM_ERR_ARG, "indicator_source: unknown flags");
    // n_k A_k into the batch scratch (a node array), then the spread of S*
    void *nA = b->d_bend_buf;
    DevBatch db = dev_batch(b);
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_area_normals_f64(db, x, nA, (cudaStream_t)stream)
                                                    : launch_area_normals_f32(db, x, nA, (cudaStream_t)stream);
    if ((rc = launch_rc(ctx, e, "indicator_source")) != IFEM_OK)
        return rc;
    if ((rc = do_bin(ctx, b, g, x, stream)) != IFEM_OK)
        return rc;
    return do_spread(ctx, b, g, x, nA, G, flags, stream);
}

extern "C" int ifem_interpolate_cc(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *field, int ncomp,
                                   const void *x, void *out, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, g);
    if (rc != IFEM_OK)
        return rc;
    if (!g || !field || ((!x || !out) && b->N > 0))
        return fail(ctx, IFEM_ERR_ARG, "interpolate_cc: null array or grid");
    if (ncomp < 1 || ncomp > 64)
        return fail(ctx, IFEM_ERR_ARG, "interpolate_cc: ncomp must be 1..64");
    if ((rc = ws_ensure(ctx, b, g, ctx->tile)) != IFEM_OK)
        return rc;
    TransferArgs a = transfer_args(ctx, b, x, nullptr, field, nullptr, out, 0, stream);
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_interp_cc_f64(a, ncomp) : launch_interp_cc_f32(a, ncomp);
    return launch_rc(ctx, e, "interpolate_cc");
}

extern "C" int ifem_fluid_stress_forces(ifem_ctx ctx, ifem_batch b, const void *x, const void *u, const void *C,
                                        const ifem_fluid_params *p, void *F, int flags, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if (!p || ((!x || !u || !F) && b->N > 0))
        return fail(ctx, IFEM_ERR_ARG, "fluid_stress_forces: null array or parameters");
    if (flags & ~IFEM_FORCES_ACCUMULATE)
        return fail(ctx, IFEM_ERR_ARG, "fluid_stress_forces: unknown flags");
    if (!(p->eta >= 0.0) || (C && !(p->lambda > 0.0)))
        return fail(ctx, IFEM_ERR_ARG, "fluid_stress_forces: need eta >= 0 and, with C, lambda > 0");
    FluidArgs a{};
    a.b = dev_batch(b);
    a.w.elem_buf = b->d_elem_buf;
    a.w.status = ctx->d_status;
    a.x = x;
    a.u = u;
    a.C = C;
    a.eta = p->eta;
    a.cp = C ? (p->eta * (1.0 - p->beta)) / p->lambda : 0.0;
    a.add = (flags & IFEM_FORCES_ACCUMULATE) ? 1 : 0;
    a.F = F;
    a.stream = (cudaStream_t)stream;
    cudaError_t e = ctx->cfg.precision == IFEM_FP64 ? launch_fluid_f64(a) : launch_fluid_f32(a);
    return launch_rc(ctx, e, "fluid_stress_forces");
}

extern "C" int ifem_interpolate(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *u, const void *x, void *v,
                                void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, g);
    if (rc != IFEM_OK)
        return rc;
    if (!g || !u || ((!x || !v) && b->N > 0))
        return fail(ctx, IFEM_ERR_ARG, "interpolate: null array or grid");
    if (ctx->cfg.precision == IFEM_FP32) {
        // the FP32 kernel walks the nodes in tile order (locality)
        if ((rc = do_bin(ctx, b, g, x, stream)) != IFEM_OK)
            return rc;
    } else if ((rc = ws_ensure(ctx, b, g, ctx->tile)) != IFEM_OK) {
        return rc;
    }
    return do_interp(ctx, b, u, x, v, stream);
}

extern "C" int ifem_reduce(ifem_ctx ctx, ifem_batch b, const void *x, const void *F, const void *v, double *red,
                           void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if (!red || (!x && b->N > 0))
        return fail(ctx, IFEM_ERR_ARG, "reduce: null array");
    if ((rc = ws_ensure(ctx, b, b->grid0, ctx->tile)) != IFEM_OK)
        return rc;
    return do_reduce(ctx, b, x, F, v, red, stream);
}

// Host-resident node arrays of ifem_step_coupling_host: positions copied in
// before the step, velocities and sums copied out after it.
struct HostIO {
    const void *x_host;
    void *v_host;
    double *red_host;
    size_t red_n;   // doubles of red
};

// The FP32 one-CTA-per-particle force kernel takes a particle range, so the
// forces of the particles whose positions have arrived can start while the
// rest are still being copied in.
static bool forces_ranged_ok(ifem_ctx ctx, ifem_batch b)
{
    return ctx->cfg.precision == IFEM_FP32 && ctx->cfg.scatter == IFEM_SCATTER_ATOMIC && b->fused_ok &&
           b->inst.size() >= 2;
}

// Copy node rows [n0, n1) of the 3 x N host array into the device array.
static cudaError_t copy_nodes_in(ifem_ctx ctx, ifem_batch b, const void *xh, void *x, long long n0, long long n1,
                                 cudaStream_t s)
{
    const size_t rs = real_size(ctx), pitch = (size_t)b->N * rs;
    if (n1 <= n0)
        return cudaSuccess;
    return cudaMemcpy2DAsync((char *)x + n0 * rs, pitch, (const char *)xh + n0 * rs, pitch, (size_t)(n1 - n0) * rs,
                             3, cudaMemcpyHostToDevice, s);
}

// One coupling step; with xn given (the caller checked vp, dt and aliasing)
// also the position update from the interpolated velocities; with io given
// the host copies in and out around it.
static int step_impl(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *u, void *F, void *f,
                     void *v, double *red, int flags, const void *vp, double dt, void *xn, void *stream,
                     const HostIO *io = nullptr)
{
    int rc;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    const size_t node_bytes = 3 * (size_t)b->N * real_size(ctx);
    if (ctx->ev_ok) {
        // profiling: stages one after the other on the caller's stream, each
        // bracketed by an event (the position update counts with the
        // interpolation; host copies lie outside the stages)
        if (io && (e = copy_nodes_in(ctx, b, io->x_host, const_cast<void *>(x), 0, b->N, s)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy in");
        // forces (ev1 -> ev0), then the binning (ev0 -> ev2): the fused
        // transfer's placement sums the forces per tile
        mark(ctx, 1, stream);
        if ((rc = do_forces(ctx, b, x, F, nullptr, 0, stream)) != IFEM_OK)
            return rc;
        mark(ctx, 0, stream);
        if ((rc = do_bin(ctx, b, g, x, stream, BIN_ALL, F)) != IFEM_OK)
            return rc;
        mark(ctx, 2, stream);
        ctx->ev_fused = use_halo(ctx);
        if (ctx->ev_fused) {
            if ((rc = do_spread_interp(ctx, b, g, x, F, u, f, v, flags, stream, vp, xn, dt)) != IFEM_OK)
                return rc;
            mark(ctx, 3, stream);
        } else {
            if ((rc = do_spread(ctx, b, g, x, F, f, flags, stream)) != IFEM_OK)
                return rc;
            mark(ctx, 3, stream);
            if ((rc = do_interp(ctx, b, u, x, v, stream, 1)) != IFEM_OK)
                return rc;
            if (xn && (rc = do_ab2(ctx, b, x, v, vp, dt, xn, stream)) != IFEM_OK)
                return rc;
        }
        mark(ctx, 4, stream);
        if (red && (rc = do_reduce(ctx, b, x, F, v, red, stream)) != IFEM_OK)
            return rc;
        mark(ctx, 5, stream);
        ctx->ev_recorded = 1;
        if (io && node_bytes > 0 &&
            (e = cudaMemcpyAsync(io->v_host, v, node_bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy out");
        if (io && io->red_host &&
            (e = cudaMemcpyAsync(io->red_host, red, io->red_n * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy out");
        return IFEM_OK;
    }
    // fork-join over the context's two auxiliary streams (also inside stream
    // capture): forces run beside binning, interpolation (and the position
    // update) beside spreading, and the x/F sums (which need only the forces)
    // beside the transfers. The sums wait for the binning too: started with
    // the forces' last blocks they slowed the binning's scan, which the
    // transfer waits for, while the transfer's CTAs take their work from a
    // counter and absorb them
    //   s:    bin ----------------------- wait(forces) spread  wait(interp) sums of v, boxes  wait(sums)
    //   aux0: forces --/ wait(bin) sums of x, F ---------------------------------------------/
    //   aux1:       wait(bin) interp [ab2] -------/
    // With the fused spread + interpolation [+ ab2] the aux1 branch is absent,
    // and the binning's placement, which sums |F| per tile for the transfer's
    // fixed-point scales, waits for the forces:
    //   s:    count, scan -- wait(forces) placement  spread+interp  sums of v, boxes  wait(sums)
    //   aux0: forces ------/ wait(placement) sums of x, F ------------------------------/
    // With host arrays the positions arrive on s in two halves (by particle)
    // when the force kernel takes particle ranges, each half's forces starting
    // on aux0 once it has landed; v goes back to the host on aux1 beside the
    // sums of v and the boxes:
    //   s:    copy x[0:h] copy x[h:N] count, scan, wait(forces) placement ... spread+interp  sums of v, boxes  copy red  wait(copy v)
    //   aux0:   wait(x[0:h]) forces[0:h] wait(x[h:N]) forces[h:N] wait(placement) sums of x, F
    //   aux1:                                           wait(v) copy v ------------------/
    const bool fused = use_halo(ctx) != 0;
    if ((rc = ws_ensure(ctx, b, g, ctx->tile)) != IFEM_OK)
        return rc;
    const bool split = io && forces_ranged_ok(ctx, b);
    if (split) {
        // halves by node count, cut at a particle boundary
        const int ni = (int)b->inst.size();
        int h = 1;
        while (h < ni - 1 && b->h_inst[h].node_off < b->N / 2)
            ++h;
        const long long nh = b->h_inst[h].node_off;
        if ((e = copy_nodes_in(ctx, b, io->x_host, const_cast<void *>(x), 0, nh, s)) == cudaSuccess &&
            (e = cudaEventRecord(ctx->fork[5], s)) == cudaSuccess &&
            (e = copy_nodes_in(ctx, b, io->x_host, const_cast<void *>(x), nh, b->N, s)) == cudaSuccess &&
            (e = cudaEventRecord(ctx->fork[6], s)) == cudaSuccess)
            e = cudaStreamWaitEvent(ctx->aux[0], ctx->fork[5], 0);
        if (e != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy in");
        if ((rc = do_forces(ctx, b, x, F, nullptr, 0, ctx->aux[0], 0, h)) != IFEM_OK)
            return rc;
        if ((e = cudaStreamWaitEvent(ctx->aux[0], ctx->fork[6], 0)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy in");
        if ((rc = do_forces(ctx, b, x, F, nullptr, 0, ctx->aux[0], h, ni - h)) != IFEM_OK)
            return rc;
    } else {
        if (io && (e = copy_nodes_in(ctx, b, io->x_host, const_cast<void *>(x), 0, b->N, s)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy in");
        e = cudaEventRecord(ctx->fork[0], s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(ctx->aux[0], ctx->fork[0], 0);
        if (e != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling fork");
        if ((rc = do_forces(ctx, b, x, F, nullptr, 0, ctx->aux[0])) != IFEM_OK)
            return rc;
    }
    if ((e = cudaEventRecord(ctx->fork[1], ctx->aux[0])) != cudaSuccess)
        return launch_rc(ctx, e, "step_coupling fork");
    // with the fused transfer the binning's count and scan run beside the
    // forces and its placement (which sums the forces per tile) after them
    if ((rc = do_bin(ctx, b, g, x, stream, fused ? BIN_COUNT : BIN_ALL)) != IFEM_OK)
        return rc;
    if (fused) {
        if ((e = cudaStreamWaitEvent(s, ctx->fork[1], 0)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling join");
        if ((rc = do_bin(ctx, b, g, x, stream, BIN_PLACE, F)) != IFEM_OK)
            return rc;
    }
    // the x/F sums, after the forces and the binning, on aux0 beside the transfers
    if (red) {
        if ((e = cudaEventRecord(ctx->fork[9], s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->aux[0], ctx->fork[9], 0)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling fork");
        if ((rc = do_reduce(ctx, b, x, F, v, red, ctx->aux[0], 1)) != IFEM_OK)
            return rc;
        if ((e = cudaEventRecord(ctx->fork[4], ctx->aux[0])) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling fork");
    }
    if (!fused) {
        if ((e = cudaEventRecord(ctx->fork[2], s)) == cudaSuccess)
            e = cudaStreamWaitEvent(ctx->aux[1], ctx->fork[2], 0);
        if (e != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling fork");
        if ((rc = do_interp(ctx, b, u, x, v, ctx->aux[1], 1)) != IFEM_OK)
            return rc;
        if (xn && (rc = do_ab2(ctx, b, x, v, vp, dt, xn, ctx->aux[1])) != IFEM_OK)
            return rc;
        if ((e = cudaEventRecord(ctx->fork[3], ctx->aux[1])) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling fork");
    }
    if ((e = cudaStreamWaitEvent(s, ctx->fork[1], 0)) != cudaSuccess)
        return launch_rc(ctx, e, "step_coupling join");
    // with host arrays and the staged transfer, one launch per lattice: row d
    // of v goes back to the host on aux1 as soon as lattice d's launch ends,
    // beside the later lattices. Lattices 1 and 2 are launched with
    // programmatic serialization: their CTAs start on the SMs that the
    // previous lattice's CTAs leave when its items run out (they read nothing
    // it writes), so the three launches share one tail instead of one each
    const bool v_rows = fused && io && ctx->staged && node_bytes > 0 && !(flags & IFEM_SPREAD_OVERWRITE);
    if (v_rows) {
        const size_t row = node_bytes / 3;
        for (int d = 0; d < 3; ++d) {
            if ((rc = do_spread_interp(ctx, b, g, x, F, u, f, v, flags, stream, vp, xn, dt, d, d > 0)) != IFEM_OK)
                return rc;
            if ((e = cudaEventRecord(ctx->fork[d == 2 ? 7 : 2 + d], s)) == cudaSuccess &&
                (e = cudaStreamWaitEvent(ctx->aux[1], ctx->fork[d == 2 ? 7 : 2 + d], 0)) == cudaSuccess)
                e = cudaMemcpyAsync((char *)io->v_host + d * row, (const char *)v + d * row, row,
                                    cudaMemcpyDeviceToHost, ctx->aux[1]);
            if (e != cudaSuccess)
                return launch_rc(ctx, e, "step_coupling_host: copy out");
        }
        // what follows on s waits for every lattice, not only the last one
        if ((e = cudaStreamWaitEvent(s, ctx->fork[2], 0)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, ctx->fork[3], 0)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling join");
        if ((e = cudaEventRecord(ctx->fork[8], ctx->aux[1])) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy out");
    } else if (fused) {
        if ((rc = do_spread_interp(ctx, b, g, x, F, u, f, v, flags, stream, vp, xn, dt)) != IFEM_OK)
            return rc;
    } else {
        if ((rc = do_spread(ctx, b, g, x, F, f, flags, stream)) != IFEM_OK)
            return rc;
        if ((e = cudaStreamWaitEvent(s, ctx->fork[3], 0)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling join");
    }
    const bool v_out = io && node_bytes > 0 && !v_rows;
    if (v_out) {
        // v is complete here: copy it back beside the remaining sums
        if ((e = cudaEventRecord(ctx->fork[7], s)) == cudaSuccess &&
            (e = cudaStreamWaitEvent(ctx->aux[1], ctx->fork[7], 0)) == cudaSuccess &&
            (e = cudaMemcpyAsync(io->v_host, v, node_bytes, cudaMemcpyDeviceToHost, ctx->aux[1])) == cudaSuccess)
            e = cudaEventRecord(ctx->fork[8], ctx->aux[1]);
        if (e != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling_host: copy out");
    }
    if (red) {
        // the sums of v and the boxes write other entries than the x/F sums,
        // which may still be running in the transfer's tail: join them after
        if ((rc = do_reduce(ctx, b, x, F, v, red, stream, 2)) != IFEM_OK)
            return rc;
        if ((e = cudaStreamWaitEvent(s, ctx->fork[4], 0)) != cudaSuccess)
            return launch_rc(ctx, e, "step_coupling join");
    }
    if (io && io->red_host &&
        (e = cudaMemcpyAsync(io->red_host, red, io->red_n * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
        return launch_rc(ctx, e, "step_coupling_host: copy out");
    if ((v_out || v_rows) && (e = cudaStreamWaitEvent(s, ctx->fork[8], 0)) != cudaSuccess)
        return launch_rc(ctx, e, "step_coupling_host: join");
    return IFEM_OK;
}

static int check_step(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *u, const void *F,
                      const void *f, const void *v, int flags, const char *who)
{
    int rc = check_call(ctx, b, g);
    if (rc != IFEM_OK)
        return rc;
    if (!g || !u || !f || ((!x || !F || !v) && b->N > 0))
        return fail(ctx, IFEM_ERR_ARG, std::string(who) + ": null array or grid");
    if (flags & ~(IFEM_SPREAD_FORCE | IFEM_SPREAD_OVERWRITE))
        return fail(ctx, IFEM_ERR_ARG, std::string(who) + ": unknown flags");
    return IFEM_OK;
}

extern "C" int ifem_step_coupling(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *u, void *F,
                                  void *f, void *v, double *red, int flags, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_step(ctx, b, g, x, u, F, f, v, flags, "step_coupling");
    if (rc != IFEM_OK)
        return rc;
    return step_impl(ctx, b, g, x, u, F, f, v, red, flags, nullptr, 0.0, nullptr, stream);
}

extern "C" int ifem_step_coupling_ab2(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *u,
                                      void *F, void *f, void *v, double *red, int flags, const void *v_prev,
                                      double dt, void *x_new, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_step(ctx, b, g, x, u, F, f, v, flags, "step_coupling_ab2");
    if (rc != IFEM_OK)
        return rc;
    if ((!v_prev || !x_new) && b->N > 0)
        return fail(ctx, IFEM_ERR_ARG, "step_coupling_ab2: null array");
    if (!std::isfinite(dt))
        return fail(ctx, IFEM_ERR_ARG, "step_coupling_ab2: dt must be finite");
    if (b->N > 0) {
        // x_new is written while x, v_prev and F are still read, and v_prev
        // is read after v is written: none of them may overlap
        const size_t nb = 3 * (size_t)b->N * real_size(ctx);
        auto overlap = [nb](const void *p, const void *q) {
            const char *a = (const char *)p, *c = (const char *)q;
            return a < c + nb && c < a + nb;
        };
        if (overlap(x_new, x) || overlap(x_new, v) || overlap(x_new, v_prev) || overlap(x_new, F) ||
            overlap(v_prev, v))
            return fail(ctx, IFEM_ERR_ARG, "step_coupling_ab2: x_new, x, v, v_prev and F must not overlap");
    }
    return step_impl(ctx, b, g, x, u, F, f, v, red, flags, v_prev, dt, x_new, stream);
}

extern "C" int ifem_step_coupling_host(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x_host, void *x,
                                       const void *u, void *F, void *f, void *v, void *v_host, double *red,
                                       double *red_host, int flags, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_step(ctx, b, g, x, u, F, f, v, flags, "step_coupling_host");
    if (rc != IFEM_OK)
        return rc;
    if ((!x_host || !v_host) && b->N > 0)
        return fail(ctx, IFEM_ERR_ARG, "step_coupling_host: null host array");
    if (red_host && !red)
        return fail(ctx, IFEM_ERR_ARG, "step_coupling_host: red_host needs the device array red");
    HostIO io{x_host, v_host, red_host, 12 * b->inst.size() + 6 * (size_t)g->n_boxes};
    return step_impl(ctx, b, g, x, u, F, f, v, red, flags, nullptr, 0.0, nullptr, stream, &io);
}

// Tile autotuner: time binning + spreading + interpolation of the batch at
// its current positions x for each candidate tile edge, with the transfer
// launches the step uses (the fused one where it fuses) (CUDA events on
// `stream`, best of two after one warm-up run) and keep the fastest. Forces
// for the spread are the batch's own (computed once); the velocity field is
// zero (the gathers cost the same for any values). Temporary buffers are
// allocated and freed here, so this must run outside stream capture.
static int autotune(ifem_ctx ctx, ifem_batch b, const void *x, void *stream)
{
    ifem_grid g = b->grid0;
    const size_t rs = real_size(ctx);
    const std::vector<int> cand = ctx->cfg.precision == IFEM_FP64 ? std::vector<int>{6, 8, 10, 12}
                                                                   : std::vector<int>{8, 12, 16};
    void *F = nullptr, *v = nullptr, *u = nullptr, *f = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = IFEM_OK;
    float best_ms = 1e30f;
    int best = ctx->tile;
    auto cleanup = [&]() {
        cudaFree(F);
        cudaFree(v);
        cudaFree(u);
        cudaFree(f);
        if (e0)
            cudaEventDestroy(e0);
        if (e1)
            cudaEventDestroy(e1);
    };
    if (cudaMalloc(&F, std::max<size_t>(16, 3 * b->N * rs)) != cudaSuccess ||
        cudaMalloc(&v, std::max<size_t>(16, 3 * b->N * rs)) != cudaSuccess ||
        cudaMalloc(&u, g->total * rs) != cudaSuccess || cudaMalloc(&f, g->total * rs) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return fail(ctx, IFEM_ERR_OOM, "autotune: temporary allocation failed");
    }
    cudaMemsetAsync(u, 0, g->total * rs, s);
    cudaMemsetAsync(f, 0, g->total * rs, s);
    if ((rc = do_forces(ctx, b, x, F, nullptr, 0, stream)) != IFEM_OK) {
        cleanup();
        return rc;
    }
    for (int t : cand) {
        if ((rc = ws_ensure(ctx, b, g, t)) != IFEM_OK)
            break;
        const int saved = ctx->tile;
        ctx->tile = t;
        float tmin = 1e30f;
        for (int rep = 0; rep < 3 && rc == IFEM_OK; ++rep) {
            cudaEventRecord(e0, s);
            if ((rc = do_bin(ctx, b, g, x, stream, BIN_ALL, F)) == IFEM_OK) {
                // the transfer launches the step will use (fused where it fuses)
                if (use_halo(ctx))
                    rc = do_spread_interp(ctx, b, g, x, F, u, f, v, 0, stream);
                else if ((rc = do_spread(ctx, b, g, x, F, f, 0, stream)) == IFEM_OK)
                    rc = do_interp(ctx, b, u, x, v, stream);
            }
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = fail(ctx, IFEM_ERR_CUDA, "autotune: event timing failed");
            if (rep > 0)
                tmin = std::min(tmin, ms);
        }
        ctx->tile = saved;
        if (rc != IFEM_OK)
            break;
        if (tmin < best_ms) {
            best_ms = tmin;
            best = t;
        }
    }
    cleanup();
    // the timing runs added to the status block; clear it
    cudaMemset(ctx->d_status, 0, sizeof(unsigned long long) * kStatusWords);
    if (rc != IFEM_OK)
        return rc;
    ctx->tile = best;
    ctx->tuned = 1;
    return ws_ensure(ctx, b, g, best);
}

extern "C" int ifem_prepare(ifem_ctx ctx, ifem_batch b, const void *x, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    int rc = check_call(ctx, b, nullptr);
    if (rc != IFEM_OK)
        return rc;
    if (ctx->cfg.tile == 0 && !ctx->tuned && b->N > 0) {
        if (!x)
            return fail(ctx, IFEM_ERR_ARG, "prepare: autotuning needs positions x");
        return autotune(ctx, b, x, stream);
    }
    return ws_ensure(ctx, b, b->grid0, ctx->tile);
}
