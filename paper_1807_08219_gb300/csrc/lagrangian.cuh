// lagrangian.cuh -- the Lagrangian update after a coupling step: the
// Adams-Bashforth position update (Eq. Bashforth_eqn), per-particle volumes
// and the membrane volume correction of Sec. "Conservation of Volume for
// Membranes" (after Mendez et al. 2014). Positions are the particles' local
// offsets; volumes and the correction's sums are FP64 in both precisions.
#pragma once
#include "forces.cuh"
#include "transfer.cuh"

namespace ifem {

// xo = x + dt*(1.5*v - 0.5*vp), componentwise over the 3N node values (in
// place when xo == x).
template <typename real>
__global__ void ab2_kernel(long long n3, const real *x, real *xo, const real *__restrict__ v,
                           const real *__restrict__ vp, real dt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3)
        xo[i] = ab2_value(x[i], v[i], vp[i], dt);
}

__device__ __forceinline__ void cross3d(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3d(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <typename real>
__device__ __forceinline__ void load_node_d(const real *x, long long N, long long node, double p[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
        p[a] = (double)x[a * N + node];
}

constexpr int kVolThreads = 256;

// Block per instance: membranes V = (1/18) sum_faces [a.(b x c) + b.(c x a)
// + c.(a x b)] (the polyhedron formula; the three terms are equal, so
// V = 1/6 sum a.(b x c)), solids V = sum_tets det(Ds)/6.
template <typename real>
__global__ void __launch_bounds__(kVolThreads) volume_kernel(DevBatch b, const real *__restrict__ x,
                                                             double *__restrict__ vol)
{
    __shared__ double sh[kVolThreads];
    const InstDev I = b.inst[blockIdx.x];
    const TmplDev T = b.tmpl[I.tmpl];
    const long long N = b.N;
    double s = 0.0;
    for (int e = threadIdx.x; e < T.n_elems; e += blockDim.x) {
        if (T.kind == 0) {
            // the three cyclic triple products of the formula are equal: one
            // per face, V = 1/6 sum a.(b x c)
            double p[3][3], t[3];
            for (int c = 0; c < 3; ++c)
                load_node_d(x, N, I.node_off + T.elems[3 * e + c], p[c]);
            cross3d(p[1], p[2], t);
            s += dot3d(p[0], t);
        } else {
            double p[4][3], Ds[3][3];
            for (int c = 0; c < 4; ++c)
                load_node_d(x, N, I.node_off + T.elems[4 * e + c], p[c]);
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < 3; ++a)
                    Ds[a][c] = p[1 + c][a] - p[0][a];
            s += det3(Ds) / 6.0;
        }
    }
    const double r = block_sum<kVolThreads>(s, sh);
    if (threadIdx.x == 0)
        vol[blockIdx.x] = T.kind == 0 ? r / 6.0 : r;
}

// Thread per (instance, node) of a membrane: alpha_I = -(1/12) sum over the
// incident faces, ascending, of x_{I2} x x_{I3} (the face's other two nodes
// in cyclic order); FP64 for FP64 positions, FP32 edge vectors for FP32
// positions (below). alpha: 3 doubles per node (batch node order).
template <typename real>
__global__ void vc_alpha_kernel(DevBatch b, const real *__restrict__ x, double *__restrict__ alpha)
{
    const InstDev I = b.inst[blockIdx.y];
    const TmplDev T = b.tmpl[I.tmpl];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (T.kind != 0 || k >= T.n_nodes)
        return;
    const long long N = b.N;
    double *o = alpha + 3 * (I.node_off + k);
    if constexpr (std::is_same<real, float>::value) {
        // FP32: over the closed ring sum x_I2 x x_I3 = sum (x_I2 - x_I) x (x_I3 - x_I)
        // (the ring's edges x_I3 - x_I2 sum to zero), so the cross products
        // take edge vectors about one cell long, exact enough in FP32; the
        // correction's sums use this same alpha in FP64, so the corrected
        // volume still meets V0
        float pk[3], acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            pk[a] = x[a * N + I.node_off + k];
        for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
            const int code = T.inc_idx[q], e = code >> 2, v = code & 3;
            const long long n1 = I.node_off + T.elems[3 * e + (v + 1) % 3];
            const long long n2 = I.node_off + T.elems[3 * e + (v + 2) % 3];
            float e1[3], e2[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                e1[a] = x[a * N + n1] - pk[a];
                e2[a] = x[a * N + n2] - pk[a];
            }
            acc[0] += e1[1] * e2[2] - e1[2] * e2[1];
            acc[1] += e1[2] * e2[0] - e1[0] * e2[2];
            acc[2] += e1[0] * e2[1] - e1[1] * e2[0];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            o[a] = (double)acc[a] * (-1.0 / 12.0);
    } else {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
            const int code = T.inc_idx[q], e = code >> 2, v = code & 3;
            const int n1 = T.elems[3 * e + (v + 1) % 3], n2 = T.elems[3 * e + (v + 2) % 3];
            double p1[3], p2[3], t[3];
            load_node_d(x, N, I.node_off + n1, p1);
            load_node_d(x, N, I.node_off + n2, p2);
            cross3d(p1, p2, t);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                acc[a] = acc[a] + t[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            o[a] = acc[a] * (-1.0 / 12.0);
    }
}

// Block per instance of a membrane: the cubic A L^3 + B L^2 + C L + D = 0 of
// the volume correction with the paper's cyclic sums (A = (1/18) sum
// alpha.(alpha x alpha), B = (1/6) sum x.(alpha x alpha), C = (1/6) sum
// alpha.(x x x), D = V(x) - V0, FP64 block trees; for A and V the three
// cyclic terms are equal and one is taken, times 3, and C is evaluated as
// -2 sum |alpha_I|^2, equal to it since alpha_I = -(1/2) grad_I V), Lambda by Newton from 0
// (|step| <= 1e-15 max(1, |L|), at most 100 steps; the root the oracle
// takes), then x_I = x_I + Lambda alpha_I. Solids: lambda = 0, x unchanged.
// status ST_DOMAIN counts instances whose Newton failed (x left unchanged).
template <typename real>
__global__ void __launch_bounds__(kVolThreads) vc_correct_kernel(DevBatch b, real *__restrict__ x,
                                                                 const double *__restrict__ alpha,
                                                                 const double *__restrict__ V0,
                                                                 double *__restrict__ lambda,
                                                                 unsigned long long *status)
{
    __shared__ double sh[kVolThreads];
    __shared__ double sL;
    const InstDev I = b.inst[blockIdx.x];
    const TmplDev T = b.tmpl[I.tmpl];
    const long long N = b.N;
    if (T.kind != 0) {
        if (threadIdx.x == 0 && lambda)
            lambda[blockIdx.x] = 0.0;
        return;
    }
    double sA = 0.0, sB = 0.0, sC = 0.0, sV = 0.0;
    for (int e = threadIdx.x; e < T.n_elems; e += blockDim.x) {
        int nd[3];
        double p[3][3], q[3][3];
        for (int c = 0; c < 3; ++c) {
            nd[c] = T.elems[3 * e + c];
            load_node_d(x, N, I.node_off + nd[c], p[c]);
            const double *al = alpha + 3 * (I.node_off + nd[c]);
            q[c][0] = al[0];
            q[c][1] = al[1];
            q[c][2] = al[2];
        }
        // cyclic (a, b, c), (b, c, a), (c, a, b): B takes all three terms;
        // the three terms of A and of V are equal, so those take one (1/6)
        double xx[3], qq[3];
        cross3d(p[1], p[2], xx);
        sV += dot3d(p[0], xx);
        for (int c = 0; c < 3; ++c) {
            const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
            cross3d(q[c1], q[c2], qq);
            sB += dot3d(p[c], qq);
            if (c == 0)
                sA += dot3d(q[0], qq);
        }
    }
    // C = 1/6 sum alpha.(x x x) (cyclic) = sum_I alpha_I . grad_I V = -2 sum_I |alpha_I|^2,
    // since alpha_I = -(1/2) grad_I V exactly
    for (int k = threadIdx.x; k < T.n_nodes; k += blockDim.x) {
        const double *al = alpha + 3 * (I.node_off + k);
        sC += al[0] * al[0] + al[1] * al[1] + al[2] * al[2];
    }
    const double A = block_sum<kVolThreads>(sA, sh) / 6.0;
    const double B = block_sum<kVolThreads>(sB, sh) / 6.0;
    const double C = -2.0 * block_sum<kVolThreads>(sC, sh);
    const double D = block_sum<kVolThreads>(sV, sh) / 6.0 - V0[blockIdx.x];
    if (threadIdx.x == 0) {
        double L = 0.0;
        bool ok = false;
        for (int it = 0; it < 100; ++it) {
            const double f = ((A * L + B) * L + C) * L + D;
            const double fp = (3.0 * A * L + 2.0 * B) * L + C;
            if (fp == 0.0)
                break;
            const double step = f / fp;
            L = L - step;
            if (fabs(step) <= 1e-15 * fmax(1.0, fabs(L))) {
                ok = true;
                break;
            }
        }
        if (!ok) {
            status_add(status, ST_DOMAIN, 1);
            L = 0.0;
        }
        sL = L;
        if (lambda)
            lambda[blockIdx.x] = L;
    }
    __syncthreads();
    const double L = sL;
    for (int k = threadIdx.x; k < T.n_nodes; k += blockDim.x) {
        const double *al = alpha + 3 * (I.node_off + k);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            real *p = x + a * N + I.node_off + k;
            *p = (real)((double)*p + L * al[a]);
        }
    }
}

}  // namespace ifem
