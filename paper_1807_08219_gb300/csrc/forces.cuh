// forces.cuh -- Lagrangian internal-force kernels (Algorithm step 1).
//
//   membranes  Eq. FEM_Membrane: F_k = -A0 P^ grad N^_k with the tangent-plane
//              deformation gradient F^ = Ds Dm^-1 and S^ = 2 dW/dC^ for the
//              neo-Hookean (Eq. neo-Hookena) and Skalak (Eq. Skalak) laws;
//   solids     Eq. FEM: F_k = -V0 P grad N_k, F = sum_k x_k (x) grad N_k,
//              P = F S, S = lambda/2 (J^2 - 1) C^-1 + mu (I - C^-1);
//   bending    F_k = 2 kb [Lap(kH - kH0) + 2 (kH - kH0)(kH^2 - kG + kH0 kH)] n_k A_k
//              (force of the Canham-Helfrich energy, Eq. Bending_Energy) with
//              the discrete operators of Meyer, Desbrun, Schroeder & Barr.
//
// Every expression follows one fixed evaluation order (written out in the
// comments of the oracle-independent specification in each function), so
// that the FP64 build, compiled without FMA contraction, is bit-reproducible.
#pragma once
#include "common.cuh"

namespace ifem {

// ------------------------------------------------------------ membranes
// Per triangle (a, b, c) with m = Dm^-1 = [m00 m01; m10 m11] and area A0:
//   d1 = xb - xa, d2 = xc - xa
//   Fh[i][0] = d1[i]*m00 + d2[i]*m10,  Fh[i][1] = d1[i]*m01 + d2[i]*m11
//   C00 = (Fh00^2 + Fh10^2) + Fh20^2, C01 = (Fh00 Fh01 + Fh10 Fh11) + Fh20 Fh21, C11 likewise
//   I1 = C00 + C11, I2 = C00*C11 - C01*C01
//   NH:     q = mu/(I2*I2); S00 = mu - q*C11; S01 = q*C01; S11 = mu - q*C00
//   Skalak: a = mu*((I1-2)+1); b = (0.5*(C*mu))*(I2-1) - mu;
//           S00 = a + b*C11; S01 = -(b*C01); S11 = a + b*C00
//   P0 = Fh[i][0]*S00 + Fh[i][1]*S01, P1 = Fh[i][0]*S01 + Fh[i][1]*S11
//   fb[i] = -(A0*(P0*m00 + P1*m01)); fc[i] = -(A0*(P0*m10 + P1*m11)); fa[i] = -(fb[i] + fc[i])
template <typename real>
__device__ __forceinline__ void membrane_kin(const real xa[3], const real xb[3], const real xc[3],
                                             const real m[4], real Fh[3][2], real &C00, real &C01,
                                             real &C11)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        real d1 = xb[i] - xa[i];
        real d2 = xc[i] - xa[i];
        Fh[i][0] = d1 * m[0] + d2 * m[2];
        Fh[i][1] = d1 * m[1] + d2 * m[3];
    }
    C00 = (Fh[0][0] * Fh[0][0] + Fh[1][0] * Fh[1][0]) + Fh[2][0] * Fh[2][0];
    C01 = (Fh[0][0] * Fh[0][1] + Fh[1][0] * Fh[1][1]) + Fh[2][0] * Fh[2][1];
    C11 = (Fh[0][1] * Fh[0][1] + Fh[1][1] * Fh[1][1]) + Fh[2][1] * Fh[2][1];
}

template <typename real>
__device__ __forceinline__ void membrane_S(int law, real mu, real C, real C00, real C01, real C11,
                                           real &S00, real &S01, real &S11)
{
    real I1 = C00 + C11;
    real I2 = C00 * C11 - C01 * C01;
    if (law == 0) {
        real q = mu / (I2 * I2);
        S00 = mu - q * C11;
        S01 = q * C01;
        S11 = mu - q * C00;
    } else {
        real a = mu * ((I1 - real(2)) + real(1));
        real b = (real(0.5) * (C * mu)) * (I2 - real(1)) - mu;
        S00 = a + b * C11;
        S01 = -(b * C01);
        S11 = a + b * C00;
    }
}

template <typename real>
__device__ __forceinline__ void membrane_force(int law, real mu, real C, const real m[4], real A0,
                                               const real xa[3], const real xb[3], const real xc[3],
                                               real f[3][3])
{
    real Fh[3][2], C00, C01, C11, S00, S01, S11;
    membrane_kin(xa, xb, xc, m, Fh, C00, C01, C11);
    membrane_S(law, mu, C, C00, C01, C11, S00, S01, S11);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        real P0 = Fh[i][0] * S00 + Fh[i][1] * S01;
        real P1 = Fh[i][0] * S01 + Fh[i][1] * S11;
        f[1][i] = -(A0 * (P0 * m[0] + P1 * m[1]));
        f[2][i] = -(A0 * (P0 * m[2] + P1 * m[3]));
        f[0][i] = -(f[1][i] + f[2][i]);
    }
}

// Directional derivative of the membrane element force along w (for the
// Hessian-vector product): dFh = dDs Dm^-1, dC = dFh^T Fh + Fh^T dFh,
//   NH:     dS = -mu (adj(dC)/I2^2 - 2 adj(C) dI2/I2^3)
//   Skalak: dS = mu dI1 I + (muD/2) dI2 adj(C) + (muD/2 (I2-1) - mu) adj(dC)
//   dP = dFh S + Fh dS,  df_k = -A0 dP grad N_k.
template <typename real>
__device__ __forceinline__ void membrane_dforce(int law, real mu, real C, const real m[4], real A0,
                                                const real xa[3], const real xb[3], const real xc[3],
                                                const real wa[3], const real wb[3], const real wc[3],
                                                real df[3][3])
{
    real Fh[3][2], C00, C01, C11, S00, S01, S11, dF[3][2];
    membrane_kin(xa, xb, xc, m, Fh, C00, C01, C11);
    membrane_S(law, mu, C, C00, C01, C11, S00, S01, S11);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        real d1 = wb[i] - wa[i], d2 = wc[i] - wa[i];
        dF[i][0] = d1 * m[0] + d2 * m[2];
        dF[i][1] = d1 * m[1] + d2 * m[3];
    }
    real dC00 = 0, dC01 = 0, dC11 = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dC00 += real(2) * dF[i][0] * Fh[i][0];
        dC11 += real(2) * dF[i][1] * Fh[i][1];
        dC01 += dF[i][0] * Fh[i][1] + Fh[i][0] * dF[i][1];
    }
    real I2 = C00 * C11 - C01 * C01;
    real dI1 = dC00 + dC11, dI2 = dC00 * C11 + C00 * dC11 - real(2) * C01 * dC01;
    real dS00, dS01, dS11;
    if (law == 0) {
        real i2 = real(1) / (I2 * I2), i3 = real(2) * dI2 / (I2 * I2 * I2);
        dS00 = -mu * (dC11 * i2 - C11 * i3);
        dS11 = -mu * (dC00 * i2 - C00 * i3);
        dS01 = mu * (dC01 * i2 - C01 * i3);
    } else {
        real muD = C * mu;
        real b = real(0.5) * muD * (I2 - real(1)) - mu, db = real(0.5) * muD * dI2;
        dS00 = mu * dI1 + db * C11 + b * dC11;
        dS11 = mu * dI1 + db * C00 + b * dC00;
        dS01 = -(db * C01 + b * dC01);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        real P0 = dF[i][0] * S00 + dF[i][1] * S01 + Fh[i][0] * dS00 + Fh[i][1] * dS01;
        real P1 = dF[i][0] * S01 + dF[i][1] * S11 + Fh[i][0] * dS01 + Fh[i][1] * dS11;
        df[1][i] = -(A0 * (P0 * m[0] + P1 * m[1]));
        df[2][i] = -(A0 * (P0 * m[2] + P1 * m[3]));
        df[0][i] = -(df[1][i] + df[2][i]);
    }
}

// ------------------------------------------------------------ solids
// det3 = M00 (M11 M22 - M12 M21) - M01 (M10 M22 - M12 M20) + M02 (M10 M21 - M11 M20)
template <typename real>
__device__ __forceinline__ real det3(const real M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
         - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
         + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

// inverse by the adjugate: R[i][j] = cofactor[j][i] / det
template <typename real>
__device__ __forceinline__ void inv3(const real M[3][3], real det, real R[3][3])
{
    R[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
    R[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
    R[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
    R[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
    R[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
    R[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
    R[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
    R[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
    R[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
}

// F = Ds M: F[i][j] = (Ds[i][0]*M[0][j] + Ds[i][1]*M[1][j]) + Ds[i][2]*M[2][j],
// Ds columns x1-x0, x2-x0, x3-x0.
template <typename real>
__device__ __forceinline__ void tet_F(const real x[4][3], const real *M, real F[3][3])
{
    real Ds[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            Ds[i][c] = x[1 + c][i] - x[0][i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            F[i][j] = (Ds[i][0] * M[0 * 3 + j] + Ds[i][1] * M[1 * 3 + j]) + Ds[i][2] * M[2 * 3 + j];
}

// J = det F; Finv = adj(F)/J; Cinv[i][j] = (Finv[i][0] Finv[j][0] + Finv[i][1] Finv[j][1]) + Finv[i][2] Finv[j][2];
// a = (0.5*lam)*(J*J - 1); S[i][j] = a*Cinv[i][j] + mu*(delta_ij - Cinv[i][j]).
template <typename real>
__device__ __forceinline__ real tet_S(real lam, real mu, const real F[3][3], real S[3][3],
                                      real Ci[3][3], real Fi[3][3])
{
    real J = det3(F);
    inv3(F, J, Fi);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Ci[i][j] = (Fi[i][0] * Fi[j][0] + Fi[i][1] * Fi[j][1]) + Fi[i][2] * Fi[j][2];
    real a = (real(0.5) * lam) * (J * J - real(1));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            S[i][j] = a * Ci[i][j] + mu * ((i == j ? real(1) : real(0)) - Ci[i][j]);
    return J;
}

// P[i][j] = (F[i][0] S[0][j] + F[i][1] S[1][j]) + F[i][2] S[2][j];
// f_k[i] = -(V0*((P[i][0] M[k-1][0] + P[i][1] M[k-1][1]) + P[i][2] M[k-1][2])), k = 1..3;
// f_0[i] = -((f_1[i] + f_2[i]) + f_3[i]). Returns J.
template <typename real>
__device__ __forceinline__ real tet_force(real lam, real mu, const real *M, real V0, const real x[4][3],
                                          real f[4][3])
{
    real F[3][3], S[3][3], Ci[3][3], Fi[3][3], P[3][3];
    tet_F(x, M, F);
    real J = tet_S(lam, mu, F, S, Ci, Fi);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P[i][j] = (F[i][0] * S[0][j] + F[i][1] * S[1][j]) + F[i][2] * S[2][j];
#pragma unroll
    for (int k = 1; k <= 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const real *g = M + 3 * (k - 1);
            f[k][i] = -(V0 * ((P[i][0] * g[0] + P[i][1] * g[1]) + P[i][2] * g[2]));
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
        f[0][i] = -((f[1][i] + f[2][i]) + f[3][i]);
    return J;
}

// dF = dDs M, dJ = J tr(F^-1 dF), dC = dF^T F + F^T dF, dC^-1 = -C^-1 dC C^-1,
// dS = lam J dJ C^-1 + (lam/2 (J^2 - 1) - mu) dC^-1, dP = dF S + F dS.
template <typename real>
__device__ __forceinline__ void tet_dforce(real lam, real mu, const real *M, real V0, const real x[4][3],
                                           const real w[4][3], real df[4][3])
{
    real F[3][3], S[3][3], Ci[3][3], Fi[3][3], dF[3][3];
    tet_F(x, M, F);
    tet_F(w, M, dF);
    real J = tet_S(lam, mu, F, S, Ci, Fi);
    real tr = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            tr += Fi[i][k] * dF[k][i];
    real dJ = J * tr;
    real dC[3][3], T[3][3], dS[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            real s = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                s += dF[k][i] * F[k][j] + F[k][i] * dF[k][j];
            dC[i][j] = s;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            real s = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                s += Ci[i][k] * dC[k][j];
            T[i][j] = s;
        }
    real a = real(0.5) * lam * (J * J - real(1)) - mu;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            real s = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                s += T[i][k] * Ci[k][j];
            dS[i][j] = lam * J * dJ * Ci[i][j] - a * s;
        }
    real dP[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            real s = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                s += dF[i][k] * S[k][j] + F[i][k] * dS[k][j];
            dP[i][j] = s;
        }
#pragma unroll
    for (int k = 1; k <= 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const real *g = M + 3 * (k - 1);
            df[k][i] = -(V0 * (dP[i][0] * g[0] + dP[i][1] * g[1] + dP[i][2] * g[2]));
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
        df[0][i] = -(df[1][i] + df[2][i] + df[3][i]);
}

template <typename real>
__device__ __forceinline__ const real *ref_ptr(const TmplDev &T);
template <>
__device__ __forceinline__ const double *ref_ptr<double>(const TmplDev &T) { return T.ref_d; }
template <>
__device__ __forceinline__ const float *ref_ptr<float>(const TmplDev &T) { return T.ref_f; }

// ------------------------------------------------------------ element pass
// Thread per (instance, element). Writes the element's nodal forces (or
// force derivatives along w, negated: the Hessian-vector contribution) to
// elem_buf[(elem_off + e)*12 + 3*v + i].
template <typename real, bool HVP>
__global__ void elem_force_kernel(DevBatch b, const real *__restrict__ x, const real *__restrict__ w,
                                  real *__restrict__ ebuf, unsigned long long *status)
{
    const int i = blockIdx.y;
    const InstDev I = b.inst[i];
    const TmplDev T = b.tmpl[I.tmpl];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long inverted = 0;
    if (e < T.n_elems) {
        const long long N = b.N;
        const real *ref = ref_ptr<real>(T);
        real *out = ebuf + (I.elem_off + e) * 12;
        if (T.kind == 0) {
            int v[3] = {T.elems[3 * e], T.elems[3 * e + 1], T.elems[3 * e + 2]};
            real xs[3][3], ws[3][3], f[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    xs[c][a] = x[a * N + I.node_off + v[c]];
                    if (HVP)
                        ws[c][a] = w[a * N + I.node_off + v[c]];
                }
            const real *r = ref + 5 * e;
            real m[4] = {r[0], r[1], r[2], r[3]};
            if (HVP) {
                membrane_dforce<real>(T.law, (real)T.mu, (real)T.C, m, r[4], xs[0], xs[1], xs[2], ws[0],
                                      ws[1], ws[2], f);
            } else {
                membrane_force<real>(T.law, (real)T.mu, (real)T.C, m, r[4], xs[0], xs[1], xs[2], f);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    out[3 * c + a] = HVP ? -f[c][a] : f[c][a];
        } else {
            real xs[4][3], ws[4][3], f[4][3];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int v = T.elems[4 * e + c];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    xs[c][a] = x[a * N + I.node_off + v];
                    if (HVP)
                        ws[c][a] = w[a * N + I.node_off + v];
                }
            }
            const real *r = ref + 10 * e;
            if (HVP) {
                tet_dforce<real>((real)T.lam, (real)T.mu, r, r[9], xs, ws, f);
            } else {
                real J = tet_force<real>((real)T.lam, (real)T.mu, r, r[9], xs, f);
                inverted = !(J > real(0));
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    out[3 * c + a] = HVP ? -f[c][a] : f[c][a];
        }
    }
    if (!HVP) {
        // one status update per warp
        unsigned long long tot = inverted;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            tot += __shfl_down_sync(0xffffffffu, tot, o);
        if ((threadIdx.x & 31) == 0)
            status_add(status, ST_INVERTED, tot);
    }
}

// Thread per (instance, node): F = sum over incident (element, vertex) in
// ascending element order, starting from 0: acc = acc + f.
template <typename real>
__global__ void node_gather_kernel(DevBatch b, const real *__restrict__ ebuf, real *__restrict__ F)
{
    const int i = blockIdx.y;
    const InstDev I = b.inst[i];
    const TmplDev T = b.tmpl[I.tmpl];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T.n_nodes)
        return;
    real acc[3] = {real(0), real(0), real(0)};
    for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
        int code = T.inc_idx[q];
        const real *src = ebuf + (I.elem_off + (code >> 2)) * 12 + 3 * (code & 3);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            acc[a] = acc[a] + src[a];
    }
    const long long N = b.N;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        F[a * N + I.node_off + k] = acc[a];
}

// ------------------------------------------------------------ fluid stress
// Newtonian and polymer fluid-stress parts of Eq. FEM inside a solid (Sec.
// "Governing Equations"; they enter F^IB with a plus sign), per tet on the
// reference configuration, in this order:
//   F = Ds M, J = det F, Fi = F^-1; G = Du M = sum_k u_k (x) grad N_k;
//   Lv[i][j] = (G[i][0] Fi[0][j] + G[i][1] Fi[1][j]) + G[i][2] Fi[2][j];
//   E[i][j] = Lv[i][j] + Lv[j][i];
//   P[i][j] = (eta J) ((E[i][0] Fi[j][0] + E[i][1] Fi[j][1]) + E[i][2] Fi[j][2]);
//   polymer: Cb[i][j] = (((c_0 + c_1) + c_2) + c_3) * 0.25, c_k = C_k[i][j] - d_ij,
//   P[i][j] = P[i][j] + (J cp) ((Cb[i][0] Fi[j][0] + Cb[i][1] Fi[j][1]) + Cb[i][2] Fi[j][2]),
//   cp = eta (1 - beta) / lambda;
//   f_k[i] = V0 ((P[i][0] M[k-1][0] + P[i][1] M[k-1][1]) + P[i][2] M[k-1][2]), k = 1..3;
//   f_0[i] = -((f_1[i] + f_2[i]) + f_3[i]).
// C per node: (xx, yy, zz, xy, xz, yz).
template <typename real>
__device__ __forceinline__ void tet_fluid_force(real eta, real cp, const real *M, real V0, const real x[4][3],
                                                const real u[4][3], const real C[4][6], bool polymer,
                                                real f[4][3])
{
    real F[3][3], G[3][3], Fi[3][3], Lv[3][3], E[3][3], P[3][3];
    tet_F(x, M, F);
    tet_F(u, M, G);
    const real J = det3(F);
    inv3(F, J, Fi);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Lv[i][j] = (G[i][0] * Fi[0][j] + G[i][1] * Fi[1][j]) + G[i][2] * Fi[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            E[i][j] = Lv[i][j] + Lv[j][i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            P[i][j] = (eta * J) * ((E[i][0] * Fi[j][0] + E[i][1] * Fi[j][1]) + E[i][2] * Fi[j][2]);
    if (polymer) {
        const int sym[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
        real Cb[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const real dij = i == j ? real(1) : real(0);
                real acc = C[0][sym[i][j]] - dij;
#pragma unroll
                for (int k = 1; k < 4; ++k)
                    acc = acc + (C[k][sym[i][j]] - dij);
                Cb[i][j] = acc * real(0.25);
            }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                P[i][j] = P[i][j] + (J * cp) * ((Cb[i][0] * Fi[j][0] + Cb[i][1] * Fi[j][1]) + Cb[i][2] * Fi[j][2]);
    }
#pragma unroll
    for (int k = 1; k <= 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const real *g = M + 3 * (k - 1);
            f[k][i] = V0 * ((P[i][0] * g[0] + P[i][1] * g[1]) + P[i][2] * g[2]);
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
        f[0][i] = -((f[1][i] + f[2][i]) + f[3][i]);
}

// Thread per (instance, element) of a solid: the element's fluid-stress
// nodal forces into elem_buf; fluid_gather_kernel then sums them per node.
// Membranes carry no fluid stress in the paper's thin-shell model.
template <typename real>
__global__ void fluid_elem_kernel(DevBatch b, const real *__restrict__ x, const real *__restrict__ u,
                                  const real *__restrict__ C, real eta, real cp, real *__restrict__ ebuf)
{
    const InstDev I = b.inst[blockIdx.y];
    const TmplDev T = b.tmpl[I.tmpl];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= T.n_elems)
        return;
    if (T.kind == 0)
        return;   // membranes: no fluid stress (fluid_gather_kernel writes their zeros)
    real *out = ebuf + (I.elem_off + e) * 12;
    const long long N = b.N;
    real xs[4][3], us[4][3], Cs[4][6], f[4][3];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const long long v = I.node_off + T.elems[4 * e + c];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xs[c][a] = x[a * N + v];
            us[c][a] = u[a * N + v];
        }
#pragma unroll
        for (int q = 0; q < 6; ++q)
            Cs[c][q] = C ? C[q * N + v] : real(0);
    }
    const real *r = ref_ptr<real>(T) + 10 * e;
    tet_fluid_force<real>(eta, cp, r, r[9], xs, us, Cs, C != nullptr, f);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            out[3 * c + a] = f[c][a];
}

// ------------------------------------------------------------ bending
// Geometry of one incident triangle (p[c] is the vertex itself, corners
// c1 = c+1, c2 = c+2): edge dots at every corner, twice the area
// (|u x w| is the same from every corner), the unnormalised face normal.
// cot at a corner = dot / (2 area); the corner is obtuse iff its dot < 0.
template <typename real>
struct TriGeom {
    real dot[3];
    real twoA;
    real fn[3];
};

template <typename real>
__device__ __forceinline__ void tri_geom(const real p[3][3], TriGeom<real> &t)
{
    real e1[3], e2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e1[a] = p[1][a] - p[0][a];
        e2[a] = p[2][a] - p[0][a];
    }
    t.fn[0] = e1[1] * e2[2] - e1[2] * e2[1];
    t.fn[1] = e1[2] * e2[0] - e1[0] * e2[2];
    t.fn[2] = e1[0] * e2[1] - e1[1] * e2[0];
    t.twoA = sqrt(t.fn[0] * t.fn[0] + t.fn[1] * t.fn[1] + t.fn[2] * t.fn[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        real u0 = p[(c + 1) % 3][0] - p[c][0], u1 = p[(c + 1) % 3][1] - p[c][1], u2 = p[(c + 1) % 3][2] - p[c][2];
        real w0 = p[(c + 2) % 3][0] - p[c][0], w1 = p[(c + 2) % 3][1] - p[c][1], w2 = p[(c + 2) % 3][2] - p[c][2];
        t.dot[c] = u0 * w0 + u1 * w1 + u2 * w2;
    }
}

// Pass 1 at vertex i (template-local id k), over its incident triangles in
// ascending order: K += cot_k (x_i - x_j) + cot_j (x_i - x_k); mixed Voronoi
// area (Voronoi region if no corner is obtuse, area/2 at an obtuse corner,
// area/4 at the others); corner angles; area-weighted normal. Outputs A,
// kH = K.n/2 (K /= 2A), kG = (2 pi - angles)/A and the unit normal n.
// The cotangents share one reciprocal of 2A per triangle. The angle deficit
// 2 pi - sum theta is minus the argument of prod (dot + i 2A) over the corners
// (each factor has argument theta), one atan2 per vertex instead of one per
// corner; it equals the angle sum's deficit while that lies in (-pi, pi), and
// the product is rescaled by an exact power of two if it grows small.
template <typename real, typename Load>
__device__ inline void bend_vertex_pass1(const TmplDev &T, int k, Load ld, real &A_out, real &kH_out,
                                         real &kG_out, real n_out[3])
{
    real K[3] = {0, 0, 0}, nrm[3] = {0, 0, 0}, A = 0;
    real zr = 1, zi = 0;   // running product of (dot + i 2A) over the corners
    for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
        // incident triangle rotated to start at this vertex: (k, j, l)
        const int2 jk = T.ring[q];
        const int c = 0, c1 = 1, c2 = 2;
        real p[3][3];
        ld(k, p[0]);
        ld(jk.x, p[1]);
        ld(jk.y, p[2]);
        TriGeom<real> t;
        tri_geom(p, t);
        const real inv2A = real(1) / t.twoA;
        real cj = t.dot[c1] * inv2A, ck = t.dot[c2] * inv2A;
        real eij[3], eik[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            eij[a] = p[c][a] - p[c1][a];
            eik[a] = p[c][a] - p[c2][a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            K[a] += ck * eij[a] + cj * eik[a];
        bool obtuse = t.dot[0] < real(0) || t.dot[1] < real(0) || t.dot[2] < real(0);
        real Ai;
        if (!obtuse)
            Ai = (ck * (eij[0] * eij[0] + eij[1] * eij[1] + eij[2] * eij[2])
                  + cj * (eik[0] * eik[0] + eik[1] * eik[1] + eik[2] * eik[2])) / real(8);
        else if (t.dot[c] < real(0))
            Ai = t.twoA / real(4);
        else
            Ai = t.twoA / real(8);
        A += Ai;
        const real pr = zr * t.dot[c] - zi * t.twoA, pi = zr * t.twoA + zi * t.dot[c];
        zr = pr;
        zi = pi;
        if (fabs(zr) + fabs(zi) < real(1e-30)) {
            zr *= real(1099511627776.0);   // 2^40, exact
            zi *= real(1099511627776.0);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            nrm[a] += t.fn[a];
    }
    real nl = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        n_out[a] = nrm[a] / nl;
        K[a] /= real(2) * A;
    }
    A_out = A;
    kH_out = real(0.5) * (K[0] * n_out[0] + K[1] * n_out[1] + K[2] * n_out[2]);
    kG_out = -atan2(zi, zr) / A;
}

// Pass 2 at vertex k: cotangent Laplacian of (kH - kH0) and the force.
template <typename real, typename Load, typename LoadH>
__device__ inline void bend_vertex_pass2(const TmplDev &T, int k, Load ld, LoadH kHof, real A, real kH,
                                         real kG, const real n[3], real Fb[3])
{
    const real kH0 = real(-0.5) * (real)T.c0;
    real lap = 0;
    for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
        const int2 jk = T.ring[q];
        real p[3][3];
        ld(k, p[0]);
        ld(jk.x, p[1]);
        ld(jk.y, p[2]);
        TriGeom<real> t;
        tri_geom(p, t);
        const real inv2A = real(1) / t.twoA;
        lap += (t.dot[2] * inv2A) * ((kHof(jk.x) - kH0) - (kH - kH0))
             + (t.dot[1] * inv2A) * ((kHof(jk.y) - kH0) - (kH - kH0));
    }
    real L = lap / (real(2) * A);
    real dh = kH - kH0;
    real mag = real(2) * (real)T.kb * (L + real(2) * dh * (kH * kH - kG + kH0 * kH)) * A;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        Fb[a] = mag * n[a];
}

// Global-memory bending passes (thread per (instance, node)), used by the
// deterministic path. bend_buf per global node: [A, kH, kG, n0, n1, n2].
template <typename real>
__global__ void bend_pass1_kernel(DevBatch b, const real *__restrict__ x, real *__restrict__ bb)
{
    const int i = blockIdx.y;
    const InstDev I = b.inst[i];
    const TmplDev T = b.tmpl[I.tmpl];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (T.kind != 0 || T.kb == 0.0 || k >= T.n_nodes)
        return;
    const long long N = b.N;
    auto ld = [&](int v, real p[3]) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            p[a] = x[a * N + I.node_off + v];
    };
    real A, kH, kG, n[3];
    bend_vertex_pass1<real>(T, k, ld, A, kH, kG, n);
    real *o = bb + 6LL * (I.node_off + k);
    o[0] = A; o[1] = kH; o[2] = kG; o[3] = n[0]; o[4] = n[1]; o[5] = n[2];
}

// Node sums of the fluid-stress element buffer for solids (ascending element
// order from 0, as node_gather_kernel); membrane nodes get 0 (ADD: unchanged).
template <typename real, bool ADD>
__global__ void fluid_gather_kernel(DevBatch b, const real *__restrict__ ebuf, real *__restrict__ F)
{
    const InstDev I = b.inst[blockIdx.y];
    const TmplDev T = b.tmpl[I.tmpl];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T.n_nodes || (ADD && T.kind == 0))
        return;
    real acc[3] = {real(0), real(0), real(0)};
    if (T.kind != 0) {
        for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
            const int code = T.inc_idx[q];
            const real *src = ebuf + (I.elem_off + (code >> 2)) * 12 + 3 * (code & 3);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                acc[a] = acc[a] + src[a];
        }
    }
    const long long N = b.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        real *p = F + a * N + I.node_off + k;
        *p = ADD ? *p + acc[a] : acc[a];
    }
}

// n_k A_k of every membrane node (unit normal times mixed area, from the
// bending pass-1 operators) as a node array; solid nodes get 0. Source of
// the indicator-function equation (Sec. "Variable Viscosity Implementation").
template <typename real>
__global__ void area_normal_kernel(DevBatch b, const real *__restrict__ x, real *__restrict__ nA)
{
    const int i = blockIdx.y;
    const InstDev I = b.inst[i];
    const TmplDev T = b.tmpl[I.tmpl];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T.n_nodes)
        return;
    const long long N = b.N;
    const long long node = I.node_off + k;
    if (T.kind != 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            nA[a * N + node] = real(0);
        return;
    }
    auto ld = [&](int v, real p[3]) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            p[a] = x[a * N + I.node_off + v];
    };
    real A, kH, kG, n[3];
    bend_vertex_pass1<real>(T, k, ld, A, kH, kG, n);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        nA[a * N + node] = n[a] * A;
}

// F = F_el + F_be (one add per component).
template <typename real>
__global__ void bend_pass2_kernel(DevBatch b, const real *__restrict__ x, const real *__restrict__ bb,
                                  real *__restrict__ F)
{
    const int i = blockIdx.y;
    const InstDev I = b.inst[i];
    const TmplDev T = b.tmpl[I.tmpl];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (T.kind != 0 || T.kb == 0.0 || k >= T.n_nodes)
        return;
    const long long N = b.N;
    auto ld = [&](int v, real p[3]) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            p[a] = x[a * N + I.node_off + v];
    };
    auto kHof = [&](int v) { return bb[6LL * (I.node_off + v) + 1]; };
    const real *me = bb + 6LL * (I.node_off + k);
    real n[3] = {me[3], me[4], me[5]}, Fb[3];
    bend_vertex_pass2<real>(T, k, ld, kHof, me[0], me[1], me[2], n, Fb);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        real *p = F + a * N + I.node_off + k;
        *p = *p + Fb[a];
    }
}

// ------------------------------------------------------- FP32 bending helpers
// The same discrete operators as bend_vertex_pass1/2 (Meyer et al. 2003),
// arranged for FP32 throughput. Per incident triangle (k, j, l) with
// e1 = x_j - x_k, e2 = x_l - x_k: 2A = |e1 x e2| from one rsqrt, the corner
// dots d_k = e1.e2, d_j = |e1|^2 - d_k, d_l = |e2|^2 - d_k, cotangents d/2A.
// The corner-angle sum enters only through 2 pi - sum(theta); it is taken as
// -arg(prod_t (cos theta_t + i sin theta_t)), one atan2 per vertex, which
// equals the deficit while it lies in (-pi, pi) (any vertex of a closed mesh
// that is not folded onto itself).
struct RingF {
    float e1[3], e2[3], fn[3], inv2A, dk, dj, dl, l1, l2;
};
__device__ __forceinline__ void ring_tri_f32(const float xk[3], const float xj[3], const float xl[3], RingF &t)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        t.e1[a] = xj[a] - xk[a];
        t.e2[a] = xl[a] - xk[a];
    }
    t.fn[0] = t.e1[1] * t.e2[2] - t.e1[2] * t.e2[1];
    t.fn[1] = t.e1[2] * t.e2[0] - t.e1[0] * t.e2[2];
    t.fn[2] = t.e1[0] * t.e2[1] - t.e1[1] * t.e2[0];
    t.inv2A = rsqrtf(t.fn[0] * t.fn[0] + t.fn[1] * t.fn[1] + t.fn[2] * t.fn[2]);
    t.l1 = t.e1[0] * t.e1[0] + t.e1[1] * t.e1[1] + t.e1[2] * t.e1[2];
    t.l2 = t.e2[0] * t.e2[0] + t.e2[1] * t.e2[1] + t.e2[2] * t.e2[2];
    t.dk = t.e1[0] * t.e2[0] + t.e1[1] * t.e2[1] + t.e1[2] * t.e2[2];
    t.dj = t.l1 - t.dk;
    t.dl = t.l2 - t.dk;
}

// Pass 1 at vertex k (positions in shared memory, SoA with stride nn):
// mixed area A, kH = (K.n)/2 with K the cotangent mean-curvature vector over
// 2A, kG = deficit / A, unit normal n (area-weighted face normals).
__device__ __forceinline__ void bend1_f32(const TmplDev &T, int k, const float *xs, int nn, float &A_out,
                                          float &kH_out, float &kG_out, float n_out[3])
{
    float K[3] = {0.f, 0.f, 0.f}, nrm[3] = {0.f, 0.f, 0.f}, A = 0.f, zr = 1.f, zi = 0.f;
    const float xk[3] = {xs[k], xs[nn + k], xs[2 * nn + k]};
    for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
        const int2 jl = T.ring[q];
        const float xj[3] = {xs[jl.x], xs[nn + jl.x], xs[2 * nn + jl.x]};
        const float xl[3] = {xs[jl.y], xs[nn + jl.y], xs[2 * nn + jl.y]};
        RingF t;
        ring_tri_f32(xk, xj, xl, t);
        const float cj = t.dj * t.inv2A, cl = t.dl * t.inv2A;
        // K += cot_l (x_k - x_j) + cot_j (x_k - x_l)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            K[a] -= cl * t.e1[a] + cj * t.e2[a];
        const float twoA = (t.fn[0] * t.fn[0] + t.fn[1] * t.fn[1] + t.fn[2] * t.fn[2]) * t.inv2A;
        float Ai;
        if (t.dk >= 0.f && t.dj >= 0.f && t.dl >= 0.f)
            Ai = (cl * t.l1 + cj * t.l2) * 0.125f;
        else
            Ai = t.dk < 0.f ? twoA * 0.25f : twoA * 0.125f;
        A += Ai;
        // unit (cos, sin) of the corner angle at k, |e1||e2| = sqrt(l1 l2)
        const float r = rsqrtf(t.l1 * t.l2);
        const float cr = t.dk * r, ci = twoA * r;
        const float nr = zr * cr - zi * ci;
        zi = zr * ci + zi * cr;
        zr = nr;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            nrm[a] += t.fn[a];
    }
    const float rn = rsqrtf(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    const float h = 0.5f / A;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        n_out[a] = nrm[a] * rn;
        K[a] *= h;
    }
    A_out = A;
    kH_out = 0.5f * (K[0] * n_out[0] + K[1] * n_out[1] + K[2] * n_out[2]);
    kG_out = -atan2f(zi, zr) / A;
}

// Pass 2 at vertex k: lap = sum (cot_l (kH_j - kH_k) + cot_j (kH_l - kH_k))
// and the unnormalised normal, in the order of pass 1.
__device__ __forceinline__ void bend2_f32(const TmplDev &T, int k, const float *xs, const float *kHs, int nn,
                                          float &lap_out, float nrm[3])
{
    float lap = 0.f;
    nrm[0] = nrm[1] = nrm[2] = 0.f;
    const float xk[3] = {xs[k], xs[nn + k], xs[2 * nn + k]};
    const float kHk = kHs[k];
    for (int q = T.inc_off[k]; q < T.inc_off[k + 1]; ++q) {
        const int2 jl = T.ring[q];
        const float xj[3] = {xs[jl.x], xs[nn + jl.x], xs[2 * nn + jl.x]};
        const float xl[3] = {xs[jl.y], xs[nn + jl.y], xs[2 * nn + jl.y]};
        RingF t;
        ring_tri_f32(xk, xj, xl, t);
        lap += (t.dl * t.inv2A) * (kHs[jl.x] - kHk) + (t.dj * t.inv2A) * (kHs[jl.y] - kHk);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            nrm[a] += t.fn[a];
    }
    lap_out = lap;
}

// ------------------------------------------------------------ FP32 fused path
// One CTA per instance: node positions and force accumulators in shared
// memory, element forces added with shared-memory atomics (order not
// reproducible), then the two bending passes, then one coalesced write of F.
// The bending force is split so that only kH is kept between the passes:
//   pass 1 (vertex i): F_i += 2 kb * 2 (kH - kH0)(kH^2 - kG + kH0 kH) A_i n_i
//   pass 2 (vertex i): F_i += 2 kb * Lap(kH - kH0) A_i n_i = kb * lap_i * n_i
// where lap_i = sum_j (cot a_ij + cot b_ij)(kH_j - kH_i) (A_i cancels) and n_i
// is recomputed from the incident faces in the same order as in pass 1.
// Shared memory: 3n (x) + 3n (F) + n (kH) floats.
static __global__ void __launch_bounds__(512, 2) forces_fused_f32_kernel(DevBatch b, const float *__restrict__ x,
                                                                      float *__restrict__ F,
                                                                      unsigned long long *status, int inst0)
{
    extern __shared__ float sm[];
    const InstDev I = b.inst[inst0 + blockIdx.x];   // particles inst0, inst0 + 1, ...
    const TmplDev T = b.tmpl[I.tmpl];
    const int nn = T.n_nodes;
    const long long N = b.N;
    float *xs = sm;               // [3][nn]
    float *Fs = sm + 3 * nn;      // [3][nn]
    float *kHs = sm + 6 * nn;     // [nn]
    const unsigned sF = smem_u32(Fs);
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xs[a * nn + k] = x[a * N + I.node_off + k];
            Fs[a * nn + k] = 0.f;
        }
    }
    __syncthreads();
    const float *ref = T.ref_f;
    unsigned long long inverted = 0;
    for (int e = threadIdx.x; e < T.n_elems; e += blockDim.x) {
        if (T.kind == 0) {
            int v[3] = {T.elems[3 * e], T.elems[3 * e + 1], T.elems[3 * e + 2]};
            float p[3][3], f[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    p[c][a] = xs[a * nn + v[c]];
            const float *r = ref + 5 * e;
            float m[4] = {r[0], r[1], r[2], r[3]};
            membrane_force<float>(T.law, (float)T.mu, (float)T.C, m, r[4], p[0], p[1], p[2], f);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    red_shared_add(sF + 4u * (unsigned)(a * nn + v[c]), f[c][a]);
        } else {
            int v[4];
            float p[4][3], f[4][3];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                v[c] = T.elems[4 * e + c];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    p[c][a] = xs[a * nn + v[c]];
            }
            const float *r = ref + 10 * e;
            float J = tet_force<float>((float)T.lam, (float)T.mu, r, r[9], p, f);
            inverted += !(J > 0.f);
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    red_shared_add(sF + 4u * (unsigned)(a * nn + v[c]), f[c][a]);
        }
    }
    if (T.kind == 0 && T.kb != 0.0) {
        const float kb = (float)T.kb, kH0 = -0.5f * (float)T.c0;
        for (int k = threadIdx.x; k < nn; k += blockDim.x) {
            float A, kH, kG, n[3];
            bend1_f32(T, k, xs, nn, A, kH, kG, n);
            kHs[k] = kH;
            const float dh = kH - kH0;
            const float mag = 2.f * kb * (2.f * dh * (kH * kH - kG + kH0 * kH)) * A;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                red_shared_add(sF + 4u * (unsigned)(a * nn + k), mag * n[a]);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nn; k += blockDim.x) {
            float lap, nrm[3];
            bend2_f32(T, k, xs, kHs, nn, lap, nrm);
            const float s = kb * lap * rsqrtf(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                red_shared_add(sF + 4u * (unsigned)(a * nn + k), s * nrm[a]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            F[a * N + I.node_off + k] = Fs[a * nn + k];
    }
    unsigned long long tot = inverted;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        tot += __shfl_down_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0)
        status_add(status, ST_INVERTED, tot);
}

}  // namespace ifem
