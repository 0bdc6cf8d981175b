/*
 * ifem_oracle.c -- plain FP64 CPU oracle of the IFEM fluid-structure coupling
 * step (Saadat, Guido, Iaccarino & Shaqfeh, arXiv:1807.08219).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct reference
 * that the CUDA library is checked against. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does. It shares no code, header or table with the CUDA library.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, no
 * reassociation), single-threaded, plain loops. Every floating-point
 * expression below is written in the exact evaluation order stated in its
 * comment, because the deterministic FP64 mode of the CUDA library promises
 * the same bits for the element forces, the nodal sums, spreading and
 * interpolation.
 *
 * Conventions
 *   x, X, F, v     node arrays, AoS (N, 3) row-major.
 *   grids          per velocity component d: n^3 values indexed
 *                  (k*n + j)*n + i, components stacked: grid[d*n^3 + ...].
 *   MAC lattices   component d has nodes at ((i,j,k) + o_d) h with
 *                  o_d = (1/2,1/2,1/2) - e_d/2, h = L/n.
 *
 * Functions and the passages they follow (section / equation of the paper):
 *   ifo_membrane_*   Sec. "Numerical Implementation": Eq. FEM_Membrane, the
 *                    tangent-plane deformation gradient, S-hat = 2 dW/dC-hat
 *                    with the neo-Hookean (Eq. neo-Hookena) and Skalak
 *                    (Eq. Skalak) energies.
 *   ifo_tet_*        Eq. FEM with the linear-tet deformation gradient and
 *                    the discrete compressible neo-Hookean P = F S.
 *   ifo_bending_*    the Helfrich bending force of the same section (force
 *                    from the Canham-Helfrich energy, Eq. Bending_Energy),
 *                    with the Meyer-Desbrun-Schroeder-Barr discrete
 *                    operators (the paper defers the operators to Sinha &
 *                    Graham without printing them).
 *   ifo_phi4         4-point discrete delta (Peskin 2002), the kernel the
 *                    benchmark workloads name.
 *   ifo_mls_weights  Sec. "Interpolation Scheme": linear MLS, Eq. norm and
 *                    the A, B, phi equations that follow, cubic-spline W.
 *   ifo_spread / ifo_interp   the S* and S operators of that section and of
 *                    Algorithm steps 2 and 4.
 *   ifo_volume       the polyhedron volume of Sec. "Conservation of Volume
 *                    for Membranes".
 *   ifo_interp_cc    interpolation S of a cell-centred multi-component
 *                    field (the conformation tensor C of the same section).
 *   ifo_tet_fluid_forces  the Newtonian and polymer fluid-stress parts of
 *                    Eq. FEM inside solids (P^{f,N}, P^{f,P} of Sec.
 *                    "Governing Equations" / "Numerical Implementation").
 *   ifo_ab2          the Adams-Bashforth position update (Eq. Bashforth_eqn).
 *   ifo_tet_volume   the current volume of a solid (sum of tet volumes).
 *   ifo_volume_correction  the membrane volume correction of Sec.
 *                    "Conservation of Volume for Membranes".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IFO_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* 4-point discrete delta (Peskin 2002), one dimension, r in cells.   */
/*   |r| <= 1     : (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8           */
/*   1 < |r| <= 2 : (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8         */
/* Evaluation order: a=|r|, q=4a; inner t=(1+q)-q*a,                  */
/* phi=((3-2a)+sqrt(t))*0.125; outer t=((12a)-7)-q*a,                 */
/* phi=((5-2a)-sqrt(t))*0.125.                                        */
/* ------------------------------------------------------------------ */
double ifo_phi4(double r)
{
    double a = fabs(r);
    double q = 4.0 * a;
    if (a <= 1.0) {
        double t = (1.0 + q) - q * a;
        return ((3.0 - 2.0 * a) + sqrt(t)) * 0.125;
    }
    if (a <= 2.0) {
        double t = ((12.0 * a) - 7.0) - q * a;
        return ((5.0 - 2.0 * a) - sqrt(t)) * 0.125;
    }
    return 0.0;
}

/* Periodic wrap of an integer lattice index into [0, n). */
static int wrap(long i, int n)
{
    long m = i % n;
    return (int)(m < 0 ? m + n : m);
}

/* Lattice coordinate s = p * (n/L) - o  of one position component. */
static double lattice_coord(double p, double inv_h, double o)
{
    return p * inv_h - o;
}

/* MAC offset of component d along axis a. */
static double mac_off(int d, int a)
{
    return a == d ? 0.0 : 0.5;
}

/* ------------------------------------------------------------------ */
/* Cubic-spline MLS weight W(r) (Sec. Interpolation Scheme), read with */
/* the first branch 2/3 - 4r^2 + 4r^3 (the printed "-4r" is not        */
/* continuous with the second branch at r = 1/2).                      */
/* ------------------------------------------------------------------ */
double ifo_mls_w(double r)
{
    if (r <= 0.5)
        return 2.0 / 3.0 - 4.0 * r * r + 4.0 * r * r * r;
    if (r <= 1.0)
        return 4.0 / 3.0 - 4.0 * r + 4.0 * r * r - 4.0 / 3.0 * r * r * r;
    return 0.0;
}

/* Solve the 4x4 symmetric positive definite system A z = b by Cholesky. */
static int chol4_solve(const double A[16], const double b[4], double z[4])
{
    double Lm[16] = {0};
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * 4 + j];
            for (int k = 0; k < j; ++k)
                s -= Lm[i * 4 + k] * Lm[j * 4 + k];
            if (i == j) {
                if (!(s > 0.0))
                    return -1;
                Lm[i * 4 + i] = sqrt(s);
            } else {
                Lm[i * 4 + j] = s / Lm[j * 4 + j];
            }
        }
    }
    double y[4];
    for (int i = 0; i < 4; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k)
            s -= Lm[i * 4 + k] * y[k];
        y[i] = s / Lm[i * 4 + i];
    }
    for (int i = 3; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 4; ++k)
            s -= Lm[k * 4 + i] * z[k];
        z[i] = s / Lm[i * 4 + i];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Linear MLS weights at one Lagrangian point (Sec. Interpolation      */
/* Scheme). s[3]: the point in lattice-index units. support: the       */
/* weight radius h_w in cells. Stencil: the 27 lattice nodes around    */
/* the nearest node c = floor(s + 1/2), ordered z-outer, x-inner.      */
/* Basis p(x_J) = (1, (x_J - x_k)/h); minimising the weighted squared  */
/* residual gives A z = B Y, so phi_J = p(x_k)^T A^-1 W_J p(x_J) with  */
/* p(x_k) = e1 in the shifted basis.                                   */
/* Writes the stencil base c-1 (per axis) and the 27 weights.          */
/* ------------------------------------------------------------------ */
int ifo_mls_weights(const double s[3], double support, int base[3], double w[27])
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        c[a] = (int)floor(s[a] + 0.5);
        base[a] = c[a] - 1;
    }
    double A[16] = {0};
    double Wj[27], P[27][4];
    int J = 0;
    for (int kz = 0; kz < 3; ++kz)
        for (int jy = 0; jy < 3; ++jy)
            for (int ix = 0; ix < 3; ++ix, ++J) {
                double y0 = (double)(base[0] + ix) - s[0];
                double y1 = (double)(base[1] + jy) - s[1];
                double y2 = (double)(base[2] + kz) - s[2];
                double r = sqrt(y0 * y0 + y1 * y1 + y2 * y2) / support;
                Wj[J] = ifo_mls_w(r);
                P[J][0] = 1.0; P[J][1] = y0; P[J][2] = y1; P[J][3] = y2;
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b)
                        A[a * 4 + b] += Wj[J] * P[J][a] * P[J][b];
            }
    const double e1[4] = {1.0, 0.0, 0.0, 0.0};
    double z[4];
    if (chol4_solve(A, e1, z) != 0)
        return -1;
    for (J = 0; J < 27; ++J)
        w[J] = Wj[J] * (z[0] * P[J][0] + z[1] * P[J][1] + z[2] * P[J][2] + z[3] * P[J][3]);
    return 0;
}

/* Peskin weights along one axis: base index i0 = floor(s) - 1 and the  */
/* four 1D weights phi(s - (i0 + m)), m = 0..3.                         */
static long peskin_axis(double s, double phi[4])
{
    long i0 = (long)floor(s) - 1;
    for (int m = 0; m < 4; ++m)
        phi[m] = ifo_phi4(s - (double)(i0 + m));
    return i0;
}

/* ------------------------------------------------------------------ */
/* Spreading S* (Algorithm step 2): f_J += sum_k phi_J(x_J - x_k) g_k,  */
/* g_k = F_k * scale with scale = (n/L)^3 for a force density or 1 for  */
/* the literal nodal-force form. Nodes in ascending order; per node and */
/* component the stencil in z, y, x order; each grid value receives     */
/* f = f + w * g with w = (phi_x * phi_y) * phi_z (Peskin) or the MLS   */
/* weight. kernel 0 = Peskin 4-point, 1 = MLS 27-point.                 */
/* x: absolute positions (N,3). f: 3 n^3 values, accumulated into.      */
/* Returns 0, or -1 if an MLS moment matrix was singular.               */
/* ------------------------------------------------------------------ */
int ifo_spread(int kernel, int n, double L, int N, const double *x, const double *F,
               double *f, int density, double support)
{
    const double inv_h = (double)n / L;
    const double scale = density ? inv_h * inv_h * inv_h : 1.0;
    const long n3 = (long)n * n * n;
    for (int k = 0; k < N; ++k) {
        for (int d = 0; d < 3; ++d) {
            double g = F[3 * k + d] * scale;
            double s[3];
            for (int a = 0; a < 3; ++a)
                s[a] = lattice_coord(x[3 * k + a], inv_h, mac_off(d, a));
            double *fd = f + d * n3;
            if (kernel == 0) {
                double px[4], py[4], pz[4];
                long ix0 = peskin_axis(s[0], px);
                long iy0 = peskin_axis(s[1], py);
                long iz0 = peskin_axis(s[2], pz);
                for (int c = 0; c < 4; ++c)
                    for (int b = 0; b < 4; ++b)
                        for (int a = 0; a < 4; ++a) {
                            double w = (px[a] * py[b]) * pz[c];
                            long idx = ((long)wrap(iz0 + c, n) * n + wrap(iy0 + b, n)) * n
                                       + wrap(ix0 + a, n);
                            fd[idx] = fd[idx] + w * g;
                        }
            } else {
                int base[3];
                double w[27];
                if (ifo_mls_weights(s, support, base, w) != 0)
                    return -1;
                int J = 0;
                for (int c = 0; c < 3; ++c)
                    for (int b = 0; b < 3; ++b)
                        for (int a = 0; a < 3; ++a, ++J) {
                            long idx = ((long)wrap(base[2] + c, n) * n + wrap(base[1] + b, n)) * n
                                       + wrap(base[0] + a, n);
                            fd[idx] = fd[idx] + w[J] * g;
                        }
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Interpolation S (Algorithm step 4): v_k = sum_J phi_J u_J, summed    */
/* from 0 in stencil order z-outer, y, x-inner: acc = acc + w * u.      */
/* ------------------------------------------------------------------ */
int ifo_interp(int kernel, int n, double L, int N, const double *x, const double *u,
               double *v, double support)
{
    const double inv_h = (double)n / L;
    const long n3 = (long)n * n * n;
    for (int k = 0; k < N; ++k) {
        for (int d = 0; d < 3; ++d) {
            double s[3];
            for (int a = 0; a < 3; ++a)
                s[a] = lattice_coord(x[3 * k + a], inv_h, mac_off(d, a));
            const double *ud = u + d * n3;
            double acc = 0.0;
            if (kernel == 0) {
                double px[4], py[4], pz[4];
                long ix0 = peskin_axis(s[0], px);
                long iy0 = peskin_axis(s[1], py);
                long iz0 = peskin_axis(s[2], pz);
                for (int c = 0; c < 4; ++c)
                    for (int b = 0; b < 4; ++b)
                        for (int a = 0; a < 4; ++a) {
                            double w = (px[a] * py[b]) * pz[c];
                            long idx = ((long)wrap(iz0 + c, n) * n + wrap(iy0 + b, n)) * n
                                       + wrap(ix0 + a, n);
                            acc = acc + w * ud[idx];
                        }
            } else {
                int base[3];
                double w[27];
                if (ifo_mls_weights(s, support, base, w) != 0)
                    return -1;
                int J = 0;
                for (int c = 0; c < 3; ++c)
                    for (int b = 0; b < 3; ++b)
                        for (int a = 0; a < 3; ++a, ++J) {
                            long idx = ((long)wrap(base[2] + c, n) * n + wrap(base[1] + b, n)) * n
                                       + wrap(base[0] + a, n);
                            acc = acc + w[J] * ud[idx];
                        }
            }
            v[3 * k + d] = acc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Interpolation S of a cell-centred field with ncomp components (the   */
/* conformation tensor C_J of Sec. "Interpolation Scheme"): every       */
/* component sits at ((i,j,k) + 1/2) h, so s = p n/L - 1/2 on all axes. */
/* Same stencil and order as ifo_interp: acc = acc + w * c_J from 0,    */
/* z-outer, x-inner, w = (phi_x * phi_y) * phi_z (Peskin).              */
/* field: ncomp blocks of n^3 values; out: (N, ncomp).                  */
/* ------------------------------------------------------------------ */
int ifo_interp_cc(int kernel, int n, double L, int N, const double *x, const double *field, int ncomp,
                  double *out, double support)
{
    const double inv_h = (double)n / L;
    const long n3 = (long)n * n * n;
    for (int k = 0; k < N; ++k) {
        double s[3];
        for (int a = 0; a < 3; ++a)
            s[a] = lattice_coord(x[3 * k + a], inv_h, 0.5);
        double px[4], py[4], pz[4], w27[27];
        long i0[3] = {0, 0, 0};
        int base[3] = {0, 0, 0};
        if (kernel == 0) {
            i0[0] = peskin_axis(s[0], px);
            i0[1] = peskin_axis(s[1], py);
            i0[2] = peskin_axis(s[2], pz);
        } else if (ifo_mls_weights(s, support, base, w27) != 0) {
            return -1;
        }
        for (int q = 0; q < ncomp; ++q) {
            const double *cq = field + q * n3;
            double acc = 0.0;
            if (kernel == 0) {
                for (int c = 0; c < 4; ++c)
                    for (int b = 0; b < 4; ++b)
                        for (int a = 0; a < 4; ++a) {
                            double w = (px[a] * py[b]) * pz[c];
                            long idx = ((long)wrap(i0[2] + c, n) * n + wrap(i0[1] + b, n)) * n
                                       + wrap(i0[0] + a, n);
                            acc = acc + w * cq[idx];
                        }
            } else {
                int J = 0;
                for (int c = 0; c < 3; ++c)
                    for (int b = 0; b < 3; ++b)
                        for (int a = 0; a < 3; ++a, ++J) {
                            long idx = ((long)wrap(base[2] + c, n) * n + wrap(base[1] + b, n)) * n
                                       + wrap(base[0] + a, n);
                            acc = acc + w27[J] * cq[idx];
                        }
            }
            out[(long)ncomp * k + q] = acc;
        }
    }
    return 0;
}

/* ================================================================== */
/* Membranes (3-node triangles)                                       */
/* ================================================================== */

/* Reference data of every triangle (a, b, c) from the stress-free     */
/* positions X: an orthonormal tangent frame e1 = E1/|E1|,              */
/* e2 = (E1 x E2)/|E1 x E2| x e1, the 2x2 matrix of reference edges in  */
/* that frame Dm = [[l1, e1.E2], [0, e2.E2]], its inverse (row 0 and    */
/* row 1 are the in-plane gradients of the shape functions of b and c) */
/* and the reference area A0 = |E1 x E2| / 2.                           */
/* Dminv layout per triangle: [m00, m01, m10, m11].                     */
void ifo_membrane_reference(int nt, const int *tri, const double *X, double *Dminv, double *A0)
{
    for (int e = 0; e < nt; ++e) {
        const double *Xa = X + 3 * tri[3 * e], *Xb = X + 3 * tri[3 * e + 1],
                     *Xc = X + 3 * tri[3 * e + 2];
        double E1[3], E2[3], e1[3], nr[3], nh[3], e2[3];
        for (int i = 0; i < 3; ++i) {
            E1[i] = Xb[i] - Xa[i];
            E2[i] = Xc[i] - Xa[i];
        }
        double l1 = sqrt((E1[0] * E1[0] + E1[1] * E1[1]) + E1[2] * E1[2]);
        for (int i = 0; i < 3; ++i)
            e1[i] = E1[i] / l1;
        nr[0] = E1[1] * E2[2] - E1[2] * E2[1];
        nr[1] = E1[2] * E2[0] - E1[0] * E2[2];
        nr[2] = E1[0] * E2[1] - E1[1] * E2[0];
        double nl = sqrt((nr[0] * nr[0] + nr[1] * nr[1]) + nr[2] * nr[2]);
        for (int i = 0; i < 3; ++i)
            nh[i] = nr[i] / nl;
        e2[0] = nh[1] * e1[2] - nh[2] * e1[1];
        e2[1] = nh[2] * e1[0] - nh[0] * e1[2];
        e2[2] = nh[0] * e1[1] - nh[1] * e1[0];
        double d01 = (e1[0] * E2[0] + e1[1] * E2[1]) + e1[2] * E2[2];
        double d11 = (e2[0] * E2[0] + e2[1] * E2[1]) + e2[2] * E2[2];
        Dminv[4 * e + 0] = 1.0 / l1;
        Dminv[4 * e + 1] = -d01 / (l1 * d11);
        Dminv[4 * e + 2] = 0.0;
        Dminv[4 * e + 3] = 1.0 / d11;
        A0[e] = 0.5 * nl;
    }
}

/* Tangent-plane deformation gradient Fh = Ds Dm^-1 (3x2) and Ch = Fh^T Fh. */
static void membrane_kinematics(const double *xa, const double *xb, const double *xc,
                                const double *m, double Fh[3][2], double *C00, double *C01,
                                double *C11)
{
    double d1[3], d2[3];
    for (int i = 0; i < 3; ++i) {
        d1[i] = xb[i] - xa[i];
        d2[i] = xc[i] - xa[i];
    }
    for (int i = 0; i < 3; ++i) {
        Fh[i][0] = d1[i] * m[0] + d2[i] * m[2];
        Fh[i][1] = d1[i] * m[1] + d2[i] * m[3];
    }
    *C00 = (Fh[0][0] * Fh[0][0] + Fh[1][0] * Fh[1][0]) + Fh[2][0] * Fh[2][0];
    *C01 = (Fh[0][0] * Fh[0][1] + Fh[1][0] * Fh[1][1]) + Fh[2][0] * Fh[2][1];
    *C11 = (Fh[0][1] * Fh[0][1] + Fh[1][1] * Fh[1][1]) + Fh[2][1] * Fh[2][1];
}

/* Second Piola-Kirchhoff tension S-hat = 2 dW/dC-hat
 *   = 2 { dW/dI1 I + I2 C-hat^-1 dW/dI2 },  I1 = tr C-hat, I2 = det C-hat = J^2,
 * and I2 C-hat^-1 = adj(C-hat) = [[C11, -C01], [-C01, C00]].
 * law 0, neo-Hookean W = mu/2 (I1 + 1/I2 - 3):
 *   S = mu (I - adj/I2^2):  q = mu/(I2*I2); S00 = mu - q*C11; S01 = q*C01;
 *   S11 = mu - q*C00.
 * law 1, Skalak W = mu/2 (I1'^2/2 + I1' - I2') + muD/8 I2'^2 with
 *   I1' = I1 - 2, I2' = I2 - 1, muD = C mu:
 *   S = mu (I1' + 1) I + (muD/2 I2' - mu) adj:
 *   a = mu*((I1-2)+1); b = (0.5*(C*mu))*(I2-1) - mu;
 *   S00 = a + b*C11; S01 = -(b*C01); S11 = a + b*C00. */
static void membrane_tension(int law, double mu, double C, double C00, double C01, double C11,
                             double *S00, double *S01, double *S11)
{
    double I1 = C00 + C11;
    double I2 = C00 * C11 - C01 * C01;
    if (law == 0) {
        double q = mu / (I2 * I2);
        *S00 = mu - q * C11;
        *S01 = q * C01;
        *S11 = mu - q * C00;
    } else {
        double a = mu * ((I1 - 2.0) + 1.0);
        double b = (0.5 * (C * mu)) * (I2 - 1.0) - mu;
        *S00 = a + b * C11;
        *S01 = -(b * C01);
        *S11 = a + b * C00;
    }
}

/* Membrane strain energy density W-hat (Eqs. neo-Hookena, Skalak). */
static double membrane_w(int law, double mu, double C, double C00, double C01, double C11)
{
    double I1 = C00 + C11;
    double I2 = C00 * C11 - C01 * C01;
    if (law == 0)
        return 0.5 * mu * (I1 + 1.0 / I2 - 3.0);
    double i1 = I1 - 2.0, i2 = I2 - 1.0;
    return 0.5 * mu * (0.5 * i1 * i1 + i1 - i2) + C * mu / 8.0 * i2 * i2;
}

/* Elastic nodal forces of a membrane (Eq. FEM_Membrane):
 *   F_k = -A0 P-hat grad N_k,  P-hat = Fh S-hat (3x2, current 3D x reference 2D,
 * i.e. the in-plane force already rotated to 3D). Per triangle, in order:
 *   P[i][j] = Fh[i][0]*S[0][j] + Fh[i][1]*S[1][j];
 *   fb[i] = -(A0*(P[i][0]*m00 + P[i][1]*m01)); fc[i] = -(A0*(P[i][0]*m10 + P[i][1]*m11));
 *   fa[i] = -(fb[i] + fc[i]).
 * Triangles in ascending order, F[node] = F[node] + f. F is overwritten
 * (starts at 0). x: current positions (N,3). */
void ifo_membrane_forces(int law, double mu, double C, int nn, int nt, const int *tri,
                         const double *Dminv, const double *A0, const double *x, double *F)
{
    memset(F, 0, sizeof(double) * 3 * (size_t)nn);
    for (int e = 0; e < nt; ++e) {
        int ia = tri[3 * e], ib = tri[3 * e + 1], ic = tri[3 * e + 2];
        const double *m = Dminv + 4 * e;
        double Fh[3][2], C00, C01, C11, S00, S01, S11;
        membrane_kinematics(x + 3 * ia, x + 3 * ib, x + 3 * ic, m, Fh, &C00, &C01, &C11);
        membrane_tension(law, mu, C, C00, C01, C11, &S00, &S01, &S11);
        double fa[3], fb[3], fc[3];
        for (int i = 0; i < 3; ++i) {
            double P0 = Fh[i][0] * S00 + Fh[i][1] * S01;
            double P1 = Fh[i][0] * S01 + Fh[i][1] * S11;
            fb[i] = -(A0[e] * (P0 * m[0] + P1 * m[1]));
            fc[i] = -(A0[e] * (P0 * m[2] + P1 * m[3]));
            fa[i] = -(fb[i] + fc[i]);
        }
        for (int i = 0; i < 3; ++i) {
            F[3 * ia + i] = F[3 * ia + i] + fa[i];
            F[3 * ib + i] = F[3 * ib + i] + fb[i];
            F[3 * ic + i] = F[3 * ic + i] + fc[i];
        }
    }
}

/* Total membrane elastic energy E = sum_e A0_e W-hat(C-hat_e). */
double ifo_membrane_energy(int law, double mu, double C, int nt, const int *tri,
                           const double *Dminv, const double *A0, const double *x)
{
    double E = 0.0;
    for (int e = 0; e < nt; ++e) {
        double Fh[3][2], C00, C01, C11;
        membrane_kinematics(x + 3 * tri[3 * e], x + 3 * tri[3 * e + 1], x + 3 * tri[3 * e + 2],
                            Dminv + 4 * e, Fh, &C00, &C01, &C11);
        E += A0[e] * membrane_w(law, mu, C, C00, C01, C11);
    }
    return E;
}

/* Hessian-vector product of the membrane elastic energy,
 * Hw = d/de [-F(x + e w)] at e = 0, by the analytic directional derivative:
 *   dFh = dDs Dm^-1, dC = dFh^T Fh + Fh^T dFh, dI1 = tr dC,
 *   dI2 = dC00 C11 + C00 dC11 - 2 C01 dC01,
 *   NH:     S = mu (I - adj(C)/I2^2)  => dS = -mu (adj(dC)/I2^2 - 2 adj(C) dI2/I2^3)
 *   Skalak: S = mu (I1' + 1) I + (muD/2 I2' - mu) adj(C)
 *           => dS = mu dI1 I + muD/2 dI2 adj(C) + (muD/2 I2' - mu) adj(dC)
 *   dP = dFh S + Fh dS, df_k = -A0 dP grad N_k, Hw = -df. */
void ifo_membrane_hvp(int law, double mu, double C, int nn, int nt, const int *tri,
                      const double *Dminv, const double *A0, const double *x, const double *w,
                      double *Hw)
{
    memset(Hw, 0, sizeof(double) * 3 * (size_t)nn);
    for (int e = 0; e < nt; ++e) {
        int id[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
        const double *m = Dminv + 4 * e;
        double Fh[3][2], C00, C01, C11;
        membrane_kinematics(x + 3 * id[0], x + 3 * id[1], x + 3 * id[2], m, Fh, &C00, &C01, &C11);
        double dF[3][2];
        for (int i = 0; i < 3; ++i) {
            double d1 = w[3 * id[1] + i] - w[3 * id[0] + i];
            double d2 = w[3 * id[2] + i] - w[3 * id[0] + i];
            dF[i][0] = d1 * m[0] + d2 * m[2];
            dF[i][1] = d1 * m[1] + d2 * m[3];
        }
        double dC00 = 0, dC01 = 0, dC11 = 0;
        for (int i = 0; i < 3; ++i) {
            dC00 += 2.0 * dF[i][0] * Fh[i][0];
            dC11 += 2.0 * dF[i][1] * Fh[i][1];
            dC01 += dF[i][0] * Fh[i][1] + Fh[i][0] * dF[i][1];
        }
        double I1 = C00 + C11, I2 = C00 * C11 - C01 * C01;
        double dI1 = dC00 + dC11, dI2 = dC00 * C11 + C00 * dC11 - 2.0 * C01 * dC01;
        double S00, S01, S11, dS00, dS01, dS11;
        membrane_tension(law, mu, C, C00, C01, C11, &S00, &S01, &S11);
        if (law == 0) {
            double i2 = 1.0 / (I2 * I2), i3 = 2.0 * dI2 / (I2 * I2 * I2);
            dS00 = -mu * (dC11 * i2 - C11 * i3);
            dS11 = -mu * (dC00 * i2 - C00 * i3);
            dS01 = mu * (dC01 * i2 - C01 * i3);
        } else {
            double muD = C * mu;
            double b = 0.5 * muD * (I2 - 1.0) - mu, db = 0.5 * muD * dI2;
            dS00 = mu * dI1 + db * C11 + b * dC11;
            dS11 = mu * dI1 + db * C00 + b * dC00;
            dS01 = -(db * C01 + b * dC01);
        }
        (void)I1;
        double df[3][3];
        for (int i = 0; i < 3; ++i) {
            double P0 = dF[i][0] * S00 + dF[i][1] * S01 + Fh[i][0] * dS00 + Fh[i][1] * dS01;
            double P1 = dF[i][0] * S01 + dF[i][1] * S11 + Fh[i][0] * dS01 + Fh[i][1] * dS11;
            df[1][i] = -(A0[e] * (P0 * m[0] + P1 * m[1]));
            df[2][i] = -(A0[e] * (P0 * m[2] + P1 * m[3]));
            df[0][i] = -(df[1][i] + df[2][i]);
        }
        for (int v = 0; v < 3; ++v)
            for (int i = 0; i < 3; ++i)
                Hw[3 * id[v] + i] -= df[v][i];
    }
}

/* ================================================================== */
/* Solids (4-node tetrahedra)                                         */
/* ================================================================== */

static double det3(const double M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
         - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
         + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* inverse by the adjugate: inv[i][j] = cof[j][i] / det. */
static void inv3(const double M[3][3], double det, double R[3][3])
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

/* Reference data of every tet: Dm = [X1-X0, X2-X0, X3-X0] (columns),  */
/* V0 = det(Dm)/6, and Dm^-1 whose rows 0..2 are grad N_1..N_3 (grad   */
/* N_0 = -(sum)). Dminv layout per tet: row-major 3x3.                 */
void ifo_tet_reference(int ne, const int *tet, const double *X, double *Dminv, double *V0)
{
    for (int e = 0; e < ne; ++e) {
        const double *X0 = X + 3 * tet[4 * e];
        double Dm[3][3], R[3][3];
        for (int c = 0; c < 3; ++c) {
            const double *Xc = X + 3 * tet[4 * e + 1 + c];
            for (int i = 0; i < 3; ++i)
                Dm[i][c] = Xc[i] - X0[i];
        }
        double det = det3(Dm);
        inv3(Dm, det, R);
        for (int i = 0; i < 9; ++i)
            Dminv[9 * e + i] = R[i / 3][i % 3];
        V0[e] = det / 6.0;
    }
}

/* F = Ds Dm^-1 = sum_k x_k (x) grad N_k (Sec. Numerical Implementation). */
static void tet_defgrad(const double *x, const int *t, const double *Mi, double F[3][3])
{
    const double *x0 = x + 3 * t[0];
    double Ds[3][3];
    for (int c = 0; c < 3; ++c) {
        const double *xc = x + 3 * t[1 + c];
        for (int i = 0; i < 3; ++i)
            Ds[i][c] = xc[i] - x0[i];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            F[i][j] = (Ds[i][0] * Mi[0 * 3 + j] + Ds[i][1] * Mi[1 * 3 + j]) + Ds[i][2] * Mi[2 * 3 + j];
}

/* Second Piola-Kirchhoff stress of the discrete compressible neo-Hookean
 * solid, S = lambda/2 (J^2 - 1) C^-1 + mu (I - C^-1), C^-1 = F^-1 F^-T:
 *   J = det F; Finv = adj(F)/J; Cinv[i][j] = (Finv[i][0]*Finv[j][0] +
 *   Finv[i][1]*Finv[j][1]) + Finv[i][2]*Finv[j][2]; a = (0.5*lam)*(J*J - 1);
 *   S[i][j] = a*Cinv[i][j] + mu*(delta_ij - Cinv[i][j]). Returns J. */
static double tet_stress(double lam, double mu, const double F[3][3], double S[3][3],
                         double Cinv[3][3], double Finv[3][3])
{
    double J = det3(F);
    inv3(F, J, Finv);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Cinv[i][j] = (Finv[i][0] * Finv[j][0] + Finv[i][1] * Finv[j][1]) + Finv[i][2] * Finv[j][2];
    double a = (0.5 * lam) * (J * J - 1.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            S[i][j] = a * Cinv[i][j] + mu * ((i == j ? 1.0 : 0.0) - Cinv[i][j]);
    return J;
}

/* Elastic nodal forces of a solid (Eq. FEM, elastic part):
 *   P = F S: P[i][j] = (F[i][0]*S[0][j] + F[i][1]*S[1][j]) + F[i][2]*S[2][j];
 *   f_k[i] = -(V0*((P[i][0]*M[k][0] + P[i][1]*M[k][1]) + P[i][2]*M[k][2])), k = 1..3
 *   (M = Dm^-1, rows = grad N_k); f_0[i] = -((f_1[i] + f_2[i]) + f_3[i]).
 * Tets ascending, F[node] = F[node] + f. Returns the number of tets with J <= 0. */
int ifo_tet_forces(double lam, double mu, int nn, int ne, const int *tet, const double *Dminv,
                   const double *V0, const double *x, double *Fout)
{
    int inverted = 0;
    memset(Fout, 0, sizeof(double) * 3 * (size_t)nn);
    for (int e = 0; e < ne; ++e) {
        const int *t = tet + 4 * e;
        const double *Mi = Dminv + 9 * e;
        double F[3][3], S[3][3], Ci[3][3], Fi[3][3], P[3][3];
        tet_defgrad(x, t, Mi, F);
        double J = tet_stress(lam, mu, F, S, Ci, Fi);
        if (!(J > 0.0))
            ++inverted;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                P[i][j] = (F[i][0] * S[0][j] + F[i][1] * S[1][j]) + F[i][2] * S[2][j];
        double f[4][3];
        for (int k = 1; k <= 3; ++k)
            for (int i = 0; i < 3; ++i) {
                const double *g = Mi + 3 * (k - 1);
                f[k][i] = -(V0[e] * ((P[i][0] * g[0] + P[i][1] * g[1]) + P[i][2] * g[2]));
            }
        for (int i = 0; i < 3; ++i)
            f[0][i] = -((f[1][i] + f[2][i]) + f[3][i]);
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 3; ++i)
                Fout[3 * t[k] + i] = Fout[3 * t[k] + i] + f[k][i];
    }
    return inverted;
}

/* Fluid-stress nodal forces inside a solid (Sec. "Governing Equations": */
/* F^IB = -int (P^s - P^{f,N} - P^{f,P}) grad N_k, so the fluid parts     */
/* enter with a plus sign). Per tet, on the reference configuration:     */
/*   F = Ds Dm^-1, J = det F, Fi = F^-1 (tet_defgrad, inv3);              */
/*   G = Du Dm^-1 = sum_k u_k (x) grad N_k (nodal velocities u);           */
/*   Lv[i][j] = (G[i][0]*Fi[0][j] + G[i][1]*Fi[1][j]) + G[i][2]*Fi[2][j]   */
/*             (velocity gradient du_i/dx_j);                              */
/*   E[i][j] = Lv[i][j] + Lv[j][i];                                        */
/*   PN[i][j] = (eta*J) * ((E[i][0]*Fi[j][0] + E[i][1]*Fi[j][1])           */
/*              + E[i][2]*Fi[j][2])   (eta J (grad u + grad u^T) F^-T);    */
/*   Cb[i][j] = (((c_0 + c_1) + c_2) + c_3) * 0.25, c_k = C_k[i][j] - d_ij */
/*   (the printed sum of (C_k - I)/4 over the four nodes);                 */
/*   PP[i][j] = (J*cp) * ((Cb[i][0]*Fi[j][0] + Cb[i][1]*Fi[j][1])          */
/*              + Cb[i][2]*Fi[j][2]),  cp = (eta*(1 - beta))/lambda;        */
/*   P = PN + PP;  f_k[i] = V0*((P[i][0]*M[k][0] + P[i][1]*M[k][1])         */
/*              + P[i][2]*M[k][2]) (k = 1..3), f_0[i] = -((f_1 + f_2) + f_3). */
/* C: (N, 6) per node in the order xx, yy, zz, xy, xz, yz, or NULL (no    */
/* polymer term). Tets ascending, Fout[node] = Fout[node] + f, from 0.    */
void ifo_tet_fluid_forces(double eta, double beta, double lambda, int nn, int ne, const int *tet,
                          const double *Dminv, const double *V0, const double *x, const double *u,
                          const double *C, double *Fout)
{
    memset(Fout, 0, sizeof(double) * 3 * (size_t)nn);
    const double cp = (eta * (1.0 - beta)) / lambda;
    static const int sym[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    for (int e = 0; e < ne; ++e) {
        const int *t = tet + 4 * e;
        const double *Mi = Dminv + 9 * e;
        double F[3][3], G[3][3], Fi[3][3], Lv[3][3], E[3][3], P[3][3];
        tet_defgrad(x, t, Mi, F);
        tet_defgrad(u, t, Mi, G);
        const double J = det3(F);
        inv3(F, J, Fi);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Lv[i][j] = (G[i][0] * Fi[0][j] + G[i][1] * Fi[1][j]) + G[i][2] * Fi[2][j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                E[i][j] = Lv[i][j] + Lv[j][i];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                P[i][j] = (eta * J) * ((E[i][0] * Fi[j][0] + E[i][1] * Fi[j][1]) + E[i][2] * Fi[j][2]);
        if (C) {
            double Cb[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double dij = i == j ? 1.0 : 0.0;
                    double acc = C[6 * t[0] + sym[i][j]] - dij;
                    for (int k = 1; k < 4; ++k)
                        acc = acc + (C[6 * t[k] + sym[i][j]] - dij);
                    Cb[i][j] = acc * 0.25;
                }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    P[i][j] = P[i][j]
                              + (J * cp) * ((Cb[i][0] * Fi[j][0] + Cb[i][1] * Fi[j][1]) + Cb[i][2] * Fi[j][2]);
        }
        double f[4][3];
        for (int k = 1; k <= 3; ++k)
            for (int i = 0; i < 3; ++i) {
                const double *g = Mi + 3 * (k - 1);
                f[k][i] = V0[e] * ((P[i][0] * g[0] + P[i][1] * g[1]) + P[i][2] * g[2]);
            }
        for (int i = 0; i < 3; ++i)
            f[0][i] = -((f[1][i] + f[2][i]) + f[3][i]);
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 3; ++i)
                Fout[3 * t[k] + i] = Fout[3 * t[k] + i] + f[k][i];
    }
}

/* Strain energy density of the compressible neo-Hookean solid:
 * W = lam/4 (I3 - 1) - (lam/2 + mu) ln(I3^(1/2)) + mu/2 (I1 - 3). */
double ifo_tet_energy(double lam, double mu, int ne, const int *tet, const double *Dminv,
                      const double *V0, const double *x)
{
    double E = 0.0;
    for (int e = 0; e < ne; ++e) {
        double F[3][3];
        tet_defgrad(x, tet + 4 * e, Dminv + 9 * e, F);
        double I1 = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                I1 += F[i][j] * F[i][j];
        double J = det3(F);
        double I3 = J * J;
        E += V0[e] * (0.25 * lam * (I3 - 1.0) - (0.5 * lam + mu) * log(sqrt(I3)) + 0.5 * mu * (I1 - 3.0));
    }
    return E;
}

/* Hessian-vector product of the solid elastic energy, Hw = -dF[w]:
 *   dF = dDs Dm^-1, dJ = J tr(F^-1 dF), dC = dF^T F + F^T dF,
 *   dC^-1 = -C^-1 dC C^-1, dS = lam J dJ C^-1 + (lam/2 (J^2-1) - mu) dC^-1,
 *   dP = dF S + F dS, df_k = -V0 dP grad N_k. */
void ifo_tet_hvp(double lam, double mu, int nn, int ne, const int *tet, const double *Dminv,
                 const double *V0, const double *x, const double *w, double *Hw)
{
    memset(Hw, 0, sizeof(double) * 3 * (size_t)nn);
    for (int e = 0; e < ne; ++e) {
        const int *t = tet + 4 * e;
        const double *Mi = Dminv + 9 * e;
        double F[3][3], S[3][3], Ci[3][3], Fi[3][3], dF[3][3];
        tet_defgrad(x, t, Mi, F);
        tet_defgrad(w, t, Mi, dF);
        double J = tet_stress(lam, mu, F, S, Ci, Fi);
        double tr = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k)
                tr += Fi[i][k] * dF[k][i];
        double dJ = J * tr;
        double dC[3][3], T[3][3], dCi[3][3], dS[3][3], dP[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    s += dF[k][i] * F[k][j] + F[k][i] * dF[k][j];
                dC[i][j] = s;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    s += Ci[i][k] * dC[k][j];
                T[i][j] = s;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    s += T[i][k] * Ci[k][j];
                dCi[i][j] = -s;
            }
        double a = 0.5 * lam * (J * J - 1.0) - mu;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                dS[i][j] = lam * J * dJ * Ci[i][j] + a * dCi[i][j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    s += dF[i][k] * S[k][j] + F[i][k] * dS[k][j];
                dP[i][j] = s;
            }
        double df[4][3];
        for (int k = 1; k <= 3; ++k)
            for (int i = 0; i < 3; ++i) {
                const double *g = Mi + 3 * (k - 1);
                df[k][i] = -(V0[e] * (dP[i][0] * g[0] + dP[i][1] * g[1] + dP[i][2] * g[2]));
            }
        for (int i = 0; i < 3; ++i)
            df[0][i] = -(df[1][i] + df[2][i] + df[3][i]);
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 3; ++i)
                Hw[3 * t[k] + i] -= df[k][i];
    }
}

/* ================================================================== */
/* Helfrich bending (membranes)                                       */
/* ================================================================== */

static void sub3(const double *a, const double *b, double *r)
{
    r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double *a, const double *b, double *r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* Discrete curvature quantities at every vertex (Meyer, Desbrun,
 * Schroeder & Barr 2003), from a plain loop over triangles:
 *   K_i   = 1/(2 A_i) sum_j (cot a_ij + cot b_ij)(x_i - x_j)   (= 2 kH n)
 *   A_i   mixed Voronoi area (Voronoi region for non-obtuse triangles,
 *           area/2 at an obtuse corner, area/4 at the other two corners)
 *   n_i   unit area-weighted normal of the incident faces (outward)
 *   kH_i  = K_i . n_i / 2   (positive 1/R on a sphere)
 *   kG_i  = (2 pi - sum of corner angles at i) / A_i
 * Arrays sized nn (n: 3 nn). Corner angles use atan2(|u x v|, u . v). */
void ifo_curvatures(int nn, int nt, const int *tri, const double *x, double *A, double *nrm,
                    double *kH, double *kG, double *Kvec)
{
    double *ang = (double *)calloc((size_t)nn, sizeof(double));
    for (int i = 0; i < nn; ++i) {
        A[i] = 0.0; kH[i] = 0.0; kG[i] = 0.0;
        for (int a = 0; a < 3; ++a) { nrm[3 * i + a] = 0.0; Kvec[3 * i + a] = 0.0; }
    }
    for (int e = 0; e < nt; ++e) {
        const int v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
        double fn[3], e1[3], e2[3];
        sub3(x + 3 * v[1], x + 3 * v[0], e1);
        sub3(x + 3 * v[2], x + 3 * v[0], e2);
        cross3(e1, e2, fn);
        double area = 0.5 * sqrt(dot3(fn, fn));
        double th[3], cot[3];
        for (int c = 0; c < 3; ++c) {
            const double *p = x + 3 * v[c], *q = x + 3 * v[(c + 1) % 3], *r = x + 3 * v[(c + 2) % 3];
            double u[3], w[3], cr[3];
            sub3(q, p, u);
            sub3(r, p, w);
            cross3(u, w, cr);
            double cl = sqrt(dot3(cr, cr)), dp = dot3(u, w);
            th[c] = atan2(cl, dp);
            cot[c] = dp / cl;
        }
        for (int c = 0; c < 3; ++c) {
            int i = v[c], j = v[(c + 1) % 3], k = v[(c + 2) % 3];
            /* edge (i,j) is opposite corner k, edge (i,k) opposite corner j */
            double eij[3], eik[3];
            sub3(x + 3 * i, x + 3 * j, eij);
            sub3(x + 3 * i, x + 3 * k, eik);
            double cj = cot[(c + 1) % 3], ck = cot[(c + 2) % 3];
            for (int a = 0; a < 3; ++a)
                Kvec[3 * i + a] += ck * eij[a] + cj * eik[a];
            double Ai;
            int obtuse = th[0] > 0.5 * IFO_PI || th[1] > 0.5 * IFO_PI || th[2] > 0.5 * IFO_PI;
            if (!obtuse)
                Ai = (ck * dot3(eij, eij) + cj * dot3(eik, eik)) / 8.0;
            else if (th[c] > 0.5 * IFO_PI)
                Ai = area / 2.0;
            else
                Ai = area / 4.0;
            A[i] += Ai;
            ang[i] += th[c];
            for (int a = 0; a < 3; ++a)
                nrm[3 * i + a] += fn[a];
        }
    }
    for (int i = 0; i < nn; ++i) {
        double nl = sqrt(dot3(nrm + 3 * i, nrm + 3 * i));
        for (int a = 0; a < 3; ++a) {
            nrm[3 * i + a] /= nl;
            Kvec[3 * i + a] /= 2.0 * A[i];
        }
        kH[i] = 0.5 * dot3(Kvec + 3 * i, nrm + 3 * i);
        kG[i] = (2.0 * IFO_PI - ang[i]) / A[i];
    }
    free(ang);
}

/* Helfrich bending force (the paper's F_be, with the Canham-Helfrich
 * energy of Eq. Bending_Energy), at every vertex:
 *   F_k = 2 kb [ Lap_s(kH - kH0) + 2 (kH - kH0)(kH^2 - kG + kH0 kH) ] n_k A_k
 * with kH0 = -c0/2 and the cotangent Laplace-Beltrami operator
 *   Lap_s g (x_i) = 1/(2 A_i) sum_j (cot a_ij + cot b_ij)(g_j - g_i).
 * F is overwritten. */
void ifo_bending_forces(double kb, double c0, int nn, int nt, const int *tri, const double *x,
                        double *F)
{
    double *A = (double *)malloc(sizeof(double) * nn), *kH = (double *)malloc(sizeof(double) * nn),
           *kG = (double *)malloc(sizeof(double) * nn), *n = (double *)malloc(sizeof(double) * 3 * nn),
           *K = (double *)malloc(sizeof(double) * 3 * nn), *lap = (double *)calloc((size_t)nn, sizeof(double));
    ifo_curvatures(nn, nt, tri, x, A, n, kH, kG, K);
    double kH0 = -0.5 * c0;
    for (int e = 0; e < nt; ++e) {
        const int v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
        double cot[3];
        for (int c = 0; c < 3; ++c) {
            double u[3], w[3], cr[3];
            sub3(x + 3 * v[(c + 1) % 3], x + 3 * v[c], u);
            sub3(x + 3 * v[(c + 2) % 3], x + 3 * v[c], w);
            cross3(u, w, cr);
            cot[c] = dot3(u, w) / sqrt(dot3(cr, cr));
        }
        for (int c = 0; c < 3; ++c) {
            int i = v[c], j = v[(c + 1) % 3], k = v[(c + 2) % 3];
            lap[i] += cot[(c + 2) % 3] * ((kH[j] - kH0) - (kH[i] - kH0))
                    + cot[(c + 1) % 3] * ((kH[k] - kH0) - (kH[i] - kH0));
        }
    }
    for (int i = 0; i < nn; ++i) {
        double L = lap[i] / (2.0 * A[i]);
        double dh = kH[i] - kH0;
        double mag = 2.0 * kb * (L + 2.0 * dh * (kH[i] * kH[i] - kG[i] + kH0 * kH[i])) * A[i];
        for (int a = 0; a < 3; ++a)
            F[3 * i + a] = mag * n[3 * i + a];
    }
    free(A); free(kH); free(kG); free(n); free(K); free(lap);
}

/* Discrete Helfrich energy E_B = sum_i A_i kb/2 (2 kH_i + c0)^2. */
double ifo_bending_energy(double kb, double c0, int nn, int nt, const int *tri, const double *x)
{
    double *A = (double *)malloc(sizeof(double) * nn), *kH = (double *)malloc(sizeof(double) * nn),
           *kG = (double *)malloc(sizeof(double) * nn), *n = (double *)malloc(sizeof(double) * 3 * nn),
           *K = (double *)malloc(sizeof(double) * 3 * nn);
    ifo_curvatures(nn, nt, tri, x, A, n, kH, kG, K);
    double E = 0.0;
    for (int i = 0; i < nn; ++i) {
        double t = 2.0 * kH[i] + c0;
        E += A[i] * 0.5 * kb * t * t;
    }
    free(A); free(kH); free(kG); free(n); free(K);
    return E;
}

/* Polyhedron volume of a closed triangulated surface (Sec. Conservation
 * of Volume for Membranes): V = 1/18 sum_faces [x1.(x2 x x3) + x2.(x3 x x1)
 * + x3.(x1 x x2)]. */
double ifo_volume(int nt, const int *tri, const double *x)
{
    double V = 0.0;
    for (int e = 0; e < nt; ++e) {
        const double *a = x + 3 * tri[3 * e], *b = x + 3 * tri[3 * e + 1], *c = x + 3 * tri[3 * e + 2];
        double t1[3], t2[3], t3[3];
        cross3(b, c, t1);
        cross3(c, a, t2);
        cross3(a, b, t3);
        V += dot3(a, t1) + dot3(b, t2) + dot3(c, t3);
    }
    return V / 18.0;
}

/* Volume of a solid in its current configuration: the sum of its tets'
 * signed volumes det(Ds)/6, Ds = [x1-x0, x2-x0, x3-x0], tets ascending. */
double ifo_tet_volume(int ne, const int *tet, const double *x)
{
    double V = 0.0;
    for (int e = 0; e < ne; ++e) {
        const int *t = tet + 4 * e;
        double Ds[3][3];
        for (int c = 0; c < 3; ++c)
            for (int i = 0; i < 3; ++i)
                Ds[i][c] = x[3 * t[1 + c] + i] - x[3 * t[0] + i];
        V = V + det3(Ds) / 6.0;
    }
    return V;
}

/* Adams-Bashforth position update (Eq. Bashforth_eqn):
 * x = x + dt*(1.5*v - 0.5*vp), componentwise, in place. */
void ifo_ab2(int n3, double *x, const double *v, const double *vp, double dt)
{
    for (int i = 0; i < n3; ++i)
        x[i] = x[i] + dt * (1.5 * v[i] - 0.5 * vp[i]);
}

/* Sum over faces (a, b, c) of the three cyclic triple products
 * p_a.(q_b x r_c) + p_b.(q_c x r_a) + p_c.(q_a x r_b), faces ascending. */
static double cyclic_triple_sum(int nt, const int *tri, const double *p, const double *q, const double *r)
{
    double s = 0.0;
    for (int e = 0; e < nt; ++e) {
        const int a = tri[3 * e], b = tri[3 * e + 1], c = tri[3 * e + 2];
        double t1[3], t2[3], t3[3];
        cross3(q + 3 * b, r + 3 * c, t1);
        cross3(q + 3 * c, r + 3 * a, t2);
        cross3(q + 3 * a, r + 3 * b, t3);
        s += dot3(p + 3 * a, t1) + dot3(p + 3 * b, t2) + dot3(p + 3 * c, t3);
    }
    return s;
}

/* Volume conservation of a closed membrane (Sec. "Conservation of Volume
 * for Membranes", after Mendez et al. 2014): the smallest displacement
 * that restores the volume V0 is dx_I = Lambda alpha_I with
 *   alpha_I = -(1/12) sum_{faces with I} x_{I2} x x_{I3} (the face's other
 *   two nodes in cyclic order), accumulated over faces ascending, then
 *   scaled by -1/12;
 * Lambda the root of A L^3 + B L^2 + C L + D = 0 with the paper's
 *   A = (1/18) sum [alpha . (alpha x alpha)] (cyclic),
 *   B = (1/6)  sum [x . (alpha x alpha)] (cyclic),
 *   C = (1/6)  sum [alpha . (x x x)] (cyclic),
 *   D = V(x) - V0.
 * The root taken is the one Newton's method reaches from Lambda = 0
 * (the small correction): L = L - f/f', f = ((A L + B) L + C) L + D,
 * f' = (3 A L + 2 B) L + C, until |step| <= 1e-15 max(1, |L|) (at most
 * 100 steps). Then x_I = x_I + Lambda alpha_I. alpha: (nn, 3) scratch.
 * Returns the Newton steps taken, or -1 if f' vanished or it did not converge. */
int ifo_volume_correction(int nn, int nt, const int *tri, double *x, double V0, double *alpha,
                          double *lambda_out)
{
    memset(alpha, 0, sizeof(double) * 3 * (size_t)nn);
    for (int e = 0; e < nt; ++e) {
        const int a = tri[3 * e], b = tri[3 * e + 1], c = tri[3 * e + 2];
        double t[3];
        cross3(x + 3 * b, x + 3 * c, t);
        for (int i = 0; i < 3; ++i)
            alpha[3 * a + i] = alpha[3 * a + i] + t[i];
        cross3(x + 3 * c, x + 3 * a, t);
        for (int i = 0; i < 3; ++i)
            alpha[3 * b + i] = alpha[3 * b + i] + t[i];
        cross3(x + 3 * a, x + 3 * b, t);
        for (int i = 0; i < 3; ++i)
            alpha[3 * c + i] = alpha[3 * c + i] + t[i];
    }
    for (int i = 0; i < 3 * nn; ++i)
        alpha[i] = alpha[i] * (-1.0 / 12.0);
    const double A = cyclic_triple_sum(nt, tri, alpha, alpha, alpha) / 18.0;
    const double B = cyclic_triple_sum(nt, tri, x, alpha, alpha) / 6.0;
    const double C = cyclic_triple_sum(nt, tri, alpha, x, x) / 6.0;
    const double D = cyclic_triple_sum(nt, tri, x, x, x) / 18.0 - V0;
    double L = 0.0;
    int it = 0, ok = 0;
    for (; it < 100; ++it) {
        const double f = ((A * L + B) * L + C) * L + D;
        const double fp = (3.0 * A * L + 2.0 * B) * L + C;
        if (fp == 0.0)
            break;
        const double step = f / fp;
        L = L - step;
        if (fabs(step) <= 1e-15 * fmax(1.0, fabs(L))) {
            ok = 1;
            ++it;
            break;
        }
    }
    for (int i = 0; i < 3 * nn; ++i)
        x[i] = x[i] + L * alpha[i];
    if (lambda_out)
        *lambda_out = L;
    return ok ? it : -1;
}
