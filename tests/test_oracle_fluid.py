"""Pins of the oracle's fluid-stress terms inside solids and of the
cell-centred interpolation that feeds them (the Newtonian and polymer parts
of Eq. FEM, Sec. "Governing Equations"; interpolation of the conformation
tensor, Sec. "Interpolation Scheme").

Fluid-stress forces: zero for rigid motion (the symmetric velocity gradient
vanishes), zero polymer force for C = I, force and torque balance (the
nominal stresses come from symmetric Cauchy stresses, so a misplaced
transpose shows up as a torque), and the virtual work of a homogeneous
deformation against its closed form V_tot P : H. Interpolation: constant
and linear fields reproduced exactly, and a single point against a brute
force sum over every cell centre with minimum-image distances.
"""
import numpy as np
import pytest

from oracle import oracle as O
from ifem_workloads import meshes

ETA, BETA, LAM = 0.7, 0.3, 2.5
CP = ETA * (1.0 - BETA) / LAM


@pytest.fixture(scope="module")
def ball():
    X, tet = meshes.kuhn_ball(5, 1.0)
    return X, tet


def _deformed(X, seed, noise=0.03):
    rng = np.random.default_rng(seed)
    A = np.eye(3) + 0.15 * rng.standard_normal((3, 3))
    assert np.linalg.det(A) > 0.3
    return X @ A.T + noise * rng.standard_normal(X.shape), A


def _sym6(M):
    return np.array([M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]])


def test_rigid_motion_gives_no_newtonian_force(ball):
    X, tet = ball
    x, _ = _deformed(X, 1)
    rng = np.random.default_rng(2)
    a, w = rng.standard_normal(3), rng.standard_normal(3)
    u_rigid = a + np.cross(w, x)
    u_gen = rng.standard_normal(x.shape)
    F_rigid = O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u_rigid)
    F_gen = O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u_gen)
    assert np.abs(F_rigid).max() <= 1e-12 * np.abs(F_gen).max()


def test_identity_conformation_gives_no_polymer_force(ball):
    X, tet = ball
    x, _ = _deformed(X, 3)
    u = np.random.default_rng(4).standard_normal(x.shape)
    C = np.tile(_sym6(np.eye(3)), (x.shape[0], 1))
    assert np.array_equal(O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u, C),
                          O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u))


def test_force_and_torque_balance(ball):
    X, tet = ball
    x, _ = _deformed(X, 5)
    rng = np.random.default_rng(6)
    u = rng.standard_normal(x.shape)
    Q = rng.standard_normal((x.shape[0], 3, 3)) * 0.2
    C = np.array([_sym6(np.eye(3) + q @ q.T) for q in Q])
    F = O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u, C)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(0)).max() <= 1e-13 * scale
    assert np.abs(np.cross(x, F).sum(0)).max() <= 1e-13 * scale * np.abs(x).max()


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_homogeneous_virtual_work_closed_form(ball, seed):
    """x = A X, u = G x, C_k = I + Q on every node: every element has the same
    P = eta J (G + G^T) A^-T + J cp Q A^-T, so sum_k F_k . (H X_k) = V_tot P : H."""
    X, tet = ball
    rng = np.random.default_rng(seed)
    A = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    G, H = rng.standard_normal((3, 3)), rng.standard_normal((3, 3))
    q = 0.3 * rng.standard_normal((3, 3))
    Q = q @ q.T
    x = X @ A.T
    u = x @ G.T
    C = np.tile(_sym6(np.eye(3) + Q), (x.shape[0], 1))
    _, V0 = O.tet_reference(tet, X)
    J = np.linalg.det(A)
    AinvT = np.linalg.inv(A).T
    P = ETA * J * (G + G.T) @ AinvT + J * CP * Q @ AinvT
    for C_arg, P_ref in ((None, ETA * J * (G + G.T) @ AinvT), (C, P)):
        F = O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u, C_arg)
        work = np.sum(F * (X @ H.T))
        expect = V0.sum() * np.sum(P_ref * H)
        assert work == pytest.approx(expect, rel=1e-11)


def test_linear_in_velocity_and_conformation(ball):
    X, tet = ball
    x, _ = _deformed(X, 10)
    rng = np.random.default_rng(11)
    u1, u2 = rng.standard_normal(x.shape), rng.standard_normal(x.shape)
    F1 = O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u1)
    F2 = O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, u2)
    F12 = O.tet_fluid_forces(ETA, BETA, LAM, tet, X, x, 2.0 * u1 - u2)
    np.testing.assert_allclose(F12, 2.0 * F1 - F2, atol=1e-12 * np.abs(F12).max())


# ------------------------------------------------------------ interpolation
def _cc_positions(n, L):
    h = L / n
    idx = np.arange(n)
    return (idx + 0.5) * h


@pytest.mark.parametrize("kernel", [O.KERNEL_PESKIN4, O.KERNEL_MLS27])
def test_cc_interp_reproduces_constant_and_linear_fields(kernel):
    n, L = 16, 1.0
    c = _cc_positions(n, L)
    Z, Y, Xg = np.meshgrid(c, c, c, indexing="ij")
    a, b = np.array([0.3, -1.2]), np.array([[0.7, -0.4, 1.1], [0.2, 0.5, -0.9]])
    field = np.stack([a[q] + b[q, 0] * Xg + b[q, 1] * Y + b[q, 2] * Z for q in range(2)])
    rng = np.random.default_rng(12)
    x = rng.uniform(0.3, 0.7, (50, 3))   # stencils do not wrap
    out = O.interp_cc(x, field, n, L, kernel)
    expect = a[None, :] + x @ b.T
    np.testing.assert_allclose(out, expect, atol=1e-13, rtol=0)
    const = O.interp_cc(rng.uniform(0, L, (50, 3)), np.full((1, n, n, n), 2.5), n, L, kernel)
    np.testing.assert_allclose(const, 2.5, atol=1e-14, rtol=0)


def test_cc_interp_single_point_bruteforce_with_wrap():
    n, L = 10, 1.7
    h = L / n
    rng = np.random.default_rng(13)
    field = rng.standard_normal((6, n, n, n))
    c = _cc_positions(n, L)
    for xk in ([0.01, 1.69, 0.8], rng.uniform(0, L, 3), [L - 1e-9, 0.0, 0.5 * L]):
        xk = np.asarray(xk, dtype=float)
        rel = [((c - xk[a] + 0.5 * L) % L - 0.5 * L) / h for a in range(3)]
        ph = [np.array([O.phi4(r) for r in rel[a]]) for a in range(3)]
        w = ph[2][:, None, None] * ph[1][None, :, None] * ph[0][None, None, :]
        ref = np.array([np.sum(w * field[q]) for q in range(6)])
        out = O.interp_cc(xk[None], field, n, L)[0]
        np.testing.assert_allclose(out, ref, atol=1e-13 * np.abs(field).max(), rtol=0)
