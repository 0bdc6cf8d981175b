"""Pins of the oracle's Lagrangian force layer.

Membrane (neo-Hookean, Skalak), solid neo-Hookean tets, Helfrich bending and
their Hessian-vector products are checked against closed-form energies,
finite-difference gradients of the paper's energy densities, rigid-motion
invariance, momentum conservation and the polyhedron-volume formula.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
import ifem_workloads as W
from ifem_workloads import meshes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def W_nh(l1, l2, mu=1.0):
    return 0.5 * mu * (l1**2 + l2**2 + 1.0 / (l1**2 * l2**2) - 3.0)


def W_sk(l1, l2, mu=1.0, C=1.0):
    i1 = l1**2 + l2**2 - 2.0
    i2 = l1**2 * l2**2 - 1.0
    return 0.5 * mu * (0.5 * i1**2 + i1 - i2) + C * mu / 8.0 * i2**2


@pytest.mark.parametrize("law", ["nh", "skalak"])
@pytest.mark.parametrize("stretch", [(1.3, 1.0), (0.8, 1.0), (1.2, 1.2), (1.1, 0.7)])
def test_flat_triangle_closed_form_energy(law, stretch):
    rng = np.random.default_rng(0)
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.9, 0.0]])
    tri = np.array([[0, 1, 2]])
    l1, l2 = stretch
    # rotate the stretched triangle out of plane: energy is frame-indifferent
    R = meshes.random_rotation(rng)
    x = (X * np.array([l1, l2, 1.0])) @ R.T + rng.standard_normal(3)
    A0 = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
    Wc = W_nh(l1, l2) if law == "nh" else W_sk(l1, l2, C=3.0)
    E = O.membrane_energy(law, 1.0, 3.0, tri, X, x)
    assert E == pytest.approx(A0 * Wc, rel=1e-13)


@pytest.mark.parametrize("law", ["nh", "skalak"])
def test_icosphere_uniform_scale_equibiaxial(law):
    v, f = meshes.icosphere(3)
    X = 0.15 * v
    lam = 1.17
    Dminv, A0 = O.membrane_reference(f, X)
    E = O.membrane_energy(law, 1.0, 2.0, f, X, lam * X)
    Wc = W_nh(lam, lam) if law == "nh" else W_sk(lam, lam, C=2.0)
    assert E == pytest.approx(A0.sum() * Wc, rel=1e-12)
    # the restoring force of a uniform inflation points inward at every node
    F = O.membrane_forces(law, 1.0, 2.0, f, X, lam * X)
    radial = np.einsum("ij,ij->i", F, v)
    assert (radial < 0).all()
    # and the work of a uniform scaling equals -dE/dlam = -A0_tot dW/dlam
    dl = 1e-6
    Wp = W_nh(lam + dl, lam + dl) if law == "nh" else W_sk(lam + dl, lam + dl, C=2.0)
    Wm = W_nh(lam - dl, lam - dl) if law == "nh" else W_sk(lam - dl, lam - dl, C=2.0)
    assert np.sum(F * X) == pytest.approx(-A0.sum() * (Wp - Wm) / (2 * dl), rel=1e-7)


def W_solid(Fm, lam, mu):
    J = np.linalg.det(Fm)
    return 0.25 * lam * (J * J - 1) - (0.5 * lam + mu) * math.log(J) + 0.5 * mu * (np.sum(Fm * Fm) - 3)


def test_tet_ball_homogeneous_deformation():
    X, t = meshes.kuhn_ball(6, 1.0)
    rng = np.random.default_rng(2)
    Fm = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    assert np.linalg.det(Fm) > 0
    x = X @ Fm.T + rng.standard_normal(3)
    lam, mu = 9.0, 1.0
    Dminv, V0 = O.tet_reference(t, X)
    E = O.tet_energy(lam, mu, t, X, x)
    assert E == pytest.approx(V0.sum() * W_solid(Fm, lam, mu), rel=1e-12)
    F = O.tet_forces(lam, mu, t, X, x)
    surf = np.unique(np.concatenate([np.flatnonzero(np.abs(np.abs(X).max(1)) > 0) ]))
    # interior nodes: the ones strictly inside the [-1,1]^3 lattice before mapping
    m = 6
    g = np.arange(m)
    K, J, I = np.meshgrid(g, g, g, indexing="ij")
    interior = ((I > 0) & (I < m - 1) & (J > 0) & (J < m - 1) & (K > 0) & (K < m - 1)).ravel()
    assert interior.sum() == (m - 2) ** 3
    assert np.abs(F[interior]).max() < 1e-12 * np.abs(F).max()
    del surf


def _fd_grad(energy, x, eps):
    g = np.zeros_like(x)
    for i in range(x.shape[0]):
        for a in range(3):
            xp = x.copy(); xp[i, a] += eps
            xm = x.copy(); xm[i, a] -= eps
            g[i, a] = (energy(xp) - energy(xm)) / (2 * eps)
    return g


@pytest.mark.parametrize("law", ["nh", "skalak"])
def test_membrane_force_is_minus_energy_gradient(law):
    v, f = meshes.icosphere(1)
    rng = np.random.default_rng(12)
    X = v
    x = X @ (np.eye(3) + 0.15 * rng.standard_normal((3, 3))).T + 0.03 * rng.standard_normal(X.shape)
    ref = O.membrane_reference(f, X)
    C = 5.0
    F = O.membrane_forces(law, 1.3, C, f, X, x, ref=ref)
    g = _fd_grad(lambda y: O.membrane_energy(law, 1.3, C, f, X, y, ref=ref), x, 1e-6)
    assert np.abs(F + g).max() < 1e-7 * np.abs(F).max()


def test_tet_force_is_minus_energy_gradient():
    X, t = meshes.kuhn_ball(3, 1.0)
    rng = np.random.default_rng(13)
    x = X @ (np.eye(3) + 0.1 * rng.standard_normal((3, 3))).T + 0.02 * rng.standard_normal(X.shape)
    ref = O.tet_reference(t, X)
    F = O.tet_forces(50.0, 1.0, t, X, x, ref=ref)
    g = _fd_grad(lambda y: O.tet_energy(50.0, 1.0, t, X, y, ref=ref), x, 1e-6)
    assert np.abs(F + g).max() < 1e-7 * np.abs(F).max()


def _all_forces(tm, x):
    return O.template_forces(tm, x)


@pytest.mark.parametrize("cfg", ["C1", "C2", "C3"])
def test_rigid_motion_zero_and_covariant(cfg):
    wl = W.make(cfg)
    tm = wl.templates[0]
    rng = np.random.default_rng(31)
    R = meshes.random_rotation(rng)
    b = rng.standard_normal(3)
    # reference state moved rigidly: zero elastic force
    if tm.kind == "membrane":
        Fel = O.membrane_forces(tm.law, tm.mu, tm.C, tm.elems, tm.X, tm.X @ R.T + b)
    else:
        Fel = O.tet_forces(tm.lam, tm.mu, tm.elems, tm.X, tm.X @ R.T + b)
    assert np.abs(Fel).max() < 1e-11 * max(tm.mu, 1.0)
    # deformed state: F(Rx + b) = R F(x), including bending
    x = wl.instances[0].x_local
    F1 = _all_forces(tm, x)
    F2 = _all_forces(tm, x @ R.T + b)
    assert np.abs(F2 - F1 @ R.T).max() < 1e-10 * np.abs(F1).max()


@pytest.mark.parametrize("cfg", ["C1", "C3"])
def test_elastic_force_and_torque_balance(cfg):
    wl = W.make(cfg)
    tm = wl.templates[0]
    x = wl.instances[0].x_local
    F = _all_forces(tm, x)
    scale = np.abs(F).max() * len(x)
    assert np.abs(F.sum(0)).max() < 1e-13 * scale
    c = x.mean(0)
    assert np.abs(np.cross(x - c, F).sum(0)).max() < 1e-13 * scale * np.abs(x - c).max()


def test_polyhedron_volume_ellipsoidal_stretch():
    v, f = meshes.icosphere(3)
    X = 0.15 * v
    V0 = O.volume(f, X)
    # closed surface volume is exact for the polyhedron: a linear map scales it by det
    V1 = O.volume(f, X @ np.diag([1.2, 0.9, 0.9]).T + np.array([0.5, 0.5, 0.5]))
    assert V1 == pytest.approx(0.972 * V0, rel=1e-14)
    # and the polyhedron volume converges to the sphere volume under refinement
    v4, f4 = meshes.icosphere(4)
    assert abs(O.volume(f4, v4) - 4 / 3 * math.pi) < abs(O.volume(f, v) - 4 / 3 * math.pi)
    # divergence-theorem cross-check via tetrahedra to an interior point
    a, b, c = X[f[:, 0]], X[f[:, 1]], X[f[:, 2]]
    assert V0 == pytest.approx(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6, rel=1e-14)


@pytest.mark.parametrize("kind", ["nh", "skalak", "tet"])
def test_hvp_symmetric_and_matches_fd(kind):
    rng = np.random.default_rng(41)
    if kind == "tet":
        X, t = meshes.kuhn_ball(4, 1.0)
        x = X @ (np.eye(3) + 0.1 * rng.standard_normal((3, 3))).T
        ref = O.tet_reference(t, X)
        force = lambda y: O.tet_forces(9.0, 1.0, t, X, y, ref=ref)  # noqa: E731
        hvp = lambda y, w: O.tet_hvp(9.0, 1.0, t, X, y, w, ref=ref)  # noqa: E731
    else:
        v, f = meshes.icosphere(2)
        X = v
        x = X @ (np.eye(3) + 0.1 * rng.standard_normal((3, 3))).T
        ref = O.membrane_reference(f, X)
        force = lambda y: O.membrane_forces(kind, 1.0, 4.0, f, X, y, ref=ref)  # noqa: E731
        hvp = lambda y, w: O.membrane_hvp(kind, 1.0, 4.0, f, X, y, w, ref=ref)  # noqa: E731
    w = rng.standard_normal(x.shape)
    z = rng.standard_normal(x.shape)
    Hw, Hz = hvp(x, w), hvp(x, z)
    assert np.sum(z * Hw) == pytest.approx(np.sum(w * Hz), rel=1e-11)
    eps = 1e-6
    fd = -(force(x + eps * w) - force(x - eps * w)) / (2 * eps)
    assert np.abs(Hw - fd).max() < 1e-7 * np.abs(Hw).max()


def test_bending_vanishes_on_sphere_with_refinement():
    """On a sphere with c0 = 0, kH^2 = kG and Lap kH = 0: the discrete force tends to 0."""
    R = 1.0
    mags = []
    for lev in (2, 3, 4):
        v, f = meshes.icosphere(lev)
        Fb = O.bending_forces(1.0, f, R * v)
        cur = O.curvatures(f, R * v)
        # per-area force density relative to the scale 2 kb kH^3 of its two terms
        mags.append(np.abs(Fb / cur["A"][:, None]).max() / (2.0 / R**3))
        assert np.median(cur["kH"]) == pytest.approx(1.0 / R, rel=2e-2)
        assert np.median(cur["kG"]) == pytest.approx(1.0 / R**2, rel=2e-2)
        assert cur["A"].sum() == pytest.approx(4 * math.pi * R**2, rel=2e-2)
    assert mags[2] < mags[1] < mags[0]


def test_bending_force_matches_energy_variation_to_discretisation_order():
    """-sum F . dx against the FD change of the discrete Helfrich energy, on an
    ellipsoid (semi-axes 1, 0.8, 0.6) under a smooth perturbation. The force
    is not the exact gradient of the discrete energy, so the two agree to the
    discretisation order only: 0.82 % at icosphere level 3 and 0.22 % at
    level 4, shrinking about 4x per refinement (second order). The bounds sit
    just above those figures, so a missing factor or a dropped term in one of
    the force's terms fails."""
    rel = []
    for lev, bound in ((3, 0.012), (4, 0.004)):
        v, f = meshes.icosphere(lev)
        x = v @ np.diag([1.0, 0.8, 0.6]).T
        kb = 1.0
        # smooth normal-ish perturbation (low mode), well resolved by the mesh
        dx = (np.sin(2 * x[:, 0]) + np.cos(3 * x[:, 1]))[:, None] * v
        Fb = O.bending_forces(kb, f, x)
        eps = 1e-5
        dE = (O.bending_energy(kb, f, x + eps * dx) - O.bending_energy(kb, f, x - eps * dx)) / (2 * eps)
        work = -np.sum(Fb * dx)
        rel.append(abs(work / dE - 1.0))
        assert rel[-1] < bound, (lev, rel[-1])
    assert rel[1] < rel[0] / 3.0, rel


def test_bending_scale_invariance():
    """The Helfrich energy of Eq. Bending_Energy (c0 = 0) is scale invariant, so F(l x) = F(x)/l."""
    wl = W.make("C2")
    tm = wl.templates[0]
    x = wl.instances[0].x_local
    F1 = O.bending_forces(tm.kb, tm.elems, x)
    F2 = O.bending_forces(tm.kb, tm.elems, 2.5 * x)
    np.testing.assert_allclose(F2, F1 / 2.5, atol=1e-12 * np.abs(F1).max())


def test_workload_constants_follow_paper():
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    from ifem_workloads import configs as C
    assert C.SKALAK_C == g["skalak_muD_over_mu"]["value"]
    assert C.PLT_LAMBDA_OVER_MU == g["solid_lambda_over_mu"]["value"]
    assert C.CA_PLT_OVER_CA_RBC == g["ca_platelet"]["value"]
    assert C.RP_OVER_D_RBC * 8.0 == pytest.approx(g["rbc_effective_radius_um"]["value"])
