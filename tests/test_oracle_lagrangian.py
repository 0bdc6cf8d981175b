"""Pins of the oracle's Lagrangian update layer: the Adams-Bashforth position
update (Eq. Bashforth_eqn), the current volume of solids, and the membrane
volume correction of Sec. "Conservation of Volume for Membranes".

AB2 is exact for velocities linear in time and converges at second order;
the solid volume scales with det A under x = A X; the corrected membrane has
exactly the target volume, its displacement directions are minus one half of
the volume gradient (central differences of the polyhedron volume), and a
membrane that already has the target volume is left untouched.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from ifem_workloads import meshes


def test_ab2_exact_for_linear_in_time_velocity():
    rng = np.random.default_rng(1)
    a, b, x0 = rng.standard_normal((3, 40, 3))
    dt = 0.013
    for n in range(1, 6):
        tn, tp = n * dt, (n - 1) * dt
        xn = x0 + a * tn + 0.5 * b * tn**2
        x1 = O.ab2(xn, a + b * tn, a + b * tp, dt)
        t1 = tn + dt
        np.testing.assert_allclose(x1, x0 + a * t1 + 0.5 * b * t1**2, rtol=0, atol=1e-14)


def test_ab2_second_order():
    def run(dt):
        x = np.array([[math.sin(dt)]])           # exact first step
        t = dt
        while t < 1.0 - 1e-12:
            x = O.ab2(x, np.array([[math.cos(t)]]), np.array([[math.cos(t - dt)]]), dt)
            t += dt
        return abs(x[0, 0] - math.sin(1.0))
    e1, e2 = run(1 / 40), run(1 / 80)
    assert 3.5 < e1 / e2 < 4.5


def test_tet_volume_scales_with_det():
    X, tet = meshes.kuhn_ball(6, 1.0)
    _, V0 = O.tet_reference(tet, X)
    V = O.tet_volume(tet, X)
    assert V == pytest.approx(V0.sum(), rel=1e-13)
    A = np.array([[1.2, 0.1, 0.0], [0.05, 0.9, 0.2], [0.0, -0.1, 1.1]])
    assert O.tet_volume(tet, X @ A.T) == pytest.approx(np.linalg.det(A) * V, rel=1e-13)


@pytest.fixture(scope="module")
def cell():
    X, tri = meshes.rbc_surface(3, 1.0)
    return np.asarray(X, dtype=float), np.asarray(tri)


def _perturbed(X, seed, scale):
    rng = np.random.default_rng(seed)
    return X * scale + 1e-3 * rng.standard_normal(X.shape) + np.array([0.3, -0.2, 0.1])


@pytest.mark.parametrize("scale", [0.999, 1.0004, 1.01])
def test_correction_restores_target_volume(cell, scale):
    X, tri = cell
    V0 = O.volume(tri, X)
    x = _perturbed(X, 2, scale)
    xc, alpha, lam = O.volume_correction(tri, x, V0)
    assert O.volume(tri, xc) == pytest.approx(V0, rel=1e-12)
    np.testing.assert_allclose(xc - x, lam * alpha, rtol=0, atol=1e-15 * np.abs(x).max())
    # the small root: close to the linearised estimate -D / C
    lin = -(O.volume(tri, x) - V0) / np.sum(alpha * (-2.0 * alpha))  # C = grad V . alpha = -2 |alpha|^2
    assert lam == pytest.approx(lin, rel=0.05)


def test_displacement_direction_is_volume_gradient(cell):
    X, tri = cell
    x = _perturbed(X, 3, 1.002)
    _, alpha, _ = O.volume_correction(tri, x, O.volume(tri, x) * 0.999)
    h = 1e-6
    rng = np.random.default_rng(4)
    for I in rng.choice(x.shape[0], 12, replace=False):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[I, a] += h
            xm[I, a] -= h
            g = (O.volume(tri, xp) - O.volume(tri, xm)) / (2 * h)
            assert alpha[I, a] == pytest.approx(-0.5 * g, rel=1e-6, abs=1e-9)


def test_no_correction_at_target_volume(cell):
    X, tri = cell
    x = _perturbed(X, 5, 1.0)
    xc, _, lam = O.volume_correction(tri, x, O.volume(tri, x))
    assert lam == 0.0 and np.array_equal(xc, x)


# ------------------------------------------------ indicator-function source
def test_mixed_areas_partition_the_surface(cell):
    """sum_k A_k equals the total triangle area (mixed Voronoi areas tile the surface)."""
    X, tri = cell
    x = _perturbed(X, 6, 1.0)
    e1 = x[tri[:, 1]] - x[tri[:, 0]]
    e2 = x[tri[:, 2]] - x[tri[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum()
    assert O.curvatures(tri, x)["A"].sum() == pytest.approx(area, rel=1e-13)


def test_area_normals_divergence_theorem_converges():
    """sum_k (n_k A_k) . x_k -> 3 V (divergence theorem) at second order on refined spheres,
    and sum_k n_k A_k -> 0 for the closed surface."""
    errs = []
    for level in (2, 3, 4):
        X, tri = meshes.icosphere(level)
        x = X * 0.8 + np.array([0.1, -0.3, 0.2])
        nA = O.area_normals(tri, x)
        V = O.volume(tri, x)
        errs.append(abs(np.sum(nA * x) - 3.0 * V) / (3.0 * V))
        assert np.abs(nA.sum(0)).max() <= 1e-12 * np.abs(nA).sum()
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0


def test_indicator_source_is_the_spread_of_area_normals():
    """Density form: the first moment sum_d h^3 sum_J G_d,J x_J,d of the source equals
    sum_k n_k A_k . x_k (the Peskin kernel reproduces linear functions; the cell does
    not touch the box faces), a non-zero quantity close to 3 V."""
    import ifem_workloads as W
    from ifem_workloads.fields import mac_offset
    w = W.make("C2")
    G = O.indicator_source(w)
    off = w.node_offsets()
    inst = w.instances[0]
    tm = w.templates[inst.tmpl]
    xl = w.x_local_all()[off[0]:off[1]]
    nA = O.area_normals(tm.elems, xl)
    xa = inst.origin[None, :] + xl
    bx = w.boxes[0]
    h = bx.L / bx.n
    idx = np.arange(bx.n)
    moment = 0.0
    for d in range(3):
        coord = (idx + mac_offset(d)[d]) * h
        shape = [1, 1, 1]
        shape[2 - d] = bx.n
        moment += h**3 * np.sum(G[0][d] * coord.reshape(shape))
    expect = np.sum(nA * xa)
    assert moment == pytest.approx(expect, rel=1e-12)
    assert expect == pytest.approx(3.0 * O.volume(tm.elems, xl), rel=0.02)
