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
