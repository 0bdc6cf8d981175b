"""Pins of the oracle's transfer operators (spreading S*, interpolation S).

Each test checks the oracle against something other than itself: closed-form
kernel values, the kernels' moment conditions, a brute-force evaluation over
every grid node, exact reproduction of linear fields, the adjoint identity
and second-order convergence on smooth fields.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
import ifem_workloads as W
from ifem_workloads.fields import eval_modes, fourier_modes, mac_offset, sample_on_mac

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_peskin_closed_form_values():
    g = json.load(open(os.path.join(GOLD, "peskin4_values.json")))
    for p in g["points"]:
        assert O.phi4(p["r"]) == pytest.approx(p["phi"], abs=2e-16)


def test_peskin_moments_random_shifts():
    rng = np.random.default_rng(7)
    for s in rng.uniform(-50, 50, 2000):
        i0 = math.floor(s) - 1
        r = [s - (i0 + m) for m in range(4)]
        ph = [O.phi4(x) for x in r]
        assert sum(ph) == pytest.approx(1.0, abs=4e-16)
        assert sum(ri * p for ri, p in zip(r, ph)) == pytest.approx(0.0, abs=1e-15)
        assert sum(p * p for p in ph) == pytest.approx(0.375, abs=4e-16)


def test_peskin_continuity_and_support():
    eps = 1e-12
    for r in (1.0, 2.0):
        assert O.phi4(r - eps) == pytest.approx(O.phi4(r + eps), abs=1e-6)
    assert O.phi4(2.0 + 1e-9) == 0.0


def test_mls_spline_branches():
    # cubic-spline weight read as 2/3 - 4r^2 + 4r^3 on r <= 1/2 (continuous at 1/2)
    assert O.mls_w(0.0) == pytest.approx(2.0 / 3.0, abs=1e-16)
    assert O.mls_w(0.5) == pytest.approx(1.0 / 6.0, abs=1e-16)
    assert O.mls_w(0.5 + 1e-12) == pytest.approx(1.0 / 6.0, abs=1e-11)
    assert O.mls_w(1.0) == pytest.approx(0.0, abs=1e-15)
    assert O.mls_w(1.2) == 0.0


def _mls_bruteforce(s, support):
    """phi = e1^T (P^T W P)^-1 P^T W by an SVD least-squares solve."""
    c = np.floor(np.asarray(s) + 0.5).astype(int)
    pts = []
    for kz in range(-1, 2):
        for jy in range(-1, 2):
            for ix in range(-1, 2):
                pts.append(c + np.array([ix, jy, kz]))
    pts = np.array(pts, dtype=float)
    Y = pts - np.asarray(s)
    r = np.linalg.norm(Y, axis=1) / support
    Wt = np.where(r <= 0.5, 2 / 3 - 4 * r**2 + 4 * r**3,
                  np.where(r <= 1.0, 4 / 3 - 4 * r + 4 * r**2 - 4 / 3 * r**3, 0.0))
    # unshifted basis p(x) = (1, x) evaluated at the absolute lattice points
    P = np.concatenate([np.ones((27, 1)), pts], axis=1)
    sw = np.sqrt(Wt)
    Z, *_ = np.linalg.lstsq(sw[:, None] * P, np.diag(sw), rcond=None)
    p_k = np.concatenate([[1.0], s])
    return p_k @ Z


def test_mls_weights_vs_bruteforce_lstsq():
    rng = np.random.default_rng(3)
    for _ in range(200):
        s = rng.uniform(-3, 20, 3)
        base, w = O.mls_weights(s)
        ref = _mls_bruteforce(s, O.MLS_SUPPORT)
        np.testing.assert_allclose(w, ref, atol=1e-11, rtol=0)
        assert (base == np.floor(s + 0.5).astype(int) - 1).all()


def test_mls_linear_reproduction():
    rng = np.random.default_rng(4)
    for _ in range(200):
        s = rng.uniform(0, 30, 3)
        base, w = O.mls_weights(s)
        pts = np.array([[base[0] + a, base[1] + b, base[2] + c]
                        for c in range(3) for b in range(3) for a in range(3)], dtype=float)
        assert w.sum() == pytest.approx(1.0, abs=1e-13)
        np.testing.assert_allclose(w @ (pts - s), 0.0, atol=1e-12)


def _brute_spread_one(xk, Fk, n, L, kernel):
    """Spread one node by looping over EVERY grid node with the minimum-image distance."""
    h = L / n
    f = np.zeros((3, n, n, n))
    idx = np.arange(n)
    for d in range(3):
        o = mac_offset(d)
        pos = [(idx + o[a]) * h for a in range(3)]
        rel = [((pos[a] - xk[a] + 0.5 * L) % L - 0.5 * L) / h for a in range(3)]
        if kernel == O.KERNEL_PESKIN4:
            ph = [np.array([O.phi4(r) for r in rel[a]]) for a in range(3)]
            w = ph[2][:, None, None] * ph[1][None, :, None] * ph[0][None, None, :]
        else:
            s = np.array([xk[a] / h - o[a] for a in range(3)])
            base, ww = O.mls_weights(s)
            w = np.zeros((n, n, n))
            J = 0
            for c in range(3):
                for b in range(3):
                    for a in range(3):
                        w[(base[2] + c) % n, (base[1] + b) % n, (base[0] + a) % n] = ww[J]
                        J += 1
        f[d] = w * Fk[d] / h**3
    return f


@pytest.mark.parametrize("kernel", [O.KERNEL_PESKIN4, O.KERNEL_MLS27])
def test_spread_single_node_bruteforce_with_wrap(kernel):
    rng = np.random.default_rng(11)
    n, L = 12, 1.3
    for xk in ([0.02, 1.27, 0.6], rng.uniform(0, L, 3), [L - 1e-9, 0.0, 0.5 * L]):
        xk = np.asarray(xk, dtype=float)
        Fk = rng.standard_normal(3)
        f = O.spread(xk[None], Fk[None], n, L, kernel)
        ref = _brute_spread_one(xk, Fk, n, L, kernel)
        np.testing.assert_allclose(f, ref, atol=1e-13 * np.abs(ref).max(), rtol=0)


@pytest.mark.parametrize("kernel", [O.KERNEL_PESKIN4, O.KERNEL_MLS27])
def test_interp_reproduces_linear_fields(kernel):
    # u_d(p) = a_d + b_d . p sampled on each MAC lattice, node far from the wrap
    rng = np.random.default_rng(5)
    n, L = 32, 1.0
    h = L / n
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    u = np.zeros((3, n, n, n))
    idx = np.arange(n)
    for d in range(3):
        o = mac_offset(d)
        Z, Y, X = np.meshgrid((idx + o[2]) * h, (idx + o[1]) * h, (idx + o[0]) * h, indexing="ij")
        u[d] = a[d] + B[d, 0] * X + B[d, 1] * Y + B[d, 2] * Z
    x = rng.uniform(0.3, 0.7, (50, 3))
    v = O.interp(x, u, n, L, kernel)
    np.testing.assert_allclose(v, a[None] + x @ B.T, atol=1e-13, rtol=0)


@pytest.mark.parametrize("kernel", [O.KERNEL_PESKIN4, O.KERNEL_MLS27])
def test_adjoint_identity(kernel):
    """<interp u, F> = h^3 <u, spread F> (density form) and = <u, spread F> (force form)."""
    wl = W.make("C1")
    rng = np.random.default_rng(9)
    n, L = wl.boxes[0].n, wl.boxes[0].L
    x = wl.origins_per_node() + wl.x_local_all()
    F = rng.standard_normal(x.shape)
    u = rng.standard_normal((3, n, n, n))
    lhs = np.sum(O.interp(x, u, n, L, kernel) * F)
    fd = O.spread(x, F, n, L, kernel, density=True)
    ff = O.spread(x, F, n, L, kernel, density=False)
    assert lhs == pytest.approx((L / n) ** 3 * np.sum(u * fd), rel=1e-13)
    assert lhs == pytest.approx(np.sum(u * ff), rel=1e-13)


@pytest.mark.parametrize("kernel", [O.KERNEL_PESKIN4, O.KERNEL_MLS27])
def test_spread_conserves_force_and_torque(kernel):
    wl = W.make("C1")
    n, L = wl.boxes[0].n, wl.boxes[0].L
    h = L / n
    x = wl.origins_per_node() + wl.x_local_all()
    F = np.random.default_rng(1).standard_normal(x.shape)
    f = O.spread(x, F, n, L, kernel)
    tot = np.array([f[d].sum() for d in range(3)]) * h**3
    np.testing.assert_allclose(tot, F.sum(0), atol=1e-11)
    idx = np.arange(n)
    torque = np.zeros(3)
    for d in range(3):
        o = mac_offset(d)
        Z, Y, X = np.meshgrid((idx + o[2]) * h, (idx + o[1]) * h, (idx + o[0]) * h, indexing="ij")
        P = np.stack([X, Y, Z], -1)
        fv = np.zeros(P.shape)
        fv[..., d] = f[d]
        torque += np.cross(P, fv).reshape(-1, 3).sum(0) * h**3
    np.testing.assert_allclose(torque, np.cross(x, F).sum(0), atol=1e-10)


@pytest.mark.parametrize("kernel", [O.KERNEL_PESKIN4, O.KERNEL_MLS27])
def test_interp_second_order_convergence(kernel):
    rng = np.random.default_rng(21)
    modes = fourier_modes(rng, n_modes=4, kmax=2)
    x = rng.uniform(0, 1, (200, 3))
    exact = eval_modes(modes, x, 1.0)
    errs = []
    for n in (32, 64, 128):
        u = sample_on_mac(modes, n, 1.0)
        errs.append(np.abs(O.interp(x, u, n, 1.0, kernel) - exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.7, (errs, rates)


# ------------------------------------------------ conservation sums (FP64)
def _sums_workload(parts):
    """A workload holding only what the per-particle sums read: one template
    per particle (its node count), instances with the given local positions."""
    tm = [W.Template(kind="solid", X=np.zeros((len(x), 3)), elems=np.zeros((0, 4), np.int32), law="nh")
          for x, _ in parts]
    inst = [W.Instance(tmpl=i, box=0, origin=np.asarray(org, dtype=np.float64), x_local=np.asarray(x, np.float64))
            for i, (x, org) in enumerate(parts)]
    return W.Workload(name="sums", templates=tm, instances=inst, boxes=[W.Box(16)], u=[], seed=0)


def test_reductions_closed_form_octahedron():
    """Force and torque balance sums (Sec. "Numerical Implementation"): six
    nodes at c +- a e_i carry F = w x (x - c) + G. About the centroid the
    torque is (tr M - M) w with M = sum r r^T = 2 a^2 I, i.e. 4 a^2 w; the
    uniform part G adds nothing (sum r = 0) and sum F = 6 G. A torque taken
    about the origin (6 c x G more), a swapped cross product (sign) or a
    dropped term fails here."""
    a, c = 0.375, np.array([0.3, -1.25, 2.5])
    w, G = np.array([0.5, -2.0, 1.5]), np.array([-0.25, 0.75, 1.0])
    r = np.concatenate([a * np.eye(3), -a * np.eye(3)])
    x = c + r
    F = np.cross(w, r) + G
    v = np.arange(18, dtype=np.float64).reshape(6, 3) * 0.125
    wl = _sums_workload([(x, [7.0, 0.0, -3.0])])
    red = O.reductions(wl, x, F, v)[0]
    np.testing.assert_array_equal(red[0:3], c)
    np.testing.assert_allclose(red[3:6], 6 * G, rtol=0, atol=1e-15)
    np.testing.assert_allclose(red[6:9], 4 * a * a * w, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(red[9:12], v.sum(0))


def test_reductions_rigid_rotation_field_about_offset_centroid():
    """Random cloud made symmetric about an offset centre c (so the centroid
    is c exactly), F = w x (x - c) + G: the torque about the centroid equals
    (tr(M) I - M) w, M the second-moment matrix of the offsets, and is
    independent of G; several particles are summed separately."""
    rng = np.random.default_rng(11)
    parts, exp = [], []
    for p in range(3):
        h = rng.standard_normal((40, 3))
        r = np.concatenate([h, -h])
        c = rng.uniform(-5, 5, 3)
        w, G = rng.standard_normal(3), rng.standard_normal(3)
        M = r.T @ r
        exp.append((c, len(r) * G, (np.trace(M) * np.eye(3) - M) @ w))
        parts.append((c + r, np.cross(w, r) + G))
    wl = _sums_workload([(x, rng.uniform(-1, 1, 3)) for x, _ in parts])
    xl = np.concatenate([x for x, _ in parts])
    F = np.concatenate([f for _, f in parts])
    red = O.reductions(wl, xl, F, np.zeros_like(xl))
    for p, (c, sF, tq) in enumerate(exp):
        np.testing.assert_allclose(red[p, 0:3], c, rtol=0, atol=1e-13)
        np.testing.assert_allclose(red[p, 3:6], sF, rtol=0, atol=1e-12)
        np.testing.assert_allclose(red[p, 6:9], tq, rtol=1e-12, atol=1e-11)
        assert np.all(red[p, 9:12] == 0.0)


def test_reductions_sums_are_correctly_rounded():
    """The FP64 sums are correctly rounded: 1e16 + 1 - 1e16 ... in any order
    gives the exact sum (a plain left-to-right loop would lose the 1s)."""
    x = np.zeros((4, 3))
    F = np.array([[1e16, 1.0, 3.0], [1.0, -1e16, 3.0], [-1e16, 1e16, 3.0], [1.0, 1.0, 3.0]])
    wl = _sums_workload([(x, [0.0, 0.0, 0.0])])
    red = O.reductions(wl, x, F, F)[0]
    np.testing.assert_array_equal(red[3:6], [2.0, 2.0, 12.0])
    np.testing.assert_array_equal(red[9:12], [2.0, 2.0, 12.0])
