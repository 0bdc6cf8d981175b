"""CUDA path vs the FP64 oracle for the Lagrangian update: the Adams-Bashforth
position update (Eq. Bashforth_eqn), per-particle volumes and the membrane
volume correction (Sec. "Conservation of Volume for Membranes").

AB2 in FP64 is bit-identical to the oracle. Volumes and the correction's
sums are FP64 block trees in both precisions, so they agree with the
oracle's sequential sums to a few ulps of the summed magnitudes (1e-12
relative); after the correction the volumes equal the targets to that
precision (FP64) or to the FP32 rounding of the corrected positions.
"""
import numpy as np
import pytest

import ifem_workloads as W
from oracle import oracle as O
from tests._helpers import rounded_workload

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
_cache = {}


def wl(name):
    if name not in _cache:
        _cache[name] = W.make(name)
    return _cache[name]


def _oracle_volumes(w, x):
    off = w.node_offsets()
    out = []
    for i, inst in enumerate(w.instances):
        tm = w.templates[inst.tmpl]
        xi = x[off[i]:off[i + 1]]
        out.append(O.volume(tm.elems, xi) if tm.kind == "membrane" else O.tet_volume(tm.elems, xi))
    return np.array(out)


def _run(w, precision, fn):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(w, precision=precision)
    try:
        return fn(cp, I, torch)
    finally:
        cp.close()


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_ab2_update(precision):
    w = wl("C2")
    if precision == FP32:
        w = rounded_workload(w, np.float32)
    rng = np.random.default_rng(1)
    dt_ = np.float32 if precision == FP32 else np.float64
    v = rng.standard_normal((w.n_nodes, 3)).astype(dt_).astype(np.float64)
    vp = rng.standard_normal((w.n_nodes, 3)).astype(dt_).astype(np.float64)
    dt = 0.0375

    def fn(cp, I, torch):
        x = cp.nodes_to_device(w.x_local_all())
        I.ifem_ab2_update(cp.ctx, cp.batch, x, cp.nodes_to_device(v), cp.nodes_to_device(vp), dt)
        torch.cuda.synchronize()
        return cp.nodes_to_host(x)

    g = _run(w, precision, fn)
    o = O.ab2(w.x_local_all(), v, vp, dt)
    if precision == FP64:
        assert np.array_equal(g, o)
    else:
        np.testing.assert_allclose(g, o, rtol=0, atol=4e-7 * np.abs(o).max())


@pytest.mark.parametrize("case", ["C2", "C3", "C4"])
@pytest.mark.parametrize("precision", [FP32, FP64])
def test_volumes(case, precision):
    w = wl(case)
    if precision == FP32:
        w = rounded_workload(w, np.float32)

    def fn(cp, I, torch):
        x = cp.nodes_to_device(w.x_local_all())
        vol = torch.empty(len(w.instances), dtype=torch.float64, device=cp.device)
        I.ifem_volumes(cp.ctx, cp.batch, x, vol)
        return vol.cpu().numpy()

    g = _run(w, precision, fn)
    o = _oracle_volumes(w, w.x_local_all())
    np.testing.assert_allclose(g, o, rtol=1e-12, atol=0)


def _perturbed(w, seed):
    rng = np.random.default_rng(seed)
    x = w.x_local_all()
    off = w.node_offsets()
    out = x.copy()
    for i in range(len(w.instances)):
        s = slice(off[i], off[i + 1])
        out[s] = x[s] * rng.uniform(0.997, 1.003) + 1e-3 * rng.standard_normal(x[s].shape)
    return out


@pytest.mark.parametrize("case", ["C2", "C4"])
@pytest.mark.parametrize("precision", [FP32, FP64])
def test_volume_correction(case, precision):
    w = wl(case)
    V0 = _oracle_volumes(w, w.x_local_all())
    xp = _perturbed(w, 2)
    if precision == FP32:
        xp = xp.astype(np.float32).astype(np.float64)

    def fn(cp, I, torch):
        x = cp.nodes_to_device(xp)
        V0d = torch.as_tensor(V0, dtype=torch.float64, device=cp.device)
        lam = torch.empty(len(w.instances), dtype=torch.float64, device=cp.device)
        I.ifem_volume_correct(cp.ctx, cp.batch, x, V0d, lam)
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        assert rc == 0, st
        return cp.nodes_to_host(x), lam.cpu().numpy()

    g, lam = _run(w, precision, fn)
    off = w.node_offsets()
    for i, inst in enumerate(w.instances):
        tm = w.templates[inst.tmpl]
        s = slice(off[i], off[i + 1])
        if tm.kind != "membrane":
            assert lam[i] == 0.0 and np.array_equal(g[s], xp[s])
            continue
        xo, _, lo = O.volume_correction(tm.elems, xp[s], V0[i])
        # FP32: alpha from FP32 edge vectors, so Lambda carries their rounding
        assert lam[i] == pytest.approx(lo, rel=1e-9 if precision == FP64 else 1e-5)
        scale = np.abs(xo).max()
        tol = 1e-12 if precision == FP64 else 2e-7
        np.testing.assert_allclose(g[s], xo, rtol=0, atol=tol * scale)
        vtol = 1e-11 if precision == FP64 else 2e-6
        assert O.volume(tm.elems, g[s]) == pytest.approx(V0[i], rel=vtol)


# ------------------------------------------------ indicator-function source
def _gpu_indicator(w, precision, kernel=0, scatter=0, flags=0):
    def fn(cp, I, torch):
        x = cp.nodes_to_device(w.x_local_all())
        G = cp.zeros_grid()
        I.ifem_indicator_source(cp.ctx, cp.batch, cp.grid, x, G, flags)
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        assert rc == 0, st
        return cp.grid_to_host(G)

    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(w, precision=precision, kernel=kernel, scatter=scatter)
    try:
        return fn(cp, I, torch)
    finally:
        cp.close()


@pytest.mark.parametrize("case", ["C2", "C4", "C5"])
@pytest.mark.parametrize("kernel", [0, 1])
def test_indicator_source_fp64(case, kernel):
    """n_k A_k comes from the vertex-ring evaluation of the bending operators,
    which associates the incident triangles' terms differently from the
    oracle's loop over triangles (last-bit differences, as for the bending
    force); the spread that follows is the bit-exact FP64 one. Bound: relative
    L2 1e-13."""
    w = wl(case)
    g = _gpu_indicator(w, FP64, kernel)
    o = O.indicator_source(w, kernel=kernel)
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(g, o)))
    den = np.sqrt(sum(np.sum(b ** 2) for b in o))
    assert num / den < 1e-13


@pytest.mark.parametrize("scatter", [0, 1])
@pytest.mark.parametrize("flags", [0, 1])
def test_indicator_source_fp32(scatter, flags):
    w = rounded_workload(wl("C2"), np.float32)
    g = _gpu_indicator(w, FP32, scatter=scatter, flags=flags)
    o = O.indicator_source(w, density=not (flags & 1))
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(g, o)))
    den = np.sqrt(sum(np.sum(b ** 2) for b in o))
    assert num / den < 1e-5
