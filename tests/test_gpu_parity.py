"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

FP64 (deterministic) mode: element forces, nodal sums, spreading and
interpolation must be bit-identical to the oracle; the bending force must
agree to 1e-13 relative L2 (the oracle sums the corner angles with one libm
atan2 each, the GPU takes the angle deficit from one CUDA atan2 of a complex
product per vertex, and the cotangents from one reciprocal of 2A per
triangle; the measured error is printed).
FP32 mode: relative L2 error against the oracle evaluated on the same
FP32-rounded inputs within 1e-5 (forces, spread field) and 1e-6 (interpolated
velocities).
"""
import numpy as np
import pytest

import ifem_workloads as W
from oracle import oracle as O
from tests._helpers import oracle_step, random_grid, rel_l2, rounded_workload, run_gpu_step

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
TOL_F, TOL_V, TOL_GRID = 1e-5, 1e-6, 1e-5
TOL_BEND64 = 1e-13

_cache = {}


def wl(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        _cache[key] = W.make(name, **kw)
    return _cache[key]


def no_bending(w):
    import dataclasses
    return dataclasses.replace(w, templates=[dataclasses.replace(t, kb=0.0) for t in w.templates])


# ------------------------------------------------------------------ FP64
@pytest.mark.parametrize("case", ["C1-nh", "C1-skalak", "C2-elastic", "C3"])
@pytest.mark.parametrize("kernel", [0, 1])
def test_fp64_step_bit_exact(case, kernel):
    if case.startswith("C1"):
        w = wl("C1", law=case.split("-")[1])
    elif case == "C2-elastic":
        w = no_bending(wl("C2"))
    else:
        w = wl("C3")
    f0 = random_grid(w, seed=3)
    g = run_gpu_step(w, FP64, kernel=kernel, f0=f0)
    o = oracle_step(w, kernel=kernel, f0=f0)
    assert g["rc"] == 0, g["stats"]
    assert np.array_equal(g["F"], o["F"]), np.abs(g["F"] - o["F"]).max()
    assert np.array_equal(g["v"], o["v"]), np.abs(g["v"] - o["v"]).max()
    for gb, ob in zip(g["f"], o["f"]):
        assert np.array_equal(gb, ob), np.abs(gb - ob).max()


@pytest.mark.parametrize("kernel", [0, 1])
def test_fp64_bending_step(kernel):
    w = wl("C2")
    g = run_gpu_step(w, FP64, kernel=kernel)
    o = oracle_step(w, kernel=kernel)
    eF, ef = rel_l2(g["F"], o["F"]), rel_l2(g["f"][0], o["f"][0])
    print(f"C2 FP64 bending step, kernel {kernel}: rel L2 F {eF:.3e}, spread field {ef:.3e}")
    assert eF < TOL_BEND64, eF
    assert rel_l2(g["v"], o["v"]) == 0.0
    assert ef < TOL_BEND64, ef


def test_fp64_deterministic_across_runs():
    w = wl("C2")
    a = run_gpu_step(w, FP64)
    b = run_gpu_step(w, FP64)
    for k in ("F", "v"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["f"][0], b["f"][0])
    assert np.array_equal(a["red"], b["red"])


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_fp64_spread_modes(flags):
    """force form (1), overwrite (2) and both (3) against the oracle."""
    w = wl("C1")
    f0 = random_grid(w, seed=5)
    g = run_gpu_step(w, FP64, flags=flags, f0=f0)
    o = oracle_step(w, density=not (flags & 1), f0=None if flags & 2 else f0)
    assert np.array_equal(g["f"][0], o["f"][0])


# ------------------------------------------------------------------ FP32
@pytest.mark.parametrize("case", ["C1", "C2", "C3"])
@pytest.mark.parametrize("scatter", [0, 1])
@pytest.mark.parametrize("kernel", [0, 1])
def test_fp32_step_tolerances(case, scatter, kernel):
    w = rounded_workload(wl(case), np.float32)
    g = run_gpu_step(w, FP32, kernel=kernel, scatter=scatter)
    o = oracle_step(w, kernel=kernel)
    assert g["rc"] == 0, g["stats"]
    eF, ev, ef = rel_l2(g["F"], o["F"]), rel_l2(g["v"], o["v"]), rel_l2(g["f"][0], o["f"][0])
    assert eF < TOL_F and ev < TOL_V and ef < TOL_GRID, (eF, ev, ef)


def test_fp32_det_scatter_reproducible():
    w = wl("C2")
    a = run_gpu_step(w, FP32, scatter=0)
    b = run_gpu_step(w, FP32, scatter=0)
    assert np.array_equal(a["F"], b["F"])
    assert np.array_equal(a["v"], b["v"])


# ------------------------------------------------------------------ reductions
@pytest.mark.parametrize("precision", [FP32, FP64])
def test_reductions(precision):
    w = wl("C2")
    if precision == FP32:
        w = rounded_workload(w, np.float32)
    g = run_gpu_step(w, precision)
    red = g["red"]
    ni = len(w.instances)
    xl = w.x_local_all()
    exp = O.reductions(w, xl, g["F"], g["v"])
    got = red[: 12 * ni].reshape(ni, 12)
    scale = np.array([np.abs(xl).max()] * 3 + [np.abs(g["F"]).max() * len(xl)] * 3
                     + [np.abs(g["F"]).max() * np.abs(xl).max() * len(xl)] * 3 + [np.abs(g["v"]).max() * len(xl)] * 3)
    assert np.all(np.abs(got - exp) <= 1e-13 * scale + 1e-300)
    # grid side: h^3 sum of the spread values equals the total nodal force
    box = red[12 * ni: 12 * ni + 3]
    tol = 1e-11 if precision == FP64 else 1e-5
    np.testing.assert_allclose(box, exp[0, 3:6], atol=tol * np.abs(g["F"]).sum(0).max())


# ------------------------------------------------------------------ HVP
def _hvp_gpu(w, precision, wvec):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(w, precision=precision)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        wd = cp.nodes_to_device(wvec)
        Hw = cp.empty_nodes()
        I.ifem_force_hvp(cp.ctx, cp.batch, x, wd, Hw)
        torch.cuda.synchronize()
        return cp.nodes_to_host(Hw)
    finally:
        cp.close()


@pytest.mark.parametrize("case", ["C1-nh", "C1-skalak", "C3"])
@pytest.mark.parametrize("precision", [FP32, FP64])
def test_hvp_vs_oracle(case, precision):
    w = wl("C1", law=case.split("-")[1]) if case.startswith("C1") else wl("C3")
    if precision == FP32:
        w = rounded_workload(w, np.float32)
    tm = w.templates[0]
    wvec = np.random.default_rng(2).standard_normal((w.n_nodes, 3))
    if precision == FP32:
        wvec = wvec.astype(np.float32).astype(np.float64)
    g = _hvp_gpu(w, precision, wvec)
    x = w.x_local_all()
    if tm.kind == "membrane":
        o = O.membrane_hvp(tm.law, tm.mu, tm.C, tm.elems, tm.X, x, wvec)
    else:
        o = O.tet_hvp(tm.lam, tm.mu, tm.elems, tm.X, x, wvec)
    e = rel_l2(g, o)
    print(f"{case} HVP {'FP64' if precision == FP64 else 'FP32'}: rel L2 {e:.3e} against the oracle")
    # FP32: the force tolerance (the HVP is the same element arithmetic, differentiated)
    assert e < (1e-12 if precision == FP64 else TOL_F), e


# ------------------------------------------------------------------ edge cases
def test_particle_across_periodic_boundary_and_outside_box():
    """Origins near the box faces and outside [0, L): wrap must match the oracle."""
    import dataclasses
    w = wl("C1")
    for org in ([0.999, 0.0005, 0.5], [1.3, -0.2, 5.0]):
        ww = dataclasses.replace(w, instances=[dataclasses.replace(w.instances[0], origin=np.array(org))])
        g = run_gpu_step(ww, FP64)
        o = oracle_step(ww)
        assert np.array_equal(g["v"], o["v"])
        assert np.array_equal(g["f"][0], o["f"][0])


def test_small_box_ragged_tiles():
    """A 9^3 box (single ragged tile per axis at t = 8) and a 27^3 box (ragged last tile)."""
    import dataclasses
    base = wl("C1")
    for n, scale in ((9, 0.02), (27, 0.06)):
        tm = dataclasses.replace(base.templates[0], X=base.templates[0].X * scale / 0.15)
        inst = dataclasses.replace(base.instances[0], x_local=base.instances[0].x_local * scale / 0.15)
        u = np.random.default_rng(n).standard_normal((3, n, n, n))
        ww = dataclasses.replace(base, templates=[tm], instances=[inst], boxes=[W.Box(n, 1.0)], u=[u])
        for tile in (6, 8):
            g = run_gpu_step(ww, FP64, tile=tile)
            o = oracle_step(ww)
            assert np.array_equal(g["f"][0], o["f"][0])
            assert np.array_equal(g["v"], o["v"])


@pytest.mark.parametrize("n,tile", [(9, 6), (9, 8), (27, 8), (27, 12), (36, 12), (40, 16)])
def test_fp32_atomic_small_boxes(n, tile):
    """FP32 ATOMIC Peskin spread (own-tile nodes, halo added with L2 reductions):
    boxes whose halo wraps onto the tile itself (n = 9), ragged last tiles
    (27, 40: scalar flush) and quad-aligned rows (36, 40 with t = 12, 16)."""
    import dataclasses
    base = wl("C1")
    scale = 0.15 * min(1.0, n / 40)
    tm = dataclasses.replace(base.templates[0], X=base.templates[0].X * scale / 0.15)
    inst = dataclasses.replace(base.instances[0], x_local=base.instances[0].x_local * scale / 0.15,
                               origin=np.array([0.93, 0.02, 0.5]))
    u = np.random.default_rng(n).standard_normal((3, n, n, n))
    ww = rounded_workload(dataclasses.replace(base, templates=[tm], instances=[inst], boxes=[W.Box(n, 1.0)], u=[u]),
                          np.float32)
    g = run_gpu_step(ww, FP32, scatter=1, tile=tile)
    o = oracle_step(ww)
    assert g["rc"] == 0, g["stats"]
    assert rel_l2(g["F"], o["F"]) < TOL_F
    assert rel_l2(g["f"][0], o["f"][0]) < TOL_GRID
    assert rel_l2(g["v"], o["v"]) < TOL_V


@pytest.mark.parametrize("org", [[0.999, 0.0005, 0.5], [1.3, -0.2, 5.0]])
def test_fp32_atomic_particle_across_boundary_and_outside_box(org):
    """FP32 ATOMIC Peskin path (one-pass binning, fused staged transfer) with
    the particle across the periodic faces and with its origin outside [0, L)
    (cells below 0 and beyond 2n, wrapped in 32-bit arithmetic)."""
    import dataclasses
    w = wl("C1")
    ww = rounded_workload(dataclasses.replace(w, instances=[dataclasses.replace(w.instances[0], origin=np.array(org))]),
                          np.float32)
    g = run_gpu_step(ww, FP32, scatter=1)
    o = oracle_step(ww)
    assert g["rc"] == 0, g["stats"]
    eF, ev, ef = rel_l2(g["F"], o["F"]), rel_l2(g["v"], o["v"]), rel_l2(g["f"][0], o["f"][0])
    assert eF < TOL_F and ev < TOL_V and ef < TOL_GRID, (eF, ev, ef)


@pytest.mark.parametrize("case", ["C2", "C3", "small"])
def test_fp32_fused_gather_kernel(case, monkeypatch):
    """The fused transfer that gathers velocities through L1
    (spread_halo_kernel<true>, selected by IFEM_TRANSFER=halo when the context
    is created) against the oracle, as the default staged kernel is."""
    import dataclasses
    monkeypatch.setenv("IFEM_TRANSFER", "halo")
    if case == "small":
        base = wl("C1")
        n = 27
        tm = dataclasses.replace(base.templates[0], X=base.templates[0].X * 0.06 / 0.15)
        inst = dataclasses.replace(base.instances[0], x_local=base.instances[0].x_local * 0.06 / 0.15,
                                   origin=np.array([0.93, 0.02, 0.5]))
        u = np.random.default_rng(n).standard_normal((3, n, n, n))
        w = dataclasses.replace(base, templates=[tm], instances=[inst], boxes=[W.Box(n, 1.0)], u=[u])
    else:
        w = wl(case)
    w = rounded_workload(w, np.float32)
    g = run_gpu_step(w, FP32, scatter=1, tile=8 if case == "small" else 0)
    o = oracle_step(w)
    assert g["rc"] == 0, g["stats"]
    eF, ev, ef = rel_l2(g["F"], o["F"]), rel_l2(g["v"], o["v"]), rel_l2(g["f"][0], o["f"][0])
    assert eF < TOL_F and ev < TOL_V and ef < TOL_GRID, (eF, ev, ef)


def test_empty_batch():
    import dataclasses
    w = dataclasses.replace(wl("C1"), instances=[])
    f0 = random_grid(w, seed=1)
    g = run_gpu_step(w, FP64, f0=f0)
    assert g["rc"] == 0
    assert np.array_equal(g["f"][0], f0[0])


def test_nan_position_reports_domain_error():
    import dataclasses
    w = wl("C1")
    x = w.instances[0].x_local.copy()
    x[5, 1] = np.nan
    ww = dataclasses.replace(w, instances=[dataclasses.replace(w.instances[0], x_local=x)])
    g = run_gpu_step(ww, FP32)
    assert g["rc"] == -6 and g["stats"]["domain_errors"] >= 1


def test_inverted_tet_is_counted_and_still_evaluated():
    import dataclasses
    w = wl("C3")
    tm = w.templates[0]
    x = w.instances[0].x_local.copy()
    t0 = tm.elems[100]
    x[t0[0]] = x[t0[1]] + 2.0 * (x[t0[0]] - x[t0[1]]) * -1.0
    ww = dataclasses.replace(w, instances=[dataclasses.replace(w.instances[0], x_local=x)])
    g = run_gpu_step(ww, FP64)
    F, ninv = O.tet_forces(tm.lam, tm.mu, tm.elems, tm.X, x, return_inverted=True)
    assert ninv >= 1
    assert g["rc"] == -5 and g["stats"]["inverted_elements"] == ninv
    assert np.array_equal(g["F"], F)


def test_autotuned_tile_matches_fixed_tile():
    import torch
    from paper_1807_08219_gb300 import ifem as I
    w = rounded_workload(wl("C2"), np.float32)
    cp = I.Coupler(w, precision=FP32, tile=0)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        I.ifem_prepare(cp.ctx, cp.batch, x)
        assert I.ifem_ctx_tile(cp.ctx) in (8, 12, 16)
        u = cp.grid_to_device(w.u)
        F, v, f = cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
        I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, None)
        I.ifem_sync_status(cp.ctx)
        g = {"F": cp.nodes_to_host(F), "v": cp.nodes_to_host(v), "f": cp.grid_to_host(f)}
    finally:
        cp.close()
    o = oracle_step(w)
    assert rel_l2(g["F"], o["F"]) < TOL_F and rel_l2(g["v"], o["v"]) < TOL_V
    assert rel_l2(g["f"][0], o["f"][0]) < TOL_GRID
