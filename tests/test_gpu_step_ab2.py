"""The coupling step with the position update of Algorithm step 4 and Eq.
Bashforth_eqn (ifem_step_coupling_ab2) against the FP64 oracle.

The oracle side is the oracle's coupling step followed by its AB2 update on
the oracle's velocities. FP64 (deterministic) mode: x_new bit-identical. FP32
mode: x_new within the bound that the velocity tolerance (relative L2 1e-6)
and the FP32 rounding of the update give; dt is chosen so that the
displacement is a tenth of the positions, so a dropped or mis-signed term
fails by orders of magnitude. Consistency of the fusion: x_new equals the
separate ifem_ab2_update applied to the velocities the same call wrote, bit
for bit, and v equals that of ifem_step_coupling (also when the step is
replayed from a CUDA graph).
"""
import numpy as np
import pytest

import ifem_workloads as W
from oracle import oracle as O
from tests._helpers import oracle_step, rel_l2, rounded_workload

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
DET, ATOMIC = 0, 1
TOL_V = 1e-6
_cache = {}


def wl(name):
    if name not in _cache:
        _cache[name] = W.make(name)
    return _cache[name]


def _v_prev(w, dtype, seed=5):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((w.n_nodes, 3)).astype(dtype).astype(np.float64)


def _dt(w, o_v, vp):
    """dt with |dt (3/2 v - 1/2 vp)| about a tenth of |x| (local positions)."""
    step = np.linalg.norm(1.5 * o_v - 0.5 * vp)
    return float(np.float32(0.1 * np.linalg.norm(w.x_local_all()) / step))


def _run(w, precision, scatter, kernel, vp, dt, tile=0):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(w, precision=precision, scatter=scatter, kernel=kernel, tile=tile)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        u = cp.grid_to_device(w.u)
        vpd = cp.nodes_to_device(vp)
        F, v, xn = cp.empty_nodes(), cp.empty_nodes(), cp.empty_nodes()
        f = cp.zeros_grid()
        red = torch.zeros(12 * len(w.instances) + 6 * len(w.boxes), dtype=torch.float64, device=cp.device)
        I.ifem_step_coupling_ab2(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, red, 0, vpd, dt, xn)
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        assert rc == 0, st
        # the separate update on the velocities this call wrote
        xs = x.clone()
        I.ifem_ab2_update(cp.ctx, cp.batch, xs, v, vpd, dt)
        # the plain step's velocities on the same inputs
        v2 = cp.empty_nodes()
        I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x, u, cp.empty_nodes(), cp.zeros_grid(), v2, None)
        I.ifem_sync_status(cp.ctx)
        assert torch.equal(v, v2)
        assert torch.equal(xn, xs)
        return {"x_new": cp.nodes_to_host(xn), "v": cp.nodes_to_host(v), "red": red.cpu().numpy()}
    finally:
        cp.close()


@pytest.mark.parametrize("case", ["C2", "C3"])
@pytest.mark.parametrize("kernel", [0, 1])
def test_fp64_step_ab2_bit_exact(case, kernel):
    w = wl(case)
    o = oracle_step(w, kernel=kernel)
    vp = _v_prev(w, np.float64)
    dt = _dt(w, o["v"], vp)
    g = _run(w, FP64, DET, kernel, vp, dt)
    assert np.array_equal(g["v"], o["v"])
    x_o = O.ab2(w.x_local_all(), o["v"], vp, dt)
    assert np.array_equal(g["x_new"], x_o), np.abs(g["x_new"] - x_o).max()


@pytest.mark.parametrize("case", ["C2", "C3"])
@pytest.mark.parametrize("scatter,kernel", [(ATOMIC, 0), (DET, 0), (ATOMIC, 1)])
def test_fp32_step_ab2(case, scatter, kernel):
    """(ATOMIC, Peskin) is the fused kernel; the others update after the interpolation."""
    w = rounded_workload(wl(case), np.float32)
    o = oracle_step(w, kernel=kernel)
    vp = _v_prev(w, np.float32)
    dt = _dt(w, o["v"], vp)
    g = _run(w, FP32, scatter, kernel, vp, dt)
    x = w.x_local_all()
    x_o = O.ab2(x, o["v"], vp, dt)
    assert rel_l2(g["v"], o["v"]) < TOL_V
    # bound: velocity error through 3/2 dt, plus one FP32 rounding of each
    # of the five operations on values no larger than |x| + |dt| (1.5|v| + 0.5|vp|)
    nv = np.linalg.norm(o["v"])
    mag = np.linalg.norm(x) + abs(dt) * (1.5 * nv + 0.5 * np.linalg.norm(vp))
    tol = (1.5 * abs(dt) * TOL_V * nv + 5 * 2.0**-24 * mag) / np.linalg.norm(x_o)
    assert rel_l2(g["x_new"], x_o) < tol
    # the update moved the nodes by about a tenth of |x|: far above tol
    assert rel_l2(x, x_o) > 1e3 * tol


def test_fp32_step_ab2_graph_replay():
    """The fused step captured in a CUDA graph gives the eager step's x_new and v."""
    import torch
    from paper_1807_08219_gb300 import ifem as I
    w = rounded_workload(wl("C2"), np.float32)
    vp = _v_prev(w, np.float32)
    cp = I.Coupler(w, precision=FP32, scatter=ATOMIC, tile=12)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        u = cp.grid_to_device(w.u)
        vpd = cp.nodes_to_device(vp)
        F, v, xn, f = cp.empty_nodes(), cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
        stream = torch.cuda.Stream(device=cp.device)
        I.ifem_prepare(cp.ctx, cp.batch, x, stream)

        def step(s):
            I.ifem_step_coupling_ab2(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, None, 0, vpd, 0.01, xn, s)

        with torch.cuda.stream(stream):
            step(stream)
        torch.cuda.synchronize()
        ref_v, ref_x = v.clone(), xn.clone()
        v.zero_()
        xn.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step(torch.cuda.current_stream())
        g.replay()
        torch.cuda.synchronize()
        I.ifem_sync_status(cp.ctx)
        assert torch.equal(v, ref_v) and torch.equal(xn, ref_x)
    finally:
        cp.close()


def test_step_ab2_argument_checks():
    import torch
    from paper_1807_08219_gb300 import ifem as I
    w = wl("C2")
    cp = I.Coupler(w, precision=FP64)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        u = cp.grid_to_device(w.u)
        F, v, vp, xn, f = (cp.empty_nodes() for _ in range(5))
        f = cp.zeros_grid()
        call = lambda **kw: I.ifem_step_coupling_ab2(  # noqa: E731
            cp.ctx, cp.batch, cp.grid, kw.get("x", x), u, kw.get("F", F), f, kw.get("v", v), None, 0,
            kw.get("vp", vp), kw.get("dt", 0.01), kw.get("xn", xn))
        for bad in ({"xn": x}, {"xn": v}, {"xn": vp}, {"xn": F}, {"vp": v}, {"dt": float("nan")},
                    {"dt": float("inf")}, {"vp": None}, {"xn": None}):
            with pytest.raises(I.IfemError):
                call(**bad)
        # a view overlapping x by one node still counts as overlap
        big = torch.empty((3 * cp.N + 1,), dtype=torch.float64, device=cp.device)
        with pytest.raises(I.IfemError):
            call(x=big[:3 * cp.N].view(3, cp.N), xn=big[1:].view(3, cp.N))
        call()
        I.ifem_sync_status(cp.ctx)
    finally:
        cp.close()


def test_step_ab2_empty_batch():
    import dataclasses
    import torch
    from paper_1807_08219_gb300 import ifem as I
    w = dataclasses.replace(wl("C3"), instances=[])
    cp = I.Coupler(w, precision=FP32, scatter=ATOMIC)
    try:
        e = torch.empty((3, 0), dtype=torch.float32, device=cp.device)
        u = cp.grid_to_device(w.u)
        f = cp.zeros_grid()
        I.ifem_step_coupling_ab2(cp.ctx, cp.batch, cp.grid, e, u, e, f, e, None, 0, e, 0.1, e)
        I.ifem_sync_status(cp.ctx)
        assert float(f.abs().max()) == 0.0
    finally:
        cp.close()
