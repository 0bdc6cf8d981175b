"""Parity at the benchmark sizes: the 500-RBC + 100-platelet suspension
(1.33M nodes, 256^3) in the bench's launch configuration, and the 64-box
mixed batch, each against the FP64 oracle over every node and grid value;
on the suspension also the step with the fused position update and the
host-array step.

FP64 mode: interpolation and spreading (of the GPU's own forces) bit-exact,
forces within 1e-13 relative L2 (the bending angle deficit is taken from a
different atan2 on each side; the measured error is printed). FP32 mode: the stated relative L2
tolerances (forces 1e-5, velocities 1e-6, grid field 1e-5).
"""
import numpy as np
import pytest

import ifem_workloads as W
from oracle import oracle as O
from tests._helpers import rel_l2, rounded_workload

pytestmark = pytest.mark.gpu

_wl = {}


def workload(name):
    if name not in _wl:
        _wl[name] = W.make(name)
    return _wl[name]


def run(wl, precision, scatter, tile):
    """One step; tile 0 autotunes in ifem_prepare first, as the benchmark does."""
    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(wl, precision=precision, scatter=scatter, tile=tile)
    try:
        dt = np.float64 if precision == I.IFEM_FP64 else np.float32
        x = cp.nodes_to_device(wl.x_local_all(dt))
        if tile == 0:
            I.ifem_prepare(cp.ctx, cp.batch, x)
        u = cp.grid_to_device(wl.u)
        F, v, f = cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
        I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, None)
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        return rc, st, cp.nodes_to_host(F), cp.nodes_to_host(v), cp.grid_to_host(f)
    finally:
        cp.close()


def oracle_parts(wl, F):
    """Oracle forces, interpolation, and spreading of the given nodal forces F."""
    xl = wl.x_local_all()
    off = wl.node_offsets()
    Fo = np.zeros_like(xl)
    for i, inst in enumerate(wl.instances):
        Fo[off[i]:off[i + 1]] = O.template_forces(wl.templates[inst.tmpl], xl[off[i]:off[i + 1]])
    xa = wl.origins_per_node() + xl
    box = np.concatenate([np.full(off[i + 1] - off[i], inst.box) for i, inst in enumerate(wl.instances)])
    v = np.zeros_like(xl)
    f = []
    for b, bx in enumerate(wl.boxes):
        rows = np.flatnonzero(box == b)
        v[rows] = O.interp(xa[rows], wl.u[b], bx.n, bx.L)
        f.append(O.spread(xa[rows], F[rows], bx.n, bx.L))
    return Fo, v, f


@pytest.mark.parametrize("name", ["C4", "C5"])
def test_fullsize_fp32_bench_configuration(name):
    wl, Fo, vo, fo = oracle_fp32(name)
    rc, st, F, v, f = run(wl, 0, 1, 0)   # atomic scatter, autotuned tile: the benchmark's configuration
    assert rc == 0, st
    assert rel_l2(F, Fo) < 1e-5
    assert rel_l2(v, vo) < 1e-6
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(f, fo)))
    den = np.sqrt(sum(np.sum(b ** 2) for b in fo))
    assert num / den < 1e-5


def oracle_parts_spread(wl, F):
    xl = wl.x_local_all()
    off = wl.node_offsets()
    xa = wl.origins_per_node() + xl
    box = np.concatenate([np.full(off[i + 1] - off[i], inst.box) for i, inst in enumerate(wl.instances)])
    return [O.spread(xa[box == b], F[box == b], bx.n, bx.L) for b, bx in enumerate(wl.boxes)]


@pytest.mark.parametrize("name", ["C4", "C5"])
def test_fullsize_fp64_deterministic(name):
    wl = workload(name)
    rc, st, F, v, f = run(wl, 1, 0, 0)
    assert rc == 0, st
    Fo, vo, fo = oracle_parts(wl, F)
    eF = rel_l2(F, Fo)
    print(f"{name} FP64 forces: rel L2 {eF:.3e} against the oracle")
    assert eF < 1e-13, eF
    assert np.array_equal(v, vo)
    for a, b in zip(f, fo):
        assert np.array_equal(a, b)


_oracle_cache = {}


def oracle_fp32(name):
    """Oracle forces, velocities and spread of its own forces on the FP32-rounded workload."""
    if name not in _oracle_cache:
        wl = rounded_workload(workload(name), np.float32)
        Fo, vo, _ = oracle_parts(wl, np.zeros((wl.n_nodes, 3)))
        _oracle_cache[name] = (wl, Fo, vo, oracle_parts_spread(wl, Fo))
    return _oracle_cache[name]


def test_fullsize_fp32_step_ab2():
    """The step with the fused position update on the suspension, bench configuration:
    x_new against the oracle's update from its own velocities, within the bound the
    velocity tolerance and FP32 rounding give."""
    import torch
    from paper_1807_08219_gb300 import ifem as I
    wl, Fo, vo, _ = oracle_fp32("C4")
    rng = np.random.default_rng(21)
    vp = rng.standard_normal(vo.shape).astype(np.float32).astype(np.float64)
    xl = wl.x_local_all()
    dt = float(np.float32(0.1 * np.linalg.norm(xl) / np.linalg.norm(1.5 * vo - 0.5 * vp)))
    cp = I.Coupler(wl, precision=0, scatter=1, tile=0)
    try:
        x = cp.nodes_to_device(xl)
        I.ifem_prepare(cp.ctx, cp.batch, x)
        u = cp.grid_to_device(wl.u)
        F, v, xn, f = cp.empty_nodes(), cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
        I.ifem_step_coupling_ab2(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, None, 0, cp.nodes_to_device(vp), dt, xn)
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        assert rc == 0, st
        g_v, g_x = cp.nodes_to_host(v), cp.nodes_to_host(xn)
    finally:
        cp.close()
    assert rel_l2(g_v, vo) < 1e-6
    x_o = O.ab2(xl, vo, vp, dt)
    nv = np.linalg.norm(vo)
    mag = np.linalg.norm(xl) + abs(dt) * (1.5 * nv + 0.5 * np.linalg.norm(vp))
    tol = (1.5 * abs(dt) * 1e-6 * nv + 5 * 2.0**-24 * mag) / np.linalg.norm(x_o)
    assert rel_l2(g_x, x_o) < tol
    assert rel_l2(xl, x_o) > 1e3 * tol


def test_fullsize_fp32_host_step():
    """The host-array step on the suspension (positions in two halves), bench configuration."""
    import torch
    from paper_1807_08219_gb300 import ifem as I
    wl, Fo, vo, fo = oracle_fp32("C4")
    cp = I.Coupler(wl, precision=0, scatter=1, tile=0)
    try:
        xh = torch.from_numpy(np.ascontiguousarray(wl.x_local_all(np.float32).T)).pin_memory()
        x = cp.empty_nodes()
        I.ifem_prepare(cp.ctx, cp.batch, cp.nodes_to_device(wl.x_local_all()))
        u = cp.grid_to_device(wl.u)
        F, v, f = cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
        vh = torch.empty((3, cp.N), dtype=torch.float32).pin_memory()
        I.ifem_step_coupling_host(cp.ctx, cp.batch, cp.grid, xh, x, u, F, f, v, vh)
        torch.cuda.synchronize()
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        assert rc == 0, st
        g_F, g_v, g_f = cp.nodes_to_host(F), vh.double().numpy().T.copy(), cp.grid_to_host(f)
    finally:
        cp.close()
    assert rel_l2(g_F, Fo) < 1e-5
    assert rel_l2(g_v, vo) < 1e-6
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(g_f, fo)))
    den = np.sqrt(sum(np.sum(b ** 2) for b in fo))
    assert num / den < 1e-5
