"""CUDA path vs the FP64 oracle for the fluid-stress forces inside solids and
the cell-centred multi-component interpolation (the conformation tensor) that
feeds them (Sec. "Governing Equations", Sec. "Interpolation Scheme").

FP64: bit-identical to the oracle (same evaluation order, per-element buffer
and fixed-order nodal sums). FP32: relative L2 within 1e-5 (forces) and 1e-6
(interpolated values), against the oracle on the same FP32-rounded inputs.
"""
import numpy as np
import pytest

import ifem_workloads as W
from ifem_workloads.fields import conformation_cc
from oracle import oracle as O
from tests._helpers import rel_l2, rounded_workload

pytestmark = pytest.mark.gpu

FP32, FP64 = 0, 1
ETA, BETA, LAM = 0.9, 0.4, 1.7
_cache = {}


def wl(name):
    if name not in _cache:
        _cache[name] = W.make(name)
    return _cache[name]


def _inputs(w, seed, dtype):
    rng = np.random.default_rng(seed)
    N = w.n_nodes
    u = rng.standard_normal((N, 3))
    q = 0.2 * rng.standard_normal((N, 3, 3))
    Cm = np.eye(3)[None] + q @ np.transpose(q, (0, 2, 1))
    C = np.stack([Cm[:, 0, 0], Cm[:, 1, 1], Cm[:, 2, 2], Cm[:, 0, 1], Cm[:, 0, 2], Cm[:, 1, 2]], axis=1)
    return u.astype(dtype).astype(np.float64), C.astype(dtype).astype(np.float64)


def _oracle_fluid(w, u, C):
    xl = w.x_local_all()
    off = w.node_offsets()
    F = np.zeros_like(xl)
    for i, inst in enumerate(w.instances):
        tm = w.templates[inst.tmpl]
        if tm.kind != "solid":
            continue
        s = slice(off[i], off[i + 1])
        F[s] = O.tet_fluid_forces(ETA, BETA, LAM, tm.elems, tm.X, xl[s], u[s], None if C is None else C[s])
    return F


def _gpu_fluid(w, precision, u, C, F0=None):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(w, precision=precision)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        ud = cp.nodes_to_device(u)
        Cd = None if C is None else torch.as_tensor(np.ascontiguousarray(C.T), dtype=cp.dtype).to(cp.device)
        F = cp.nodes_to_device(F0) if F0 is not None else cp.empty_nodes()
        I.ifem_fluid_stress_forces(cp.ctx, cp.batch, x, ud, Cd, ETA, BETA, LAM, F,
                                   I.IFEM_FORCES_ACCUMULATE if F0 is not None else 0)
        I.ifem_sync_status(cp.ctx)
        return cp.nodes_to_host(F)
    finally:
        cp.close()


@pytest.mark.parametrize("case", ["C3", "C5"])
@pytest.mark.parametrize("polymer", [False, True])
def test_fluid_forces_fp64_bit_exact(case, polymer):
    w = wl(case)
    u, C = _inputs(w, 1, np.float64)
    C = C if polymer else None
    g = _gpu_fluid(w, FP64, u, C)
    o = _oracle_fluid(w, u, C)
    assert np.array_equal(g, o), np.abs(g - o).max()


def test_fluid_forces_accumulate_fp64():
    w = wl("C3")
    u, C = _inputs(w, 2, np.float64)
    F0 = np.random.default_rng(3).standard_normal((w.n_nodes, 3))
    g = _gpu_fluid(w, FP64, u, C, F0=F0)
    assert np.array_equal(g, F0 + _oracle_fluid(w, u, C))


def test_fluid_forces_fp32_tolerance():
    w = rounded_workload(wl("C3"), np.float32)
    u, C = _inputs(w, 4, np.float32)
    g = _gpu_fluid(w, FP32, u, C)
    o = _oracle_fluid(w, u, C)
    assert rel_l2(g, o) < 1e-5


def test_membranes_get_no_fluid_force():
    w = wl("C2")
    u, C = _inputs(w, 5, np.float64)
    g = _gpu_fluid(w, FP64, u, C)
    assert np.array_equal(g, np.zeros_like(g))


def _gpu_interp_cc(w, precision, fields, kernel=0):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(w, precision=precision, kernel=kernel)
    try:
        ncomp = fields[0].shape[0]
        x = cp.nodes_to_device(w.x_local_all())
        fd = torch.as_tensor(np.concatenate([f.reshape(-1) for f in fields]), dtype=cp.dtype).to(cp.device)
        out = torch.empty((ncomp, cp.N), dtype=cp.dtype, device=cp.device)
        I.ifem_interpolate_cc(cp.ctx, cp.batch, cp.grid, fd, ncomp, x, out)
        I.ifem_sync_status(cp.ctx)
        return out.cpu().double().numpy().T.copy()
    finally:
        cp.close()


def _oracle_interp_cc(w, fields, kernel=0):
    xa = w.origins_per_node() + w.x_local_all()
    off = w.node_offsets()
    box = np.concatenate([np.full(off[i + 1] - off[i], inst.box) for i, inst in enumerate(w.instances)])
    out = np.zeros((xa.shape[0], fields[0].shape[0]))
    for b, bx in enumerate(w.boxes):
        rows = np.flatnonzero(box == b)
        out[rows] = O.interp_cc(xa[rows], fields[b], bx.n, bx.L, kernel)
    return out


@pytest.mark.parametrize("case", ["C1", "C3", "C5"])
@pytest.mark.parametrize("kernel", [0, 1])
def test_interp_cc_fp64_bit_exact(case, kernel):
    w = wl(case)
    rng = np.random.default_rng(6)
    fields = [conformation_cc(rng, bx.n, bx.L) for bx in w.boxes]
    g = _gpu_interp_cc(w, FP64, fields, kernel)
    o = _oracle_interp_cc(w, fields, kernel)
    assert np.array_equal(g, o), np.abs(g - o).max()


@pytest.mark.parametrize("ncomp", [1, 6])
def test_interp_cc_fp32_tolerance(ncomp):
    w = rounded_workload(wl("C3"), np.float32)
    rng = np.random.default_rng(7)
    fields = [conformation_cc(rng, bx.n, bx.L)[:ncomp].astype(np.float32).astype(np.float64) for bx in w.boxes]
    g = _gpu_interp_cc(w, FP32, fields)
    o = _oracle_interp_cc(w, fields)
    assert rel_l2(g, o) < 1e-6
