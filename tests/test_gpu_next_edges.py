"""Edge cases of the Lagrangian-update, fluid-stress, conformation-interpolation
and indicator-source entry points: empty batches, argument checks, batches
without membranes, and the overwrite / accumulate flags."""
import dataclasses

import numpy as np
import pytest

import ifem_workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu
FP32, FP64 = 0, 1
_cache = {}


def wl(name):
    if name not in _cache:
        _cache[name] = W.make(name)
    return _cache[name]


def _coupler(w, precision=FP64):
    from paper_1807_08219_gb300 import ifem as I
    return I, I.Coupler(w, precision=precision)


def test_empty_batch_entry_points():
    import torch
    w = dataclasses.replace(wl("C3"), instances=[])
    I, cp = _coupler(w)
    try:
        e = torch.empty((3, 0), dtype=torch.float64, device=cp.device)
        G = cp.zeros_grid()
        field = torch.ones(2 * cp.G // 3, dtype=torch.float64, device=cp.device)
        out = torch.empty((2, 0), dtype=torch.float64, device=cp.device)
        vol = torch.empty(1, dtype=torch.float64, device=cp.device)
        I.ifem_interpolate_cc(cp.ctx, cp.batch, cp.grid, field, 2, e, out)
        I.ifem_fluid_stress_forces(cp.ctx, cp.batch, e, e, None, 1.0, 0.5, 1.0, e)
        I.ifem_ab2_update(cp.ctx, cp.batch, e, e, e, 0.1)
        I.ifem_volumes(cp.ctx, cp.batch, e, vol)
        I.ifem_volume_correct(cp.ctx, cp.batch, e, vol, None)
        I.ifem_indicator_source(cp.ctx, cp.batch, cp.grid, e, G)
        I.ifem_sync_status(cp.ctx)
        assert float(G.abs().max()) == 0.0
    finally:
        cp.close()


def test_argument_checks():
    import torch
    w = wl("C3")
    I, cp = _coupler(w)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        F = cp.empty_nodes()
        C = torch.ones((6, cp.N), dtype=torch.float64, device=cp.device)
        field = torch.ones(cp.G, dtype=torch.float64, device=cp.device)
        out = torch.empty((3, cp.N), dtype=torch.float64, device=cp.device)
        for bad in (0, 65):
            with pytest.raises(I.IfemError):
                I.ifem_interpolate_cc(cp.ctx, cp.batch, cp.grid, field, bad, x, out)
        with pytest.raises(I.IfemError):   # polymer term needs lambda > 0
            I.ifem_fluid_stress_forces(cp.ctx, cp.batch, x, x, C, 1.0, 0.5, 0.0, F)
        with pytest.raises(I.IfemError):
            I.ifem_fluid_stress_forces(cp.ctx, cp.batch, x, x, None, -1.0, 0.5, 1.0, F)
        with pytest.raises(I.IfemError):
            I.ifem_fluid_stress_forces(cp.ctx, cp.batch, x, x, None, 1.0, 0.5, 1.0, F, 4)
        with pytest.raises(I.IfemError):
            I.ifem_ab2_update(cp.ctx, cp.batch, x, x, x, float("nan"))
        with pytest.raises(I.IfemError):
            I.ifem_indicator_source(cp.ctx, cp.batch, cp.grid, x, field, 8)
    finally:
        cp.close()


def test_volume_correction_leaves_solids_alone():
    import torch
    w = wl("C3")
    I, cp = _coupler(w)
    try:
        x = cp.nodes_to_device(w.x_local_all() * 1.01)
        x_before = x.clone()
        V0 = torch.full((len(w.instances),), 1.0, dtype=torch.float64, device=cp.device)
        lam = torch.full_like(V0, 7.0)
        I.ifem_volume_correct(cp.ctx, cp.batch, x, V0, lam)
        I.ifem_sync_status(cp.ctx)
        assert torch.equal(x, x_before)
        assert float(lam.abs().max()) == 0.0
    finally:
        cp.close()


def test_indicator_overwrite_and_fluid_accumulate():
    import torch
    w = wl("C2")
    I, cp = _coupler(w)
    try:
        x = cp.nodes_to_device(w.x_local_all())
        G = torch.full((cp.G,), 3.0, dtype=torch.float64, device=cp.device)
        I.ifem_indicator_source(cp.ctx, cp.batch, cp.grid, x, G, I.IFEM_SPREAD_OVERWRITE)
        ref = cp.zeros_grid()
        I.ifem_indicator_source(cp.ctx, cp.batch, cp.grid, x, ref, 0)
        assert torch.equal(G, ref)
        # membranes carry no fluid stress: accumulate leaves F as it was
        F = torch.full((3, cp.N), 2.5, dtype=torch.float64, device=cp.device)
        I.ifem_fluid_stress_forces(cp.ctx, cp.batch, x, x, None, 1.0, 0.5, 1.0, F, I.IFEM_FORCES_ACCUMULATE)
        I.ifem_sync_status(cp.ctx)
        assert float((F - 2.5).abs().max()) == 0.0
    finally:
        cp.close()
