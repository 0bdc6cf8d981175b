"""Conservation sums and binning of the FP32 halo coupling step.

The step's sums come from the per-particle sum kernel in two launches (the
x/F sums beside the transfer, the sums of v and the boxes after it); the
same quantities from ifem_reduce called afterwards on the step's own x, F
and v (one launch, all parts) are equal bit for bit, the partials and tree
of a quantity not depending on the parts a launch computes. The step's
one-pass binning is checked through the transfers: the step's v agrees with
the standalone interpolation of the same positions (another kernel:
relative L2 within the velocity tolerance 1e-6), and the step without sums
(red = null) gives the same v as the step with them, bit for bit. Device
arrays and host arrays (positions in two halves, two force launches) are
both covered.
"""
import dataclasses

import numpy as np
import pytest

import ifem_workloads as W
from tests._helpers import rel_l2

pytestmark = pytest.mark.gpu

_cache = {}


def wl(name):
    if name not in _cache:
        if name == "C5-12":
            w = W.make("C5")
            _cache[name] = dataclasses.replace(w, instances=w.instances[:12])
        else:
            _cache[name] = W.make(name)
    return _cache[name]


def _coupler(w):
    from paper_1807_08219_gb300 import ifem as I
    return I.Coupler(w, precision=I.IFEM_FP32, scatter=I.IFEM_SCATTER_ATOMIC, tile=12)


@pytest.mark.parametrize("case", ["C2", "C3", "C5-12"])
@pytest.mark.parametrize("host", [False, True])
def test_step_sums_equal_standalone_reduction(case, host):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    w = wl(case)
    cp = _coupler(w)
    try:
        n_red = 12 * len(w.instances) + 6 * len(w.boxes)
        u = cp.grid_to_device(w.u)
        F, v, f = cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
        red = torch.full((n_red,), float("nan"), dtype=torch.float64, device=cp.device)
        if host:
            x = cp.empty_nodes()
            x_host = torch.from_numpy(np.ascontiguousarray(w.x_local_all().T)).to(cp.dtype).pin_memory()
            v_host = torch.empty((3, cp.N), dtype=cp.dtype).pin_memory()
            red_host = torch.empty(n_red, dtype=torch.float64).pin_memory()
            I.ifem_step_coupling_host(cp.ctx, cp.batch, cp.grid, x_host, x, u, F, f, v, v_host, red, red_host, 0)
        else:
            x = cp.nodes_to_device(w.x_local_all())
            I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, red, 0)
        torch.cuda.synchronize()
        got = red.cpu().numpy()
        assert np.isfinite(got).all()
        ref = torch.full_like(red, float("nan"))
        I.ifem_reduce(cp.ctx, cp.batch, x, F, v, ref)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        ni = len(w.instances)
        assert np.array_equal(got[: 12 * ni].reshape(ni, 12)[:, :9], ref[: 12 * ni].reshape(ni, 12)[:, :9])
        assert np.array_equal(got, ref)
        if host:
            assert np.array_equal(red_host.numpy(), got)
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        assert rc == 0, st
    finally:
        cp.close()


@pytest.mark.parametrize("case", ["C2", "C5-12"])
def test_step_velocities_from_epilogue_binning(case):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    w = wl(case)
    cp = _coupler(w)
    try:
        n_red = 12 * len(w.instances) + 6 * len(w.boxes)
        u = cp.grid_to_device(w.u)
        x = cp.nodes_to_device(w.x_local_all())
        vs = []
        for with_red in (True, False):
            F, v, f = cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
            red = torch.zeros(n_red, dtype=torch.float64, device=cp.device) if with_red else None
            I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, red, 0)
            torch.cuda.synchronize()
            vs.append(cp.nodes_to_host(v))
        # standalone binning + interpolation of the same positions
        v2 = cp.empty_nodes()
        I.ifem_interpolate(cp.ctx, cp.batch, cp.grid, u, x, v2)
        torch.cuda.synchronize()
        assert np.array_equal(vs[0], vs[1])
        e = rel_l2(vs[0], cp.nodes_to_host(v2))
        print(f"{case}: step v against ifem_interpolate, relative L2 {e:.3e}")
        assert e < 1e-6, e
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        assert rc == 0, st
    finally:
        cp.close()
