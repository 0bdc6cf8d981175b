"""ifem_compute_forces_noalloc against ifem_compute_forces, through the C ABI.

The allocation-free entry point exists for callers that cannot call
cudaMalloc: hosts whose own pool or allocator owns all device memory from
start-up, and real-time loops that forbid allocation once running (an
allocation may synchronise the device and take unbounded time).
It must give the forces of the ordinary entry point: bit-identical in the
deterministic FP64 mode, within the FP32 tolerance (relative L2 1e-5)
otherwise, on two calls in a row (the second call reuses the shared scratch
array the first one left behind). Batches whose scratch does not fit the
fixed array are rejected before any launch.
"""
import dataclasses

import numpy as np
import pytest

import ifem_workloads as W

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["C2", "C3"])
@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_compute_forces_twice(case, precision):
    import torch
    from paper_1807_08219_gb300 import ifem as I
    wl = W.make(case)
    cp = I.Coupler(wl, precision=precision, scatter=I.IFEM_SCATTER_DET)
    try:
        x = cp.nodes_to_device(wl.x_local_all())
        F_ref = cp.empty_nodes()
        I.ifem_compute_forces(cp.ctx, cp.batch, x, F_ref)
        ref = cp.nodes_to_host(F_ref)
        for _ in range(2):
            F = torch.full_like(F_ref, float("nan"))
            I.ifem_compute_forces_noalloc(cp.ctx, cp.batch, x, F)
            torch.cuda.synchronize()
            got = cp.nodes_to_host(F)
            if precision == I.IFEM_FP64:
                assert np.array_equal(got, ref)
            else:
                assert _rel_l2(got, ref) < 1e-5
        I.ifem_sync_status(cp.ctx)
    finally:
        cp.close()


def test_noalloc_rejects_batches_beyond_the_fixed_scratch():
    from paper_1807_08219_gb300 import ifem as I
    base = W.make("C3")
    # 40 copies of the 20250-tet ball: 810k tets x 12 doubles, far above 32 MiB
    inst = [dataclasses.replace(base.instances[0], origin=base.instances[0].origin + 0.01 * k) for k in range(40)]
    wl = dataclasses.replace(base, instances=inst)
    cp = I.Coupler(wl, precision=I.IFEM_FP64)
    try:
        x = cp.nodes_to_device(wl.x_local_all())
        F = cp.empty_nodes()
        with pytest.raises(I.IfemError) as e:
            I.ifem_compute_forces_noalloc(cp.ctx, cp.batch, x, F)
        assert e.value.code == -7
    finally:
        cp.close()
