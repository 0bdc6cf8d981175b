"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import oracle as O

KER_NAMES = {0: "peskin4", 1: "mls27"}


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def rounded_workload(wl, dtype):
    """The workload as the CUDA path sees it in `dtype`: positions and grid
    velocities rounded to that precision (then held in FP64 for the oracle)."""
    inst = [dataclasses.replace(i, x_local=i.x_local.astype(dtype).astype(np.float64)) for i in wl.instances]
    u = [np.asarray(ub).astype(dtype).astype(np.float64) for ub in wl.u]
    return dataclasses.replace(wl, instances=inst, u=u)


def random_grid(wl, seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return [scale * rng.standard_normal((3, b.n, b.n, b.n)) for b in wl.boxes]


def run_gpu_step(wl, precision, kernel=0, scatter=0, tile=0, flags=0, f0=None, with_red=True):
    """One ifem_step_coupling on the GPU. Returns host arrays (FP64)."""
    import torch
    from paper_1807_08219_gb300 import ifem as I
    cp = I.Coupler(wl, precision=precision, kernel=kernel, scatter=scatter, tile=tile)
    try:
        x = cp.nodes_to_device(wl.x_local_all())
        u = cp.grid_to_device(wl.u)
        F = cp.empty_nodes()
        v = cp.empty_nodes()
        f = cp.grid_to_device(f0) if f0 is not None else cp.zeros_grid()
        red = torch.zeros(12 * len(wl.instances) + 6 * len(wl.boxes), dtype=torch.float64, device=cp.device)
        I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, red if with_red else None, flags)
        rc, st = I.ifem_sync_status(cp.ctx, raise_on_error=False)
        out = {"F": cp.nodes_to_host(F), "v": cp.nodes_to_host(v), "f": cp.grid_to_host(f),
               "red": red.cpu().numpy(), "rc": rc, "stats": st}
    finally:
        cp.close()
    return out


def oracle_step(wl, kernel=0, density=True, f0=None):
    return O.oracle_step(wl, kernel=kernel, density=density, f0=f0)
