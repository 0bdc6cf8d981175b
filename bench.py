"""Coupling-step benchmark: Lagrangian nodes coupled per second on the dense
blood suspension (500 RBC + 100 platelets, 1.33M nodes, 256^3 periodic MAC
grid), FP32, through the C ABI of libifem.

One step = node binning + element forces (membrane Skalak + Helfrich bending,
platelet neo-Hookean tets) + spreading + interpolation + FP64 conservation
sums, replayed from a CUDA graph. Inputs are resident in HBM; L2 (129 MB) is
flushed between timed steps by writing a 256 MB buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ifem|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
repository) on the same workload, on the host cores.
Under torchrun (N > 1) every rank runs its own replica of the workload (the
step has no cross-rank exchange); value = all ranks' nodes / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Lagrangian nodes coupled/s (force+spread+interp) and HBM GB/s; FP32-batched vs FP64 at stated err"
WORKLOADS = {
    "C4": ("dense blood suspension: 500 RBC (2562 nodes, Skalak C=100 + bending) + 100 platelets "
           "(512 nodes / 2058 tets, NH), 256^3 periodic MAC grid, Ht 0.20, 4-point delta"),
    "C5": ("batch of 64 independent periodic boxes (32^3..96^3 cells, h = 1/64) with 1-20 mixed particles "
           "each (capsules 642/2562, RBC 2562, Kuhn balls 512-3375 nodes), one launch per stage, 4-point delta"),
}
WORKLOAD = WORKLOADS["C4"]
REF_BUDGET_S = 150.0   # --impl reference: warm-up + timed oracle steps


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the current kernels on the C4 suspension (profiles/*_c4_fp32.md),
# reported for that workload only; set an entry to None when its kernel changes.
NCU_TRAFFIC = {"spread+interp": None, "spread": None, "interp": None, "forces": None, "bin": None}
# The unit that bounds each kernel in that capture and its fraction of peak (context for the HBM
# fraction: the fused transfer kernel is latency-bound at 12 warps per SM, with the L1 load/store
# pipe the busiest unit; the forces kernel is bound by shared-memory wavefronts).
NCU_LIMITER = {"forces": ("shared-memory wavefronts", 0.598)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu: int, interval_ms: int = 20):
        self.gpu = gpu
        self.interval_ms = interval_ms
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, busy, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [s.strip() for s in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            try:
                if float(f[9]) >= 50.0:
                    busy.append(sm[-1])
            except (IndexError, ValueError):
                pass
            for n, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(busy or sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_busy": len(busy),
                "interval_ms": self.interval_ms,
                "window": "every timed GPU loop of the run (headline steps, stage times, end-to-end, extras, FP64)"}


def algorithmic_bytes(N, T, P, real=4):
    """Algorithmic bytes per stage: the bytes each stage must move at least.

    N nodes, T touched lattice values (over the 3 lattices), P (tile, node)
    candidate pairs (0 when the spread walks each tile's own nodes instead),
    `real` bytes per value. Node arrays are read or written once per stage;
    each touched lattice value is read once (interpolation) or read and
    written once (spreading)."""
    lists = P if P else N
    return {
        "bin": 2 * 3 * real * N + 4 * (N + P),          # x read (count + fill), pair/own lists written
        "forces": 2 * 3 * real * N,                     # x read, F written
        "spread": 2 * 3 * real * N + 4 * lists + 2 * real * T,  # x, F read; node list read; f read + written
        "interp": 2 * 3 * real * N + 4 * N + real * T,  # x read, v written, order list read; u read
        # spread with the interpolation fused: x, F read, v written; f read + written, u read
        "spread+interp": 3 * 3 * real * N + 3 * real * T,
        "reduce": 3 * 3 * real * N,                     # x, F, v read
        # the coupling step as one operation: x read, v written; u read, f read + written
        "step": 2 * 3 * real * N + 3 * real * T,
        # the same with the nodal forces F written and read back (the step's F output)
        "step_with_F": 4 * 3 * real * N + 3 * real * T,
    }


def flush_l2(flush, stream):
    """Write a buffer larger than L2 (129 MB) on the timed stream, so that the
    next timed work on that stream starts only after the write has finished."""
    import torch
    with torch.cuda.stream(stream):
        flush.fill_(1.0)


def max_over_ranks(values, device, dist=None):
    """Element-wise maximum of per-rank timings (ms) over all ranks."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(n_nodes_per_rank, world, t_ms):
    """Whole-job nodes per second: every rank couples its own replica in t_ms."""
    return world * n_nodes_per_rank / (t_ms * 1e-3)


def _even_sample(wl, n_target):
    """Evenly spaced particles whose node count first reaches n_target (at least one)."""
    sizes = [wl.templates[i.tmpl].n_nodes for i in wl.instances]
    if n_target >= sum(sizes):
        return list(range(len(sizes))), int(sum(sizes))
    k = 1
    while True:
        sel = sorted(set(np.linspace(0, len(sizes) - 1, k).astype(int).tolist()))
        n = int(sum(sizes[i] for i in sel))
        if n >= n_target or k >= len(sizes):
            return sel, n
        k += 1


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the same workload (rank 0 only), over all host cores.

    Each step is one oracle coupling step (forces, spread, interpolation, sums)
    run by the multi-core timing driver around the unchanged oracle functions
    (cpu_baseline_parallel) over the whole workload, or over an evenly spaced
    sample of its particles when --warmup + --steps whole steps would take
    more than about REF_BUDGET_S seconds."""
    if rank != 0:
        return
    import dataclasses
    import ifem_workloads as W
    from oracle import oracle as O
    O.build()
    wl = W.make(args.workload)
    N = wl.n_nodes
    probe = cpu_baseline_parallel(wl, steps=1, warmup=1)
    per_node = probe["step_s"][0] / N
    per_step = REF_BUDGET_S / max(1, args.steps + max(0, args.warmup))
    sel, n_sel = _even_sample(wl, int(per_step / per_node))
    sub = wl if n_sel == N else dataclasses.replace(wl, instances=[wl.instances[i] for i in sel])
    r = cpu_baseline_parallel(sub, steps=args.steps, warmup=max(1, args.warmup))
    t = float(np.mean(r["step_s"]))
    val = n_sel / t
    sample = (f"{len(sel)} of {len(wl.instances)} particles evenly spaced ({n_sel} of {N} nodes), one full "
              f"oracle step (forces + spread + interp + sums) on the whole grid per timed step, "
              f"{r['cores']} host threads over the unchanged single-threaded oracle functions")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "nodes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "nodes": N,
                   "grid": [bx.n for bx in wl.boxes] if len(wl.boxes) > 1 else wl.boxes[0].n,
                   "sample_nodes": n_sel},
        "cpu_baseline": {"value": val, "unit": "nodes/s", "cores": r["cores"], "kind": "oracle", "sample": sample,
                         "host": r["host"]},
        "e2e": {"value": val, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def host_description():
    """The host CPU: model name (lscpu, else /proc/cpuinfo, else platform) and usable cores."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    return {"cpu_model": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "nproc": cores}


def cpu_baseline_sample(wl):
    """Oracle timed on the whole workload (host cores, one thread): full coupling
    steps repeated until at least 10 s of CPU work (at most 8 steps)."""
    from oracle import oracle as O
    O.build()
    xl = wl.x_local_all(np.float32).astype(np.float64)
    sel = list(range(len(wl.instances)))
    ts = []
    while sum(ts) < 10.0 and len(ts) < 8:
        t0 = time.perf_counter()
        O.oracle_step(wl, x_local=xl, instances=sel)
        ts.append(time.perf_counter() - t0)
    t = float(np.mean(ts))
    return {"value": wl.n_nodes / t, "unit": "nodes/s", "cores": 1, "kind": "oracle",
            "sample": f"the whole workload ({wl.n_nodes} nodes), {len(ts)} full oracle steps (forces + spread + "
                      f"interp + sums), single thread, {sum(ts):.1f} s"}


# ---- the oracle over all host cores (a timing driver around the unchanged,
# single-threaded oracle functions)
_SUMS_WL = {}


def _sums_init(chunks):
    global _SUMS_WL
    _SUMS_WL = chunks


def _sums_task(args):
    """Per-particle FP64 sums of one chunk of particles (runs in a worker process)."""
    from oracle import oracle as O
    c, xl, F, v = args
    return O.reductions(_SUMS_WL[c], xl, F, v)


def _chunks_by_nodes(wl, parts):
    """Contiguous particle ranges with about equal node counts."""
    off = wl.node_offsets()
    N = int(off[-1])
    bounds = [0]
    for p in range(1, parts):
        bounds.append(int(np.searchsorted(off, p * N / parts)))
    bounds.append(len(wl.instances))
    return [(a, b) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


def cpu_baseline_parallel(wl, threads=None, min_s=3.0, max_steps=8, steps=None, warmup=1):
    """The oracle's coupling step over all host cores: one thread per chunk of
    particles (contiguous, equal node counts) runs the oracle's element and
    bending forces, its spreading into a private grid per chunk and its
    interpolation (the C calls release the interpreter lock); the private
    grids are summed in chunk order (fixed order, split over the threads by
    slabs); the per-particle FP64 sums, which the oracle takes with
    math.fsum under the interpreter lock, run in a process pool (spawn). The
    oracle itself is unchanged and single-threaded."""
    import concurrent.futures as cf
    import dataclasses
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    host = host_description()
    P = threads or host["nproc"]
    xl = wl.x_local_all(np.float32).astype(np.float64)
    off = wl.node_offsets()
    chunks = _chunks_by_nodes(wl, P)
    light = {c: dataclasses.replace(wl, instances=[dataclasses.replace(i, x_local=np.zeros((0, 3)))
                                                   for i in wl.instances[a:b]], u=[])
             for c, (a, b) in enumerate(chunks)}
    origins = wl.origins_per_node()
    box_of = np.concatenate([np.full(off[i + 1] - off[i], inst.box) for i, inst in enumerate(wl.instances)])

    def local_work(c):
        a, b = chunks[c]
        lo, hi = int(off[a]), int(off[b])
        F = np.zeros((hi - lo, 3))
        for ii in range(a, b):
            F[off[ii] - lo:off[ii + 1] - lo] = O.template_forces(wl.templates[wl.instances[ii].tmpl],
                                                                 xl[off[ii]:off[ii + 1]])
        xa = origins[lo:hi] + xl[lo:hi]
        v = np.zeros_like(F)
        grids = {}
        for bi, bx in enumerate(wl.boxes):
            rows = np.flatnonzero(box_of[lo:hi] == bi)
            if rows.size:
                grids[bi] = O.spread(xa[rows], F[rows], bx.n, bx.L)
                v[rows] = O.interp(xa[rows], wl.u[bi], bx.n, bx.L)
        return F, v, grids

    def grid_sum(parts, out, s0, s1):
        out[s0:s1] = 0.0
        for g in parts:        # chunk order: fixed summation order
            out[s0:s1] += g[s0:s1]

    ctx = mp.get_context("spawn")
    ts = []
    with cf.ThreadPoolExecutor(P) as tp, cf.ProcessPoolExecutor(P, mp_context=ctx, initializer=_sums_init,
                                                                initargs=(light,)) as pp:
        fields = [np.zeros((3, bx.n, bx.n, bx.n)) for bx in wl.boxes]
        warm = max(1, warmup)   # the first step starts the worker processes: never timed

        def more():
            if steps is not None:
                return len(ts) < steps
            return (sum(ts) < min_s or len(ts) < 2) and len(ts) < max_steps

        while more():
            t0 = time.perf_counter()
            res = list(tp.map(local_work, range(len(chunks))))
            jobs = []
            for bi, bx in enumerate(wl.boxes):
                parts = [r[2][bi].reshape(-1) for r in res if bi in r[2]]
                flat = fields[bi].reshape(-1)
                step = -(-flat.size // P)
                jobs += [tp.submit(grid_sum, parts, flat, s0, min(s0 + step, flat.size))
                         for s0 in range(0, flat.size, step)]
            sums = list(pp.map(_sums_task, [(c, xl[off[a]:off[b]], r[0], r[1])
                                            for c, ((a, b), r) in enumerate(zip(chunks, res))]))
            for j in jobs:
                j.result()
            if warm == 0:
                ts.append(time.perf_counter() - t0)
            else:
                warm -= 1
            del res, sums
    t = float(np.mean(ts))
    return {"value": wl.n_nodes / t, "unit": "nodes/s", "cores": P, "kind": "oracle",
            "sample": (f"the whole workload ({wl.n_nodes} nodes), {len(ts)} full oracle steps on {P} threads "
                       f"(forces, spread into per-chunk private grids, interp; grids summed in chunk order; "
                       f"per-particle sums in {P} processes), {sum(ts):.1f} s wall"),
            "host": host, "step_s": ts}


def time_extras(wl, I, torch, dev, flush, T, reps=20, warm=3):
    """CUDA-event times of the Lagrangian-update and fluid-stress entry points
    on the resident workload (FP32, same context kind as the step), each with
    its algorithmic bytes: every node array read or written once, grid values
    read (or read and written) once over the touched footprint. The coupling
    step with the fused position update is timed beside the plain step, both
    launched eagerly (no graph), so that their difference is the cost of the
    update inside the step."""
    import math
    N = wl.n_nodes
    n_solid = int(sum(wl.templates[i.tmpl].n_nodes for i in wl.instances if wl.templates[i.tmpl].kind == "solid"))
    cp = I.Coupler(wl, precision=I.IFEM_FP32, scatter=I.IFEM_SCATTER_ATOMIC, tile=16)
    s = torch.cuda.Stream(device=dev)
    x0 = cp.nodes_to_device(wl.x_local_all(np.float32))
    x = x0.clone()
    v = torch.randn((3, N), device=dev) * 0.1
    vp = torch.randn((3, N), device=dev) * 0.1
    F = cp.empty_nodes()
    # cell-centred conformation field I + smooth perturbation, 6 components per box
    parts = []
    for bx in wl.boxes:
        c = (torch.arange(bx.n, device=dev, dtype=torch.float32) + 0.5) * (2 * math.pi / bx.n)
        z, y, xg = torch.meshgrid(c, c, c, indexing="ij")
        base = 0.05 * torch.cos(xg + 2 * y - z)
        parts.append(torch.stack([1 + base, 1 - base, 1 + 0.5 * base, 0.3 * base, -0.2 * base, 0.1 * base]).reshape(-1))
    field = torch.cat(parts)
    Cn = torch.empty((6, N), device=dev)
    G = cp.zeros_grid()
    vol = torch.empty(len(wl.instances), dtype=torch.float64, device=dev)
    I.ifem_volumes(cp.ctx, cp.batch, x0, vol, s)
    V0 = vol.clone()
    lam = torch.empty_like(vol)
    u = cp.grid_to_device(wl.u)
    vs, xn, f = cp.empty_nodes(), cp.empty_nodes(), cp.zeros_grid()
    red = torch.zeros(12 * len(wl.instances) + 6 * len(wl.boxes), dtype=torch.float64, device=dev)
    I.ifem_prepare(cp.ctx, cp.batch, x0, s)
    step_bytes = 4 * 12 * N + 12 * T
    calls = {
        "step_coupling": (lambda: I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x0, u, F, f, vs, red, 0, s),
                          step_bytes),
        "step_coupling_ab2": (lambda: I.ifem_step_coupling_ab2(cp.ctx, cp.batch, cp.grid, x0, u, F, f, vs, red, 0,
                                                               vp, 1e-4, xn, s), step_bytes + 24 * N),
        "interp_cc6": (lambda: I.ifem_interpolate_cc(cp.ctx, cp.batch, cp.grid, field, 6, x0, Cn, s),
                       12 * N + 24 * N + 6 * 4 * (T // 3)),
        "fluid_stress_forces": (lambda: I.ifem_fluid_stress_forces(cp.ctx, cp.batch, x0, v, Cn, 1.0, 0.5, 1.0, F,
                                                                   0, s), 12 * N + 48 * n_solid),
        "ab2_update": (lambda: I.ifem_ab2_update(cp.ctx, cp.batch, x, v, vp, 1e-4, s), 48 * N),
        "volumes": (lambda: I.ifem_volumes(cp.ctx, cp.batch, x0, vol, s), 12 * N),
        "volume_correct": (lambda: I.ifem_volume_correct(cp.ctx, cp.batch, x, V0, lam, s), 24 * N + 24 * N),
        "indicator_source": (lambda: I.ifem_indicator_source(cp.ctx, cp.batch, cp.grid, x0, G, 0, s),
                             12 * N + 8 * T),
    }
    out = {}
    for name, (call, nbytes) in calls.items():
        ts = []
        for it in range(warm + reps):
            flush_l2(flush, s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            call()
            e1.record(s)
            e1.synchronize()
            if it >= warm:
                ts.append(e0.elapsed_time(e1))
        ms = float(np.mean(ts))
        out[name] = {"ms": ms, "nodes_per_s": N / (ms * 1e-3), "algorithmic_bytes": int(nbytes),
                     "gbs": nbytes / (ms * 1e-3) / 1e9}
    I.ifem_sync_status(cp.ctx)
    cp.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ifem", choices=["ifem", "reference"])
    ap.add_argument("--scatter", default="atomic", choices=["atomic", "det"])
    ap.add_argument("--tile", type=int, default=0, help="tile edge; 0 = autotune (ifem_prepare)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip timing the Lagrangian-update entry points")
    ap.add_argument("--workload", default="C4", choices=sorted(WORKLOADS),
                    help="C4 (default, the headline suspension) or C5 (64 mixed boxes)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import ifem_workloads as W
    from paper_1807_08219_gb300 import ifem as I

    wl = W.make(args.workload)
    N = wl.n_nodes
    scatter = I.IFEM_SCATTER_ATOMIC if args.scatter == "atomic" else I.IFEM_SCATTER_DET
    cp = I.Coupler(wl, precision=I.IFEM_FP32, scatter=scatter, tile=args.tile, device=local)
    dev = cp.device
    xl32 = wl.x_local_all(np.float32)
    x = cp.nodes_to_device(xl32)
    u = cp.grid_to_device(wl.u)
    F, v = cp.empty_nodes(), cp.empty_nodes()
    f = cp.zeros_grid()
    red = torch.zeros(12 * len(wl.instances) + 6 * len(wl.boxes), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step(s):
        I.ifem_step_coupling(cp.ctx, cp.batch, cp.grid, x, u, F, f, v, red, 0, s)

    # work buffers (and, with --tile 0, the tile autotuner) before capture
    I.ifem_prepare(cp.ctx, cp.batch, x, stream)
    tile = I.ifem_ctx_tile(cp.ctx)

    # first step outside capture: allocates the work buffers, gives the counts
    with torch.cuda.stream(stream):
        step(stream)
    torch.cuda.synchronize()
    _, st = I.ifem_sync_status(cp.ctx)
    # touched lattice values: the non-zero values of the first step's spread
    # into the zero field (each counted once, whichever tiles added to it)
    T, P = int(torch.count_nonzero(f)), st["pairs"]

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step(torch.cuda.current_stream())
    torch.cuda.synchronize()

    # clock samples: from before the headline steps to after the last timed
    # GPU loop (the headline region alone can be shorter than one sample)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(1.0)   # nvidia-smi's first sample lands before the timed steps
    for _ in range(args.warmup):
        flush_l2(flush, stream)
        with torch.cuda.stream(stream):
            g.replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush_l2(flush, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            g.replay()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    t_ms = max_over_ranks([float(np.mean(times))], dev, dist)[0]
    value = job_throughput(N, world, t_ms)

    # per-stage times of the same step (profiled context, same stream, same flush)
    cpp = I.Coupler(wl, precision=I.IFEM_FP32, scatter=scatter, tile=tile, device=local, profile=1)
    stages = {k: [] for k in ("bin", "forces", "spread", "interp", "reduce")}
    fp = cpp.zeros_grid()
    for it in range(args.warmup + args.steps):
        flush_l2(flush, stream)
        with torch.cuda.stream(stream):
            I.ifem_step_coupling(cpp.ctx, cpp.batch, cpp.grid, x, u, F, fp, v, red, 0, stream)
        ms = I.ifem_stage_times(cpp.ctx)
        if it >= args.warmup:
            for k in stages:
                stages[k].append(ms[k])
    I.ifem_sync_status(cpp.ctx)
    stage_ms = {k: float(np.mean(vv)) for k, vv in stages.items()}
    cpp.close()
    ab = algorithmic_bytes(N, T, P)
    hbm, peak_kind = peaks()
    fused = stage_ms["interp"] == 0.0   # interpolation ran inside the spread kernel
    if fused:
        stage_ms["spread+interp"] = stage_ms.pop("spread")
        stage_ms.pop("interp")
    dom = max((k for k in ("spread+interp", "spread", "interp", "forces", "bin") if k in stage_ms),
              key=lambda k: stage_ms[k])
    achieved = ab[dom] / (stage_ms[dom] * 1e-3) / 1e9
    step_gbs = ab["step"] / (t_ms * 1e-3) / 1e9
    step_gbs_F = ab["step_with_F"] / (t_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers (pinned): ifem_step_coupling_host
    # copies x in, runs the step and copies v and the sums out, all inside the
    # timed region; beside it the same with the caller doing the copies around
    # ifem_step_coupling (no overlap of copies and kernels)
    x_host = torch.from_numpy(np.ascontiguousarray(xl32.T)).pin_memory()
    v_host = torch.empty((3, N), dtype=torch.float32).pin_memory()
    red_host = torch.empty(red.numel(), dtype=torch.float64).pin_memory()

    def host_step(s):
        I.ifem_step_coupling_host(cp.ctx, cp.batch, cp.grid, x_host, x, u, F, f, v, v_host, red, red_host, 0, s)

    def caller_copies(s):
        x.copy_(x_host, non_blocking=True)
        step(s)
        v_host.copy_(v, non_blocking=True)
        red_host.copy_(red, non_blocking=True)

    def time_e2e(fn):
        ts = []
        for it in range(args.warmup + args.steps):
            flush_l2(flush, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                fn(stream)
                e1.record(stream)
            e1.synchronize()
            if it >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        return max_over_ranks([float(np.mean(ts))], dev, dist)[0]

    def graphed(fn):
        """The same call captured once into a CUDA graph (host copies included, as
        memcpy nodes from the pinned host arrays) and replayed every step."""
        gh = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gh, stream=stream):
            fn(torch.cuda.current_stream())
        torch.cuda.synchronize()
        return lambda s: gh.replay()

    e2e_eager_ms = time_e2e(host_step)
    e2e_ms = time_e2e(graphed(host_step))
    e2e_caller_ms = time_e2e(caller_copies)

    # Lagrangian update, fluid-stress and indicator entry points (reported beside)
    extras = None if args.no_extras else time_extras(wl, I, torch, dev, flush, T)

    # FP64 deterministic GPU path on the same workload (reported beside)
    fp64 = None
    if not args.no_fp64:
        c64 = I.Coupler(wl, precision=I.IFEM_FP64, tile=0, device=local)
        x64 = c64.nodes_to_device(xl32.astype(np.float64))
        I.ifem_prepare(c64.ctx, c64.batch, x64)   # tile autotuner (FP64 candidates)
        u64 = c64.grid_to_device(wl.u)
        F64, v64, f64 = c64.empty_nodes(), c64.empty_nodes(), c64.zeros_grid()
        for _ in range(2):
            I.ifem_step_coupling(c64.ctx, c64.batch, c64.grid, x64, u64, F64, f64, v64, None, 0, stream)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            flush_l2(flush, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            I.ifem_step_coupling(c64.ctx, c64.batch, c64.grid, x64, u64, F64, f64, v64, None, 0, stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        I.ifem_sync_status(c64.ctx)
        # error of the FP32 step against the FP64 GPU step (same inputs)
        Fd = F.double()
        vd = v.double()
        eF = float(torch.linalg.norm(Fd - F64) / torch.linalg.norm(F64))
        ev = float(torch.linalg.norm(vd - v64) / torch.linalg.norm(v64))
        t64 = float(np.mean(ts))
        fp64 = {"value": N / (t64 * 1e-3), "unit": "nodes/s", "ms_per_step": t64, "tile": I.ifem_ctx_tile(c64.ctx),
                "fp32_rel_l2_vs_fp64": {"F": eF, "v": ev}}
        c64.close()
    ck = clocks.stop()

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline_parallel(wl)
        cpu["single_thread"] = cpu_baseline_sample(wl)
    # bin (halo path: count + rank, scan, placement + list of tiles with own nodes; candidate path:
    # count, 2 scans, fill), forces, spread and interp (one fused launch on the halo path), 2 reductions
    launches_per_step = (3 if fused else 4) + 1 + (1 if fused else 2) + 2
    if scatter == I.IFEM_SCATTER_DET:
        launches_per_step += 3
    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "nodes": N, "particles": len(wl.instances),
                   "grid": [b.n for b in wl.boxes] if len(wl.boxes) > 1 else wl.boxes[0].n,
                   "kernel": "peskin4", "scatter": args.scatter, "tile": tile,
                   "tile_autotuned": args.tile == 0, "cuda_graph": True,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "hbm_gbs_step": step_gbs,
        "step_roofline_frac": step_gbs / hbm,
        "step_algorithmic_bytes": {"per_step": ab["step"], "formula": "24N + 12T (x read, v written; u read, "
                                   "f read + written over the touched values)",
                                   "with_F_round_trip": ab["step_with_F"], "hbm_gbs_with_F": step_gbs_F},
        "stage_ms": stage_ms,
        "touched_values": T, "pairs": P,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": NCU_TRAFFIC.get(dom) if args.workload == "C4" else None,
                     "limiter": ({"unit": NCU_LIMITER[dom][0], "frac_of_peak": NCU_LIMITER[dom][1],
                                  "source": "ncu capture on this workload (profiles/)"}
                                 if args.workload == "C4" and dom in NCU_LIMITER else None), "peak_kind": peak_kind,
                     "algorithmic_bytes": ab[dom],
                     "bytes_formula": {"spread+interp": "36N + 12T", "spread": "24N + 4N + 8T",
                                       "interp": "24N + 4N + 4T", "forces": "24N", "bin": "24N + 4N"}.get(dom)},
        "cpu_baseline": cpu,
        "e2e": {"value": job_throughput(N, world, e2e_ms), "unit": "nodes/s", "h2d_bytes_per_step": 12 * N,
                "d2h_bytes_per_step": 12 * N + 8 * red.numel(), "ms_per_step": e2e_ms,
                "api": "ifem_step_coupling_host", "launch": "cuda_graph (captured once, replayed per step)",
                "eager": {"value": job_throughput(N, world, e2e_eager_ms), "ms_per_step": e2e_eager_ms},
                "caller_copies": {"value": job_throughput(N, world, e2e_caller_ms), "ms_per_step": e2e_caller_ms,
                                  "api": "copies around ifem_step_coupling"}},
        "fp64": fp64,
        "extras": extras,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": ck,
        "wall_s_timed": wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
