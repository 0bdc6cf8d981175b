"""Thin ctypes binding of libifem (the C ABI in include/ifem.h).

Functions keep the C names and only marshal arguments: torch tensors become
device pointers, the current torch CUDA stream becomes the cudaStream_t,
status codes become exceptions. Every computation runs in libifem's CUDA
kernels; there is no CPU fallback, and importing this module on a machine
where libifem.so cannot be loaded raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

IFEM_OK = 0
STATUS_NAMES = {
    -1: "IFEM_ERR_ARG", -2: "IFEM_ERR_OOM", -3: "IFEM_ERR_CUDA", -4: "IFEM_ERR_TIMEOUT",
    -5: "IFEM_ERR_INVERTED", -6: "IFEM_ERR_DOMAIN", -7: "IFEM_ERR_CAPACITY",
}
IFEM_FP32, IFEM_FP64 = 0, 1
IFEM_KERNEL_PESKIN4, IFEM_KERNEL_MLS27 = 0, 1
IFEM_SCATTER_DET, IFEM_SCATTER_ATOMIC = 0, 1
IFEM_LAW_NEO_HOOKE, IFEM_LAW_SKALAK = 0, 1
IFEM_SPREAD_DENSITY, IFEM_SPREAD_FORCE, IFEM_SPREAD_OVERWRITE = 0, 1, 2
IFEM_FORCES_ACCUMULATE = 1

# Every entry point declared in include/ifem.h.
EXPORTS = (
    "ifem_config_default", "ifem_ctx_create", "ifem_ctx_destroy", "ifem_last_error", "ifem_sync_status",
    "ifem_ctx_tile", "ifem_stage_times", "ifem_tmpl_create_membrane", "ifem_tmpl_create_solid", "ifem_tmpl_destroy",
    "ifem_grid_create", "ifem_grid_destroy", "ifem_grid_values", "ifem_grid_box_offset",
    "ifem_batch_create", "ifem_batch_destroy", "ifem_batch_nodes", "ifem_batch_instances",
    "ifem_batch_set_origins", "ifem_prepare", "ifem_compute_forces", "ifem_spread", "ifem_interpolate",
    "ifem_reduce", "ifem_step_coupling", "ifem_step_coupling_ab2", "ifem_step_coupling_host", "ifem_force_hvp", "ifem_compute_forces_noalloc",
    "ifem_interpolate_cc", "ifem_fluid_stress_forces", "ifem_ab2_update", "ifem_volumes", "ifem_volume_correct",
    "ifem_indicator_source",
)


class ifem_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("kernel", ctypes.c_int), ("scatter", ctypes.c_int),
                ("tile", ctypes.c_int), ("mls_support", ctypes.c_double), ("device", ctypes.c_int),
                ("profile", ctypes.c_int)]


class ifem_membrane_params(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("C", ctypes.c_double), ("kb", ctypes.c_double),
                ("c0", ctypes.c_double)]


class ifem_solid_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("mu", ctypes.c_double)]


class ifem_fluid_params(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("beta", ctypes.c_double), ("lambda_", ctypes.c_double)]


class ifem_instance_desc(ctypes.Structure):
    _fields_ = [("tmpl", ctypes.c_int), ("box", ctypes.c_int), ("origin", ctypes.c_double * 3)]


class ifem_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("inverted_elements", "domain_errors", "capacity_errors",
                                              "timeouts", "pairs", "active_tiles", "touched_cells")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class IfemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libifem.so (building it first if needed). Raises if it cannot load."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    L = ctypes.CDLL(path)
    p, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "ifem_config_default": (i, [p]),
        "ifem_ctx_create": (i, [p, p]),
        "ifem_ctx_destroy": (i, [p]),
        "ifem_last_error": (ctypes.c_char_p, [p]),
        "ifem_sync_status": (i, [p, p]),
        "ifem_ctx_tile": (i, [p]),
        "ifem_stage_times": (i, [p, p]),
        "ifem_tmpl_create_membrane": (i, [p, i, i, p, p, i, p, p]),
        "ifem_tmpl_create_solid": (i, [p, i, i, p, p, p, p]),
        "ifem_tmpl_destroy": (i, [p]),
        "ifem_grid_create": (i, [p, i, p, p, p]),
        "ifem_grid_destroy": (i, [p]),
        "ifem_grid_values": (i64, [p]),
        "ifem_grid_box_offset": (i64, [p, i]),
        "ifem_batch_create": (i, [p, i, p, i, p, p, p]),
        "ifem_batch_destroy": (i, [p]),
        "ifem_batch_nodes": (i64, [p]),
        "ifem_batch_instances": (i, [p]),
        "ifem_batch_set_origins": (i, [p, p]),
        "ifem_prepare": (i, [p, p, p, p]),
        "ifem_compute_forces": (i, [p, p, p, p, p]),
        "ifem_spread": (i, [p, p, p, p, p, p, i, p]),
        "ifem_interpolate": (i, [p, p, p, p, p, p, p]),
        "ifem_reduce": (i, [p, p, p, p, p, p, p]),
        "ifem_step_coupling": (i, [p, p, p, p, p, p, p, p, p, i, p]),
        "ifem_step_coupling_ab2": (i, [p, p, p, p, p, p, p, p, p, i, p, d, p, p]),
        "ifem_step_coupling_host": (i, [p, p, p, p, p, p, p, p, p, p, p, p, i, p]),
        "ifem_force_hvp": (i, [p, p, p, p, p, p]),
        "ifem_compute_forces_noalloc": (i, [p, p, p, p, p]),
        "ifem_interpolate_cc": (i, [p, p, p, p, i, p, p, p]),
        "ifem_fluid_stress_forces": (i, [p, p, p, p, p, p, p, i, p]),
        "ifem_ab2_update": (i, [p, p, p, p, p, d, p]),
        "ifem_volumes": (i, [p, p, p, p, p]),
        "ifem_volume_correct": (i, [p, p, p, p, p, p]),
        "ifem_indicator_source": (i, [p, p, p, p, p, i, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(ctx, rc: int):
    if rc != IFEM_OK:
        msg = load().ifem_last_error(ctx).decode() if ctx else ""
        raise IfemError(rc, msg)
    return rc


def _ptr(t) -> Optional[int]:
    """Device (or host numpy) pointer of a tensor/array; None passes NULL."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------- C names
def ifem_ctx_create(precision: int = IFEM_FP32, kernel: int = IFEM_KERNEL_PESKIN4,
                    scatter: int = IFEM_SCATTER_DET, tile: int = 0, mls_support: float = 0.0,
                    device: int = 0, profile: int = 0):
    L = load()
    cfg = ifem_config()
    L.ifem_config_default(ctypes.byref(cfg))
    cfg.precision, cfg.kernel, cfg.scatter, cfg.tile = precision, kernel, scatter, tile
    cfg.mls_support, cfg.device, cfg.profile = mls_support, device, profile
    h = ctypes.c_void_p()
    rc = L.ifem_ctx_create(ctypes.byref(cfg), ctypes.byref(h))
    if rc != IFEM_OK:
        raise IfemError(rc, "ifem_ctx_create failed")
    return h


def ifem_ctx_tile(ctx) -> int:
    return int(load().ifem_ctx_tile(ctx))


def ifem_stage_times(ctx):
    ms = (ctypes.c_double * 5)()
    _check(ctx, load().ifem_stage_times(ctx, ms))
    return dict(zip(("bin", "forces", "spread", "interp", "reduce"), list(ms)))


def ifem_ctx_destroy(ctx):
    return _check(None, load().ifem_ctx_destroy(ctx))


def ifem_sync_status(ctx, raise_on_error: bool = True):
    st = ifem_stats()
    rc = load().ifem_sync_status(ctx, ctypes.byref(st))
    if raise_on_error:
        _check(ctx, rc)
    return rc, st.as_dict()


def ifem_tmpl_create_membrane(ctx, tris: np.ndarray, X_ref: np.ndarray, law: int, mu: float, C: float = 1.0,
                              kb: float = 0.0, c0: float = 0.0):
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    X_ref = np.ascontiguousarray(X_ref, dtype=np.float64)
    prm = ifem_membrane_params(mu, C, kb, c0)
    h = ctypes.c_void_p()
    _check(ctx, load().ifem_tmpl_create_membrane(ctx, X_ref.shape[0], tris.shape[0], _ptr(tris), _ptr(X_ref),
                                                 law, ctypes.byref(prm), ctypes.byref(h)))
    return h


def ifem_tmpl_create_solid(ctx, tets: np.ndarray, X_ref: np.ndarray, lam: float, mu: float):
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    X_ref = np.ascontiguousarray(X_ref, dtype=np.float64)
    prm = ifem_solid_params(lam, mu)
    h = ctypes.c_void_p()
    _check(ctx, load().ifem_tmpl_create_solid(ctx, X_ref.shape[0], tets.shape[0], _ptr(tets), _ptr(X_ref),
                                              ctypes.byref(prm), ctypes.byref(h)))
    return h


def ifem_tmpl_destroy(t):
    return load().ifem_tmpl_destroy(t)


def ifem_grid_create(ctx, n: Sequence[int], L: Sequence[float]):
    n = np.ascontiguousarray(n, dtype=np.int32)
    Ls = np.ascontiguousarray(L, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(ctx, load().ifem_grid_create(ctx, n.shape[0], _ptr(n), _ptr(Ls), ctypes.byref(h)))
    return h


def ifem_grid_destroy(g):
    return load().ifem_grid_destroy(g)


def ifem_grid_values(g) -> int:
    return int(load().ifem_grid_values(g))


def ifem_grid_box_offset(g, b: int) -> int:
    return int(load().ifem_grid_box_offset(g, b))


def ifem_batch_create(ctx, tmpls: Sequence, inst: Sequence[tuple], grid):
    """inst: sequence of (template index, box index, origin (3,))."""
    arr_t = (ctypes.c_void_p * len(tmpls))(*[t.value for t in tmpls])
    descs = (ifem_instance_desc * max(1, len(inst)))()
    for k, (ti, bi, org) in enumerate(inst):
        descs[k].tmpl, descs[k].box = int(ti), int(bi)
        for a in range(3):
            descs[k].origin[a] = float(org[a])
    h = ctypes.c_void_p()
    _check(ctx, load().ifem_batch_create(ctx, len(tmpls), arr_t, len(inst), descs, grid, ctypes.byref(h)))
    return h


def ifem_batch_destroy(b):
    return load().ifem_batch_destroy(b)


def ifem_batch_nodes(b) -> int:
    return int(load().ifem_batch_nodes(b))


def ifem_batch_instances(b) -> int:
    return int(load().ifem_batch_instances(b))


def ifem_batch_set_origins(ctx, b, origins: np.ndarray):
    o = np.ascontiguousarray(origins, dtype=np.float64)
    return _check(ctx, load().ifem_batch_set_origins(b, _ptr(o)))


def ifem_prepare(ctx, b, x=None, stream=None):
    return _check(ctx, load().ifem_prepare(ctx, b, _ptr(x), _stream(stream)))


def ifem_compute_forces(ctx, b, x, F, stream=None):
    return _check(ctx, load().ifem_compute_forces(ctx, b, _ptr(x), _ptr(F), _stream(stream)))


def ifem_compute_forces_noalloc(ctx, b, x, F, stream=None):
    """ifem_compute_forces without allocation in the call (fixed 32 MiB device scratch)."""
    return _check(ctx, load().ifem_compute_forces_noalloc(ctx, b, _ptr(x), _ptr(F), _stream(stream)))


def ifem_spread(ctx, b, g, x, F, f, flags: int = 0, stream=None):
    return _check(ctx, load().ifem_spread(ctx, b, g, _ptr(x), _ptr(F), _ptr(f), flags, _stream(stream)))


def ifem_interpolate(ctx, b, g, u, x, v, stream=None):
    return _check(ctx, load().ifem_interpolate(ctx, b, g, _ptr(u), _ptr(x), _ptr(v), _stream(stream)))


def ifem_interpolate_cc(ctx, b, g, field, ncomp: int, x, out, stream=None):
    return _check(ctx, load().ifem_interpolate_cc(ctx, b, g, _ptr(field), int(ncomp), _ptr(x), _ptr(out),
                                                  _stream(stream)))


def ifem_fluid_stress_forces(ctx, b, x, u, C, eta: float, beta: float, lam: float, F, flags: int = 0,
                             stream=None):
    prm = ifem_fluid_params(eta, beta, lam)
    return _check(ctx, load().ifem_fluid_stress_forces(ctx, b, _ptr(x), _ptr(u), _ptr(C), ctypes.byref(prm),
                                                       _ptr(F), flags, _stream(stream)))


def ifem_indicator_source(ctx, b, g, x, G, flags: int = 0, stream=None):
    return _check(ctx, load().ifem_indicator_source(ctx, b, g, _ptr(x), _ptr(G), flags, _stream(stream)))


def ifem_ab2_update(ctx, b, x, v, v_prev, dt: float, stream=None):
    return _check(ctx, load().ifem_ab2_update(ctx, b, _ptr(x), _ptr(v), _ptr(v_prev), float(dt), _stream(stream)))


def ifem_volumes(ctx, b, x, vol, stream=None):
    return _check(ctx, load().ifem_volumes(ctx, b, _ptr(x), _ptr(vol), _stream(stream)))


def ifem_volume_correct(ctx, b, x, V0, lam=None, stream=None):
    return _check(ctx, load().ifem_volume_correct(ctx, b, _ptr(x), _ptr(V0), _ptr(lam), _stream(stream)))


def ifem_reduce(ctx, b, x, F, v, red, stream=None):
    return _check(ctx, load().ifem_reduce(ctx, b, _ptr(x), _ptr(F), _ptr(v), _ptr(red), _stream(stream)))


def ifem_step_coupling(ctx, b, g, x, u, F, f, v, red=None, flags: int = 0, stream=None):
    return _check(ctx, load().ifem_step_coupling(ctx, b, g, _ptr(x), _ptr(u), _ptr(F), _ptr(f), _ptr(v),
                                                 _ptr(red), flags, _stream(stream)))


def ifem_step_coupling_ab2(ctx, b, g, x, u, F, f, v, red, flags: int, v_prev, dt: float, x_new, stream=None):
    return _check(ctx, load().ifem_step_coupling_ab2(ctx, b, g, _ptr(x), _ptr(u), _ptr(F), _ptr(f), _ptr(v),
                                                     _ptr(red), flags, _ptr(v_prev), float(dt), _ptr(x_new),
                                                     _stream(stream)))


def ifem_step_coupling_host(ctx, b, g, x_host, x, u, F, f, v, v_host, red=None, red_host=None, flags: int = 0,
                            stream=None):
    """x_host, v_host, red_host: CPU tensors (pinned for overlap); the rest device tensors."""
    for t in (x_host, v_host, red_host):
        if t is not None and getattr(t, "is_cuda", False):
            raise ValueError("ifem_step_coupling_host: x_host, v_host and red_host must be host tensors")
    return _check(ctx, load().ifem_step_coupling_host(ctx, b, g, _ptr(x_host), _ptr(x), _ptr(u), _ptr(F), _ptr(f),
                                                      _ptr(v), _ptr(v_host), _ptr(red), _ptr(red_host), flags,
                                                      _stream(stream)))


def ifem_force_hvp(ctx, b, x, w, Hw, stream=None):
    return _check(ctx, load().ifem_force_hvp(ctx, b, _ptr(x), _ptr(w), _ptr(Hw), _stream(stream)))


# ---------------------------------------------------------------- workload helper
class Coupler:
    """Owns the libifem handles and device buffers for one workload.

    Built from an ``ifem_workloads.Workload``: one template per workload
    template, one box per workload box, instances in workload order. Node
    arrays are (3, N) tensors (SoA); grid fields are 1-D tensors of
    ``ifem_grid_values`` entries.
    """

    def __init__(self, wl, precision: int = IFEM_FP32, kernel: int = IFEM_KERNEL_PESKIN4,
                 scatter: int = IFEM_SCATTER_DET, tile: int = 0, device: int = 0, profile: int = 0):
        import torch
        self.torch = torch
        self.wl = wl
        self.precision = precision
        self.dtype = torch.float64 if precision == IFEM_FP64 else torch.float32
        self.device = torch.device("cuda", device)
        self.ctx = ifem_ctx_create(precision, kernel, scatter, tile, 0.0, device, profile)
        self.tmpls = []
        for tm in wl.templates:
            if tm.kind == "membrane":
                law = IFEM_LAW_NEO_HOOKE if tm.law == "nh" else IFEM_LAW_SKALAK
                self.tmpls.append(ifem_tmpl_create_membrane(self.ctx, tm.elems, tm.X, law, tm.mu, tm.C, tm.kb))
            else:
                self.tmpls.append(ifem_tmpl_create_solid(self.ctx, tm.elems, tm.X, tm.lam, tm.mu))
        self.grid = ifem_grid_create(self.ctx, [bx.n for bx in wl.boxes], [bx.L for bx in wl.boxes])
        self.batch = ifem_batch_create(self.ctx, self.tmpls, [(i.tmpl, i.box, i.origin) for i in wl.instances],
                                       self.grid)
        self.N = ifem_batch_nodes(self.batch)
        self.G = ifem_grid_values(self.grid)
        self.box_off = [ifem_grid_box_offset(self.grid, b) for b in range(len(wl.boxes))]

    # host <-> device helpers (layout conversions only)
    def nodes_to_device(self, a: np.ndarray):
        """(N, 3) host array -> (3, N) device tensor of the context precision."""
        t = self.torch.as_tensor(np.ascontiguousarray(np.asarray(a).T), dtype=self.dtype)
        return t.to(self.device).contiguous()

    def nodes_to_host(self, t) -> np.ndarray:
        return t.detach().cpu().double().numpy().T.copy()

    def grid_to_device(self, fields: Sequence[np.ndarray]):
        """per-box (3, n, n, n) host arrays -> one flat device field."""
        flat = np.concatenate([np.asarray(f).reshape(-1) for f in fields])
        return self.torch.as_tensor(flat, dtype=self.dtype).to(self.device)

    def grid_to_host(self, t):
        h = t.detach().cpu().double().numpy()
        out = []
        for b, bx in enumerate(self.wl.boxes):
            n = bx.n
            out.append(h[self.box_off[b]: self.box_off[b] + 3 * n ** 3].reshape(3, n, n, n))
        return out

    def empty_nodes(self):
        return self.torch.empty((3, self.N), dtype=self.dtype, device=self.device)

    def zeros_grid(self):
        return self.torch.zeros(self.G, dtype=self.dtype, device=self.device)

    def close(self):
        if self.batch is not None:
            ifem_batch_destroy(self.batch)
            ifem_grid_destroy(self.grid)
            for t in self.tmpls:
                ifem_tmpl_destroy(t)
            ifem_ctx_destroy(self.ctx)
            self.batch = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
