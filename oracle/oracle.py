"""ctypes binding of the plain FP64 CPU oracle (``ifem_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the benchmark's CPU-baseline leg; never by the product path.

Besides thin wrappers of the C functions, ``oracle_step`` evaluates one whole
coupling step (element forces + bending, spreading, interpolation and the
FP64 conservation sums) for a workload from ``ifem_workloads``, following the
paper's Algorithm steps 1, 2 and 4 in that order.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ifem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libifem_oracle.so")
_lib = None
_lock = threading.Lock()

KERNEL_PESKIN4 = 0
KERNEL_MLS27 = 1
LAW_NH = 0
LAW_SKALAK = 1
MLS_SUPPORT = math.sqrt(3.0)


def build(force: bool = False) -> str:
    """Compile the oracle with FMA contraction off (plain IEEE FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["cc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            L.ifo_phi4.restype = d
            L.ifo_phi4.argtypes = [d]
            L.ifo_mls_w.restype = d
            L.ifo_mls_w.argtypes = [d]
            L.ifo_mls_weights.restype = i
            L.ifo_mls_weights.argtypes = [p, d, p, p]
            L.ifo_spread.restype = i
            L.ifo_spread.argtypes = [i, i, d, i, p, p, p, i, d]
            L.ifo_interp.restype = i
            L.ifo_interp.argtypes = [i, i, d, i, p, p, p, d]
            L.ifo_membrane_reference.argtypes = [i, p, p, p, p]
            L.ifo_membrane_forces.argtypes = [i, d, d, i, i, p, p, p, p, p]
            L.ifo_membrane_energy.restype = d
            L.ifo_membrane_energy.argtypes = [i, d, d, i, p, p, p, p]
            L.ifo_membrane_hvp.argtypes = [i, d, d, i, i, p, p, p, p, p, p]
            L.ifo_tet_reference.argtypes = [i, p, p, p, p]
            L.ifo_tet_forces.restype = i
            L.ifo_tet_forces.argtypes = [d, d, i, i, p, p, p, p, p]
            L.ifo_tet_energy.restype = d
            L.ifo_tet_energy.argtypes = [d, d, i, p, p, p, p]
            L.ifo_tet_hvp.argtypes = [d, d, i, i, p, p, p, p, p, p]
            L.ifo_curvatures.argtypes = [i, i, p, p, p, p, p, p, p]
            L.ifo_bending_forces.argtypes = [d, d, i, i, p, p, p]
            L.ifo_bending_energy.restype = d
            L.ifo_bending_energy.argtypes = [d, d, i, i, p, p]
            L.ifo_volume.restype = d
            L.ifo_volume.argtypes = [i, p, p]
            L.ifo_interp_cc.restype = i
            L.ifo_interp_cc.argtypes = [i, i, d, i, p, p, i, p, d]
            L.ifo_tet_fluid_forces.argtypes = [d, d, d, i, i, p, p, p, p, p, p, p]
            L.ifo_tet_volume.restype = d
            L.ifo_tet_volume.argtypes = [i, p, p]
            L.ifo_ab2.argtypes = [i, p, p, p, d]
            L.ifo_volume_correction.restype = i
            L.ifo_volume_correction.argtypes = [i, i, p, p, d, p, p]
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------ kernels
def phi4(r: float) -> float:
    return lib().ifo_phi4(float(r))


def mls_w(r: float) -> float:
    return lib().ifo_mls_w(float(r))


def mls_weights(s, support: float = MLS_SUPPORT):
    s = _f64(s)
    base = np.zeros(3, dtype=np.int32)
    w = np.zeros(27)
    if lib().ifo_mls_weights(_ptr(s), support, _ptr(base), _ptr(w)) != 0:
        raise FloatingPointError("singular MLS moment matrix")
    return base, w


# ------------------------------------------------------------ transfer
def spread(x_abs, F, n: int, L: float, kernel: int = KERNEL_PESKIN4, density: bool = True,
           f0=None, support: float = MLS_SUPPORT) -> np.ndarray:
    """S*: returns f0 + spread (3, n, n, n). x_abs, F: (N, 3)."""
    x_abs, F = _f64(x_abs), _f64(F)
    f = np.zeros((3, n, n, n)) if f0 is None else _f64(f0).copy()
    rc = lib().ifo_spread(kernel, n, float(L), x_abs.shape[0], _ptr(x_abs), _ptr(F), _ptr(f),
                          int(density), support)
    if rc != 0:
        raise FloatingPointError("singular MLS moment matrix")
    return f


def interp(x_abs, u, n: int, L: float, kernel: int = KERNEL_PESKIN4,
           support: float = MLS_SUPPORT) -> np.ndarray:
    """S: returns v (N, 3) interpolated from u (3, n, n, n)."""
    x_abs, u = _f64(x_abs), _f64(u)
    v = np.zeros_like(x_abs)
    rc = lib().ifo_interp(kernel, n, float(L), x_abs.shape[0], _ptr(x_abs), _ptr(u), _ptr(v), support)
    if rc != 0:
        raise FloatingPointError("singular MLS moment matrix")
    return v


def interp_cc(x_abs, field, n: int, L: float, kernel: int = KERNEL_PESKIN4,
              support: float = MLS_SUPPORT) -> np.ndarray:
    """S of a cell-centred field (ncomp, n, n, n): returns (N, ncomp)."""
    x_abs, field = _f64(x_abs), _f64(field)
    ncomp = field.shape[0]
    out = np.zeros((x_abs.shape[0], ncomp))
    rc = lib().ifo_interp_cc(kernel, n, float(L), x_abs.shape[0], _ptr(x_abs), _ptr(field), ncomp, _ptr(out),
                             support)
    if rc != 0:
        raise FloatingPointError("singular MLS moment matrix")
    return out


# ------------------------------------------------------------ membranes
def membrane_reference(tri, X):
    tri, X = _i32(tri), _f64(X)
    Dminv = np.zeros((tri.shape[0], 4))
    A0 = np.zeros(tri.shape[0])
    lib().ifo_membrane_reference(tri.shape[0], _ptr(tri), _ptr(X), _ptr(Dminv), _ptr(A0))
    return Dminv, A0


def _law(law) -> int:
    if isinstance(law, str):
        return {"nh": LAW_NH, "skalak": LAW_SKALAK}[law]
    return int(law)


def membrane_forces(law, mu, C, tri, X, x, ref=None):
    tri, x = _i32(tri), _f64(x)
    Dminv, A0 = membrane_reference(tri, X) if ref is None else ref
    F = np.zeros_like(x)
    lib().ifo_membrane_forces(_law(law), mu, C, x.shape[0], tri.shape[0], _ptr(tri), _ptr(Dminv),
                              _ptr(A0), _ptr(x), _ptr(F))
    return F


def membrane_energy(law, mu, C, tri, X, x, ref=None) -> float:
    tri, x = _i32(tri), _f64(x)
    Dminv, A0 = membrane_reference(tri, X) if ref is None else ref
    return lib().ifo_membrane_energy(_law(law), mu, C, tri.shape[0], _ptr(tri), _ptr(Dminv),
                                     _ptr(A0), _ptr(x))


def membrane_hvp(law, mu, C, tri, X, x, w, ref=None):
    tri, x, w = _i32(tri), _f64(x), _f64(w)
    Dminv, A0 = membrane_reference(tri, X) if ref is None else ref
    Hw = np.zeros_like(x)
    lib().ifo_membrane_hvp(_law(law), mu, C, x.shape[0], tri.shape[0], _ptr(tri), _ptr(Dminv),
                           _ptr(A0), _ptr(x), _ptr(w), _ptr(Hw))
    return Hw


# ------------------------------------------------------------ solids
def tet_reference(tet, X):
    tet, X = _i32(tet), _f64(X)
    Dminv = np.zeros((tet.shape[0], 9))
    V0 = np.zeros(tet.shape[0])
    lib().ifo_tet_reference(tet.shape[0], _ptr(tet), _ptr(X), _ptr(Dminv), _ptr(V0))
    return Dminv, V0


def tet_forces(lam, mu, tet, X, x, ref=None, return_inverted=False):
    tet, x = _i32(tet), _f64(x)
    Dminv, V0 = tet_reference(tet, X) if ref is None else ref
    F = np.zeros_like(x)
    inv = lib().ifo_tet_forces(lam, mu, x.shape[0], tet.shape[0], _ptr(tet), _ptr(Dminv), _ptr(V0),
                               _ptr(x), _ptr(F))
    return (F, inv) if return_inverted else F


def tet_fluid_forces(eta, beta, lam_relax, tet, X, x, u, C=None, ref=None):
    """Newtonian (+ polymer, if C (N, 6) is given) fluid-stress nodal forces of a solid."""
    tet, x, u = _i32(tet), _f64(x), _f64(u)
    Dminv, V0 = tet_reference(tet, X) if ref is None else ref
    Cp = None if C is None else _f64(C)
    F = np.zeros_like(x)
    lib().ifo_tet_fluid_forces(eta, beta, lam_relax, x.shape[0], tet.shape[0], _ptr(tet), _ptr(Dminv), _ptr(V0),
                               _ptr(x), _ptr(u), None if Cp is None else _ptr(Cp), _ptr(F))
    return F


def tet_energy(lam, mu, tet, X, x, ref=None) -> float:
    tet, x = _i32(tet), _f64(x)
    Dminv, V0 = tet_reference(tet, X) if ref is None else ref
    return lib().ifo_tet_energy(lam, mu, tet.shape[0], _ptr(tet), _ptr(Dminv), _ptr(V0), _ptr(x))


def tet_hvp(lam, mu, tet, X, x, w, ref=None):
    tet, x, w = _i32(tet), _f64(x), _f64(w)
    Dminv, V0 = tet_reference(tet, X) if ref is None else ref
    Hw = np.zeros_like(x)
    lib().ifo_tet_hvp(lam, mu, x.shape[0], tet.shape[0], _ptr(tet), _ptr(Dminv), _ptr(V0), _ptr(x),
                      _ptr(w), _ptr(Hw))
    return Hw


# ------------------------------------------------------------ bending
def curvatures(tri, x):
    tri, x = _i32(tri), _f64(x)
    nn = x.shape[0]
    A, kH, kG = np.zeros(nn), np.zeros(nn), np.zeros(nn)
    n, K = np.zeros((nn, 3)), np.zeros((nn, 3))
    lib().ifo_curvatures(nn, tri.shape[0], _ptr(tri), _ptr(x), _ptr(A), _ptr(n), _ptr(kH), _ptr(kG),
                         _ptr(K))
    return {"A": A, "n": n, "kH": kH, "kG": kG, "K": K}


def bending_forces(kb, tri, x, c0: float = 0.0):
    tri, x = _i32(tri), _f64(x)
    F = np.zeros_like(x)
    lib().ifo_bending_forces(kb, c0, x.shape[0], tri.shape[0], _ptr(tri), _ptr(x), _ptr(F))
    return F


def bending_energy(kb, tri, x, c0: float = 0.0) -> float:
    tri, x = _i32(tri), _f64(x)
    return lib().ifo_bending_energy(kb, c0, x.shape[0], tri.shape[0], _ptr(tri), _ptr(x))


def volume(tri, x) -> float:
    tri, x = _i32(tri), _f64(x)
    return lib().ifo_volume(tri.shape[0], _ptr(tri), _ptr(x))


def tet_volume(tet, x) -> float:
    tet, x = _i32(tet), _f64(x)
    return lib().ifo_tet_volume(tet.shape[0], _ptr(tet), _ptr(x))


def ab2(x, v, vp, dt: float):
    """Adams-Bashforth step: returns x + dt (3/2 v - 1/2 vp)."""
    out = _f64(x).copy()
    v, vp = _f64(v), _f64(vp)
    lib().ifo_ab2(out.size, _ptr(out), _ptr(v), _ptr(vp), float(dt))
    return out


def volume_correction(tri, x, V0: float):
    """Volume-corrected positions, the displacement directions alpha and Lambda."""
    tri = _i32(tri)
    out = _f64(x).copy()
    alpha = np.zeros_like(out)
    lam = ctypes.c_double(0.0)
    it = lib().ifo_volume_correction(out.shape[0], tri.shape[0], _ptr(tri), _ptr(out), float(V0), _ptr(alpha),
                                     ctypes.byref(lam))
    if it < 0:
        raise FloatingPointError("volume correction: Newton did not converge")
    return out, alpha, lam.value


# ------------------------------------------------------------ whole step
def template_forces(tm, x_local):
    """Elastic (+ bending) nodal forces of one particle: F = F_el + F_be (Algorithm step 1)."""
    if tm.kind == "membrane":
        F = membrane_forces(tm.law, tm.mu, tm.C, tm.elems, tm.X, x_local)
        if tm.kb != 0.0:
            F = F + bending_forces(tm.kb, tm.elems, x_local)
        return F
    return tet_forces(tm.lam, tm.mu, tm.elems, tm.X, x_local)


def fsum3(a: np.ndarray) -> np.ndarray:
    """Correctly rounded FP64 sum of the rows of an (N, 3) array."""
    return np.array([math.fsum(a[:, c]) for c in range(3)])


def oracle_step(wl, x_local=None, kernel: int = KERNEL_PESKIN4, density: bool = True,
                f0=None, instances=None, with_reductions: bool = True):
    """One coupling step on the CPU in FP64.

    x_local: optional (N, 3) local positions (e.g. the FP32-rounded values the
    GPU sees); defaults to the workload's own. Returns dict with F (N,3),
    f (list per box of (3,n,n,n)), v (N,3), and per-particle / per-box sums.
    instances: optional subset of instance indices (for timing samples).
    """
    if x_local is None:
        x_local = wl.x_local_all()
    x_local = _f64(x_local)
    off = wl.node_offsets()
    sel = range(len(wl.instances)) if instances is None else instances
    F = np.zeros_like(x_local)
    for ii in sel:
        inst = wl.instances[ii]
        a, b = off[ii], off[ii + 1]
        F[a:b] = template_forces(wl.templates[inst.tmpl], x_local[a:b])
    out = {"F": F, "f": [], "v": np.zeros_like(x_local)}
    x_abs = np.zeros_like(x_local)
    for ii in sel:
        inst = wl.instances[ii]
        a, b = off[ii], off[ii + 1]
        x_abs[a:b] = inst.origin[None, :] + x_local[a:b]
    for bi, box in enumerate(wl.boxes):
        rows = np.concatenate([np.arange(off[ii], off[ii + 1]) for ii in sel
                               if wl.instances[ii].box == bi] or [np.zeros(0, dtype=np.int64)])
        base = None if f0 is None else f0[bi]
        out["f"].append(spread(x_abs[rows], F[rows], box.n, box.L, kernel, density, f0=base))
        if rows.size:
            out["v"][rows] = interp(x_abs[rows], wl.u[bi], box.n, box.L, kernel)
    if with_reductions:
        out["red"] = reductions(wl, x_local, F, out["v"], sel)
    return out


def area_normals(tri, x):
    """n_k A_k of every vertex of a membrane: the unit vertex normal times the
    mixed Voronoi area of the bending operators (Sec. "Variable Viscosity
    Implementation" names n_k and A_k without defining them)."""
    c = curvatures(tri, x)
    return c["n"] * c["A"][:, None]


def indicator_source(wl, x_local=None, kernel: int = KERNEL_PESKIN4, density: bool = True, f0=None):
    """Source of the indicator-function Poisson equation (Sec. "Variable
    Viscosity Implementation"): G_J = sum_k n_k A_k phi(x_J - x_k) over the
    membrane nodes of each box, spread like a force (S*) onto the three MAC
    lattices. Returns a list per box of (3, n, n, n)."""
    if x_local is None:
        x_local = wl.x_local_all()
    x_local = _f64(x_local)
    off = wl.node_offsets()
    nA = np.zeros_like(x_local)
    x_abs = np.zeros_like(x_local)
    for ii, inst in enumerate(wl.instances):
        a, b = off[ii], off[ii + 1]
        tm = wl.templates[inst.tmpl]
        if tm.kind == "membrane":
            nA[a:b] = area_normals(tm.elems, x_local[a:b])
        x_abs[a:b] = inst.origin[None, :] + x_local[a:b]
    out = []
    for bi, box in enumerate(wl.boxes):
        rows = np.concatenate([np.arange(off[ii], off[ii + 1]) for ii, inst in enumerate(wl.instances)
                               if inst.box == bi] or [np.zeros(0, dtype=np.int64)])
        base = None if f0 is None else f0[bi]
        out.append(spread(x_abs[rows], nA[rows], box.n, box.L, kernel, density, f0=base))
    return out


def reductions(wl, x_local, F, v, sel=None):
    """Per-particle FP64 sums: centroid c, sum F, sum (x - c) x F, sum v (correctly rounded)."""
    off = wl.node_offsets()
    sel = range(len(wl.instances)) if sel is None else sel
    rows = []
    for ii in sel:
        a, b = off[ii], off[ii + 1]
        xl, Fk, vk = x_local[a:b], F[a:b], v[a:b]
        c = fsum3(xl) / (b - a)
        r = xl - c
        tq = np.cross(r, Fk)
        rows.append(np.concatenate([c, fsum3(Fk), fsum3(tq), fsum3(vk)]))
    return np.array(rows)
