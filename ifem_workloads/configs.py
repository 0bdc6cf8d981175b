"""The five seeded synthetic coupling-step workloads.

Every workload is a set of structure *templates* (reference mesh plus
material constants, shared by all particles of that type), a list of particle
*instances* (template, box, FP64 origin, current node positions as offsets
from that origin), a list of periodic *boxes* (cells per side n, side L) and
one MAC velocity field per box. Sizes are in box units unless a name says
"cells". All randomness comes from numpy's PCG64 seeded with 1000 + index.

C1  single spherical capsule (642 nodes), 64^3, neo-Hookean or Skalak
C2  single biconcave RBC (2562 nodes, D = 20 cells), 128^3, Skalak C=100 + bending
C3  tetrahedral ball (4096 nodes / 20250 tets, R = 12 cells), 128^3, solid NH nu=0.45
C4  500 RBC + 100 platelets at ~20% volume fraction in 256^3
C5  64 boxes (n ~ U{32..96}) with 1-20 mixed particles each
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import meshes
from .fields import fourier_modes, sample_on_mac

KAPPA_B_HAT = 0.01          # dimensionless bending modulus k_b / (R_p mu_p)
SKALAK_C = 100.0            # mu_D / mu_p for red cells
PLT_LAMBDA_OVER_MU = 50.0   # lambda_p / mu_p of deformable platelets
CA_PLT_OVER_CA_RBC = 0.0421 # platelet capillary number at Ca_RBC = 1
RP_OVER_D_RBC = 2.82 / 8.0  # effective RBC radius over diameter


@dataclasses.dataclass
class Template:
    kind: str                 # "membrane" | "solid"
    X: np.ndarray             # (n, 3) float64 stress-free reference positions
    elems: np.ndarray         # (E, 3) or (E, 4) int32
    law: str                  # "nh" | "skalak" (membranes) | "nh" (solids)
    mu: float = 1.0           # shear modulus (membrane: areal)
    C: float = 1.0            # mu_D / mu (Skalak only)
    kb: float = 0.0           # bending modulus (membranes)
    lam: float = 0.0          # Lame lambda (solids)
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return self.X.shape[0]

    @property
    def n_elems(self) -> int:
        return self.elems.shape[0]


@dataclasses.dataclass
class Instance:
    tmpl: int
    box: int
    origin: np.ndarray        # (3,) float64
    x_local: np.ndarray       # (n, 3) float64 current positions minus origin


@dataclasses.dataclass
class Box:
    n: int
    L: float = 1.0

    @property
    def h(self) -> float:
        return self.L / self.n


@dataclasses.dataclass
class Workload:
    name: str
    templates: List[Template]
    instances: List[Instance]
    boxes: List[Box]
    u: List[np.ndarray]       # per box (3, n, n, n) float64 [d, k, j, i]
    seed: int
    note: str = ""

    @property
    def n_nodes(self) -> int:
        return sum(self.templates[i.tmpl].n_nodes for i in self.instances)

    def node_offsets(self) -> np.ndarray:
        off = [0]
        for i in self.instances:
            off.append(off[-1] + self.templates[i.tmpl].n_nodes)
        return np.asarray(off, dtype=np.int64)

    def x_local_all(self, dtype=np.float64) -> np.ndarray:
        """(N, 3) concatenated local positions, rounded to dtype."""
        if not self.instances:
            return np.zeros((0, 3), dtype=dtype)
        return np.concatenate([i.x_local for i in self.instances]).astype(dtype)

    def origins_per_node(self) -> np.ndarray:
        if not self.instances:
            return np.zeros((0, 3))
        return np.concatenate([np.broadcast_to(i.origin, (self.templates[i.tmpl].n_nodes, 3))
                               for i in self.instances])


def _jitter(rng, shape, sigma):
    return rng.normal(0.0, sigma, size=shape)


# ---------------------------------------------------------------- C1
def config1(law: str = "nh", seed: int = 1001, n: int = 64) -> Workload:
    """Single spherical capsule, 642 nodes, R = 0.15, stretch (1.2, 0.9, 0.9) + N(0, 1e-3)."""
    rng = np.random.default_rng(seed)
    v, f = meshes.icosphere(3)
    c = np.array([0.5, 0.5, 0.5])
    X = 0.15 * v
    S = np.diag([1.2, 0.9, 0.9])
    x = X @ S.T + _jitter(rng, X.shape, 1e-3)
    tm = Template("membrane", X, f, law, mu=1.0, C=1.0, kb=0.0, name=f"capsule642-{law}")
    u = sample_on_mac(fourier_modes(rng), n, 1.0)
    return Workload("C1", [tm], [Instance(0, 0, c.copy(), x)], [Box(n, 1.0)], [u], seed,
                    note=f"capsule 642 nodes, {law}, {n}^3")


# ---------------------------------------------------------------- C2
def rbc_template(D: float, level: int = 4, mu: float = 1.0) -> Template:
    X, f = meshes.rbc_surface(level, D)
    kb = KAPPA_B_HAT * (RP_OVER_D_RBC * D) * mu
    return Template("membrane", X, f, "skalak", mu=mu, C=SKALAK_C, kb=kb, name="rbc2562")


def deform_rbc(rng, X: np.ndarray, D: float) -> np.ndarray:
    R = meshes.random_rotation(rng)
    S = np.diag(1.0 + 0.1 * rng.standard_normal(3))
    return X @ (R @ S).T + _jitter(rng, X.shape, 1e-3 * D)


def config2(seed: int = 1002, n: int = 128) -> Workload:
    """Single RBC, D = 20 cells, Skalak C = 100, kappa_b = 0.01, 128^3."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    D = 20.0 * h
    tm = rbc_template(D)
    c = np.array([0.5, 0.5, 0.5]) + rng.uniform(-0.5, 0.5, 3) * h
    x = deform_rbc(rng, tm.X, D)
    u = sample_on_mac(fourier_modes(rng), n, 1.0)
    return Workload("C2", [tm], [Instance(0, 0, c, x)], [Box(n, 1.0)], [u], seed,
                    note="RBC 2562 nodes, Skalak C=100 + bending, 128^3")


# ---------------------------------------------------------------- C3
def ball_template(m: int, radius: float, mu: float = 1.0, nu: float = 0.45,
                  semi_axes: Optional[np.ndarray] = None, lam: Optional[float] = None) -> Template:
    X, t = meshes.kuhn_ball(m, radius)
    if semi_axes is not None:
        X = X * (np.asarray(semi_axes) / radius)
    if lam is None:
        lam = mu * 2.0 * nu / (1.0 - 2.0 * nu)
    assert (meshes.tet_signed_volumes(X, t) > 0).all()
    return Template("solid", X, t, "nh", mu=mu, lam=lam, name=f"ball{m}")


def config3(seed: int = 1003, n: int = 128) -> Workload:
    """Solid ball R = 12 cells (4096 nodes / 20250 tets), affine + sinusoidal deformation."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    tm = ball_template(16, 12.0 * h)
    c = np.array([0.5, 0.5, 0.5]) + rng.uniform(-0.5, 0.5, 3) * h
    A = np.eye(3) + 0.1 * rng.standard_normal((3, 3))
    q = rng.standard_normal(3)
    q /= np.linalg.norm(q)
    a = rng.standard_normal(3)
    a /= np.linalg.norm(a)
    X = tm.X
    x = X @ A.T + 0.5 * h * np.sin(2.0 * np.pi * (X @ q) / (24.0 * h))[:, None] * a
    u = sample_on_mac(fourier_modes(rng), n, 1.0)
    return Workload("C3", [tm], [Instance(0, 0, c, x)], [Box(n, 1.0)], [u], seed,
                    note="solid ball 4096 nodes / 20250 tets, NH nu=0.45, 128^3")


# ---------------------------------------------------------------- RSA
class _Occupancy:
    """Voxel occupancy of a periodic box (one voxel per grid cell).

    A particle is rasterised once, as a set of voxel offsets around an integer
    cell plus a fixed fractional shift; each random sequential addition trial
    is then a batch of table lookups.
    """

    def __init__(self, n: int):
        self.n = n
        self.occ = np.zeros(n ** 3, dtype=bool)

    @staticmethod
    def offsets(frac, inside_fn, half_extent):
        e = int(np.ceil(half_extent)) + 1
        r = np.arange(-e, e + 1)
        Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
        p = np.stack([X + 0.5, Y + 0.5, Z + 0.5], axis=-1) - frac
        m = inside_fn(p)
        return X[m], Y[m], Z[m]

    def place(self, rng, offs, tries: int, batch: int = 64):
        """Try up to `tries` random integer centres; returns the centre or None."""
        n = self.n
        ox, oy, oz = offs
        for start in range(0, tries, batch):
            k = min(batch, tries - start)
            c = rng.integers(0, n, size=(k, 3))
            idx = (((c[:, 2:3] + oz[None]) % n) * n + ((c[:, 1:2] + oy[None]) % n)) * n \
                + ((c[:, 0:1] + ox[None]) % n)
            hit = self.occ[idx].any(axis=1)
            free = np.flatnonzero(~hit)
            if free.size:
                j = free[0]
                self.occ[idx[j]] = True
                return c[j]
        return None


def _rbc_inside_fn(Minv, D_cells, gap):
    def f(p):
        q = p @ Minv.T
        return meshes.rbc_inside(q, D_cells, gap)
    return f


def _ellipsoid_inside_fn(Minv, semi, gap):
    def f(p):
        q = p @ Minv.T
        return ((q / (np.asarray(semi) + gap)) ** 2).sum(-1) <= 1.0
    return f


# ---------------------------------------------------------------- C4
def config4(seed: int = 1004, n: int = 256, n_rbc: int = 500, n_plt: int = 100,
            target_ht: float = 0.20, max_tries: int = 20000) -> Workload:
    """Dense blood suspension: n_rbc RBCs (2562 nodes) + n_plt platelets (512 nodes, 2058 tets)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    # RBC volume is 0.1968 D^3 for this profile; platelet (a, a, a/2), a = 0.1875 D.
    v_rbc = 0.19676
    v_plt = 4.0 / 3.0 * np.pi * 0.1875 ** 3 * 0.5
    D_cells = (target_ht * n ** 3 / (n_rbc * v_rbc + n_plt * v_plt)) ** (1.0 / 3.0)
    D = D_cells * h
    rbc = rbc_template(D)
    a_cells = 0.1875 * D_cells
    R_plt = a_cells * h
    mu_plt = 1.0 / (CA_PLT_OVER_CA_RBC * R_plt)
    plt = ball_template(8, R_plt, mu=mu_plt, semi_axes=np.array([R_plt, R_plt, 0.5 * R_plt]),
                        lam=PLT_LAMBDA_OVER_MU * mu_plt)
    plt.name = "platelet512"
    kinds = np.array([0] * n_rbc + [1] * n_plt)[rng.permutation(n_rbc + n_plt)]
    occ = _Occupancy(n)
    instances = []
    for kind in kinds:
        Rm = meshes.random_rotation(rng)
        frac = rng.uniform(0.0, 1.0, 3)
        if kind == 0:
            M = Rm @ np.diag(1.0 + 0.1 * rng.standard_normal(3))
            offs = occ.offsets(frac, _rbc_inside_fn(np.linalg.inv(M), D_cells, 0.5),
                               0.5 * D_cells * 1.4 + 1.0)
        else:
            M = Rm @ (np.eye(3) + 0.05 * rng.uniform(-1, 1, (3, 3)))
            offs = occ.offsets(frac, _ellipsoid_inside_fn(np.linalg.inv(M),
                                                          [a_cells, a_cells, 0.5 * a_cells], 0.5),
                               a_cells * 1.3 + 1.0)
        c = occ.place(rng, offs, max_tries)
        if c is None:
            continue
        tm = rbc if kind == 0 else plt
        x = tm.X @ M.T
        if kind == 0:
            x = x + _jitter(rng, x.shape, 1e-3 * D)
        instances.append(Instance(int(kind), 0, (c + frac) * h, x))
    # RBCs first, then platelets (node order is the instance order)
    instances.sort(key=lambda i: i.tmpl)
    u = sample_on_mac(fourier_modes(rng), n, 1.0, dtype=np.float32)
    nr = sum(1 for i in instances if i.tmpl == 0)
    npl = len(instances) - nr
    ht = (nr * v_rbc + npl * v_plt) * D_cells ** 3 / n ** 3
    return Workload("C4", [rbc, plt], instances, [Box(n, 1.0)], [u], seed,
                    note=f"{nr} RBC + {npl} PLT, D={D_cells:.2f} cells, Ht={ht:.3f}, {n}^3")


# ---------------------------------------------------------------- C5
def config5(seed: int = 1005, n_boxes: int = 64, nmin: int = 32, nmax: int = 96,
            max_per_box: int = 20, max_tries: int = 1000, h: float = 1.0 / 64) -> Workload:
    """64 independent periodic boxes of n ~ U{32..96} cells (spacing h), 1-20 mixed particles each."""
    rng = np.random.default_rng(seed)
    cap642 = meshes.icosphere(3)
    cap2562 = meshes.icosphere(4)
    templates: List[Template] = []
    R1, R2, Drbc = 9.6 * h, 14.0 * h, 20.0 * h
    templates.append(Template("membrane", R1 * cap642[0], cap642[1], "nh", mu=1.0,
                              kb=KAPPA_B_HAT * R1, name="capsule642"))
    templates.append(Template("membrane", R2 * cap2562[0], cap2562[1], "nh", mu=1.0,
                              kb=KAPPA_B_HAT * R2, name="capsule2562"))
    templates.append(rbc_template(Drbc))
    ball_m = list(range(8, 16))
    for m in ball_m:
        templates.append(ball_template(m, 0.5 * (m - 1) * h))
    boxes, instances, us = [], [], []
    for b in range(n_boxes):
        n = int(rng.integers(nmin, nmax + 1))
        box = Box(n, n * h)
        boxes.append(box)
        occ = _Occupancy(n)
        k = int(rng.integers(1, max_per_box + 1))
        for _ in range(k):
            typ = int(rng.integers(0, 4))
            Rm = meshes.random_rotation(rng)
            frac = rng.uniform(0.0, 1.0, 3)
            if typ == 3:
                m = int(rng.integers(8, 16))
                ti = 3 + ball_m.index(m)
                rad = 0.5 * (m - 1)
                M = Rm @ (np.eye(3) + 0.05 * rng.uniform(-1, 1, (3, 3)))
                inside = _ellipsoid_inside_fn(np.linalg.inv(M), [rad] * 3, 0.5)
                ext = rad * 1.2 + 1.0
            elif typ == 2:
                ti = 2
                M = Rm @ np.diag(1.0 + 0.1 * rng.standard_normal(3))
                inside = _rbc_inside_fn(np.linalg.inv(M), 20.0, 0.5)
                ext = 10.0 * 1.4 + 1.0
            else:
                ti = typ
                rad = (9.6, 14.0)[typ]
                M = Rm @ np.diag(1.0 + 0.1 * rng.standard_normal(3))
                inside = _ellipsoid_inside_fn(np.linalg.inv(M), [rad] * 3, 0.5)
                ext = rad * 1.4 + 1.0
            if 2 * ext + 2 > n:
                continue
            c = occ.place(rng, occ.offsets(frac, inside, ext), max_tries)
            if c is None:
                continue
            x = templates[ti].X @ M.T
            if templates[ti].kind == "membrane":
                # solids get the affine map only: their thinnest slivers are
                # ~0.02 cells high and would invert under positional noise
                x = x + _jitter(rng, x.shape, 1e-4 * n * h)
            instances.append(Instance(ti, b, (c + frac) * h, x))
        us.append(sample_on_mac(fourier_modes(rng), n, box.L, dtype=np.float32))
    return Workload("C5", templates, instances, boxes, us, seed,
                    note=f"{n_boxes} boxes, {len(instances)} particles")


def make(name: str, **kw) -> Workload:
    return {"C1": config1, "C2": config2, "C3": config3, "C4": config4, "C5": config5}[name](**kw)
