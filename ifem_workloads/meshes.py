"""Seeded synthetic Lagrangian meshes for the coupling-step workloads.

Pure geometry and topology: icosphere membranes, the biconcave red-cell
surface, Kuhn-split tetrahedral balls. Nothing here evaluates the IFEM
method itself; both the CPU oracle and the CUDA path consume these arrays.

Conventions
-----------
* Node coordinates are float64 arrays of shape (n_nodes, 3).
* Triangles are int32 (n_tris, 3), oriented so that (b - a) x (c - a)
  points out of the enclosed volume.
* Tetrahedra are int32 (n_tets, 4), oriented so that
  det[x1 - x0, x2 - x0, x3 - x0] > 0.
"""
from __future__ import annotations

import numpy as np

# Evans & Fung (1972) biconcave profile coefficients, in units of the cell
# radius R0 = D/2: thickness T(rho) = R0 * sqrt(1 - rho^2) * (C0 + C2 rho^2 +
# C4 rho^4) with C0 = 0.81, C2 = 7.83, C4 = -4.39 (um) over R0 = 3.91 um.
EVANS_FUNG_C = (0.81 / 3.91, 7.83 / 3.91, -4.39 / 3.91)


def icosahedron() -> tuple[np.ndarray, np.ndarray]:
    """Regular icosahedron on the unit sphere, outward-oriented faces."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    return v, _orient_outward(v, f)


def _orient_outward(v: np.ndarray, f: np.ndarray) -> np.ndarray:
    f = f.copy()
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    f[flip, 1], f[flip, 2] = f[flip, 2].copy(), f[flip, 1].copy()
    return f


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere by repeated 4-way midpoint subdivision.

    level 3 -> 642 nodes / 1280 triangles; level 4 -> 2562 / 5120.
    """
    v, f = icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}
        nf = []

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            k = cache.get(key)
            if k is None:
                p = (np.asarray(verts[i]) + np.asarray(verts[j])) * 0.5
                p /= np.linalg.norm(p)
                verts.append(tuple(p))
                k = len(verts) - 1
                cache[key] = k
            return k

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.asarray(nf, dtype=np.int32)
    v = np.asarray(verts, dtype=np.float64)
    return v, _orient_outward(v, f)


def rbc_surface(level: int, diameter: float) -> tuple[np.ndarray, np.ndarray]:
    """Biconcave resting red-cell surface of the given diameter.

    Maps the unit icosphere through the Evans-Fung profile: a sphere point
    (x, y, z) goes to (R0 x, R0 y, sign(z) T(rho)/2) with rho = hypot(x, y),
    R0 = diameter / 2 and T the full thickness of the profile above.
    """
    v, f = icosphere(level)
    r0 = 0.5 * diameter
    rho2 = np.clip(v[:, 0] ** 2 + v[:, 1] ** 2, 0.0, 1.0)
    c0, c2, c4 = EVANS_FUNG_C
    half_t = 0.5 * r0 * np.sqrt(1.0 - rho2) * (c0 + c2 * rho2 + c4 * rho2 ** 2)
    out = np.empty_like(v)
    out[:, 0] = r0 * v[:, 0]
    out[:, 1] = r0 * v[:, 1]
    out[:, 2] = np.sign(v[:, 2]) * half_t
    return out, _orient_by_volume(out, f)


def _orient_by_volume(v: np.ndarray, f: np.ndarray) -> np.ndarray:
    # The map above preserves the outward orientation of every face of the
    # sphere (it is monotone in z on each hemisphere), so only a global
    # check is needed.
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    if vol < 0:
        f = f[:, [0, 2, 1]].copy()
    return f


def rbc_inside(p: np.ndarray, diameter: float, gap: float = 0.0) -> np.ndarray:
    """Point-in-cell test for the resting biconcave shape (local frame)."""
    r0 = 0.5 * diameter
    rho2 = (p[..., 0] ** 2 + p[..., 1] ** 2) / (r0 + gap) ** 2
    c0, c2, c4 = EVANS_FUNG_C
    rr = np.clip(rho2, 0.0, 1.0)
    half_t = 0.5 * r0 * np.sqrt(1.0 - rr) * (c0 + c2 * rr + c4 * rr ** 2)
    return (rho2 <= 1.0) & (np.abs(p[..., 2]) <= half_t + gap)


def kuhn_ball(m: int, radius: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Tetrahedral ball: an m^3 cube lattice mapped onto a sphere.

    Every hexahedral cell of the [-1, 1]^3 lattice is split into the six
    Kuhn tetrahedra along its main diagonal; the lattice is then mapped onto
    the ball by the smooth cube-to-sphere map
    x' = x sqrt(1 - y^2/2 - z^2/2 + y^2 z^2/3) (and cyclic), which sends the
    cube surface to the unit sphere. Unlike the plain radial projection
    p |p|_inf / |p|_2 it keeps every tetrahedron well shaped (smallest volume
    about 1/60 of the largest instead of 1/1000).
    m = 16 gives 4096 nodes / 20250 tets; m = 8 gives 512 / 2058.
    """
    g = np.linspace(-1.0, 1.0, m)
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    nid = lambda i, j, k: (k * m + j) * m + i  # noqa: E731
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for k in range(m - 1):
        for j in range(m - 1):
            for i in range(m - 1):
                for perm in perms:
                    c = [0, 0, 0]
                    path = [nid(i, j, k)]
                    for ax in perm:
                        c[ax] += 1
                        path.append(nid(i + c[0], j + c[1], k + c[2]))
                    tets.append(path)
    t = np.asarray(tets, dtype=np.int32)
    x2, y2, z2 = p[:, 0] ** 2, p[:, 1] ** 2, p[:, 2] ** 2
    q = np.stack([p[:, 0] * np.sqrt(1 - y2 / 2 - z2 / 2 + y2 * z2 / 3),
                  p[:, 1] * np.sqrt(1 - z2 / 2 - x2 / 2 + z2 * x2 / 3),
                  p[:, 2] * np.sqrt(1 - x2 / 2 - y2 / 2 + x2 * y2 / 3)], axis=1)
    q *= radius
    t = _orient_tets(q, t)
    return q, t


def _orient_tets(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    t = t.copy()
    d = np.linalg.det(np.stack([x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]],
                                x[t[:, 3]] - x[t[:, 0]]], axis=2))
    neg = d < 0
    t[neg, 2], t[neg, 3] = t[neg, 3].copy(), t[neg, 2].copy()
    return t


def tet_signed_volumes(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Signed volume of every tetrahedron (input sanity checks only)."""
    d = np.stack([x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]],
                  x[t[:, 3]] - x[t[:, 0]]], axis=2)
    return np.linalg.det(d) / 6.0


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix (QR of a Gaussian matrix)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q
