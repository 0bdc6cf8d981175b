"""Seeded synthetic Eulerian velocity fields on periodic staggered (MAC) grids.

Grid convention shared by every consumer in this repository: a box of side
L holds n^3 cells of spacing h = L/n. Velocity component d lives on its own
lattice with node (i, j, k) at ((i, j, k) + o_d) h, where
o_d = (1/2, 1/2, 1/2) - e_d / 2 (u_x on x-faces, u_y on y-faces, u_z on
z-faces). Each component is stored as an (n, n, n) array indexed [k, j, i],
x fastest.
"""
from __future__ import annotations

import numpy as np


def mac_offset(d: int) -> np.ndarray:
    """Lattice offset o_d (in cells) of velocity component d."""
    o = np.full(3, 0.5)
    o[d] = 0.0
    return o


def fourier_modes(rng: np.random.Generator, n_modes: int = 8, kmax: int = 4,
                  amplitude: float = 0.1):
    """Random divergence-free Fourier modes.

    Each mode has an integer wave vector k in {-kmax..kmax}^3 without 0, a unit
    direction e orthogonal to k, and a phase uniform on [0, 2 pi).
    """
    ks, es, ph = [], [], []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            continue
        e = rng.standard_normal(3)
        kn = k / np.linalg.norm(k)
        e -= e.dot(kn) * kn
        e /= np.linalg.norm(e)
        ks.append(k.astype(np.float64))
        es.append(e)
        ph.append(rng.uniform(0.0, 2.0 * np.pi))
    return np.array(ks), np.array(es), amplitude * np.ones(n_modes), np.array(ph)


def eval_modes(modes, p: np.ndarray, L: float) -> np.ndarray:
    """Evaluate the velocity sum_m a_m e_m cos(2 pi k_m . p / L + phi_m) at points p (..., 3)."""
    ks, es, amp, ph = modes
    out = np.zeros(p.shape[:-1] + (3,))
    for k, e, a, f in zip(ks, es, amp, ph):
        arg = 2.0 * np.pi * (p @ k) / L + f
        out += (a * np.cos(arg))[..., None] * e
    return out


def sample_on_mac(modes, n: int, L: float, dtype=np.float64) -> np.ndarray:
    """Sample the modes on the three MAC lattices: returns (3, n, n, n) [d, k, j, i]."""
    ks, es, amp, ph = modes
    h = L / n
    out = np.zeros((3, n, n, n), dtype=np.float64)
    idx = np.arange(n, dtype=np.float64)
    for d in range(3):
        o = mac_offset(d)
        cx = (idx + o[0]) * h
        cy = (idx + o[1]) * h
        cz = (idx + o[2]) * h
        acc = np.zeros((n, n, n), dtype=np.complex128)
        for k, e, a, f in zip(ks, es, amp, ph):
            if e[d] == 0.0:
                continue
            ex = np.exp(2j * np.pi * k[0] * cx / L)
            ey = np.exp(2j * np.pi * k[1] * cy / L)
            ez = np.exp(2j * np.pi * k[2] * cz / L)
            acc += (a * e[d] * np.exp(1j * f)) * (ez[:, None, None] * ey[None, :, None] * ex[None, None, :])
        out[d] = acc.real
    return out.astype(dtype, copy=False)


def conformation_cc(rng: np.random.Generator, n: int, L: float, n_modes: int = 6, kmax: int = 3,
                    amplitude: float = 0.05) -> np.ndarray:
    """Seeded smooth cell-centred conformation-tensor field: (6, n, n, n) in the
    component order xx, yy, zz, xy, xz, yz, equal to I plus a sum of cosine
    modes with random symmetric amplitude matrices (the perturbation stays
    below the identity, so every sample is symmetric positive definite)."""
    c = (np.arange(n, dtype=np.float64) + 0.5) * (L / n)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    out = np.zeros((6, n, n, n))
    out[0] = out[1] = out[2] = 1.0
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    for _ in range(n_modes):
        k = rng.integers(-kmax, kmax + 1, size=3).astype(np.float64)
        M = rng.standard_normal((3, 3))
        M = amplitude * (M + M.T) / 2.0
        arg = 2.0 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) / L + rng.uniform(0.0, 2.0 * np.pi)
        cos = np.cos(arg)
        for q, (i, j) in enumerate(pairs):
            out[q] += M[i, j] * cos
    return out
