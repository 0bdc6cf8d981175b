"""Host-side logic of bench.py (no GPU): the algorithmic byte counts behind the
roofline fraction and the particle sampling of the oracle baselines."""
import dataclasses

import numpy as np
import pytest

import ifem_workloads as W


def test_algorithmic_bytes_closed_forms():
    """The per-unit bytes of the hot path: a fused transfer launch moves x and
    F in and v out (36 B per node) and reads u, reads and writes f once per
    touched lattice value (12 B); the coupling step as one operation moves x
    in and v out (24 B per node) plus the same 12 B per touched value; the F
    round trip adds 24 B per node and is reported separately."""
    import bench
    N, T = 1_332_200, 18_680_000
    ab = bench.algorithmic_bytes(N, T, 0)
    assert ab["spread+interp"] == 36 * N + 12 * T
    assert ab["step"] == 24 * N + 12 * T
    assert ab["step_with_F"] == 48 * N + 12 * T
    assert ab["forces"] == 24 * N and ab["reduce"] == 36 * N
    # with candidate lists the spread reads one entry per (tile, node) pair
    P = 3 * N
    assert bench.algorithmic_bytes(N, T, P)["spread"] == 24 * N + 4 * P + 8 * T
    # FP64 doubles every real-valued byte
    ab8 = bench.algorithmic_bytes(N, T, 0, real=8)
    assert ab8["spread+interp"] == 2 * (36 * N + 12 * T)
    # C4 figures: 0.272 GB per fused launch, 0.256 GB per step
    assert ab["spread+interp"] == pytest.approx(272.1e6, rel=1e-3)
    assert ab["step"] == pytest.approx(256.1e6, rel=1e-3)


def test_chunks_by_nodes_cover_every_particle_once():
    import bench
    w = W.make("C2")
    w7 = dataclasses.replace(w, instances=[w.instances[0]] * 7)
    for parts in (1, 3, 7, 16):
        ch = bench._chunks_by_nodes(w7, parts)
        assert ch[0][0] == 0 and ch[-1][1] == 7
        assert all(a < b for a, b in ch) and all(ch[i][1] == ch[i + 1][0] for i in range(len(ch) - 1))
        assert len(ch) == min(parts, 7)


def test_even_sample_reaches_target_evenly():
    import bench
    w = W.make("C2")
    w10 = dataclasses.replace(w, instances=[w.instances[0]] * 10)
    size = w.templates[0].n_nodes
    sel, n = bench._even_sample(w10, 3 * size)
    assert n == len(sel) * size and n >= 3 * size
    assert sel[0] == 0 and sel[-1] == 9 and sel == sorted(set(sel))
    sel, n = bench._even_sample(w10, 1)
    assert sel == [0] and n == size
    sel, n = bench._even_sample(w10, 10**9)
    assert sel == list(range(10)) and n == 10 * size


def test_roofline_denominator_is_the_measured_copy_bandwidth():
    import bench
    hbm, kind = bench.peaks()
    assert hbm > 1000.0 and kind in ("measured", "fallback")
    if kind == "fallback":
        assert hbm == pytest.approx(6800.0)
