"""Host-side logic of bench.py (no GPU): the algorithmic byte counts behind the
roofline fraction and the particle sampling of the oracle baselines."""
import dataclasses

import numpy as np
import pytest

import ifem_workloads as W


def test_algorithmic_bytes_closed_forms():
    import bench
    N, T = 1_332_200, 18_680_000
    ab = bench.algorithmic_bytes(N, T, 0)
    # fused transfer: x, F read + v written (36N), own-node list (4N), u read + f read and written (12T)
    assert ab["spread+interp"] == 40 * N + 12 * T
    # whole step: x, v, F written and read, u read, f read and written
    assert ab["step"] == 48 * N + 12 * T
    assert ab["forces"] == 24 * N and ab["reduce"] == 36 * N
    # with candidate lists the spread reads one entry per (tile, node) pair
    P = 3 * N
    assert bench.algorithmic_bytes(N, T, P)["spread"] == 24 * N + 4 * P + 8 * T
    # FP64 doubles every real-valued byte, not the int32 lists
    ab8 = bench.algorithmic_bytes(N, T, 0, real=8)
    assert ab8["spread+interp"] == 2 * (36 * N + 12 * T) + 4 * N


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
