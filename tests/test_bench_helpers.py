"""Host logic of bench.py that picks the roofline unit of the coupling.

The double-float coupling runs one of two kernels; bench.py reads which one
from the tuning table (keys "coupling_dd/..."), else applies the library's
untuned default (the digit split from 8 columns per pass).  A fake of the
binding's save call stands in for the library.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeSm:
    def __init__(self, entries):
        self.entries = entries

    def smash_autotune_save(self, path):  # like the binding: returns None, raises on failure
        with open(path, "w") as f:
            json.dump({"smash_autotune": 1, "entries": self.entries}, f)


def test_recorded_choice_wins():
    sm = _FakeSm({"ksum_dd/sm152/k1/d3": 1, "coupling_dd/sm152/k1/d3/ld16/n65536": 1})
    assert bench._coupling_choice(sm, 16) == 1
    sm = _FakeSm({"coupling_dd/sm152/k1/d3/ld16/n65536": 0})
    assert bench._coupling_choice(sm, 4) == 0


def test_pinned_coupling_wins_over_the_table():
    sm = _FakeSm({"coupling_dd/sm152/k1/d3/ld16/n65536": 0})
    assert bench._coupling_choice(sm, 16, "tcgen05") == 2
    assert bench._coupling_choice(sm, 16, "fp32") == 1
    assert bench._coupling_choice(sm, 16, "warp") == 0
    assert bench._coupling_choice(sm, 16, "auto") == 0


def test_untuned_default_follows_the_column_count():
    sm = _FakeSm({"compress/sm152/d3/p4/m512/n4096": 256})
    assert bench._coupling_choice(sm, 16) == 0
    assert bench._coupling_choice(sm, 8) == 0
    assert bench._coupling_choice(sm, 5) == 0   # 5 columns pass as 8
    assert bench._coupling_choice(sm, 4) == 1
    assert bench._coupling_choice(sm, 1) == 1


# ---------------------------------------------------------------- roofline units
import numpy as np  # noqa: E402


def test_build_flops_counts_the_algorithmic_work_per_node():
    ranks = {"m": np.array([0, 32, 100]), "k": np.array([0, 8, 64])}
    r, d = 64, 3

    def one(m, k):
        return m * r * (d + 1) + (4 * r * m * k - 2 * k * k * (r + m) + 4 * k ** 3 / 3) + k * k * (m - k)

    assert bench.build_flops(ranks, r, d) == one(32, 8) + one(100, 64)


def test_pass_bytes_counts_G_and_the_vectors():
    ranks = {"m": np.array([10, 4]), "k": np.array([3, 4])}
    assert bench.pass_bytes(ranks, 16) == 8 * (7 * 3 + 0) + 8 * 16 * (13 + 8)


def test_entry_errors_scale_each_entry_by_its_sum_of_magnitudes():
    zo = np.array([[1.0, 0.0], [2.0, -3.0]])
    sc = np.array([[10.0, 0.0], [4.0, 6.0]])
    e = bench.entry_errors(zo + np.array([[1e-3, 0.0], [4e-3, 0.0]]), zo, sc)
    assert abs(e["worst_entry_vs_sum_abs_terms"] - 1e-3) < 1e-15
    assert np.isinf(bench.entry_errors(zo + np.array([[0, 1e-30], [0, 0]]), zo, sc)["worst_entry_vs_sum_abs_terms"])


def test_rooflines_use_method_work_and_the_stated_peaks():
    class Sm:
        SMASH_PREC_F64 = 0

    info = {"coupling_pairs": 1000, "near_pairs": 200, "r": 8, "dim": 1}
    ranks = {"m": np.array([16]), "k": np.array([4])}
    prof = {"coupling": 2.0, "near": 1.0, "compression": 0.5, "upward": 0.1, "downward": 0.2}
    peaks = {"fp32_tflops": 80.0, "fp64_tflops": 1.25, "hbm_gbs": 7000.0}
    r = bench.rooflines(info, ranks, prof, 16, 16, peaks, 1, Sm)
    assert abs(r["coupling"]["achieved"] - 1000 * 42 / 2e-3 / 1e12) < 1e-18
    assert r["coupling"]["peak"] == 80.0 and r["compression"]["peak"] == 1.25
    r64 = bench.rooflines(info, ranks, prof, 16, 16, peaks, 0, Sm)
    assert r64["coupling"]["peak"] == 1.25
    assert r["upward"]["unit"] == "GB/s" and r["upward"]["peak"] == 7000.0
