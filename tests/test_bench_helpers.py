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


def test_untuned_default_follows_the_column_count():
    sm = _FakeSm({"compress/sm152/d3/p4/m512/n4096": 256})
    assert bench._coupling_choice(sm, 16) == 0
    assert bench._coupling_choice(sm, 8) == 0
    assert bench._coupling_choice(sm, 5) == 0   # 5 columns pass as 8
    assert bench._coupling_choice(sm, 4) == 1
    assert bench._coupling_choice(sm, 1) == 1
