"""The -fopenmp build of the oracle (used only for the multi-core CPU
baseline) computes the same bits as the serial build: every loop it runs in
parallel writes only its own node's or row's results."""
import os
import subprocess
import sys

import numpy as np

import oracle
import smash_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import oracle, smash_inputs as si
assert oracle.openmp()
x = si.uniform_cube(6000, 3, 810)
q = si.rhs(6000, 3, 811)
h = oracle.H2(x, 1, 32, 3, 1e-8)
e = h.export()
np.savez(sys.argv[2], z=h.matvec(q), za=h.matvec_abs(q), G=e["G_row"], skel=e["skel_row"],
         d=oracle.dense_rows(x, 1, q, rows=np.arange(0, 6000, 7)))
"""


def test_openmp_build_gives_the_serial_bits(tmp_path):
    out = tmp_path / "omp.npz"
    env = dict(os.environ, ORACLE_OPENMP="1", OMP_NUM_THREADS="4")
    subprocess.run([sys.executable, "-c", _CHILD, ROOT, str(out)], env=env, check=True, timeout=300)
    got = np.load(out)
    assert not oracle.openmp()
    x = si.uniform_cube(6000, 3, 810)
    q = si.rhs(6000, 3, 811)
    h = oracle.H2(x, 1, 32, 3, 1e-8)
    e = h.export()
    assert np.array_equal(got["G"], e["G_row"]) and np.array_equal(got["skel"], e["skel_row"])
    assert np.array_equal(got["z"], h.matvec(q))
    assert np.array_equal(got["za"], h.matvec_abs(q))
    assert np.array_equal(got["d"], oracle.dense_rows(x, 1, q, rows=np.arange(0, 6000, 7)))
