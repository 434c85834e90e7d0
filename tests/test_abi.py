"""The C-ABI library builds, loads and exports what include/smash.h declares;
host-only logic (validation, the Section 6.1 heuristic, struct layouts) works
without a GPU.  No test here launches a kernel."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_1705_05443_gb300 as sm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smash.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SMASH_API [^;{]*?\b(smash_\w+)\(", text)))


def test_library_builds_and_loads():
    lib = sm.load_library()
    assert os.path.exists(sm.library_path())
    assert lib is not None


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", sm.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (smash_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = sm.load_library()
    for n in names:
        assert hasattr(lib, n)


def test_struct_layouts_match_the_header(tmp_path):
    """Compile a probe against include/smash.h with the host C compiler and
    compare sizes and offsets with the ctypes mirrors of the binding."""
    src = tmp_path / "probe.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "smash.h"', "int main(void){"]
    for st, cls in (("smash_info_t", sm.smash_info_t), ("smash_export_t", sm.smash_export_t),
                    ("smash_options", sm.smash_options)):
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for name, _ in cls._fields_:
            lines.append(f'printf("{st}.{name} %zu\\n", offsetof({st}, {name}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for st, cls in (("smash_info_t", sm.smash_info_t), ("smash_export_t", sm.smash_export_t),
                    ("smash_options", sm.smash_options)):
        assert int(got[st]) == C.sizeof(cls), st
        for name, _ in cls._fields_:
            assert int(got[f"{st}.{name}"]) == getattr(cls, name).offset, f"{st}.{name}"


def test_suggest_rank_host_function():
    # Section 6.1 worked values, computed by the library's host code
    assert sm.smash_suggest_rank(1e-7, 0.65) == 22
    assert sm.smash_suggest_rank(1e-8, 0.6) == 21
    assert sm.smash_suggest_rank(1e-10, 0.6) == 25


@pytest.mark.parametrize("kw,msg", [
    (dict(dim=4), "dim"),
    (dict(n=0), "n must"),
    (dict(leaf=0), "leaf_size"),
    (dict(order=0), "order"),
    (dict(order=9), "order^dim"),
    (dict(tol=0.0), "tol"),
    (dict(tol=float("nan")), "tol"),
    (dict(kernel=7), "kernel_id"),
    (dict(kernel=3), "Cauchy"),
])
def test_invalid_input_is_rejected_before_any_device_work(kw, msg):
    import numpy as np
    lib = sm.load_library()
    x = np.random.default_rng(0).random((16, 3))
    h = C.c_void_p(12345)
    st = lib.smash_build(C.c_void_p(x.ctypes.data), kw.get("dim", 3), kw.get("n", 16), kw.get("kernel", 1),
                         kw.get("leaf", 8), kw.get("order", 3), kw.get("tol", 1e-8), C.byref(h))
    assert st == 1                     # SMASH_EINVAL
    assert h.value is None             # *out = NULL on failure
    assert msg in lib.smash_last_error().decode()


def test_predict_footprint_grows_with_n():
    a = sm.smash_predict_footprint(1 << 16, 3, 128, 4, 16)
    b = sm.smash_predict_footprint(1 << 20, 3, 128, 4, 16)
    assert 0 < a < b
    assert sm.smash_predict_footprint(0, 3, 128, 4, 16) == 0


def test_free_and_info_accept_null():
    lib = sm.load_library()
    lib.smash_free(None)
    assert lib.smash_footprint_bytes(None) == 0
    assert lib.smash_info(None, None) == 1


@pytest.mark.parametrize("offsets,msg", [
    ([], "nproblems"),
    ([1, 5], "offsets[0]"),
    ([0, 5, 5], "at least one point"),
    ([0, 7, 3], "at least one point"),
])
def test_batch_offsets_are_validated_before_any_device_work(offsets, msg):
    import numpy as np
    lib = sm.load_library()
    x = np.random.default_rng(1).random((16, 3))
    off = np.asarray(offsets, dtype=np.int64)
    h = C.c_void_p(12345)
    st = lib.smash_build_batch(C.c_void_p(x.ctypes.data), C.c_void_p(off.ctypes.data) if off.size else None,
                               max(len(off) - 1, 0), 3, 1, 8, 3, 1e-8, None, C.byref(h))
    assert st == 1
    assert h.value is None
    assert msg in lib.smash_last_error().decode()


def test_autotune_table_round_trips_through_a_file(tmp_path):
    """The autotune table is host state: load, look up, save and reload
    without a device."""
    sm.smash_autotune_clear()
    assert sm.smash_autotune_entries() == 0
    src = tmp_path / "in.json"
    src.write_text('{"smash_autotune": 1, "entries": {"compress/sm152/d3/p4/m512/n1024": 256,\n'
                   ' "ksum_dd/sm152/k1/d3/x1/rc16/ld16/t128/n32768": 3}}')
    assert sm.smash_autotune_load(str(src)) == 2
    assert sm.smash_autotune_lookup("compress/sm152/d3/p4/m512/n1024") == 256
    assert sm.smash_autotune_lookup("no/such/key") is None
    out = tmp_path / "out.json"
    sm.smash_autotune_save(str(out))
    sm.smash_autotune_clear()
    assert sm.smash_autotune_load(str(out)) == 2
    assert sm.smash_autotune_lookup("ksum_dd/sm152/k1/d3/x1/rc16/ld16/t128/n32768") == 3
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": {"a": x}}')
    assert sm.smash_autotune_load(str(bad)) == -1
    assert sm.smash_autotune_load(str(tmp_path / "missing.json")) == -1
    assert sm.smash_autotune_entries() == 2   # unchanged by the failed loads
    sm.smash_autotune_clear()


def test_matvec_graph_rejects_null_handle():
    lib = sm.load_library()
    assert lib.smash_matvec_graph(None, None, None, 1, 0, None) == 1
    assert "NULL" in lib.smash_last_error().decode()
    assert lib.smash_matvec_graph_count(None) == 0


def test_cauchy_like_rejects_bad_arguments_without_a_device():
    lib = sm.load_library()
    assert lib.smash_matvec_cauchy_like(None, None, None, 2, None, None, 1, 0, None) == 1
    assert "NULL" in lib.smash_last_error().decode()


def test_double_layer_kernels_need_two_dimensions():
    import numpy as np
    lib = sm.load_library()
    x = np.random.default_rng(2).random((16, 3))
    h = C.c_void_p(12345)
    st = lib.smash_build(C.c_void_p(x.ctypes.data), 3, 16, sm.SMASH_K_DLP1, 8, 3, 1e-8, C.byref(h))
    assert st == 1 and h.value is None
    assert "dim == 2" in lib.smash_last_error().decode()
    assert lib.smash_matvec_double_layer(None, None, None, None, None, None, 1, 0, None) == 1
    assert lib.smash_matvec_kernel(None, 4, None, None, 1, 0, None) == 1
