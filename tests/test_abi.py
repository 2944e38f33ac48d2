"""The C ABI library: it builds, loads, exports every declared symbol, and its
host-side logic (encoding, built-in matrix, argument validation) is right.
No GPU is needed: every call here fails or returns before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2309_09609_gb300 import build as nvbuild
from paper_2309_09609_gb300 import swgb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nvbuild.build()
    return swgb.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "swgb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", swgb.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)$", out, flags=re.M))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n), n


def test_default_matrix_equals_oracle_table(lib):
    assert (swgb.default_matrix().astype(np.int32) == oracle.blosum62()).all()


def test_encode_matches_oracle(lib):
    text = "ARNDCQEGHILKMFPSTWYVBZX*uojarnd?!. "
    assert (swgb.encode(text) == oracle.encode(text)).all()
    # every byte value, including those above 127
    every = bytes(range(256)).decode("latin-1")
    got = swgb.encode(every)
    assert (got == oracle.encode(every)).all() and got.max() < 24
    assert swgb.encode("").size == 0


def test_options_default(lib):
    o = swgb.options()
    assert o.rows_per_thread in (16, 32) and o.intra_rows in (8, 16)
    assert o.warps_per_block >= 1 and o.long_cutoff > 0 and o.use_graph == 1
    assert o.wide_min_len >= 0


def test_options_struct_layout_matches_the_header(lib):
    # every field of sw_options, as the library fills it in, at the offset
    # the binding reads it from (a mismatched layout shifts these values)
    o = swgb.options()
    assert {k: getattr(o, k) for k, _ in swgb.Options._fields_} == {
        "rows_per_thread": 32, "warps_per_block": 8, "long_cutoff": 1500, "intra_rows": 8,
        "use_graph": 1, "force_int32": 0, "auto_cutoff": 0, "wide_min_len": 0,
        "wide_min_subject": 4096, "inter_columns": 8, "overlap_kernels": 0, "two_query": 1,
        "two_query_rows": 32, "two_query_pairs": 0, "flag_capacity": 0,
        "two_query_long": 1}
    header = open(os.path.join(ROOT, "include", "swgb.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\} sw_options;", header).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"int32_t\s+(\w+);", body)
    assert fields == [k for k, _ in swgb.Options._fields_]


def test_stats_struct_fields_match_the_header(lib):
    header = open(os.path.join(ROOT, "include", "swgb.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\} sw_stats;", header).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(int32_t|int64_t|float)\s+(\w+);", body)
    ctype = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "float": ctypes.c_float}
    assert [(n, ctype[t]) for t, n in fields] == list(swgb.Stats._fields_)


def test_db_create_rejects_bad_input_before_touching_the_gpu(lib):
    with pytest.raises(swgb.SwError) as e:
        swgb.Database(np.array([0, 1, 30], np.uint8), np.array([3], np.int32))
    assert e.value.status == swgb.SW_EINVAL and "code 30" in str(e.value)
    with pytest.raises(swgb.SwError) as e:
        swgb.Database(np.array([0, 1], np.uint8), np.array([2, -1], np.int32))
    assert e.value.status == swgb.SW_EINVAL
    st = lib.sw_db_create(None, None, -1, 0, ctypes.byref(ctypes.c_void_p()))
    assert st == swgb.SW_EINVAL and "n_subjects" in swgb.last_error()
    assert lib.sw_db_create(None, None, 0, 0, None) == swgb.SW_EINVAL


def test_null_handles_are_rejected(lib):
    z = ctypes.c_void_p()
    assert lib.sw_search(None, None, None, 0, 10, 2, None, None, None) == swgb.SW_EINVAL
    assert lib.sw_plan_create(None, 1, 1, None, ctypes.byref(z)) == swgb.SW_EINVAL
    assert lib.sw_plan_search(None, None, None, 0, 10, 2, None, None, None) == swgb.SW_EINVAL
    assert lib.sw_plan_wait(None, 0) == swgb.SW_EINVAL
    assert lib.sw_align(None, None, None, 0, None, None, 0, 10, 2, None, None, None, 0,
                        None) == swgb.SW_EINVAL
    lib.sw_db_destroy(None)
    lib.sw_plan_destroy(None)
    assert lib.sw_db_subjects(None) == 0


def test_intpeak_rejects_bad_arguments_before_touching_the_gpu(lib):
    out = np.zeros(3, dtype=np.float64)
    p = out.ctypes.data_as(ctypes.c_void_p)
    assert lib.sw_intpeak(len(swgb.INTPEAK_OPS), 8, 256, 100, p) == swgb.SW_EINVAL
    assert lib.sw_intpeak(-1, 8, 256, 100, p) == swgb.SW_EINVAL
    assert lib.sw_intpeak(0, 0, 256, 100, p) == swgb.SW_EINVAL
    assert lib.sw_intpeak(0, 8, 2048, 100, p) == swgb.SW_EINVAL
    assert lib.sw_intpeak(0, 8, 256, 100, None) == swgb.SW_EINVAL
