"""The C ABI (include/*.h): the shared library builds, loads and exports every function the
headers declare; host-side validation rejects malformed patterns before any device work.
No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_11681_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(s_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_documented_calls():
    names = declared_functions()
    for must in ("s_pattern_create", "s_plan_create", "s_mul_masked", "s_mul_masked_adjoint", "s_add", "s_funm",
                 "s_norm_est", "s_build_create", "s_build_values", "s_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_validation_without_gpu():
    from paper_2211_11681_gb300 import sformat as sf
    bad = [
        (np.array([0, 3, 5]), np.array([0, 1]), np.array([0, 2, 3]), np.array([1, 0, 1])),   # unsorted row
        (np.array([0, 3, 5]), np.array([0, 1]), np.array([0, 1, 2]), np.array([0, 7])),      # column out of range
        (np.array([0, 3, 3]), np.array([0, 1]), np.array([0, 1, 2]), np.array([0, 1])),      # block on empty cluster
        (np.array([1, 3, 5]), np.array([0, 1]), np.array([0, 1, 2]), np.array([0, 1])),      # offsets not from 0
    ]
    for bo, lv, rp, ci in bad:
        with pytest.raises(sf.SFormatError) as e:
            sf.Pattern(bo, lv, rp, ci)
        assert e.value.status == sf.S_ERR_PATTERN


def test_null_arguments_are_rejected():
    from paper_2211_11681_gb300 import sformat as sf
    assert sf.lib.s_mul_masked(None, None, None, None, None) == sf.S_ERR_ARG
    assert sf.lib.s_plan_create(None, None, None, 0, None) == sf.S_ERR_ARG
    assert sf.lib.s_pattern_nnz(None) == -1
    assert "s_plan_create" in sf.lib.s_last_error().decode()


def test_binding_enums_match_the_header():
    # the ctypes binding passes plain ints: its precision and status values must be the
    # header's enumerators
    from paper_2211_11681_gb300 import sformat as sf
    text = open(os.path.join(ROOT, "include", "sformat.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(S_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    for name in ("S_FP64", "S_FP32", "S_BF16X3", "S_FP64_DF", "S_TF32X3", "S_OK", "S_ERR_ARG", "S_ERR_PATTERN",
                 "S_ERR_MISMATCH"):
        assert getattr(sf, name) == enums[name], name
    assert sf.PREC == {"fp64": enums["S_FP64"], "fp32": enums["S_FP32"], "bf16x3": enums["S_BF16X3"],
                       "fp64_df": enums["S_FP64_DF"], "tf32x3": enums["S_TF32X3"]}
