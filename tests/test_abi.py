"""The C-ABI library builds, loads and exports every symbol include/fa.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1505_07959_gb300 import build, fa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fa_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return fa.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "fa_parareal_solve" in names and "fa_fine_sweep" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(fa.SYMBOLS), set(names) - set(fa.SYMBOLS)


def test_status_strings(lib):
    for s in range(8):
        assert fa.fa_status_string(s)
    assert fa.fa_status_string(0) == "ok"


@pytest.mark.parametrize("field,value", [("n", 0), ("N", 0), ("fine_steps", 0), ("coarse_steps", 0),
                                         ("T", 0.0), ("T", -1.0), ("max_iters", -1), ("flow", 3),
                                         ("fine_dtype", 9), ("coarse_dtype", 2), ("tol", -1.0),
                                         ("n", 20000), ("refine_steps", -2)])
def test_plan_rejects_bad_descriptors(lib, field, value):
    d = fa.fa_problem_desc(n=8, flow=0, T=1.0, N=2, coarse_steps=1, fine_steps=2, max_iters=2,
                           tol=0.0, fine_dtype=fa.FA_BF16X4, coarse_dtype=fa.FA_BF16X4,
                           refine_steps=0)
    setattr(d, field, value)
    h, ws = ctypes.c_void_p(), ctypes.c_size_t()
    st = lib.fa_plan(ctypes.byref(h), ctypes.byref(d), None, ctypes.byref(ws))
    assert st == 1, (field, value, st)
    assert fa.fa_last_error()
    assert not h.value


def test_null_plan_is_rejected(lib):
    assert lib.fa_fine_sweep(None, None, None) == 1
    assert lib.fa_parareal_solve(None, None, None, None, None) == 1
    assert lib.fa_plan_destroy(None) == 0


def test_product_pair_sets_match_header():
    """The dtype table of the binding follows the header's enum order."""
    src = open(os.path.join(ROOT, "include", "fa.h")).read()
    for name, val in fa.DTYPES.items():
        assert re.search(rf"FA_{name.upper()}\s*=\s*{val}\b", src), name
