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
                                         ("T", 0.0), ("T", -1.0), ("max_iters", -1), ("flow", -1),
                                         ("fine_dtype", 9), ("coarse_dtype", 2), ("tol", -1.0),
                                         ("n", 20000), ("refine_steps", -2),
                                         ("coarse_kind", 2), ("coarse_kind", -1), ("flow", 4),
                                         ("method", 2), ("fine_scheme", 4), ("coarse_scheme", 4),
                                         ("coarse_scheme", -1)])
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
    assert lib.fa_plan_set_learned_check(None, 1) == 1


def test_product_pair_sets_match_header():
    """The dtype table of the binding follows the header's enum order."""
    src = open(os.path.join(ROOT, "include", "fa.h")).read()
    for name, val in fa.DTYPES.items():
        assert re.search(rf"FA_{name.upper()}\s*=\s*{val}\b", src), name


def test_learned_descriptor_rules(lib):
    """The learned coarse propagator takes one step per slice (FA_ERR_ARG otherwise) and has no
    square-root form (FA_ERR_UNSUPPORTED), both checked before any device query."""
    def plan(**kw):
        d = fa.fa_problem_desc(n=8, flow=0, T=1.0, N=2, coarse_steps=1, fine_steps=2, max_iters=2,
                               tol=0.0, fine_dtype=fa.FA_BF16X6, coarse_dtype=fa.FA_BF16X6,
                               refine_steps=0, coarse_kind=fa.FA_COARSE_LEARNED)
        for k, v in kw.items():
            setattr(d, k, v)
        h, ws = ctypes.c_void_p(), ctypes.c_size_t()
        return lib.fa_plan(ctypes.byref(h), ctypes.byref(d), None, ctypes.byref(ws))
    assert plan(coarse_steps=2) == 1
    assert plan(flow=2) == 7


def test_network_entry_points_check_arguments(lib):
    """Argument errors of the network kernels' entry points, reported without launching."""
    b = ctypes.c_size_t()
    assert lib.fa_mlp_scratch_bytes(0, ctypes.byref(b)) == 1
    assert lib.fa_mlp_scratch_bytes(4096, ctypes.byref(b)) == 0 and b.value > 4096 * 2000
    assert lib.fa_mlp_forward(None, 4, None, 32, None, None) == 1
    one = ctypes.c_void_p(256)   # never dereferenced: the call fails on its arguments first
    assert lib.fa_mlp_forward(one, 4, one, 7, one, None) == 1
    assert lib.fa_mlp_adam(one, one, one, one, 0, 1e-3, 0.9, 0.999, 1e-8, None) == 1
    assert lib.fa_mlp_loss_grad(one, 0, one, one, one, one, 1 << 20, None) == 1
    assert lib.fa_mlp_loss_grad(one, 16, one, one, one, one, 8, None) == 3
    assert lib.fa_plan_set_learned(None, None) == 1
    assert lib.fa_learned_records(None, None, None, None, None, 0) == 1
    assert lib.fa_plan_set_recorder(None, None, 0, None, 0) == 1


def test_blob_and_record_sizes_match_header():
    src = open(os.path.join(ROOT, "include", "fa.h")).read()
    from oracle import learned as L
    assert fa.FA_MLP_PARAMS == 2 * L.NFEAT + L.HID * L.NFEAT + L.HID + L.HID * L.HID + L.HID \
        + L.NOUT * L.HID + L.NOUT
    for name in ("FA_MLP_PARAMS", "FA_RECORD_DOUBLES", "FA_MLP_FEATURES", "FA_MLP_HIDDEN",
                 "FA_MLP_COEFS", "FA_PROBES"):
        assert re.search(rf"#define {name} {getattr(fa, name)}\b", src), name
    assert re.search(r"#define FA_PROBE_SEED 0x150507959ULL", src)
    assert fa.FA_PROBE_SEED == L.PROBE_SEED
    assert L.to_blob(L.init_params(0)).size == fa.FA_MLP_PARAMS


def test_wait_fault_switch_checks_its_argument(lib):
    assert lib.fa_debug_set_wait_fault(-1, 0) == 1          # FA_ERR_ARG
    assert lib.fa_debug_set_wait_fault(0, -1) == 0          # normal operation
