"""Host-side checks of the C-ABI (no GPU): the library loads, exports every call the header
declares, plans and sizes workspaces, and rejects bad arguments before launching anything."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0809_2407_gb300 import build, tsqr

    build.build()
    return tsqr


def header_functions():
    text = open(os.path.join(ROOT, "include", "tsqr.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|tsqr_status_t)\s+(tsqr_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    so = ctypes.CDLL(lib.LIB_PATH)
    for nm in names:
        assert hasattr(so, nm), nm
    assert set(names) == set(lib.EXPORTED)


def test_status_strings(lib):
    L = lib.load()
    for s, nm in enumerate(["TSQR_OK", "TSQR_ERR_INVALID_ARG", "TSQR_ERR_UNSUPPORTED", "TSQR_ERR_CUDA",
                            "TSQR_ERR_WORKSPACE", "TSQR_ERR_TIMEOUT"]):
        assert L.tsqr_status_string(s).decode() == nm


def test_workspace_size_grows_with_m(lib):
    a = lib.tsqr_workspace_size(lib.TSQR_F64, 4096, 16, {"leaf_h": 256, "chain": 1, "arity": 2})
    b = lib.tsqr_workspace_size(lib.TSQR_F64, 8192, 16, {"leaf_h": 256, "chain": 1, "arity": 2})
    assert 0 < a < b
    # in-place storage drops the m x n reflector copy
    c = lib.tsqr_workspace_size(lib.TSQR_F64, 8192, 16, {"leaf_h": 256, "chain": 1, "arity": 2, "inplace": 1})
    assert b - c >= 8192 * 16 * 8


@pytest.mark.parametrize("m,n,opts,status", [
    (10, 20, None, 1),                      # m < n
    (100, 0, None, 1),                      # n < 1
    (10000, 5000, None, 2),                 # n > 4096
    (1000, 200, {"precision": 4}, 2),       # every panel's plan is checked
    (1000, 16, {"arity": 1}, 1),
    (1000, 16, {"arity": 9}, 1),
    (1000, 16, {"leaf_h": 12}, 1),          # not a multiple of 8
    (1000, 16, {"leaf_h": 8}, 1),           # below padded n
    (1000, 16, {"leaf_h": 384}, 1),         # above 256 but not a multiple of 256
    (1000, 16, {"precision": 4}, 2),
])
def test_invalid_plans(lib, m, n, opts, status):
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_workspace_size(lib.TSQR_F64, m, n, opts)
    assert ei.value.status == status


def test_factor_rejects_before_launch(lib):
    L = lib.load()
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every case fails validation first
    # lda < n
    assert L.tsqr_factor(0, 0, 100, 3, fake, 2, fake, 3, fake, 1 << 20, None, None, ctypes.byref(h)) == 1
    # A not even 8-byte aligned
    assert L.tsqr_factor(0, 0, 100, 4, ctypes.c_void_p(0x1004), 4, fake, 4, fake, 1 << 20, None, None,
                         ctypes.byref(h)) == 1
    # in place needs a TMA-compatible A (even lda, 16-byte aligned)
    inpl = lib.Opts(inplace=1)
    assert L.tsqr_factor(0, 0, 100, 3, fake, 3, fake, 3, fake, 1 << 20, ctypes.byref(inpl), None,
                         ctypes.byref(h)) == 1
    assert L.tsqr_factor(0, 0, 100, 4, ctypes.c_void_p(0x1008), 4, fake, 4, fake, 1 << 20, ctypes.byref(inpl),
                         None, ctypes.byref(h)) == 1
    # column-major needs lda >= m; FP32 keeps A read-only, runs precision 0 only, and checks its
    # workspace and 4-byte alignment like FP64
    assert L.tsqr_factor(0, 1, 100, 4, fake, 4, fake, 4, fake, 1 << 20, None, None, ctypes.byref(h)) == 1
    assert L.tsqr_factor(1, 0, 100, 4, fake, 4, fake, 4, fake, 1 << 20, ctypes.byref(inpl), None,
                         ctypes.byref(h)) == 2
    assert L.tsqr_factor(1, 0, 100, 4, fake, 4, fake, 4, fake, 1 << 20, ctypes.byref(lib.Opts(precision=1)), None,
                         ctypes.byref(h)) == 2
    assert L.tsqr_factor(1, 0, 100, 4, fake, 4, fake, 4, fake, 16, None, None, ctypes.byref(h)) == 4
    assert L.tsqr_factor(1, 0, 100, 4, ctypes.c_void_p(0x1002), 4, fake, 4, fake, 1 << 20, None, None,
                         ctypes.byref(h)) == 1
    assert L.tsqr_factor(7, 0, 100, 4, fake, 4, fake, 4, fake, 1 << 20, None, None, ctypes.byref(h)) == 1
    # workspace too small
    assert L.tsqr_factor(0, 0, 100, 4, fake, 4, fake, 4, fake, 16, None, None, ctypes.byref(h)) == 4
    assert h.value is None
    assert b"workspace" in L.tsqr_last_error()
    # NULL handle everywhere
    assert L.tsqr_form_q(None, fake, 4, None) == 1
    assert L.tsqr_apply_qt(None, 1, fake, 1, None) == 1
    assert L.tsqr_apply_q(None, 1, fake, 1, None) == 1
    assert L.tsqr_status_poll(None, None) == 1
    assert L.tsqr_destroy(None) == 0


def test_batch_plans_and_errors(lib):
    m, n = [1000, 5000, 300, 77777], [8, 16, 50, 64]
    size = lib.tsqr_batch_workspace_size(lib.TSQR_F64, 4, m, n)
    single = sum(lib.tsqr_workspace_size(lib.TSQR_F64, mm, nn) for mm, nn in zip(m, n))
    assert size >= single // 2  # every item keeps its own factors
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_batch_workspace_size(lib.TSQR_F64, 2, [10, 100], [20, 4])  # item 0: m < n
    assert ei.value.status == 1 and "item 0" in str(ei.value)
    with pytest.raises(lib.TsqrError):
        lib.tsqr_batch_workspace_size(lib.TSQR_F64, 0, [], [])
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_batch_workspace_size(lib.TSQR_F64, 1, [100], [4], {"inplace": 1})
    assert ei.value.status == 2


def test_batch_per_item_plans(lib):
    """tsqr_batch_workspace_size_plans: a plan per matrix; the workspace follows each plan (shorter
    leaves keep more T factors), mixed precisions and bad plans are refused with the item named."""
    m, n = [20000, 5000, 3000], [64, 16, 50]
    O = lib.Opts
    base = lib.tsqr_batch_workspace_size_plans(lib.TSQR_F64, 3, m, n, [O(), O(), O()])
    assert base == lib.tsqr_batch_workspace_size(lib.TSQR_F64, 3, m, n)
    small_leaves = lib.tsqr_batch_workspace_size_plans(lib.TSQR_F64, 3, m, n,
                                                       [O(leaf_h=64), O(leaf_h=64), O(leaf_h=64)])
    assert small_leaves > base
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_batch_workspace_size_plans(lib.TSQR_F64, 3, m, n, [O(), O(precision=1), O()])
    assert ei.value.status == 2
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_batch_workspace_size_plans(lib.TSQR_F64, 3, m, n, [O(), O(), O(leaf_h=20)])
    assert ei.value.status == 1 and "item 2" in str(ei.value)


def test_autotune_candidates_and_key(lib):
    c = lib.candidate_opts(1 << 20, 64)
    assert len(c) >= 6
    assert all(o.leaf_h >= 64 for o in c)
    assert lib.tune_key(1 << 20, 50, 0) == (20, 64, 0, lib.TSQR_F64)
    assert lib.tune_key(3 << 19, 9, 1) == (20, 16, 1, lib.TSQR_F64)
    assert lib.tune_key(3 << 19, 9, 0, lib.TSQR_F32) == (20, 16, 0, lib.TSQR_F32)
    assert len(lib.candidate_opts(1 << 20, 64, 0, lib.TSQR_F32)) >= 6


def test_panel_workspace(lib):
    """n > 64: a staged copy of A plus one in-place TSQR workspace per 64-column panel."""
    m = 100000
    one = lib.tsqr_workspace_size(lib.TSQR_F64, m, 64, {"inplace": 1})
    two = lib.tsqr_workspace_size(lib.TSQR_F64, m, 128)
    two_inplace = lib.tsqr_workspace_size(lib.TSQR_F64, m, 128, {"inplace": 1})
    assert two - two_inplace >= m * 128 * 8
    assert two_inplace >= one + lib.tsqr_workspace_size(lib.TSQR_F64, m - 64, 64, {"inplace": 1})
    # a 65th column adds a narrow panel
    assert lib.tsqr_workspace_size(lib.TSQR_F64, m, 65, {"inplace": 1}) > one


def test_f32_workspace(lib):
    """FP32 storage: A is always widened into the workspace, so its size matches FP64's non-inplace
    layout; in-place factorizations and the other precision modes stay FP64 only."""
    for m, n in [(4096, 16), (100000, 64), (100000, 100)]:
        assert lib.tsqr_workspace_size(lib.TSQR_F32, m, n) > 0
    assert lib.tsqr_workspace_size(lib.TSQR_F32, 100000, 64) == lib.tsqr_workspace_size(lib.TSQR_F64, 100000, 64)
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_workspace_size(lib.TSQR_F32, 1000, 16, {"inplace": 1})
    assert ei.value.status == 2
    assert lib.tsqr_batch_workspace_size(lib.TSQR_F32, 2, [1000, 5000], [16, 50]) > 0
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_batch_workspace_size(lib.TSQR_F32, 1, [1000], [16], {"precision": 1})
    assert ei.value.status == 2


def test_panel_factor_rejects_before_launch(lib):
    L = lib.load()
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    inpl = lib.Opts(inplace=1)
    # in place needs an even lda for the panels too
    assert L.tsqr_factor(0, 0, 1000, 100, fake, 101, fake, 100, fake, 1 << 30, ctypes.byref(inpl), None,
                         ctypes.byref(h)) == 1
    # workspace too small
    assert L.tsqr_factor(0, 0, 1000, 100, fake, 100, fake, 100, fake, 1 << 10, None, None, ctypes.byref(h)) == 4
    assert h.value is None


def test_r_only_plans(lib):
    """R alone keeps no reflectors, tau or T: a smaller workspace; it excludes inplace, panels
    and batches."""
    m, n = 100000, 64
    full = lib.tsqr_workspace_size(lib.TSQR_F64, m, n)
    r = lib.tsqr_workspace_size(lib.TSQR_F64, m, n, {"r_only": 1})
    assert 0 < r < full
    assert full - r >= (m // 96) * 64 * 64 * 8  # the per-leaf T factors at least
    for opts, n_, status in [({"r_only": 1, "inplace": 1}, 64, 1), ({"r_only": 1}, 100, 2)]:
        with pytest.raises(lib.TsqrError) as ei:
            lib.tsqr_workspace_size(lib.TSQR_F64, m, n_, opts)
        assert ei.value.status == status
    with pytest.raises(lib.TsqrError) as ei:
        lib.tsqr_batch_workspace_size(lib.TSQR_F64, 1, [1000], [16], {"r_only": 1})
    assert ei.value.status == 2


def test_column_major_checks(lib):
    """Column-major A needs lda >= m, n <= 64 and no inplace; all rejected before any launch."""
    L = lib.load()
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    col = lib.TSQR_COL_MAJOR
    assert L.tsqr_factor(0, col, 100, 4, fake, 99, fake, 4, fake, 1 << 20, None, None, ctypes.byref(h)) == 1
    assert L.tsqr_factor(0, col, 1000, 100, fake, 1000, fake, 100, fake, 1 << 30, None, None, ctypes.byref(h)) == 2
    inpl = lib.Opts(inplace=1)
    assert L.tsqr_factor(0, col, 100, 4, fake, 100, fake, 4, fake, 1 << 20, ctypes.byref(inpl), None,
                         ctypes.byref(h)) == 1
    assert L.tsqr_factor(0, 7, 100, 4, fake, 100, fake, 4, fake, 1 << 20, None, None, ctypes.byref(h)) == 1
    assert h.value is None
