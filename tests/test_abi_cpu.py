"""CPU-side checks of the C-ABI library: it loads, exports every entry
point declared in include/rp.h, and rejects bad arguments before launching
anything (these calls never reach a GPU)."""
import ctypes as C
import os
import re

import pytest

import paper_1906_00142_gb300 as rp
from paper_1906_00142_gb300 import build as rpbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    rpbuild.build()
    return rp.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rp_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "rp_fit" in names and "rp_eval_search" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_strerror(lib):
    assert rp.rp_version() == 3
    assert rp.rp_strerror(0) == "ok"
    assert rp.rp_strerror(-1) == "invalid argument"
    assert rp.rp_strerror(-999) == "unknown error"


def test_program_size(lib):
    for K, d in [(1, 1), (7, 3), (1024, 3), (5, 4)]:
        a16 = lambda v: (v + 15) & ~15
        expect = 2 * a16(4 * K * 8) + a16(4 * K) + 4 * K * 66 * 8 * 2 * (d + 1)
        assert rp.rp_program_size(K, d) == expect
    assert rp.rp_program_size(3, 9) == 0


def test_argument_validation_without_launch(lib):
    d = rp.FitDesc(4, 100, 9, 1, 4, 0, 1e-12, None)          # degree 9: invalid
    assert lib.rp_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0, None) == -1
    d = rp.FitDesc(4, 100, 3, 17, 4, 0, 1e-12, None)         # bad precision
    assert lib.rp_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0, None) == -1
    d = rp.FitDesc(4, 100, 3, 1, 4, 0, 1e-12, None)          # null outputs
    assert lib.rp_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0, None) == -1
    d = rp.FitDesc(4, 100, 3, 1, 4, 0, 1e-8, None, 1234, 10, 0)   # point sets of 0 fits
    assert lib.rp_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0, None) == -1
    d = rp.FitDesc(4, 100, 3, 1, 4, 0, 1e-8, None, None, 0, 0, 7)     # reserved field set
    assert lib.rp_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0, None) == -1
    d = rp.FitDesc(0, 0, 3, 1, 4, 0, 1e-12, None)            # empty batch: ok, nothing launched
    assert lib.rp_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0, None) == 0
    ws = C.c_size_t(123)
    assert lib.rp_fit_workspace_size(C.byref(d), C.byref(ws)) == 0 and ws.value == 0
    hw = rp.hw_struct()
    hw_bad = rp.hw_struct(dict(issue_cycles=0.0))
    assert lib.rp_eval_search(None, 4, 3, C.byref(hw_bad), None, 10, None, None, None, None, None,
                              0, None) == -1
    assert lib.rp_eval_search(None, 4, 3, C.byref(hw), None, 10, None, None, None, None, None,
                              0, None) == -1
    assert lib.rp_eval_search(None, 4, 3, C.byref(hw), None, 0, None, None, None, None, None,
                              0, None) == 0
    assert lib.rp_program_pack(4, 0, None, None, None, None, None, None, 0, None) == -1
    assert lib.rp_adam_step(10, None, None, None, None, None, 0, 1e-3, 0.9, 0.999, 1e-8, None) == -1
    assert lib.rp_relmse_fwd(-1, 0, None, None, None, None, None, None, None, None) == -1


def test_tuning_argument_validation_without_launch(lib):
    d = rp.FitDesc(4, 100, 9, 1, 4, 0, 1e-12, None)          # degree 9: invalid
    c = C.c_int32(0)
    assert lib.rp_tune_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0,
                           None, C.byref(c)) == -1
    d = rp.FitDesc(4, 100, 3, 1, 4, 0, 1e-12, None)
    assert lib.rp_tune_fit(C.byref(d), None, None, None, None, None, None, None, None, None, 0,
                           None, None) == -1
    h = rp.hw_struct()
    t = C.c_int32(0)
    assert lib.rp_tune_search(None, 1, 3, C.byref(h), None, 10, None, None, None, None, None,
                              0, None, C.byref(t), None) == -1
    ws = C.c_size_t(0)
    d = rp.FitDesc(5, 100, 3, 1, 4, 0, 1e-12, None)
    assert lib.rp_fit_workspace_size(C.byref(d), C.byref(ws)) == 0 and ws.value == 32
    # the basis cache: none at FP64 precision (the counters only); bad
    # arguments rejected
    d64 = rp.FitDesc(5, 100, 3, 0, 4, 0, 1e-12, None)
    assert lib.rp_fit_cache_workspace_size(C.byref(d64), C.byref(ws)) == 0 and ws.value == 32
    assert lib.rp_fit_cache_workspace_size(C.byref(d), None) == -1
    bad = rp.FitDesc(5, 100, 9, 1, 4, 0, 1e-12, None)
    assert lib.rp_fit_cache_workspace_size(C.byref(bad), C.byref(ws)) == -1


def test_search_workspace_size(lib):
    """Closed form of rp_search_workspace_size: offsets int32[K+2], cursors
    int32[K+1], bucketed indices int32[Q], each rounded up to 16 bytes; 0
    below 32 queries per kernel and outside int32 positions."""
    a16 = lambda v: (v + 15) & ~15
    for K, Q in [(1, 32), (8, 5000), (1024, 1_000_000), (1024, 10_000_000), (3, 97)]:
        assert rp.rp_search_workspace_size(K, Q) == a16(4 * (K + 2)) + a16(4 * (K + 1)) + a16(4 * Q)
    for K, Q in [(1024, 3000), (1, 31), (0, 100), (5, 0), (1, 2**31 - 1)]:
        assert rp.rp_search_workspace_size(K, Q) == 0
    b = C.c_size_t(7)
    assert lib.rp_search_workspace_size(-1, 10, C.byref(b)) == -1
    assert lib.rp_search_workspace_size(1, 10, None) == -1


def test_search_workspace_checked_before_launch(lib):
    """A workspace that is too small or misaligned is rejected before any
    device work (the other pointers are never dereferenced)."""
    hw = rp.hw_struct()
    fake = C.c_void_p(1 << 20)      # 16-byte aligned, never dereferenced
    need = rp.rp_search_workspace_size(8, 5000)
    args = (fake, 8, 3, C.byref(hw), fake, 5000, fake, fake, fake, fake)
    assert lib.rp_eval_search(*args, fake, need - 16, None) == -3
    assert lib.rp_eval_search(*args, C.c_void_p((1 << 20) + 4), need, None) == -5
