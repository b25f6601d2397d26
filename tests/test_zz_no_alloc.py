"""tsqr_factor_r_noalloc: R with no workspace, for callers that cannot allocate device memory.

Its scratch is a static device array inside libtsqr.so that every call reuses.  The tests call
the entry point several times in a row through the C-ABI, on different matrices, so each call
starts from the previous call's leftovers in that array.  R is held per element to the FP64
oracle's R (the sign-normalised Householder R) on a small ragged case, and to tsqr_factor's R on
two tall cases: n = 64 at m = 2^20, whose chain count is capped so the tree's R factors fit the
array, and n = 16 at m = 2^22; all within the parity tests' R tolerance (1e-10 relative to
max |R|).  The failure path is
checked without a GPU fault: the status word a timed-out device wait would set is set from the
host, the poll reports TSQR_ERR_TIMEOUT, and the next call clears it.  This file sorts last so a
stop-at-first-failure run has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0809_2407_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_R = 1e-10


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_2407_gb300 import build, tsqr

    build.build()
    tsqr.load()
    return tsqr


def noalloc_r(T, A):
    import torch

    m, n = A.shape
    lib = T.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    R = torch.full((n, n), np.nan, dtype=torch.float64, device="cuda")
    st = lib.tsqr_factor_r_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(R.data_ptr()), n, stream)
    assert st == 0, lib.tsqr_last_error().decode()
    poll, _ = T.tsqr_noalloc_status_poll(stream)
    assert poll == T.TSQR_OK
    return R.cpu().numpy()


def check_r(R, R_ref):
    assert np.all(np.isfinite(R))
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    assert np.abs(R - R_ref).max() <= TOL_R * np.abs(R_ref).max()


def test_noalloc_matches_oracle_and_factor(T):
    import torch

    # a short case with a ragged last leaf against the oracle, then tall cases against
    # tsqr_factor (n = 64: chain count capped to fit the scratch), then the short case again
    small = inputs.gaussian(5000 + 77, 24, 902)
    R_oracle = oracle.qr(small, want_q=False)["R"]
    check_r(noalloc_r(T, torch.from_numpy(small).cuda()), R_oracle)
    for m, n, seed in ((1 << 20, 64, 901), (1 << 22, 16, 903)):
        A = torch.from_numpy(inputs.gaussian(m, n, seed)).cuda()
        R = noalloc_r(T, A)
        f = T.Factorization(A)
        torch.cuda.synchronize()
        assert f.status() == T.TSQR_OK
        R_ref = f.R.cpu().numpy()
        f.close()
        check_r(R, R_ref)
        del A
    check_r(noalloc_r(T, torch.from_numpy(small).cuda()), R_oracle)


def test_noalloc_timeout_reaches_the_host(T):
    """The status word of the static scratch, set here from the host as a timed-out device wait
    would set it, is reported by tsqr_noalloc_status_poll; the next call clears it."""
    import torch

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    A_h = inputs.gaussian(3000, 16, 904)
    A = torch.from_numpy(A_h).cuda()
    noalloc_r(T, A)
    st, addr = T.tsqr_noalloc_status_poll(stream)
    assert st == T.TSQR_OK and addr
    word = _device_int(addr)
    word.fill_(1)
    st, _ = T.tsqr_noalloc_status_poll(stream)
    assert st == T.TSQR_ERR_TIMEOUT
    R = noalloc_r(T, A)  # clears the word, and R is right again
    check_r(R, oracle.qr(A_h, want_q=False)["R"])


class _DeviceWord:
    """A 4-byte int32 at a device address, exposed to torch through the CUDA array interface."""

    def __init__(self, addr):
        self.__cuda_array_interface__ = {"shape": (1,), "typestr": "<i4", "data": (addr, False), "version": 3}


def _device_int(addr):
    import torch

    return torch.as_tensor(_DeviceWord(addr), device="cuda")


def test_noalloc_rejects_bad_arguments(T):
    import torch

    lib = T.load()
    A = torch.zeros((100, 4), dtype=torch.float64, device="cuda")
    R = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert lib.tsqr_factor_r_noalloc(3, 4, ctypes.c_void_p(A.data_ptr()), 4, ctypes.c_void_p(R.data_ptr()), 4,
                                     None) == T.TSQR_ERR_INVALID_ARG
    assert lib.tsqr_factor_r_noalloc(100, 3, ctypes.c_void_p(A.data_ptr()), 3, ctypes.c_void_p(R.data_ptr()), 4,
                                     None) == T.TSQR_ERR_INVALID_ARG
