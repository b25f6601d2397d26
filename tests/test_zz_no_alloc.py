"""tsqr_factor_r_noalloc: R with no workspace, for callers that cannot allocate device memory.

Its scratch is a static device array inside libtsqr.so that every call reuses.  The test calls
the entry point twice in a row through the C-ABI, on two different matrices, so the second call
starts from the first call's leftovers in that array, and compares each R with tsqr_factor's
R on the same input, within the parity tests' R tolerance (1e-10 relative).  This file sorts
last so a stop-at-first-failure run has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_0809_2407_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_matches_factor_twice():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_2407_gb300 import build, tsqr

    build.build()
    lib = tsqr.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a long tall case (chain count capped to fit the scratch) and a short one with a ragged tail
    for m, n, seed in ((1 << 20, 64, 901), (5000 + 77, 24, 902)):
        A = torch.from_numpy(inputs.gaussian(m, n, seed)).cuda()
        R_static = torch.full((n, n), np.nan, dtype=torch.float64, device="cuda")
        st = lib.tsqr_factor_r_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(R_static.data_ptr()),
                                       n, stream)
        assert st == 0, lib.tsqr_last_error().decode()
        f = tsqr.Factorization(A)
        torch.cuda.synchronize()
        assert f.status() == tsqr.TSQR_OK
        R_ref = f.R.cpu().numpy()
        R = R_static.cpu().numpy()
        f.close()
        assert np.all(np.isfinite(R))
        assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
        assert np.linalg.norm(R - R_ref) / np.linalg.norm(R_ref) <= 1e-10


def test_noalloc_rejects_bad_arguments():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_2407_gb300 import build, tsqr

    build.build()
    lib = tsqr.load()
    A = torch.zeros((100, 4), dtype=torch.float64, device="cuda")
    R = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert lib.tsqr_factor_r_noalloc(3, 4, ctypes.c_void_p(A.data_ptr()), 4, ctypes.c_void_p(R.data_ptr()), 4,
                                     None) == tsqr.TSQR_ERR_INVALID_ARG
    assert lib.tsqr_factor_r_noalloc(100, 3, ctypes.c_void_p(A.data_ptr()), 3, ctypes.c_void_p(R.data_ptr()), 4,
                                     None) == tsqr.TSQR_ERR_INVALID_ARG
