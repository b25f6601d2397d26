"""GPU parity: the CUDA TSQR against the FP64 CPU oracle, through the C-ABI.

Both arithmetic modes are held to the FP64-level bar: backward error ||A - QR||_F/||A||_F
<= 1e-12 and orthogonality ||I - Q^T Q||_F <= 1e-12 everywhere; R within 1e-10 relative of the
oracle's R when kappa(A) <= 1e6, where the sign-normalised thin QR is unique.  Q is compared
elementwise with a bound from QR perturbation theory: two backward-stable factorizations differ
in Q by about kappa(A) * n * u, so the test allows 50 * kappa * n * u (at least 1e-13), with u
the unit roundoff of the mode: 2^-53 for native FP64, 2^-46 for double-float (two FP32 halves
with 24 + 24 significant bits, less the guard bits the sloppy sum gives up), 2^-50 for the
Ozaki tensor-core products (56-bit fixed point per row/column, 9-term truncation).
"""
import numpy as np
import pytest

import oracle
from paper_0809_2407_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_BACK = 1e-12
TOL_ORTH = 1e-12
TOL_R = 1e-10
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_2407_gb300 import build, tsqr

    build.build()
    tsqr.load()
    return tsqr


def run(T, A_h, lda=None, **opts):
    import torch

    m, n = A_h.shape
    if lda is not None and lda != n:
        buf = torch.zeros((m, lda), dtype=torch.float64, device="cuda")
        buf[:, :n] = torch.from_numpy(A_h).cuda()
        A = buf[:, :n]
    else:
        A = torch.from_numpy(np.ascontiguousarray(A_h)).cuda()
    f = T.Factorization(A, **opts)
    Q = f.form_q()
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    return f, f.R.cpu().numpy(), Q.cpu().numpy()


UNIT = {0: 2.0 ** -53, 1: 2.0 ** -46, 2: 2.0 ** -50, 3: 2.0 ** -46}


@pytest.fixture(params=[0, 1, 2, 3], ids=["f64", "df", "ozaki", "df_ozaki"])
def prec(request):
    return request.param


def check_against_oracle(A_h, R, Q, unique=True, precision=0):
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    assert oracle.backward_error(A_h, Q, R) <= TOL_BACK
    assert oracle.orthogonality(Q) <= TOL_ORTH
    if unique:
        ref = oracle.qr(A_h)
        assert np.linalg.norm(R - ref["R"]) / np.linalg.norm(ref["R"]) <= TOL_R
        assert np.abs(R - ref["R"]).max() <= TOL_R * np.abs(ref["R"]).max()  # and per element
        kappa = np.linalg.cond(ref["R"])
        n = A_h.shape[1]
        assert np.abs(Q - ref["Q"]).max() <= max(1e-13, 50 * kappa * n * UNIT[precision])


def test_config1_binary_tree(T, prec):
    """4096 x 16 N(0,1), leaf height 256, binary tree over 16 leaves."""
    A_h = inputs.gaussian(4096, 16, inputs.seed_for(1, 0))
    f, R, Q = run(T, A_h, leaf_h=256, chain=1, arity=2, precision=prec)
    info = f.info()
    assert (info.leaves, info.chains, info.depth) == (16, 16, 4)
    check_against_oracle(A_h, R, Q, precision=prec)


@pytest.mark.parametrize("chain,arity", [(1, 2), (1, 3), (1, 4), (1, 8), (2, 2), (3, 2), (5, 3), (0, 2), (1000, 2)])
def test_tree_shapes(T, chain, arity, prec):
    """Any tree gives the QR of A (Sec. 2): binary, k-ary, flat chains, hybrids, single chain."""
    A_h = inputs.gaussian(3000, 24, inputs.seed_for(2, chain * 10 + arity))
    _, R, Q = run(T, A_h, leaf_h=128, chain=chain, arity=arity, precision=prec)
    check_against_oracle(A_h, R, Q, precision=prec)


@pytest.mark.parametrize("m,n,h", [(4096 + 77, 16, 256), (1000, 64, 128), (129, 64, 64), (65, 64, 64),
                                   (130, 30, 64), (16, 16, 16), (1, 1, 16), (777, 1, 16), (5000, 5, 512),
                                   (2000, 50, 128), (3333, 33, 128), (64 * 7 + 3, 64, 64)])
def test_ragged_and_edge_shapes(T, m, n, h, prec):
    A_h = inputs.gaussian(m, n, inputs.seed_for(3, m + n + h))
    lda = n + (n % 2)
    _, R, Q = run(T, A_h, lda=lda, leaf_h=h, chain=0 if m > 1000 else 2, arity=2, precision=prec)
    check_against_oracle(A_h, R, Q, precision=prec)


@pytest.mark.parametrize("m,n", [(40000 + 13, 64), (30000, 50), (60000 + 7, 32), (50000, 33), (100000 + 3, 16),
                                 (70000, 17), (9000, 64)])
def test_default_plan_shapes(T, m, n, prec):
    """The default plans (leaf height 96/256/512 for n up to 64/32/16) run the scheduled chain step."""
    A_h = inputs.gaussian(m, n, inputs.seed_for(3, m + n))
    f, R, Q = run(T, A_h, precision=prec)
    assert f.info().leaf_h == {64: 96, 32: 256, 16: 512}[f.info().np]
    check_against_oracle(A_h, R, Q, precision=prec)


BLOCKED_SHAPES = [(40000 + 13, 64, {}), (30000, 50, {}), (50000, 33, {}), (20000, 64, {"chain": 5}),
                  (64 * 7 + 5, 64, {"chain": 8}), (8000, 40, {}), (100000 + 77, 64, {"chain": 40})]


@pytest.mark.parametrize("m,n,opts", BLOCKED_SHAPES)
def test_blocked_tensor_core_step_ozaki(T, m, n, opts):
    """Precision mode 2 with 64-row leaves at padded width 64 runs the blocked flat-tree step: FP64
    reflectors panel by panel, the panels' WY products and the Gram entries feeding T as Ozaki
    tensor-core products.  R, Q and Q^T b against the oracle; R alone bitwise the full R."""
    import torch

    A_h = inputs.gaussian(m, n, inputs.seed_for(30, m + n))
    f, R, Q = run(T, A_h, precision=2, leaf_h=64, **opts)
    assert f.info().leaf_h == 64 and f.info().np == 64
    check_against_oracle(A_h, R, Q, precision=2)
    b_h = inputs.gaussian(m, 1, inputs.seed_for(31, m))
    b = torch.from_numpy(b_h.copy()).cuda()
    f.apply_qt(b)
    torch.cuda.synchronize()
    assert np.abs(b[:n].cpu().numpy() - oracle.thin_qt(A_h, b_h)[:n]).max() <= 1e-12 * np.linalg.norm(b_h)
    fr = T.Factorization(torch.from_numpy(A_h).cuda(), precision=2, leaf_h=64, r_only=True, **opts)
    torch.cuda.synchronize()
    assert fr.status() == T.TSQR_OK
    assert np.array_equal(fr.R.cpu().numpy(), R)
    fr.close()
    f.close()


OZAKI_PHASE_SHAPES = [
    (96 * 40 + 50, 64, {"chain": 1}),   # every leaf starts a chain: no leaf products kernel work
    (96 * 40 + 50, 64, {"chain": 41}),  # one chain, no tree: the recurrence starts from the signs
    (96 * 41 + 20, 64, {"chain": 5}),   # a short last leaf joins the last chain, taken whole
    (96 * 37 + 70, 33, {"chain": 4}),   # odd n, ragged last leaf of at least n rows
    (96 * 300 + 1, 64, {}),             # the default plan; a one-row last leaf
]


@pytest.mark.parametrize("m,n,opts", OZAKI_PHASE_SHAPES)
@pytest.mark.parametrize("precision", [2, 3], ids=["ozaki", "df_ozaki"])
def test_ozaki_thin_q_phases(T, m, n, opts, precision):
    """The tensor-core thin Q of modes 2 and 3 runs as the chains' recurrences (M = T C into
    each later leaf's rows of Q), the chains' first leaves, and the other leaves' products -V M.
    Q against the oracle elementwise and against the FP64-pipe thin Q of the same factorization's
    arithmetic (mode 0 for mode 2, mode 1 for mode 3), in row- and column-major layout."""
    import torch

    A_h = inputs.gaussian(m, n, inputs.seed_for(43, m + n))
    f, R, Q = run(T, A_h, precision=precision, **opts)
    check_against_oracle(A_h, R, Q, precision=precision)
    _, R0, Q0 = run(T, A_h, precision=precision - 2, **opts)
    assert np.array_equal(R, R0)  # the factorization is the same; only the thin Q's products differ
    assert np.abs(Q - Q0).max() <= 1e-13
    # column-major: the same Q, bitwise
    A_col = torch.from_numpy(np.ascontiguousarray(A_h.T)).cuda().t()
    fc = T.Factorization(A_col, precision=precision, **opts)
    Qc = fc.form_q()
    torch.cuda.synchronize()
    assert fc.status() == T.TSQR_OK and Qc.stride(0) == 1
    assert np.array_equal(Qc.cpu().numpy(), Q)
    fc.close()
    f.close()


def test_short_last_leaf_is_merged(T):
    """A last leaf with fewer than n rows joins the previous chain instead of starting one."""
    A_h = inputs.gaussian(64 * 4 + 5, 32, 77)
    f, R, Q = run(T, A_h, leaf_h=64, chain=1, arity=2)
    assert f.info().chains == 4
    check_against_oracle(A_h, R, Q)


@pytest.mark.parametrize("lda_extra,offset", [(0, 0), (1, 0), (0, 1), (3, 1)])
def test_staged_layouts(T, lda_extra, offset):
    """Odd leading dimensions and 8-byte (not 16-byte) aligned A go through the staging copy."""
    import torch

    m, n = 3001, 21
    A_h = inputs.gaussian(m, n, 404 + lda_extra)
    lda = n + lda_extra
    buf = torch.zeros(m * lda + 2, dtype=torch.float64, device="cuda")
    A = buf[offset:offset + m * lda].view(m, lda)[:, :n]
    A.copy_(torch.from_numpy(A_h))
    f = T.Factorization(A)
    Q = f.form_q()
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    check_against_oracle(A_h, f.R.cpu().numpy(), Q.cpu().numpy())
    assert np.array_equal(A.cpu().numpy(), A_h)  # A untouched


def test_strided_and_inplace(T):
    import torch

    A_h = inputs.gaussian(2500, 20, 31)
    _, R1, Q1 = run(T, A_h, lda=36, leaf_h=128, chain=3)
    check_against_oracle(A_h, R1, Q1)
    A = torch.from_numpy(A_h.copy()).cuda()
    f = T.Factorization(A, leaf_h=128, chain=3, inplace=True)
    Q2 = f.form_q().cpu().numpy()
    assert np.array_equal(f.R.cpu().numpy(), R1)
    assert np.array_equal(Q2, Q1)
    # the reflectors now live in A
    assert not np.array_equal(A.cpu().numpy(), A_h)


@pytest.mark.parametrize("kind,k", [("usv", 0), ("usv", 6), ("usv", 12), ("krylov", None)])
def test_conditioning(T, kind, k, prec):
    m, n = 1 << 14, 32
    A_h = inputs.usv(m, n, k, 55 + (k or 0)) if kind == "usv" else inputs.krylov(m, n, 56)
    _, R, Q = run(T, A_h, leaf_h=256, precision=prec)
    check_against_oracle(A_h, R, Q, unique=(kind == "usv" and k <= 6), precision=prec)


def test_apply_qt_apply_q(T, prec):
    import torch

    m, n, k = 5000, 24, 7
    A_h = inputs.gaussian(m, n, 91)
    B_h = inputs.gaussian(m, k, 92)
    f, R, Q = run(T, A_h, leaf_h=128, chain=4, arity=3, precision=prec)
    tol = 1e-11 if prec == 0 else 1e-10
    B = torch.from_numpy(B_h.copy()).cuda()
    f.apply_qt(B)
    QtB = B.cpu().numpy()
    # thin part against the oracle: D (H_{n-1} ... H_0 B)_{0:n}
    assert np.abs(QtB[:n] - oracle.thin_qt(A_h, B_h)).max() <= tol
    # Q^T is orthogonal: norms of columns kept
    assert np.allclose(np.linalg.norm(QtB, axis=0), np.linalg.norm(B_h, axis=0), rtol=100 * UNIT[prec])
    # Q^T A = [R; 0]
    Ad = torch.from_numpy(A_h.copy()).cuda()
    f.apply_qt(Ad)
    QtA = Ad.cpu().numpy()
    assert np.abs(QtA[:n] - R).max() <= tol * np.abs(R).max()
    assert np.abs(QtA[n:]).max() <= tol * np.abs(R).max()
    # Q Q^T B = B
    f.apply_q(B)
    assert np.abs(B.cpu().numpy() - B_h).max() <= 100 * tol
    # form_q equals Q [I; 0]
    E = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    E[:n] = torch.eye(n, dtype=torch.float64, device="cuda")
    f.apply_q(E)
    assert np.abs(E.cpu().numpy() - Q).max() <= 100 * n * UNIT[prec]


@pytest.mark.parametrize("k", [1, 2, 33, 64 * 32 + 5])
def test_apply_column_counts(T, k):
    import torch

    m, n = 3000, 16
    A_h = inputs.gaussian(m, n, 101)
    B_h = inputs.gaussian(m, k, 102)
    f, _, _ = run(T, A_h, leaf_h=256, chain=2)
    B = torch.from_numpy(B_h.copy()).cuda()
    f.apply_qt(B)
    assert np.abs(B.cpu().numpy()[:n] - oracle.thin_qt(A_h, B_h)).max() <= 1e-11
    f.apply_q(B)
    assert np.abs(B.cpu().numpy() - B_h).max() <= 1e-12


@pytest.mark.parametrize("m,n,k,opts", [
    (20000, 64, 64, {}),                                # default plan (h = 96): W over 64 + 32 rows
    (20000 + 37, 48, 100, {"leaf_h": 128, "chain": 3}),  # n < 64, 2 x 64 rows, ragged leaf, 64 + 36 columns
    (9000, 64, 33, {"leaf_h": 64, "chain": 1}),          # one part of 64 rows; every leaf a chain's first
    (700, 64, 129, {"leaf_h": 96, "chain": 64}),        # one chain: no tree, the signs in the chain kernel
    (6000, 40, 32, {"leaf_h": 80, "chain": 2, "arity": 3}),  # ternary tree levels after the chains
])
def test_apply_ozaki(T, m, n, k, opts):
    """Q^T B and Q B with the chains' WY products as Ozaki splits on the tensor cores (precision
    modes 2 and 3 from 32 columns of B on).  Where mode 2 factors in native FP64 exactly as mode
    0 does (plans other than the blocked step's: leaf height other than 64), its Q^T B and Q B
    must equal mode 0's FP64-pipe results over all m rows to the accuracy of the split products
    (2^-50 relative to the rows and columns involved); otherwise, and in mode 3, Q^T B is held to
    the oracle's thin part and to the invariants Q^T A = [R; 0], Q Q^T B = B and
    Q [I; 0] = thin Q."""
    import torch

    A_h = inputs.gaussian(m, n, inputs.seed_for(18, m + n + k))
    B_h = inputs.gaussian(m, k, inputs.seed_for(19, m + k))
    A = torch.from_numpy(A_h).cuda()
    f0 = T.Factorization(A, precision=0, **opts)
    B0 = torch.from_numpy(B_h.copy()).cuda()
    f0.apply_qt(B0)
    for prec in (2, 3):
        f = T.Factorization(A, precision=prec, **opts)
        Q = f.form_q()
        R = f.R
        B = torch.from_numpy(B_h.copy()).cuda()
        f.apply_qt(B)
        torch.cuda.synchronize()
        assert f.status() == T.TSQR_OK
        QtB = B.cpu().numpy()
        assert np.abs(QtB[:n] - oracle.thin_qt(A_h, B_h)).max() <= 1e-10
        info = f.info()
        blocked = info.np == 64 and info.leaf_h == 64 and info.arity == 2
        if prec == 2 and not blocked:
            assert torch.equal(R, f0.R)  # the same FP64 factorization
            assert (B - B0).abs().max().item() <= 1e-12 * B0.abs().max().item()
        Ad = A.clone()
        f.apply_qt(Ad)
        Rn = R.cpu().numpy()
        QtA = Ad.cpu().numpy()
        assert np.abs(QtA[:n] - Rn).max() <= 1e-10 * np.abs(Rn).max()
        assert np.abs(QtA[n:]).max() <= 1e-10 * np.abs(Rn).max()
        f.apply_q(B)
        assert np.abs(B.cpu().numpy() - B_h).max() <= 1e-10
        E = torch.zeros((m, max(n, 32)), dtype=torch.float64, device="cuda")
        E[:n, :n] = torch.eye(n, dtype=torch.float64, device="cuda")
        f.apply_q(E)
        assert (E[:, :n] - Q).abs().max().item() <= 100 * n * UNIT[prec]
        assert torch.all(E[:, n:] == 0)
        f.close()
    f0.close()


@pytest.mark.parametrize("m,n,k,opts", [
    (20000, 64, 64, {}),
    (20000 + 37, 48, 100, {"leaf_h": 128, "chain": 3}),
    (9000, 64, 33, {"leaf_h": 64, "chain": 1}),
    (700, 64, 129, {"leaf_h": 96, "chain": 64}),
    (6000, 40, 32, {"leaf_h": 80, "chain": 2, "arity": 3}),
])
def test_apply_tc_matches_narrow(T, m, n, k, opts):
    """From 32 columns of B on, Q^T B and Q B take the tensor-core chain kernels (Ozaki splits in
    mode 3, bf16x3 terms in FP32 storage); narrower blocks run the FP64 / double-float / FP32
    pipe kernels.  On the same factorization the two must agree column block by column block:
    B in one call against B in slices of 16 columns, to the accuracy of the form (1e-12 relative
    for mode 3; FP32: 50 n u with u = 2^-24)."""
    import torch

    A_h = inputs.gaussian(m, n, inputs.seed_for(21, m + n + k))
    B_h = inputs.gaussian(m, k, inputs.seed_for(22, m + k))
    for dt, prec, tol in ((torch.float64, 3, 1e-12), (torch.float32, 0, 50 * n * U32)):
        A = torch.from_numpy(A_h).to(dt).cuda()
        f = T.Factorization(A, precision=prec, **opts)
        B = torch.from_numpy(B_h).to(dt).cuda()
        Bn = B.clone()
        f.apply_qt(B)
        for c in range(0, k, 16):
            blk = Bn[:, c:c + 16].contiguous()
            f.apply_qt(blk)
            Bn[:, c:c + 16] = blk
        torch.cuda.synchronize()
        assert f.status() == T.TSQR_OK
        scale = B.abs().max().item()
        assert (B - Bn).abs().max().item() <= tol * scale, (dt, (B - Bn).abs().max().item() / scale)
        B_thin = B[:n].double().cpu().numpy()
        ref = oracle.thin_qt(A.double().cpu().numpy(), B_h.astype(np.float64) if dt == torch.float64 else
                             torch.from_numpy(B_h).float().double().numpy())
        assert np.abs(B_thin - ref).max() <= (1e-10 if dt == torch.float64 else 50 * n * U32 * np.abs(ref).max())
        f.apply_q(B)
        for c in range(0, k, 16):
            blk = Bn[:, c:c + 16].contiguous()
            f.apply_q(blk)
            Bn[:, c:c + 16] = blk
        torch.cuda.synchronize()
        assert (B - Bn).abs().max().item() <= tol * scale
        B0 = torch.from_numpy(B_h).to(dt).cuda()
        assert (B - B0).abs().max().item() <= tol * B0.abs().max().item()  # Q Q^T B = B
        f.close()


def test_apply_bf16x3_panels(T):
    """FP32 storage with n > 64: the panels' trailing updates take the bf16x3 Q^T B / Q B (64
    trailing columns at n = 128); backward error and orthogonality within the FP32 bar."""
    import torch

    m, n = 30000, 128
    A32 = inputs.gaussian(m, n, inputs.seed_for(23, 1)).astype(np.float32)
    A = torch.from_numpy(A32).cuda()
    f = T.Factorization(A)
    Q = f.form_q()
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK and f.info().panels == 2
    Qd, Rd = Q.double().cpu().numpy(), f.R.double().cpu().numpy()
    assert oracle.backward_error(A32.astype(np.float64), Qd, Rd) <= TOL_F32
    assert oracle.orthogonality(Qd) <= TOL_F32
    f.close()


@pytest.mark.parametrize("dtype,prec", [("float64", 2), ("float32", 0)])
def test_apply_tc_column_major(T, dtype, prec):
    """The tensor-core Q^T B and Q B (Ozaki in mode 2, bf16x3 in FP32 storage) read and write B in
    a column-major handle's layout: bitwise the row-major results."""
    import torch

    tdt = getattr(torch, dtype)
    m, n, k = 7000, 64, 70
    A_h = inputs.gaussian(m, n, inputs.seed_for(20, 1))
    B_h = inputs.gaussian(m, k, inputs.seed_for(20, 2))
    A_row = torch.from_numpy(A_h).to(tdt).cuda()
    A_col = torch.from_numpy(A_h.T.copy()).to(tdt).cuda().t()
    f_row, f_col = T.Factorization(A_row, precision=prec), T.Factorization(A_col, precision=prec)
    B_row = torch.from_numpy(B_h).to(tdt).cuda()
    B_col = torch.from_numpy(B_h.T.copy()).to(tdt).cuda().t()
    f_row.apply_qt(B_row)
    f_col.apply_qt(B_col)
    torch.cuda.synchronize()
    assert torch.equal(B_col, B_row)
    f_row.apply_q(B_row)
    f_col.apply_q(B_col)
    torch.cuda.synchronize()
    assert torch.equal(B_col, B_row)
    tol = 1e-10 if dtype == "float64" else 50 * n * U32 * np.abs(B_h).max()
    assert np.abs(B_row.double().cpu().numpy() - torch.from_numpy(B_h).to(tdt).double().numpy()).max() <= tol


@pytest.mark.parametrize("m,n,opts", [(20000, 128, {}), (5000 + 33, 65, {"leaf_h": 128}),
                                      (3001, 100, {"chain": 2, "arity": 3}), (2000, 200, {}), (300, 150, {}),
                                      (129, 129, {}), (64 * 9 + 7, 128, {"leaf_h": 64, "chain": 1})])
def test_panels_n_above_64(T, m, n, opts, prec):
    """n > 64: right-looking blocked QR over 64-column TSQR panels (Sec. 6, Algorithm 3)."""
    import torch

    A_h = inputs.gaussian(m, n, inputs.seed_for(9, m + n))
    f, R, Q = run(T, A_h, precision=prec, **opts)
    assert f.info().panels == (n + 63) // 64
    check_against_oracle(A_h, R, Q, precision=prec)
    tol = 1e-11 if prec == 0 else 1e-10
    k = 5
    B_h = inputs.gaussian(m, k, inputs.seed_for(10, m + n))
    B = torch.from_numpy(B_h.copy()).cuda()
    f.apply_qt(B)
    QtB = B.cpu().numpy()
    assert np.abs(QtB[:n] - oracle.thin_qt(A_h, B_h)).max() <= tol
    Ad = torch.from_numpy(A_h.copy()).cuda()
    f.apply_qt(Ad)
    QtA = Ad.cpu().numpy()
    assert np.abs(QtA[:n] - R).max() <= tol * np.abs(R).max()
    if m > n:
        assert np.abs(QtA[n:]).max() <= tol * np.abs(R).max()
    f.apply_q(B)
    assert np.abs(B.cpu().numpy() - B_h).max() <= 100 * tol
    E = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    E[:n] = torch.eye(n, dtype=torch.float64, device="cuda")
    f.apply_q(E)
    assert np.abs(E.cpu().numpy() - Q).max() <= 100 * n * UNIT[prec]


def test_panels_staged_and_inplace(T):
    """n > 64 with an odd lda (staged) and in place: the same arithmetic, bitwise."""
    import torch

    m, n = 4000, 96
    A_h = inputs.gaussian(m, n, 812)
    _, R1, Q1 = run(T, A_h)
    _, R2, Q2 = run(T, A_h, lda=n + 1)
    assert np.array_equal(R1, R2) and np.array_equal(Q1, Q2)
    A = torch.from_numpy(A_h.copy()).cuda()
    f = T.Factorization(A, inplace=True)
    Q3 = f.form_q()
    torch.cuda.synchronize()
    assert np.array_equal(f.R.cpu().numpy(), R1) and np.array_equal(Q3.cpu().numpy(), Q1)
    check_against_oracle(A_h, R1, Q1)


@pytest.mark.parametrize("m,n,h,arity", [(2048, 16, 128, 4), (2048, 16, 128, 2), (4096, 32, 128, 2),
                                         (4096 + 64, 64, 64, 2), (6000, 50, 96, 2)])
def test_node_structure_eq_fact_2rs(T, m, n, h, arity):
    """Tree-node reflectors: lower blocks upper triangular (eq. fact_2rs), T upper triangular,
    for k-ary nodes and for the structured binary node step; R and Q against the oracle."""
    A_h = inputs.gaussian(m, n, 5)
    f, R, Q = run(T, A_h, leaf_h=h, chain=1, arity=arity)
    check_against_oracle(A_h, R, Q)
    info = f.info()
    assert info.arity == arity and info.depth >= 2
    np_ = info.np
    Y = workspace_view(f, info.node_y, info.tree_nodes * (info.arity - 1) * np_ * np_)
    Y = Y.reshape(info.tree_nodes, info.arity - 1, np_, np_)
    assert np.all(np.tril(Y, -1) == 0.0)
    assert np.count_nonzero(np.triu(Y[:, :, :16, :16])) > 0
    Tn = workspace_view(f, info.node_t, info.tree_nodes * np_ * np_).reshape(info.tree_nodes, np_, np_)
    assert np.all(np.tril(Tn, -1) == 0.0)
    tau = workspace_view(f, info.node_tau, info.tree_nodes * np_).reshape(info.tree_nodes, np_)
    assert np.array_equal(np.diagonal(Tn, axis1=1, axis2=2), tau)


def leaf_factors(f, info, precision):
    """V (m x n), tau (leaves x np) and T (leaves x np x np) of a factorization as FP64, decoding
    the double-float pairs of modes 1 and 3 (hi in the low word) into hi + lo."""
    import torch

    np_, leaves = info.np, info.leaves

    def decode(ptr, count):
        raw = workspace_view(f, ptr, count)
        if precision in (1, 3):
            pairs = raw.view(np.float32).reshape(-1, 2).astype(np.float64)
            return pairs[:, 0] + pairs[:, 1]
        return raw

    torch.cuda.synchronize()
    V = decode(info.v, info.m * info.ldv).reshape(info.m, info.ldv)[:, :info.n]
    tau = decode(info.tau_leaf, leaves * np_).reshape(leaves, np_)
    Tl = decode(info.t_leaf, leaves * np_ * np_).reshape(leaves, np_, np_)
    return V, tau, Tl


@pytest.mark.parametrize("n", [64, 50, 33])
def test_gram_entries_on_tensor_cores(T, n):
    """The Ozaki WY form (mode 2) takes the Gram entries v_p^T v_q of each flat-tree step's T on
    the tensor cores; modes 0 and 3 take them in the column loop.  For every step, in every mode,
    T^-1 = diag(1/tau) + the strict upper part of V^T V (Sec. 3.2: the
    compact-WY T of reflectors with tau = 2 / v^T v; the unit top parts are orthogonal, so V^T V
    is the leaf rows' Gram), checked with numpy's FP64 Gram of the stored reflectors; in mode 2
    R, V and tau are bitwise mode 0's and T agrees with mode 0's to the products' accuracy."""
    import torch

    h, chain, chains = 96, 4, 3
    m = h * chain * chains
    A_h = inputs.gaussian(m, n, inputs.seed_for(41, n))
    A = torch.from_numpy(A_h).cuda()
    got = {}
    for prec in (0, 2, 3):
        f = T.Factorization(A, precision=prec, leaf_h=h, chain=chain, arity=2)
        info = f.info()
        assert (info.np, info.leaf_h, info.chain, info.leaves) == (64, h, chain, chain * chains)
        V, tau, Tl = leaf_factors(f, info, prec)
        got[prec] = (f.R.cpu().numpy(), V, tau, Tl)
        for leaf in range(info.leaves):
            if leaf % chain == 0:
                continue  # a chain's first leaf: plain Householder QR, T by its own recurrence
            Vb = V[leaf * h:(leaf + 1) * h]
            M = np.triu(Vb.T @ Vb, 1) + np.diag(1.0 / tau[leaf, :n])
            Tn = Tl[leaf, :n, :n]
            assert np.all(np.tril(Tl[leaf], -1) == 0.0) and np.all(Tl[leaf, n:] == 0.0)
            assert np.abs(Tn @ M - np.eye(n)).max() <= (1e-12 if prec != 3 else 1e-9), (prec, leaf)
        f.close()
    R0, V0, tau0, T0 = got[0]
    R2, V2, tau2, T2 = got[2]
    assert np.array_equal(R2, R0) and np.array_equal(V2, V0) and np.array_equal(tau2, tau0)
    assert np.abs(T2 - T0).max() <= 1e-13 * np.abs(T0).max()


def workspace_view(f, ptr, count):
    """`count` doubles of the factorization's workspace starting at device pointer ptr."""
    import torch

    torch.cuda.synchronize()
    off = ptr - f.work.data_ptr()
    assert 0 <= off and off + 8 * count <= f.work.numel()
    return f.work[off:off + 8 * count].view(torch.float64).cpu().numpy()


def test_deterministic(T):
    A_h = inputs.gaussian(20000, 32, 17)
    _, R1, Q1 = run(T, A_h)
    _, R2, Q2 = run(T, A_h)
    assert np.array_equal(R1, R2) and np.array_equal(Q1, Q2)


def test_virtual_ranks(T):
    """Distributed TSQR algebra on one GPU: factor P row slabs separately, then the stacked R's."""
    import torch

    A_h = inputs.gaussian(8000, 16, 23)
    _, R_one, _ = run(T, A_h)
    Rs = []
    for s in np.array_split(np.arange(8000), 4):
        _, Rp, _ = run(T, A_h[s])
        Rs.append(Rp)
    _, R_two, _ = run(T, np.vstack(Rs), leaf_h=16, chain=1)
    assert np.abs(R_two - R_one).max() <= 1e-12 * np.abs(R_one).max()


@pytest.fixture(scope="module")
def full_size_oracle():
    """The oracle on the benchmark's own matrix (m = 2^22, n = 64, A = U Sigma V^T with kappa = 1,
    the benchmark's seed) and on b: R and the top n rows of Q^T b, sign-normalised.  Computed
    once per module: about a minute of single-threaded FP64 work on the host."""
    m, n = 1 << 22, 64
    A_h = inputs.usv(m, n, 0.0, inputs.seed_for(2, 0))
    b = inputs.gaussian(m, 1, inputs.seed_for(2, 101))[:, 0]
    ref = oracle.qr(A_h, want_q=False)
    qtb = ref["D"] * oracle.apply_qt(ref["V"], ref["tau"], b)[:n]
    return A_h, b, ref["R"], qtb


@pytest.mark.timeout(1500, method="thread")
def test_full_size_against_oracle(T, full_size_oracle, prec):
    """Parity at the benchmark's configuration: every FP64-storage precision form's R equals the
    oracle's per element within 1e-10 of max |R|, and its Q^T b (top n rows) the oracle's within
    1e-12 of ||b||, on the benchmark's matrix and launch configuration."""
    import torch

    A_h, b_h, R_ref, qtb_ref = full_size_oracle
    n = A_h.shape[1]
    A = torch.from_numpy(A_h).cuda()
    f = T.Factorization(A, precision=prec)
    b = torch.from_numpy(b_h.copy()).cuda().reshape(-1, 1)
    f.apply_qt(b)
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    R = f.R.cpu().numpy()
    qtb = b[:n, 0].cpu().numpy()
    f.close()
    del A, b
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    assert np.abs(R - R_ref).max() <= TOL_R * np.abs(R_ref).max()
    assert np.abs(qtb - qtb_ref).max() <= 1e-12 * np.linalg.norm(b_h)


def test_full_size_properties(T, prec):
    """m = 2^22, n = 64, A = U Sigma V^T with kappa = 1 (the benchmark's workload and launch
    configuration).  At kappa = 1 the Cholesky factor of A^T A (a library routine on the Gram
    matrix) equals R to ~eps, which pins R elementwise; A = QR and Q^T Q = I are checked with
    FP64 GEMMs on the device.  Q^T b (the benchmark's k = 1) and Q^T B, Q B with 64 columns (on
    the tensor cores in modes 2 and 3) are held to Q_thin^T B from an FP64 GEMM with the thin Q,
    and to Q Q^T B = B."""
    import torch

    m, n = 1 << 22, 64
    A_h = inputs.usv(m, n, 0.0, inputs.seed_for(2, 0))
    A = torch.from_numpy(A_h).cuda()
    f = T.Factorization(A, precision=prec)
    Q = f.form_q()
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    R = f.R
    G = A_h.T @ A_h
    L = np.linalg.cholesky(G)
    Rc = L.T
    assert np.abs(R.cpu().numpy() - Rc).max() <= 1e-12 * (1 if prec == 0 else 16)
    be = (torch.linalg.norm(A - Q @ R) / torch.linalg.norm(A)).item()
    orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - Q.T @ Q).item()
    assert be <= TOL_BACK and orth <= TOL_ORTH
    del A
    for k in (1, 64):
        B0 = torch.from_numpy(inputs.gaussian(m, k, inputs.seed_for(2, 100 + k))).cuda()
        B = B0.clone()
        f.apply_qt(B)
        ref = Q.T @ B0
        torch.cuda.synchronize()
        assert f.status() == T.TSQR_OK
        scale = torch.linalg.norm(B0, dim=0).max().item()
        assert (B[:n] - ref).abs().max().item() <= 1e-12 * scale, (k, (B[:n] - ref).abs().max().item() / scale)
        f.apply_q(B)
        assert (B - B0).abs().max().item() <= 1e-12 * scale
        del B0, B, ref
    f.close()


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_batched_uneven(T, precision):
    """One launch for many matrices of uneven m and n (block Krylov / s-step batches); in modes 2
    and 3 the thin Q of the matrices of n in 33..64 runs its WY products on the tensor cores."""
    import torch

    rng = np.random.default_rng(4)
    ms = [int(x) for x in np.exp(rng.uniform(np.log(300), np.log(40000), 14)).astype(int)]
    ns = [int(x) for x in rng.choice([8, 16, 32, 50, 64], 14)]
    ms = [max(m_, n_) for m_, n_ in zip(ms, ns)]
    hs = [inputs.gaussian(m_, n_, 5000 + i) for i, (m_, n_) in enumerate(zip(ms, ns))]
    mats = [torch.from_numpy(a).cuda() for a in hs]
    b = T.Batch(mats, precision=precision)
    b.factor()
    b.form_q()
    torch.cuda.synchronize()
    assert b.status() == T.TSQR_OK
    for a, R, Q in zip(hs, b.R, b.Q):
        check_against_oracle(a, R.cpu().numpy(), Q.cpu().numpy(), precision=precision)
    b.close()


def test_batched_per_item_plans(T):
    """A plan per matrix (leaf height, arity, chain length) in one persistent launch, FP64 and
    double-float, and the plans autotune_batch picks on the batch itself: every matrix against
    the oracle."""
    import torch

    rng = np.random.default_rng(41)
    ms = [int(x) for x in np.exp(rng.uniform(np.log(500), np.log(60000), 12)).astype(int)]
    ns = [int(x) for x in rng.choice([8, 16, 32, 50, 64], 12)]
    ms = [max(m_, n_) for m_, n_ in zip(ms, ns)]
    hs = [inputs.gaussian(m_, n_, 6000 + i) for i, (m_, n_) in enumerate(zip(ms, ns))]
    mats = [torch.from_numpy(a).cuda() for a in hs]
    choice = {16: (512, 4), 32: (128, 2), 64: (128, 4)}
    for precision in (0, 1):
        plans = [T.Opts(leaf_h=choice[T.padded_width(n_)][0], arity=choice[T.padded_width(n_)][1],
                        chain=(3 if i % 3 == 0 else 0), precision=precision) for i, n_ in enumerate(ns)]
        b = T.Batch(mats, precision=precision, plans=plans)
        b.factor()
        b.form_q()
        torch.cuda.synchronize()
        assert b.status() == T.TSQR_OK
        for a, R, Q in zip(hs, b.R, b.Q):
            check_against_oracle(a, R.cpu().numpy(), Q.cpu().numpy(), precision=precision)
        b.close()
    plans, picked = T.autotune_batch(mats, leaf_hs=(64, 256), arities=(2, 4), reps=1)
    assert set(picked) == {T.padded_width(n_) for n_ in ns}
    b = T.Batch(mats, plans=plans)
    b.factor()
    b.form_q()
    torch.cuda.synchronize()
    assert b.status() == T.TSQR_OK
    for a, R, Q in zip(hs, b.R, b.Q):
        check_against_oracle(a, R.cpu().numpy(), Q.cpu().numpy())
    b.close()
    # mixed precisions are refused before anything launches
    bad = [T.Opts(precision=i % 2) for i in range(len(ns))]
    with pytest.raises(T.TsqrError):
        T.Batch(mats, plans=bad)


def test_batched_cuda_graph(T):
    """tsqr_batch_factor / tsqr_batch_form_q captured once in a CUDA graph and replayed."""
    import torch

    hs = [inputs.gaussian(4000 + 37 * i, 16 + 8 * (i % 3), 6000 + i) for i in range(6)]
    mats = [torch.from_numpy(a).cuda() for a in hs]
    b = T.Batch(mats)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.factor()
        b.form_q()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    R0 = [R.clone() for R in b.R]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.factor()
        b.form_q()
    for R in b.R:
        R.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for R, r0, a, Q in zip(b.R, R0, hs, b.Q):
        assert torch.equal(R, r0)
        check_against_oracle(a, R.cpu().numpy(), Q.cpu().numpy())
    b.close()


def test_autotune_returns_valid_plan(T):
    import torch

    o = T.autotune(20000, 24, reps=1, proxy_rows=20000)
    A_h = inputs.gaussian(20000, 24, 31337)
    _, R, Q = run(T, A_h, leaf_h=o.leaf_h, chain=o.chain, arity=o.arity)
    check_against_oracle(A_h, R, Q)
    assert T.autotune(20000, 24) is not None  # cached
    o32 = T.autotune(20000, 24, reps=1, proxy_rows=20000, dtype=torch.float32)  # FP32 storage, own key
    A32 = torch.from_numpy(A_h).float().cuda()
    f = T.Factorization(A32, leaf_h=o32.leaf_h, chain=o32.chain, arity=o32.arity)
    Q = f.form_q().double()
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    assert torch.linalg.norm(torch.eye(24, dtype=torch.float64, device="cuda") - Q.T @ Q).item() <= 5e-5
    f.close()


# ---- FP32 storage (TSQR_F32): FP32-level bar, 5e-5 on backward error and orthogonality -------
TOL_F32 = 5e-5
U32 = 2.0 ** -24


def run32(T, A64, lda=None, offset=0, **opts):
    """Factor the float32 rounding of A64; returns the handle, R and Q as float64 arrays."""
    import torch

    m, n = A64.shape
    lda = lda or n
    buf = torch.zeros(m * lda + offset, dtype=torch.float32, device="cuda")
    A = buf[offset:offset + m * lda].view(m, lda)[:, :n]
    A.copy_(torch.from_numpy(A64.astype(np.float32)))
    f = T.Factorization(A, **opts)
    Q = f.form_q()
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    assert f.R.dtype == torch.float32 and Q.dtype == torch.float32
    assert np.array_equal(A.cpu().numpy(), A64.astype(np.float32))  # A is read only
    return f, f.R.cpu().numpy().astype(np.float64), Q.cpu().numpy().astype(np.float64)


def check_f32(A32, R, Q, unique=True):
    """A32: the float32 input as float64.  Measures against it; R and Q against the oracle's QR
    of it within the perturbation bound 50 kappa n u with u = 2^-24."""
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    assert oracle.backward_error(A32, Q, R) <= TOL_F32
    assert oracle.orthogonality(Q) <= TOL_F32
    if unique:
        ref = oracle.qr(A32)
        kappa = np.linalg.cond(ref["R"])
        bound = 50 * kappa * A32.shape[1] * U32
        assert np.linalg.norm(R - ref["R"]) / np.linalg.norm(ref["R"]) <= bound
        assert np.abs(Q - ref["Q"]).max() <= bound


@pytest.mark.parametrize("m,n,opts", OZAKI_PHASE_SHAPES)
def test_f32_thin_q_phases(T, m, n, opts):
    """FP32 storage at padded width 64 forms the thin Q as the chains' recurrences (M = T C on the
    FP32 pipe, into each later leaf's rows of Q), the chains' first leaves, and the other leaves'
    products -Y M as bf16x3 tensor-core terms.  Q against the oracle's QR of the float32 input,
    and the column-major layout bitwise the same."""
    import torch

    A32 = inputs.gaussian(m, n, inputs.seed_for(44, m + n)).astype(np.float32).astype(np.float64)
    f, R, Q = run32(T, A32, **opts)
    check_f32(A32, R, Q)
    A_col = torch.from_numpy(np.ascontiguousarray(A32.T.astype(np.float32))).cuda().t()
    fc = T.Factorization(A_col, **opts)
    Qc = fc.form_q()
    torch.cuda.synchronize()
    assert fc.status() == T.TSQR_OK and Qc.stride(0) == 1
    assert np.array_equal(Qc.cpu().numpy().astype(np.float64), Q)
    fc.close()
    f.close()


@pytest.mark.parametrize("m,n,opts", [(4096, 16, {"leaf_h": 256, "chain": 1, "arity": 2}),
                                      (3000, 24, {"leaf_h": 128, "chain": 3, "arity": 3}),
                                      (40000 + 13, 64, {}), (30000, 50, {}), (100000 + 3, 16, {}),
                                      (60000 + 7, 32, {}), (777, 1, {"leaf_h": 16}), (65, 64, {"leaf_h": 64}),
                                      (20000, 128, {}), (5000 + 33, 65, {"leaf_h": 128})])
def test_f32_shapes(T, m, n, opts):
    """FP32 storage and arithmetic on the tree shapes, default plans, ragged tails and panels."""
    A64 = inputs.gaussian(m, n, inputs.seed_for(11, m + n))
    A32 = A64.astype(np.float32).astype(np.float64)
    f, R, Q = run32(T, A64, **opts)
    assert f.info().dtype == T.TSQR_F32
    check_f32(A32, R, Q)


@pytest.mark.parametrize("m,n,opts", BLOCKED_SHAPES)
def test_blocked_tensor_core_step_f32(T, m, n, opts):
    """FP32 storage with 64-row leaves at padded width 64 runs the blocked flat-tree step: FP32
    reflectors panel by panel, the panels' WY products and the Gram entries feeding T as bf16x3
    tensor-core products.  R and Q against the oracle at the FP32 bar; R alone bitwise the full R."""
    import torch

    A64 = inputs.gaussian(m, n, inputs.seed_for(32, m + n))
    A32 = A64.astype(np.float32).astype(np.float64)
    f, R, Q = run32(T, A64, leaf_h=64, **opts)
    assert f.info().leaf_h == 64 and f.info().np == 64
    check_f32(A32, R, Q)
    fr = T.Factorization(torch.from_numpy(A64.astype(np.float32)).cuda(), leaf_h=64, r_only=True, **opts)
    torch.cuda.synchronize()
    assert fr.status() == T.TSQR_OK
    assert np.array_equal(fr.R.cpu().numpy().astype(np.float64), R)
    fr.close()
    f.close()


@pytest.mark.parametrize("lda_extra,offset", [(1, 0), (0, 1), (5, 3)])
def test_f32_strided(T, lda_extra, offset):
    A64 = inputs.gaussian(3001, 21, 912 + lda_extra)
    A32 = A64.astype(np.float32).astype(np.float64)
    _, R, Q = run32(T, A64, lda=21 + lda_extra, offset=offset)
    check_f32(A32, R, Q)


@pytest.mark.parametrize("k", [0, 4, 8])
def test_f32_conditioning(T, k):
    """kappa = 1, 1e4, 1e8 (the precision-form inputs); at 1e8 > 1/u the float32 matrix is
    numerically rank deficient, so only backward error and orthogonality are checked."""
    A64 = inputs.usv(1 << 15, 64, k, 57 + k)
    A32 = A64.astype(np.float32).astype(np.float64)
    _, R, Q = run32(T, A64)
    check_f32(A32, R, Q, unique=(k <= 4))


@pytest.mark.parametrize("n", [24, 100])
def test_f32_apply(T, n):
    import torch

    m, k = 7001, 6
    A64 = inputs.gaussian(m, n, 93 + n)
    A32 = A64.astype(np.float32).astype(np.float64)
    B32 = inputs.gaussian(m, k, 94).astype(np.float32)
    f, R, Q = run32(T, A64)
    B = torch.from_numpy(B32.copy()).cuda()
    f.apply_qt(B)
    QtB = B.cpu().numpy().astype(np.float64)
    scale = np.linalg.norm(B32.astype(np.float64), axis=0).max()
    assert np.abs(QtB[:n] - oracle.thin_qt(A32, B32.astype(np.float64))).max() <= 1e-4 * scale
    f.apply_q(B)
    assert np.abs(B.cpu().numpy() - B32).max() <= 1e-5 * scale
    E = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    E[:n] = torch.eye(n, dtype=torch.float32, device="cuda")
    f.apply_q(E)
    assert np.abs(E.cpu().numpy() - Q).max() <= 100 * n * U32


def test_f32_batched_uneven_and_graph(T):
    """FP32 batch: uneven m and n in one persistent launch, widened on the device, replayed from a
    CUDA graph with bitwise equal R."""
    import torch

    rng = np.random.default_rng(14)
    ms = [int(x) for x in np.exp(rng.uniform(np.log(300), np.log(40000), 12)).astype(int)]
    ns = [int(x) for x in rng.choice([8, 16, 32, 50, 64], 12)]
    ms = [max(m_, n_) for m_, n_ in zip(ms, ns)]
    hs = [inputs.gaussian(m_, n_, 7000 + i).astype(np.float32) for i, (m_, n_) in enumerate(zip(ms, ns))]
    mats = [torch.from_numpy(a).cuda() for a in hs]
    b = T.Batch(mats)
    b.factor()
    b.form_q()
    torch.cuda.synchronize()
    assert b.status() == T.TSQR_OK
    R0 = [R.clone() for R in b.R]
    for a, R, Q in zip(hs, b.R, b.Q):
        assert R.dtype == torch.float32
        check_f32(a.astype(np.float64), R.cpu().numpy().astype(np.float64), Q.cpu().numpy().astype(np.float64))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.factor()
        b.form_q()
    for R in b.R:
        R.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for R, r0 in zip(b.R, R0):
        assert torch.equal(R, r0)
    b.close()


def test_f32_full_size_properties(T):
    """m = 2^22, n = 64 in FP32 storage (the benchmark's launch configuration: 144-leaf chains and
    the bf16x3 tensor-core thin Q).  Long chains are where an inexact C recurrence would show;
    backward error and orthogonality are checked with FP64 GEMMs on the device, R against the
    Cholesky factor of the float32 A's Gram matrix within the FP32 perturbation bound."""
    import torch

    m, n = 1 << 22, 64
    A32 = inputs.usv(m, n, 0.0, inputs.seed_for(2, 0)).astype(np.float32)
    A = torch.from_numpy(A32).cuda()
    f = T.Factorization(A)
    Q = f.form_q()
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    Ad, Qd, Rd = A.double(), Q.double(), f.R.double()
    be = (torch.linalg.norm(Ad - Qd @ Rd) / torch.linalg.norm(Ad)).item()
    orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - Qd.T @ Qd).item()
    assert be <= TOL_F32 and orth <= TOL_F32
    Rc = np.linalg.cholesky(A32.astype(np.float64).T @ A32.astype(np.float64)).T
    assert np.abs(Rd.cpu().numpy() - Rc).max() <= 50 * n * U32 * np.abs(Rc).max()


@pytest.mark.parametrize("n", [32, 64, 128])
def test_precision_forms_conditioning(T, n):
    """The precision forms on the conditioning sweep of their workload (A = U S V^T, kappa = 1,
    1e4, 1e8, m = 2^20): every FP64-level form within 1e-12 on backward error and orthogonality,
    the FP32 form within 5e-5, whatever kappa (Householder QR is backward stable)."""
    import torch

    m = 1 << 20
    for k in (0, 4, 8):
        A_h = inputs.usv(m, n, k, inputs.seed_for(12, 10 * n + k))
        A = torch.from_numpy(A_h).cuda()
        for prec in (0, 1, 2, 3):
            f = T.Factorization(A, precision=prec)
            Q = f.form_q()
            torch.cuda.synchronize()
            assert f.status() == T.TSQR_OK
            be = (torch.linalg.norm(A - Q @ f.R) / torch.linalg.norm(A)).item()
            orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - Q.T @ Q).item()
            assert be <= TOL_BACK and orth <= TOL_ORTH, (k, prec, be, orth)
            f.close()
        A32 = A.float()
        f = T.Factorization(A32)
        Q = f.form_q().double()
        torch.cuda.synchronize()
        Ad = A32.double()
        be = (torch.linalg.norm(Ad - Q @ f.R.double()) / torch.linalg.norm(Ad)).item()
        orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device="cuda") - Q.T @ Q).item()
        assert be <= TOL_F32 and orth <= TOL_F32, (k, "f32", be, orth)
        f.close()


@pytest.mark.parametrize("kind", ["zero_matrix", "zero_first_last", "zero_middle", "duplicate_columns"])
def test_degenerate_inputs(T, kind, prec):
    """Degenerate cases of the method: H = I reflectors (tau = 0) everywhere or in some columns,
    and exact rank deficiency.  Householder QR stays backward stable and Q orthonormal.  R is
    compared with the oracle where it is unique: a zero first column leaves q_0 = e_0 in both
    (their first reflector is the identity), a zero last column has nothing to its right.  After
    a zero middle column j, q_j and row j of R depend on the reflectors before it, which differ
    between the tree and the oracle, so only the invariants are checked there."""
    m, n = 5000, 40
    A_h = inputs.gaussian(m, n, inputs.seed_for(14, n))
    if kind == "zero_matrix":
        A_h[:] = 0.0
    elif kind == "zero_first_last":
        A_h[:, [0, 39]] = 0.0
    elif kind == "zero_middle":
        A_h[:, 7] = 0.0
    else:
        A_h[:, 5] = A_h[:, 3]
        A_h[:, 20] = 2.0 * A_h[:, 11]
    f, R, Q = run(T, A_h, leaf_h=128, chain=3, precision=prec)
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    assert oracle.orthogonality(Q) <= TOL_ORTH
    if kind == "zero_matrix":
        assert np.all(R == 0.0)
        assert np.array_equal(Q[:n], np.eye(n)) and np.all(Q[n:] == 0.0)  # Q = [I; 0], the oracle's
    else:
        assert np.linalg.norm(A_h - Q @ R) <= TOL_BACK * np.linalg.norm(A_h)
    if kind == "zero_first_last":
        ref = oracle.qr(A_h)
        assert np.abs(R - ref["R"]).max() <= 1e-10 * np.abs(ref["R"]).max()
        assert R[0, 0] == 0.0 and R[39, 39] == 0.0


@pytest.mark.parametrize("kind", ["zero_matrix", "zero_first_last", "zero_middle", "duplicate_columns", "nan",
                                  "scale_-600", "scale_600"])
def test_blocked_step_degenerate_inputs(T, kind):
    """The blocked tensor-core step (precision mode 2, 64-row leaves) on the degenerate cases of
    the method: H = I reflectors, exact rank deficiency, NaN propagating without a fault, and
    entries near the ends of the exponent range (the Ozaki products scale every operand row and
    column by its own exponent)."""
    m, n = 6000, 50
    A_h = inputs.gaussian(m, n, inputs.seed_for(33, n))
    if kind == "zero_matrix":
        A_h[:] = 0.0
    elif kind == "zero_first_last":
        A_h[:, [0, n - 1]] = 0.0
    elif kind == "zero_middle":
        A_h[:, 20] = 0.0
    elif kind == "duplicate_columns":
        A_h[:, 5] = A_h[:, 3]
        A_h[:, 40] = 2.0 * A_h[:, 17]
    elif kind == "nan":
        A_h[3333, 7] = np.nan
    else:
        A_h *= 2.0 ** int(kind.split("_")[1])
    f, R, Q = run(T, A_h, precision=2, leaf_h=64, chain=5)
    if kind == "nan":
        assert np.isnan(R).any()
        return
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    assert oracle.orthogonality(Q) <= TOL_ORTH
    if kind == "zero_matrix":
        assert np.all(R == 0.0)
        assert np.array_equal(Q[:n], np.eye(n)) and np.all(Q[n:] == 0.0)
        return
    assert oracle.backward_error(A_h, Q, R) <= TOL_BACK
    if kind in ("zero_first_last", "scale_-600", "scale_600"):
        ref = oracle.qr(A_h)
        s = 2.0 ** -int(kind.split("_")[1]) if kind.startswith("scale") else 1.0
        assert np.abs((R - ref["R"]) * s).max() <= 1e-10 * np.abs(ref["R"] * s).max()


@pytest.mark.parametrize("scale_exp", [-600, -90, 90, 600])
def test_extreme_scaling(T, scale_exp, prec):
    """Entries near the ends of the exponent range: the FP64 norms rescale by the largest
    magnitude; double-float (modes 1 and 3) keeps full accuracy within about [2^-100, 2^100]
    (its FP32 exponent range), so it is held to that range only."""
    if prec in (1, 3) and abs(scale_exp) > 100:
        pytest.skip("outside the double-float range the header states")
    A_h = inputs.gaussian(3000, 24, inputs.seed_for(15, abs(scale_exp))) * 2.0 ** scale_exp
    f, R, Q = run(T, A_h, leaf_h=128, precision=prec)
    assert oracle.backward_error(A_h, Q, R) <= TOL_BACK
    assert oracle.orthogonality(Q) <= TOL_ORTH
    ref = oracle.qr(A_h)
    s = 2.0 ** -scale_exp  # exact rescaling, so the norms below neither underflow nor overflow
    assert np.linalg.norm((R - ref["R"]) * s) / np.linalg.norm(ref["R"] * s) <= TOL_R


def test_timeout_flag_reaches_the_host(T):
    """Failure detection without a GPU fault: the status word that a bounded device wait sets
    when it gives up is set here from the host; tsqr_status_poll then reports TSQR_ERR_TIMEOUT,
    and clearing the word restores TSQR_OK.  The factorization itself ran normally."""
    import torch

    A = torch.from_numpy(inputs.gaussian(4096, 16, inputs.seed_for(24, 0))).cuda()
    f = T.Factorization(A, leaf_h=256, chain=1)
    torch.cuda.synchronize()
    assert f.status() == T.TSQR_OK
    off = f.info().status - f.work.data_ptr()
    assert 0 <= off and off + 4 <= f.work.numel() and off % 4 == 0
    word = f.work[off:off + 4].view(torch.int32)
    word.fill_(1)
    assert f.status() == T.TSQR_ERR_TIMEOUT
    word.zero_()
    assert f.status() == T.TSQR_OK
    f.close()


@pytest.mark.parametrize("m,n,opts", [(2000, 16, {"leaf_h": 128}), (4096, 64, {"leaf_h": 64, "chain": 1, "arity": 2}),
                                      (4096, 32, {"leaf_h": 64, "chain": 1, "arity": 2}),
                                      (8192, 16, {"leaf_h": 64, "chain": 1, "arity": 2})])
def test_nan_propagates_without_fault(T, m, n, opts):
    """NaN in A propagates to R (no check, no trap); the device status word stays clear.  With
    one-leaf chains under a binary tree the NaN reaches the structured node steps, which keep
    the structural zeros exact, so only some lanes of a reflector's reductions see it: the
    reductions must still end with one value on every lane (their branches hold full-warp
    shuffles)."""
    A_h = inputs.gaussian(m, n, 99)
    A_h[1234, 5] = np.nan
    f, R, Q = run(T, A_h, **opts)
    assert np.isnan(R).any()


@pytest.mark.parametrize("m,n,opts", [(40000 + 13, 64, {}), (30000, 50, {}), (60000 + 7, 32, {}), (100000 + 3, 16, {}),
                                      (3000, 24, {"leaf_h": 128, "chain": 5, "arity": 3}), (777, 1, {"leaf_h": 16})])
def test_r_only_matches_full_factorization(T, m, n, opts, prec):
    """R alone (no reflectors, T or tree factors built or stored) is bitwise the R of the full
    factorization, and the handle refuses to apply or form a Q it does not have."""
    import torch

    A_h = inputs.gaussian(m, n, inputs.seed_for(16, m + n))
    A = torch.from_numpy(A_h).cuda()
    f_full = T.Factorization(A, precision=prec, **opts)
    f_r = T.Factorization(A, precision=prec, r_only=True, **opts)
    torch.cuda.synchronize()
    assert f_r.status() == T.TSQR_OK
    assert torch.equal(f_r.R, f_full.R)
    assert f_r.work.numel() < f_full.work.numel()
    with pytest.raises(T.TsqrError):
        f_r.form_q()
    with pytest.raises(T.TsqrError):
        f_r.apply_qt(torch.zeros((m, 1), dtype=torch.float64, device="cuda"))
    A32 = A.float()
    g_full, g_r = T.Factorization(A32, **opts), T.Factorization(A32, r_only=True, **opts)
    torch.cuda.synchronize()
    assert torch.equal(g_r.R, g_full.R)


@pytest.mark.parametrize("m,n,dtype", [(40000 + 13, 64, "float64"), (3001, 21, "float64"), (50000, 33, "float32"),
                                       (777, 1, "float64")])
def test_column_major(T, m, n, dtype):
    """TSQR_COL_MAJOR: A, R, Q and B column-major (a unit row stride, lda >= m).  The same
    factorization as the row-major copy of A, bitwise (A is transposed into the same staging
    buffer), with Q, R and Q^T B returned in column-major order."""
    import torch

    tdt = getattr(torch, dtype)
    A_h = inputs.gaussian(m, n, inputs.seed_for(17, m + n))
    A_row = torch.from_numpy(A_h).to(tdt).cuda()
    lda = m + 5
    buf = torch.zeros((n, lda), dtype=tdt, device="cuda")
    buf[:, :m] = A_row.t()
    A_col = buf[:, :m].t()  # m x n, strides (1, lda)
    f_row, f_col = T.Factorization(A_row), T.Factorization(A_col)
    Q_row, Q_col = f_row.form_q(), f_col.form_q()
    torch.cuda.synchronize()
    assert f_col.info().layout == T.TSQR_COL_MAJOR and f_col.status() == T.TSQR_OK
    assert Q_col.stride(0) == 1 and f_col.R.stride(0) == 1
    assert torch.equal(f_col.R, f_row.R) and torch.equal(Q_col, Q_row)
    assert torch.equal(A_col, A_row)  # A is read only
    B_h = inputs.gaussian(m, 3, 5)
    B_row = torch.from_numpy(B_h).to(tdt).cuda()
    B_col = torch.from_numpy(B_h.T.copy()).to(tdt).cuda().t()
    f_row.apply_qt(B_row)
    f_col.apply_qt(B_col)
    assert torch.equal(B_col, B_row)
    f_row.apply_q(B_row)
    f_col.apply_q(B_col)
    assert torch.equal(B_col, B_row)
    with pytest.raises(ValueError):
        f_col.apply_qt(torch.zeros((m, 3), dtype=tdt, device="cuda"))  # row-major B for a column-major handle
