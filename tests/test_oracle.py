"""Pins for the FP64 CPU oracle (CPU only).

The oracle is checked against facts that do not come from itself: exact rational arithmetic,
matrices built with a known QR, a library QR, closed forms and structural zeros printed in the
paper.  ``test_oracle_mutants`` plants plausible mistakes in a copy of the oracle's C source and
checks that these pins catch each of them.
"""
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

from paper_0809_2407_gb300 import inputs

EPS = np.finfo(np.float64).eps
HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- exact rational Gram-Schmidt
def rational_gs(A_int):
    """Classical Gram-Schmidt in exact rationals on an integer matrix.

    Returns d (d_j = R_jj^2) and e (e_ij = R_ii * R_ij for i < j), both exact Fractions.
    With qt_j the unnormalised orthogonal vectors: R_jj^2 = qt_j.qt_j, R_ii R_ij = qt_i.a_j.
    """
    m, n = A_int.shape
    cols = [[Fraction(int(A_int[r, c])) for r in range(m)] for c in range(n)]
    qt = []
    d = []
    e = {}
    for j in range(n):
        v = list(cols[j])
        for i in range(j):
            num = sum(qt[i][r] * cols[j][r] for r in range(m))
            e[(i, j)] = num
            coef = num / d[i]
            v = [v[r] - coef * qt[i][r] for r in range(m)]
        qt.append(v)
        d.append(sum(x * x for x in v))
    return d, e


@pytest.mark.parametrize("shape,seed", [((6, 3), 1), ((8, 4), 2), ((5, 5), 3), ((7, 1), 4), ((9, 6), 5)])
def test_rational_gram_schmidt(oracle_mod, shape, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-6, 7, size=shape).astype(np.float64)
    while np.linalg.matrix_rank(A) < shape[1]:
        A = rng.integers(-6, 7, size=shape).astype(np.float64)
    d, e = rational_gs(A)
    R = oracle_mod.qr(A, want_q=False)["R"]
    n = shape[1]
    scale = np.linalg.norm(A)
    tol = 16 * EPS * scale
    for j in range(n):
        assert abs(R[j, j] - float(d[j]) ** 0.5) <= tol
        for i in range(j):
            ref = float(e[(i, j)]) / float(d[i]) ** 0.5
            assert abs(R[i, j] - ref) <= tol
    # R^T R = A^T A, the latter exact in integers
    AtA = A.T @ A  # exact: small integers
    assert np.abs(R.T @ R - AtA).max() <= 32 * EPS * scale * scale
    assert np.all(np.tril(R, -1) == 0.0)


# ---------------------------------------------------------------- known-QR construction
def householder_product_matrix(m, n, seed):
    """A = H_0 ... H_{n-1} [R0; 0] with random unit vectors and positive-diagonal R0.

    Built by applying 2 v v^T reflections one at a time (no factorization involved); returns
    A, the thin factor Q0 = H_0 ... H_{n-1} [I; 0], and R0 (kappa(R0) <= ~1e3).
    """
    rng = np.random.default_rng(seed)
    R0 = np.triu(rng.standard_normal((n, n)) * 0.1) + np.diag(rng.uniform(1.0, 2.0, n))
    X = np.zeros((m, n))
    X[:n] = R0
    E = np.zeros((m, n))
    E[:n] = np.eye(n)
    for j in reversed(range(n)):
        v = rng.standard_normal(m)
        v /= np.linalg.norm(v)
        X -= 2.0 * np.outer(v, v @ X)
        E -= 2.0 * np.outer(v, v @ E)
    return X, E, R0


@pytest.mark.parametrize("m,n,seed", [(50, 5, 11), (300, 16, 12), (1024, 32, 13), (64, 64, 14)])
def test_householder_product_recovery(oracle_mod, m, n, seed):
    A, Q0, R0 = householder_product_matrix(m, n, seed)
    f = oracle_mod.qr(A)
    assert np.abs(f["R"] - R0).max() <= 1e-13 * np.abs(R0).max()
    assert np.abs(f["Q"] - Q0).max() <= 1e-13


# ---------------------------------------------------------------- invariants + library QR
@pytest.mark.parametrize("m,n,kind", [(4096, 64, "gaussian"), (1000, 17, "gaussian"), (64, 64, "gaussian"),
                                      (33, 1, "gaussian"), (2000, 24, "usv6"), (1500, 12, "krylov")])
def test_invariants(oracle_mod, m, n, kind):
    seed = inputs.seed_for(0, m + n)
    if kind == "gaussian":
        A = inputs.gaussian(m, n, seed)
    elif kind == "usv6":
        A = inputs.usv(m, n, 6, seed)
    else:
        A = inputs.krylov(m, n, seed)
    f = oracle_mod.qr(A)
    Q, R = f["Q"], f["R"]
    # Householder QR is backward stable and its Q orthonormal to machine precision (Sec. 5)
    assert oracle_mod.backward_error(A, Q, R) <= 10 * n * EPS
    assert oracle_mod.orthogonality(Q) <= 10 * n * EPS
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    # independent metric computation in numpy
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 10 * n * EPS
    assert np.linalg.norm(np.eye(n) - Q.T @ Q) <= 10 * n * EPS
    if kind != "krylov":  # full-rank: R is unique once diag(R) >= 0; compare with LAPACK's
        q_l, r_l = np.linalg.qr(A)
        s = np.where(np.diag(r_l) < 0, -1.0, 1.0)
        r_l = s[:, None] * r_l
        assert np.linalg.norm(R - r_l) / np.linalg.norm(r_l) <= 1e-12


# ---------------------------------------------------------------- special cases
def test_single_column(oracle_mod):
    a = inputs.gaussian(257, 1, 5)
    f = oracle_mod.qr(a)
    nrm = np.sqrt(np.sum(a * a))
    assert abs(f["R"][0, 0] - nrm) <= 4 * EPS * nrm
    assert np.abs(f["Q"] - a / nrm).max() <= 4 * EPS


def test_already_triangular_is_exact(oracle_mod):
    rng = np.random.default_rng(7)
    n = 9
    R0 = np.triu(rng.standard_normal((n, n)))
    R0[2, 2] = -abs(R0[2, 2])
    R0[5, 5] = -abs(R0[5, 5])
    A = np.vstack([R0, np.zeros((20, n))])
    f = oracle_mod.qr(A)
    D = np.where(np.diag(R0) < 0, -1.0, 1.0)
    assert np.array_equal(f["R"], D[:, None] * R0)
    Qref = np.zeros((n + 20, n))
    Qref[:n] = np.diag(D)
    assert np.array_equal(f["Q"], Qref)
    assert np.all(f["tau"] == 0.0)


def test_zero_column_gives_identity_reflector(oracle_mod):
    A = inputs.gaussian(40, 6, 8)
    A[:, 3] = 0.0
    f = oracle_mod.qr(A)
    # column 3 is zero below the diagonal after reflectors 0..2 only if it started at zero:
    # the reflectors map a zero column to a zero column, so tau_3 = 0 and R_33 = 0.
    assert f["tau"][3] == 0.0
    assert f["R"][3, 3] == 0.0
    assert np.all(f["R"][:, 3] == 0.0)


@pytest.mark.parametrize("k", [-600, 600])
def test_power_of_two_scaling_is_exact(oracle_mod, k):
    """QR commutes with scaling by 2^k: every step (max-scaled norms, beta, tau, v, the
    reflections) scales exactly when nothing over- or underflows, so R(2^k A) = 2^k R(A) and
    Q(2^k A) = Q(A) bitwise; the backward error, a ratio of norms, is unchanged.  At k = -600 the
    entries' squares underflow, so an unscaled norm or sum of squares would fail this."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((300, 12))
    f = oracle_mod.qr(A)
    g = oracle_mod.qr(A * 2.0 ** k)
    assert np.array_equal(g["R"], f["R"] * 2.0 ** k)
    assert np.array_equal(g["Q"], f["Q"])
    assert oracle_mod.backward_error(A * 2.0 ** k, g["Q"], g["R"]) == oracle_mod.backward_error(A, f["Q"], f["R"])
    assert oracle_mod.backward_error(A * 2.0 ** k, g["Q"], g["R"]) <= 10 * 12 * EPS


def test_zero_padding_is_exact(oracle_mod):
    A = inputs.gaussian(100, 8, 9)
    f1 = oracle_mod.qr(A)
    f2 = oracle_mod.qr(np.vstack([A, np.zeros((37, 8))]))
    assert np.array_equal(f1["R"], f2["R"])
    assert np.array_equal(f1["Q"], f2["Q"][:100])
    assert np.all(f2["Q"][100:] == 0.0)


def test_block_diagonal(oracle_mod):
    A1 = inputs.gaussian(30, 4, 10)
    A2 = inputs.gaussian(25, 3, 11)
    A = np.zeros((55, 7))
    A[:30, :4] = A1
    A[30:, 4:] = A2
    R = oracle_mod.qr(A)["R"]
    assert np.all(R[4:, :4] == 0.0) and np.all(R[:4, 4:] == 0.0)
    assert np.abs(R[:4, :4] - oracle_mod.qr(A1)["R"]).max() <= 1e-14 * 8
    assert np.abs(R[4:, 4:] - oracle_mod.qr(A2)["R"]).max() <= 1e-14 * 8


def test_apply_round_trip_and_formq(oracle_mod):
    A = inputs.gaussian(120, 10, 12)
    f = oracle_mod.qr(A, want_q=False)
    B = inputs.gaussian(120, 5, 13)
    QtB = oracle_mod.apply_qt(f["V"], f["tau"], B)
    assert np.abs(oracle_mod.apply_q(f["V"], f["tau"], QtB) - B).max() <= 1e-14
    assert abs(np.linalg.norm(QtB) - np.linalg.norm(B)) <= 1e-13 * np.linalg.norm(B)
    # Q^T A = [R_raw; 0]
    QtA = oracle_mod.apply_qt(f["V"], f["tau"], A)
    assert np.abs(QtA[:10] - np.triu(f["V"][:10])).max() <= 1e-13
    assert np.abs(QtA[10:]).max() <= 1e-13
    # thin Q from org2r equals Q [I; 0]
    E = np.zeros((120, 10))
    E[:10] = np.eye(10)
    assert np.array_equal(oracle_mod.org2r(f["V"], f["tau"]), oracle_mod.apply_q(f["V"], f["tau"], E))
    # sign-normalised thin part: D (Q^T B)_top equals Q_norm^T B with Q_norm the explicit factor
    fq = oracle_mod.qr(A)
    assert np.abs(oracle_mod.thin_qt(A, B) - fq["Q"].T @ B).max() <= 1e-13


def _load_pattern():
    rows = []
    with open(os.path.join(HERE, "golden", "fact_2rs_pattern.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    return rows


def test_structured_pair_pattern(oracle_mod):
    """Eq. fact_2rs: the reflectors of [R0; R1] have identity on top and a triangle below."""
    pat = _load_pattern()
    assert len(pat) == 10 and all(len(r) == 5 for r in pat)
    rng = np.random.default_rng(21)
    R0 = np.triu(rng.standard_normal((5, 5)))
    R1 = np.triu(rng.standard_normal((5, 5)))
    VR, tau = oracle_mod.geqr2(np.vstack([R0, R1]))
    assert np.all(tau != 0.0)
    for r in range(10):
        for c in range(5):
            sym = pat[r][c]
            if r < 5:  # top block of the vectors is stored implicitly: strict lower must be zero
                if r > c:
                    assert sym == "." and VR[r, c] == 0.0
                if r == c:
                    assert sym == "1"
            else:
                if sym == ".":
                    assert VR[r, c] == 0.0
                else:
                    assert sym == "x" and VR[r, c] != 0.0


def test_metrics_closed_forms(oracle_mod):
    n = 7
    Q = np.zeros((30, n))
    Q[:n] = np.eye(n)
    assert oracle_mod.orthogonality(Q) == 0.0
    delta = 1e-6
    # ||I - (1+d)^2 I||_F = sqrt(n) * |2d + d^2|
    got = oracle_mod.orthogonality((1 + delta) * Q)
    assert abs(got - np.sqrt(n) * (2 * delta + delta ** 2)) <= 1e-15
    A = inputs.gaussian(30, n, 3)
    f = oracle_mod.qr(A)
    assert oracle_mod.backward_error(A, f["Q"], f["R"]) < 1e-15
    # a rank-one perturbation of known norm: ||E||_F / ||A||_F
    E = np.outer(np.ones(30), np.arange(n, dtype=float)) * 1e-9
    got = oracle_mod.backward_error(A + E, f["Q"], f["R"])
    assert abs(got - np.linalg.norm(E) / np.linalg.norm(A + E)) <= 1e-6 * got


def test_flop_formulas_consistent():
    """Sec. 3.1: dense QR of a 2n x n pair costs about 10n^3/3 = Householder count at m=2n."""
    f = {}
    with open(os.path.join(HERE, "golden", "flop_counts.txt")) as fh:
        for line in fh:
            if line.startswith("#") or "=" not in line:
                continue
            k, v = line.split("=", 1)
            f[k.strip()] = v.strip()
    for n in (4, 16, 50, 64):
        m = 2 * n
        hh = eval(f["householder_qr"], {}, {"m": m, "n": n})
        dense = eval(f["node_pair_dense"], {}, {"m": m, "n": n})
        assert abs(hh - dense) <= 1e-9 * dense
        assert abs(eval(f["node_pair_structured"], {}, {"n": n}) * 5 - dense) <= 1e-9 * dense


# ---------------------------------------------------------------- planted mistakes
MUTANTS = {
    # the trailing update forgets tau
    "drop_tau": ("A[j * lda + c] -= tau[j] * w;", "A[j * lda + c] -= w;"),
    # tau computed with the wrong denominator
    "tau_denominator": ("*tau = (beta - alpha) / beta;", "*tau = (beta - alpha) / alpha;"),
    # thin Q accumulated in the wrong order
    "formq_order": ("for (int64_t j = n - 1; j >= 0; --j) apply_reflector(m, j, V, ldv, j, tau[j], n, Q, ldq);",
                    "for (int64_t j = 0; j < n; ++j) apply_reflector(m, j, V, ldv, j, tau[j], n, Q, ldq);"),
    # the dot product uses the transposed index
    "transposed_index": ("w += A[i * lda + j] * A[i * lda + c];", "w += A[j * lda + i] * A[i * lda + c];"),
    # the sign normalisation of diag(R) left out
    "drop_sign_normalisation": ("D[j] = (V[j * ldv + j] < 0.0) ? -1.0 : 1.0;", "D[j] = 1.0;"),
}


def _build_mutant(src_text, name, tmpdir):
    path = os.path.join(tmpdir, name + ".c")
    with open(path, "w") as fh:
        fh.write(src_text)
    so = os.path.join(tmpdir, name + ".so")
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, path, "-lm"])
    return so


def _pins_pass(lib_path):
    """Runs a subset of the pins against the library at lib_path; True if all hold."""
    import ctypes
    import oracle as O

    saved = O._load()  # the serial build, whose argument types the mutant library takes
    try:
        lib = ctypes.CDLL(lib_path)
        for nm in ("oracle_geqr2", "oracle_org2r", "oracle_apply_qt", "oracle_apply_q", "oracle_signs",
                   "oracle_qr", "oracle_backward_error", "oracle_orthogonality"):
            getattr(lib, nm).argtypes = getattr(saved, nm).argtypes
            getattr(lib, nm).restype = getattr(saved, nm).restype
        O._libs["serial"] = lib
        try:
            A, Q0, R0 = householder_product_matrix(60, 6, 5)
            f = O.qr(A)
            if np.abs(f["R"] - R0).max() > 1e-13 or np.abs(f["Q"] - Q0).max() > 1e-13:
                return False
            A = np.random.default_rng(4).integers(-6, 7, size=(8, 4)).astype(float)
            d, e = rational_gs(A)
            R = O.qr(A, want_q=False)["R"]
            for j in range(4):
                if abs(R[j, j] - float(d[j]) ** 0.5) > 1e-12:
                    return False
            G = inputs.gaussian(200, 9, 6)
            g = O.qr(G)
            if O.orthogonality(g["Q"]) > 1e-13 or O.backward_error(G, g["Q"], g["R"]) > 1e-13:
                return False
            return True
        except Exception:
            return False
    finally:
        O._libs["serial"] = saved


def test_oracle_mutants(oracle_mod):
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "tsqr_oracle.c")).read()
    with tempfile.TemporaryDirectory() as td:
        assert _pins_pass(_build_mutant(src, "clean", td)), "pins must pass on the unmodified oracle"
        for name, (old, new) in MUTANTS.items():
            assert src.count(old) == 1, name
            so = _build_mutant(src.replace(old, new), name, td)
            assert not _pins_pass(so), "pins missed planted mistake %s" % name


def test_householder_stability_contrast_with_cholesky_qr(oracle_mod):
    """Householder QR is unconditionally stable: its Q stays orthonormal to O(u) whatever
    kappa(A) (Sec. 5), while CholeskyQR (R from the Cholesky factor of A^T A, Q = A R^-1; the
    paper's comparison) loses orthogonality like kappa^2 u.  At kappa = 1e6 the two differ by
    many orders of magnitude."""
    from paper_0809_2407_gb300 import inputs

    A = inputs.usv(4000, 20, 6.0, inputs.seed_for(30, 1))
    ref = oracle_mod.qr(A)
    assert oracle_mod.orthogonality(ref["Q"]) <= 1e-13
    Rc = np.linalg.cholesky(A.T @ A).T
    Qc = np.linalg.solve(Rc.T, A.T).T
    assert oracle_mod.orthogonality(Qc) >= 1e-6


def test_paper_p4_binary_and_flat_trees(oracle_mod):
    """The paper's P = 4 examples (Sec. 2): A in four row blocks, each factored locally; the
    binary tree combines R_0 with R_1 and R_2 with R_3, then the two results (eq. par4:final), and
    the flat tree folds the blocks one by one into a running R (eq. seq4:final).  Both reach the
    QR of the whole matrix: the same R after sign normalisation, and Q from the tree factors
    reproduces A."""
    from paper_0809_2407_gb300 import inputs

    m, n, P = 400, 6, 4
    A = inputs.gaussian(m, n, inputs.seed_for(31, 0))
    blocks = np.split(A, P)
    whole = oracle_mod.qr(A)

    def R_of(X):
        return oracle_mod.qr(X, want_q=False)["R"]

    # binary: level 1 pairs (0,1) and (2,3), level 2 the root
    R01 = R_of(np.vstack([R_of(blocks[0]), R_of(blocks[1])]))
    R23 = R_of(np.vstack([R_of(blocks[2]), R_of(blocks[3])]))
    R_bin = R_of(np.vstack([R01, R23]))
    # flat: R <- QR([R; A_k]) for k = 1, 2, 3
    R_flat = R_of(blocks[0])
    for k in range(1, P):
        R_flat = R_of(np.vstack([R_flat, blocks[k]]))
    tol = 1e-12 * np.abs(whole["R"]).max()
    assert np.abs(R_bin - whole["R"]).max() <= tol
    assert np.abs(R_flat - whole["R"]).max() <= tol
    # Q of the binary tree: block-diagonal leaf factors times the node factors, applied to [I; 0]
    leaf = [oracle_mod.qr(b) for b in blocks]
    n1 = [oracle_mod.qr(np.vstack([leaf[0]["R"], leaf[1]["R"]])), oracle_mod.qr(np.vstack([leaf[2]["R"], leaf[3]["R"]]))]
    root = oracle_mod.qr(np.vstack([n1[0]["R"], n1[1]["R"]]))
    Qroot = root["Q"]                                    # 2n x n
    Q1 = [n1[i]["Q"] @ Qroot[i * n:(i + 1) * n] for i in range(2)]           # 2n x n each
    Q = np.vstack([leaf[2 * i + j]["Q"] @ Q1[i][j * n:(j + 1) * n] for i in range(2) for j in range(2)])
    assert np.abs(Q @ root["R"] - A).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(Q - whole["Q"]).max() <= 1e-12


def test_openmp_timing_build_is_bitwise_serial(oracle_mod):
    """The oracle's -fopenmp build, used only to time it on all host cores, runs each column's
    sums in the serial order, so its R, Q and reflectors are the serial build's bit for bit."""
    oracle = oracle_mod
    A = inputs.gaussian(3000, 24, 77)
    ref = oracle.qr(A)
    oracle.set_variant("openmp")
    try:
        par = oracle.qr(A)
    finally:
        oracle.set_variant("serial")
    for k in ("R", "Q", "V", "tau", "D"):
        assert np.array_equal(ref[k], par[k]), k
