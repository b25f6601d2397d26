"""Seeded synthetic inputs shaped like the paper's tall-skinny workloads.

The paper never says how its test matrices were drawn.  These generators produce the shapes
and structures it discusses: tall-skinny blocks with n around 4..128 and m up to millions of
rows (Sec. 7.1, Sec. 7.2), and s-step Krylov bases (Sec. 1).  They draw random numbers
and build matrices; they hold none of TSQR's arithmetic, and both the CUDA path's tests and
the oracle's take their inputs from here.

Every generator is a pure function of its arguments and a seed, drawn with numpy's PCG64
(``numpy.random.default_rng``), in FP64 on the host.  Seeds follow
``SEED_BASE + 1000 * workload + index``.
"""
import numpy as np

SEED_BASE = 20080809


def seed_for(workload: int, index: int = 0) -> int:
    """Seed of input ``index`` of workload number ``workload``."""
    return SEED_BASE + 1000 * int(workload) + int(index)


def gaussian(m: int, n: int, seed: int) -> np.ndarray:
    """m x n matrix of iid N(0, 1) entries."""
    return np.random.default_rng(seed).standard_normal((m, n))


def _haar_columns(m: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """m x n matrix with orthonormal columns, Haar distributed.

    Polar factor of a Gaussian matrix G: U = G (G^T G)^(-1/2).  G and O G have the same
    distribution for any orthogonal O and the polar factor commutes with that action, so U is
    Haar distributed on the Stiefel manifold.  A tall Gaussian is well conditioned, so the
    inverse square root through a symmetric eigendecomposition loses nothing.
    """
    G = rng.standard_normal((m, n))
    w, E = np.linalg.eigh(G.T @ G)
    return G @ ((E * (1.0 / np.sqrt(w))) @ E.T)


def usv(m: int, n: int, log10_kappa: float, seed: int) -> np.ndarray:
    """A = U diag(s) V^T with Haar U (m x n), Haar V (n x n) and s_j = 10^(-k j / (n-1)).

    The singular values are log-spaced from 1 down to 10^-k, so kappa_2(A) = 10^k.
    """
    rng = np.random.default_rng(seed)
    U = _haar_columns(m, n, rng)
    V = _haar_columns(n, n, rng)
    if n == 1:
        s = np.ones(1)
    else:
        s = 10.0 ** (-float(log10_kappa) * np.arange(n) / (n - 1))
    return (U * s) @ V.T


def usv_family(m: int, n: int, log10_kappas, seed: int):
    """usv(m, n, k, seed) for every k in log10_kappas, drawing U and V once: the same rng draws
    in the same order, so each matrix equals usv's bit for bit.  Yields the matrices one by one."""
    rng = np.random.default_rng(seed)
    U = _haar_columns(m, n, rng)
    V = _haar_columns(n, n, rng)
    for k in log10_kappas:
        s = np.ones(1) if n == 1 else 10.0 ** (-float(k) * np.arange(n) / (n - 1))
        yield (U * s) @ V.T


def sparse_symmetric(m: int, seed: int, partners: int = 4):
    """Random sparse symmetric m x m matrix, about 2 * partners nonzeros per row.

    Each row i draws ``partners`` distinct columns j != i uniformly; S_ij = S_ji ~ N(0, 1).
    Returned as a scipy CSR matrix (duplicates summed).
    """
    import scipy.sparse as sp

    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(m), partners)
    cols = np.empty(m * partners, dtype=np.int64)
    for i0 in range(0, m, 1 << 16):
        i1 = min(m, i0 + (1 << 16))
        cnt = i1 - i0
        # distinct offsets in 1..m-1 per row: draw without replacement from a small pool
        offs = np.stack([rng.permutation(m - 1)[:partners] + 1 for _ in range(cnt)]) if m <= 64 \
            else _distinct_offsets(rng, cnt, partners, m - 1)
        cols[i0 * partners:i1 * partners] = ((np.arange(i0, i1)[:, None] + offs) % m).ravel()
    vals = rng.standard_normal(m * partners)
    S = sp.coo_matrix((np.concatenate([vals, vals]),
                       (np.concatenate([rows, cols]), np.concatenate([cols, rows]))),
                      shape=(m, m)).tocsr()
    S.sum_duplicates()
    return S


def _distinct_offsets(rng, cnt, k, hi):
    """cnt rows of k distinct integers in 1..hi (rejection on duplicates, hi >> k)."""
    out = rng.integers(1, hi + 1, size=(cnt, k))
    while True:
        srt = np.sort(out, axis=1)
        dup = np.any(srt[:, 1:] == srt[:, :-1], axis=1)
        if not dup.any():
            return out
        out[dup] = rng.integers(1, hi + 1, size=(int(dup.sum()), k))


def krylov(m: int, n: int, seed: int, power_steps: int = 100) -> np.ndarray:
    """s-step monomial Krylov basis [x, Sx, ..., S^(n-1) x] with unit-norm columns.

    S is ``sparse_symmetric(m)`` scaled to spectral radius ~1 by ``power_steps`` power
    iterations; x ~ N(0, I).  Column j is S v_{j-1} / ||S v_{j-1}||, which spans the same
    direction as S^j x.  At n beyond ~20 the basis is numerically rank deficient.
    """
    rng = np.random.default_rng(seed)
    S = sparse_symmetric(m, seed + 1)
    z = rng.standard_normal(m)
    lam = 1.0
    for _ in range(power_steps):
        y = S @ z
        lam = np.linalg.norm(y)
        z = y / lam
    S = S * (1.0 / lam)
    x = rng.standard_normal(m)
    A = np.empty((m, n))
    A[:, 0] = x / np.linalg.norm(x)
    for j in range(1, n):
        y = S @ A[:, j - 1]
        A[:, j] = y / np.linalg.norm(y)
    return A


def make(kind: str, m: int, n: int, seed: int, **kw) -> np.ndarray:
    """Dispatch by name: 'gaussian', 'usv' (kw: log10_kappa), 'krylov'."""
    if kind == "gaussian":
        return gaussian(m, n, seed)
    if kind == "usv":
        return usv(m, n, kw.get("log10_kappa", 0.0), seed)
    if kind == "krylov":
        return krylov(m, n, seed)
    raise ValueError("unknown input kind %r" % kind)
