"""Python binding of libtsqr.so (include/tsqr.h): the same calls, marshalled through ctypes.

Every step of TSQR runs in the library's CUDA kernels; this module only passes pointers,
sizes and the current CUDA stream, and turns status codes into exceptions.  PyTorch provides
device memory and streams.  If the library is missing the import fails loudly: there is no
CPU or PyTorch fallback.

Low level (same names as the C-ABI): ``tsqr_workspace_size``, ``tsqr_factor``,
``tsqr_apply_qt``, ``tsqr_apply_q``, ``tsqr_form_q``, ``tsqr_status_poll``,
``tsqr_handle_info``, ``tsqr_destroy``, the batch calls ``tsqr_batch_*`` and
``tsqr_backward``.  Convenience on torch tensors: ``Factorization`` (one matrix), ``Batch``
(many matrices in one launch, capturable in a CUDA graph), ``qr_autograd`` (differentiable QR)
and ``autotune`` (plan search, cached per shape bucket).

Example::

    import torch
    from paper_0809_2407_gb300 import tsqr
    A = torch.randn(1 << 20, 64, dtype=torch.float64, device="cuda")
    f = tsqr.Factorization(A)           # R in f.R, the implicit Q in the workspace
    Q = f.form_q()                      # explicit thin Q
    B = torch.randn(1 << 20, 64, dtype=torch.float64, device="cuda")
    f.apply_qt(B)                       # B <- Q^T B in place (rows 0..63: Q_thin^T B)
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtsqr.so")

TSQR_OK, TSQR_ERR_INVALID_ARG, TSQR_ERR_UNSUPPORTED, TSQR_ERR_CUDA, TSQR_ERR_WORKSPACE, TSQR_ERR_TIMEOUT = range(6)
TSQR_F64, TSQR_F32 = 0, 1
TSQR_ROW_MAJOR, TSQR_COL_MAJOR = 0, 1

EXPORTED = ("tsqr_workspace_size", "tsqr_factor", "tsqr_apply_qt", "tsqr_apply_q", "tsqr_form_q",
            "tsqr_status_poll", "tsqr_handle_info", "tsqr_destroy", "tsqr_status_string", "tsqr_last_error",
            "tsqr_factor_r_noalloc", "tsqr_noalloc_status_poll", "tsqr_batch_workspace_size", "tsqr_batch_create",
            "tsqr_batch_workspace_size_plans", "tsqr_batch_create_plans",
            "tsqr_batch_factor", "tsqr_batch_form_q", "tsqr_batch_status_poll", "tsqr_batch_destroy", "tsqr_backward")


class Opts(ctypes.Structure):
    _fields_ = [("leaf_h", ctypes.c_int32), ("chain", ctypes.c_int32), ("arity", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("inplace", ctypes.c_int32), ("r_only", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("np", ctypes.c_int64),
                ("leaf_h", ctypes.c_int32), ("chain", ctypes.c_int32), ("arity", ctypes.c_int32),
                ("depth", ctypes.c_int32),
                ("leaves", ctypes.c_int64), ("chains", ctypes.c_int64), ("tree_nodes", ctypes.c_int64),
                ("v", ctypes.c_void_p), ("ldv", ctypes.c_int64),
                ("tau_leaf", ctypes.c_void_p), ("t_leaf", ctypes.c_void_p), ("node_y", ctypes.c_void_p),
                ("node_tau", ctypes.c_void_p), ("node_t", ctypes.c_void_p), ("signs", ctypes.c_void_p),
                ("panels", ctypes.c_int32), ("dtype", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("status", ctypes.c_void_p)]


class TsqrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_status_name(status), msg))
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Loads libtsqr.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libtsqr.so not found at %s: run __graft_entry__.build() first" % path)
    lib = ctypes.CDLL(path)
    i64, vp, sz = ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
    lib.tsqr_workspace_size.argtypes = [ctypes.c_int, i64, i64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    lib.tsqr_factor.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, vp, i64, vp, i64, vp, sz,
                                ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.tsqr_apply_qt.argtypes = [vp, i64, vp, i64, vp]
    lib.tsqr_apply_q.argtypes = [vp, i64, vp, i64, vp]
    lib.tsqr_form_q.argtypes = [vp, vp, i64, vp]
    lib.tsqr_status_poll.argtypes = [vp, vp]
    lib.tsqr_handle_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.tsqr_destroy.argtypes = [vp]
    lib.tsqr_factor_r_noalloc.argtypes = [i64, i64, vp, i64, vp, i64, vp]
    lib.tsqr_noalloc_status_poll.argtypes = [vp, ctypes.POINTER(vp)]
    i32, pi64, pvp = ctypes.c_int32, ctypes.POINTER(i64), ctypes.POINTER(vp)
    lib.tsqr_batch_workspace_size.argtypes = [ctypes.c_int, i32, pi64, pi64, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
    lib.tsqr_batch_workspace_size_plans.argtypes = [ctypes.c_int, i32, pi64, pi64, ctypes.POINTER(Opts),
                                                    ctypes.POINTER(sz)]
    lib.tsqr_batch_create.argtypes = [ctypes.c_int, i32, pi64, pi64, pvp, pi64, pvp, pi64, pvp, pi64, vp, sz,
                                      ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.tsqr_batch_create_plans.argtypes = [ctypes.c_int, i32, pi64, pi64, pvp, pi64, pvp, pi64, pvp, pi64, vp, sz,
                                            ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.tsqr_batch_factor.argtypes = [vp, vp]
    lib.tsqr_batch_form_q.argtypes = [vp, vp]
    lib.tsqr_batch_status_poll.argtypes = [vp, vp]
    lib.tsqr_batch_destroy.argtypes = [vp]
    lib.tsqr_backward.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, i64, vp]
    lib.tsqr_status_string.argtypes = [ctypes.c_int]
    lib.tsqr_status_string.restype = ctypes.c_char_p
    lib.tsqr_last_error.argtypes = []
    lib.tsqr_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        f = getattr(lib, name)
        if name not in ("tsqr_status_string", "tsqr_last_error"):
            f.restype = ctypes.c_int
    _lib = lib
    return lib


def _status_name(s):
    try:
        return load().tsqr_status_string(s).decode()
    except OSError:
        return "status %d" % s


def _check(status):
    if status != TSQR_OK:
        raise TsqrError(status, load().tsqr_last_error().decode())


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, Opts):
        return ctypes.byref(opts)
    return ctypes.byref(Opts(**opts))


# ---------------------------------------------------------------- C-ABI, one to one
def tsqr_workspace_size(dtype, m, n, opts=None):
    out = ctypes.c_size_t(0)
    _check(load().tsqr_workspace_size(dtype, m, n, _opts(opts), ctypes.byref(out)))
    return out.value


def tsqr_factor(dtype, layout, m, n, dA, lda, dR, ldr, dWork, work_bytes, opts, stream):
    h = ctypes.c_void_p()
    _check(load().tsqr_factor(dtype, layout, m, n, dA, lda, dR, ldr, dWork, work_bytes, _opts(opts), stream,
                              ctypes.byref(h)))
    return h


def tsqr_apply_qt(h, k, dB, ldb, stream):
    _check(load().tsqr_apply_qt(h, k, dB, ldb, stream))


def tsqr_apply_q(h, k, dB, ldb, stream):
    _check(load().tsqr_apply_q(h, k, dB, ldb, stream))


def tsqr_form_q(h, dQ, ldq, stream):
    _check(load().tsqr_form_q(h, dQ, ldq, stream))


def tsqr_status_poll(h, stream):
    return load().tsqr_status_poll(h, stream)


def tsqr_handle_info(h):
    info = Info()
    _check(load().tsqr_handle_info(h, ctypes.byref(info)))
    return info


def tsqr_destroy(h):
    load().tsqr_destroy(h)


def tsqr_factor_r_noalloc(m, n, dA, lda, dR, ldr, stream):
    """R only, using the library's static device scratch: for callers that cannot allocate."""
    _check(load().tsqr_factor_r_noalloc(m, n, dA, lda, dR, ldr, stream))


def tsqr_noalloc_status_poll(stream):
    """Status of the latest tsqr_factor_r_noalloc on the current device (waits for `stream`):
    returns (status code, device address of the static scratch's status word)."""
    word = ctypes.c_void_p()
    st = load().tsqr_noalloc_status_poll(stream, ctypes.byref(word))
    return st, word.value


def tsqr_backward(h, dQbar, ldqb, dRbar, ldrb, dR, ldr, dAbar, ldab, stream):
    _check(load().tsqr_backward(h, dQbar, ldqb, dRbar, ldrb, dR, ldr, dAbar, ldab, stream))


def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


def tsqr_batch_workspace_size(dtype, count, m, n, opts=None):
    out = ctypes.c_size_t(0)
    _check(load().tsqr_batch_workspace_size(dtype, count, _arr(ctypes.c_int64, m), _arr(ctypes.c_int64, n),
                                            _opts(opts), ctypes.byref(out)))
    return out.value


def tsqr_batch_create(dtype, count, m, n, dA, lda, dR, ldr, dQ, ldq, dWork, work_bytes, opts, stream):
    h = ctypes.c_void_p()
    vp = ctypes.c_void_p
    _check(load().tsqr_batch_create(dtype, count, _arr(ctypes.c_int64, m), _arr(ctypes.c_int64, n), _arr(vp, dA),
                                    _arr(ctypes.c_int64, lda), _arr(vp, dR), _arr(ctypes.c_int64, ldr),
                                    _arr(vp, dQ) if dQ is not None else None,
                                    _arr(ctypes.c_int64, ldq) if ldq is not None else None,
                                    dWork, work_bytes, _opts(opts), stream, ctypes.byref(h)))
    return h


def _opts_array(plans):
    arr = (Opts * len(plans))()
    for i, o in enumerate(plans):
        arr[i] = o
    return arr


def tsqr_batch_workspace_size_plans(dtype, count, m, n, plans):
    out = ctypes.c_size_t(0)
    _check(load().tsqr_batch_workspace_size_plans(dtype, count, _arr(ctypes.c_int64, m), _arr(ctypes.c_int64, n),
                                                  _opts_array(plans), ctypes.byref(out)))
    return out.value


def tsqr_batch_create_plans(dtype, count, m, n, dA, lda, dR, ldr, dQ, ldq, dWork, work_bytes, plans, stream):
    h = ctypes.c_void_p()
    vp = ctypes.c_void_p
    _check(load().tsqr_batch_create_plans(dtype, count, _arr(ctypes.c_int64, m), _arr(ctypes.c_int64, n),
                                          _arr(vp, dA), _arr(ctypes.c_int64, lda), _arr(vp, dR),
                                          _arr(ctypes.c_int64, ldr), _arr(vp, dQ) if dQ is not None else None,
                                          _arr(ctypes.c_int64, ldq) if ldq is not None else None,
                                          dWork, work_bytes, _opts_array(plans), stream, ctypes.byref(h)))
    return h


def tsqr_batch_factor(b, stream):
    _check(load().tsqr_batch_factor(b, stream))


def tsqr_batch_form_q(b, stream):
    _check(load().tsqr_batch_form_q(b, stream))


def tsqr_batch_status_poll(b, stream):
    return load().tsqr_batch_status_poll(b, stream)


def tsqr_batch_destroy(b):
    load().tsqr_batch_destroy(b)


# ---------------------------------------------------------------- torch convenience layer
def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check_matrix(X, name, dtype=None, layout=None):
    """Checks a CUDA matrix argument; returns (layout, leading dimension).  A unit column stride
    means row-major, else a unit row stride means column-major; layout, if given, must match."""
    import torch

    ok = (torch.float64, torch.float32) if dtype is None else (dtype,)
    if not (X.is_cuda and X.dtype in ok and X.dim() == 2 and (X.stride(1) == 1 or X.stride(0) == 1)):
        raise ValueError("%s must be a CUDA %s matrix with unit column or row stride"
                         % (name, " or ".join(str(t).replace("torch.", "") for t in ok)))
    got = TSQR_ROW_MAJOR if X.stride(1) == 1 and (layout != TSQR_COL_MAJOR or X.stride(0) != 1) else TSQR_COL_MAJOR
    if layout is not None and got != layout:
        raise ValueError("%s must be %s like A" % (name, "row-major" if layout == TSQR_ROW_MAJOR else "column-major"))
    return got, (X.stride(0) if got == TSQR_ROW_MAJOR else max(X.stride(1), X.shape[0]))


def _empty_like_layout(rows, cols, dtype, device, layout):
    import torch

    if layout == TSQR_COL_MAJOR:
        return torch.empty((cols, rows), dtype=dtype, device=device).t()
    return torch.empty((rows, cols), dtype=dtype, device=device)


class Factorization:
    """TSQR of a CUDA float64 or float32 matrix A (m x n, row-major, or column-major: a unit row
    stride, e.g. the transpose of a contiguous n x m tensor).  Holds R, the workspace and the
    handle.  A float32 A selects TSQR_F32 (FP32 storage and arithmetic); R, Q and the matrices
    given to apply_qt / apply_q then have A's dtype and layout.

    ``inplace=True`` lets the reflectors overwrite A (A must then stay alive; float64 only);
    ``r_only=True`` computes R alone and keeps no Q.  Options: leaf_h, chain, arity, precision
    (0 native FP64, 1 double-float, 2 Ozaki WY products, 3 double-float + Ozaki WY; see
    tsqr_opts_t).
    """

    def __init__(self, A, leaf_h=0, chain=0, arity=0, inplace=False, precision=0, r_only=False):
        import torch

        self.layout, lda = _check_matrix(A, "A")
        m, n = A.shape
        self.m, self.n = m, n
        self.dtype = A.dtype
        self.code = TSQR_F32 if A.dtype == torch.float32 else TSQR_F64
        self.opts = Opts(leaf_h=leaf_h, chain=chain, arity=arity, precision=precision, inplace=1 if inplace else 0,
                         r_only=1 if r_only else 0)
        nbytes = tsqr_workspace_size(self.code, m, n, self.opts)
        self.work = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=A.device)
        self.R = _empty_like_layout(n, n, A.dtype, A.device, self.layout)
        self.A = A
        self.handle = tsqr_factor(self.code, self.layout, m, n, A.data_ptr(), lda, self.R.data_ptr(), n,
                                  self.work.data_ptr(), nbytes, self.opts, _stream())

    def form_q(self, out=None):
        Q = out if out is not None else _empty_like_layout(self.m, self.n, self.dtype, self.R.device, self.layout)
        _, ldq = _check_matrix(Q, "Q", self.dtype, self.layout)
        tsqr_form_q(self.handle, Q.data_ptr(), ldq, _stream())
        return Q

    def apply_qt(self, B):
        """B <- Q^T B in place (B: m x k CUDA matrix of A's dtype and layout)."""
        _, ldb = _check_matrix(B, "B", self.dtype, self.layout)
        tsqr_apply_qt(self.handle, B.shape[1], B.data_ptr(), ldb, _stream())
        return B

    def apply_q(self, B):
        """B <- Q B in place."""
        _, ldb = _check_matrix(B, "B", self.dtype, self.layout)
        tsqr_apply_q(self.handle, B.shape[1], B.data_ptr(), ldb, _stream())
        return B

    def info(self):
        return tsqr_handle_info(self.handle)

    def status(self):
        return tsqr_status_poll(self.handle, _stream())

    def close(self):
        if self.handle:
            tsqr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qr(A, **opts):
    """Thin QR of a CUDA float64 or float32 matrix by TSQR: returns (Q, R), diag(R) >= 0."""
    f = Factorization(A, **opts)
    Q = f.form_q()
    R = f.R
    f.close()
    return Q, R


class Batch:
    """Many CUDA float64 (or, all of them, float32) tall-skinny matrices factored together (one
    launch for all R factors, one launch per tree depth plus one for all thin Q factors).  The
    launches only enqueue work on the current stream, so ``factor()`` and ``form_q()`` can be
    captured in a CUDA graph.
    """

    def __init__(self, mats, want_q=True, leaf_h=0, chain=0, arity=0, precision=0, plans=None):
        """plans: an Opts per matrix (its leaf height, arity and chain length; chain 0 takes the
        batch's shared chain length), e.g. from autotune_batch; otherwise one plan for all."""
        import torch

        dt = mats[0].dtype
        for i, A in enumerate(mats):
            _check_matrix(A, "A[%d]" % i, dt, TSQR_ROW_MAJOR)
        self.mats = list(mats)
        dev = self.mats[0].device
        self.code = TSQR_F32 if dt == torch.float32 else TSQR_F64
        self.m = [A.shape[0] for A in self.mats]
        self.n = [A.shape[1] for A in self.mats]
        count = len(self.mats)
        self.opts = Opts(leaf_h=leaf_h, chain=chain, arity=arity, precision=precision, inplace=0)
        self.plans = list(plans) if plans is not None else None
        if self.plans is not None:
            assert len(self.plans) == count
            nbytes = tsqr_batch_workspace_size_plans(self.code, count, self.m, self.n, self.plans)
        else:
            nbytes = tsqr_batch_workspace_size(self.code, count, self.m, self.n, self.opts)
        self.work = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        self.R = [torch.empty((k, k), dtype=dt, device=dev) for k in self.n]
        self.Q = [torch.empty((mm, k), dtype=dt, device=dev) for mm, k in zip(self.m, self.n)] \
            if want_q else None
        args = (self.code, count, self.m, self.n, [A.data_ptr() for A in self.mats], [A.stride(0) for A in self.mats],
                [R.data_ptr() for R in self.R], [R.stride(0) for R in self.R],
                [Q.data_ptr() for Q in self.Q] if want_q else None, [Q.stride(0) for Q in self.Q] if want_q else None,
                self.work.data_ptr(), nbytes)
        if self.plans is not None:
            self.handle = tsqr_batch_create_plans(*args, self.plans, _stream())
        else:
            self.handle = tsqr_batch_create(*args, self.opts, _stream())

    def factor(self):
        tsqr_batch_factor(self.handle, _stream())

    def form_q(self):
        tsqr_batch_form_q(self.handle, _stream())

    def status(self):
        return tsqr_batch_status_poll(self.handle, _stream())

    def close(self):
        if self.handle:
            tsqr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- autotuner
_TUNE_CACHE = {}


def tune_key(m, n, precision, dtype=TSQR_F64):
    """Cache key: (log2 bucket of m, n rounded up to the padded width, precision, dtype code)."""
    mb = max(0, int(m).bit_length() - 1)
    np_ = 16
    while np_ < n:
        np_ *= 2
    return (mb, np_, int(precision), int(dtype))


def candidate_opts(m, n, precision=0, dtype=TSQR_F64):
    """Plans the library accepts for an m x n problem: leaf height 64..1024, arity 2/4/8, flat
    chains (auto) or a pure tree (chain 1)."""
    out = []
    for h in (64, 96, 128, 192, 256, 512, 1024):
        for arity in (2, 4, 8):
            for chain in (0, 1):
                o = Opts(leaf_h=h, chain=chain, arity=arity, precision=precision, inplace=0)
                try:
                    tsqr_workspace_size(dtype, m, n, o)
                except TsqrError:
                    continue
                out.append(o)
    return out


def autotune(m, n, precision=0, reps=2, proxy_rows=1 << 18, path=None, dtype=None):
    """Times factor + thin Q for each candidate plan on a seeded N(0,1) matrix of min(m, proxy_rows)
    rows and returns the fastest Opts, caching it by tune_key (and in the JSON file `path` if given).
    dtype: torch.float64 (default) or torch.float32 (FP32 storage, precision 0).
    """
    import json

    import torch

    dtype = torch.float64 if dtype is None else dtype
    code = TSQR_F32 if dtype == torch.float32 else TSQR_F64
    key = tune_key(m, n, precision, code)
    if path and not _TUNE_CACHE and os.path.exists(path):
        with open(path) as fh:
            for k, v in json.load(fh).items():
                _TUNE_CACHE[tuple(int(x) for x in k.split(","))] = v
    if key in _TUNE_CACHE:
        return Opts(**_TUNE_CACHE[key])
    rows = int(min(m, proxy_rows))
    g = torch.Generator(device="cuda").manual_seed(20080809)
    A = torch.randn((rows, n), dtype=torch.float64, device="cuda", generator=g).to(dtype)
    best, best_ms = None, float("inf")
    for o in candidate_opts(rows, n, precision, code):
        times = []
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f = Factorization(A, leaf_h=o.leaf_h, chain=o.chain, arity=o.arity, precision=precision)
            f.form_q()
            e1.record()
            torch.cuda.synchronize()
            f.close()
            times.append(e0.elapsed_time(e1))
        ms = min(times[1:])
        if ms < best_ms:
            best, best_ms = o, ms
    _TUNE_CACHE[key] = {"leaf_h": best.leaf_h, "chain": best.chain, "arity": best.arity, "precision": precision,
                        "inplace": 0}
    if path:
        with open(path, "w") as fh:
            json.dump({",".join(map(str, k)): v for k, v in _TUNE_CACHE.items()}, fh, indent=1)
    return best


_BATCH_TUNE_CACHE = {}


def padded_width(n):
    np_ = 16
    while np_ < n:
        np_ *= 2
    return np_


def autotune_batch(mats, precision=0, leaf_hs=(64, 96, 128, 256, 512), arities=(2, 4), reps=2):
    """Per-shape plans for a batch, tuned on the batch itself: for each padded width present
    (16, 32, 64), one pass of coordinate descent over the leaf height and the tree arity of the
    matrices of that width, the others held at their current choice, timing the whole batch's
    factor + thin Q.  Returns (an Opts per matrix, {padded width: (leaf_h, arity)}); the choices
    are cached by (padded widths present, precision, dtype)."""
    import torch

    code = TSQR_F32 if mats[0].dtype == torch.float32 else TSQR_F64
    widths = sorted({padded_width(A.shape[1]) for A in mats})
    key = (tuple(widths), int(precision), int(code))

    def plans_for(choice):
        return [Opts(leaf_h=choice[padded_width(A.shape[1])][0], arity=choice[padded_width(A.shape[1])][1],
                     chain=0, precision=precision, inplace=0) for A in mats]

    def time_plans(choice):
        try:
            b = Batch(mats, want_q=True, plans=plans_for(choice))
        except TsqrError:
            return float("inf")
        ts = []
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.factor()
            b.form_q()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        b.close()
        return min(ts[1:])

    if key not in _BATCH_TUNE_CACHE:
        choice = {w: (0, 2) for w in widths}  # 0: the library's default leaf height
        best = time_plans(choice)
        for w in widths:
            for h in leaf_hs:
                if h < w:
                    continue
                for a in arities:
                    trial = dict(choice)
                    trial[w] = (h, a)
                    t = time_plans(trial)
                    if t < best:
                        best, choice = t, trial
        _BATCH_TUNE_CACHE[key] = choice
    choice = _BATCH_TUNE_CACHE[key]
    return plans_for(choice), dict(choice)


# ---------------------------------------------------------------- differentiation
def _qr_function():
    import torch

    class QR(torch.autograd.Function):
        """(Q, R) = qr(A) by TSQR with a hand-written backward (tsqr_backward).

        keep="tree": the forward keeps its workspace (the implicit Q tree: reflectors, T, tree
        nodes) for the backward.  keep="recompute": the forward frees it and the backward
        factors A again (A is alive anyway), so between forward and backward only Q and R are
        held.  Neither stores an explicit Q for the backward.
        """

        @staticmethod
        def forward(ctx, A, keep, opts):
            f = Factorization(A, **opts)
            Q = f.form_q()
            R = f.R.clone()
            ctx.keep, ctx.opts = keep, opts
            if keep == "tree":
                ctx.fact = f
            else:
                f.close()
                del f
                ctx.fact = None
            ctx.save_for_backward(A, R)
            return Q, R

        @staticmethod
        def backward(ctx, Qbar, Rbar):
            A, R = ctx.saved_tensors
            f = ctx.fact if ctx.fact is not None else Factorization(A, **ctx.opts)
            m, n = A.shape
            Abar = torch.empty((m, n), dtype=A.dtype, device=A.device)
            qb = Qbar.contiguous() if Qbar is not None else None
            rb = Rbar.contiguous() if Rbar is not None else None
            tsqr_backward(f.handle, qb.data_ptr() if qb is not None else None, n,
                          rb.data_ptr() if rb is not None else None, n, R.data_ptr(), n,
                          Abar.data_ptr(), n, _stream())
            if ctx.fact is None:
                torch.cuda.current_stream().synchronize()
                f.close()
            ctx.fact = None
            return Abar, None, None

    class QRBatch(torch.autograd.Function):
        """A batch of independent QRs (A: B x m x n).  Each matrix alone leaves most SMs idle
        during its reduction tree, so the matrices are spread round-robin over a few CUDA streams
        and their launches overlap; the calling stream waits for all of them.  keep as in QR."""

        @staticmethod
        def forward(ctx, A, keep, opts):
            nb, m, n = A.shape
            cur = torch.cuda.current_stream(A.device)
            streams = _side_streams(A.device)
            Q = torch.empty_like(A)
            R = torch.empty((nb, n, n), dtype=A.dtype, device=A.device)
            ready = torch.cuda.Event()
            ready.record(cur)
            facts = []
            for i in range(nb):
                s = streams[i % len(streams)]
                s.wait_event(ready)
                with torch.cuda.stream(s):
                    f = Factorization(A[i], **opts)
                    f.form_q(out=Q[i])
                    R[i].copy_(f.R)
                    if keep == "tree":
                        facts.append(f)
                    else:
                        f.close()
            for s in streams:
                cur.wait_stream(s)
            ctx.keep, ctx.opts, ctx.facts = keep, opts, facts
            ctx.save_for_backward(A, R)
            return Q, R

        @staticmethod
        def backward(ctx, Qbar, Rbar):
            A, R = ctx.saved_tensors
            nb, m, n = A.shape
            cur = torch.cuda.current_stream(A.device)
            streams = _side_streams(A.device)
            Abar = torch.empty_like(A)
            qb = Qbar.contiguous() if Qbar is not None else None
            rb = Rbar.contiguous() if Rbar is not None else None
            ready = torch.cuda.Event()
            ready.record(cur)
            for i in range(nb):
                s = streams[i % len(streams)]
                s.wait_event(ready)
                with torch.cuda.stream(s):
                    f = ctx.facts[i] if ctx.keep == "tree" else Factorization(A[i], **ctx.opts)
                    tsqr_backward(f.handle, qb[i].data_ptr() if qb is not None else None, n,
                                  rb[i].data_ptr() if rb is not None else None, n, R[i].data_ptr(), n,
                                  Abar[i].data_ptr(), n, _stream())
                    if ctx.keep != "tree":
                        f.close()
            for s in streams:
                cur.wait_stream(s)
            ctx.facts = None
            return Abar, None, None

    return QR, QRBatch


_QR = None
_QRB = None
_SIDE = {}


def _side_streams(device, count=8):
    """The pool of CUDA streams a batch of factorizations is spread over (one pool per device)."""
    import torch

    key = torch.device(device).index
    if key not in _SIDE:
        _SIDE[key] = [torch.cuda.Stream(device) for _ in range(count)]
    return _SIDE[key]


def qr_autograd(A, keep="tree", **opts):
    """Differentiable thin QR of a CUDA float64 or float32 matrix, or of a batch (B x m x n, the
    matrices factored concurrently on several streams).  Returns (Q, R) with diag(R) >= 0;
    gradients flow through tsqr_backward."""
    global _QR, _QRB
    if _QR is None:
        _QR, _QRB = _qr_function()
    if A.dim() == 2:
        return _QR.apply(A.contiguous(), keep, dict(opts))
    if A.dim() != 3:
        raise ValueError("A must be m x n or B x m x n")
    return _QRB.apply(A.contiguous(), keep, dict(opts))
