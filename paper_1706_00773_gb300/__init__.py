"""GB300 (sm_103a) rank-k symmetric eigen-update (Oh & Hu, arXiv 1706.00773).

Thin Python binding of the C ABI in ``include/eig_update.h``: the functions
below carry the same names and only marshal arguments (torch CUDA tensors to
device pointers, streams, structs).  Every step of the update runs in the CUDA
kernels of ``libeigupdate.so``; there is no CPU or PyTorch fallback, and
loading fails with an error when the library has not been built.

Layout: matrices are FP64, column-major (a torch tensor ``Q`` of shape (n, n)
with strides (1, n), e.g. ``torch.empty(n, n).t()`` or ``colmajor(t)``).
Q's columns are eigenvectors; lambda is ascending.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "EIG_OK", "EIG_EINVAL", "EIG_ENOMEM", "EIG_ENOTCONV", "EIG_ETIMEOUT", "EIG_ECUDA",
    "EIG_ENOTSUP", "EIG_EBUSY", "EIG_FP64", "EIG_MIXED", "EIG_VALUES", "EIG_VECTORS",
    "EIG_REPORT", "EIG_ASYNC", "EIG_MAX_K", "EIG_Q_STATUS", "EIG_Q_REPORT", "EIG_Q_LAST_STATUS",
    "EIG_Q_COUNT", "EIG_Q_WORKSPACE", "EIG_Q_METRICS", "EigError", "lib", "library_path", "colmajor",
    "eig_update_init", "eig_update_destroy", "eig_update_rank_k", "eig_update_batch", "eig_update_release",
    "eig_update_query", "eig_project", "eig_secular_values", "eig_make_rank2", "eig_version", "eig_last_cuda_error",
    "eig_count", "Updater", "eig_secular_values_static", "EIG_ETOOBIG", "EIG_STATIC_MAX_N",
    "eig_server_create", "eig_server_destroy", "eig_server_add_resident", "eig_server_submit",
    "eig_server_poll", "eig_server_query", "eig_server_pending", "Server", "eig_location_rank2",
    "eig_perturbation", "eig_update_select", "eig_pole_counts", "eig_fp64_fma_rate", "EIG_TUNE",
]

EIG_OK, EIG_EINVAL, EIG_ENOMEM, EIG_ENOTCONV = 0, -1, -2, -3
EIG_ETIMEOUT, EIG_ECUDA, EIG_ENOTSUP, EIG_EBUSY, EIG_ETOOBIG = -4, -5, -6, -7, -8
EIG_STATIC_MAX_N = 8192
EIG_MAX_K = 16
EIG_FP64, EIG_MIXED = 0, 1
EIG_VALUES, EIG_VECTORS, EIG_REPORT, EIG_ASYNC = 1, 2, 4, 8
EIG_TUNE = 1
EIG_Q_STATUS, EIG_Q_REPORT, EIG_Q_LAST_STATUS, EIG_Q_COUNT, EIG_Q_WORKSPACE, EIG_Q_METRICS = 1, 2, 3, 4, 5, 6

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libeigupdate.so")

_NAMES = {EIG_OK: "EIG_OK", EIG_EINVAL: "EIG_EINVAL", EIG_ENOMEM: "EIG_ENOMEM",
          EIG_ENOTCONV: "EIG_ENOTCONV", EIG_ETIMEOUT: "EIG_ETIMEOUT", EIG_ECUDA: "EIG_ECUDA",
          EIG_ENOTSUP: "EIG_ENOTSUP", EIG_EBUSY: "EIG_EBUSY", EIG_ETOOBIG: "EIG_ETOOBIG"}


class EigError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        super().__init__("%s failed: %s (%d)%s" % (what, _NAMES.get(code, "?"), code,
                                                   (": " + detail) if detail else ""))
        self.code = code
        self.detail = detail


class eig_init_params(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("mode", ctypes.c_uint32), ("hbm_budget", ctypes.c_uint64),
                ("max_iter", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class eig_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("Q", ctypes.c_void_p), ("lambda_", ctypes.c_void_p), ("K", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("Q_out", ctypes.c_void_p), ("want", ctypes.c_uint32),
                ("pad2_", ctypes.c_uint32), ("errors", ctypes.c_void_p)]


class eig_metrics(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("updates", ctypes.c_int64), ("eigenpairs", ctypes.c_int64),
                ("updates_ok", ctypes.c_int64), ("updates_failed", ctypes.c_int64),
                ("updates_pending", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("workspace_allocs", ctypes.c_int64), ("workspace_bytes", ctypes.c_uint64),
                ("tune_trials", ctypes.c_int64), ("tune_hits", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class eig_report(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_deflated", ctypes.c_int64), ("iters_total", ctypes.c_int64),
                ("n_notconv", ctypes.c_int64), ("k", ctypes.c_int32), ("status", ctypes.c_int32),
                ("iters_max", ctypes.c_int32), ("n_checked", ctypes.c_int32),
                ("max_residual", ctypes.c_double), ("max_orth", ctypes.c_double),
                ("norm_A", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_project", ctypes.c_double), ("ms_deflate", ctypes.c_double),
                ("ms_counts", ctypes.c_double), ("ms_roots", ctypes.c_double),
                ("ms_assemble", ctypes.c_double), ("ms_slice", ctypes.c_double), ("ms_gemm", ctypes.c_double),
                ("launches", ctypes.c_int32), ("n_runs", ctypes.c_int32), ("iters32_total", ctypes.c_int64),
                ("redo32_total", ctypes.c_int64), ("taylor_total", ctypes.c_int64),
                ("max_pair_residual", ctypes.c_double), ("max_pair_rayleigh", ctypes.c_double),
                ("max_pair_orth", ctypes.c_double), ("tc_pair_tiles", ctypes.c_int64),
                ("asm_fp64_cols", ctypes.c_int64), ("gj32_total", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class eig_server_params(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("mode", ctypes.c_uint32), ("hbm_budget", ctypes.c_uint64),
                ("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32)]


class eig_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("resident", ctypes.c_int32), ("k", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("submit_ms", ctypes.c_double), ("launch_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class eig_count_args(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int32), ("npts", ctypes.c_int32),
                ("lambda_", ctypes.c_void_p), ("U", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("counts", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded C library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError("libeigupdate.so is not built (run __graft_entry__.build() or "
                               "python paper_1706_00773_gb300/build.py); the update has no CPU path")
        L = ctypes.CDLL(library_path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.eig_update_init.argtypes = [ctypes.POINTER(eig_init_params), ctypes.POINTER(vp)]
        L.eig_update_destroy.argtypes = [vp]
        L.eig_update_rank_k.argtypes = [vp, ctypes.POINTER(eig_problem), ctypes.POINTER(eig_report), vp]
        L.eig_update_batch.argtypes = [vp, i32, ctypes.POINTER(eig_problem), ctypes.POINTER(ctypes.c_uint64), vp]
        L.eig_update_release.argtypes = [vp, ctypes.c_uint64]
        L.eig_update_query.argtypes = [vp, i32, vp, vp, ctypes.c_size_t]
        L.eig_project.argtypes = [vp, i64, i32, vp, vp, vp, vp]
        L.eig_secular_values.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp, vp]
        L.eig_make_rank2.argtypes = [i64, i64, vp, vp, vp, vp]
        L.eig_location_rank2.argtypes = [i64, vp, vp, vp, vp, vp, vp]
        L.eig_perturbation.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp, vp, vp]
        L.eig_update_select.argtypes = [vp, i64, i32, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, i64,
                                        vp, vp, ctypes.POINTER(i64), vp]
        L.eig_secular_values_static.argtypes = [i64, i32, vp, vp, vp, vp, vp, i32, vp]
        L.eig_pole_counts.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64), vp]
        L.eig_fp64_fma_rate.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double), vp]
        L.eig_server_create.argtypes = [ctypes.POINTER(eig_server_params), ctypes.POINTER(vp)]
        L.eig_server_destroy.argtypes = [vp]
        L.eig_server_add_resident.argtypes = [vp, i64, vp, vp, ctypes.POINTER(i32)]
        L.eig_server_submit.argtypes = [vp, i32, i32, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.eig_server_poll.argtypes = [vp, i32]
        L.eig_server_query.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(eig_request_info)]
        L.eig_server_pending.argtypes = [vp]
        for f in ("eig_server_create", "eig_server_destroy", "eig_server_add_resident", "eig_server_submit",
                  "eig_server_poll", "eig_server_query", "eig_server_pending"):
            getattr(L, f).restype = ctypes.c_int
        L.eig_version.restype = ctypes.c_char_p
        L.eig_last_cuda_error.argtypes = [ctypes.c_char_p, i32]
        L.eig_last_cuda_error.restype = ctypes.c_int
        for f in ("eig_update_init", "eig_update_destroy", "eig_update_rank_k", "eig_update_batch",
                  "eig_update_release", "eig_update_query", "eig_project", "eig_secular_values", "eig_make_rank2",
                  "eig_secular_values_static", "eig_location_rank2", "eig_perturbation",
                  "eig_update_select", "eig_pole_counts", "eig_fp64_fma_rate"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def colmajor(t):
    """Column-major (Fortran-order) FP64 copy of a 2-D tensor."""
    import torch

    t = t.to(torch.float64)
    return t.t().contiguous().t()


def _ptr(t, what: str, cols_major: bool = False):
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != torch.float64:
        raise TypeError("%s must be float64" % what)
    if t.dim() == 2 and cols_major and t.shape[0] > 1 and t.shape[1] > 1 and t.stride() != (1, t.shape[0]):
        raise ValueError("%s must be column-major (strides (1, rows)); use colmajor()" % what)
    if t.dim() == 1 and t.stride(0) != 1:
        raise ValueError("%s must be contiguous" % what)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _sigma_buf(sigma, k):
    if sigma is None:
        return None, None
    vals = [int(v) for v in (sigma.tolist() if hasattr(sigma, "tolist") else sigma)]
    if len(vals) != k:
        raise ValueError("sigma must have k entries")
    buf = (ctypes.c_int8 * k)(*vals)
    return buf, ctypes.cast(buf, ctypes.c_void_p)


def eig_last_cuda_error():
    """(code, message) of the CUDA error behind this thread's last EIG_ECUDA (0, "" if none)."""
    buf = ctypes.create_string_buffer(256)
    code = lib().eig_last_cuda_error(buf, 256)
    return code, buf.value.decode(errors="replace")


def _check(rc: int, what: str, ok=(EIG_OK,)):
    if rc not in ok:
        detail = ""
        if rc == EIG_ECUDA:
            code, msg = eig_last_cuda_error()
            detail = msg if code else ""
        raise EigError(rc, what, detail)
    return rc


# ---------------------------------------------------------------------------
# C-ABI functions (same names)
# ---------------------------------------------------------------------------
def eig_version() -> str:
    return lib().eig_version().decode()


def eig_update_init(device: int = 0, mode: int = EIG_FP64, hbm_budget: int = 0, max_iter: int = 0,
                    flags: int = 0):
    p = eig_init_params(device, mode, hbm_budget, max_iter, flags)
    h = ctypes.c_void_p()
    _check(lib().eig_update_init(ctypes.byref(p), ctypes.byref(h)), "eig_update_init")
    return h


def eig_update_destroy(h) -> None:
    _check(lib().eig_update_destroy(h), "eig_update_destroy")


def _problem(Q, lam, K, sigma, want, Q_out=None, errors=None):
    n = int(lam.shape[0])
    k = int(K.shape[1]) if K.dim() == 2 else 1
    sbuf, sp = _sigma_buf(sigma, k)
    if errors is not None and (tuple(errors.shape) != (n, 4) or errors.stride() != (1, n)):
        raise ValueError("errors must be an n x 4 column-major float64 tensor (e.g. torch.empty(4, n).t())")
    P = eig_problem(n, k, 0, _ptr(Q, "Q", True), _ptr(lam, "lambda"), _ptr(K, "K", True), sp,
                    _ptr(Q_out, "Q_out", True) if Q_out is not None else None, want, 0,
                    _ptr(errors, "errors") if errors is not None else None)
    return P, sbuf


def eig_update_rank_k(h, Q, lam, K, sigma=None, want: int = EIG_VALUES | EIG_VECTORS, Q_out=None,
                      stream=None, raise_on_error: bool = True, errors=None):
    """One update in place (lam, and Q unless Q_out); errors: optional n x 4
    column-major per-eigenpair report.  Returns (status, report dict)."""
    P, keep = _problem(Q, lam, K, sigma, want, Q_out, errors)
    rep = eig_report()
    rc = lib().eig_update_rank_k(h, ctypes.byref(P), ctypes.byref(rep), _stream(stream))
    del keep
    if raise_on_error:
        _check(rc, "eig_update_rank_k", ok=(EIG_OK, EIG_ENOTCONV))
    return rc, rep.as_dict()


def eig_update_batch(h, problems, stream=None):
    """problems: list of dicts with Q, lam, K[, sigma, want, Q_out].  Returns ticket ids."""
    arr = (eig_problem * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        P, sb = _problem(p["Q"], p["lam"], p["K"], p.get("sigma"),
                         p.get("want", EIG_VALUES | EIG_VECTORS), p.get("Q_out"), p.get("errors"))
        arr[i] = P
        keep.append(sb)
    tickets = (ctypes.c_uint64 * max(1, len(problems)))()
    _check(lib().eig_update_batch(h, len(problems), arr, tickets, _stream(stream)), "eig_update_batch")
    ids = [int(tickets[i]) for i in range(len(problems))]
    for t in ids:  # the call's host buffers live until its tickets are released
        _batch_keepalive[(h.value if hasattr(h, "value") else h, t)] = (arr, keep)
    return ids


def eig_update_release(h, ticket: int) -> int:
    """Free a finished batch ticket (EIG_EBUSY while it runs, EIG_EINVAL if unknown)."""
    rc = lib().eig_update_release(h, int(ticket))
    if rc == EIG_OK:
        _batch_keepalive.pop((h.value if hasattr(h, "value") else h, int(ticket)), None)
    return rc


_batch_keepalive = {}


def eig_update_query(h, what: int, ticket: int | None = None):
    L = lib()
    if what in (EIG_Q_STATUS, EIG_Q_REPORT):
        t = ctypes.c_uint64(ticket)
        if what == EIG_Q_STATUS:
            out = ctypes.c_int32()
            rc = L.eig_update_query(h, what, ctypes.byref(t), ctypes.byref(out), ctypes.sizeof(out))
            return rc
        rep = eig_report()
        rc = L.eig_update_query(h, what, ctypes.byref(t), ctypes.byref(rep), ctypes.sizeof(rep))
        return rc, rep.as_dict()
    if what == EIG_Q_LAST_STATUS:
        out = ctypes.c_int32()
        return L.eig_update_query(h, what, None, ctypes.byref(out), ctypes.sizeof(out))
    if what == EIG_Q_METRICS:
        m = eig_metrics()
        _check(L.eig_update_query(h, what, None, ctypes.byref(m), ctypes.sizeof(m)), "eig_update_query(METRICS)")
        return m.as_dict()
    raise ValueError("use eig_count / workspace_bytes for this query")


def workspace_bytes(h, n: int, k: int, want: int = EIG_VALUES | EIG_VECTORS, in_place: bool = True) -> int:
    P = eig_problem(n, k, 0, None, None, None, None, None if in_place else ctypes.c_void_p(1), want, 0)
    out = ctypes.c_uint64()
    _check(lib().eig_update_query(h, EIG_Q_WORKSPACE, ctypes.byref(P), ctypes.byref(out),
                                  ctypes.sizeof(out)), "eig_update_query(WORKSPACE)")
    return int(out.value)


def eig_count(h, lam, U, sigma, x, counts, stream=None) -> None:
    """#{mu < x_j} for diag(lam) + U Sigma U^T at device points x into int32 counts."""
    import torch

    n = int(lam.shape[0])
    k = int(U.shape[1])
    if counts.dtype != torch.int32 or not counts.is_cuda:
        raise TypeError("counts must be a CUDA int32 tensor")
    sbuf, sp = _sigma_buf(sigma, k)
    a = eig_count_args(n, k, int(x.shape[0]), _ptr(lam, "lambda"), _ptr(U, "U", True), sp,
                       _ptr(x, "x"), ctypes.c_void_p(counts.data_ptr()), _stream(stream))
    _check(lib().eig_update_query(h, EIG_Q_COUNT, ctypes.byref(a), None, 0), "eig_update_query(COUNT)")
    del sbuf


def eig_project(h, Q, K, U, stream=None) -> None:
    n = int(Q.shape[0])
    k = int(K.shape[1])
    _check(lib().eig_project(h, n, k, _ptr(Q, "Q", True), _ptr(K, "K", True), _ptr(U, "U", True),
                             _stream(stream)), "eig_project")


def eig_secular_values(h, lam, U, sigma, mu, iters=None, stream=None) -> int:
    n = int(lam.shape[0])
    k = int(U.shape[1])
    sbuf, sp = _sigma_buf(sigma, k)
    ip = ctypes.c_void_p(iters.data_ptr()) if iters is not None else None
    rc = lib().eig_secular_values(h, n, k, _ptr(lam, "lambda"), _ptr(U, "U", True), sp, _ptr(mu, "mu"),
                                  ip, _stream(stream))
    del sbuf
    return _check(rc, "eig_secular_values", ok=(EIG_OK, EIG_ENOTCONV))


def _iptr(t, what: str):
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32 or t.dim() != 1 or t.stride(0) != 1:
        raise TypeError("%s must be a contiguous CUDA int32 vector" % what)
    return ctypes.c_void_p(t.data_ptr())


def eig_pole_counts(h, lam, U, sigma, counts, counts32=None, idx_keep=None, stream=None):
    """Pole counts of the deflated sub-problem as the update computes them in the
    handle's mode (device int32 outputs of n entries).  Returns (status, n_keep)."""
    n = int(lam.shape[0])
    k = int(U.shape[1])
    for t, nm in ((counts, "counts"), (counts32, "counts32"), (idx_keep, "idx_keep")):
        if t is not None and int(t.numel()) < n:
            raise ValueError("%s needs n entries" % nm)
    sbuf, sp = _sigma_buf(sigma, k)
    nk = ctypes.c_int64()
    rc = lib().eig_pole_counts(h, n, k, _ptr(lam, "lambda"), _ptr(U, "U", True), sp, _iptr(counts, "counts"),
                               _iptr(counts32, "counts32"), _iptr(idx_keep, "idx_keep"), ctypes.byref(nk),
                               _stream(stream))
    del sbuf
    _check(rc, "eig_pole_counts")
    return rc, int(nk.value)


def eig_secular_values_static(lam, U, sigma, mu, iters=None, max_iter: int = 0, stream=None) -> int:
    """eig_secular_values without any device allocation (fixed library scratch,
    n <= EIG_STATIC_MAX_N); returns the status code without raising."""
    n = int(lam.shape[0])
    k = int(U.shape[1])
    sbuf, sp = _sigma_buf(sigma, k)
    ip = ctypes.c_void_p(iters.data_ptr()) if iters is not None else None
    rc = lib().eig_secular_values_static(n, k, _ptr(lam, "lambda"), _ptr(U, "U", True), sp, _ptr(mu, "mu"),
                                         ip, max_iter, _stream(stream))
    del sbuf
    return rc


def eig_fp64_fma_rate(device: int = 0, reps: int = 10, stream=None) -> float:
    """Measured FP64 FMA throughput of the device, GFLOP/s (2 flops per FMA)."""
    out = ctypes.c_double()
    _check(lib().eig_fp64_fma_rate(int(device), int(reps), ctypes.byref(out), _stream(stream)),
           "eig_fp64_fma_rate")
    return float(out.value)


def eig_make_rank2(n: int, j: int, a, K, stream=None):
    """K (n x 2, column-major) and sigma = (+1, -1) with K Sigma K^T = e_j a^T + a e_j^T."""
    sig = (ctypes.c_int8 * 2)()
    _check(lib().eig_make_rank2(n, j, _ptr(a, "a"), _ptr(K, "K", True), ctypes.cast(sig, ctypes.c_void_p),
                                _stream(stream)), "eig_make_rank2")
    return [int(sig[0]), int(sig[1])]


def eig_location_rank2(lam, U, sigma, alpha, L, stream=None) -> None:
    """Residues (device n) and location vector (device int32 n+1) of a rank-2
    update diag(lam) + U Sigma U^T (Algorithms 1a-1c)."""
    import torch

    n = int(lam.shape[0])
    if int(U.shape[1]) != 2:
        raise ValueError("the location vector is defined for rank 2")
    if L.dtype != torch.int32 or not L.is_cuda or int(L.numel()) < n + 1:
        raise TypeError("L must be a CUDA int32 tensor of n+1 entries")
    sbuf, sp = _sigma_buf(sigma, 2)
    _check(lib().eig_location_rank2(n, _ptr(lam, "lambda"), _ptr(U, "U", True), sp, _ptr(alpha, "alpha"),
                                    ctypes.c_void_p(L.data_ptr()), _stream(stream)), "eig_location_rank2")
    del sbuf


def eig_perturbation(h, Q, lam, K, sigma, mu, X, stream=None) -> None:
    """First-order estimate of eq. (11): mu (device n) and X = Q W (device n x n,
    column-major); mu_j pairs with column j of X."""
    n = int(Q.shape[0])
    k = int(K.shape[1])
    sbuf, sp = _sigma_buf(sigma, k)
    _check(lib().eig_perturbation(h, n, k, _ptr(Q, "Q", True), _ptr(lam, "lambda"), _ptr(K, "K", True), sp,
                                  _ptr(mu, "mu"), _ptr(X, "X", True), _stream(stream)), "eig_perturbation")
    del sbuf


def eig_update_select(h, Q, lam, K, sigma, vl, vu, mu, X=None, stream=None):
    """Eigenpairs of A' with eigenvalues in [vl, vu): mu (device, capacity
    max_m = len(mu)) and X (device n x max_m column-major, or None).  Returns
    (status, m); EIG_ETOOBIG (nothing written) when m > max_m."""
    n = int(Q.shape[0])
    k = int(K.shape[1])
    max_m = int(mu.shape[0])
    if X is not None and (int(X.shape[0]) != n or int(X.shape[1]) < max_m):
        raise ValueError("X must be n x max_m")
    sbuf, sp = _sigma_buf(sigma, k)
    m = ctypes.c_int64()
    rc = lib().eig_update_select(h, n, k, _ptr(Q, "Q", True), _ptr(lam, "lambda"), _ptr(K, "K", True), sp,
                                 float(vl), float(vu), max_m, _ptr(mu, "mu"),
                                 _ptr(X, "X", True) if X is not None else None, ctypes.byref(m), _stream(stream))
    del sbuf
    _check(rc, "eig_update_select", ok=(EIG_OK, EIG_ENOTCONV, EIG_ETOOBIG))
    return rc, int(m.value)


class Updater:
    """Handle wrapper: ``Updater(mode).update(Q, lam, K, sigma)``."""

    def __init__(self, device: int = 0, mode: int = EIG_FP64, hbm_budget: int = 0, max_iter: int = 0):
        self.h = eig_update_init(device, mode, hbm_budget, max_iter)

    def update(self, Q, lam, K, sigma=None, want: int = EIG_VALUES | EIG_VECTORS, Q_out=None, stream=None):
        return eig_update_rank_k(self.h, Q, lam, K, sigma, want, Q_out, stream)

    def close(self):
        if self.h:
            eig_update_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Serving (continuous batching over resident decompositions)
# ---------------------------------------------------------------------------
def eig_server_create(device: int = 0, mode: int = EIG_MIXED, hbm_budget: int = 0, slots: int = 0,
                      max_batch: int = 0):
    p = eig_server_params(device, mode, hbm_budget, slots, max_batch)
    s = ctypes.c_void_p()
    _check(lib().eig_server_create(ctypes.byref(p), ctypes.byref(s)), "eig_server_create")
    return s


def eig_server_destroy(srv) -> None:
    _check(lib().eig_server_destroy(srv), "eig_server_destroy")


def eig_server_add_resident(srv, Q, lam) -> int:
    out = ctypes.c_int32()
    _check(lib().eig_server_add_resident(srv, int(lam.shape[0]), _ptr(Q, "Q", True), _ptr(lam, "lambda"),
                                         ctypes.byref(out)), "eig_server_add_resident")
    return int(out.value)


def eig_server_submit(srv, resident: int, K_host, sigma=None) -> int:
    """K_host: numpy (n, k) float64 (any layout; copied column-major)."""
    import numpy as np

    K = np.asfortranarray(np.asarray(K_host, dtype=np.float64))
    if K.ndim == 1:
        K = K.reshape(-1, 1, order="F")
    k = int(K.shape[1])
    sbuf, sp = _sigma_buf(sigma, k)
    t = ctypes.c_uint64()
    _check(lib().eig_server_submit(srv, int(resident), k, K.ctypes.data_as(ctypes.c_void_p), sp, ctypes.byref(t)),
           "eig_server_submit")
    del sbuf
    return int(t.value)


def eig_server_poll(srv, wait_us: int = 0) -> int:
    rc = lib().eig_server_poll(srv, int(wait_us))
    if rc < 0:
        raise EigError(rc, "eig_server_poll")
    return rc


def eig_server_query(srv, ticket: int) -> dict:
    info = eig_request_info()
    lib().eig_server_query(srv, ctypes.c_uint64(ticket), ctypes.byref(info))
    return info.as_dict()


def eig_server_pending(srv) -> int:
    return int(lib().eig_server_pending(srv))


class Server:
    """``Server(mode=...)``: add_resident(Q, lam) -> id, submit(id, K_host, sigma) -> ticket,
    poll(), drain(), query(ticket)."""

    def __init__(self, device: int = 0, mode: int = EIG_MIXED, hbm_budget: int = 0, slots: int = 0,
                 max_batch: int = 0):
        self.s = eig_server_create(device, mode, hbm_budget, slots, max_batch)

    def add_resident(self, Q, lam) -> int:
        return eig_server_add_resident(self.s, Q, lam)

    def submit(self, resident: int, K_host, sigma=None) -> int:
        return eig_server_submit(self.s, resident, K_host, sigma)

    def poll(self, wait_us: int = 0) -> int:
        return eig_server_poll(self.s, wait_us)

    def pending(self) -> int:
        return eig_server_pending(self.s)

    def drain(self, wait_us: int = 200) -> None:
        while self.pending() > 0:
            self.poll(wait_us)

    def query(self, ticket: int) -> dict:
        return eig_server_query(self.s, ticket)

    def close(self):
        if self.s:
            eig_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
