"""GB300 (sm_103a) mixed precision preconditioned Jacobi eigensolver and SVD.

A thin binding over the C ABI of ``libmpjacobi.so`` (include/mpjacobi.h): it
marshals torch CUDA tensors (device memory and the current stream) into the
plain-pointer calls.  Every step of the computation runs in the library's CUDA
kernels; there is no CPU or library fallback, and a missing library raises.

Matrices are exchanged column-major: a column-major n x n buffer is the
transpose of torch's row-major view, so outputs are returned as transposed
views of the column-major buffers.

Entry points (Zhang & Bai, arXiv 2211.03339):
  syevj_mp / syevj_plain   Algorithm 4.1 / Algorithm 3.2
  gesvj_mp / gesvj_plain   Algorithm 5.2 / Algorithm 5.1
  stage1_syevj32, mgs, congruence, sweeps   single steps of Algorithm 4.1
"""
from __future__ import annotations

import ctypes
import os
import threading

U = 2.0 ** -53
UPS = 2.0 ** -24

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmpjacobi.so")

_lock = threading.Lock()
_lib = None

STATUS = {0: "success", 1: "invalid argument", 2: "input holds NaN or Inf",
          3: "not converged within max_sweeps", 4: "rank deficient", 5: "CUDA error",
          6: "no sm_103 device"}

EXPORTS = ["mpj_syevj_mp", "mpj_syevj_plain", "mpj_syevj_workspace_bytes",
           "mpj_gesvj_mp", "mpj_gesvj_plain", "mpj_gesvj_workspace_bytes",
           "mpj_stage1_syevj32", "mpj_mgs", "mpj_mgs_workspace_bytes", "mpj_mgs_noalloc",
           "mpj_congruence", "mpj_congruence_workspace_bytes",
           "mpj_sweeps", "mpj_sweeps_workspace_bytes",
           "mpj_profile_enable", "mpj_profile_reset", "mpj_profile_read", "mpj_profile_units", "mpj_profile_name",
           "mpj_profile_classes", "mpj_kernel_launches",
           "mpj_batch_plan_create", "mpj_batch_plan_info", "mpj_syevj_batched",
           "mpj_batch_plan_destroy", "mpj_syev_backward_batched",
           "mpj_syev_backward_workspace_bytes",
           "mpj_status_string", "mpj_last_error", "mpj_version"]


class Stats(ctypes.Structure):
    """Mirror of ``mpj_stats``."""
    _fields_ = [("sweeps", ctypes.c_int), ("sweeps_stage1", ctypes.c_int),
                ("rotations", ctypes.c_double), ("rotations_stage1", ctypes.c_double),
                ("off_T0", ctypes.c_double), ("off_final", ctypes.c_double),
                ("norm_A", ctypes.c_double), ("ms_stage", ctypes.c_float * 4),
                ("block", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_stage"}
        d["ms_stage"] = list(self.ms_stage)
        return d


class Options(ctypes.Structure):
    """Mirror of ``mpj_options`` (zero fields mean 'default'); ``flags`` takes the
    OPT_* bits below."""
    _fields_ = [("max_sweeps", ctypes.c_int), ("max_sweeps_stage1", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("tol_stage1", ctypes.c_double),
                ("ju_ratio", ctypes.c_double), ("block", ctypes.c_int),
                ("flags", ctypes.c_int), ("stage1_tf32_terms", ctypes.c_int)]


# mpj_options.flags (include/mpjacobi.h)
OPT_SIMT_STAGE1 = 1
OPT_SIMT_SWEEPS = 2
OPT_FP64_PRODUCTS = 4
OPT_FULL_INNER = 8
OPT_MGS_GLOBAL = 16
OPT_TRACE = 32
OPT_FP64_SOLVES = 64


class BatchTuning(ctypes.Structure):
    """Mirror of ``mpj_batch_tuning`` (zero fields mean 'default')."""
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("block_large", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("max_sweeps_stage1", ctypes.c_int)]


class MPJError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


def lib():
    """The loaded C library with argument types declared (raises if not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2211_03339_gb300.build` "
                "(the library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        p, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        op, sp = ctypes.POINTER(Options), ctypes.POINTER(Stats)
        for name in ("mpj_syevj_mp", "mpj_syevj_plain"):
            f = getattr(L, name)
            f.argtypes = [p, i, i, p, p, i, d, op, sp, p, sz, p]
            f.restype = i
        for name in ("mpj_gesvj_mp", "mpj_gesvj_plain"):
            f = getattr(L, name)
            f.argtypes = [p, i, i, i, p, p, i, p, i, d, op, sp, p, sz, p]
            f.restype = i
        L.mpj_syevj_workspace_bytes.argtypes = [i]; L.mpj_syevj_workspace_bytes.restype = sz
        L.mpj_gesvj_workspace_bytes.argtypes = [i, i]; L.mpj_gesvj_workspace_bytes.restype = sz
        L.mpj_stage1_syevj32.argtypes = [p, i, i, p, i, p, op, sp, p, sz, p]
        L.mpj_stage1_syevj32.restype = i
        L.mpj_mgs.argtypes = [p, i, i, i, p, i, p, sz, p]; L.mpj_mgs.restype = i
        L.mpj_mgs_workspace_bytes.argtypes = [i, i]; L.mpj_mgs_workspace_bytes.restype = sz
        L.mpj_mgs_noalloc.argtypes = [p, i, i, i, p, i, p]; L.mpj_mgs_noalloc.restype = i
        L.mpj_congruence.argtypes = [p, i, p, i, i, p, i, p, sz, p]; L.mpj_congruence.restype = i
        L.mpj_congruence_workspace_bytes.argtypes = [i]
        L.mpj_congruence_workspace_bytes.restype = sz
        L.mpj_sweeps.argtypes = [p, i, p, i, i, d, d, op, sp, p, sz, p]; L.mpj_sweeps.restype = i
        L.mpj_sweeps_workspace_bytes.argtypes = [i]; L.mpj_sweeps_workspace_bytes.restype = sz
        L.mpj_status_string.argtypes = [i]; L.mpj_status_string.restype = ctypes.c_char_p
        L.mpj_last_error.argtypes = []; L.mpj_last_error.restype = ctypes.c_char_p
        L.mpj_version.argtypes = []; L.mpj_version.restype = ctypes.c_char_p
        L.mpj_profile_enable.argtypes = [i]; L.mpj_profile_enable.restype = None
        L.mpj_profile_reset.argtypes = []; L.mpj_profile_reset.restype = None
        L.mpj_profile_read.argtypes = [i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(d)]
        L.mpj_profile_read.restype = i
        L.mpj_profile_units.argtypes = [i, ctypes.POINTER(d)]; L.mpj_profile_units.restype = i
        L.mpj_profile_name.argtypes = [i]; L.mpj_profile_name.restype = ctypes.c_char_p
        L.mpj_profile_classes.argtypes = []; L.mpj_profile_classes.restype = i
        L.mpj_kernel_launches.argtypes = []; L.mpj_kernel_launches.restype = ctypes.c_ulonglong
        L.mpj_batch_plan_create.argtypes = [p, i, i, ctypes.POINTER(BatchTuning), ctypes.POINTER(p)]
        L.mpj_batch_plan_create.restype = i
        L.mpj_batch_plan_info.argtypes = [p, ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i),
                                          ctypes.POINTER(sz)]
        L.mpj_batch_plan_info.restype = i
        L.mpj_syevj_batched.argtypes = [p, p, p, p, d, p, p, p]; L.mpj_syevj_batched.restype = i
        L.mpj_batch_plan_destroy.argtypes = [p]; L.mpj_batch_plan_destroy.restype = None
        L.mpj_syev_backward_batched.argtypes = [p, p, p, p, i, i, p, p, sz, p]
        L.mpj_syev_backward_batched.restype = i
        L.mpj_syev_backward_workspace_bytes.argtypes = [i, i]
        L.mpj_syev_backward_workspace_bytes.restype = sz
        _lib = L
        return L


# ---------------------------------------------------------------- torch helpers
def _torch():
    import torch
    return torch


def _stream_ptr(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _colmajor(A):
    """Column-major copy of a 2-D CUDA float64 tensor (its .t().contiguous())."""
    torch = _torch()
    if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2):
        raise TypeError("expected a 2-D torch.float64 CUDA tensor")
    return A.t().contiguous()          # memory = A in column-major order


def _workspace(nbytes, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def _opts(options):
    if options is None:
        return None
    if isinstance(options, Options):
        return ctypes.byref(options)
    o = Options(**options)
    return ctypes.byref(o)


def _check(rc, where, allow_not_converged=False):
    if rc == 0 or (rc == 3 and allow_not_converged):
        return
    detail = lib().mpj_last_error().decode() if rc == 5 else ""
    raise MPJError(rc, where, detail)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- public API
def _syevj(name, A, tol, options, allow_not_converged):
    torch = _torch()
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("A must be square")
    Ac = _colmajor(A)
    lam = torch.empty(n, dtype=torch.float64, device=A.device)
    Vc = torch.empty((n, n), dtype=torch.float64, device=A.device)   # column-major buffer
    ws = _workspace(lib().mpj_syevj_workspace_bytes(n), A.device)
    st = Stats()
    tol = n * U if tol is None else float(tol)
    rc = getattr(lib(), name)(_ptr(Ac), n, n, _ptr(lam), _ptr(Vc), n, tol, _opts(options),
                              ctypes.byref(st), _ptr(ws), ws.numel(), _stream_ptr(A.device))
    _check(rc, name, allow_not_converged)
    return lam, Vc.t(), st.as_dict()


def syevj_mp(A, tol=None, options=None, allow_not_converged=False):
    """Algorithm 4.1: (Lambda ascending, V, stats) of a symmetric float64 CUDA tensor."""
    return _syevj("mpj_syevj_mp", A, tol, options, allow_not_converged)


def syevj_plain(A, tol=None, options=None, allow_not_converged=False):
    """Algorithm 3.2 (parallel block order): (Lambda ascending, V, stats)."""
    return _syevj("mpj_syevj_plain", A, tol, options, allow_not_converged)


def _gesvj(name, A, tol, options, allow_not_converged):
    torch = _torch()
    m, n = A.shape
    if m < n:
        raise ValueError("gesvj needs m >= n")
    Ac = _colmajor(A)
    sig = torch.empty(n, dtype=torch.float64, device=A.device)
    Uc = torch.empty((n, m), dtype=torch.float64, device=A.device)   # column-major m x n
    Vc = torch.empty((n, n), dtype=torch.float64, device=A.device)
    ws = _workspace(lib().mpj_gesvj_workspace_bytes(m, n), A.device)
    st = Stats()
    tol = 8 * U if tol is None else float(tol)
    rc = getattr(lib(), name)(_ptr(Ac), m, n, m, _ptr(sig), _ptr(Uc), m, _ptr(Vc), n, tol,
                              _opts(options), ctypes.byref(st), _ptr(ws), ws.numel(),
                              _stream_ptr(A.device))
    _check(rc, name, allow_not_converged)
    return sig, Uc.t(), Vc.t(), st.as_dict()


def gesvj_mp(A, tol=None, options=None, allow_not_converged=False):
    """Algorithm 5.2: (Sigma descending, U, V, stats) of an m x n float64 CUDA tensor."""
    return _gesvj("mpj_gesvj_mp", A, tol, options, allow_not_converged)


def gesvj_plain(A, tol=None, options=None, allow_not_converged=False):
    """Algorithm 5.1 + ordering/normalisation: (Sigma descending, U, V, stats)."""
    return _gesvj("mpj_gesvj_plain", A, tol, options, allow_not_converged)


def stage1_syevj32(A, options=None):
    """Step 1 of Algorithm 4.1: (Z, D) from FP32 block Jacobi of fl32(A), widened to FP64."""
    torch = _torch()
    n = A.shape[0]
    Ac = _colmajor(A)
    Zc = torch.empty((n, n), dtype=torch.float64, device=A.device)
    D = torch.empty(n, dtype=torch.float64, device=A.device)
    ws = _workspace(lib().mpj_syevj_workspace_bytes(n), A.device)
    st = Stats()
    rc = lib().mpj_stage1_syevj32(_ptr(Ac), n, n, _ptr(Zc), n, _ptr(D), _opts(options),
                                  ctypes.byref(st), _ptr(ws), ws.numel(), _stream_ptr(A.device))
    _check(rc, "mpj_stage1_syevj32", allow_not_converged=True)
    return Zc.t(), D, st.as_dict()


def mgs(Z):
    """Modified Gram-Schmidt (Lemma 2.1): the orthonormal factor Q of Z = Q R."""
    torch = _torch()
    m, n = Z.shape
    Zc = _colmajor(Z)
    Qc = torch.empty((n, m), dtype=torch.float64, device=Z.device)
    ws = _workspace(lib().mpj_mgs_workspace_bytes(m, n), Z.device)
    rc = lib().mpj_mgs(_ptr(Zc), m, n, m, _ptr(Qc), m, _ptr(ws), ws.numel(), _stream_ptr(Z.device))
    _check(rc, "mpj_mgs")
    return Qc.t()


def mgs_noalloc(Z):
    """mgs() without any device allocation: scratch comes from a fixed array in the
    library (for callers that cannot allocate at call time; see include/mpjacobi.h
    for the size limit and the rule that overlapping calls must be serialised)."""
    torch = _torch()
    m, n = Z.shape
    Zc = _colmajor(Z)
    Qc = torch.empty((n, m), dtype=torch.float64, device=Z.device)
    rc = lib().mpj_mgs_noalloc(_ptr(Zc), m, n, m, _ptr(Qc), m, _stream_ptr(Z.device))
    _check(rc, "mpj_mgs_noalloc")
    return Qc.t()


def congruence(A, Q):
    """Step 3 of Algorithm 4.1: T = Q^T A Q (exactly symmetric)."""
    torch = _torch()
    n = A.shape[0]
    Ac, Qc = _colmajor(A), _colmajor(Q)
    Tc = torch.empty((n, n), dtype=torch.float64, device=A.device)
    ws = _workspace(lib().mpj_congruence_workspace_bytes(n), A.device)
    rc = lib().mpj_congruence(_ptr(Ac), n, _ptr(Qc), n, n, _ptr(Tc), n, _ptr(ws), ws.numel(),
                              _stream_ptr(A.device))
    _check(rc, "mpj_congruence")
    return Tc.t()


def sweeps(T, P, tol=None, normA=None, options=None, allow_not_converged=False):
    """Step 4 of Algorithm 4.1 on (T, P): returns (T_final, P_final, stats)."""
    torch = _torch()
    n = T.shape[0]
    Tc, Pc = _colmajor(T), _colmajor(P)
    if normA is None:
        raise ValueError("normA (the ||A||_F of the while-test) is required")
    ws = _workspace(lib().mpj_sweeps_workspace_bytes(n), T.device)
    st = Stats()
    tol = n * U if tol is None else float(tol)
    rc = lib().mpj_sweeps(_ptr(Tc), n, _ptr(Pc), n, n, tol, float(normA), _opts(options),
                          ctypes.byref(st), _ptr(ws), ws.numel(), _stream_ptr(T.device))
    _check(rc, "mpj_sweeps", allow_not_converged)
    return Tc.t(), Pc.t(), st.as_dict()


# ---------------------------------------------------------------- diagnostics
def profile_enable(on=True):
    """Count and time (CUDA events on the launching stream) every library launch."""
    lib().mpj_profile_enable(1 if on else 0)


def profile_reset():
    lib().mpj_profile_reset()


def profile_read():
    """{kernel class: (launches, total_ms)} since the last reset."""
    L = lib()
    out = {}
    for k in range(L.mpj_profile_classes()):
        n, ms = ctypes.c_longlong(), ctypes.c_double()
        L.mpj_profile_read(k, ctypes.byref(n), ctypes.byref(ms))
        out[L.mpj_profile_name(k).decode()] = (n.value, ms.value)
    return out


def profile_units():
    """{kernel class: algorithmic bytes counted by the library} since the last reset."""
    L = lib()
    out = {}
    for k in range(L.mpj_profile_classes()):
        v = ctypes.c_double()
        L.mpj_profile_units(k, ctypes.byref(v))
        out[L.mpj_profile_name(k).decode()] = v.value
    return out


def kernel_launches():
    return int(lib().mpj_kernel_launches())


# ---------------------------------------------------------------- batched solver
class BatchPlan:
    """Plan for many independent eigendecompositions (n_i <= 256) in one launch.

    ``ns``: the sizes; ``method``: "mp" (Alg. 4.1) or "plain" (Alg. 3.2).  The
    packed layouts (column-major, ld n_i) are: A_i and V_i at offset
    sum_{j<i} n_j^2, Lambda_i at sum_{j<i} n_j.  ``run`` enqueues one memset and
    one kernel on the current stream (no host synchronisation, capturable).
    """

    def __init__(self, ns, method="mp", tuning=None):
        import numpy as np
        self.ns = np.asarray(ns, dtype=np.int32)
        self.method = 1 if method == "mp" else 0
        arr = (ctypes.c_int * len(self.ns))(*[int(x) for x in self.ns])
        handle = ctypes.c_void_p()
        tun = None
        if tuning is not None:
            tun = tuning if isinstance(tuning, BatchTuning) else BatchTuning(**tuning)
        rc = lib().mpj_batch_plan_create(ctypes.cast(arr, ctypes.c_void_p), len(self.ns), self.method,
                                         ctypes.byref(tun) if tun is not None else None,
                                         ctypes.byref(handle))
        _check(rc, "mpj_batch_plan_create")
        self.handle = handle
        a, l, c, b = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int(), ctypes.c_size_t()
        lib().mpj_batch_plan_info(handle, ctypes.byref(a), ctypes.byref(l), ctypes.byref(c), ctypes.byref(b))
        self.a_elems, self.lambda_elems, self.ctas, self.scratch_bytes = a.value, l.value, c.value, b.value
        self.a_offsets = np.concatenate([[0], np.cumsum(self.ns.astype(np.int64) ** 2)])[:-1]
        self.l_offsets = np.concatenate([[0], np.cumsum(self.ns.astype(np.int64))])[:-1]

    def outputs(self, device="cuda"):
        torch = _torch()
        return (torch.empty(self.lambda_elems, dtype=torch.float64, device=device),
                torch.empty(self.a_elems, dtype=torch.float64, device=device),
                torch.empty(len(self.ns), dtype=torch.int32, device=device),
                torch.empty(len(self.ns), dtype=torch.int32, device=device))

    def run(self, A_packed, Lam, V, status=None, sweeps=None, tol=0.0):
        """Enqueue the batched solve of the packed A on the current stream."""
        rc = lib().mpj_syevj_batched(self.handle, _ptr(A_packed), _ptr(Lam), _ptr(V), float(tol),
                                     _ptr(status) if status is not None else None,
                                     _ptr(sweeps) if sweeps is not None else None,
                                     _stream_ptr(A_packed.device))
        _check(rc, "mpj_syevj_batched")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.mpj_batch_plan_destroy(h)
            self.handle = None


def pack_symmetric(mats):
    """Concatenate column-major copies of square float64 numpy matrices."""
    import numpy as np
    return np.concatenate([np.asarray(M, dtype=np.float64).ravel(order="F") for M in mats])


# ---------------------------------------------------------------- differentiation
def syev_backward(lam, V, glam, gV):
    """A_bar of a batch (b, n, n): V, gV are the logical matrices (b, n, n)."""
    torch = _torch()
    b, n = lam.shape
    Vc = V.transpose(-1, -2).contiguous()               # column-major buffers
    gVc = gV.transpose(-1, -2).contiguous() if gV is not None else None
    gl = glam.contiguous() if glam is not None else None
    gA = torch.empty((b, n, n), dtype=torch.float64, device=V.device)
    ws = _workspace(lib().mpj_syev_backward_workspace_bytes(n, b), V.device)
    rc = lib().mpj_syev_backward_batched(_ptr(lam.contiguous()), _ptr(Vc),
                                         _ptr(gl) if gl is not None else None,
                                         _ptr(gVc) if gVc is not None else None, n, b, _ptr(gA),
                                         _ptr(ws), ws.numel(), _stream_ptr(V.device))
    _check(rc, "mpj_syev_backward_batched")
    return gA.transpose(-1, -2)                         # symmetric: either layout


_plans = {}


def _eigh_batched_forward(A, method):
    b, n, _ = A.shape
    key = (n, b, method, A.device.index)
    plan = _plans.get(key)
    if plan is None:
        plan = _plans[key] = BatchPlan([n] * b, method=method)
    Ac = A.transpose(-1, -2).contiguous().reshape(-1)   # column-major packed
    Lam, V, st, sw = plan.outputs(A.device)
    plan.run(Ac, Lam, V, st, sw)
    if int((st != 0).sum().item()) != 0:
        raise MPJError(int(st[st != 0][0].item()), "mpj_syevj_batched")
    return Lam.view(b, n), V.view(b, n, n).transpose(-1, -2)


def _make_function():
    torch = _torch()

    class EighFunction(torch.autograd.Function):
        """Batched symmetric eigendecomposition (Alg. 4.1 forward) with the
        hand-written backward kernel."""

        @staticmethod
        def forward(ctx, A, method="mp"):
            lam, V = _eigh_batched_forward(A, method)
            ctx.save_for_backward(lam, V)
            return lam, V

        @staticmethod
        def backward(ctx, glam, gV):
            lam, V = ctx.saved_tensors
            return syev_backward(lam, V, glam, gV), None

    return EighFunction


_EighFunction = None


def eigh(A, method="mp"):
    """Differentiable (lambda ascending, V) of a batch (b, n, n) of symmetric float64
    CUDA matrices, n <= 256: forward by the batched solver, backward by
    mpj_syev_backward_batched."""
    global _EighFunction
    if _EighFunction is None:
        _EighFunction = _make_function()
    if A.dim() == 2:
        lam, V = _EighFunction.apply(A.unsqueeze(0), method)
        return lam[0], V[0]
    return _EighFunction.apply(A, method)
