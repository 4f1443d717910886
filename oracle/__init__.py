"""CPU oracle for the mixed precision preconditioned Jacobi method.

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, links or runs anything in this directory; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.
The oracle shares no code with the CUDA path.

``oracle.c`` holds the arithmetic (plain scalar C, double precision, no FMA
contraction).  This module compiles it with gcc on first use and exposes
numpy wrappers.  Every wrapper takes and returns column-major (Fortran order)
float64 arrays.

Passages followed (Zhang & Bai, arXiv 2211.03339):
  rotation      -- Lemma 3.1
  jacobi_step   -- eq. (3.1) and the update formulas in the proofs of Lemmas 3.4/3.5
  syev_cyclic   -- Algorithm 3.2 (row-cyclic), skip rule of Remark 3.7
  mgs           -- Lemma 2.1 (modified Gram-Schmidt)
  congruence    -- Algorithm 4.1 step 3
  syevj_plain   -- Algorithm 3.2 from P = I
  syevj_mp      -- Algorithm 4.1
  gesvj_plain   -- Algorithm 5.1 (+ ordering/normalisation of Alg. 5.2 steps 11-13)
  gesvj_mp      -- Algorithm 5.2

One-sided Jacobi stopping (a reading): Sec. 6 runs Alg. 5.1/5.2 with eps = omega
and stops when a sweep applies fewer than 2e-4 N rotations.  The Frobenius test
on the unscaled Gram matrix cannot see the columns of small norm (with sigma down
to 1e-10 their inner products are far below omega ||C^T C||_F), so the wrappers
default to eps = 0: the iteration is ended by the rotation-count rule, and a pair
is rotated only while |c_i^T c_j| > tol_rot ||c_i|| ||c_j|| (tol_rot = sqrt(m) u).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

U = 2.0 ** -53     # omega = u, double precision unit roundoff (Sec. 6)
UPS = 2.0 ** -24   # upsilon, single precision unit roundoff (Sec. 6)

_lock = threading.Lock()
_lib = None


class Stats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int),
        ("rotations", ctypes.c_long),
        ("off_initial", ctypes.c_double),
        ("off_final", ctypes.c_double),
        ("sweeps_stage1", ctypes.c_int),
        ("rotations_stage1", ctypes.c_long),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        sp = ctypes.POINTER(Stats)
        lib.orc_rotation.argtypes = [d, d, d, ctypes.POINTER(d), ctypes.POINTER(d)]
        lib.orc_rotation_f.argtypes = [ctypes.c_float] * 3 + [ctypes.POINTER(ctypes.c_float)] * 2
        lib.orc_offnorm.argtypes = [p, i]; lib.orc_offnorm.restype = d
        lib.orc_fnorm.argtypes = [p, i, i]; lib.orc_fnorm.restype = d
        lib.orc_jacobi_step.argtypes = [p, p, i, i, i]
        lib.orc_syev_cyclic.argtypes = [p, p, i, d, d, d, i, sp, p]; lib.orc_syev_cyclic.restype = i
        lib.orc_syev_cyclic_f.argtypes = [p, p, i, d, d, ctypes.c_float, i, sp]
        lib.orc_syev_cyclic_f.restype = i
        lib.orc_mgs.argtypes = [p, i, i, p, p]; lib.orc_mgs.restype = i
        lib.orc_congruence.argtypes = [p, p, i, p]
        lib.orc_syevj_plain.argtypes = [p, i, p, p, d, i, sp]; lib.orc_syevj_plain.restype = i
        lib.orc_stage1_syev_f.argtypes = [p, i, d, i, p, p, sp]; lib.orc_stage1_syev_f.restype = i
        lib.orc_syevj_mp.argtypes = [p, i, p, p, d, d, i, sp, p, p]; lib.orc_syevj_mp.restype = i
        lib.orc_gesvj_cyclic.argtypes = [p, p, i, i, d, d, d, i, sp]; lib.orc_gesvj_cyclic.restype = i
        lib.orc_gesvj_plain.argtypes = [p, i, i, p, p, p, d, d, d, i, sp]
        lib.orc_gesvj_plain.restype = i
        lib.orc_stage1_gesvj_f.argtypes = [p, i, i, ctypes.c_float, d, i, p, sp]
        lib.orc_stage1_gesvj_f.restype = i
        lib.orc_gesvj_mp.argtypes = [p, i, i, p, p, p, d, d, d, i, sp]
        lib.orc_gesvj_mp.restype = i
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------- primitives
def rotation(aii: float, ajj: float, aij: float):
    """(c, s) of Lemma 3.1 in double precision."""
    c, s = ctypes.c_double(), ctypes.c_double()
    _load().orc_rotation(aii, ajj, aij, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def rotation_f(aii: float, ajj: float, aij: float):
    """(c, s) of Lemma 3.1 evaluated in single precision."""
    c, s = ctypes.c_float(), ctypes.c_float()
    f = ctypes.c_float
    _load().orc_rotation_f(f(aii), f(ajj), f(aij), ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def offnorm(A) -> float:
    A = _f64(A)
    return _load().orc_offnorm(_ptr(A), A.shape[0])


def jacobi_step(T, P, p: int, q: int):
    """One rotation in the (p, q) plane: returns (J^T T J, P J)."""
    T = _f64(T).copy(order="F"); P = _f64(P).copy(order="F")
    _load().orc_jacobi_step(_ptr(T), _ptr(P), T.shape[0], p, q)
    return T, P


def syev_cyclic(T, P=None, tol: float | None = None, normA: float | None = None,
                eps_skip: float = U, max_sweeps: int = 100, history: bool = False):
    """Algorithm 3.2 (row-cyclic) in place on copies of T and P."""
    T = _f64(T).copy(order="F"); n = T.shape[0]
    P = np.asfortranarray(np.eye(n)) if P is None else _f64(P).copy(order="F")
    if tol is None:
        tol = n * U
    if normA is None:
        normA = float(np.linalg.norm(T))
    st = Stats()
    hist = np.zeros(max_sweeps + 1)
    rc = _load().orc_syev_cyclic(_ptr(T), _ptr(P), n, tol, normA, eps_skip, max_sweeps,
                                 ctypes.byref(st), _ptr(hist))
    out = dict(status=rc, T=T, P=P, stats=st.as_dict())
    if history:
        out["off_history"] = hist[: st.sweeps + 1].copy()
    return out


def syev_cyclic_f(T, P=None, tol: float = 4 * UPS, normA: float | None = None,
                  eps_skip: float = UPS, max_sweeps: int = 100):
    """Algorithm 3.2 carried out in single precision (step 1 of Alg. 4.1)."""
    T = np.asfortranarray(np.asarray(T, dtype=np.float32)).copy(order="F"); n = T.shape[0]
    P = np.asfortranarray(np.eye(n, dtype=np.float32)) if P is None else \
        np.asfortranarray(np.asarray(P, dtype=np.float32)).copy(order="F")
    if normA is None:
        normA = float(np.linalg.norm(T.astype(np.float64)))
    st = Stats()
    rc = _load().orc_syev_cyclic_f(_ptr(T), _ptr(P), n, tol, normA, ctypes.c_float(eps_skip),
                                   max_sweeps, ctypes.byref(st))
    return dict(status=rc, T=T, P=P, stats=st.as_dict())


def mgs(Z):
    """Modified Gram-Schmidt QR of Z (m x n): returns (Q, R, status)."""
    Z = _f64(Z); m, n = Z.shape
    Q = np.zeros((m, n), order="F"); R = np.zeros((n, n), order="F")
    rc = _load().orc_mgs(_ptr(Z), m, n, _ptr(Q), _ptr(R))
    return Q, R, rc


def congruence(A, Q):
    """T = Q^T A Q (upper triangle computed, mirrored)."""
    A = _f64(A); Q = _f64(Q); n = A.shape[0]
    T = np.zeros((n, n), order="F")
    _load().orc_congruence(_ptr(A), _ptr(Q), n, _ptr(T))
    return T


# ---------------------------------------------------------------- drivers
def syevj_plain(A, tol: float | None = None, max_sweeps: int = 100):
    """Algorithm 3.2 from T = A, P = I; returns (Lambda ascending, V, stats, status)."""
    A = _f64(A); n = A.shape[0]
    if tol is None:
        tol = n * U
    lam = np.zeros(n); V = np.zeros((n, n), order="F"); st = Stats()
    rc = _load().orc_syevj_plain(_ptr(A), n, _ptr(lam), _ptr(V), tol, max_sweeps, ctypes.byref(st))
    return lam, V, st.as_dict(), rc


def stage1_syev_f(A, tol1: float = 4 * UPS, max_sweeps: int = 100):
    """Step 1 of Alg. 4.1: single precision Jacobi of fl32(A); returns (Z, D, stats)."""
    A = _f64(A); n = A.shape[0]
    Z = np.zeros((n, n), order="F"); D = np.zeros(n); st = Stats()
    _load().orc_stage1_syev_f(_ptr(A), n, tol1, max_sweeps, _ptr(Z), _ptr(D), ctypes.byref(st))
    return Z, D, st.as_dict()


def syevj_mp(A, tol: float | None = None, tol1: float = 4 * UPS, max_sweeps: int = 100,
             intermediates: bool = False):
    """Algorithm 4.1; returns (Lambda ascending, V, stats, status[, Q, T0])."""
    A = _f64(A); n = A.shape[0]
    if tol is None:
        tol = n * U
    lam = np.zeros(n); V = np.zeros((n, n), order="F"); st = Stats()
    Q = np.zeros((n, n), order="F"); T0 = np.zeros((n, n), order="F")
    rc = _load().orc_syevj_mp(_ptr(A), n, _ptr(lam), _ptr(V), tol, tol1, max_sweeps,
                              ctypes.byref(st), _ptr(Q), _ptr(T0))
    if intermediates:
        return lam, V, st.as_dict(), rc, Q, T0
    return lam, V, st.as_dict(), rc


def gesvj_cyclic(C, V=None, eps: float = 0.0, tol_rot: float | None = None,
                 ju_ratio: float = 2e-4, max_sweeps: int = 100):
    """Algorithm 5.1 in place on copies of C (m x n) and V."""
    C = _f64(C).copy(order="F"); m, n = C.shape
    V = np.asfortranarray(np.eye(n)) if V is None else _f64(V).copy(order="F")
    if tol_rot is None:
        tol_rot = np.sqrt(m) * U
    st = Stats()
    rc = _load().orc_gesvj_cyclic(_ptr(C), _ptr(V), m, n, eps, tol_rot, ju_ratio, max_sweeps,
                                  ctypes.byref(st))
    return dict(status=rc, C=C, V=V, stats=st.as_dict())


def gesvj_plain(A, eps: float = 0.0, tol_rot: float | None = None, ju_ratio: float = 2e-4,
                max_sweeps: int = 100):
    """Algorithm 5.1 + Alg. 5.2 steps 11-13; returns (Sigma desc, U, V, stats, status)."""
    A = _f64(A); m, n = A.shape
    if tol_rot is None:
        tol_rot = np.sqrt(m) * U
    sig = np.zeros(n); Uo = np.zeros((m, n), order="F"); Vo = np.zeros((n, n), order="F")
    st = Stats()
    rc = _load().orc_gesvj_plain(_ptr(A), m, n, _ptr(sig), _ptr(Uo), _ptr(Vo), eps, tol_rot,
                                 ju_ratio, max_sweeps, ctypes.byref(st))
    return sig, Uo, Vo, st.as_dict(), rc


def stage1_gesvj_f(A, tol_rot: float | None = None, ju_ratio: float = 2e-4, max_sweeps: int = 100):
    """Step 1 of Alg. 5.2 in single precision; returns (Z, stats)."""
    A = _f64(A); m, n = A.shape
    if tol_rot is None:
        tol_rot = np.sqrt(m) * UPS
    Z = np.zeros((n, n), order="F"); st = Stats()
    _load().orc_stage1_gesvj_f(_ptr(A), m, n, ctypes.c_float(tol_rot), ju_ratio, max_sweeps,
                               _ptr(Z), ctypes.byref(st))
    return Z, st.as_dict()


def gesvj_mp(A, eps: float = 0.0, tol_rot: float | None = None, ju_ratio: float = 2e-4,
             max_sweeps: int = 100):
    """Algorithm 5.2; returns (Sigma desc, U, V, stats, status)."""
    A = _f64(A); m, n = A.shape
    if tol_rot is None:
        tol_rot = np.sqrt(m) * U
    sig = np.zeros(n); Uo = np.zeros((m, n), order="F"); Vo = np.zeros((n, n), order="F")
    st = Stats()
    rc = _load().orc_gesvj_mp(_ptr(A), m, n, _ptr(sig), _ptr(Uo), _ptr(Vo), eps, tol_rot,
                              ju_ratio, max_sweeps, ctypes.byref(st))
    return sig, Uo, Vo, st.as_dict(), rc
