"""GPU test of mpj_mgs_noalloc, the MGS entry point for callers that cannot
allocate device memory at call time (its scratch is a fixed array inside the
library).  Its results must match those of mpj_mgs, the allocating entry point,
within the MGS tolerance the parity tests use (10 n u kappa(Z), elementwise),
on two calls in a row -- the second call reuses the array the first one left
behind.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2211_03339_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def mpj():
    if not torch.cuda.is_available():
        pytest.fail("gpu tests selected but no CUDA device is visible")
    from paper_2211_03339_gb300 import build
    build.build()
    import paper_2211_03339_gb300 as m
    return m


def _col(Z):
    """Column-major device copy of a numpy matrix."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(Z).T)).cuda()


def _call(fn_name, mpj, Z, expect=0):
    m, n = Z.shape
    L = mpj.lib()
    Zd = _col(Z)
    Qd = torch.empty((n, m), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if fn_name == "mpj_mgs":
        ws = torch.empty(L.mpj_mgs_workspace_bytes(m, n), dtype=torch.uint8, device="cuda")
        rc = L.mpj_mgs(ctypes.c_void_p(Zd.data_ptr()), m, n, m, ctypes.c_void_p(Qd.data_ptr()), m,
                       ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream)
    else:
        rc = L.mpj_mgs_noalloc(ctypes.c_void_p(Zd.data_ptr()), m, n, m,
                               ctypes.c_void_p(Qd.data_ptr()), m, stream)
    assert rc == expect, (fn_name, rc)
    return Qd.cpu().numpy().T


def test_mgs_noalloc_matches_mgs_on_two_calls(mpj):
    cases = []
    A, _ = synth.sym_matrix(300, "uniform", seed=7301)
    Z1, _, _ = oracle.stage1_syev_f(A)                       # nearly orthonormal, as in step 2
    cases.append(Z1)
    rng = np.random.default_rng(7302)
    cases.append(rng.standard_normal((257, 200)))           # general m x n, ragged panels
    for Z in cases:
        n = Z.shape[1]
        kappa = np.linalg.cond(Z)
        Q_ref = _call("mpj_mgs", mpj, Z)
        Q_new = _call("mpj_mgs_noalloc", mpj, Z)
        assert np.abs(Q_new - Q_ref).max() <= 10 * n * U * kappa
        assert np.linalg.norm(Q_new.T @ Q_new - np.eye(n)) <= 10 * n * U * kappa


def test_mgs_noalloc_clears_the_rank_flag_between_calls(mpj):
    """The rank flag lives in the shared array: a call on a Z with a zero column
    reports MPJ_RANK_DEFICIENT (4), and the next call on a full-rank Z must start
    from a cleared flag, return 0 and match mpj_mgs."""
    rng = np.random.default_rng(7303)
    Zbad = rng.standard_normal((200, 96))
    Zbad[:, 40] = 0.0
    _call("mpj_mgs_noalloc", mpj, Zbad, expect=4)
    Z = rng.standard_normal((200, 96))
    n = Z.shape[1]
    kappa = np.linalg.cond(Z)
    Q_new = _call("mpj_mgs_noalloc", mpj, Z)
    Q_ref = _call("mpj_mgs", mpj, Z)
    assert np.abs(Q_new - Q_ref).max() <= 10 * n * U * kappa


def test_mgs_noalloc_rejects_sizes_beyond_its_scratch(mpj):
    L = mpj.lib()
    big = 4096    # 32 * 4096 * (1 + 16) doubles > the fixed 2^20
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = L.mpj_mgs_noalloc(p, big, big, big, p, big,
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"MPJ_MGS_NOALLOC_MAX_SCRATCH_DOUBLES" in L.mpj_last_error()
