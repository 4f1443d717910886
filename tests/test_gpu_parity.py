"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (binding, from the stated accuracy targets; u = 2^-53):
  relative residual   ||A V - V Lambda||_F / ||A||_F   <= 10 n u
  orthogonality       ||V^T V - I||_F                  <= 10 n u
  eigenvalues         |lambda_i - lambda_i^oracle|     <= 10 n u ||A||_2
The oracle runs at sizes it finishes in seconds (several 64-wide tiles plus a
ragged tail); the full-size cases are checked through properties that hold at
any size (residual, orthogonality, the constructed spectrum).
"""
import functools
import os

import numpy as np
import pytest

import oracle
from paper_2211_03339_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
UPS = 2.0 ** -24


@pytest.fixture(scope="module")
def mpj():
    if not torch.cuda.is_available():
        pytest.fail("gpu tests selected but no CUDA device is visible")
    from paper_2211_03339_gb300 import build
    build.build()
    import paper_2211_03339_gb300 as m
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def evd_metrics(A, lam, V):
    n = A.shape[0]
    res = np.linalg.norm(A @ V - V * lam) / np.linalg.norm(A)
    orth = np.linalg.norm(V.T @ V - np.eye(n))
    return res, orth


def sign_fix(V):
    idx = np.argmax(np.abs(V), axis=0)
    s = np.sign(V[idx, np.arange(V.shape[1])])
    s[s == 0] = 1
    return V * s


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("n", [33, 64, 200, 300])
def test_mgs_parity(mpj, n):
    A, _ = synth.sym_matrix(n, "uniform", seed=100 + n)
    Z, D, _ = oracle.stage1_syev_f(A)          # a nearly orthonormal Z, as in step 2
    Qo, Ro, rc = oracle.mgs(Z)
    assert rc == 0
    Qg = host(mpj.mgs(dev(Z)))
    assert np.abs(Qg - Qo).max() <= 10 * n * U
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n)) <= 10 * n * U


@pytest.mark.parametrize("m,n", [(40, 40), (130, 70), (257, 100)])
def test_mgs_parity_general(mpj, m, n):
    rng = np.random.default_rng(m + n)
    Z = rng.standard_normal((m, n))
    Qo, Ro, rc = oracle.mgs(Z)
    kappa = np.linalg.cond(Z)
    Qg = host(mpj.mgs(dev(Z)))
    assert np.abs(Qg - Qo).max() <= 10 * n * U * kappa


@pytest.mark.parametrize("m,n", [(6500, 45), (13000, 40)])
def test_mgs_parity_tall(mpj, m, n):
    """Tall panels: up to 12800 rows a 32-column panel is held in the shared memory
    of a 16-CTA cluster (more than 400 rows per CTA from 6401 rows on); beyond
    that the panel kernel works from global memory.  Both against the oracle."""
    rng = np.random.default_rng(m + n)
    Z = rng.standard_normal((m, n))
    Qo, Ro, rc = oracle.mgs(Z)
    kappa = np.linalg.cond(Z)
    Qg = host(mpj.mgs(dev(Z)))
    assert np.abs(Qg - Qo).max() <= 10 * n * U * kappa
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n)) <= 10 * n * U


@pytest.mark.parametrize("n", [17, 64, 129, 300])
def test_congruence_parity(mpj, n):
    A, _ = synth.sym_matrix(n, "uniform", seed=200 + n)
    Q = synth.haar(synth.rng_for(300 + n), n)
    To = oracle.congruence(A, Q)
    Tg = host(mpj.congruence(dev(A), dev(Q)))
    assert np.array_equal(Tg, Tg.T)
    gn = n * U / (1 - n * U)
    bound = gn * (2 + gn) * (np.abs(Q).T @ np.abs(A) @ np.abs(Q))
    assert (np.abs(Tg - To) <= 2 * bound).all()


@pytest.mark.parametrize("kind", ["uniform", "geometric", "cluster"])
@pytest.mark.parametrize("n", [64, 200, 257, 513])
def test_sweeps_parity(mpj, n, kind):
    """Step 4 alone from the oracle's T_0 and Q: n <= 256 runs the b = 16 SIMT
    engine, n > 256 the b = 32 engine whose block rotations are applied on the
    tensor cores by exact splitting (a ragged last 128-row slab at 257 and 513)."""
    A, lam = synth.sym_matrix(n, kind, seed=400 + n)
    Lo, Vo, sto, rco, Qo, T0 = oracle.syevj_mp(A, intermediates=True)
    normA = np.linalg.norm(A)
    Tg, Pg, st = mpj.sweeps(dev(T0), dev(Qo), tol=n * U, normA=normA)
    Tg, Pg = host(Tg), host(Pg)
    lam_g = np.sort(np.diag(Tg))
    a2 = np.abs(lam).max()
    assert np.abs(lam_g - Lo).max() <= 10 * n * U * a2
    assert oracle.offnorm(Tg) <= n * U * normA
    assert 1 <= st["sweeps"] <= 12
    res, orth = evd_metrics(A, np.diag(Tg), Pg)
    assert res <= 10 * n * U and orth <= 10 * n * U


@pytest.mark.parametrize("n", [64, 200])
def test_stage1_fp32(mpj, n):
    A, lam = synth.sym_matrix(n, "uniform", seed=500 + n)
    Z, D, st = mpj.stage1_syevj32(dev(A))
    Z, D = host(Z), host(D)
    a2 = np.abs(lam).max()
    assert (np.diff(D) >= 0).all()
    # FP32 eigenvalues within single precision accuracy of the exact spectrum
    assert np.abs(D - lam).max() <= 10 * n * UPS * a2
    init_res = np.linalg.norm(A @ Z - Z * D) / np.linalg.norm(A)
    assert init_res <= 10 * n * UPS
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= 10 * n * UPS
    # Z is exactly representable in single precision (step 1 stores it at omega)
    assert np.array_equal(Z, Z.astype(np.float32).astype(np.float64))


# ------------------------------------------------------------------ end to end (EVD)
@pytest.mark.parametrize("kind", ["uniform", "geometric", "cluster"])
@pytest.mark.parametrize("n", [5, 64, 100, 257])
@pytest.mark.parametrize("method", ["mp", "plain"])
def test_syevj_parity(mpj, n, kind, method):
    A, lam = synth.sym_matrix(n, kind, seed=synth.seed_for(1, n))
    Lo, Vo, sto, rco = oracle.syevj_plain(A)
    f = mpj.syevj_mp if method == "mp" else mpj.syevj_plain
    Lg, Vg, st = f(dev(A))
    Lg, Vg = host(Lg), host(Vg)
    a2 = np.abs(lam).max()
    assert np.abs(Lg - Lo).max() <= 10 * n * U * a2
    res, orth = evd_metrics(A, Lg, Vg)
    assert res <= 10 * n * U, res
    assert orth <= 10 * n * U, orth
    # eigenvectors of well separated eigenvalues agree with the oracle's up to sign
    gaps = np.minimum(np.abs(np.diff(Lo, prepend=-np.inf)), np.abs(np.diff(Lo, append=np.inf)))
    sep = gaps > 1e-3 * a2
    if sep.any():
        dv = np.abs(sign_fix(Vg)[:, sep] - sign_fix(Vo)[:, sep]).max(axis=0)
        assert (dv <= 100 * n * U * a2 / gaps[sep]).all()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_syevj_tiny(mpj, n):
    A, lam = synth.sym_matrix(n, "uniform", seed=7 + n)
    for f in (mpj.syevj_mp, mpj.syevj_plain):
        Lg, Vg, st = f(dev(A))
        Lg, Vg = host(Lg), host(Vg)
        assert np.abs(Lg - np.sort(lam)).max() <= 64 * U
        res, orth = evd_metrics(A, Lg, Vg)
        assert res <= 64 * U and orth <= 64 * U


def test_syevj_diagonal_and_zero(mpj):
    n = 70
    d = np.linspace(-3, 2, n)[::-1].copy()
    A = np.diag(d)
    for f in (mpj.syevj_mp, mpj.syevj_plain):
        Lg, Vg, st = f(dev(A))
        assert np.array_equal(host(Lg), np.sort(d))
    Z = np.zeros((40, 40))
    Lg, Vg, st = mpj.syevj_plain(dev(Z))
    assert (host(Lg) == 0).all()
    assert np.array_equal(host(Vg), np.eye(40))


def test_syevj_nonfinite_input(mpj):
    A, _ = synth.sym_matrix(32, "uniform", seed=1)
    A[3, 5] = A[5, 3] = np.nan
    with pytest.raises(mpj.MPJError) as e:
        mpj.syevj_mp(dev(A))
    assert e.value.status == 2


def test_syevj_lda_larger_than_n(mpj):
    import ctypes
    n, lda = 50, 64
    A, lam = synth.sym_matrix(n, "geometric", seed=3)
    buf = np.zeros((lda, n), order="F"); buf[:n, :] = A
    Ad = dev(buf.T)                              # row-major (n, lda) view = column-major lda x n
    L = mpj.lib()
    lamd = torch.empty(n, dtype=torch.float64, device="cuda")
    Vd = torch.zeros((n, 72), dtype=torch.float64, device="cuda")   # ldv = 72
    st = mpj.Stats()
    rc = L.mpj_syevj_mp(ctypes.c_void_p(Ad.data_ptr()), n, lda, ctypes.c_void_p(lamd.data_ptr()),
                        ctypes.c_void_p(Vd.data_ptr()), 72, n * U, None, ctypes.byref(st), None, 0,
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    V = host(Vd).T[:n, :]
    res, orth = evd_metrics(A, host(lamd), V)
    assert res <= 10 * n * U and orth <= 10 * n * U
    assert (host(Vd).T[n:, :] == 0).all()         # rows beyond n of the ldv slab untouched


def test_not_converged_status(mpj):
    A, lam = synth.sym_matrix(128, "uniform", seed=9)
    Lg, Vg, st = mpj.syevj_plain(dev(A), options={"max_sweeps": 1, "max_inner": 1},
                                 allow_not_converged=True)
    assert st["status"] == 3 and st["sweeps"] == 1
    with pytest.raises(mpj.MPJError):
        mpj.syevj_plain(dev(A), options={"max_sweeps": 1, "max_inner": 1})


# ------------------------------------------------------------------ full size, properties
@pytest.mark.parametrize("n", [1024, 4096])
def test_syevj_full_size_properties(mpj, n):
    A, lam = synth.sym_matrix(n, "uniform", seed=synth.seed_for(1, n))
    a2 = np.abs(lam).max()
    for f in (mpj.syevj_mp, mpj.syevj_plain):
        Lg, Vg, st = f(dev(A))
        Lg, Vg = host(Lg), host(Vg)
        res, orth = evd_metrics(A, Lg, Vg)
        assert res <= 10 * n * U, (f.__name__, res)
        assert orth <= 10 * n * U, (f.__name__, orth)
        # constructed spectrum, with the slack of forming fl(Q diag(lam) Q^T)
        assert np.abs(Lg - lam).max() <= 10 * n * U * a2 + 4 * n * U * a2


# ------------------------------------------------------------------ SVD
@pytest.mark.parametrize("m,n", [(48, 24), (200, 100), (300, 257), (301, 257)])
@pytest.mark.parametrize("method", ["mp", "plain"])
def test_gesvj_parity(mpj, m, n, method):
    """SVD against the oracle. n <= 256 runs the SIMT engines; 300 x 257 the
    tensor-core FP32 step 1 and FP64 sweeps; 301 x 257 (odd m) the tensor-core step 1
    and the SIMT FP64 sweeps (the FP64 tile maps need an even row count)."""
    A, sig, Uc, Vc = synth.svd_matrix(m, n, seed=synth.seed_for(2, n), sigma_min=1e-10)
    So, Uo, Vo, sto, rco = oracle.gesvj_plain(A)
    f = mpj.gesvj_mp if method == "mp" else mpj.gesvj_plain
    Sg, Ug, Vg, st = f(dev(A))
    Sg, Ug, Vg = host(Sg), host(Ug), host(Vg)
    assert (np.diff(Sg) <= 0).all()
    assert np.abs(Sg - So).max() <= 10 * n * U * sig[0]
    assert np.abs(Sg - sig).max() <= 10 * n * U * sig[0] + 4 * n * U * sig[0]
    assert np.linalg.norm(A @ Vg - Ug * Sg) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(Vg.T @ Vg - np.eye(n)) <= 10 * n * U
    assert np.linalg.norm(Ug.T @ Ug - np.eye(n)) <= 10 * n * U


@functools.lru_cache(maxsize=1)
def _oracle_sigma_520x448():
    A = synth.svd_matrix(520, 448, seed=synth.seed_for(2, 7), sigma_min=1e-10)[0]
    return oracle.gesvj_plain(A)[0]


@pytest.mark.parametrize("method", ["mp", "plain"])
def test_gesvj_tensor_core_sweeps_vs_simt(mpj, method):
    """The FP64 one-sided sweeps with exactly split Grams and rotations on the tensor
    cores (n > 256: b = 32, N = 448, m = 520 rows: four full slabs and a ragged one)
    with the block solves' Gram in FP32/FP64 (default) or all FP64 (MPJ_OPT_FP64_SOLVES),
    and the SIMT engine (MPJ_OPT_SIMT_SWEEPS) on the same matrix, all against the
    oracle's singular values; step 1 on the TF32 tensor cores (default) and on the
    SIMT FP32 engine (MPJ_OPT_SIMT_STAGE1)."""
    m, n = 520, 448
    A, sig, _, _ = synth.svd_matrix(m, n, seed=synth.seed_for(2, 7), sigma_min=1e-10)
    So = _oracle_sigma_520x448()
    f = mpj.gesvj_mp if method == "mp" else mpj.gesvj_plain
    for flags in (0, mpj.OPT_FP64_SOLVES, mpj.OPT_SIMT_SWEEPS, mpj.OPT_SIMT_STAGE1):
        Sg, Ug, Vg, st = f(dev(A), options={"flags": flags, "max_sweeps": 100})
        Sg, Ug, Vg = host(Sg), host(Ug), host(Vg)
        assert (np.diff(Sg) <= 0).all()
        assert np.abs(Sg - So).max() <= 10 * n * U * sig[0]
        assert np.linalg.norm(A @ Vg - Ug * Sg) / np.linalg.norm(A) <= 10 * n * U
        assert np.linalg.norm(Vg.T @ Vg - np.eye(n)) <= 10 * n * U
        assert np.linalg.norm(Ug.T @ Ug - np.eye(n)) <= 10 * n * U


@pytest.mark.parametrize("flags", ["tensor", "simt"])
def test_gesvj_plain_graded_relative_accuracy(mpj, flags):
    """One-sided Jacobi keeps every singular value of a column-graded A = B D (B
    Gaussian 600 x 320, D over 12 decades) to high relative accuracy.  On the
    tensor cores the digits of C are scaled per column, so a small column is not
    cut relative to a large one in the same rows; a per-row scale would leave the
    small singular values with errors relative to the largest."""
    m, n = 600, 320
    A = synth.graded_matrix(m, n, seed=synth.seed_for(2, 11), decades=12.0)
    So = oracle.gesvj_plain(A)[0]
    opts = {"max_sweeps": 100, "flags": mpj.OPT_SIMT_SWEEPS if flags == "simt" else 0}
    Sg, Ug, Vg, st = mpj.gesvj_plain(dev(A), options=opts)
    Sg = host(Sg)
    assert So.min() < 1e-11 * So.max()
    assert (np.abs(Sg - So) / So).max() <= 1e-11


def test_gesvj_full_size_properties(mpj):
    m, n = 4096, 2048
    A, sig, _, _ = synth.svd_matrix(m, n, seed=synth.seed_for(2, 0), sigma_min=1e-10)
    Sg, Ug, Vg, st = mpj.gesvj_mp(dev(A))
    Sg, Ug, Vg = host(Sg), host(Ug), host(Vg)
    assert np.abs(Sg - sig).max() <= 10 * n * U * sig[0] + 4 * n * U * sig[0]
    assert np.linalg.norm(A @ Vg - Ug * Sg) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(Vg.T @ Vg - np.eye(n)) <= 10 * n * U
    assert np.linalg.norm(Ug.T @ Ug - np.eye(n)) <= 10 * n * U


# ------------------------------------------------------------------ multiple eigenvalues (Example 2)
@pytest.mark.parametrize("mode", [1, 2, 3, 4, 5])
def test_syevj_multiple_eigenvalues(mpj, mode):
    """Example 2 stand-in, (r, s) = (4, 128): eigenvalues of multiplicity 4.  Within a
    multiple eigenvalue only the invariant subspace is unique, so the checks are the
    residual, orthogonality and eigenvalues (against the exact spectrum)."""
    r, s = 4, 128
    n = r * s
    A, lam = synth.sym_matrix_multiple(r, s, mode, kappa=1e4, seed=synth.seed_for(4, mode))
    for f in (mpj.syevj_mp, mpj.syevj_plain):
        L, V, st = f(dev(A))
        L, V = host(L), host(V)
        res, orth = evd_metrics(A, L, V)
        assert res <= 10 * n * U and orth <= 10 * n * U, (f.__name__, res, orth)
        assert np.abs(L - lam).max() <= 14 * n * U * np.abs(lam).max()


def test_syevj_mp_geometric_late_b16(mpj):
    """Geometric spectrum at n = 1024: after preconditioning T is nearly diagonal but
    needs more than two FP64 sweeps, so the sweeps from the third on run with b = 16.
    Residual, orthogonality and the constructed eigenvalues within the bounds."""
    n = 1024
    A, lam = synth.sym_matrix(n, "geometric", seed=synth.seed_for(1, 77))
    L, V, st = mpj.syevj_mp(dev(A))
    L, V = host(L), host(V)
    assert st["sweeps"] > 2, st
    res, orth = evd_metrics(A, L, V)
    assert res <= 10 * n * U and orth <= 10 * n * U, (res, orth)
    a2 = np.abs(lam).max()
    assert np.abs(L - lam).max() <= 10 * n * U * a2 + 4 * n * U * a2


def test_syevj_mp_n8192_properties(mpj):
    """Largest single-matrix size of the workload (n = 8192), preconditioned path."""
    n = 8192
    A, lam = synth.sym_matrix(n, "uniform", seed=synth.seed_for(1, n))
    Ad = dev(A)
    Lg, Vg, st = mpj.syevj_mp(Ad)
    Vt = Vg.contiguous()
    R = Ad @ Vt - Vt * Lg[None, :]
    res = (torch.linalg.matrix_norm(R) / torch.linalg.matrix_norm(Ad)).item()
    orth = torch.linalg.matrix_norm(Vt.T @ Vt - torch.eye(n, dtype=torch.float64, device="cuda")).item()
    assert res <= 10 * n * U and orth <= 10 * n * U
    a2 = np.abs(lam).max()
    assert np.abs(host(Lg) - lam).max() <= 14 * n * U * a2


def test_gesvj_8192x1024_properties(mpj):
    m, n = 8192, 1024
    A, sig, _, _ = synth.svd_matrix(m, n, seed=synth.seed_for(2, 1), sigma_min=1e-10)
    Sg, Ug, Vg, st = mpj.gesvj_mp(dev(A))
    Sg, Ug, Vg = host(Sg), host(Ug), host(Vg)
    assert np.abs(Sg - sig).max() <= 10 * n * U * sig[0] + 4 * n * U * sig[0]
    assert np.linalg.norm(A @ Vg - Ug * Sg) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(Vg.T @ Vg - np.eye(n)) <= 10 * n * U
    assert np.linalg.norm(Ug.T @ Ug - np.eye(n)) <= 10 * n * U


@pytest.mark.parametrize("n", [129, 1000, 2500])
def test_congruence_tensor_core_accuracy(mpj, n):
    """Step 3 on the tensor cores (exact bf16 splitting) against an FP64 product
    formed in numpy: the error must stay within the FP64 bound of the plain product
    and near FP64 rounding in the Frobenius norm (a plausible slicing error -- a
    dropped slice, a wrong exponent -- is orders of magnitude above both)."""
    A, _ = synth.sym_matrix(n, "uniform", seed=700 + n)
    Q = synth.haar(synth.rng_for(800 + n), n)
    Tg = host(mpj.congruence(dev(A), dev(Q)))
    Tn = Q.T @ (A @ Q)
    Tn = np.triu(Tn) + np.triu(Tn, 1).T
    assert np.array_equal(Tg, Tg.T)
    gn = n * U / (1 - n * U)
    bound = gn * (2 + gn) * (np.abs(Q).T @ np.abs(A) @ np.abs(Q))
    assert (np.abs(Tg - Tn) <= 2 * bound).all()
    assert np.linalg.norm(Tg - Tn) <= 4 * np.sqrt(n) * U * np.linalg.norm(A)


def test_mgs_block_tensor_core_parity(mpj):
    """n >= 1024 takes the block MGS (256-column panels, panel projections on the
    tensor cores by exact splitting): same Q as the oracle's column MGS within
    10 n u kappa(Z), orthonormal to working precision."""
    m, n = 1300, 1100
    rng = np.random.default_rng(m + n)
    Z = rng.standard_normal((m, n))
    Qo, Ro, rc = oracle.mgs(Z)
    kappa = np.linalg.cond(Z)
    Qg = host(mpj.mgs(dev(Z)))
    assert np.abs(Qg - Qo).max() <= 10 * n * U * kappa
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n)) <= 10 * n * U


# ------------------------------------------------------------------ stored oracle results (n = 512, 1024)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def oracle_fixture(name):
    """Eigenvalues the oracle computed for a seeded input (tests/golden/
    make_oracle_fixtures.py, which calls only oracle/ and the input generators)."""
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if not line.startswith("#"):
                vals.extend(float(v) for v in line.split())
    return np.array(vals)


@pytest.mark.parametrize("kind", ["uniform", "geometric", "cluster"])
@pytest.mark.parametrize("method", ["mp", "plain"])
def test_syevj_parity_n1024(mpj, kind, method):
    """n = 1024 (b = 32, tensor-core FP64 sweeps, 8 slabs of 128 rows) against the
    oracle's plain Jacobi eigenvalues of the same seeded matrix."""
    n = 1024
    A, lam = synth.sym_matrix(n, kind, seed=synth.seed_for(1, n))
    Lo = oracle_fixture(f"oracle_eig_n1024_{kind}.txt")
    f = mpj.syevj_mp if method == "mp" else mpj.syevj_plain
    Lg, Vg, st = f(dev(A))
    Lg, Vg = host(Lg), host(Vg)
    a2 = np.abs(lam).max()
    assert np.abs(Lg - Lo).max() <= 10 * n * U * a2
    res, orth = evd_metrics(A, Lg, Vg)
    assert res <= 10 * n * U and orth <= 10 * n * U, (res, orth)


@pytest.mark.parametrize("mode", [1, 2, 3, 4, 5])
def test_syevj_multiple_eigenvalues_vs_oracle(mpj, mode):
    """Example 2 stand-in (r, s) = (4, 128), n = 512: both methods against the
    oracle's eigenvalues of the same matrix (not only the constructed spectrum)."""
    n = 512
    A, lam = synth.sym_matrix_multiple(4, 128, mode, kappa=1e4, seed=synth.seed_for(4, mode))
    Lo = oracle_fixture(f"oracle_eig_n512_multiple_mode{mode}.txt")
    for f in (mpj.syevj_mp, mpj.syevj_plain):
        L, V, st = f(dev(A))
        assert np.abs(host(L) - Lo).max() <= 10 * n * U * np.abs(lam).max(), f.__name__


@pytest.mark.parametrize("n", [257, 1024])
def test_stage1_tensor_core_parity(mpj, n):
    """Step 1 on the tensor-core FP32 engine (b = 32): the FP32 eigenvalues against
    the oracle's single precision Jacobi (oracle.stage1_syev_f) within 10 n upsilon
    ||A||_2, init-Res and orthogonality of Z within 10 n upsilon (Table 6.2)."""
    A, lam = synth.sym_matrix(n, "uniform", seed=500 + n)
    if n <= 300:
        _, Do, _ = oracle.stage1_syev_f(A)
    else:
        Do = oracle_fixture(f"oracle_stage1_n{n}_uniform.txt")
    Z, D, st = mpj.stage1_syevj32(dev(A))
    Z, D = host(Z), host(D)
    a2 = np.abs(lam).max()
    assert np.abs(D - Do).max() <= 10 * n * UPS * a2
    assert np.linalg.norm(A @ Z - Z * D) / np.linalg.norm(A) <= 10 * n * UPS
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= 10 * n * UPS


@pytest.mark.parametrize("n", [257, 1024])
def test_syevj_mp_one_term_tf32_stage1(mpj, n):
    """A lower-precision step 1 (TF32 hi*hi products only, about 2^-11; Sec. 6,
    Figs. 6.2-6.3): the FP64 sweeps still reach the FP64 bars against the oracle,
    with at least as many FP64 sweeps as the three-term step 1."""
    kind = "uniform"
    A, lam = synth.sym_matrix(n, kind, seed=synth.seed_for(1, n))
    Lo = oracle.syevj_plain(A)[0] if n <= 300 else oracle_fixture(f"oracle_eig_n{n}_{kind}.txt")
    L1, V1, st1 = mpj.syevj_mp(dev(A), options={"stage1_tf32_terms": 1, "tol_stage1": 2.0 ** -10})
    L3, V3, st3 = mpj.syevj_mp(dev(A))
    L1, V1 = host(L1), host(V1)
    a2 = np.abs(lam).max()
    assert np.abs(L1 - Lo).max() <= 10 * n * U * a2
    res, orth = evd_metrics(A, L1, V1)
    assert res <= 10 * n * U and orth <= 10 * n * U, (res, orth)
    assert st1["sweeps"] >= st3["sweeps"]
    assert st1["off_T0"] > st3["off_T0"]


@pytest.mark.parametrize("kind", ["uniform", "geometric", "cluster"])
@pytest.mark.parametrize("method", ["mp", "plain"])
def test_syevj_parity_simt_engines(mpj, kind, method):
    """The SIMT engines kept for comparison (MPJ_OPT_SIMT_STAGE1 / SIMT_SWEEPS /
    FP64_PRODUCTS: double-float and FP64 tile products, FP64 GEMMs) at b = 32
    against the oracle."""
    n = 257
    A, lam = synth.sym_matrix(n, kind, seed=synth.seed_for(1, n))
    Lo, Vo, sto, rco = oracle.syevj_plain(A)
    flags = mpj.OPT_SIMT_STAGE1 | mpj.OPT_SIMT_SWEEPS | mpj.OPT_FP64_PRODUCTS
    f = mpj.syevj_mp if method == "mp" else mpj.syevj_plain
    Lg, Vg, st = f(dev(A), options={"flags": flags})
    Lg, Vg = host(Lg), host(Vg)
    assert np.abs(Lg - Lo).max() <= 10 * n * U * np.abs(lam).max()
    res, orth = evd_metrics(A, Lg, Vg)
    assert res <= 10 * n * U and orth <= 10 * n * U


def test_syevj_mp_full_inner_schedule(mpj):
    """The full-tournament inner schedule of the tensor-core FP64 sweeps
    (MPJ_OPT_FULL_INNER) against the oracle."""
    n = 513
    A, lam = synth.sym_matrix(n, "cluster", seed=synth.seed_for(1, n))
    Lo = oracle.syevj_plain(A)[0]
    Lg, Vg, st = mpj.syevj_mp(dev(A), options={"flags": mpj.OPT_FULL_INNER})
    Lg, Vg = host(Lg), host(Vg)
    assert np.abs(Lg - Lo).max() <= 10 * n * U * np.abs(lam).max()
    res, orth = evd_metrics(A, Lg, Vg)
    assert res <= 10 * n * U and orth <= 10 * n * U


def test_congruence_parity_n1024(mpj):
    """Step 3 at n = 1024 elementwise against oracle.congruence (extended
    precision) within the FP64 bound of Sec. 4."""
    n = 1024
    A, _ = synth.sym_matrix(n, "uniform", seed=200 + n)
    Q = synth.haar(synth.rng_for(300 + n), n)
    To = oracle.congruence(A, Q)
    Tg = host(mpj.congruence(dev(A), dev(Q)))
    assert np.array_equal(Tg, Tg.T)
    gn = n * U / (1 - n * U)
    bound = gn * (2 + gn) * (np.abs(Q).T @ np.abs(A) @ np.abs(Q))
    assert (np.abs(Tg - To) <= 2 * bound).all()


@pytest.mark.parametrize("method", ["mp", "plain"])
def test_gesvj_parity_1300x1100(mpj, method):
    """SVD at n >= 1024: the block MGS with tensor-core panel projections (step 2)
    and C = A Q by exact splitting (step 3) on the preconditioned path; singular
    values against the oracle's one-sided Jacobi of the same matrix."""
    m, n = 1300, 1100
    A, sig, _, _ = synth.svd_matrix(m, n, seed=synth.seed_for(2, n), sigma_min=1e-10)
    So = oracle_fixture("oracle_svd_1300x1100.txt")
    f = mpj.gesvj_mp if method == "mp" else mpj.gesvj_plain
    Sg, Ug, Vg, st = f(dev(A), options={"max_sweeps": 100})
    Sg, Ug, Vg = host(Sg), host(Ug), host(Vg)
    assert np.abs(Sg - So).max() <= 10 * n * U * sig[0]
    assert np.linalg.norm(A @ Vg - Ug * Sg) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(Vg.T @ Vg - np.eye(n)) <= 10 * n * U
    assert np.linalg.norm(Ug.T @ Ug - np.eye(n)) <= 10 * n * U
