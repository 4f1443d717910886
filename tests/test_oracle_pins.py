"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

None of these compare the oracle with itself.  The pins are:
  * hand-derived 2x2 rotations (Lemma 3.1) and an explicit J from eq. (3.1);
  * the exact invariants stated after Lemma 3.1 (zeroed entry, b_ii^2 + b_jj^2,
    the off-norm drop by 2 a_ij^2, untouched entries, trace, Frobenius norm);
  * brute force for n <= 4: the quadratic formula, the trigonometric closed form
    for 3x3, exact characteristic polynomials with rational bisection, and
    exactly representable matrices with exactly known spectra;
  * constructed spectra Q diag(lam) Q^T;
  * MGS against a hand example, Householder QR (unique QR with r_jj > 0) and
    the bounds of Lemma 2.1 / Lemma 4.1;
  * the congruence against an extended-precision product and the bound
    |T - Q^T A Q| <= gamma_n (2 + gamma_n) |Q|^T |A| |Q|;
  * the bound ||off(Q^T A Q)||_F <= 10 bd, bd = n ||A|| upsilon (Sec. 6, Fig. 6.1);
  * one-sided Jacobi (Lemma 5.1, Alg. 5.1/5.2) against constructed singular values.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2211_03339_gb300 import synth

U = 2.0 ** -53
UPS = 2.0 ** -24
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# ------------------------------------------------------------------ Lemma 3.1
def test_rotation_golden_cases():
    for row in _rows("rotation_2x2.txt"):
        aii, ajj, aij, mu, t, c, s, bii, bjj = [float(x) for x in row]
        cc, ss = oracle.rotation(aii, ajj, aij)
        assert cc == pytest.approx(c, abs=2 * U), row
        assert ss == pytest.approx(s, abs=2 * U), row
        T = np.array([[aii, aij], [aij, ajj]], order="F")
        B, P = oracle.jacobi_step(T, np.eye(2), 0, 1)
        scale = abs(aii) + abs(ajj) + abs(aij)
        assert B[0, 0] == pytest.approx(bii, abs=8 * U * scale)
        assert B[1, 1] == pytest.approx(bjj, abs=8 * U * scale)
        assert B[0, 1] == 0.0 and B[1, 0] == 0.0


def test_rotation_properties_random():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        aii, ajj, aij = rng.standard_normal(3) * 10.0 ** rng.uniform(-6, 6, 3)
        c, s = oracle.rotation(aii, ajj, aij)
        assert abs(c * c + s * s - 1.0) <= 4 * U
        assert abs(s) <= c + 4 * U           # |theta| <= pi/4, the inner rotation
        # b_ij of J^T A J with the explicit 2x2 J of eq. (3.1) vanishes (Lemma 3.1)
        J = np.array([[c, s], [-s, c]])
        A = np.array([[aii, aij], [aij, ajj]])
        B = J.T @ A @ J
        assert abs(B[0, 1]) <= 8 * U * (abs(aii) + abs(ajj) + abs(aij))


def test_rotation_single_precision_matches_lemma():
    rng = np.random.default_rng(2)
    for _ in range(500):
        aii, ajj, aij = rng.standard_normal(3)
        c, s = oracle.rotation_f(aii, ajj, aij)
        J = np.array([[c, s], [-s, c]], dtype=np.float64)
        A = np.array([[aii, aij], [aij, ajj]], dtype=np.float32).astype(np.float64)
        B = J.T @ A @ J
        assert abs(B[0, 1]) <= 16 * UPS * (abs(aii) + abs(ajj) + abs(aij))


def _explicit_J(n, p, q, c, s):
    """J(p,q;c,s) of eq. (3.1): I + [e_p e_q] [[c-1, s], [-s, c-1]] [e_p e_q]^T."""
    J = np.eye(n)
    J[p, p] = c; J[q, q] = c; J[p, q] = s; J[q, p] = -s
    return J


def test_single_step_invariants_and_explicit_J():
    rng = np.random.default_rng(3)
    n = 9
    G = rng.standard_normal((n, n)); A = np.asfortranarray(G + G.T)
    for (p, q) in [(0, 1), (2, 7), (3, 8), (0, 8)]:
        B, P = oracle.jacobi_step(A, np.eye(n), p, q)
        c, s = oracle.rotation(A[p, p], A[q, q], A[p, q])
        J = _explicit_J(n, p, q, c, s)
        ref = J.T @ A @ J
        ref[p, q] = ref[q, p] = 0.0
        assert np.abs(B - ref).max() <= 16 * U * np.abs(A).max()
        assert np.abs(P - J).max() == 0.0
        # exact zero at (p,q), element invariance outside rows/cols p,q (eq. (3.2))
        assert B[p, q] == 0.0 and B[q, p] == 0.0
        mask = np.ones((n, n), bool); mask[[p, q], :] = False; mask[:, [p, q]] = False
        assert np.array_equal(B[mask], A[mask])
        # b_pp^2 + b_qq^2 = a_pp^2 + a_qq^2 + 2 a_pq^2 (Lemma 3.1)
        lhs = B[p, p] ** 2 + B[q, q] ** 2
        rhs = A[p, p] ** 2 + A[q, q] ** 2 + 2 * A[p, q] ** 2
        assert lhs == pytest.approx(rhs, rel=32 * U)
        # ||off(B)||^2 = ||off(A)||^2 - 2 a_pq^2 (text after Lemma 3.1)
        assert oracle.offnorm(B) ** 2 == pytest.approx(oracle.offnorm(A) ** 2 - 2 * A[p, q] ** 2,
                                                       rel=64 * n * U)
        assert np.trace(B) == pytest.approx(np.trace(A), abs=16 * U * np.abs(A).sum())
        assert np.linalg.norm(B) == pytest.approx(np.linalg.norm(A), rel=16 * n * U)


# ------------------------------------------------------------------ brute force, n <= 4
def test_n2_quadratic_formula():
    rng = np.random.default_rng(4)
    for _ in range(200):
        a, d, b = rng.standard_normal(3)
        A = np.array([[a, b], [b, d]], order="F")
        lam, V, st, rc = oracle.syevj_plain(A)
        disc = np.sqrt(((a - d) / 2) ** 2 + b * b)
        ref = np.sort([(a + d) / 2 - disc, (a + d) / 2 + disc])
        assert rc == 0
        assert np.abs(lam - ref).max() <= 16 * U * (abs(a) + abs(b) + abs(d))


def _eig3_trig(A):
    """Closed-form eigenvalues of a real symmetric 3x3 (Smith, CACM 1961)."""
    q = np.trace(A) / 3.0
    p1 = A[0, 1] ** 2 + A[0, 2] ** 2 + A[1, 2] ** 2
    p2 = (A[0, 0] - q) ** 2 + (A[1, 1] - q) ** 2 + (A[2, 2] - q) ** 2 + 2 * p1
    p = np.sqrt(p2 / 6.0)
    B = (A - q * np.eye(3)) / p
    r = np.clip(np.linalg.det(B) / 2.0, -1.0, 1.0)
    phi = np.arccos(r) / 3.0
    e1 = q + 2 * p * np.cos(phi)
    e3 = q + 2 * p * np.cos(phi + 2 * np.pi / 3)
    e2 = 3 * q - e1 - e3
    return np.sort([e1, e2, e3])


def test_n3_trigonometric_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(100):
        G = rng.standard_normal((3, 3)); A = np.asfortranarray(G + G.T)
        lam, V, st, rc = oracle.syevj_plain(A)
        assert rc == 0
        assert np.abs(lam - _eig3_trig(A)).max() <= 1e-13 * np.abs(A).max()


def _charpoly_exact(A):
    """Characteristic polynomial of a rational matrix by Faddeev-LeVerrier, exact Fractions."""
    n = len(A)
    M = [[Fraction(0)] * n for _ in range(n)]
    coeffs = [Fraction(1)]
    I = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    c = Fraction(1)
    for k in range(1, n + 1):
        # M_k = A M_{k-1} + c_{k-1} I ; c_k = -tr(A M_k)/k
        AM = [[sum(A[i][l] * M[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
        M = [[AM[i][j] + c * I[i][j] for j in range(n)] for i in range(n)]
        AM = [[sum(A[i][l] * M[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
        c = -sum(AM[i][i] for i in range(n)) / k
        coeffs.append(c)
    return coeffs  # x^n + c1 x^(n-1) + ... + cn


def _peval(coeffs, x):
    v = Fraction(0)
    for c in coeffs:
        v = v * x + c
    return v


def _real_roots_bisect(coeffs, lo, hi, grid=4000, iters=70):
    xs = [lo + (hi - lo) * Fraction(i, grid) for i in range(grid + 1)]
    vals = [_peval(coeffs, x) for x in xs]
    roots = []
    for i in range(grid):
        a, b, fa, fb = xs[i], xs[i + 1], vals[i], vals[i + 1]
        if fa == 0:
            roots.append(a); continue
        if fa * fb < 0:
            for _ in range(iters):
                mid = (a + b) / 2
                fm = _peval(coeffs, mid)
                if fa * fm <= 0:
                    b = mid
                else:
                    a, fa = mid, fm
            roots.append((a + b) / 2)
    return [float(r) for r in roots]


@pytest.mark.parametrize("n", [3, 4])
def test_brute_force_exact_charpoly(n):
    rng = np.random.default_rng(10 + n)
    for _ in range(3):
        Ai = rng.integers(-9, 10, (n, n)); Ai = Ai + Ai.T
        A = [[Fraction(int(x)) for x in row] for row in Ai]
        coeffs = _charpoly_exact(A)
        R = int(np.abs(Ai).sum(axis=1).max()) + 1          # Gershgorin radius bound
        roots = _real_roots_bisect(coeffs, Fraction(-R), Fraction(R))
        if len(roots) != n:        # a double root or two roots inside one grid cell
            continue
        lam, V, st, rc = oracle.syevj_plain(np.asfortranarray(Ai.astype(np.float64)))
        assert rc == 0
        assert np.abs(lam - np.sort(roots)).max() <= 64 * U * R


def test_exactly_representable_spectra():
    v = np.ones(4)
    H = np.eye(4) - 0.5 * np.outer(v, v)
    for row in _rows("exact_spectra.txt"):
        d = np.array([float(x) for x in row])
        A = np.asfortranarray(H @ np.diag(d) @ H)
        assert np.array_equal(A, A.T)
        lam, V, st, rc = oracle.syevj_plain(A)
        assert rc == 0
        assert np.abs(lam - np.sort(d)).max() <= 32 * U * np.abs(d).max()
        assert np.linalg.norm(A @ V - V * lam) <= 64 * U * np.abs(d).max()


# ------------------------------------------------------------------ Alg. 3.2 / 4.1
@pytest.mark.parametrize("kind", ["uniform", "geometric", "cluster"])
@pytest.mark.parametrize("n", [16, 48])
def test_constructed_spectra_plain(n, kind):
    A, lam = synth.sym_matrix(n, kind, seed=synth.seed_for(0, n))
    L, V, st, rc = oracle.syevj_plain(A)
    assert rc == 0
    a2 = np.abs(lam).max()
    build_err = 4 * n * U * a2        # fl(Q diag(lam) Q^T) differs from an exact similarity
    assert np.abs(L - lam).max() <= 10 * n * U * a2 + build_err
    assert np.linalg.norm(A @ V - V * L) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 20 * n * U
    # second opinion from LAPACK
    assert np.abs(L - np.linalg.eigvalsh(A)).max() <= 10 * n * U * a2


def test_sweep_invariants_trace_and_frobenius():
    n = 24
    A, lam = synth.sym_matrix(n, "uniform", seed=7)
    T, P = A.copy(order="F"), np.eye(n)
    tr0, f0 = np.trace(A), np.linalg.norm(A)
    for _ in range(4):
        r = oracle.syev_cyclic(T, P, tol=0.0, max_sweeps=1)
        T, P = r["T"], r["P"]
        assert np.trace(T) == pytest.approx(tr0, abs=10 * n * U * f0)
        assert np.linalg.norm(T) == pytest.approx(f0, rel=10 * n * U)
        # P^T A P reproduces the iterate (the rotations are accumulated consistently)
        assert np.abs(P.T @ A @ P - T).max() <= 50 * n * U * f0


def test_quadratic_convergence_of_sweeps():
    """Once ||off|| is small the sweep-to-sweep decay is quadratic (Thms 3.9/3.10)."""
    n = 40
    A, lam = synth.sym_matrix(n, "uniform", seed=11)
    r = oracle.syev_cyclic(A, tol=0.0, max_sweeps=12, history=True)
    h = r["off_history"] / np.linalg.norm(A)
    seen = 0
    for k in range(len(h) - 1):
        if 1e-13 < h[k + 1] and h[k] < 1e-3:
            assert h[k + 1] <= 50 * h[k] ** 2 / 1e-3 * 1e-3 + 1e-15 or h[k + 1] <= h[k] ** 1.5
            seen += 1
    assert seen >= 1


def test_planted_mistake_is_caught(tmp_path):
    """A sign error in the row update of the oracle must fail the explicit-J pin."""
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    bad = src.replace("double bqj = s * apj + c * aqj;", "double bqj = s * apj - c * aqj;", 1)
    assert bad != src
    c_file = tmp_path / "bad.c"; so = tmp_path / "bad.so"
    c_file.write_text(bad)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", str(c_file),
                           "-o", str(so), "-lm"])
    lib = ctypes.CDLL(str(so))
    n, p, q = 5, 1, 3
    rng = np.random.default_rng(0)
    G = rng.standard_normal((n, n)); A = np.asfortranarray(G + G.T)
    B = A.copy(order="F"); P = np.asfortranarray(np.eye(n))
    lib.orc_jacobi_step(ctypes.c_void_p(B.ctypes.data), ctypes.c_void_p(P.ctypes.data),
                        ctypes.c_int(n), ctypes.c_int(p), ctypes.c_int(q))
    c, s = oracle.rotation(A[p, p], A[q, q], A[p, q])
    J = _explicit_J(n, p, q, c, s)
    ref = J.T @ A @ J
    ref[p, q] = ref[q, p] = 0
    assert np.abs(B - ref).max() > 1e-3


def test_alg41_preconditioned_stagewise():
    n = 64
    A, lam = synth.sym_matrix(n, "uniform", seed=synth.seed_for(0, 0))
    L, V, st, rc, Q, T0 = oracle.syevj_mp(A, intermediates=True)
    assert rc == 0
    normA = np.linalg.norm(A, 2)
    # Q from MGS is orthogonal to double precision (Lemma 2.1 with kappa(Z) ~ 1)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 10 * n * U
    # ||off(T0)||_F <= 10 bd, bd = n ||A|| upsilon (Sec. 6, Fig. 6.1)
    assert oracle.offnorm(T0) <= 10 * n * normA * UPS
    # a handful of sweeps (Tables 6.1/6.3/6.4 report 1-6)
    assert 1 <= st["sweeps"] <= 6
    assert np.abs(L - lam).max() <= 10 * n * U * normA + 4 * n * U * normA
    assert np.linalg.norm(A @ V - V * L) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 10 * n * U


def test_stage1_quality():
    """Step 1 (single precision Jacobi) meets Lemma 2.2's form ||E|| <= p(n)||A|| upsilon.

    Table 6.2 reports init-Res = ||A Z - Z Phi||_F/||A||_F of 1e-6..3e-6 at n = 2048 for
    LAPACK's single precision solver, i.e. p(n) ~ n/8; the scalar Jacobi of the oracle
    is pinned to p(n) <= 10 n.  Lemma 4.1's ||Z - Q||_F and r_ss = 1 + O(upsilon) are
    checked against the first-order relation R - I ~ triu(Z^T Z - I) of a QR of a
    nearly orthonormal Z.
    """
    n = 128
    A, lam = synth.sym_matrix(n, "mode4", seed=5, kappa=1e3)
    Z, D, st = oracle.stage1_syev_f(A)
    init_res = np.linalg.norm(A @ Z - Z * D) / np.linalg.norm(A)
    assert UPS < init_res < 10 * n * UPS
    Q, R, rc = oracle.mgs(Z)
    assert rc == 0
    G = Z.T @ Z - np.eye(n)
    assert np.linalg.norm(G) < 1e-2
    assert np.linalg.norm(Z - Q) <= 2 * np.linalg.norm(G) + 10 * n * U
    assert np.abs(np.diag(R) - 1).max() <= np.abs(np.diag(G)).max() + 10 * n * U
    # init-OR-Q = ||Q^T Q - I||_F / sqrt(n) of order 1e-15 (Table 6.2)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) / np.sqrt(n) < 1e-14


# ------------------------------------------------------------------ MGS (Lemma 2.1)
def test_mgs_golden():
    rows = {r[0]: np.array([float(x) for x in r[1:]]) for r in _rows("mgs_small.txt")}
    Z = rows["Z"].reshape(2, 2, order="F")
    Q, R, rc = oracle.mgs(Z)
    assert rc == 0
    assert np.abs(Q - rows["Q"].reshape(2, 2, order="F")).max() <= 4 * U
    assert np.abs(R - rows["R"].reshape(2, 2, order="F")).max() <= 8 * U


@pytest.mark.parametrize("m,n", [(30, 30), (50, 20), (7, 1)])
def test_mgs_against_householder_qr(m, n):
    rng = np.random.default_rng(m * 100 + n)
    Z = rng.standard_normal((m, n))
    Q, R, rc = oracle.mgs(Z)
    assert rc == 0
    assert np.allclose(np.triu(R), R) and (np.diag(R) > 0).all()
    assert np.linalg.norm(Z - Q @ R) <= 10 * n * U * np.linalg.norm(Z)
    kappa = np.linalg.cond(Z)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 10 * n * U * kappa
    Qh, Rh = np.linalg.qr(Z)
    sg = np.sign(np.diag(Rh))
    assert np.abs(Q - Qh * sg).max() <= 100 * n * U * kappa


def test_mgs_rank_deficient_status():
    Z = np.zeros((4, 3)); Z[:, 0] = 1.0; Z[:, 1] = 2.0; Z[:, 2] = [1, 2, 3, 4]
    Q, R, rc = oracle.mgs(Z)
    assert rc == 4


# ------------------------------------------------------------------ congruence (step 3)
def test_congruence_bound_extended_precision():
    n = 20
    A, _ = synth.sym_matrix(n, "uniform", seed=3)
    Q = synth.haar(synth.rng_for(4), n)
    T = oracle.congruence(A, Q)
    assert np.array_equal(T, T.T)
    Al, Ql = A.astype(np.longdouble), Q.astype(np.longdouble)
    Tx = Ql.T @ (Al @ Ql)
    gn = n * U / (1 - n * U)
    bound = gn * (2 + gn) * (np.abs(Q).T @ np.abs(A) @ np.abs(Q))
    assert (np.abs(T - Tx.astype(np.float64)) <= bound + 1e-300).all()


def test_congruence_identity_is_exact():
    A, _ = synth.sym_matrix(12, "geometric", seed=9)
    T = oracle.congruence(A, np.eye(12))
    assert np.array_equal(T, np.triu(A) + np.triu(A, 1).T)


# ------------------------------------------------------------------ one-sided Jacobi (Sec. 5)
def test_one_sided_rotation_orthogonalises_pair():
    """Lemma 5.1: after one rotation of columns i, j their inner product vanishes."""
    rng = np.random.default_rng(21)
    C = rng.standard_normal((30, 2))
    r = oracle.gesvj_cyclic(C, max_sweeps=1, ju_ratio=0.0)
    Cn = r["C"]
    assert abs(Cn[:, 0] @ Cn[:, 1]) <= 64 * U * np.linalg.norm(C) ** 2
    assert np.linalg.norm(Cn) == pytest.approx(np.linalg.norm(C), rel=16 * U)
    # the same J applied to V: C_new = C V
    assert np.abs(C @ r["V"] - Cn).max() <= 64 * U * np.abs(C).max()


@pytest.mark.parametrize("mp", [False, True])
def test_svd_constructed(mp):
    m, n = 48, 24
    A, sig, Uc, Vc = synth.svd_matrix(m, n, seed=2, sigma_min=1e-6)
    f = oracle.gesvj_mp if mp else oracle.gesvj_plain
    S, Uo, Vo, st, rc = f(A)
    assert rc == 0
    assert (np.diff(S) <= 0).all()
    assert np.abs(S - sig).max() <= 10 * n * U * sig[0] + 4 * n * U * sig[0]
    assert np.linalg.norm(A @ Vo - Uo * S) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(Vo.T @ Vo - np.eye(n)) <= 10 * n * U
    assert np.linalg.norm(Uo.T @ Uo - np.eye(n)) <= 10 * n * U
    # second opinion from LAPACK
    assert np.abs(S - np.linalg.svd(A, compute_uv=False)).max() <= 10 * n * U * sig[0]
    if mp:
        assert st["sweeps"] <= 6


def test_stage1_gesvj_f_alone():
    """Step 1 of Alg. 5.2 in the oracle, pinned on its own: Z orthogonal to the
    single precision level, its columns ordered by decreasing ||fl32(A) z_j||, and
    each z_j the right singular vector LAPACK gives for sigma_j, up to sign and to
    the single precision accuracy that the gap to the neighbouring singular values
    allows (a transposed Z or a wrong column order fails these)."""
    m, n = 60, 24
    A, sig, _, _ = synth.svd_matrix(m, n, seed=31, sigma_min=1e-2)
    Z, st = oracle.stage1_gesvj_f(A)
    assert st["sweeps_stage1"] >= 1
    assert np.linalg.norm(Z.T @ Z - np.eye(n)) <= 10 * n * UPS
    A32 = A.astype(np.float32).astype(np.float64)
    norms = np.linalg.norm(A32 @ Z, axis=0)
    assert (np.diff(norms) <= 4 * UPS * norms[0]).all()
    _, s, Vt = np.linalg.svd(A)
    gaps = np.minimum(np.abs(np.diff(s, prepend=np.inf)), np.abs(np.diff(s, append=-np.inf)))
    for j in range(n):
        v = Vt[j]
        zj = Z[:, j] * np.sign(Z[:, j] @ v)
        assert np.abs(zj - v).max() <= 100 * UPS * s[0] / gaps[j], j
