"""GPU tests of the differentiable batched eigendecomposition (forward by the
batched solver, backward by mpj_syev_backward_batched).

Loss (the workload's loss, read as Sum_i w_i lambda_i + ||B V[:, :n/2]||_F^2 with
Gaussian w and a 3 x n Gaussian B; the literal ||V^T B||_F^2 equals ||B||_F^2 for
every orthogonal V and has zero gradient, which is checked separately).
Checks: central finite differences (h = 1e-6) along random symmetric
directions; the closed form d(Sum w_i lambda_i)/dA = Sum w_i v_i v_i^T with the
oracle's eigenvectors; and an FP64 reference gradient from the oracle's
eigenpairs."""
import numpy as np
import pytest

import oracle
from paper_2211_03339_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpj():
    if not torch.cuda.is_available():
        pytest.fail("gpu tests selected but no CUDA device is visible")
    from paper_2211_03339_gb300 import build
    build.build()
    import paper_2211_03339_gb300 as m
    return m


def _batch(n, b, seed):
    mats = [synth.sym_matrix(n, "gapped", seed=synth.seed_for(5, seed + i))[0] for i in range(b)]
    rng = synth.rng_for(synth.seed_for(5, 999 + seed))
    w = rng.standard_normal((b, n))
    Bm = rng.standard_normal((b, 3, n))
    return np.stack(mats), w, Bm


def _loss(mpj, A, w, Bm, k):
    lam, V = mpj.eigh(A)
    return (w * lam).sum() + (torch.matmul(Bm, V[..., :, :k]) ** 2).sum()


@pytest.mark.parametrize("n,b", [(64, 6), (128, 3)])
def test_backward_finite_differences(mpj, n, b):
    A_np, w_np, B_np = _batch(n, b, 10 * n)
    A = torch.from_numpy(A_np).cuda().requires_grad_(True)
    w = torch.from_numpy(w_np).cuda()
    Bm = torch.from_numpy(B_np).cuda()
    k = n // 2
    L = _loss(mpj, A, w, Bm, k)
    (gA,) = torch.autograd.grad(L, A)
    assert torch.equal(gA, gA.transpose(-1, -2))
    rng = np.random.default_rng(n)
    h = 1e-6
    with torch.no_grad():
        for _ in range(3):
            E = rng.standard_normal((b, n, n)); E = (E + E.transpose(0, 2, 1)) / 2
            Ed = torch.from_numpy(E).cuda()
            fd = (_loss(mpj, A + h * Ed, w, Bm, k) - _loss(mpj, A - h * Ed, w, Bm, k)) / (2 * h)
            an = (gA * Ed).sum()
            assert abs(fd.item() - an.item()) <= 1e-6 * max(1.0, abs(an.item())), (fd.item(), an.item())


def test_backward_eigenvalue_part_closed_form_and_reference(mpj):
    n, b = 64, 4
    A_np, w_np, B_np = _batch(n, b, 500)
    A = torch.from_numpy(A_np).cuda().requires_grad_(True)
    w = torch.from_numpy(w_np).cuda()
    lam, V = mpj.eigh(A)
    (gA,) = torch.autograd.grad((w * lam).sum(), A)
    gA = gA.cpu().numpy()
    for i in range(b):
        Lo, Vo, st, rc = oracle.syevj_plain(A_np[i])
        ref = (Vo * w_np[i]) @ Vo.T                      # sum_j w_j v_j v_j^T
        assert np.abs(gA[i] - ref).max() <= 1e-12 * max(1.0, np.abs(w_np[i]).max())


def test_backward_against_fp64_reference_gradient(mpj):
    n, b = 128, 2
    A_np, w_np, B_np = _batch(n, b, 700)
    k = n // 2
    A = torch.from_numpy(A_np).cuda().requires_grad_(True)
    L = _loss(mpj, A, torch.from_numpy(w_np).cuda(), torch.from_numpy(B_np).cuda(), k)
    (gA,) = torch.autograd.grad(L, A)
    gA = gA.cpu().numpy()
    for i in range(b):
        lam, Vo, st, rc = oracle.syevj_plain(A_np[i])
        s = np.sign(Vo[np.argmax(np.abs(Vo), axis=0), np.arange(n)])   # loss is sign invariant
        Vo = Vo * s
        Vbar = np.zeros((n, n))
        Vbar[:, :k] = 2.0 * B_np[i].T @ (B_np[i] @ Vo[:, :k])
        G = Vo.T @ Vbar
        D = lam[None, :] - lam[:, None]
        np.fill_diagonal(D, 1.0)
        M = (G - G.T) / (2.0 * D)
        np.fill_diagonal(M, w_np[i])
        ref = Vo @ M @ Vo.T
        gap = np.min(np.diff(lam))
        assert np.abs(gA[i] - ref).max() <= 1e-12 / gap * np.abs(ref).max()


def test_literal_vtb_loss_has_zero_gradient(mpj):
    n, b = 64, 3
    A_np, w_np, B_np = _batch(n, b, 900)
    A = torch.from_numpy(A_np).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B_np).cuda().transpose(-1, -2)          # n x 3
    lam, V = mpj.eigh(A)
    L = (torch.matmul(V.transpose(-1, -2), Bt) ** 2).sum()        # = ||B||_F^2 for orthogonal V
    (gA,) = torch.autograd.grad(L, A)
    assert gA.abs().max().item() <= 1e-10 * float((Bt ** 2).sum())
