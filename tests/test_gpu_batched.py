"""GPU parity of the batched solver (one persistent launch, n_i <= 256) against
the CPU oracle, per matrix, with the same tolerances as the single-matrix path:
||A V - V L||_F/||A||_F <= 10 n u, ||V^T V - I||_F <= 10 n u and
|l_i - l_i^oracle| <= 10 n u ||A||_2.  Sizes cover the three block sizes
(n <= 16, <= 32, <= 64 as one block pair) and the block sweeps (n > 64), with
ragged tails."""
import numpy as np
import pytest

import oracle
from paper_2211_03339_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53
SIZES = [1, 2, 3, 8, 16, 17, 31, 32, 33, 50, 63, 64, 65, 96, 100, 127, 128, 129, 160, 200, 255, 256]


@pytest.fixture(scope="module")
def mpj():
    if not torch.cuda.is_available():
        pytest.fail("gpu tests selected but no CUDA device is visible")
    from paper_2211_03339_gb300 import build
    build.build()
    import paper_2211_03339_gb300 as m
    return m


def _batch(sizes, seed0):
    mats, lams = [], []
    for i, n in enumerate(sizes):
        A, lam = synth.sym_matrix(n, "uniform", seed=synth.seed_for(3, seed0 + i))
        mats.append(A); lams.append(lam)
    return mats, lams


def _check(mats, lams, plan, Lam, V, status, check_oracle=True):
    Lh, Vh, sh = Lam.cpu().numpy(), V.cpu().numpy(), status.cpu().numpy()
    assert (sh == 0).all(), sh
    for i, (A, lam) in enumerate(zip(mats, lams)):
        n = A.shape[0]
        lo, ao = plan.l_offsets[i], plan.a_offsets[i]
        L = Lh[lo:lo + n]
        Vi = Vh[ao:ao + n * n].reshape(n, n, order="F")
        a2 = max(np.abs(lam).max(), 1e-300)
        assert (np.diff(L) >= 0).all()
        res = np.linalg.norm(A @ Vi - Vi * L) / np.linalg.norm(A)
        orth = np.linalg.norm(Vi.T @ Vi - np.eye(n))
        assert res <= 10 * n * U, (n, res)
        assert orth <= 10 * n * U, (n, orth)
        if check_oracle and n <= 160:
            Lo, Vo, st, rc = oracle.syevj_plain(A)
            assert np.abs(L - Lo).max() <= 10 * n * U * a2, n
        else:
            assert np.abs(L - lam).max() <= 14 * n * U * a2, n


@pytest.mark.parametrize("method", ["mp", "plain"])
def test_batched_parity(mpj, method):
    mats, lams = _batch(SIZES, 0)
    plan = mpj.BatchPlan([A.shape[0] for A in mats], method=method)
    Ad = torch.from_numpy(mpj.pack_symmetric(mats)).cuda()
    Lam, V, status, sweeps = plan.outputs()
    plan.run(Ad, Lam, V, status, sweeps)
    torch.cuda.synchronize()
    _check(mats, lams, plan, Lam, V, status)


def test_batched_graph_replay_and_tuning(mpj):
    sizes = list(synth.batch_sizes(40, 8, 256, seed=77))
    mats, lams = _batch(sizes, 100)
    Ad = torch.from_numpy(mpj.pack_symmetric(mats)).cuda()
    ref = None
    for tun in ({"ctas_per_sm": 2, "max_inner": 1, "block_large": 32},
                {"ctas_per_sm": 1, "max_inner": 2, "block_large": 16}):
        plan = mpj.BatchPlan(sizes, method="mp", tuning=tun)
        Lam, V, status, sweeps = plan.outputs()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            plan.run(Ad, Lam, V, status, sweeps)          # warm-up outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.run(Ad, Lam, V, status, sweeps)
        Lam.zero_(); V.zero_()
        g.replay()
        torch.cuda.synchronize()
        _check(mats, lams, plan, Lam, V, status, check_oracle=False)
        if ref is None:
            ref = Lam.clone()
        else:   # different schedules, same eigenvalues within the tolerance
            assert (ref - Lam).abs().max().item() <= 10 * 256 * U


def test_batched_rejects_bad_sizes(mpj):
    with pytest.raises(mpj.MPJError):
        mpj.BatchPlan([10, 257])
    with pytest.raises(mpj.MPJError):
        mpj.BatchPlan([0, 5])
