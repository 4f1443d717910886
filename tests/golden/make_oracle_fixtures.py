"""Write the oracle's results for the GPU parity cases whose oracle run takes
minutes (n = 512 and 1024): the plain FP64 Jacobi eigenvalues (Algorithm 3.2,
oracle.syevj_plain), the FP32 step-1 eigenvalues (oracle.stage1_syev_f) and the
singular values of the one-sided Jacobi SVD (Algorithm 5.1, oracle.gesvj_plain).

Only oracle/ and the seeded input generators (paper_2211_03339_gb300.synth, no
arithmetic of the method) are called; nothing comes from the CUDA path.  The
inputs are regenerated from the same seeds by the tests.

    python tests/golden/make_oracle_fixtures.py      # about 10 minutes on 8 cores
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# (file name, kind, arguments): the tests build the same inputs from these seeds
CASES = [("oracle_eig_n1024_%s.txt" % k, "eig", ("sym", 1024, k, 1000 + 1024)) for k in
         ("uniform", "geometric", "cluster")]
CASES += [("oracle_stage1_n1024_uniform.txt", "stage1", ("sym", 1024, "uniform", 500 + 1024))]
CASES += [("oracle_eig_n512_multiple_mode%d.txt" % m, "eig", ("multiple", 4, 128, m, 1e4, 4000 + m))
          for m in (1, 2, 3, 4, 5)]
CASES += [("oracle_svd_1300x1100.txt", "svd", ("svd", 1300, 1100, 1e-10, 2000 + 1100))]
ONLY = sys.argv[1:]        # optional file names: write only these


def make_input(spec):
    from paper_2211_03339_gb300 import synth
    if spec[0] == "sym":
        _, n, kind, seed = spec
        return synth.sym_matrix(n, kind, seed=seed)[0]
    if spec[0] == "svd":
        _, m, n, smin, seed = spec
        return synth.svd_matrix(m, n, seed=seed, sigma_min=smin)[0]
    _, r, s, mode, kappa, seed = spec
    return synth.sym_matrix_multiple(r, s, mode, kappa=kappa, seed=seed)[0]


def run(case):
    import numpy as np
    import oracle
    name, what, spec = case
    A = make_input(spec)
    if what == "eig":
        L, V, st, rc = oracle.syevj_plain(A)
        assert rc == 0
        vals = np.asarray(L)
        head = "# oracle.syevj_plain eigenvalues (ascending), %s, sweeps %d" % (spec, st["sweeps"])
    elif what == "svd":
        S, Uo, Vo, st, rc = oracle.gesvj_plain(A)
        assert rc == 0
        vals = np.asarray(S)
        head = "# oracle.gesvj_plain singular values (descending), %s, sweeps %d" % (spec, st["sweeps"])
    else:
        Z, D, st = oracle.stage1_syev_f(A)
        vals = np.asarray(D)
        head = "# oracle.stage1_syev_f FP32 eigenvalues (in the order of Z), %s" % (spec,)
    with open(os.path.join(HERE, name), "w") as f:
        f.write(head + "\n")
        for i in range(0, len(vals), 4):
            f.write(" ".join("%.17g" % v for v in vals[i:i + 4]) + "\n")
    return name


if __name__ == "__main__":
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(min(len(CASES), os.cpu_count() or 1)) as pool:
        cases = [c for c in CASES if not ONLY or c[0] in ONLY]
        for name in pool.imap_unordered(run, cases):
            print("wrote", name, flush=True)
