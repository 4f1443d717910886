"""CPU tests of host-side logic: the multi-rank timing reduction of bench.py
(world_size 2 over gloo, the replica path of --gpus N), the autotuner's cache
key and candidate set, and argument checks of the batched plan."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    out[rank] = v
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == 15.0 and out[1] == 15.0


def test_max_over_ranks_single():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_autotune_key_and_candidates():
    from paper_2211_03339_gb300 import autotune
    ns = [8, 20, 40, 100, 200, 256] * 10
    k1 = autotune._key(ns, "mp")
    k2 = autotune._key(list(reversed(ns)), "mp")
    assert k1 == k2 and k1.startswith("mp:")
    assert autotune._key(ns, "plain") != k1
    assert len(autotune.CANDIDATES) == 8
    assert {c["block_large"] for c in autotune.CANDIDATES} == {16, 32}


def test_batched_plan_rejects_bad_sizes_on_host():
    import ctypes
    from paper_2211_03339_gb300 import build
    build.build()
    import paper_2211_03339_gb300 as m
    L = m.lib()
    h = ctypes.c_void_p()
    for sizes in ([10, 257], [0, 4]):
        arr = (ctypes.c_int * len(sizes))(*sizes)
        rc = L.mpj_batch_plan_create(ctypes.cast(arr, ctypes.c_void_p), len(sizes), 1, None,
                                     ctypes.byref(h))
        assert rc == 1
    arr = (ctypes.c_int * 1)(5)
    assert L.mpj_batch_plan_create(ctypes.cast(arr, ctypes.c_void_p), 1, 7, None, ctypes.byref(h)) == 1


def test_synth_batch_sizes_range_and_seed():
    from paper_2211_03339_gb300 import synth
    a = synth.batch_sizes(10000, 8, 256, seed=3000)
    b = synth.batch_sizes(10000, 8, 256, seed=3000)
    assert np.array_equal(a, b) and a.min() >= 8 and a.max() <= 256


@pytest.mark.parametrize("n", [512, 1024, 1280, 4096])
def test_alg_counts_closed_forms(n):
    """bench.alg_counts follows the library's schedule; its totals must equal the
    method's own counts: MGS 2 n^3 (column MGS inside 32-column panels, their
    projections and updates, and for n >= 1024 the exactly split projections
    between 256-column panels), the congruence 2 n^3 + n^2 (n + 1) on the tensor
    cores (A Q in full, Q^T W on the upper triangle), and 3 n^3 per FP64 sweep for T."""
    import bench
    c, realised = bench.alg_counts(n, 2, 11)
    oz_fp64 = c["oz_gemm"] / 36.0
    congruence = 2.0 * n ** 3 + n * n * (n + 1)
    mgs_fp64 = c["mgs_panel"] + c["mgs_proj"] + c["dgemm_f64"] + (oz_fp64 - congruence)
    assert mgs_fp64 == pytest.approx(2.0 * n ** 3, rel=1e-12)
    if n < 1024:
        assert oz_fp64 == pytest.approx(congruence, rel=1e-12)
    assert c["apply2_f64"] == 2 * 3.0 * n ** 3
    Np = -(-n // 64) * 64
    assert realised["apply2_f64"] == 2 * 4.0 * Np ** 3
    # one-pass tile update: the off-diagonal tiles (K (K - 1) / 2 of 64 x 64 FP32)
    # read once and written twice per round
    K = Np // 64
    assert c["tile_f32"] == K * (K - 1) / 2 * 3 * 64 * 64 * 4 * (Np // 32 - 1) * 11


def test_library_reads_no_environment():
    """Every switch of the numerical path is an mpj_options field: the library's
    sources call no getenv, so a default C-ABI call cannot change path with the
    caller's environment."""
    import glob
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2211_03339_gb300", "csrc")
    files = glob.glob(os.path.join(root, "*.cu")) + glob.glob(os.path.join(root, "*.cuh")) + \
        glob.glob(os.path.join(root, "*.h"))
    assert files
    for f in files:
        assert "getenv" not in open(f).read(), f


def test_options_mirror_matches_header():
    """The Python mirror of mpj_options has the header's fields in the header's
    order, and the OPT_* constants have the header's values."""
    import re
    import paper_2211_03339_gb300 as m
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "mpjacobi.h")).read()
    body = hdr[hdr.index("typedef struct mpj_options {"):hdr.index("} mpj_options;")]
    fields = re.findall(r"^\s+(?:int|double)\s+(\w+);", body, re.M)
    assert fields == [f for f, _ in m.Options._fields_]
    for name, val in re.findall(r"#define MPJ_(OPT_\w+)\s+(\d+)", hdr):
        assert getattr(m, name) == int(val), name
