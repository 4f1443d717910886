"""Autotuner for the batched solver's schedule (mpj_batch_tuning).

The tunable choices are the number of resident CTAs per SM (1 or 2), the
block size b of the sweeps of matrices with n > 64 (16 or 32) and the number
of inner sweeps of each block-pair solve (1 or 2).  ``tune`` times every
candidate on a sample of the batch (same size distribution, the caller's own
matrices) with CUDA events, keeps the fastest, and caches the choice per
(method, size histogram) in a JSON file (``MPJ_AUTOTUNE_CACHE``, default
``~/.cache/mpjacobi_autotune.json``).
"""
from __future__ import annotations

import itertools
import json
import os

CANDIDATES = [dict(ctas_per_sm=c, block_large=b, max_inner=i)
              for c, b, i in itertools.product((2, 1), (32, 16), (1, 2))]


def _cache_path():
    return os.environ.get("MPJ_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mpjacobi_autotune.json"))


def _key(ns, method):
    import numpy as np
    hist = np.histogram(np.asarray(ns), bins=[1, 17, 33, 65, 129, 193, 257])[0]
    frac = np.round(hist / max(1, len(ns)), 2).tolist()
    return f"{method}:{frac}"


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass


def tune(mats, method="mp", sample=1000, use_cache=True, seed=0, verbose=False):
    """Return (tuning dict, {candidate: ms}) for a list of square numpy matrices."""
    import numpy as np
    import torch

    import paper_2211_03339_gb300 as mpj

    ns = [int(A.shape[0]) for A in mats]
    key = _key(ns, method)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key], {}
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(mats), size=min(sample, len(mats)), replace=False)
    sub = [mats[i] for i in idx]
    sub_ns = [ns[i] for i in idx]
    Ad = torch.from_numpy(mpj.pack_symmetric(sub)).cuda()
    timings = {}
    for cand in CANDIDATES:
        plan = mpj.BatchPlan(sub_ns, method=method, tuning=cand)
        Lam, V, st, sw = plan.outputs()
        plan.run(Ad, Lam, V, st, sw)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.run(Ad, Lam, V, st, sw)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if int((st != 0).sum().item()) != 0:
            ms = float("inf")                 # a schedule that fails to converge is not eligible
        timings[json.dumps(cand, sort_keys=True)] = ms
        if verbose:
            print(f"autotune {method} {cand}: {ms:.1f} ms")
    best = json.loads(min(timings, key=timings.get))
    cache[key] = best
    if use_cache:
        _store(cache)
    return best, timings
