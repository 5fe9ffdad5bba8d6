"""Launch-option autotuner for the node-aware apply.

Searches the engine (overlapped, phased, fused), lanes per row (``vec``), the
SpMV tile shape (``tile_rows``, ``tile_nnz``: the entries one shared-memory
stage holds), the pipeline depth (``stages``), CTA or warp tiles
(``pipeline``), resident CTAs per SM (``ctas_per_sm``, 0 = occupancy maximum)
and the elements per message unit of the fused engine (``chunk``) by
coordinate descent: starting from the plan's defaults, each parameter in turn
is set to each candidate while the others stay fixed, the fastest is kept, and
the sweep repeats until nothing improves.  Each candidate is timed with CUDA
events over chained applies (inputs already on the device).  The winner is
installed with napspmv_set_default_opts and cached per (N, nnz, nnz-per-row
histogram, n_p, ppn, precision) key, in memory and optionally in a JSON file.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import napspmv as nap

CANDIDATES = {
    "engine": [nap.ENGINE_OVERLAP, nap.ENGINE_PHASED, nap.ENGINE_FUSED],
    "vec": [1, 2, 4, 8],
    "tile_nnz": [1024, 1536, 2048, 3072],
    "tile_rows": [256, 384, 512, 1024],
    "stages": [2, 3],
    "pipeline": [nap.PIPELINE_SELL, nap.PIPELINE_CTA, nap.PIPELINE_WARP],
    "ctas_per_sm": [0, 2, 3, 4],
    "chunk": [2048, 4096, 8192],
}

_cache: dict = {}


def matrix_key(row_ptr, n_p, ppn, precision):
    lens = np.diff(np.asarray(row_ptr))
    hist = np.histogram(np.minimum(lens, 64), bins=[0, 2, 4, 8, 12, 16, 24, 32, 48, 65])[0]
    hist = tuple(int(round(10 * h / max(1, len(lens)))) for h in hist)
    return f"n{len(lens)}_nnz{int(lens.sum())}_h{hist}_np{n_p}_ppn{ppn}_p{precision}"


def time_opts(plan, v, w, opts, reps=20, trials=3, stream=None):
    import torch
    s = stream or torch.cuda.current_stream()
    nap.napspmv_apply_ex(plan, v, w, reps, 1.0 / 16.0, opts, stream=s)  # warm-up
    best = float("inf")
    for _ in range(trials):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        nap.napspmv_apply_ex(plan, v, w, reps, 1.0 / 16.0, opts, stream=s)
        b.record(s)
        b.synchronize()
        best = min(best, a.elapsed_time(b) / reps)
    if nap.napspmv_status(plan, s) != 0:
        return float("inf")
    return best  # ms per apply


def _load(cache_file):
    if cache_file and os.path.exists(cache_file):
        for k, v in json.load(open(cache_file)).items():
            _cache.setdefault(k, v)


def apply_cached(plan, row_ptr, precision=nap.PREC_F64, cache_file=None):
    """Install the tuned options cached for this matrix key (in memory or in
    `cache_file`) as the plan's defaults, without measuring anything; returns
    them, or None when the matrix was never tuned."""
    key = matrix_key(row_ptr, plan.n_p, plan.ppn, precision)
    if key not in _cache:
        _load(cache_file)
    if key not in _cache:
        return None
    best = dict(_cache[key]["opts"])
    nap.napspmv_set_default_opts(plan, nap.make_opts(precision=precision, **best))
    return best


def tune(plan, row_ptr, precision=nap.PREC_F64, reps=20, max_sweeps=2, cache_file=None,
         verbose=False):
    """Tune `plan` in place; returns (best options dict, ms per apply)."""
    import torch
    key = matrix_key(row_ptr, plan.n_p, plan.ppn, precision)
    if cache_file and os.path.exists(cache_file) and not _cache:
        _cache.update(json.load(open(cache_file)))
    if key in _cache:
        best = dict(_cache[key]["opts"])
        nap.napspmv_set_default_opts(plan, nap.make_opts(precision=precision, **best))
        return best, _cache[key]["ms"]
    d = nap.napspmv_get_default_opts(plan)
    cur = {k: int(getattr(d, k)) for k in CANDIDATES}
    v = torch.rand(plan.n, dtype=torch.float64, device="cuda") * 2 - 1
    w = torch.empty_like(v)

    def measure(c):
        try:
            o = nap.make_opts(precision=precision, **c)
            return time_opts(plan, v, w, o, reps=reps)
        except nap.NapError:
            return float("inf")

    best_ms = measure(cur)
    for _ in range(max_sweeps):
        improved = False
        for k, cands in CANDIDATES.items():
            for val in cands:
                if val == cur[k]:
                    continue
                trial = dict(cur, **{k: val})
                ms = measure(trial)
                if verbose:
                    print(f"  {trial} -> {ms:.4f} ms")
                if ms < best_ms * 0.99:
                    best_ms, cur, improved = ms, trial, True
        if not improved:
            break
    nap.napspmv_set_default_opts(plan, nap.make_opts(precision=precision, **cur))
    _cache[key] = {"opts": cur, "ms": best_ms}
    if cache_file:
        with open(cache_file, "w") as f:
            json.dump(_cache, f, indent=1)
    return cur, best_ms


def main(argv=None):
    """python -m paper_1612_08060_gb300.autotune --config K: tune workload K
    (see inputs.workload) and print each candidate's time and the winner."""
    import argparse

    import torch

    from . import inputs
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--scale-down", type=int, default=1)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--precision", default="f64", choices=["f64", "f32"])
    ap.add_argument("--cache", default=None)
    a = ap.parse_args(argv)
    w = inputs.workload(a.config, a.scale_down)
    A = w.build()
    plan = nap.napspmv_plan(A.row_ptr, A.col, A.val, w.n_p, w.ppn, nap.F32_VALUES)
    torch.cuda.synchronize()
    prec = nap.PREC_F32 if a.precision == "f32" else nap.PREC_F64
    best, ms = tune(plan, A.row_ptr, precision=prec, reps=a.reps, cache_file=a.cache,
                    verbose=True)
    print(json.dumps({"workload": w.name, "precision": a.precision, "best": best,
                      "ms_per_apply": ms}))


if __name__ == "__main__":
    main()
