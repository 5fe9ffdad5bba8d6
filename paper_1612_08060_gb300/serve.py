"""Continuous-batching request server for node-aware SpMV and CG-IR solves.

Requests (an SpMV, or a CG solve to ||b - A x|| <= rtol ||b|| with FP32-stored
values inside FP64 iterative refinement) arrive over time on matrices of
differing size: Poisson matrices named by a generator spec (``dim``, ``side``)
or the caller's own CSR (``matrix``, with ``n_p``, ``ppn`` and an optional
cache ``key``) and right-hand side (``rhs``).  The server:

* admits an arrived request when a slot is free (at most ``max_active`` in
  flight) and its device memory fits the budget; plans (built on first use, with
  the autotuner's cached launch options for that matrix when a tuning cache is
  given) stay resident in an LRU cache, evicted only when unused and memory is
  short;
* keeps the admitted requests on matrices of fewer than ``SOLO_NNZ`` stored
  entries in two groups served in turn: while the GPU runs one group's step,
  the host reads the other group's scalars (one device-to-host copy per step,
  awaited on its own event), retires what finished and queues that group's next
  step, so the device never idles on a host decision;
* a step of those groups launches one batched fused apply for the group's SpMV
  requests, one batched CG-residual step (FP64 values) for the solves entering
  an outer iteration and ``iters_per_step`` batched CG iterations (FP32 values)
  for the solves in their inner loop;
* keeps the requests on larger matrices in a third group on a second stream,
  with their products on the phased engine and ``solo_iters_per_step`` CG
  iterations per step.  That group steps on its own: the host polls its event
  and neither kind of request waits for the other's steps.  A large 2D solve
  needs thousands of CG iterations, and with 8 per step its host round trips,
  not its arithmetic, set the slowest latencies.

Each request's arithmetic is independent of what else is in flight: a fixed
engine per request (the fused engine with its own plan's options, or the phased
engine on a large matrix), a fixed number of CG iterations per step (by its
matrix's size), fixed per-row and per-slot reduction orders and the same
sequence of steps whatever its group holds, so a request served alone and in a
mix gives the same bits.  ``max_active=1`` is the plain per-request loop
(same kernels, same plan cache, one request at a time in arrival order).

PyTorch provides device memory and the streams; all compute is in libnapspmv.
"""
from __future__ import annotations

import collections
import hashlib
import math
import time

import numpy as np
import torch

from . import autotune, inputs
from . import napspmv as nap


class Matrix:
    def __init__(self, key, A, n_p, ppn):
        t0 = time.perf_counter()
        self.key = key
        self.n = A.n
        self.solo = A.nnz >= nap.SOLO_NNZ
        self.plan = nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, nap.F32_VALUES)
        self.build_s = time.perf_counter() - t0
        st = nap.napspmv_plan_stats(self.plan)
        bufs = st["bll_total"] + st["lbuf_total"] + 2 * st["nap_inter_vals"] + st["bnl_total"]
        # matrix (col, values FP64 + FP32, row pointer) + index arrays + one
        # workspace (receive buffers, chain vector, two FP32 vector copies)
        self.plan_bytes = A.nnz * 16 + A.n * 12 + bufs * 12 + 16 * A.n
        self.ws_bytes = bufs * 8 + A.n * 16
        self.users = 0


class Request:
    def __init__(self, spec):
        self.spec = spec
        self.id = spec["id"]
        self.arrival = spec["arrival"]
        self.kind = spec["kind"]
        self.state = "queued"
        self.t_done = None
        self.outer = 0
        self.inner = 0
        self.result = None


SOLO = 2  # group of the requests on large matrices


class Server:
    def __init__(self, mem_budget=None, max_active=64, iters_per_step=8,
                 solo_iters_per_step=64, rtol=1e-10,
                 inner_rtol=1e-4, max_outer=40, max_inner=200000, device=None, keep_results=False,
                 cache=None, tune_cache=None):
        self.dev = torch.device(device or "cuda")
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = int(mem_budget if mem_budget else 0.5 * free)
        self.max_active = max_active
        self.iters = iters_per_step
        self.solo_iters = solo_iters_per_step
        self.rtol, self.inner_rtol = rtol, inner_rtol
        self.max_outer, self.max_inner = max_outer, max_inner
        self.keep = keep_results
        self.stream = torch.cuda.Stream(self.dev)       # fused launches and CG kernels
        self.solo_stream = torch.cuda.Stream(self.dev)  # products on large matrices
        self.solo_opts = nap.make_opts(engine=nap.ENGINE_PHASED)
        # unset fields: each plan's own defaults (one launch per option set)
        self.fused_opts = nap.make_opts(engine=nap.ENGINE_FUSED)
        self.tune_cache = tune_cache
        self.hbuf = [torch.zeros(max_active, 2, 8, dtype=torch.float64).pin_memory()
                     for _ in range(3)]
        # plans may be shared between servers (a warm cache): their bytes are
        # then counted by whoever built them
        self.cache: "collections.OrderedDict[str, Matrix]" = (
            cache if cache is not None else collections.OrderedDict())
        self.mem_used = 0
        self.steps = 0
        self.batch_sizes = []

    # ------------------------------------------------------------ matrices
    @staticmethod
    def _key(spec):
        if "matrix" in spec:
            if spec.get("key"):
                return f"user_{spec['key']}_np{spec['n_p']}_ppn{spec['ppn']}"
            A = spec["matrix"]
            h = hashlib.sha256()
            for arr in (A.row_ptr, A.col, A.val):
                h.update(np.ascontiguousarray(arr).tobytes())
            return f"user_{h.hexdigest()[:24]}_np{spec['n_p']}_ppn{spec['ppn']}"
        return f"{spec['dim']}d_{spec['side']}_np{spec['n_p']}_ppn{spec['ppn']}"

    def _matrix(self, spec):
        key = self._key(spec)
        if key in self.cache:
            self.cache.move_to_end(key)
            return self.cache[key]
        if "matrix" in spec:
            A = spec["matrix"]
        else:
            A = inputs.poisson2d(spec["side"]) if spec["dim"] == 2 else inputs.poisson3d(spec["side"])
        with torch.cuda.stream(self.stream):
            m = Matrix(key, A, spec["n_p"], spec["ppn"])
            if self.tune_cache:
                autotune.apply_cached(m.plan, A.row_ptr, nap.PREC_F64, cache_file=self.tune_cache)
        self.cache[key] = m
        self.mem_used += m.plan_bytes
        return m

    def _evict(self, need):
        for key in list(self.cache):
            if self.mem_used + need <= self.budget:
                return
            m = self.cache[key]
            if m.users == 0:
                self.mem_used -= m.plan_bytes
                del self.cache[key]

    def _request_bytes(self, spec, m):
        vecs = 2 if spec["kind"] == "spmv" else 9
        return vecs * 8 * m.n + m.ws_bytes

    # ------------------------------------------------------------ admission
    def _admit(self, r):
        spec = r.spec
        m = self._matrix(spec)
        need = self._request_bytes(spec, m)
        if self.mem_used + need > self.budget:
            self._evict(need)
            if self.mem_used + need > self.budget:
                return False
        r.m = m
        m.users += 1
        r.bytes = need
        self.mem_used += need
        n = m.n
        d = self.dev
        # the request's buffers live on the stream its steps run on
        with torch.cuda.stream(self.solo_stream if m.solo else self.stream):
            r.ws = nap.Workspace(m.plan)
            host_rhs = spec["rhs"] if "rhs" in spec else inputs.vector(n, spec["seed"])
            rhs = torch.from_numpy(np.ascontiguousarray(host_rhs, np.float64)).to(d, non_blocking=True)
            if r.kind == "spmv":
                r.v = rhs
                r.w = torch.empty(n, dtype=torch.float64, device=d)
                r.state = "spmv"
            else:
                r.b = rhs
                z = lambda: torch.zeros(n, dtype=torch.float64, device=d)  # noqa: E731
                r.x, r.ro, r.po, r.qo = z(), z(), z(), z()
                r.d, r.ri, r.pi, r.qi = z(), z(), z(), z()
                r.scal = torch.zeros(2, 8, dtype=torch.float64, device=d)
                r.outer_slot = dict(plan=m.plan, ws=r.ws, b=r.b, x=r.x, r=r.ro, p=r.po, q=r.qo,
                                    scal=r.scal[0])
                r.inner_slot = dict(plan=m.plan, ws=r.ws, b=r.ro, x=r.d, r=r.ri, p=r.pi, q=r.qi,
                                    scal=r.scal[1])
                r.state = "outer"
        return True

    def _retire(self, r, now):
        r.t_done = now
        r.state = "done"
        if self.keep:
            r.result = (r.w if r.kind == "spmv" else r.x).cpu().numpy()
        r.m.users -= 1
        self.mem_used -= r.bytes
        for a in ("ws", "v", "w", "b", "x", "ro", "po", "qo", "d", "ri", "pi", "qi", "scal",
                  "outer_slot", "inner_slot"):
            if hasattr(r, a):
                delattr(r, a)

    # ------------------------------------------------------------ one step
    @staticmethod
    def _chunks(xs, k=64):
        return [xs[i:i + k] for i in range(0, len(xs), k)]

    def _stream(self, g):
        return self.solo_stream if g == SOLO else self.stream

    def _iters(self, g):
        return self.solo_iters if g == SOLO else self.iters

    def _enqueue(self, g, reqs):
        """Queue one step of a group's work on the group's stream; returns
        (event, solves whose scalars the event's copy brings back)."""
        s = self._stream(g)
        spmv = [r for r in reqs if r.state == "spmv"]
        outer = [r for r in reqs if r.state == "outer"]
        inner = [r for r in reqs if r.state == "inner"]
        self.batch_sizes.append(len(reqs))
        with torch.cuda.stream(s):
            if g == SOLO:
                # one phased-engine apply each (a batch of several would share
                # one fused launch)
                for r in spmv:
                    nap.napspmv_apply_batch([r.m.plan], [r.v], [r.w], [1], opts=self.solo_opts,
                                            ws=[r.ws], stream=s)
            else:
                for grp in self._chunks(spmv):
                    nap.napspmv_apply_batch([r.m.plan for r in grp], [r.v for r in grp],
                                            [r.w for r in grp], [1] * len(grp),
                                            opts=self.fused_opts, ws=[r.ws for r in grp], stream=s)
            for grp in self._chunks(outer):
                nap.napspmv_cg_batch_init([r.outer_slot for r in grp], nap.PREC_F64, stream=s)
            for grp in self._chunks(inner):
                nap.napspmv_cg_batch_iterate([r.inner_slot for r in grp], nap.PREC_F32,
                                             self._iters(g), stream=s)
            cg = outer + inner
            if cg:
                self.hbuf[g][:len(cg)].copy_(torch.stack([r.scal for r in cg]), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return ev, cg

    def _finish(self, g, reqs, ev, cg):
        """Wait for a group's step, retire what finished and queue the state
        transitions of its solves (before the group's next step)."""
        ev.synchronize()
        now = time.perf_counter()
        host = self.hbuf[g][:len(cg)].numpy() if cg else None
        for r in reqs:
            if r.state == "spmv":
                self._retire(r, now)
        to_inner, to_outer = [], []
        for q, r in enumerate(cg):
            sc = host[q]
            if r.state == "outer":
                rel = math.sqrt(max(sc[0][0], 0.0)) / math.sqrt(max(sc[0][5], 1e-300))
                r.relres = rel
                if rel <= self.rtol or r.outer >= self.max_outer or not math.isfinite(rel):
                    self._retire(r, now)
                else:
                    to_inner.append(r)
            else:
                r.inner += self._iters(g)
                rr, bb = sc[1][0], sc[1][5]
                if math.sqrt(max(rr, 0.0)) <= self.inner_rtol * math.sqrt(max(bb, 1e-300)) \
                        or r.inner >= self.max_inner or not math.isfinite(rr):
                    to_outer.append(r)
        s = self._stream(g)
        with torch.cuda.stream(s):
            for grp in self._chunks(to_inner):
                nap.napspmv_cg_batch_init([r.inner_slot for r in grp], nap.PREC_F32,
                                          x_is_zero=True, stream=s)
            for grp in self._chunks(to_outer):
                nap.napspmv_batch_add([r.x for r in grp], [r.d for r in grp], stream=s)
        for r in to_inner:
            r.state = "inner"
        for r in to_outer:
            r.state = "outer"
            r.outer += 1
        self.steps += 1

    @staticmethod
    def _chunks(xs, k=64):
        return [xs[i:i + k] for i in range(0, len(xs), k)]

    # ------------------------------------------------------------ driver
    def run(self, specs, realtime=True):
        """Serve `specs` (dicts from inputs.serving_requests, or caller specs
        with ``matrix`` / ``rhs``).  With realtime, request q becomes visible at
        t0 + arrival; otherwise all are queued at once.  Returns the list of
        finished Request objects."""
        reqs = [Request(s) for s in specs]
        pending = collections.deque(sorted(reqs, key=lambda r: r.arrival))
        queue: collections.deque = collections.deque()
        groups = [[], [], []]
        inflight = [None, None, None]
        t0 = time.perf_counter()
        for r in reqs:
            r.t_arrive = t0 + (r.arrival if realtime else 0.0)
        while pending or queue or any(groups):
            now = time.perf_counter()
            while pending and pending[0].t_arrive <= now:
                queue.append(pending.popleft())
            while queue and sum(len(x) for x in groups) < self.max_active:
                if not self._admit(queue[0]):
                    break
                r = queue.popleft()
                g = SOLO if r.m.solo else (0 if len(groups[0]) <= len(groups[1]) else 1)
                groups[g].append(r)
            if not any(groups):
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].t_arrive - time.perf_counter())))
                    continue
                if queue:
                    raise RuntimeError("request does not fit the memory budget")
            progress = False
            for g in (0, 1, SOLO):
                if inflight[g] is not None:
                    ev, cg, stepped = inflight[g]
                    if g == SOLO and not ev.query():
                        continue  # the large requests' step is still running
                    self._finish(g, stepped, ev, cg)
                    inflight[g] = None
                    groups[g] = [r for r in groups[g] if r.state != "done"]
                    progress = True
                if groups[g]:
                    ev, cg = self._enqueue(g, groups[g])
                    inflight[g] = (ev, cg, list(groups[g]))
                    progress = True
            if not progress:
                time.sleep(0.0002)
        return reqs


def summarize(reqs, wall_s):
    lat = np.array([r.t_done - r.t_arrive for r in reqs])
    return {"requests": len(reqs), "throughput_rps": len(reqs) / wall_s,
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}


def warm_cache(specs, device=None):
    """Build (once) the plan of every matrix the requests use."""
    srv = Server(max_active=1, device=device)
    t0 = time.perf_counter()
    for sp in specs:
        srv._matrix(sp)
    return srv.cache, time.perf_counter() - t0


def compare(count=512, n_lo=1e3, n_hi=2e5, seed=1239, load=0.8, device=None, sweep=()):
    """Continuous batching vs the plain per-request loop on the same requests.

    The plain loop's saturated throughput (all requests queued at once) sets the
    arrival rate lambda = load * throughput; both loops then serve the same
    Poisson arrivals in real time.  Plans are built beforehand and shared.
    `sweep`: further loads, each reported under "sweep" the same way."""
    base = inputs.serving_requests(count, 1.0, seed, n_lo=n_lo, n_hi=n_hi)
    cache, build_s = warm_cache(base, device)
    t0 = time.perf_counter()
    plain_sat = Server(max_active=1, cache=cache, device=device).run(base, realtime=False)
    sat_s = time.perf_counter() - t0
    # saturated throughput of the batching server: every request queued at once
    t0 = time.perf_counter()
    Server(max_active=64, cache=cache, device=device).run(base, realtime=False)
    batched_sat_s = time.perf_counter() - t0

    def at(ld):
        rate = ld * count / sat_s
        specs = inputs.serving_requests(count, rate, seed, n_lo=n_lo, n_hi=n_hi)
        res = {"load": ld, "rate_hz": rate,
               "mix": {"spmv": sum(r["kind"] == "spmv" for r in specs),
                       "cg": sum(r["kind"] == "cg" for r in specs)}}
        for name, act in (("batched", 64), ("plain", 1)):
            srv = Server(max_active=act, cache=cache, device=device)
            t1 = time.perf_counter()
            reqs = srv.run(specs, realtime=True)
            wall = time.perf_counter() - t1
            res[name] = summarize(reqs, wall)
            res[name]["mean_batch"] = float(np.mean(srv.batch_sizes)) if srv.batch_sizes else 0.0
        return res

    main = at(load)
    out = {"requests": count, "n_range": [n_lo, n_hi], "rate_hz": main["rate_hz"],
           "plan_build_s": build_s, "plain_saturated_rps": count / sat_s,
           "batched_saturated_rps": count / batched_sat_s, "mix": main["mix"],
           "tolerance": "SpMV FP64 <= 1e-13 normwise; CG-IR ||b - Ax|| / ||b|| <= 1e-10",
           "batched": main["batched"], "plain": main["plain"]}
    if sweep:
        out["sweep"] = [at(ld) for ld in sweep]
    del plain_sat
    return out
