"""Benchmark of the node-aware SpMV apply on one GB300 (or N replicas).

Workload (default): the 2^23-row banded random matrix (N = 8,388,608, about 1.68e8
stored entries: Poisson(20) entries per row clipped to [4, 64], 80% of the
off-diagonals within +-0.5% of N of the diagonal, 20% uniform), FP64 CSR,
n_p = 8192 simulated processes, ppn = 32 (256 simulated nodes); one step = 10
chained applies x <- s A x (s the power of two at or above the largest row sum of
|A|), captured once into a CUDA graph and replayed.  Metric: algorithmic GB/s of
the apply (plain-SpMV stream plus every value moved by the node-aware message
steps), as a fraction of measured HBM bandwidth; beside it, the 3D 7-point
128^3 workload (100 chained applies per step), the same 2^23-row workload with
FP32-stored values, and the request server against the plain per-request loop.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica on its own GPU (the path is
simulated on one GPU and has no exchange between GPUs): value = all replicas'
bytes / max-over-ranks time.  ``--impl reference`` times the CPU oracle (plain
FP64 CSR SpMV) on the host cores instead, one apply per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NAPSpMV GB/s (% of HBM peak); served p50/p99 vs plain loop at stated rel err"
NOMINAL_GBS = 8000.0  # GB300 HBM3e nominal bandwidth, beside the measured copy peak
DEFAULT_REPS = {1: 100, 2: 100, 3: 20, 4: 10}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device=None):
    """Max of a float over all ranks of the default process group (the identity
    without one).  Works with nccl (CUDA tensor) and gloo (CPU tensor)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = device if (device is not None and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size, bytes_per_apply, reps, steps, max_ms):
    """Whole-job GB/s: every replica's bytes over the slowest rank's time."""
    return world_size * bytes_per_apply * reps * steps / (max_ms * 1e-3) / 1e9


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_hash():
    """Hash of the apply sources with comments and blank space removed: the
    committed ncu traffic counts only while the code they measured is unchanged."""
    import re
    h = hashlib.sha256()
    for f in ("apply.cu", "internal.h"):
        src = open(os.path.join(ROOT, "paper_1612_08060_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_record(workload, what):
    """An ncu DRAM-traffic record committed under profiles/ for this workload and
    launch configuration, if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d.get("records", {}).get(f"{workload}|{what}")


# kernels of an apply and of the SpMV step, as ncu names them
_APPLY_KERNELS = re.compile(r"k_gather2|k_pack|k_transfer|k_unpack|k_spmv|k_to_f32|k_fused")


def ncu_launches(csv_path):
    """Per-launch metrics of an `ncu --csv` log: [(kernel name, {metric: value})]
    in launch order."""
    import csv
    lines = [ln for ln in open(csv_path) if not ln.startswith("==")]
    rows = list(csv.reader(lines))
    hdr = rows[0]
    i_id, i_name = hdr.index("ID"), hdr.index("Kernel Name")
    i_met, i_val = hdr.index("Metric Name"), hdr.index("Metric Value")
    per = {}
    for r in rows[1:]:
        if len(r) <= i_val:
            continue
        per.setdefault((int(r[i_id]), r[i_name]), {})[r[i_met]] = float(r[i_val].replace(",", ""))
    return [(name, m) for (_, name), m in sorted(per.items())]


def ncu_summary(csv_path, nsteps=2, per_step=1):
    """DRAM record of one `--profile-spmv nsteps` run: the kernels after the
    last plan-build kernel are one apply, then nsteps SpMV steps of per_step
    launches each (FP32 values: the FP32 copy of x, then the SpMV)."""
    items = []
    for name, m in ncu_launches(csv_path):
        short = name.split("(")[0].replace("void ", "").replace("nap::", "")
        items.append((short.replace("<unnamed>::", ""), m))
    first = max(j for j, (n, _) in enumerate(items) if not _APPLY_KERNELS.search(n))
    rest = items[first + 1:]
    steps, apply_ = rest[len(rest) - nsteps * per_step:], rest[:len(rest) - nsteps * per_step]
    b = lambda m: m.get("dram__bytes_read.sum", 0) + m.get("dram__bytes_write.sum", 0)  # noqa: E731
    t = lambda m: m.get("gpu__time_duration.sum", 0) / 1e3  # noqa: E731
    return {
        "apply_bytes": sum(b(m) for _, m in apply_),
        "apply_us_serialised": round(sum(t(m) for _, m in apply_), 2),
        "per_kernel": [{"kernel": n, "dram_read": m.get("dram__bytes_read.sum"),
                        "dram_write": m.get("dram__bytes_write.sum"), "us": round(t(m), 2)}
                       for n, m in apply_],
        "spmv_step_bytes": sum(b(m) for _, m in steps) / nsteps,
        "spmv_step_kernels": [n for n, _ in steps[:per_step]],
        "spmv_step_us": round(sum(t(m) for _, m in steps) / nsteps, 2),
    }


def write_ncu_records(pairs, out_path):
    """profiles/dram_traffic.json from `workload|precision|engine|pipeline=csv`
    pairs, stamped with the current kernel-source hash."""
    out = {"kernel_hash": kernel_hash(), "records": {}}
    for arg in pairs:
        key, path = arg.split("=", 1)
        out["records"][key] = ncu_summary(path, per_step=2 if "|f32|" in key else 1)
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
    return out


def build_workload(cfg, rows=0):
    """Workload `cfg` (inputs.workload).  rows > 0 with cfg 4: the banded random
    structure at that many rows, with the 2^23-row workload's absolute band
    (+-41,943 columns), 1,024 rows per process and ppn 32 (a smaller case of the
    same kernels, for profiling)."""
    from paper_1612_08060_gb300 import inputs
    if rows and cfg == 4:
        band = 41943.0 / rows
        w = inputs.Workload(f"banded_random_N{rows}_band41943_np{rows // 1024}_ppn32",
                            max(1, rows // 1024), 32, 1238,
                            lambda: inputs.banded_random(rows, 1238, band=band))
    else:
        w = inputs.workload(cfg)
    A = w.build()
    v = inputs.vector(A.n, w.seed)
    return w, A, v


def chain_scale(A):
    """The power of two at or above the largest row sum of |A|, inverted: chained
    applies x <- s A x stay bounded and the scaling is exact."""
    rs = np.add.reduceat(np.abs(A.val), A.row_ptr[:-1][np.diff(A.row_ptr) > 0])
    mx = float(rs.max()) if len(rs) else 1.0
    return 2.0 ** -math.ceil(math.log2(max(mx, 1.0)))


def bytes_per_apply(A, st):
    n, nnz = A.n, A.nnz
    b_csr = 4.0 * (n + 1) + nnz * 12.0 + 16.0 * n
    b_msg = 20.0 * (st["bll_total"] + st["lbuf_total"] + 2 * st["nap_inter_vals"] +
                    st["bnl_total"])
    return b_csr + b_msg


def oracle_stats(A, w):
    """The oracle's plan statistics of this workload: the stored table written by
    oracle/workload_stats.py when its fingerprint matches, else a fresh oracle
    plan (minutes for the 2^23-row workload)."""
    import oracle
    from oracle import workload_stats
    rec = workload_stats.lookup(A.row_ptr, A.col, w.n_p, w.ppn)
    if rec is not None:
        return rec["stats"], rec.get("oracle_plan_s"), "stored (oracle/workload_stats.json)"
    t0 = time.perf_counter()
    st = oracle.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn).stats()
    return st, time.perf_counter() - t0, "built"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleThreads:
    """The oracle's plain SpMV run unchanged on every host core: the rows are cut
    into one block of about equal stored entries per thread, and each thread
    calls the oracle on its block (the foreign call releases the GIL)."""

    def __init__(self, A, threads):
        from concurrent.futures import ThreadPoolExecutor
        rp = np.asarray(A.row_ptr)
        cuts = np.searchsorted(rp, np.linspace(0, rp[-1], threads + 1), side="left")
        cuts = np.clip(cuts, 0, A.n)
        cuts[0], cuts[-1] = 0, A.n
        self.blocks = [(a, b, rp[a:b + 1] - rp[a], A.col[rp[a]:rp[b]], A.val[rp[a]:rp[b]])
                       for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        self.n = A.n
        self.threads = threads
        self.pool = ThreadPoolExecutor(max_workers=threads)

    def spmv(self, v):
        import oracle
        w = np.empty(self.n)

        def one(blk):
            a, b, rp, col, val = blk
            w[a:b] = oracle.spmv(rp, col, val, v)
        list(self.pool.map(one, self.blocks))
        return w

    def close(self):
        self.pool.shutdown()


def run_reference(args):
    """The CPU oracle on the host cores: one plain FP64 CSR SpMV per step."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    w, A, v = build_workload(args.config)
    st, plan_s, src = oracle_stats(A, w)
    B = bytes_per_apply(A, st)
    T = host_cores()
    ot = OracleThreads(A, T)
    for _ in range(args.warmup):
        ot.spmv(v)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ot.spmv(v)
    el = time.perf_counter() - t0
    ot.close()
    val = B * args.steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(el / args.steps * 1e3, 3), "ms_per_apply": round(el / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n": A.n, "nnz": A.nnz, "n_p": w.n_p, "ppn": w.ppn,
                   "partition": "contiguous", "gathers": "literal", "applies_per_step": 1},
        "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": T, "kind": "oracle",
                         "sample": f"{args.steps} plain FP64 CSR SpMVs of the full matrix on {T} "
                                   "threads (row blocks of equal stored entries); bytes counted as "
                                   "for the GPU apply, so the ratio of the two values is the "
                                   "ratio of their times per apply",
                         "ms_per_apply": round(el / args.steps * 1e3, 3),
                         "plan_stats": src,
                         "plan_build_s": None if plan_s is None else round(plan_s, 3)},
        "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def modelled_comm(nap, plan, w):
    """Sec. 3 cost models (max-rate inter-node, intra-node) with the paper's
    Blue Waters parameters, applied to this plan's messages: the modelled
    communication time of one standard and one node-aware exchange."""
    from paper_1612_08060_gb300 import model
    lists = {k: nap.export_list(plan, getattr(nap, "LIST_" + k))[:3]
             for k in ("STD", "INTER", "J0", "J1", "J2")}
    m = model.modelled(lists, w.ppn, w.n_p)
    return {k: float(f"{v:.4g}") for k, v in m.items()} | {
        "machine": "Blue Waters parameters of Sec. 3 (not this GPU)"}


def time_bounded(fn, budget_s):
    """Run fn once, then as often as fits in budget_s; (runs, seconds)."""
    t0 = time.perf_counter()
    fn()
    one = time.perf_counter() - t0
    reps = max(1, int(budget_s / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    return reps, time.perf_counter() - t0


def cpu_baseline_leg(A, v, w_gpu_one, B, budget_s, n_p, ppn, gpu_ms_per_apply, strided=False):
    """The oracle timed on this host's cores on a bounded sample (single thread,
    and on every core), its plan build timed once where that takes seconds, and
    the relative error of one GPU apply against it."""
    import oracle
    plan_s = None
    if A.nnz <= 5 * 10**7:
        t0 = time.perf_counter()
        oracle.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=oracle.STRIDED if strided else 0)
        plan_s = round(time.perf_counter() - t0, 3)
    ref = oracle.spmv(A.row_ptr, A.col, A.val, v)
    rel = float(np.linalg.norm(w_gpu_one - ref) / np.linalg.norm(ref))
    r1, e1 = time_bounded(lambda: oracle.spmv(A.row_ptr, A.col, A.val, v), budget_s / 2)
    T = host_cores()
    ot = OracleThreads(A, T)
    assert np.array_equal(ot.spmv(v), ref)
    rT, eT = time_bounded(lambda: ot.spmv(v), budget_s / 2)
    ot.close()
    cpu_ms = eT / rT * 1e3
    return {"value": round(B * rT / eT / 1e9, 3), "unit": "GB/s", "cores": T, "kind": "oracle",
            "sample": f"{rT} plain FP64 CSR SpMVs of the full matrix on {T} threads (row blocks "
                      f"of equal stored entries, {eT:.1f} s); bytes counted as for the GPU apply "
                      "(the plain SpMV moves only the CSR part of them), so compare the times",
            "ms_per_apply": round(cpu_ms, 3),
            "gpu_ms_per_apply": round(gpu_ms_per_apply, 5),
            "gpu_speedup_per_apply": round(cpu_ms / gpu_ms_per_apply, 1),
            "single_thread": {"value": round(B * r1 / e1 / 1e9, 3), "cores": 1,
                              "ms_per_apply": round(e1 / r1 * 1e3, 3),
                              "sample": f"{r1} SpMVs in {e1:.1f} s"},
            "plan_build_s": plan_s,
            "plan_build_note": None if plan_s is not None else
            "the oracle's plan of this workload takes minutes on one core; not timed here",
            "gpu_vs_oracle_relerr": rel}


def make_opts(nap, args, precision):
    return nap.make_opts(engine={"default": nap.ENGINE_DEFAULT, "fused": nap.ENGINE_FUSED,
                                 "phased": nap.ENGINE_PHASED,
                                 "overlap": nap.ENGINE_OVERLAP}[args.engine],
                         vec=args.vec, chunk=args.chunk, tile_rows=args.tile_rows,
                         tile_nnz=args.tile_nnz, stages=args.stages,
                         pipeline={"default": 0, "cta": nap.PIPELINE_CTA,
                                   "warp": nap.PIPELINE_WARP, "sell": nap.PIPELINE_SELL}[args.pipeline],
                         halo={"default": 0, "on": nap.HALO_ON, "off": nap.HALO_OFF}[args.halo],
                         precision=nap.PREC_F32 if precision == "f32" else nap.PREC_F64,
                         ctas_per_sm=args.ctas_per_sm)


def measure(nap, torch, dev, args, cfg, precision, reps, steps, warmup, ws=1, with_clocks=False,
            keep=False):
    """One workload timed through the library: build the plan, warm up, time
    `steps` steps of `reps` chained applies with CUDA events on the launching
    stream, then time the SpMV step kernel alone.  Returns (line fields, ctx)."""
    w, A, v = build_workload(cfg)
    t0 = time.perf_counter()
    pflags = nap.F32_VALUES | (nap.PARTITION_STRIDED if args.partition == "strided" else 0) | (
        nap.COMPOSED_GATHERS if args.gathers == "composed" else 0)
    plan = nap.napspmv_plan(A.row_ptr, A.col, A.val, w.n_p, w.ppn, pflags)
    plan_ms = (time.perf_counter() - t0) * 1e3
    st = nap.napspmv_plan_stats(plan)
    f32 = precision == "f32"
    scale = chain_scale(A)
    B = bytes_per_apply(A, st) - (4.0 * A.nnz if f32 else 0.0)
    B_csr = st["bytes_csr_f32"] if f32 else st["bytes_csr_f64"]
    assert abs(B - (B_csr + st["bytes_msg"])) < 1.0
    opts = make_opts(nap, args, precision)
    eff = nap.napspmv_get_default_opts(plan)
    engine = opts.engine or eff.engine
    # FP32 mode of the phased / overlapped engines moves FP32 copies through the
    # message steps: 4 B read + 4 B write + 4 B index per element and hop
    # instead of 8 + 8 + 4 (the fused engine keeps FP64 messages)
    if args.gathers == "composed":
        # two gathers from v: 8 B read + 8 B write + 4 B index per value
        B = B_csr + 20.0 * (st["bll_total"] + st["bnl_total"])
        if f32:
            B -= 8.0 * (st["bll_total"] + st["bnl_total"])
    elif f32 and engine != nap.ENGINE_FUSED:
        B -= st["bytes_msg"] * 8.0 / 20.0
    # SpMV step alone: row pointer, column + value streams, each x and each
    # received value read once, w written once; in FP32 mode the step also
    # makes the FP32 copy of x (8 B read + 4 B written per row) and reads
    # 4-byte copies
    if f32:
        B_spmv = 4.0 * (A.n + 1) + 8.0 * A.nnz + 24.0 * A.n + 4.0 * (
            st["bll_total"] + st["bnl_total"])
    else:
        B_spmv = 4.0 * (A.n + 1) + 12.0 * A.nnz + 16.0 * A.n + 8.0 * (
            st["bll_total"] + st["bnl_total"])
    stream = torch.cuda.Stream(device=dev)
    vd = torch.from_numpy(v).to(dev)
    wd = torch.empty_like(vd)

    def step():
        nap.napspmv_apply_ex(plan, vd, wd, reps, scale, opts, stream=stream)

    clocks = None
    with torch.cuda.stream(stream):
        # one plain apply for the parity figure of the CPU leg
        nap.napspmv_apply_ex(plan, vd, wd, 1, 1.0, opts, stream=stream)
        assert nap.napspmv_status(plan, stream) == 0
        w_one = wd.cpu().numpy()
        for _ in range(warmup):
            step()
        assert nap.napspmv_status(plan, stream) == 0
        sampler = ClockSampler(dev.index)
        if with_clocks:
            sampler.start()
            time.sleep(0.3)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        launches0 = nap.napspmv_launch_count()
        ev[0].record(stream)
        for i in range(steps):
            step()
            ev[i + 1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        launches = nap.napspmv_launch_count() - launches0
        if ws > 1:
            torch.distributed.barrier()
        if with_clocks:
            clocks = sampler.stop()
        rc = nap.napspmv_status(plan, stream)
        assert rc == 0, rc
    # the dominant kernel (three-block SpMV, a11) timed alone on the same stream
    # (FP32: after a phased apply, whose receive buffers hold the FP32 copies)
    with torch.cuda.stream(stream):
        ro = opts
        if f32:
            ro = nap.make_opts(**{k: getattr(opts, k) for k, _ in opts._fields_})
            ro.engine = nap.ENGINE_PHASED
        nap.napspmv_apply_ex(plan, vd, wd, 1, 1.0, ro, stream=stream)
        sp_n = 50 if A.nnz < 5 * 10**7 else 20
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        xd = torch.empty_like(vd)
        for _ in range(3):
            nap.napspmv_spmv_step(plan, vd, xd, 1.0, opts, stream=stream)
        e0.record(stream)
        for _ in range(sp_n):
            nap.napspmv_spmv_step(plan, vd, xd, 1.0, opts, stream=stream)
        e1.record(stream)
        e1.synchronize()
        spmv_ms = e0.elapsed_time(e1) / sp_n
        # same rows, same products; with more than one lane per row the engines
        # may sum in a different order
        err = float(torch.linalg.norm(xd - wd) / torch.linalg.norm(wd))
        assert err <= 1e-13, f"SpMV step does not reproduce the apply: {err}"
        assert nap.napspmv_status(plan, stream) == 0
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(total_ms, dev)
    value = job_value(ws, B, reps, steps, total_ms)
    avg_launch = statistics.mean(per)
    achieved = B * reps / (avg_launch * 1e-3) / 1e9
    peak, peak_kind = peaks()
    ms_apply = total_ms / steps / reps
    cfgd = {"workload": w.name + ("_strided" if args.partition == "strided" else "") + (
                "_composed" if args.gathers == "composed" else ""),
            "n": A.n, "nnz": A.nnz, "n_p": w.n_p, "ppn": w.ppn,
            "partition": args.partition, "gathers": args.gathers,
            "applies_per_step": reps, "scale": scale,
            "engine": {1: "fused", 2: "phased", 3: "overlap"}[engine],
            "pipeline": {1: "cta", 2: "warp", 3: "sell"}[opts.pipeline or eff.pipeline],
            "vec": opts.vec or eff.vec, "chunk": opts.chunk or eff.chunk,
            "tile_rows": opts.tile_rows or eff.tile_rows,
            "tile_nnz": opts.tile_nnz or eff.tile_nnz, "stages": opts.stages or eff.stages,
            "halo": {1: "on", 2: "off"}[opts.halo or eff.halo],
            "l2": "inputs larger than L2 (129 MB): each apply streams the matrix "
                  f"({(12 if not f32 else 8) * A.nnz / 1e6:.0f} MB of columns and values); "
                  "not flushed between steps"}
    what = f"{precision}|{cfgd['engine']}|{cfgd['pipeline']}"
    rec = ncu_record(w.name, what)
    spmv_traffic = None if rec is None else rec.get("spmv_step_bytes")
    out = {
        "value": value, "ms_per_step": total_ms / steps, "ms_per_step_median": statistics.median(per),
        "ms_per_apply": ms_apply, "dtype": "f32-values/f64-sums" if f32 else "f64",
        "config": cfgd,
        "bytes_per_apply": {"total": B, "csr": B_csr, "msg": B - B_csr},
        "csr_gbs": round(B_csr * reps / (avg_launch * 1e-3) / 1e9, 3),
        "gflops": round(2.0 * A.nnz * reps / (avg_launch * 1e-3) / 1e9, 3),
        "roofline": {"bound": "hbm", "achieved": round(B_spmv / (spmv_ms * 1e-3) / 1e9, 3),
                     "peak": peak, "unit": "GB/s",
                     "frac": round(B_spmv / (spmv_ms * 1e-3) / 1e9 / peak, 4),
                     "frac_of_nominal_8tbs": round(B_spmv / (spmv_ms * 1e-3) / 1e9 / NOMINAL_GBS, 4),
                     "peak_kind": peak_kind, "traffic": spmv_traffic,
                     "kernel": "the three-block SpMV step (one launch = every row of one apply)",
                     "timing": f"CUDA events around {sp_n} back-to-back napspmv_spmv_step launches "
                               "on the benchmark stream after the timed region" + (
                                   "; inside it the overlapped engine runs the same rows as a "
                                   "local and a remote launch" if engine == nap.ENGINE_OVERLAP
                                   else "; inside it the phased engine runs the same launch"
                                   if engine == nap.ENGINE_PHASED
                                   else "; inside it the fused kernel's last level sums the "
                                   "same rows"),
                     "algorithmic_bytes": B_spmv, "launch_ms": round(spmv_ms, 5)},
        "step_roofline": {"bound": "hbm", "achieved": round(achieved, 3), "peak": peak,
                          "frac": round(achieved / peak, 4),
                          "frac_of_nominal_8tbs": round(achieved / NOMINAL_GBS, 4),
                          "what": "whole apply (message steps + SpMV), algorithmic bytes"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "plan": {"gpu_plan_ms": round(plan_ms, 2), "std_msgs": st["std_msgs"],
                 "std_inter_msgs": st["std_inter_msgs"], "std_inter_vals": st["std_inter_vals"],
                 "nap_inter_msgs": st["nap_inter_msgs"], "nap_inter_vals": st["nap_inter_vals"],
                 "nap_intra_msgs": st["nap_intra_msgs"], "nap_intra_vals": st["nap_intra_vals"]},
    }
    if rec is not None and rec.get("apply_bytes"):
        # ncu DRAM bytes of one apply (each of its kernels captured on its own)
        # against the apply time: the HBM fraction of the whole apply
        db = rec["apply_bytes"]
        out["apply_dram"] = {"bytes_per_apply": db, "gbs": round(db / (ms_apply * 1e-3) / 1e9, 3),
                             "frac": round(db / (ms_apply * 1e-3) / 1e9 / peak, 4),
                             "per_kernel": rec.get("per_kernel"),
                             "source": "profiles/dram_traffic.json (ncu, one kernel per capture)"}
    else:
        out["apply_dram"] = None
    ctx = dict(w=w, A=A, v=v, plan=plan, st=st, B=B, scale=scale, w_one=w_one, stream=stream,
               opts=opts, ms_apply=ms_apply) if keep else None
    if not keep:
        del plan
    return out, ctx


def e2e_host(nap, torch, dev, ctx, reps, steps, ws):
    """The same metric through the host-buffer entry point: every call copies v
    in from pinned host memory, runs `reps` chained applies and copies w out."""
    A, B, plan, stream, scale = ctx["A"], ctx["B"], ctx["plan"], ctx["stream"], ctx["scale"]
    # the host-buffer call applies the plan's default options: make them the
    # timed region's (its engine, precision and tiles), as the library resolves them
    o, d = ctx["opts"], nap.napspmv_get_default_opts(plan)
    for f, _ in type(o)._fields_:
        if f == "precision" or getattr(o, f):
            setattr(d, f, getattr(o, f))
    nap.napspmv_set_default_opts(plan, d)
    vh = torch.from_numpy(ctx["v"].copy()).pin_memory()
    wh = torch.empty_like(vh).pin_memory()
    nap.napspmv_apply_host(plan, vh, wh, reps, scale, stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(steps):
        nap.napspmv_apply_host(plan, vh, wh, reps, scale, stream=stream)
    el = time.perf_counter() - t0
    return {"value": round(ws * B * reps * steps / el / 1e9, 3), "unit": "GB/s",
            "h2d_bytes_per_step": int(vh.numel() * 8), "d2h_bytes_per_step": int(wh.numel() * 8),
            "applies_per_call": reps, "ms_per_call": round(el / steps * 1e3, 4)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--reps", type=int, default=0, help="chained applies per step (0: the "
                    "workload's default: 100 for the stencils, 10 for the 2^23-row matrix)")
    ap.add_argument("--engine", default="default", choices=["default", "fused", "phased", "overlap"])
    ap.add_argument("--vec", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--tile-nnz", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--pipeline", default="default", choices=["default", "cta", "warp", "sell"])
    ap.add_argument("--halo", default="default", choices=["default", "on", "off"],
                    help="overlapped engine: stage each process's receive buffers in shared "
                         "memory for its remote rows")
    ap.add_argument("--gathers", default="literal", choices=["literal", "composed"],
                    help="composed: receive buffers gathered straight from v (an ablation "
                         "of the node-aware exchange's hops)")
    ap.add_argument("--partition", default="contiguous", choices=["contiguous", "strided"],
                    help="strided: row i on process i mod n_p (the SuiteSparse runs' partition)")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--precision", default="f64", choices=["f64", "f32"],
                    help="f32: FP32-stored values, FP32 products, FP64 sums")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads measured beside the headline")
    ap.add_argument("--serve", type=int, default=256,
                    help="requests of the serving mix served by both loops (0: skip)")
    ap.add_argument("--serve-nmax", type=float, default=2e6)
    ap.add_argument("--serve-sweep", default="",
                    help="comma-separated further loads (fractions of the plain loop's "
                         "saturated throughput), e.g. 0.5,1.0,1.2")
    ap.add_argument("--rows", type=int, default=0,
                    help="with --config 4 and --profile-spmv: the banded random structure at "
                         "this many rows (same band, rows per process and ppn)")
    ap.add_argument("--ncu-record", nargs="+", default=None, metavar="KEY=CSV",
                    help="write profiles/dram_traffic.json from the ncu CSV logs of "
                         "`--profile-spmv 2` runs, KEY = workload|precision|engine|pipeline; "
                         "no GPU needed")
    ap.add_argument("--profile-spmv", type=int, default=0,
                    help="profiling mode: one apply, then this many SpMV-step launches; "
                         "prints nothing")
    args = ap.parse_args()
    if args.ncu_record:
        write_ncu_records(args.ncu_record, os.path.join(ROOT, "profiles", "dram_traffic.json"))
        return
    if args.warmup < 3:
        args.warmup = 3
    reps = args.reps or DEFAULT_REPS.get(args.config, 10)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import __graft_entry__
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    __graft_entry__.build()
    from paper_1612_08060_gb300 import napspmv as nap

    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    if args.profile_spmv:
        w, A, v = build_workload(args.config, args.rows)
        plan = nap.napspmv_plan(A.row_ptr, A.col, A.val, w.n_p, w.ppn, nap.F32_VALUES)
        opts = make_opts(nap, args, args.precision)
        stream = torch.cuda.Stream(device=dev)
        vd = torch.from_numpy(v).to(dev)
        wd, xd = torch.empty_like(vd), torch.empty_like(vd)
        ro = nap.make_opts(**{k: getattr(opts, k) for k, _ in opts._fields_})
        if args.precision == "f32":
            ro.engine = nap.ENGINE_PHASED
        nap.napspmv_apply_ex(plan, vd, wd, 1, 1.0, ro, stream=stream)
        for _ in range(args.profile_spmv):
            nap.napspmv_spmv_step(plan, vd, xd, 1.0, opts, stream=stream)
        stream.synchronize()
        assert nap.napspmv_status(plan, stream) == 0
        return

    main_fields, ctx = measure(nap, torch, dev, args, args.config, args.precision, reps,
                               args.steps, args.warmup, ws=ws, with_clocks=not args.no_clocks,
                               keep=True)
    e2e = e2e_host(nap, torch, dev, ctx, reps, max(3, min(args.steps, 20)), ws)
    e2e_one = e2e_host(nap, torch, dev, ctx, 1, 20, ws)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    w = ctx["w"]
    line = {"metric": METRIC, "value": round(main_fields["value"], 3), "unit": "GB/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(main_fields["ms_per_step"], 4),
            "ms_per_step_median": round(main_fields["ms_per_step_median"], 4),
            "ms_per_apply": round(main_fields["ms_per_apply"], 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": main_fields["dtype"], "data": "synthetic",
            "config": main_fields["config"] | {"parallelism": f"replicas{ws}"}}
    for k in ("bytes_per_apply", "csr_gbs", "gflops", "roofline", "step_roofline", "apply_dram",
              "gpu_launches", "plan"):
        line[k] = main_fields[k]
    line["modelled_comm"] = modelled_comm(nap, ctx["plan"], w)
    line["paper_context"] = ("no GPU and no SpMV-throughput result in the paper; its CPU MPI runs "
                             "on Blue Waters (Cray XE, two AMD 6276 Interlagos per node) show "
                             "node-aware SpMV up to about 100x faster than standard SpMV at scale "
                             "(context only, not a target)")
    line["e2e"] = e2e
    line["e2e_one_apply"] = e2e_one | {"what": "one apply per call: copy v in, one apply, copy "
                                               "w out, synchronise"}
    line["clocks"] = main_fields["clocks"]
    if not args.no_cpu and ws == 1:
        line["cpu_baseline"] = cpu_baseline_leg(ctx["A"], ctx["v"], ctx["w_one"], ctx["B"],
                                                args.cpu_budget, w.n_p, w.ppn,
                                                main_fields["ms_per_apply"],
                                                args.partition == "strided")
    del ctx
    torch.cuda.empty_cache()
    if not args.no_extras and ws == 1 and args.config == 4 and args.precision == "f64":
        extras = []
        for cfg, prec in ((2, "f64"), (4, "f32")):
            f, _ = measure(nap, torch, dev, args, cfg, prec, DEFAULT_REPS[cfg],
                           max(5, args.steps // 2), args.warmup)
            extras.append({"workload": f["config"]["workload"], "dtype": f["dtype"],
                           "value": round(f["value"], 3), "unit": "GB/s",
                           "ms_per_step": round(f["ms_per_step"], 4),
                           "ms_per_apply": round(f["ms_per_apply"], 5),
                           "config": f["config"], "bytes_per_apply": f["bytes_per_apply"],
                           "roofline": f["roofline"], "step_roofline": f["step_roofline"],
                           "apply_dram": f["apply_dram"]})
            torch.cuda.empty_cache()
        line["extra"] = extras
    if args.serve > 0 and ws == 1:
        from paper_1612_08060_gb300 import serve
        sweep = tuple(float(x) for x in args.serve_sweep.split(",") if x.strip())
        line["serving"] = serve.compare(args.serve, n_hi=args.serve_nmax, device=dev, sweep=sweep)
        line["serving"]["cut"] = (f"{args.serve} requests of the serving mix's 4096 (N log-uniform "
                                  f"in [1e3, {args.serve_nmax:.0e}]) so that the default run "
                                  "stays within minutes")
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
