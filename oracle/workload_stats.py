"""Plan statistics of the benchmark workloads, computed by the oracle and stored.

Test and benchmark infrastructure.  The CPU reference arm of the benchmark
reports the same metric as the GPU arm, whose byte count per apply includes the
node-aware plan's message volumes (Sec. 4.1-4.2: every value moved by the
on->on, on->off, pack, transfer and off->on steps).  Building the oracle's plan
of the 2^23-row banded random workload takes minutes on one core, so this
script computes the statistics once with the oracle and stores them beside it,
keyed by a fingerprint of the matrix pattern, n_p, ppn and the plan flags.  A
reader that finds no matching entry builds the oracle's plan itself.

    python oracle/workload_stats.py [cfg ...]     (default: 1 2 3 4)
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PATH = os.path.join(HERE, "workload_stats.json")


def fingerprint(row_ptr, col, n_p, ppn, flags=0):
    h = hashlib.sha256()
    h.update(row_ptr.tobytes())
    h.update(col.tobytes())
    h.update(f"{n_p},{ppn},{flags}".encode())
    return h.hexdigest()[:24]


def load():
    if not os.path.exists(PATH):
        return {}
    with open(PATH) as f:
        return json.load(f)


def lookup(row_ptr, col, n_p, ppn, flags=0):
    """The stored oracle statistics of this matrix pattern and partition, or None."""
    return load().get(fingerprint(row_ptr, col, n_p, ppn, flags))


def main(cfgs):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    from paper_1612_08060_gb300 import inputs
    table = load()
    for cfg in cfgs:
        w = inputs.workload(cfg)
        A = w.build()
        key = fingerprint(A.row_ptr, A.col, w.n_p, w.ppn)
        t0 = time.perf_counter()
        st = oracle.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn).stats()
        table[key] = {"workload": w.name, "n": A.n, "nnz": A.nnz, "n_p": w.n_p, "ppn": w.ppn,
                      "flags": 0, "stats": {k: int(v) for k, v in st.items()},
                      "oracle_plan_s": round(time.perf_counter() - t0, 1)}
        print(w.name, key, flush=True)
    with open(PATH, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [1, 2, 3, 4])
