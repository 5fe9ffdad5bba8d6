"""Communication-cost models of Sec. 3 applied to a plan's messages.

* Inter-node messages, max-rate model (Eq. max_rate):
      T = alpha + ppn * s / min(B_N, B_max + (ppn - 1) * B_inj)
* Intra-node messages (Eq. intra_comm):
      T_l = alpha_l + s_l / B_max_l
with s the message size in bytes (8 per FP64 value) and the Blue Waters
parameters the paper prints for the short, eager and rendezvous protocols
(Tables inter_comm and intra_comm).

Readings where the paper is silent:
* the protocol cut-offs are not given; short is taken for s <= 512 B, eager for
  s <= 8192 B, rendezvous above (typical MPICH defaults, not the paper's);
* the short protocol's B_max is printed as negative (-1.8e7); where the
  denominator min(...) is not positive the bandwidth term is dropped
  (latency only);
* a process sends its messages one after the other: its time is the sum of its
  messages' times; the modelled time of a step is the maximum over processes.
"""
from __future__ import annotations

import math

import numpy as np

INF = math.inf
# (alpha [s], B_inj [B/s], B_max [B/s], B_N [B/s]) per protocol, Table inter_comm
INTER = {"short": (4.0e-6, 6.3e8, -1.8e7, INF), "eager": (1.1e-5, 1.7e9, 6.2e7, INF),
         "rend": (2.0e-5, 3.6e9, 6.1e8, 5.5e9)}
# (alpha_l [s], B_max_l [B/s]), Table intra_comm
INTRA = {"short": (1.3e-6, 4.2e8), "eager": (1.6e-6, 7.4e8), "rend": (4.2e-6, 3.1e9)}
SHORT_MAX, EAGER_MAX = 512, 8192


def protocol(nbytes):
    return "short" if nbytes <= SHORT_MAX else ("eager" if nbytes <= EAGER_MAX else "rend")


def inter_time(nbytes, ppn):
    a, b_inj, b_max, b_n = INTER[protocol(nbytes)]
    rate = min(b_n, b_max + (ppn - 1) * b_inj)
    return a + (ppn * nbytes / rate if rate > 0 else 0.0)


def intra_time(nbytes):
    a, b = INTRA[protocol(nbytes)]
    return a + nbytes / b


def step_times(src, dst, ptr, ppn, n_p, inter=None):
    """Per-process summed time of a list of messages (src/dst processes, ptr
    offsets).  `inter`: None = decide by node (src // ppn != dst // ppn),
    True/False = all messages inter/intra."""
    t = np.zeros(n_p)
    for k in range(len(src)):
        nb = 8 * int(ptr[k + 1] - ptr[k])
        is_inter = (src[k] // ppn != dst[k] // ppn) if inter is None else inter
        t[src[k]] += inter_time(nb, ppn) if is_inter else intra_time(nb)
    return t


def modelled(lists, ppn, n_p):
    """lists: {'STD': (src, dst, ptr), 'INTER': ..., 'J0': ..., 'J1': ..., 'J2': ...}.
    Returns modelled maximum-over-processes times in seconds: the standard
    exchange (inter and intra parts, Alg. standard_spmv) and the node-aware one
    (the three local steps and the inter-node step, Alg. NAPSpMV, in sequence:
    on->off, inter-node, off->on; on->on overlaps and is counted on its own)."""
    std = lists["STD"]
    s_int = step_times(*std, ppn, n_p)
    out = {"std_max_s": float(s_int.max()) if n_p else 0.0}
    j0 = step_times(*lists["J0"], ppn, n_p, inter=False)
    it = step_times(*lists["INTER"], ppn, n_p, inter=True)
    j1 = step_times(*lists["J1"], ppn, n_p, inter=False)
    j2 = step_times(*lists["J2"], ppn, n_p, inter=False)
    out["nap_on_off_max_s"] = float(j0.max())
    out["nap_inter_max_s"] = float(it.max())
    out["nap_off_on_max_s"] = float(j1.max())
    out["nap_on_on_max_s"] = float(j2.max())
    out["nap_max_s"] = float(j0.max() + it.max() + j1.max())
    return out
