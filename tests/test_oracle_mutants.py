"""The pins pin the oracle: each plausible mistake planted in a copy of
oracle.c (a wrong operand or index, a dropped term or condition, a flipped
ordering, a lost dedup, a swapped counter) makes the oracle's CPU pin tests
fail.  Each mutant is compiled with the oracle's own flags and loaded in a
separate pytest process through NAPSPMV_ORACLE_LIB; nothing here touches the
CUDA path.  CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
OUT = os.path.join(ROOT, "oracle", "_build", "mutants")
PINS = ["tests/test_oracle_brute.py", "tests/test_oracle_closed_forms.py",
        "tests/test_oracle_worked_example.py"]

# (name, the passage as written, the planted mistake); every passage occurs
# exactly once in oracle.c, so a change there that moves it fails loudly here
MUTANTS = [
    # Sec. 1 product: the column index dropped
    ("spmv_wrong_operand", "s += val[k] * v[col[k]];", "s += val[k] * v[i];"),
    # FP32-stored values: the product not rounded to FP32
    ("spmv_f32_unrounded_product", "float p = val[k] * x;", "double p = (double)val[k] * x;"),
    # Eq. R: the extra rows on the last ranks instead of the first
    ("partition_extra_rows_last", "return r * q + (r < rem ? r : rem);",
     "return r * q + (r > np - rem ? r - (np - rem) : 0);"),
    # the node of a rank taken modulo instead of by division
    ("node_by_rank_mod", "} else if (r / ppn == t / ppn) {", "} else if (r % ppn == t % ppn) {"),
    # on_node entries counted as off_node in the split
    ("split_on_node_as_off_node", "P->split[3 * i + 1]++;", "P->split[3 * i + 2]++;"),
    # T: the sending side ordered by ascending instead of descending |D(n, m)|
    ("send_order_ascending", "qsort(e, (size_t)c, sizeof(tu_entry), tu_desc);",
     "qsort(e, (size_t)c, sizeof(tu_entry), tu_asc);"),
    # U: receive processes counted from the front instead of from ppn - 1
    ("recv_order_not_reversed",
     "for (int64_t k = 0; k < c; k++) P->recv_proc[e[k].msg] = pn - 1 - (k % pn);",
     "for (int64_t k = 0; k < c; k++) P->recv_proc[e[k].msg] = k % pn;"),
    # the prose mapping rule and the tables' rule exchanged
    ("text_rule_swapped", "(flags & ORC_MAP_TEXT) ? tu_desc : tu_asc",
     "(flags & ORC_MAP_TEXT) ? tu_asc : tu_desc"),
    # majority mapping: ties go to the last process instead of the first
    ("majority_tie_last", "== sn * ppn + p) c++;\n                    if (c > best)",
     "== sn * ppn + p) c++;\n                    if (c >= best)"),
    # J0: the aggregator also "sends itself" the values it owns
    ("j0_includes_own_values", "if (p != s && (tpush(&j0, p, s, j) || tpush(&lbuf, s, s, j))) {",
     "if ((tpush(&j0, p, s, j) || tpush(&lbuf, s, s, j))) {"),
    # J1: every received value forwarded to every rank of the node
    ("j1_forwards_everything",
     "if (lfind(B, bs, I->idx[x]) >= 0 && tpush(&j1, q, s, I->idx[x])) {",
     "if (tpush(&j1, q, s, I->idx[x])) {"),
    # the sets keep their repeats
    ("dedup_dropped", "if (tcmp(&t->v[i], &t->v[w - 1]) != 0) t->v[w++] = t->v[i];",
     "t->v[w++] = t->v[i];"),
    # statistics: intra- and inter-node standard messages exchanged
    ("stats_intra_inter_swapped", "out[inter ? 4 : 2]++;", "out[inter ? 2 : 4]++;"),
    # Algorithm NAPSpMV: the off_node block's local_spmv dropped
    ("napspmv_off_node_dropped", "for (int blk = 0; blk < 3; blk++) {",
     "for (int blk = 0; blk < 2; blk++) {"),
    # the strided partition shifted by one row
    ("strided_shifted", "if (P->flags & ORC_STRIDED) return j % P->np;",
     "if (P->flags & ORC_STRIDED) return (j + 1) % P->np;"),
    # node splitting: the larger groups given to the last partners, not the first
    ("split_extra_processes_last",
     "int64_t size = pn / c + (k < pn % c ? 1 : 0);\n                        P->send_proc[e[k].msg] = first;",
     "int64_t size = pn / c + (k >= c - pn % c ? 1 : 0);\n                        P->send_proc[e[k].msg] = first;"),
    # node splitting: pieces received by the receiving group in reverse order
    ("split_pieces_reversed", "int64_t d = N->dst[k] * ppn + P->recv_proc[k] + i % nr;",
     "int64_t d = N->dst[k] * ppn + P->recv_proc[k] + (nr - 1 - i % nr);"),
    # node splitting: pieces cut by a rounded-up size instead of floor(i e / c)
    ("split_ceil_pieces", "int64_t lo = i * len / c, hi = (i + 1) * len / c;",
     "int64_t z = (len + c - 1) / c, lo = i * z < len ? i * z : len,\n"
     "                        hi = (i + 1) * z < len ? (i + 1) * z : len;"),
    # CG: the search direction's update with the wrong sign
    ("cg_beta_sign", "p[i] = r[i] + beta * p[i];", "p[i] = r[i] - beta * p[i];"),
]


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


def _run_pins(name, text):
    sys.path.insert(0, ROOT)
    from oracle import build as obuild
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(OUT, name + ".c")
    with open(src, "w") as f:
        f.write(text)
    lib = obuild.compile_to(src, os.path.join(OUT, name + ".so"))
    env = dict(os.environ, NAPSPMV_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-m", "not gpu",
                           "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=600)


def test_unmodified_copy_passes(source):
    """The control: the same harness on an unmodified copy passes every pin."""
    r = _run_pins("control", source)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-2000:])


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(source, name, orig, bad):
    assert source.count(orig) == 1, f"{name}: passage not found exactly once in oracle.c"
    r = _run_pins(name, source.replace(orig, bad))
    # exit code 1: tests ran and at least one failed (not a crash or a collection error)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-2000:], r.stderr[-2000:])
