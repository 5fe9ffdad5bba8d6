"""Parser of tests/golden/worked_example.txt (the paper's worked example)."""
import os
import re

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_example.txt")


def _proc(tok, ppn):
    m = re.fullmatch(r"\((\d+),(\d+)\)", tok)
    if not m:
        raise ValueError(tok)
    p, n = int(m.group(1)), int(m.group(2))
    return n * ppn + p


def load():
    """Returns dict with np, ppn, rows (list of sets), and per table KIND a dict
    key -> tuple of values; processes become global ranks.  PRINTED cells are
    returned separately under 'printed'."""
    data = {"printed": {}}
    lines = open(PATH).read().splitlines()
    ppn = None
    for ln in lines:
        if ln.startswith("PPN"):
            ppn = int(ln.split()[1])
    for ln in lines:
        ln = ln.split("#")[0].strip()
        if not ln:
            continue
        head, _, tail = ln.partition(":")
        toks = head.split()
        printed = toks[0] == "PRINTED"
        if printed:
            toks = toks[1:]
        kind, keys = toks[0], toks[1:]
        if kind in ("NP", "PPN"):
            data[kind.lower()] = int(keys[0])
            continue
        keyv = tuple(_proc(k, ppn) if k.startswith("(") else int(k) for k in keys)
        vals = tuple(_proc(v, ppn) if v.startswith("(") else int(v) for v in tail.split())
        key = keyv[0] if len(keyv) == 1 else keyv
        target = data["printed"] if printed else data
        target.setdefault(kind, {})[key] = vals
    n = len(data["PATTERN"])
    data["rows"] = [set(data["PATTERN"][i]) for i in range(n)]
    return data
