"""Table of tuned launch shapes (sg_autotune results) by problem size.

`tune_table.json` beside this file holds, for the benchmark workloads, the
shapes sg_autotune chose on a GB300 (CGS2 blocks per SM, persistent operator
CTAs per SM, transform tile width) and the times it measured.  `SG(...)`
applies the entry of its problem size through sg_tune_set (`lookup`); sizes
without an entry keep the built-in rules.  Regenerate on the GPU with

    python -m paper_2209_14740_gb300.tune_table --out paper_2209_14740_gb300/tune_table.json

which assembles each workload, runs sg_autotune on it and writes the table.
"""
from __future__ import annotations

import argparse
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_PATH = os.path.join(HERE, "tune_table.json")
KEY = ("dim", "mx", "my", "s", "r")
CHOICES = {"cgs_blocks_per_sm": range(0, 9), "op_ctas_per_sm": range(0, 17), "tc_tile_n": (0, 64, 128, 256),
           "tf32_transforms": (0, 1)}

_cache = None


def load_table(path: str = TABLE_PATH) -> dict:
    """{(dim, mx, my, s, r): entry} of the table file (empty if absent)."""
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        doc = json.load(fh)
    out = {}
    for e in doc.get("entries", []):
        k = tuple(int(e[f]) for f in KEY)
        if k in out:
            raise ValueError("duplicate tuning entry %r" % (k,))
        for name, allowed in CHOICES.items():
            if int(e.get(name, 0)) not in allowed:
                raise ValueError("tuning entry %r: %s = %r out of range" % (k, name, e[name]))
        out[k] = {name: int(e.get(name, 0)) for name in CHOICES}
    return out


def lookup(dim, mx, my, s, r):
    """Shapes for this problem size, or None."""
    global _cache
    if _cache is None:
        _cache = load_table()
    return _cache.get((int(dim), int(mx), int(my), int(s), int(r)))


def workloads():
    """(name, problem) of every size the table covers: the 511^2 and 127^2
    2D workloads, the 1D workload and the 64 sizes of the batched workload."""
    from . import inputs
    out = [("helmholtz_2d_511x511_s6_deg3", inputs.config_2d_511()),
           ("helmholtz_2d_127x127_s3_deg3", inputs.config_2d_127()),
           ("helmholtz_1d_200_s1_deg5", inputs.helmholtz_1d_c1())]
    seen = set()
    for k, p in enumerate(inputs.batch_64()):
        key = (p.dim, p.nx, p.ny, p.s, p.r)
        if key not in seen:
            seen.add(key)
            out.append(("batch_64 member %d (g=%d, s=%d, degree %d)" % (k, p.nx, p.s, p.r), p))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE_PATH)
    ap.add_argument("--restart", type=int, default=30)
    a = ap.parse_args(argv)
    import torch

    from . import binding as B
    B.load()
    entries = []
    seen = set()
    for name, prob in workloads():
        op = B.SG(prob, tuned=False)
        key = tuple(int(op.info[f]) for f in KEY)
        if key in seen:
            op.close()
            continue
        seen.add(key)
        t = op.autotune(restart=a.restart)
        e = {f: v for f, v in zip(KEY, key)}
        e.update(t)
        e["P"] = op.P
        e["workload"] = name
        entries.append(e)
        print(json.dumps(e), flush=True)
        op.close()
    doc = {"device": torch.cuda.get_device_name(0), "restart": a.restart,
           "note": "sg_autotune choices and times (microseconds) per problem size", "entries": entries}
    with open(a.out, "w") as fh:
        json.dump(doc, fh, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
