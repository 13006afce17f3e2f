#!/usr/bin/env python3
"""Writes tests/golden/batch_hashes.json: for every tile of the two full-size
batch workloads (64 tiles of 4096 x 4096, and 1000 tiles of uneven sizes; the
concurrently processed 4K x 4K tiles of Sec. V), a hash of its inputs (I, J)
and of the oracle's reconstruction R.

Only the oracle and the seeded input generator are called. Each R is computed
twice, by the oracle's raster / anti-raster sweeps to stability and by its
maximum-bottleneck flood (two pinned, independent exact routes), and the
script stops if they disagree on any tile.

Hashes: the first 24 hex digits of SHA-256 over the tile's bytes (rows of W
bytes, no padding); the input hash covers I followed by J.

Usage: python tests/golden/make_batch_hashes.py [--workloads batch64,uneven1000]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "batch_hashes.json")
DIGITS = 24


def h(*arrays) -> str:
    d = hashlib.sha256()
    for a in arrays:
        d.update(memoryview(a).cast("B"))
    return d.hexdigest()[:DIGITS]


def hash_workload(name: str, chunk: int = 32) -> dict:
    w = synth.workload(name)
    specs = list(w.tiles)
    nt = os.cpu_count() or 1
    rows = []
    t0 = time.time()
    # largest tiles first inside each chunk keeps the host threads balanced
    for c0 in range(0, len(specs), chunk):
        part = specs[c0:c0 + chunk]
        pairs = synth.generate(part, w.seed)
        conns = [s.conn for s in part]
        R_sweep, _ = oracle.recon_tiles(pairs, conns, "sweep", nthreads=nt)
        R_wide, _ = oracle.recon_tiles(pairs, conns, "widest", nthreads=nt)
        for k, (s, (I, J), a, b) in enumerate(zip(part, pairs, R_sweep, R_wide)):
            if not (a == b).all():
                raise SystemExit("%s tile %d: sweeps and flood disagree" % (name, c0 + k))
            rows.append({"t": c0 + k, "H": s.H, "W": s.W, "conn": s.conn, "marker": s.marker,
                         "in": h(I, J), "R": h(a)})
        print("%s: %d / %d tiles, %.0f s" % (name, c0 + len(part), len(specs), time.time() - t0),
              file=sys.stderr, flush=True)
    return {"seed": w.seed, "tiles": rows}


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="batch64,uneven1000")
    args = ap.parse_args()
    out = {"what": "per-tile SHA-256 (first %d hex digits) of the inputs I||J and of the oracle's R; "
                   "R from sweeps to stability, equal to the maximum-bottleneck flood on every tile" % DIGITS,
           "script": "tests/golden/make_batch_hashes.py", "workloads": {}}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out["workloads"] = json.load(f).get("workloads", {})
    for name in args.workloads.split(","):
        out["workloads"][name] = hash_workload(name)
    tmp = OUT + ".tmp"
    with open(tmp, "w") as f:
        json.dump(out, f, indent=0, separators=(",", ":"))
        f.write("\n")
    os.replace(tmp, OUT)
    return 0


if __name__ == "__main__":
    sys.exit(main())
