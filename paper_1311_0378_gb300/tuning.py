"""Persistence of the autotuner's cache (results keyed by size bucket,
connectivities and marker class; see recon_autotune in include/recon.h) as a
small JSON file, so a later process reuses them without timing trials."""
from __future__ import annotations

import json
import os

import paper_1311_0378_gb300 as rc

FIELDS = ("size_bucket", "connectivities", "marker_class", "block_h", "bands", "scan_pairs", "scan_gain")


def write_entries(path: str, entries) -> None:
    """Stores cache entries (7-tuples in FIELDS order) as JSON, atomically."""
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump({"entries": [dict(zip(FIELDS, (int(x) for x in e))) for e in entries]}, f, indent=1)
    os.replace(tmp, path)


def read_entries(path: str):
    """Cache entries stored by write_entries (ValueError on a malformed file)."""
    with open(path) as f:
        data = json.load(f)
    try:
        return [tuple(int(e[k]) for k in FIELDS) for e in data["entries"]]
    except (KeyError, TypeError, ValueError) as err:
        raise ValueError("not an autotuner cache file: %s (%s)" % (path, err))


def save_cache(ctx, path: str) -> int:
    """Writes the context's cache to `path`; returns the number of entries."""
    st, entries = rc.recon_autotune_cache(ctx)
    rc.check(st, "recon_autotune_cache")
    write_entries(path, entries)
    return len(entries)


def load_cache(ctx, path: str) -> int:
    """Adds the entries stored at `path` to the context's cache; returns their number."""
    entries = read_entries(path)
    if entries:
        rc.check(rc.recon_autotune_cache_load(ctx, entries), "recon_autotune_cache_load")
    return len(entries)
