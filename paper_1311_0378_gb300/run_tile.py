"""Reconstructs one tile of a synthetic workload through the C ABI and prints
the device time and work counters (a driver for profilers and for quick checks).

    python -m paper_1311_0378_gb300.run_tile --workload single4096 --marker 1 --conn 8 --reps 3
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    import torch
    import paper_1311_0378_gb300 as rc
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="single4096")
    ap.add_argument("--marker", type=int, default=1)
    ap.add_argument("--conn", type=int, default=8)
    ap.add_argument("--tile", type=int, default=-1, help="tile index (default: first with marker/conn)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--param", action="append", default=[], help="KEY=VALUE, KEY a RECON_P_* suffix")
    a = ap.parse_args(argv)
    w = synth.workload(a.workload)
    if a.tile >= 0:
        spec = w.tiles[a.tile]
    else:
        spec = [t for t in w.tiles if t.marker == a.marker and t.conn == a.conn][0]
    I, J = synth.tile_pair(spec, w.seed)
    ctx = rc.recon_init(0, 0, 0)
    for kv in a.param:
        k, v = kv.split("=")
        rc.check(rc.recon_set_param(ctx, getattr(rc, "RECON_P_" + k.upper()), int(v)), kv)
    dI = torch.from_numpy(I).cuda()
    J0 = torch.from_numpy(J).cuda()
    dJ = J0.clone()
    torch.cuda.synchronize()
    for r in range(a.reps):
        dJ.copy_(J0)
        torch.cuda.synchronize()
        rc.check(rc.recon_run(ctx, dI.data_ptr(), dJ.data_ptr(), spec.H, spec.W, spec.conn), "recon_run")
        rc.check(rc.recon_sync_for(ctx, 120000), "sync")
        print(json.dumps({"rep": r, "ms": rc.recon_last_kernel_ms(ctx), **rc.recon_get_work(ctx, 1)[0]}),
              flush=True)
    rc.recon_free(ctx)
    return 0


if __name__ == "__main__":
    sys.exit(main())
