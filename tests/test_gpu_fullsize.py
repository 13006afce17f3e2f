"""Full-size parity in the launch configuration bench.py times: the whole
64-tile 4096^2 batch and the whole 1000-tile uneven batch (the concurrently
processed 4K x 4K tiles of Sec. V) are each reconstructed in one persistent
launch, once with the learned schedule and once with the plain one, with the
default 128-row blocks. EVERY tile's result is hashed and compared with the
hash of the oracle's reconstruction stored in tests/golden/batch_hashes.json
(written by tests/golden/make_batch_hashes.py, which calls only the oracle and
the input generator; there the oracle's sweeps and its maximum-bottleneck
flood agree on every tile). The inputs are hashed too, so a generator that
produced other bytes on this machine is reported as such."""
import hashlib
import json
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402
from paper_1311_0378_gb300 import cost_model  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch_hashes.json")


def _h(*arrays):
    d = hashlib.sha256()
    for a in arrays:
        d.update(memoryview(a).cast("B"))
    return d


def _hashes(flat, off, digits, other=None):
    """Per-tile hashes of a flat uint8 host tensor (of I||J when `other` is given),
    computed on host threads (hashlib releases the GIL on large buffers)."""
    a = flat.numpy()
    b = other.numpy() if other is not None else None

    def one(t):
        s = slice(int(off[t]), int(off[t + 1]))
        d = _h(a[s], b[s]) if b is not None else _h(a[s])
        return d.hexdigest()[:digits]
    with ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, range(len(off) - 1)))


@pytest.mark.parametrize("name", ["batch64", "uneven1000"])
def test_fullsize_batch_every_tile_matches_oracle(name):
    import paper_1311_0378_gb300.build as b
    b.build()
    with open(GOLDEN) as f:
        gold = json.load(f)["workloads"][name]
    w = synth.workload(name)
    specs = list(w.tiles)
    assert gold["seed"] == w.seed and len(gold["tiles"]) == len(specs)
    digits = len(gold["tiles"][0]["R"])
    off = np.concatenate([[0], np.cumsum([s.H * s.W for s in specs])]).astype(np.int64)
    tot = int(off[-1])
    hI = torch.empty(tot, dtype=torch.uint8).pin_memory()
    hJ = torch.empty(tot, dtype=torch.uint8).pin_memory()
    synth.generate_into(specs, w.seed, [hI.data_ptr() + int(o) for o in off[:-1]],
                        [hJ.data_ptr() + int(o) for o in off[:-1]])
    ins = _hashes(hI, off, digits, other=hJ)
    bad_in = [t for t, g in enumerate(gold["tiles"]) if g["in"] != ins[t]]
    assert not bad_in, "input generator gave other bytes for tiles %s" % bad_in[:10]
    dI, dJ0 = hI.cuda(), hJ.cuda()
    dJ = torch.empty_like(dJ0)
    torch.cuda.synchronize()
    for schedule in ("learned", "plain"):
        dJ.copy_(dJ0)
        torch.cuda.synchronize()
        flags = rc.RECON_FLAG_SYNC | (rc.RECON_FLAG_LEARNED if schedule == "learned" else 0)
        ctx = rc.recon_init(0, 0, flags)
        try:
            if schedule == "learned":
                cost_model.install(ctx)
            tiles = [(dI.data_ptr() + int(off[t]), dJ.data_ptr() + int(off[t]), s.H, s.W, s.W, s.conn)
                     for t, s in enumerate(specs)]
            rc.check(rc.recon_batch(ctx, tiles), "recon_batch %s %s" % (name, schedule))
            R = dJ.cpu()
        finally:
            rc.recon_free(ctx)
        got = _hashes(R, off, digits)
        bad = [t for t, g in enumerate(gold["tiles"]) if g["R"] != got[t]]
        assert not bad, "%s, %s schedule: %d of %d tiles differ from the oracle, first %s" % (
            name, schedule, len(bad), len(specs), bad[:10])
