"""Full-size parity in the launch configuration bench.py times: the whole
64-tile 4096^2 batch and the whole 1000-tile uneven batch are reconstructed
in one persistent launch each, with the learned schedule and the default
128-row blocks. A deterministic sample of tiles (the largest fill-holes tiles
among them) is then compared byte for byte with the CPU oracle; every tile of
the sample also satisfies J <= R <= I."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402
from paper_1311_0378_gb300 import cost_model  # noqa: E402


def _sample(specs, k):
    """Every len/k-th tile plus the two largest fill-holes tiles."""
    idx = set(range(0, len(specs), max(1, len(specs) // k)))
    fills = sorted((i for i, s in enumerate(specs) if s.marker == synth.FILLHOLES),
                   key=lambda i: -specs[i].H * specs[i].W)
    idx.update(fills[:2])
    return sorted(idx)


@pytest.mark.parametrize("name,k", [("batch64", 6), ("uneven1000", 10)])
def test_fullsize_batch_sampled_parity(name, k):
    import paper_1311_0378_gb300.build as b
    b.build()
    w = synth.workload(name)
    specs = list(w.tiles)
    tot = sum(s.H * s.W for s in specs)
    off = np.concatenate([[0], np.cumsum([s.H * s.W for s in specs])]).astype(np.int64)
    hI = torch.empty(tot, dtype=torch.uint8).pin_memory()
    hJ = torch.empty(tot, dtype=torch.uint8).pin_memory()
    synth.generate_into(specs, w.seed, [hI.data_ptr() + int(o) for o in off[:-1]],
                        [hJ.data_ptr() + int(o) for o in off[:-1]])
    dI, dJ = hI.cuda(), hJ.cuda()
    torch.cuda.synchronize()
    ctx = rc.recon_init(0, 0, rc.RECON_FLAG_LEARNED | rc.RECON_FLAG_SYNC)
    try:
        cost_model.install(ctx)
        tiles = [(dI.data_ptr() + int(off[t]), dJ.data_ptr() + int(off[t]), s.H, s.W, s.W, s.conn)
                 for t, s in enumerate(specs)]
        rc.check(rc.recon_batch(ctx, tiles), "recon_batch " + name)
        R = dJ.cpu()
    finally:
        rc.recon_free(ctx)
    picks = _sample(specs, k)
    pairs = [(hI[off[t]:off[t + 1]].numpy().reshape(specs[t].H, specs[t].W),
              hJ[off[t]:off[t + 1]].numpy().reshape(specs[t].H, specs[t].W)) for t in picks]
    wants, _ = oracle.recon_tiles(pairs, [specs[t].conn for t in picks], "sweep")
    for t, (I, J), want in zip(picks, pairs, wants):
        got = R[off[t]:off[t + 1]].numpy().reshape(specs[t].H, specs[t].W)
        assert (J <= got).all() and (got <= I).all()
        np.testing.assert_array_equal(got, want, err_msg="%s tile %d" % (name, t))
