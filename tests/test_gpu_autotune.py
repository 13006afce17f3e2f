"""The autotuner (a6) through the C ABI: it installs one of its candidates,
leaves every marker as it found it, the tuned context still reconstructs
bit-exactly, and its results are cached by (size bucket, connectivities,
marker class), reused without trials and persisted through a JSON file."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402
from paper_1311_0378_gb300 import tuning  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import paper_1311_0378_gb300.build as b
    b.build()


def batch(marker, n=2):
    base = synth.workload("single512").tiles[0]
    pairs = [synth.tile_pair(synth.with_marker(base, marker), 1 + k) for k in range(n)]
    dev = [(torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()) for I, J in pairs]
    torch.cuda.synchronize()
    desc = [(dI.data_ptr(), dJ.data_ptr(), 512, 512, 512, 8) for dI, dJ in dev]
    return pairs, dev, desc


def test_autotune_installs_restores_and_caches(tmp_path):
    c = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    try:
        pairs, dev, desc = batch(synth.HDOME)
        st, best = rc.recon_autotune(c, desc, 1)
        rc.check(st, "recon_autotune")
        assert rc.recon_get_param(c, rc.RECON_P_TUNE_FROM_CACHE) == 0
        assert best[0] in (32, 64, 128) and best[1] in (2, 4) and best[2] in (0, 1, 2) and best[3] in (0, 2048)
        assert (rc.recon_get_param(c, rc.RECON_P_BLOCK_H), rc.recon_get_param(c, rc.RECON_P_BANDS),
                rc.recon_get_param(c, rc.RECON_P_SWEEPS), rc.recon_get_param(c, rc.RECON_P_SCAN_GAIN)) == tuple(best)
        for (I, J), (_, dJ) in zip(pairs, dev):   # markers untouched
            np.testing.assert_array_equal(dJ.cpu().numpy(), J)
        rc.check(rc.recon_batch(c, desc), "tuned batch")
        for (I, J), (_, dJ) in zip(pairs, dev):
            np.testing.assert_array_equal(dJ.cpu().numpy(), oracle.recon(I, J, 8))

        # the same kind of batch again: from the cache, no trials
        pairs2, dev2, desc2 = batch(synth.HDOME)
        st, best2 = rc.recon_autotune(c, desc2, 1)
        rc.check(st, "recon_autotune (cached)")
        assert best2 == best and rc.recon_get_param(c, rc.RECON_P_TUNE_FROM_CACHE) == 1
        st, entries = rc.recon_autotune_cache(c)
        assert st == rc.RECON_OK and len(entries) == 1
        assert entries[0][:3] == (18, 2, 0) and tuple(entries[0][3:]) == tuple(best)

        # a border-seeded batch is another key: trials again
        pairs3, dev3, desc3 = batch(synth.FILLHOLES)
        st, best3 = rc.recon_autotune(c, desc3, 1)
        rc.check(st, "recon_autotune (fill-holes)")
        assert rc.recon_get_param(c, rc.RECON_P_TUNE_FROM_CACHE) == 0
        st, entries = rc.recon_autotune_cache(c)
        assert len(entries) == 2 and {e[2] for e in entries} == {0, 1}

        # persisted, then reused by a fresh context
        path = str(tmp_path / "tune.json")
        assert tuning.save_cache(c, path) == 2
    finally:
        rc.recon_free(c)
    c2 = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    try:
        assert tuning.load_cache(c2, path) == 2
        st, best4 = rc.recon_autotune(c2, desc2, 1)
        rc.check(st, "recon_autotune (loaded cache)")
        assert best4 == best and rc.recon_get_param(c2, rc.RECON_P_TUNE_FROM_CACHE) == 1
        assert rc.recon_autotune_cache_load(c2, [(18, 2, 0, 96, 4, 1, 0)]) == rc.RECON_EINVAL   # bad height
        assert len(rc.recon_autotune_cache(c2)[1]) == 2
        assert rc.recon_autotune_cache_load(c2, []) == rc.RECON_OK                              # clears
        assert rc.recon_autotune_cache(c2)[1] == []
    finally:
        rc.recon_free(c2)
