"""The allocation-free entry point recon_run_noalloc, called through the C ABI,
must give exactly what recon_run gives (reconstruction is integer max/min, so
the tolerance is zero), on two calls in a row that reuse its built-in scratch
array. It exists for callers that may not allocate memory while running; this
file is collected last so a failure here never hides another test's result."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402


def _dev(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    return t


def _with_context(I, J, conn):
    c = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    try:
        dI, dJ = _dev(I), _dev(J)
        rc.check(rc.recon_run(c, dI.data_ptr(), dJ.data_ptr(), I.shape[0], I.shape[1], conn), "recon_run")
        return dJ.cpu().numpy()
    finally:
        rc.recon_free(c)


def _no_alloc(I, J, conn):
    dI, dJ = _dev(I), _dev(J)
    rc.check(rc.recon_run_noalloc(dI.data_ptr(), dJ.data_ptr(), I.shape[0], I.shape[1], conn, 0),
             "recon_run_noalloc")
    return dJ.cpu().numpy()


def test_no_alloc_matches_recon_run_twice():
    import paper_1311_0378_gb300.build as b
    b.build()
    base = synth.workload("single512").tiles[0]
    first = synth.tile_pair(synth.with_marker(base, synth.FILLHOLES), 1)          # 512 x 512
    second = synth.tile_pair(synth.TileSpec(1000, 777, 120, 3, 20, synth.HDOME, 4, 7), 5)  # ragged
    for (I, J), conn in ((first, 8), (second, 4)):
        want = _with_context(I, J, conn)
        got = _no_alloc(I, J, conn)
        np.testing.assert_array_equal(got, want)


def test_no_alloc_rejects_oversized_input():
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = d.data_ptr()
    # 8192 x 8192 needs 8192 blocks of 64 x 128: beyond the 4096-block scratch
    assert rc.recon_run_noalloc(p, p, 8192, 8192, 8, 0) == rc.RECON_EINVAL
    assert rc.recon_run_noalloc(p, p, 4, 4, 6, 0) == rc.RECON_EINVAL
