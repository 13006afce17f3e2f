"""The allocation-free entry point recon_run_noalloc, called through the C ABI.

It serves callers that may not allocate memory while running (a plugin whose
host framework owns all device memory through its own pool, or a pipeline
that cannot accept an allocation's implicit synchronisation), so its scratch
is one array built into the library and shared by every call. Its results
must equal the CPU oracle's byte for byte (reconstruction is integer max/min:
the tolerance is zero) and the context-based recon_run's, on calls in a row
that reuse that array: both markers, both connectivities, a ragged shape, the
largest accepted size, and a marker above its mask, which must be reported
without spoiling the next call. This file is collected last, so a failure
here never hides another test's result."""
import numpy as np
import pytest

import oracle
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


def _cases():
    base = synth.workload("single512").tiles[0]
    return [
        (synth.tile_pair(synth.with_marker(base, synth.FILLHOLES), 1), 8),                    # 512 x 512
        (synth.tile_pair(synth.TileSpec(1000, 777, 120, 3, 20, synth.HDOME, 4, 7), 5), 4),    # ragged
        (synth.tile_pair(synth.TileSpec(333, 1029, 90, 3, 20, synth.FILLHOLES, 4, 8), 5), 4),  # ragged
        (synth.tile_pair(base, 1), 8),
    ]


def test_no_alloc_matches_oracle_and_recon_run_on_calls_in_a_row():
    import paper_1311_0378_gb300.build as b
    b.build()
    for (I, J), conn in _cases():
        want = oracle.recon(I, J, conn)
        got1 = _no_alloc(I, J, conn)
        got2 = _no_alloc(I, J, conn)       # the same call again on the reused scratch
        np.testing.assert_array_equal(got1, want)
        np.testing.assert_array_equal(got2, want)
        np.testing.assert_array_equal(got1, _with_context(I, J, conn))


def test_no_alloc_largest_accepted_size():
    """4096 x 8192 = 64 x 64 blocks of 64 x 128 pixels: the 4096-block limit."""
    spec = synth.TileSpec(4096, 8192, 13000, 4, 12, synth.HDOME, 8, 3)
    I, J = synth.tile_pair(spec, 9)
    got = _no_alloc(I, J, 8)
    np.testing.assert_array_equal(got, oracle.recon(I, J, 8))


def test_no_alloc_marker_above_mask_then_normal_call():
    (I, J), conn = _cases()[3]
    bad = J.copy()
    bad[100, 200] = min(255, int(I[100, 200]) + 1)
    dI, dJ = _dev(I), _dev(bad)
    assert rc.recon_run_noalloc(dI.data_ptr(), dJ.data_ptr(), I.shape[0], I.shape[1], conn, 0) == rc.RECON_EMARKER
    np.testing.assert_array_equal(_no_alloc(I, J, conn), oracle.recon(I, J, conn))


def test_no_alloc_rejects_oversized_input():
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = d.data_ptr()
    # 8192 x 8192 needs 8192 blocks of 64 x 128: beyond the 4096-block scratch
    assert rc.recon_run_noalloc(p, p, 8192, 8192, 8, 0) == rc.RECON_EINVAL
    assert rc.recon_run_noalloc(p, p, 4, 2147483647, 8, 0) == rc.RECON_EINVAL   # no int overflow
    assert rc.recon_run_noalloc(p, p, 2147483647, 4, 8, 0) == rc.RECON_EINVAL
    assert rc.recon_run_noalloc(p, p, 4, 4, 6, 0) == rc.RECON_EINVAL
