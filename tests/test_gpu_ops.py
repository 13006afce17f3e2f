"""GPU parity for the two operations that run on the reconstruction engine
besides reconstruction by dilation: reconstruction by erosion (the dual) and
FillHoles (Table II). The CUDA path, through the C ABI, against the CPU oracle,
bit for bit, on ragged shapes (TMA and plain-load tiles, every block height),
on synthetic tiles, in mixed batches with the learned schedule, and through
the host-buffer entry point.
"""
import glob
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402

ERODE, FILL = rc.RECON_OP_ERODE, rc.RECON_OP_FILL_HOLES
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1311_0378_gb300.build as b
    b.build()
    c = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    yield c
    rc.recon_free(c)


def dev(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    return t


def gpu_op(c, I, J, conn, op, params=None):
    """One tile through recon_run_op; J = None leaves the output buffer
    uninitialised (filled with a pattern) for FillHoles."""
    for k, v in (params or {}).items():
        rc.check(rc.recon_set_param(c, k, v), "set_param")
    dI = dev(I)
    dJ = dev(J) if J is not None else dev(np.full(I.shape, 0xA5, np.uint8))
    rc.check(rc.recon_run_op(c, dI.data_ptr(), dJ.data_ptr(), I.shape[0], I.shape[1], conn, op), "recon_run_op")
    return dJ.cpu().numpy()


def border_marker(I):
    F = np.full_like(I, 255)
    F[0, :], F[-1, :], F[:, 0], F[:, -1] = I[0, :], I[-1, :], I[:, 0], I[:, -1]
    return F


def reset(c, bh=128, tma=1):
    for k, v in ((rc.RECON_P_BLOCK_H, bh), (rc.RECON_P_SWEEPS, 1), (rc.RECON_P_TMA, tma),
                 (rc.RECON_P_GRID, 0), (rc.RECON_P_SCAN_GAIN, 0)):
        rc.check(rc.recon_set_param(c, k, v))


SHAPES = [(1, 1), (1, 129), (129, 1), (3, 3), (37, 53), (64, 128), (65, 129), (130, 256),
          (257, 130), (300, 1000), (1000, 31), (515, 512)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bh,tma", [(128, 1), (64, 0), (32, 1)])
def test_erosion_ragged(ctx, shape, bh, tma):
    reset(ctx, bh, tma)
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W + bh)
    I = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    I = np.where(rng.random((H, W)) < 0.25, 255, I).astype(np.uint8)   # walls for the dual
    markers = [np.where(rng.random((H, W)) < 0.02, I, 255).astype(np.uint8),
               np.minimum(I.astype(int) + 10, 255).astype(np.uint8),
               border_marker(I)]
    for J in markers:
        for conn in (4, 8):
            np.testing.assert_array_equal(gpu_op(ctx, I, J, conn, ERODE), oracle.recon_erode(I, J, conn),
                                          err_msg="%s conn %d" % (shape, conn))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bh,tma", [(128, 1), (64, 0)])
def test_fill_holes_ragged(ctx, shape, bh, tma):
    reset(ctx, bh, tma)
    H, W = shape
    rng = np.random.default_rng(H * 7 + W * 13 + bh)
    fg = rng.random((H, W)) < 0.55
    I = np.where(fg, rng.integers(120, 256, size=(H, W)), rng.integers(0, 60, size=(H, W))).astype(np.uint8)
    for conn in (4, 8):
        np.testing.assert_array_equal(gpu_op(ctx, I, None, conn, FILL), oracle.fill_holes(I, conn),
                                      err_msg="%s conn %d" % (shape, conn))


def test_golden_fixtures(ctx):
    import test_oracle_pins as pins
    import test_oracle_pins_dual as dual
    reset(ctx)
    for path in sorted(glob.glob(os.path.join(GOLDEN, "erosion", "*.txt"))):
        conns, b = pins.read_golden(path)
        for conn in conns:
            np.testing.assert_array_equal(gpu_op(ctx, b["I"], b["J"], conn, ERODE), b["R"], err_msg=path)
    for path in sorted(glob.glob(os.path.join(GOLDEN, "fill_holes", "*.txt"))):
        conn, b = dual.read_fill(path)
        np.testing.assert_array_equal(gpu_op(ctx, b["I"], None, conn, FILL), b["F"], err_msg=path)


@pytest.mark.parametrize("marker", [synth.HDOME, synth.FILLHOLES])
@pytest.mark.parametrize("conn", [4, 8])
def test_synthetic_tiles(ctx, marker, conn):
    """The 512^2 synthetic tile: erosion of its complemented pair, and
    FillHoles of its mask."""
    reset(ctx)
    spec = synth.with_marker(synth.workload("single512").tiles[0], marker)
    I, J = synth.tile_pair(spec, 1)
    Ic, Jc = 255 - I, 255 - J
    np.testing.assert_array_equal(gpu_op(ctx, Ic, Jc, conn, ERODE), oracle.recon_erode(Ic, Jc, conn))
    np.testing.assert_array_equal(gpu_op(ctx, I, None, conn, FILL), oracle.fill_holes(I, conn))


def test_erosion_marker_below_mask_is_rejected(ctx):
    reset(ctx)
    I = np.full((64, 200), 50, np.uint8)
    J = np.full_like(I, 200)
    J[33, 150] = 49
    dI, dJ = dev(I), dev(J)
    st = rc.recon_run_op(ctx, dI.data_ptr(), dJ.data_ptr(), 64, 200, 8, ERODE)
    assert st == rc.RECON_EMARKER
    assert rc.recon_run_op(ctx, dI.data_ptr(), dJ.data_ptr(), 64, 200, 8, 3) == rc.RECON_EINVAL


def _mixed_specs():
    w = synth.workload("uneven1000")
    return [s for s in w.tiles[:36] if s.H * s.W <= 1 << 21][:18], w.seed


@pytest.mark.parametrize("learned", [False, True])
def test_mixed_batch(learned):
    """Dilation, erosion and FillHoles tiles in one persistent launch, each
    tile against its own oracle; with the learned schedule planning all three."""
    import paper_1311_0378_gb300.build as b
    from paper_1311_0378_gb300 import cost_model
    b.build()
    specs, seed = _mixed_specs()
    flags = rc.RECON_FLAG_SYNC | (rc.RECON_FLAG_LEARNED if learned else 0)
    c = rc.recon_init(0, 0, flags)
    try:
        if learned:
            cost_model.install(c)
        tiles, keep, wants = [], [], []
        for t, s in enumerate(specs):
            I, J = synth.tile_pair(s, seed)
            op = t % 3
            if op == ERODE:
                I, J = 255 - I, 255 - J
                want = oracle.recon_erode(I, J, s.conn)
            elif op == FILL:
                want = oracle.fill_holes(I, s.conn)
                J = np.zeros_like(I)
            else:
                want = oracle.recon(I, J, s.conn)
            dI, dJ = dev(I), dev(J)
            keep.append((dI, dJ))
            wants.append(want)
            tiles.append((dI.data_ptr(), dJ.data_ptr(), s.H, s.W, s.W, s.conn, op))
        rc.check(rc.recon_batch(c, tiles), "recon_batch")
        for t, (want, (_, dJ)) in enumerate(zip(wants, keep)):
            np.testing.assert_array_equal(dJ.cpu().numpy(), want, err_msg="tile %d op %d" % (t, t % 3))
    finally:
        rc.recon_free(c)


def test_host_entry_point_fill_holes():
    """recon_batch_host with FillHoles tiles: J is output only (not uploaded)."""
    import paper_1311_0378_gb300.build as b
    b.build()
    spec = synth.workload("single512").tiles[0]
    I, _ = synth.tile_pair(spec, 1)
    I = np.ascontiguousarray(I[:300, :411])
    J = np.full(I.shape, 7, np.uint8)
    c = rc.recon_init(0, 0, 0)
    try:
        tile = (I.ctypes.data, J.ctypes.data, I.shape[0], I.shape[1], I.shape[1], 4, FILL)
        rc.check(rc.recon_batch_host(c, [tile]), "recon_batch_host")
    finally:
        rc.recon_free(c)
    np.testing.assert_array_equal(J, oracle.fill_holes(I, 4))


@pytest.mark.parametrize("conn", [4, 8])
def test_full_size_4096(ctx, conn):
    """The 4096^2 mask of the bench workload at full size: FillHoles, and the
    erosion of its complemented fill-holes pair, byte for byte."""
    reset(ctx)
    w = synth.workload("single4096")
    spec = [t for t in w.tiles if t.marker == synth.FILLHOLES and t.conn == conn][0]
    I, J = synth.tile_pair(spec, w.seed)
    np.testing.assert_array_equal(gpu_op(ctx, I, None, conn, FILL), oracle.fill_holes(I, conn))
    Ic, Jc = 255 - I, 255 - J
    np.testing.assert_array_equal(gpu_op(ctx, Ic, Jc, conn, ERODE), oracle.recon_erode(Ic, Jc, conn))
