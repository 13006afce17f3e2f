"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for
bit. Reconstruction is integer max/min only, so the bar is exact equality.

R is unique (every monotone schedule reaches the same least fixed point), so
every block shape, scan count, band count, grid size and packing order must
return identical bytes.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1311_0378_gb300.build as b
    b.build()
    c = rc.recon_init(0, torch.cuda.current_stream().cuda_stream, rc.RECON_FLAG_SYNC)
    yield c
    rc.recon_free(c)


@pytest.fixture
def fresh_ctx():
    c = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    yield c
    rc.recon_free(c)


def dev(a):
    """Device copy, complete before the library's own stream touches it."""
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    torch.cuda.synchronize()
    return t


def gpu_recon(c, I, J, conn, params=None):
    """Reconstructs one tile through recon_run; returns R as numpy."""
    for k, v in (params or {}).items():
        rc.check(rc.recon_set_param(c, k, v), "set_param")
    dI, dJ = dev(I), dev(J)
    st = rc.recon_run(c, dI.data_ptr(), dJ.data_ptr(), I.shape[0], I.shape[1], conn)
    rc.check(st, "recon_run")
    return dJ.cpu().numpy()


DEFAULTS = {rc.RECON_P_BLOCK_H: 64, rc.RECON_P_SWEEPS: 1, rc.RECON_P_BANDS: 4, rc.RECON_P_GRID: 0,
            rc.RECON_P_ORDER: 1, rc.RECON_P_TMA: 1}


def reset(c):
    for k, v in DEFAULTS.items():
        rc.check(rc.recon_set_param(c, k, v))


def test_single512_hdome_8conn(ctx):
    spec = synth.workload("single512").tiles[0]
    I, J = synth.tile_pair(spec, 1)
    np.testing.assert_array_equal(gpu_recon(ctx, I, J, 8), oracle.recon(I, J, 8))


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("marker", [synth.HDOME, synth.FILLHOLES])
def test_single512_both(ctx, conn, marker):
    reset(ctx)
    spec = synth.with_marker(synth.workload("single512").tiles[0], marker)
    I, J = synth.tile_pair(spec, 1)
    np.testing.assert_array_equal(gpu_recon(ctx, I, J, conn), oracle.recon(I, J, conn))


SHAPES = [(1, 1), (1, 129), (129, 1), (3, 3), (37, 53), (64, 128), (65, 129), (130, 257),
          (257, 130), (300, 1000), (1000, 31)]


@pytest.mark.parametrize("shape", SHAPES)
def test_ragged_shapes(ctx, shape):
    reset(ctx)
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W)
    I = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    I = np.where(rng.random((H, W)) < 0.25, 0, I).astype(np.uint8)   # walls
    markers = [np.where(rng.random((H, W)) < 0.02, I, 0).astype(np.uint8),
               np.maximum(I.astype(int) - 10, 0).astype(np.uint8)]
    fh = np.zeros_like(I)
    fh[0, :], fh[-1, :], fh[:, 0], fh[:, -1] = I[0, :], I[-1, :], I[:, 0], I[:, -1]
    markers.append(fh)
    for J in markers:
        for conn in (4, 8):
            np.testing.assert_array_equal(gpu_recon(ctx, I, J, conn), oracle.recon(I, J, conn))


def test_golden_fixtures(ctx):
    import glob
    import os
    import test_oracle_pins as pins
    reset(ctx)
    for path in sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.txt"))):
        conns, b = pins.read_golden(path)
        for conn in conns:
            np.testing.assert_array_equal(gpu_recon(ctx, b["I"], b["J"], conn), b["R"], err_msg=path)


VARIANTS = [
    {rc.RECON_P_BLOCK_H: 32}, {rc.RECON_P_BLOCK_H: 128},
    {rc.RECON_P_SWEEPS: -1}, {rc.RECON_P_SWEEPS: 0}, {rc.RECON_P_SWEEPS: 4},
    {rc.RECON_P_BANDS: 1}, {rc.RECON_P_BANDS: 2},
    {rc.RECON_P_GRID: 1}, {rc.RECON_P_GRID: 3}, {rc.RECON_P_GRID: 7, rc.RECON_P_BLOCK_H: 32},
    {rc.RECON_P_SWEEPS: -1, rc.RECON_P_BLOCK_H: 128, rc.RECON_P_BANDS: 1},
    {rc.RECON_P_TMA: 0}, {rc.RECON_P_TMA: 0, rc.RECON_P_BLOCK_H: 128},
    {rc.RECON_P_TMA: 0, rc.RECON_P_SWEEPS: -1, rc.RECON_P_BLOCK_H: 32},
]


@pytest.mark.parametrize("vi", range(len(VARIANTS)))
def test_schedule_independence(ctx, vi):
    """Uniqueness of R: every schedule returns identical bytes."""
    reset(ctx)
    base = synth.workload("single512").tiles[0]
    for marker in (synth.HDOME, synth.FILLHOLES):
        I, J = synth.tile_pair(synth.with_marker(base, marker), 1)
        for conn in (4, 8):
            got = gpu_recon(ctx, I, J, conn, VARIANTS[vi])
            np.testing.assert_array_equal(got, oracle.recon(I, J, conn))
    reset(ctx)


def test_batch_mixed_sizes_and_pitches(ctx):
    reset(ctx)
    specs = [synth.TileSpec(H, W, nb, 3, 20, m, conn, t) for t, (H, W, nb, m, conn) in enumerate([
        (256, 256, 60, 0, 8), (512, 768, 300, 1, 8), (37, 1000, 20, 1, 4), (700, 130, 50, 0, 4),
        (1, 500, 0, 1, 8), (300, 300, 90, 1, 8), (129, 129, 10, 0, 8), (1024, 256, 200, 1, 4)])]
    pitches = [s.W + pad for s, pad in zip(specs, [0, 64, 3, 1, 0, 16, 7, 0])]
    hosts = [(np.zeros((s.H, p), np.uint8), np.zeros((s.H, p), np.uint8)) for s, p in zip(specs, pitches)]
    synth.generate_into(specs, 17, [a.ctypes.data for a, _ in hosts], [b.ctypes.data for _, b in hosts],
                        pitches=pitches)
    devs = [(dev(a), dev(b)) for a, b in hosts]
    tiles = [(dI.data_ptr(), dJ.data_ptr(), s.H, s.W, p, s.conn) for (dI, dJ), s, p in zip(devs, specs, pitches)]
    rc.check(rc.recon_batch(ctx, tiles), "recon_batch")
    for (dI, dJ), (hI, hJ), s, p in zip(devs, hosts, specs, pitches):
        got = dJ.cpu().numpy()
        want = oracle.recon(hI[:, :s.W], hJ[:, :s.W], s.conn)
        np.testing.assert_array_equal(got[:, :s.W], want)
        np.testing.assert_array_equal(got[:, s.W:], hJ[:, s.W:])   # padding untouched
    work = rc.recon_get_work(ctx, len(specs))
    assert all(w["visits"] >= 1 for w in work)


def test_batch_order_and_variants(ctx):
    reset(ctx)
    specs = synth.workload("uneven1000").tiles[:12]
    specs = [synth.TileSpec(max(1, s.H // 8), max(1, s.W // 8), s.nblobs // 64, s.rmin, s.rmax,
                            s.marker, s.conn, s.tile) for s in specs]
    pairs = synth.generate(specs, 4)
    want = [oracle.recon(I, J, s.conn) for (I, J), s in zip(pairs, specs)]
    rng = np.random.default_rng(0)
    for trial in range(3):
        devs = [(dev(I), dev(J)) for I, J in pairs]
        tiles = [(dI.data_ptr(), dJ.data_ptr(), s.H, s.W, s.W, s.conn) for (dI, dJ), s in zip(devs, specs)]
        variant = rng.integers(-1, 4, size=len(specs)).tolist()
        order = rng.permutation(len(specs)).tolist()
        rc.check(rc.recon_batch_ex(ctx, tiles, variant, order), "recon_batch_ex")
        for (dI, dJ), w in zip(devs, want):
            np.testing.assert_array_equal(dJ.cpu().numpy(), w)


def test_repeated_batch_replays_graph(ctx):
    reset(ctx)
    spec = synth.with_marker(synth.workload("single512").tiles[0], synth.FILLHOLES)
    I, J = synth.tile_pair(spec, 1)
    want = oracle.recon(I, J, 8)
    dI, dJ = dev(I), dev(J)
    J0 = dJ.clone()
    for _ in range(3):
        dJ.copy_(J0)
        torch.cuda.synchronize()
        rc.check(rc.recon_batch(ctx, [(dI.data_ptr(), dJ.data_ptr(), 512, 512, 512, 8)]))
        np.testing.assert_array_equal(dJ.cpu().numpy(), want)


def test_marker_violation_reports_tile(ctx):
    reset(ctx)
    specs = [synth.TileSpec(200, 300, 40, 3, 9, 0, 8, t) for t in range(4)]
    pairs = synth.generate(specs, 5)
    pairs[2][1][100, 150] = min(255, int(pairs[2][0][100, 150]) + 1)   # J > I at one pixel
    devs = [(dev(I), dev(J)) for I, J in pairs]
    tiles = [(dI.data_ptr(), dJ.data_ptr(), 200, 300, 300, 8) for dI, dJ in devs]
    assert rc.recon_batch(ctx, tiles) == rc.RECON_EMARKER
    assert rc.recon_last_error_tile(ctx) == 2
    for t in (0, 1, 3):   # the other tiles are still reconstructed
        np.testing.assert_array_equal(devs[t][1].cpu().numpy(), oracle.recon(*pairs[t], 8))


def test_invalid_arguments(ctx):
    dI = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = dI.data_ptr()
    assert rc.recon_run(ctx, p, p + 8, 2, 4, 6) == rc.RECON_EINVAL
    assert rc.recon_run(ctx, p, p + 8, 0, 4, 8) == rc.RECON_EINVAL
    assert rc.recon_run(ctx, 0, p, 2, 4, 8) == rc.RECON_EINVAL
    assert rc.recon_batch(ctx, [(p, p + 8, 2, 4, 3, 8)]) == rc.RECON_EINVAL   # pitch < W
    assert rc.recon_set_param(ctx, rc.RECON_P_BLOCK_H, 48) == rc.RECON_EINVAL
    assert rc.recon_batch_ex(ctx, [(p, p + 8, 2, 4, 4, 8)], None, [1]) == rc.RECON_EINVAL


def test_bounded_wait_reports_timeout(fresh_ctx):
    """A phantom unit of work that never finishes: every CTA's idle wait must
    run out after the configured limit, and the status must say so; the
    context stays usable afterwards."""
    c = fresh_ctx
    I, J = synth.tile_pair(synth.TileSpec(64, 128, 5, 3, 6, 0, 8, 0), 1)
    rc.check(rc.recon_set_param(c, rc.RECON_P_WAIT_NS, 20_000_000))
    rc.check(rc.recon_set_param(c, rc.RECON_P_TEST_STALL, 1))
    dI, dJ = dev(I), dev(J)
    st = rc.recon_run(c, dI.data_ptr(), dJ.data_ptr(), 64, 128, 8)
    assert st == rc.RECON_ETIMEOUT
    rc.check(rc.recon_set_param(c, rc.RECON_P_TEST_STALL, 0))
    np.testing.assert_array_equal(gpu_recon(c, I, J, 8), oracle.recon(I, J, 8))


def test_host_entry_points(fresh_ctx):
    c = fresh_ctx
    specs = [synth.TileSpec(300, 400, 60, 3, 12, 1, 8, 0), synth.TileSpec(129, 77, 9, 3, 12, 0, 4, 1)]
    pairs = synth.generate(specs, 8)
    I0, J0 = pairs[0]
    R = J0.copy()
    rc.check(rc.recon_run_host(c, I0.ctypes.data, R.ctypes.data, 300, 400, 8), "run_host")
    np.testing.assert_array_equal(R, oracle.recon(I0, J0, 8))
    outs = [J.copy() for _, J in pairs]
    tiles = [(I.ctypes.data, o.ctypes.data, s.H, s.W, s.W, s.conn) for (I, _), o, s in zip(pairs, outs, specs)]
    rc.check(rc.recon_batch_host(c, tiles), "batch_host")
    for (I, J), o, s in zip(pairs, outs, specs):
        np.testing.assert_array_equal(o, oracle.recon(I, J, s.conn))


def test_single4096_all_runs(ctx):
    """Full-size tile, 4- and 8-connectivity x h-dome and fill-holes markers."""
    reset(ctx)
    w = synth.workload("single4096")
    pairs = synth.generate(w.tiles, w.seed)
    want, _ = oracle.recon_tiles(pairs, [s.conn for s in w.tiles], "sweep")
    for (I, J), s, R in zip(pairs, w.tiles, want):
        np.testing.assert_array_equal(gpu_recon(ctx, I, J, s.conn), R)


def test_allocation_failure_is_reported_and_context_recovers(fresh_ctx):
    """A host batch whose device copy cannot fit (about 600 GB) fails with
    RECON_ENOMEM before any copy or launch (the host buffers are never read),
    and the same context then reconstructs normally."""
    small = np.zeros(64, np.uint8)
    huge = (small.ctypes.data, small.ctypes.data, 550000, 550000, 550000, 8)
    assert rc.recon_batch_host(fresh_ctx, [huge]) == rc.RECON_ENOMEM
    spec = synth.workload("single512").tiles[0]
    I, J = synth.tile_pair(spec, 1)
    np.testing.assert_array_equal(gpu_recon(fresh_ctx, I, J, 8), oracle.recon(I, J, 8))


def test_environment_overrides():
    """RECON_* environment variables set the context defaults; a bad value
    fails recon_init (checked in a child process with its own environment)."""
    import os
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_1311_0378_gb300 as rc\n"
            "try:\n    c = rc.recon_init(0, 0, 0)\nexcept rc.ReconError as e:\n    print('status', e.status); sys.exit(0)\n"
            "print(rc.recon_get_param(c, rc.RECON_P_BLOCK_H), rc.recon_get_param(c, rc.RECON_P_SCAN_GAIN))\n"
            "rc.recon_free(c)\n" % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    env = dict(os.environ, RECON_BLOCK_H="32", RECON_SCAN_GAIN="256")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120).stdout
    assert out.split() == ["32", "256"]
    env["RECON_BLOCK_H"] = "96"
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120).stdout
    assert out.split() == ["status", str(rc.RECON_EINVAL)]


def test_back_to_back_batches_without_sync():
    """Two different batches, then the first again (a graph replay), issued
    without a host wait in between: the staging buffer of the tile descriptors
    is released right after its copy, so the host stages the next batch while
    the previous kernel may still run. Every result is bit-exact."""
    c = rc.recon_init(0, 0, 0)   # asynchronous context
    try:
        specs_a = [synth.TileSpec(512, 384, 80, 3, 20, m, 8, t) for t, m in enumerate((1, 0, 1))]
        specs_b = [synth.TileSpec(300, 700, 60, 3, 20, m, 4, t) for t, m in enumerate((0, 1))]
        pa, pb = synth.generate(specs_a, 21), synth.generate(specs_b, 22)
        want_a = [oracle.recon(I, J, 8) for I, J in pa]
        want_b = [oracle.recon(I, J, 4) for I, J in pb]
        da = [(dev(I), dev(J)) for I, J in pa]
        db = [(dev(I), dev(J)) for I, J in pb]
        da2 = [(dev(I), dev(J)) for I, J in pa]
        ta = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, 8) for (I, J), s in zip(da, specs_a)]
        tb = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, 4) for (I, J), s in zip(db, specs_b)]
        ta2 = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, 8) for (I, J), s in zip(da2, specs_a)]
        rc.check(rc.recon_batch(c, ta), "batch a")
        rc.check(rc.recon_batch(c, tb), "batch b")
        rc.check(rc.recon_batch(c, ta2), "batch a again")
        rc.check(rc.recon_batch(c, ta2), "batch a, graph replay on its own output (a fixed point)")
        rc.check(rc.recon_sync(c), "sync")
        for (_, J), w in zip(da, want_a):
            np.testing.assert_array_equal(J.cpu().numpy(), w)
        for (_, J), w in zip(db, want_b):
            np.testing.assert_array_equal(J.cpu().numpy(), w)
        for (_, J), w in zip(da2, want_a):
            np.testing.assert_array_equal(J.cpu().numpy(), w)
    finally:
        rc.recon_free(c)
