"""GPU parity for the distance transform (Table II) through the C ABI. The
propagation's result depends on the processing order (like the oracle's, it
approximates the exact Euclidean transform), so the GPU result is checked for
what every correct result satisfies (tests/test_dt_oracle_pins.py:
dt_violations): each site is a background pixel, d2 is the squared distance
to it, no 8-neighbour holds a strictly better site, and d2 is the exact value
up to a bounded error on a bounded fraction of pixels. Pixels next to the
background, and images with one background pixel, must match exactly."""
import numpy as np
import pytest

import oracle
import synth
from test_dt_oracle_pins import brute_d2, dt_violations, exact_d2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1311_0378_gb300.build as b
    b.build()
    c = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    yield c
    rc.recon_free(c)


def gpu_dt(c, B, want_site=True):
    H, W = B.shape
    dB = torch.from_numpy(np.ascontiguousarray(B != 0, dtype=np.uint8)).cuda()
    d2 = torch.empty((H, W), dtype=torch.int32, device="cuda")
    site = torch.empty((H, W), dtype=torch.int32, device="cuda") if want_site else None
    torch.cuda.synchronize()
    rc.check(rc.recon_dt(c, dB.data_ptr(), d2.data_ptr(), site.data_ptr() if want_site else 0, H, W), "recon_dt")
    d2n = d2.cpu().numpy().view(np.uint32)
    return (site.cpu().numpy() if want_site else None), d2n


SHAPES = [(1, 1), (1, 37), (41, 1), (3, 3), (17, 29), (64, 64), (130, 257), (300, 111)]


@pytest.mark.parametrize("shape", SHAPES)
def test_random_images_vs_brute_force(ctx, shape):
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W)
    for density in (0.5, 0.8, 0.95, 0.995):
        B = (rng.random((H, W)) < density).astype(np.uint8)
        site, d2 = gpu_dt(ctx, B)
        ex = brute_d2(B) if H * W <= 40000 else exact_d2(B)
        if ex is None:
            ex = np.full(B.shape, 0xFFFFFFFF, np.int64)
        assert dt_violations(B, site, d2, ex) == [], (shape, density)
        # next to the background the answer is unique: 1 or 2
        near = (B != 0) & (ex <= 2)
        np.testing.assert_array_equal(d2[near].astype(np.int64), ex[near])


def test_single_background_pixel_is_exact(ctx):
    rng = np.random.default_rng(5)
    for _ in range(8):
        H, W = rng.integers(2, 300, size=2)
        B = np.ones((H, W), np.uint8)
        B[rng.integers(0, H), rng.integers(0, W)] = 0
        _, d2 = gpu_dt(ctx, B, want_site=False)
        np.testing.assert_array_equal(d2.astype(np.int64), exact_d2(B))


@pytest.mark.parametrize("polarity", ["blobs", "between_blobs"])
@pytest.mark.parametrize("workload", ["single512", "single4096"])
def test_synthetic_masks(ctx, polarity, workload):
    """Objects = blob pixels (I >= 100) of the synthetic tiles, or the space
    between them; against scipy's exact transform and the CPU oracle."""
    spec = synth.workload(workload).tiles[0]
    I, _ = synth.tile_pair(spec, synth.workload(workload).seed)
    B = ((I >= 100) if polarity == "blobs" else (I < 100)).astype(np.uint8)
    site, d2 = gpu_dt(ctx, B)
    ex = exact_d2(B)
    assert dt_violations(B, site, d2, ex) == []
    if workload == "single512":
        _, od2 = oracle.distance_transform(B)
        assert (od2 == d2).mean() > 0.999


def test_degenerate_images(ctx):
    site, d2 = gpu_dt(ctx, np.ones((5, 9), np.uint8))
    assert (site == -1).all() and (d2 == 0xFFFFFFFF).all()
    site, d2 = gpu_dt(ctx, np.zeros((5, 9), np.uint8))
    assert (d2 == 0).all() and (site.reshape(-1) == np.arange(45)).all()
    assert rc.recon_dt(ctx, 0, 0, 0, 5, 9) == rc.RECON_EINVAL
    dB = torch.zeros(4, dtype=torch.uint8, device="cuda")
    assert rc.recon_dt(ctx, dB.data_ptr(), dB.data_ptr(), 0, 40000, 1) == rc.RECON_EINVAL
