"""Pins for the distance-transform oracle (oracle/dt_oracle.c), against things
other than itself:

* the exact squared Euclidean distance transform by brute force (nearest
  background pixel over all background pixels) on small images, and by
  scipy.ndimage.distance_transform_edt on synthetic tiles;
* cases where the propagation is exact by construction (one background
  pixel; a row);
* the properties every correct result of the propagation has (shared with the
  GPU parity tests): each site is a background pixel, d2 is the squared
  distance to it, no 8-neighbour holds a strictly better site (the fixed point
  of Algorithm 1's propagation condition), and d2 is at least the exact value
  and at most DT_MAX_ERR pixels above it in distance;
* planted mistakes in a copy of the oracle's source must fail these pins.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

DT_MAX_ERR = 0.5        # pixels: bound on sqrt(d2) - exact distance
DT_MAX_INEXACT = 1e-3   # fraction of foreground pixels allowed above the exact value


def brute_d2(B):
    ys, xs = np.nonzero(B == 0)
    H, W = B.shape
    if len(ys) == 0:
        return None
    gy, gx = np.mgrid[0:H, 0:W]
    d = (gy[..., None] - ys) ** 2 + (gx[..., None] - xs) ** 2
    return d.min(axis=-1).astype(np.int64)


def dt_violations(B, site, d2, exact_d2):
    """Human-readable list of broken properties (empty when the result is valid)."""
    bad = []
    B = B != 0
    H, W = B.shape
    if not (~B).any():
        if not ((site == -1).all() and (d2 == 0xFFFFFFFF).all()):
            bad.append("no background: site -1 and d2 max expected")
        return bad
    if (site < 0).any() or (site >= H * W).any():
        return ["site out of range"]
    sy, sx = site // W, site % W
    if B.reshape(-1)[site.reshape(-1)].any():
        bad.append("a site is a foreground pixel")
    gy, gx = np.mgrid[0:H, 0:W]
    if not np.array_equal(d2.astype(np.int64), (gy - sy) ** 2 + (gx - sx) ** 2):
        bad.append("d2 is not the squared distance to the site")
    if not (site[~B] == (gy * W + gx)[~B]).all():
        bad.append("a background pixel is not its own site")
    # fixed point: no 8-neighbour offers a strictly smaller key (d2, site)
    key = d2.astype(np.int64) * (1 << 32) + site.astype(np.int64)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if not (dy or dx):
                continue
            ys0, ys1 = max(0, -dy), H - max(0, dy)
            xs0, xs1 = max(0, -dx), W - max(0, dx)
            s_n = site[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx].astype(np.int64)
            py, px = gy[ys0:ys1, xs0:xs1], gx[ys0:ys1, xs0:xs1]
            cand = ((py - s_n // W) ** 2 + (px - s_n % W) ** 2) * (1 << 32) + s_n
            fg = B[ys0:ys1, xs0:xs1]
            if (cand[fg] < key[ys0:ys1, xs0:xs1][fg]).any():
                bad.append("not a fixed point (direction %d,%d)" % (dy, dx))
    ex = exact_d2.astype(np.int64)
    if (d2.astype(np.int64) < ex).any():
        bad.append("d2 below the exact value")
    err = np.sqrt(d2.astype(np.float64)) - np.sqrt(ex.astype(np.float64))
    if err.max(initial=0.0) > DT_MAX_ERR:
        bad.append("error %.3f px above the bound" % err.max())
    if B.any() and (d2.astype(np.int64) != ex)[B].mean() > DT_MAX_INEXACT:
        bad.append("too many inexact pixels: %.5f" % (d2.astype(np.int64) != ex)[B].mean())
    return bad


def exact_d2(B):
    if not (B == 0).any():
        return np.full(B.shape, 0xFFFFFFFF, np.int64)
    return np.rint(ndimage.distance_transform_edt(B != 0) ** 2).astype(np.int64)


def dt_pin_failures(dt_fn, quick=False):
    fails = []
    # exact by construction: one background pixel; one row between two background ends
    rng = np.random.default_rng(1)
    for _ in range(10 if quick else 40):
        H, W = rng.integers(1, 30, size=2)
        B = np.ones((H, W), np.uint8)
        y, x = rng.integers(0, H), rng.integers(0, W)
        B[y, x] = 0
        site, d2 = dt_fn(B)
        if not np.array_equal(d2.astype(np.int64), brute_d2(B)):
            fails.append("single site %dx%d" % (H, W))
    site, d2 = dt_fn(np.array([[0, 1, 1, 1, 1, 1, 0]], np.uint8))
    if list(d2[0]) != [0, 1, 4, 9, 4, 1, 0]:
        fails.append("row")
    # brute force on random small images
    for k in range(40 if quick else 200):
        H, W = rng.integers(1, 28, size=2)
        B = (rng.random((H, W)) < rng.choice([0.5, 0.8, 0.95, 0.99])).astype(np.uint8)
        site, d2 = dt_fn(B)
        ex = brute_d2(B)
        if ex is None:
            ex = np.full(B.shape, 0xFFFFFFFF, np.int64)
        v = dt_violations(B, site, d2, ex)
        if v:
            fails.append("random %d: %s" % (k, v[0]))
    return fails


def test_oracle_passes_pins():
    assert dt_pin_failures(oracle.distance_transform) == []


@pytest.mark.parametrize("polarity", ["blobs", "between_blobs"])
def test_against_scipy_edt_on_synthetic_tile(polarity):
    spec = synth.workload("single512").tiles[0]
    I, _ = synth.tile_pair(spec, 1)
    B = ((I >= 100) if polarity == "blobs" else (I < 100)).astype(np.uint8)
    site, d2 = oracle.distance_transform(B)
    assert dt_violations(B, site, d2, exact_d2(B)) == []
    assert d2.max() > (4 if polarity == "blobs" else 400)


def test_no_background_and_no_foreground():
    site, d2 = oracle.distance_transform(np.ones((3, 4), np.uint8))
    assert (site == -1).all() and (d2 == 0xFFFFFFFF).all()
    site, d2 = oracle.distance_transform(np.zeros((3, 4), np.uint8))
    assert (d2 == 0).all() and (site.reshape(-1) == np.arange(12)).all()


MUTANTS = {
    "4 of 8 directions": ("for (int k = 0; k < 8; ++k) {", "for (int k = 0; k < 4; ++k) {"),
    "transposed stride": ("int64_t qy = q / W, qx = q % W, sy = s / W, sx = s % W;",
                          "int64_t qy = q % W, qx = q / W, sy = s / W, sx = s % W;"),
    "distance without the x term": ("(qx - sx) * (qx - sx)", "0"),
    "keeps the first site found": ("if (key_of(W, r, s) < key_of(W, r, site[r])) {", "if (site[r] < 0) {"),
}


def _mutant_runner(so_path):
    L = ctypes.CDLL(so_path)
    L.oracle_dt.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]

    def mut(B):
        B = np.ascontiguousarray(B != 0, dtype=np.uint8)
        site = np.empty(B.shape, np.int32)
        d2 = np.empty(B.shape, np.uint32)
        if L.oracle_dt(B.ctypes.data, B.shape[0], B.shape[1], site.ctypes.data, d2.ctypes.data) != 0:
            raise RuntimeError("status")
        return site, d2

    return 1 if dt_pin_failures(mut, quick=True) else 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_pins(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dt_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, "mutation site not found: " + name
    src = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(c)])
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_dt_oracle_pins as T; sys.exit(T._mutant_runner(%r))"
            % (os.path.dirname(here), here, str(so)))
    try:
        rc = subprocess.run([sys.executable, "-c", code], timeout=15).returncode
    except subprocess.TimeoutExpired:
        rc = "timeout"
    assert rc != 0, "planted mistake not caught: " + name
