"""Pins for the CPU oracle: checks against things other than the oracle itself.

* hand-worked fixtures (tests/golden, derived from the definition of
  reconstruction by dilation, Table II after Vincent 1993);
* brute-force Jacobi iteration of the geodesic dilation min(delta(J), I) to a
  fixed point, written here in NumPy (the definition itself);
* exhaustive small cases: every (I, J) pair with J <= I on 2x3 images over
  {0..3}, and every 3x3 mask over {0..3} with a seeded marker;
* an independent exact algorithm (maximum-bottleneck flood) on synthetic tiles;
* special cases that reduce to textbook or library routines (J = I, J = 0,
  constant masks, binary images via scipy.ndimage.label);
* invariants J <= R <= I, stability under one more dilation, idempotence;
* planted mistakes in a copy of the oracle's C source must fail these pins.
"""
import ctypes
import glob
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

OFFS4 = [(-1, 0), (1, 0), (0, -1), (0, 1)]
OFFS8 = OFFS4 + [(-1, -1), (-1, 1), (1, -1), (1, 1)]


def brute(I, J, conn):
    """Iterates X <- min(max over the closed neighbourhood of X, I) over whole
    arrays (leading axes are independent images) until nothing changes."""
    I = I.astype(np.int16)
    X = J.astype(np.int16)
    H, W = X.shape[-2:]
    pad = [(0, 0)] * (X.ndim - 2) + [(1, 1), (1, 1)]
    while True:
        P = np.pad(X, pad)  # outside the image contributes 0, the identity of max
        m = X.copy()
        for dy, dx in (OFFS8 if conn == 8 else OFFS4):
            m = np.maximum(m, P[..., 1 + dy:1 + dy + H, 1 + dx:1 + dx + W])
        Y = np.minimum(m, I)
        if np.array_equal(Y, X):
            return X.astype(np.uint8)
        X = Y


def pack(cases, per_row):
    """Lays N small h x w images on one canvas with zero gutters (I = 0 there,
    so nothing crosses a gutter, for 4- and 8-connectivity alike)."""
    n, h, w = cases.shape
    rows = -(-n // per_row)
    canvas = np.zeros((rows * (h + 1), per_row * (w + 1)), np.uint8)
    idx = np.arange(n)
    r, c = idx // per_row, idx % per_row
    for dy in range(h):
        for dx in range(w):
            canvas[r * (h + 1) + dy, c * (w + 1) + dx] = cases[:, dy, dx]
    return canvas


def unpack(canvas, n, h, w, per_row):
    idx = np.arange(n)
    r, c = idx // per_row, idx % per_row
    out = np.empty((n, h, w), np.uint8)
    for dy in range(h):
        for dx in range(w):
            out[:, dy, dx] = canvas[r * (h + 1) + dy, c * (w + 1) + dx]
    return out


def read_golden(path):
    blocks, conn, cur = {}, None, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("conn"):
                conn = line.split()[1]
            elif line in ("I", "J", "R"):
                cur = line
                blocks[cur] = []
            else:
                blocks[cur].append([int(v) for v in line.split()])
    conns = (4, 8) if conn == "both" else (int(conn),)
    return conns, {k: np.array(v, np.uint8) for k, v in blocks.items()}


GOLDEN_FILES = sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


def test_golden_files_present():
    assert len(GOLDEN_FILES) >= 6


# ---------------------------------------------------------------------------
# the pin suite, parameterised by the reconstruction under test so that the
# planted-mistake tests can run it against a broken copy of the oracle

def pin_failures(recon_fn, quick=False):
    fails = []
    for path in GOLDEN_FILES:
        conns, b = read_golden(path)
        for conn in conns:
            if not np.array_equal(recon_fn(b["I"], b["J"], conn), b["R"]):
                fails.append("golden %s conn %d" % (os.path.basename(path), conn))
    rng = np.random.default_rng(7)
    for k in range(60 if quick else 300):
        h, w = rng.integers(1, 17, size=2)
        hi = int(rng.choice([2, 4, 16, 256]))
        I = rng.integers(0, hi, size=(h, w)).astype(np.uint8)
        J = np.minimum(rng.integers(0, hi, size=(h, w)), I).astype(np.uint8)
        if k % 3 == 0:
            J = np.where(rng.random((h, w)) < 0.1, J, 0).astype(np.uint8)
        for conn in (4, 8):
            if not np.array_equal(recon_fn(I, J, conn), brute(I, J, conn)):
                fails.append("random %d conn %d" % (k, conn))
    # every 3x3 mask over {0..3} (a strided subset when quick), seeded marker
    vals = np.array(np.meshgrid(*[np.arange(4)] * 9, indexing="ij")).reshape(9, -1).T
    if quick:
        vals = vals[::37]
    Is = vals.reshape(-1, 3, 3).astype(np.uint8)
    Js = np.minimum(np.random.default_rng(11).integers(0, 4, size=Is.shape), Is).astype(np.uint8)
    Js = np.where(np.random.default_rng(12).random(Is.shape) < 0.35, Js, 0).astype(np.uint8)
    per_row = 512
    for conn in (4, 8):
        got = unpack(recon_fn(pack(Is, per_row), pack(Js, per_row), conn), len(Is), 3, 3, per_row)
        if not np.array_equal(got, brute(Is, Js, conn)):
            fails.append("3x3 masks conn %d" % conn)
    return fails


def test_oracle_passes_pins():
    assert pin_failures(oracle.recon) == []


def test_exhaustive_2x3_pairs():
    """Every (I, J) with J <= I on a 2x3 image over {0..3}: 10^6 cases."""
    pair_vals = np.array([(i, j) for i in range(4) for j in range(i + 1)], np.uint8)  # 10 per pixel
    idx = np.array(np.meshgrid(*[np.arange(10)] * 6, indexing="ij")).reshape(6, -1).T
    Is = pair_vals[idx, 0].reshape(-1, 2, 3)
    Js = pair_vals[idx, 1].reshape(-1, 2, 3)
    per_row = 1000
    for conn in (4, 8):
        got = unpack(oracle.recon(pack(Is, per_row), pack(Js, per_row), conn), len(Is), 2, 3, per_row)
        np.testing.assert_array_equal(got, brute(Is, Js, conn))


def test_golden_by_widest_and_brute():
    for path in GOLDEN_FILES:
        conns, b = read_golden(path)
        for conn in conns:
            np.testing.assert_array_equal(brute(b["I"], b["J"], conn), b["R"])
            np.testing.assert_array_equal(oracle.recon_widest(b["I"], b["J"], conn), b["R"])


@pytest.mark.parametrize("marker", [synth.HDOME, synth.FILLHOLES])
@pytest.mark.parametrize("conn", [4, 8])
def test_widest_flood_agrees_with_sweeps(marker, conn):
    spec = synth.with_marker(synth.workload("single512").tiles[0], marker)
    I, J = synth.tile_pair(spec, 1)
    np.testing.assert_array_equal(oracle.recon(I, J, conn), oracle.recon_widest(I, J, conn))


def test_widest_vs_brute_random():
    rng = np.random.default_rng(3)
    for _ in range(100):
        h, w = rng.integers(1, 40, size=2)
        I = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
        J = np.where(rng.random((h, w)) < 0.05, I, 0).astype(np.uint8)
        for conn in (4, 8):
            np.testing.assert_array_equal(oracle.recon_widest(I, J, conn), brute(I, J, conn))


def test_special_cases():
    rng = np.random.default_rng(5)
    I = rng.integers(0, 256, size=(37, 53)).astype(np.uint8)
    for conn in (4, 8):
        np.testing.assert_array_equal(oracle.recon(I, I, conn), I)                 # J = I
        np.testing.assert_array_equal(oracle.recon(I, np.zeros_like(I), conn), 0)   # J = 0
        C = np.full((19, 23), 77, np.uint8)                                         # constant mask
        J = np.zeros_like(C)
        J[7, 11] = 77
        np.testing.assert_array_equal(oracle.recon(C, J, conn), C)
        J[7, 11] = 30                                                               # lower source
        np.testing.assert_array_equal(oracle.recon(C, J, conn), 30)


@pytest.mark.parametrize("conn", [4, 8])
def test_binary_equals_connected_components(conn):
    """Binary I, J in {0, 255}: R = union of the components of {I = 255} that
    meet {J = 255} (components from scipy.ndimage.label)."""
    rng = np.random.default_rng(conn)
    for density in (0.45, 0.6, 0.75):
        fg = rng.random((120, 97)) < density
        I = np.where(fg, 255, 0).astype(np.uint8)
        J = np.where(fg & (rng.random(fg.shape) < 0.01), 255, 0).astype(np.uint8)
        struct = ndimage.generate_binary_structure(2, 2 if conn == 8 else 1)
        lab, _ = ndimage.label(fg, structure=struct)
        keep = np.unique(lab[J == 255])
        want = np.where(np.isin(lab, keep[keep > 0]), 255, 0).astype(np.uint8)
        np.testing.assert_array_equal(oracle.recon(I, J, conn), want)


@pytest.mark.parametrize("marker", [synth.HDOME, synth.FILLHOLES])
@pytest.mark.parametrize("conn", [4, 8])
def test_invariants_on_synthetic_tile(marker, conn):
    spec = synth.with_marker(synth.workload("single512").tiles[0], marker)
    I, J = synth.tile_pair(spec, 1)
    R, pairs = oracle.recon(I, J, conn, return_pairs=True)
    assert pairs >= 2
    assert (J <= R).all() and (R <= I).all()
    R2, changed = oracle.dilate_step(I, R, conn)       # stability
    assert not changed and np.array_equal(R2, R)
    np.testing.assert_array_equal(oracle.recon(I, R, conn), R)   # idempotence
    assert (R != J).any()                                # something propagated


def test_marker_above_mask_is_rejected():
    I = np.full((4, 4), 10, np.uint8)
    J = I.copy()
    J[2, 2] = 11
    with pytest.raises(ValueError):
        oracle.recon(I, J, 8)
    with pytest.raises(ValueError):
        oracle.recon(I, I, 6)


# ---------------------------------------------------------------------------
# planted mistakes: each edit of a copy of the oracle's source must break a pin

MUTANTS = {
    "dropped diagonal term": ("if (x > 0) m = u8max(m, J[p - W - 1]);", ""),
    "wrong diagonal index": ("m = u8max(m, J[p + W + 1]);", "m = u8max(m, J[p + W]);"),
    "max instead of min with the mask": ("uint8_t v = u8min(m, I[p]);\n            if (v != J[p]) { J[p] = v; changed = 1; }\n        }\n    return changed;\n}\n\n/* Anti",
                                         "uint8_t v = u8max(m, I[p]);\n            if (v != J[p]) { J[p] = v; changed = 1; }\n        }\n    return changed;\n}\n\n/* Anti"),
    "single pair only": ("if (!c1 && !c2) break;", "break;"),
    "anti-raster drops the right neighbour": ("if (x < W - 1) m = u8max(m, J[p + 1]);", ""),
    "transposed row stride": ("m = u8max(m, J[p - W]);", "m = u8max(m, J[p - 1]);"),
}


def _mutant_runner(so_path):
    L = ctypes.CDLL(so_path)
    L.oracle_recon.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_void_p]

    def mut(I, J, conn):
        I = np.ascontiguousarray(I, np.uint8)
        R = np.array(J, np.uint8, order="C", copy=True)
        if L.oracle_recon(I.ctypes.data, R.ctypes.data, I.shape[0], I.shape[1], conn, None) != 0:
            raise RuntimeError("status")
        return R

    return 1 if pin_failures(mut, quick=True) else 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_pins(name, tmp_path):
    """The mutant runs in a child process: a mutant whose sweeps never settle
    (e.g. max in place of min with the mask) is caught by the time limit."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "recon_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, "mutation site not found: " + name
    src = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(so), str(c)])
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_oracle_pins as T; sys.exit(T._mutant_runner(%r))"
            % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
               os.path.dirname(os.path.abspath(__file__)), str(so)))
    try:
        rc = subprocess.run([sys.executable, "-c", code], timeout=15).returncode
    except subprocess.TimeoutExpired:
        rc = "timeout"
    assert rc != 0, "planted mistake not caught: " + name
