"""Pins for the oracle's reconstruction by erosion and FillHoles, against
things other than the oracle itself.

* hand-worked fixtures (tests/golden/erosion, tests/golden/fill_holes);
* brute-force Jacobi iteration of the geodesic erosion max(eps(X), I) to a
  fixed point, written here in NumPy (the definition itself);
* every 3x3 mask over {0..3} with a seeded marker above it;
* duality with the (separately pinned) reconstruction by dilation:
  R^eps_I(J) = 255 - R^delta_{255-I}(255-J);
* FillHoles two ways: the complement form of the oracle and the erosion form
  (marker I on the border, 255 inside), plus binary images against
  scipy.ndimage.binary_fill_holes;
* invariants I <= R <= J, stability, idempotence, F >= I;
* planted mistakes in a copy of the oracle's erosion code must fail these pins.
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
from test_oracle_pins import OFFS4, OFFS8, pack, read_golden, unpack

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EROSION_FILES = sorted(glob.glob(os.path.join(GOLDEN, "erosion", "*.txt")))
FILL_FILES = sorted(glob.glob(os.path.join(GOLDEN, "fill_holes", "*.txt")))


def brute_erode(I, J, conn):
    """Iterates X <- max(min over the closed neighbourhood of X, I) over whole
    arrays (leading axes are independent images) until nothing changes.
    Absent neighbours are padded with 255, the identity of min."""
    I = I.astype(np.int16)
    X = J.astype(np.int16)
    H, W = X.shape[-2:]
    pad = [(0, 0)] * (X.ndim - 2) + [(1, 1), (1, 1)]
    while True:
        P = np.pad(X, pad, constant_values=255)
        m = X.copy()
        for dy, dx in (OFFS8 if conn == 8 else OFFS4):
            m = np.minimum(m, P[..., 1 + dy:1 + dy + H, 1 + dx:1 + dx + W])
        Y = np.maximum(m, I)
        if np.array_equal(Y, X):
            return X.astype(np.uint8)
        X = Y


def border_marker(I):
    """I on the one-pixel image border, 255 inside: the erosion form of FillHoles."""
    F = np.full_like(I, 255)
    F[0, :], F[-1, :], F[:, 0], F[:, -1] = I[0, :], I[-1, :], I[:, 0], I[:, -1]
    return F


def read_fill(path):
    blocks, conn, cur = {}, None, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("conn"):
                conn = int(line.split()[1])
            elif line in ("I", "F"):
                cur = line
                blocks[cur] = []
            else:
                blocks[cur].append([int(v) for v in line.split()])
    return conn, {k: np.array(v, np.uint8) for k, v in blocks.items()}


def test_fixture_files_present():
    assert len(EROSION_FILES) >= 3 and len(FILL_FILES) >= 4


def erode_pin_failures(erode_fn, quick=False):
    fails = []
    for path in EROSION_FILES:
        conns, b = read_golden(path)
        for conn in conns:
            if not np.array_equal(erode_fn(b["I"], b["J"], conn), b["R"]):
                fails.append("golden %s conn %d" % (os.path.basename(path), conn))
    rng = np.random.default_rng(17)
    for k in range(60 if quick else 300):
        h, w = rng.integers(1, 17, size=2)
        hi = int(rng.choice([2, 4, 16, 256]))
        I = rng.integers(0, hi, size=(h, w)).astype(np.uint8)
        J = np.maximum(rng.integers(0, hi, size=(h, w)), I).astype(np.uint8)
        if k % 3 == 0:
            J = np.where(rng.random((h, w)) < 0.1, J, 255).astype(np.uint8)
        for conn in (4, 8):
            if not np.array_equal(erode_fn(I, J, conn), brute_erode(I, J, conn)):
                fails.append("random %d conn %d" % (k, conn))
    vals = np.array(np.meshgrid(*[np.arange(4)] * 9, indexing="ij")).reshape(9, -1).T
    if quick:
        vals = vals[::37]
    Is = vals.reshape(-1, 3, 3).astype(np.uint8)
    Js = np.maximum(np.random.default_rng(21).integers(0, 4, size=Is.shape), Is).astype(np.uint8)
    Js = np.where(np.random.default_rng(22).random(Is.shape) < 0.35, Js, 3).astype(np.uint8)
    per_row = 512
    for conn in (4, 8):
        # gutters between the packed images: I = J = 3 there, the largest value,
        # so no lower value crosses a gutter
        inside = pack(np.ones_like(Is), per_row).astype(bool)
        cI = np.where(inside, pack(Is, per_row), 3).astype(np.uint8)
        cJ = np.where(inside, pack(Js, per_row), 3).astype(np.uint8)
        got = unpack(erode_fn(cI, cJ, conn), len(Is), 3, 3, per_row)
        if not np.array_equal(got, brute_erode(Is, Js, conn)):
            fails.append("3x3 masks conn %d" % conn)
    return fails


def test_erosion_oracle_passes_pins():
    assert erode_pin_failures(oracle.recon_erode) == []


def test_erosion_golden_by_brute():
    for path in EROSION_FILES:
        conns, b = read_golden(path)
        for conn in conns:
            np.testing.assert_array_equal(brute_erode(b["I"], b["J"], conn), b["R"])


@pytest.mark.parametrize("marker", [synth.HDOME, synth.FILLHOLES])
@pytest.mark.parametrize("conn", [4, 8])
def test_duality_with_dilation(marker, conn):
    """R^eps_I(J) = 255 - R^delta_{255-I}(255-J) on a synthetic 512^2 tile:
    the dilation tile (I, J) complemented gives an erosion tile."""
    spec = synth.with_marker(synth.workload("single512").tiles[0], marker)
    I, J = synth.tile_pair(spec, 1)
    Ic, Jc = 255 - I, 255 - J
    R = oracle.recon_erode(Ic, Jc, conn)
    np.testing.assert_array_equal(R, 255 - oracle.recon(I, J, conn))
    assert (Ic <= R).all() and (R <= Jc).all() and (R != Jc).any()


@pytest.mark.parametrize("conn", [4, 8])
def test_erosion_invariants(conn):
    rng = np.random.default_rng(30 + conn)
    I = rng.integers(0, 200, size=(97, 131)).astype(np.uint8)
    J = np.where(rng.random(I.shape) < 0.02, I, 255).astype(np.uint8)
    R, pairs = oracle.recon_erode(I, J, conn, return_pairs=True)
    assert pairs >= 2
    assert (I <= R).all() and (R <= J).all()
    R2, changed = oracle.erode_step(I, R, conn)
    assert not changed and np.array_equal(R2, R)
    np.testing.assert_array_equal(oracle.recon_erode(I, R, conn), R)


def test_erosion_special_cases():
    rng = np.random.default_rng(9)
    I = rng.integers(0, 256, size=(37, 53)).astype(np.uint8)
    for conn in (4, 8):
        np.testing.assert_array_equal(oracle.recon_erode(I, I, conn), I)                  # J = I
        np.testing.assert_array_equal(oracle.recon_erode(I, np.full_like(I, 255), conn), 255)
        C = np.full((19, 23), 77, np.uint8)
        J = np.full_like(C, 255)
        J[7, 11] = 100                                                                     # one lower source
        np.testing.assert_array_equal(oracle.recon_erode(C, J, conn), 100)


def test_erosion_marker_below_mask_is_rejected():
    I = np.full((4, 4), 10, np.uint8)
    J = I.copy()
    J[1, 3] = 9
    with pytest.raises(ValueError):
        oracle.recon_erode(I, J, 8)


@pytest.mark.parametrize("path", FILL_FILES, ids=os.path.basename)
def test_fill_holes_golden(path):
    conn, b = read_fill(path)
    np.testing.assert_array_equal(oracle.fill_holes(b["I"], conn), b["F"])
    np.testing.assert_array_equal(brute_erode(b["I"], border_marker(b["I"]), conn), b["F"])


@pytest.mark.parametrize("conn", [4, 8])
def test_fill_holes_binary_equals_scipy(conn):
    """Binary images in {0, 255}: FillHoles = scipy.ndimage.binary_fill_holes
    with the background connected by the same neighbourhood."""
    rng = np.random.default_rng(40 + conn)
    struct = ndimage.generate_binary_structure(2, 2 if conn == 8 else 1)
    for density in (0.35, 0.5, 0.65):
        fg = rng.random((90, 117)) < density
        I = np.where(fg, 255, 0).astype(np.uint8)
        want = np.where(ndimage.binary_fill_holes(fg, structure=struct), 255, 0).astype(np.uint8)
        got = oracle.fill_holes(I, conn)
        np.testing.assert_array_equal(got, want)
        assert (got != I).any()   # some holes were filled


@pytest.mark.parametrize("conn", [4, 8])
def test_fill_holes_erosion_form_and_invariants(conn):
    spec = synth.workload("single512").tiles[0]
    I, _ = synth.tile_pair(spec, 1)
    F = oracle.fill_holes(I, conn)
    np.testing.assert_array_equal(F, oracle.recon_erode(I, border_marker(I), conn))
    assert (F >= I).all() and (F != I).any()
    np.testing.assert_array_equal(oracle.fill_holes(F, conn), F)                  # idempotent
    np.testing.assert_array_equal(F[0, :], I[0, :])                               # border kept
    np.testing.assert_array_equal(F[:, -1], I[:, -1])


# ---------------------------------------------------------------------------
# planted mistakes in the erosion code

MUTANTS = {
    "erosion: max of neighbours instead of min": ("if (x > 0) m = u8min(m, J[p - 1]);",
                                                  "if (x > 0) m = u8max(m, J[p - 1]);"),
    "erosion: dropped diagonal term": ("if (x > 0) m = u8min(m, J[p - W - 1]);", ""),
    "erosion: wrong anti-raster diagonal": ("if (x > 0) m = u8min(m, J[p + W - 1]);",
                                            "if (x > 0) m = u8min(m, J[p + W]);"),
    "erosion: single pair only": ("int c2 = antiraster_erode(I, J, H, W, conn);\n        ++n;\n        if (!c1 && !c2) break;",
                                  "int c2 = antiraster_erode(I, J, H, W, conn);\n        ++n;\n        break;"),
    "erosion: min with the mask": ("uint8_t v = u8max(m, I[p]);", "uint8_t v = u8min(m, I[p]);"),
}


def _mutant_runner(so_path):
    L = ctypes.CDLL(so_path)
    L.oracle_recon_erode.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p]

    def mut(I, J, conn):
        I = np.ascontiguousarray(I, np.uint8)
        R = np.array(J, np.uint8, order="C", copy=True)
        if L.oracle_recon_erode(I.ctypes.data, R.ctypes.data, I.shape[0], I.shape[1], conn, None) != 0:
            raise RuntimeError("status")
        return R

    return 1 if erode_pin_failures(mut, quick=True) else 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_erosion_mistake_fails_pins(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "recon_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, "mutation site not found: " + name
    src = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(so), str(c)])
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import test_oracle_pins_dual as T; sys.exit(T._mutant_runner(%r))"
            % (os.path.dirname(here), here, str(so)))
    try:
        rc = subprocess.run([sys.executable, "-c", code], timeout=15).returncode
    except subprocess.TimeoutExpired:
        rc = "timeout"
    assert rc != 0, "planted mistake not caught: " + name
