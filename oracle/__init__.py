"""CPU oracle for grayscale morphological reconstruction (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package. The library never does, and the two share no code: the oracle is
plain C (``recon_oracle.c``) plus NumPy for the cost model (``mlp.py``).

Functions follow the definition of reconstruction by dilation (Table II,
"Morphological Reconstruction", after Vincent 1993): R = lim delta_I^n(J) with
delta_I(X)(p) = min(max_{q in N(p)} X(q), I(p)), N(p) the closed 4- or
8-neighbourhood inside the image. ``recon_erode`` is the dual (max and min
exchanged, J >= I), and ``fill_holes`` is Table II's FillHoles: a flood of the
background from the image border, written as complement -> reconstruction by
dilation from the border -> complement.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recon_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "dt_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EMARKER, ENOMEM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compiles liboracle.so (plain C, -O2, no vector intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, *_SRCS])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u8p = ctypes.c_void_p
        L.oracle_recon.argtypes = [u8p, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]
        L.oracle_recon_widest.argtypes = [u8p, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_dilate_step.argtypes = [u8p, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_recon_tiles.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.oracle_recon_erode.argtypes = [u8p, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]
        L.oracle_erode_step.argtypes = [u8p, u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_dt.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_dt.restype = ctypes.c_int
        for f in (L.oracle_recon, L.oracle_recon_widest, L.oracle_dilate_step, L.oracle_recon_tiles,
                  L.oracle_recon_erode, L.oracle_erode_step):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _prep(I: np.ndarray, J: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    I = np.ascontiguousarray(I, dtype=np.uint8)
    R = np.array(J, dtype=np.uint8, order="C", copy=True)
    if I.ndim != 2 or I.shape != R.shape:
        raise ValueError("I and J must be 2-D arrays of one shape")
    return I, R


def recon(I: np.ndarray, J: np.ndarray, conn: int = 8, return_pairs: bool = False):
    """Raster / anti-raster sweeps until a full pair changes nothing.

    Returns R (a new array); J is not modified. Raises ValueError on J > I
    (status 2) or bad arguments (status 1)."""
    I, R = _prep(I, J)
    pairs = ctypes.c_int(0)
    rc = lib().oracle_recon(I.ctypes.data, R.ctypes.data, I.shape[0], I.shape[1], conn,
                            ctypes.byref(pairs))
    if rc != OK:
        raise ValueError("oracle_recon status %d" % rc)
    return (R, pairs.value) if return_pairs else R


def recon_widest(I: np.ndarray, J: np.ndarray, conn: int = 8) -> np.ndarray:
    """Maximum-bottleneck flood (exact; independent of the sweeps)."""
    I, R = _prep(I, J)
    rc = lib().oracle_recon_widest(I.ctypes.data, R.ctypes.data, I.shape[0], I.shape[1], conn)
    if rc != OK:
        raise ValueError("oracle_recon_widest status %d" % rc)
    return R


def dilate_step(I: np.ndarray, X: np.ndarray, conn: int = 8) -> Tuple[np.ndarray, bool]:
    """One whole-image geodesic dilation min(delta(X), I); returns (new X, changed)."""
    I, Y = _prep(I, X)
    rc = lib().oracle_dilate_step(I.ctypes.data, Y.ctypes.data, I.shape[0], I.shape[1], conn)
    if rc < 0:
        raise ValueError("oracle_dilate_step status %d" % -rc)
    return Y, bool(rc)


def recon_erode(I: np.ndarray, J: np.ndarray, conn: int = 8, return_pairs: bool = False):
    """Reconstruction by erosion: R = lim eps_I^n(J), eps_I(X)(p) =
    max(min_{q in N(p)} X(q), I(p)), by raster / anti-raster sweeps until a
    full pair changes nothing. Requires J >= I (ValueError, status 2,
    otherwise). Returns R; J is not modified."""
    I, R = _prep(I, J)
    pairs = ctypes.c_int(0)
    rc = lib().oracle_recon_erode(I.ctypes.data, R.ctypes.data, I.shape[0], I.shape[1], conn,
                                  ctypes.byref(pairs))
    if rc != OK:
        raise ValueError("oracle_recon_erode status %d" % rc)
    return (R, pairs.value) if return_pairs else R


def erode_step(I: np.ndarray, X: np.ndarray, conn: int = 8) -> Tuple[np.ndarray, bool]:
    """One whole-image geodesic erosion max(eps(X), I); returns (new X, changed)."""
    I, Y = _prep(I, X)
    rc = lib().oracle_erode_step(I.ctypes.data, Y.ctypes.data, I.shape[0], I.shape[1], conn)
    if rc < 0:
        raise ValueError("oracle_erode_step status %d" % -rc)
    return Y, bool(rc)


def fill_holes(I: np.ndarray, conn: int = 8) -> np.ndarray:
    """FillHoles (Table II): flood the background from the image border and
    raise every pixel the flood cannot reach (a hole) to the lowest level that
    encloses it. Definition used: C = 255 - I; marker M = C on the one-pixel
    image border, 0 inside; result = 255 - R^delta_C(M), with R^delta the
    reconstruction by dilation of ``recon``."""
    I = np.ascontiguousarray(I, dtype=np.uint8)
    if I.ndim != 2:
        raise ValueError("I must be a 2-D array")
    C = (255 - I.astype(np.int16)).astype(np.uint8)
    M = np.zeros_like(C)
    M[0, :], M[-1, :], M[:, 0], M[:, -1] = C[0, :], C[-1, :], C[:, 0], C[:, -1]
    return (255 - recon(C, M, conn).astype(np.int16)).astype(np.uint8)


def distance_transform(B: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Distance transform by irregular wavefront propagation (Table II; Algorithm
    1 with nearest-background-site elements, 8-connected, FIFO order; see
    dt_oracle.c). B: 2-D array, nonzero = foreground. Returns (site, d2):
    int32 index y*W+x of the site found for each pixel (-1 if the image has no
    background) and uint32 squared Euclidean distance to it (0 on background,
    0xFFFFFFFF without a site)."""
    B = np.ascontiguousarray(B != 0, dtype=np.uint8)
    if B.ndim != 2:
        raise ValueError("B must be a 2-D array")
    site = np.empty(B.shape, np.int32)
    d2 = np.empty(B.shape, np.uint32)
    rc = lib().oracle_dt(B.ctypes.data, B.shape[0], B.shape[1], site.ctypes.data, d2.ctypes.data)
    if rc != OK:
        raise ValueError("oracle_dt status %d" % rc)
    return site, d2


def recon_tiles(pairs: Sequence[Tuple[np.ndarray, np.ndarray]], conns: Sequence[int],
                method: str = "sweep", nthreads: int = 0) -> Tuple[List[np.ndarray], int]:
    """Reconstructs independent tiles on host threads (0 = all cores).

    Returns ([R_t], threads used). method is "sweep" or "widest" (reconstruction
    by dilation) or "erode" (reconstruction by erosion, J >= I)."""
    n = len(pairs)
    Is, Rs = [], []
    for I, J in pairs:
        a, b = _prep(I, J)
        Is.append(a)
        Rs.append(b)
    Ip = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in Is])
    Rp = (ctypes.c_void_p * max(n, 1))(*[b.ctypes.data for b in Rs])
    Hs = (ctypes.c_int * max(n, 1))(*[a.shape[0] for a in Is])
    Ws = (ctypes.c_int * max(n, 1))(*[a.shape[1] for a in Is])
    Cs = (ctypes.c_int * max(n, 1))(*conns)
    st = (ctypes.c_int * max(n, 1))()
    nt = nthreads or (os.cpu_count() or 1)
    code = {"sweep": 0, "widest": 1, "erode": 2}[method]
    used = lib().oracle_recon_tiles(n, Ip, Rp, Hs, Ws, Cs, code, nt, st)
    bad = [i for i in range(n) if st[i] != OK]
    if bad:
        raise ValueError("oracle tiles failed: %s" % [(i, st[i]) for i in bad[:5]])
    return Rs, used
