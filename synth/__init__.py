"""Seeded synthetic inputs for grayscale reconstruction (mask I, marker J).

Input source only: no step of the reconstruction lives here. The CUDA path's
tests and benchmark and the CPU oracle's tests both draw their tiles from this
module, so both sides see identical bytes.

The five workload families follow the tile sizes, blob law and marker types of
the nuclei-segmentation study this library serves (4K x 4K tiles of brain-tumour
slides, Sec. V); the slides themselves are replaced by noise plus Gaussian blobs
(the recipe is in ``synth.c``'s header).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

HDOME, FILLHOLES = 0, 1
PURPOSE_PARAMS = 3


class _Desc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int),
                ("nblobs", ctypes.c_int), ("rmin", ctypes.c_int), ("rmax", ctypes.c_int),
                ("marker", ctypes.c_int), ("pad", ctypes.c_int), ("tile", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compiles libsynth.so next to its source (plain C, host only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.synth_batch.argtypes = [ctypes.c_int, ctypes.POINTER(_Desc),
                                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                  ctypes.c_uint64, ctypes.c_int]
        L.synth_batch.restype = ctypes.c_int
        L.synth_stream.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.synth_stream.restype = ctypes.c_uint64
        L.synth_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.synth_u64.restype = ctypes.c_uint64
        _lib = L
    return _lib


@dataclass(frozen=True)
class TileSpec:
    H: int
    W: int
    nblobs: int
    rmin: int
    rmax: int
    marker: int   # HDOME or FILLHOLES
    conn: int     # 4 or 8
    tile: int     # index inside the seed's family


@dataclass(frozen=True)
class Workload:
    name: str
    seed: int
    tiles: Tuple[TileSpec, ...]

    @property
    def pixels(self) -> int:
        return sum(t.H * t.W for t in self.tiles)


def _u(seed: int, tile: int, n: int) -> int:
    L = lib()
    return int(L.synth_u64(L.synth_stream(seed, tile, PURPOSE_PARAMS), n))


def _uneven_tiles(seed: int, n: int, conn: int = 8) -> Tuple[TileSpec, ...]:
    """H, W each uniform in {256, 512, ..., 4096}; blobs uniform in [0, H*W/1000];
    radius 3..20; marker h-dome or fill-holes with probability 1/2 each."""
    out = []
    for t in range(n):
        H = 256 * (1 + _u(seed, t, 1) % 16)
        W = 256 * (1 + _u(seed, t, 2) % 16)
        nb = _u(seed, t, 3) % (round(H * W / 1000) + 1)
        out.append(TileSpec(H, W, nb, 3, 20, _u(seed, t, 4) & 1, conn, t))
    return tuple(out)


def _batch64_tiles(n: int) -> Tuple[TileSpec, ...]:
    """4096 x 4096 tiles, blobs uniform in [0, H*W/1000], r 4..12, 8-conn,
    marker h-dome or fill-holes with probability 1/2 each (seed 3)."""
    tiles = []
    for t in range(n):
        nb = _u(3, t, 3) % (round(4096 * 4096 / 1000) + 1)
        tiles.append(TileSpec(4096, 4096, nb, 4, 12, _u(3, t, 4) & 1, 8, t))
    return tuple(tiles)


def scaled_workload(name: str, copies: int) -> Workload:
    """The workload's family with `copies` times as many tiles (weak scaling
    across GPUs): batch64 and uneven1000 continue their tile sequences (tile
    indices 0 .. copies * n - 1 of the same seed, so copies = 1 is the workload
    itself); single512 and single4096 repeat their tiles."""
    w = workload(name)
    if copies == 1:
        return w
    if copies < 1:
        raise ValueError("copies must be >= 1")
    if name == "batch64":
        return Workload(name, w.seed, _batch64_tiles(64 * copies))
    if name == "uneven1000":
        return Workload(name, w.seed, _uneven_tiles(w.seed, 1000 * copies))
    return Workload(name, w.seed, w.tiles * copies)


def workload(name: str) -> Workload:
    """The named synthetic workloads.

    single512     512x512, 300 blobs r 4..12, 8-conn, h-dome, seed 1
    single4096    4096x4096, 6711 blobs (1 per 2500 px) r 4..12, seed 2; four runs:
                  conn {4, 8} x marker {h-dome, fill-holes} on the same mask
    batch64       64 tiles 4096x4096, blobs uniform in [0, H*W/1000], r 4..12,
                  marker h-dome/fill-holes 50/50 per tile, 8-conn, seed 3
    uneven1000    1000 tiles, H, W uniform in {256..4096 step 256}, r 3..20,
                  blobs uniform in [0, H*W/1000], markers 50/50, 8-conn, seed 4
    train20k      20000 tiles drawn like uneven1000, seed 5 (cost-model training)
    eval1000      1000 tiles drawn like uneven1000, seed 6 (cost-model evaluation)
    """
    if name == "single512":
        return Workload(name, 1, (TileSpec(512, 512, 300, 4, 12, HDOME, 8, 0),))
    if name == "single4096":
        nb = round(4096 * 4096 / 2500)
        return Workload(name, 2, tuple(TileSpec(4096, 4096, nb, 4, 12, m, c, 0)
                                       for c in (4, 8) for m in (HDOME, FILLHOLES)))
    if name == "batch64":
        return Workload(name, 3, _batch64_tiles(64))
    if name == "uneven1000":
        return Workload(name, 4, _uneven_tiles(4, 1000))
    if name == "train20k":
        return Workload(name, 5, _uneven_tiles(5, 20000))
    if name == "eval1000":
        return Workload(name, 6, _uneven_tiles(6, 1000))
    raise KeyError(name)


def generate_into(specs: Sequence[TileSpec], seed: int, I_ptrs: Sequence[int],
                  J_ptrs: Sequence[int], pitches: Optional[Sequence[int]] = None,
                  nthreads: Optional[int] = None) -> None:
    """Writes the tiles into caller-owned host buffers given by address."""
    n = len(specs)
    D = (_Desc * max(n, 1))()
    for i, s in enumerate(specs):
        D[i] = _Desc(s.H, s.W, pitches[i] if pitches else s.W, s.nblobs, s.rmin, s.rmax,
                     s.marker, 0, s.tile)
    Ip = (ctypes.c_void_p * max(n, 1))(*I_ptrs)
    Jp = (ctypes.c_void_p * max(n, 1))(*J_ptrs)
    nt = nthreads or min(os.cpu_count() or 1, 64)
    rc = lib().synth_batch(n, D, Ip, Jp, ctypes.c_uint64(seed), nt)
    if rc != 0:
        raise RuntimeError("synth_batch failed with code %d" % rc)


def generate(specs: Sequence[TileSpec], seed: int,
             nthreads: Optional[int] = None) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Returns [(I, J)] as contiguous uint8 arrays of shape (H, W)."""
    out = [(np.empty((s.H, s.W), np.uint8), np.empty((s.H, s.W), np.uint8)) for s in specs]
    generate_into(specs, seed, [I.ctypes.data for I, _ in out], [J.ctypes.data for _, J in out],
                  nthreads=nthreads)
    return out


def tile_pair(spec: TileSpec, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    return generate([spec], seed, nthreads=1)[0]


def with_marker(spec: TileSpec, marker: int) -> TileSpec:
    return replace(spec, marker=marker)
