"""CPU oracle for the device micro-benchmarks (TEST INFRASTRUCTURE ONLY:
imported by the tests and the benchmark, never by the library).

The micro-benchmarks are the paper's Table III (random reads / writes of 32-bit
integers in a matrix) and Table IV (atomic adds on one variable or on an array
indexed by thread). What they compute is fixed so that the GPU results can be
checked exactly:

* access k (k = 0 .. ops-1) goes to element SplitMix64(seed, k + 1) >> (64 - log2n),
  SplitMix64(s, n) being output n of the SplitMix64 generator (Steele, Lea &
  Flood 2014) seeded with s: z = s + n * 0x9E3779B97F4A7C15, then its published
  mixing steps; written here in NumPy from that definition;
* a read run returns the sum of the values read, mod 2^64;
* a write run leaves element i = (i * 0x9E3779B1 mod 2^32) xor 0x5A5A5A5A at
  every touched index and the rest unchanged;
* atomic adds of 1: counts are threads x iterations (one variable), iterations
  per element (array), threads-per-CTA x iterations per CTA (shared word).
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n) -> np.ndarray:
    """Outputs n (an array of integers >= 1) of the SplitMix64 stream seeded with seed."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.asarray(n, dtype=np.uint64) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def indices(log2n: int, ops: int, seed: int, chunk: int = 1 << 22):
    """The element indices of accesses 0 .. ops-1, in chunks (a generator)."""
    for k0 in range(0, ops, chunk):
        k = np.arange(k0 + 1, min(ops, k0 + chunk) + 1, dtype=np.uint64)
        yield splitmix64(seed, k) >> np.uint64(64 - log2n)


def written_value(idx: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        return ((idx.astype(np.uint64) * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)).astype(np.uint32) \
            ^ np.uint32(0x5A5A5A5A)


def random_read_checksum(M: np.ndarray, log2n: int, ops: int, seed: int) -> int:
    """Sum (mod 2^64) of the values the read run reads from M."""
    total = np.uint64(0)
    with np.errstate(over="ignore"):
        for idx in indices(log2n, ops, seed):
            total = total + M[idx.astype(np.int64)].astype(np.uint64).sum(dtype=np.uint64)
    return int(total)


def random_write_result(M: np.ndarray, log2n: int, ops: int, seed: int) -> np.ndarray:
    """M after the write run (a new array)."""
    out = np.array(M, dtype=np.uint32, copy=True)
    for idx in indices(log2n, ops, seed):
        i = idx.astype(np.int64)
        out[i] = written_value(idx)
    return out
