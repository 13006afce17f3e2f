"""Pins for the micro-benchmark oracle (oracle/microbench.py): its SplitMix64
against the input generator's own C implementation (synth) and against a
pure-Python big-integer restatement; its read checksum and write result
against plain Python loops."""
import numpy as np

import synth
from oracle import microbench as mbo

MASK = (1 << 64) - 1


def splitmix_py(seed, n):
    z = (seed + n * 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_splitmix_matches_synth_and_python():
    L = synth.lib()
    for seed in (0, 1, 12345, 0xDEADBEEFCAFEF00D, MASK):
        ns = np.array([1, 2, 3, 1000, 10 ** 9, 2 ** 40 + 7], dtype=np.uint64)
        got = mbo.splitmix64(seed, ns)
        for n, g in zip(ns, got):
            assert int(g) == splitmix_py(seed, int(n)) == int(L.synth_u64(seed, int(n)))


def test_indices_in_range_and_spread():
    idx = np.concatenate(list(mbo.indices(10, 200000, 7, chunk=65536)))
    assert idx.dtype == np.uint64 and len(idx) == 200000
    assert int(idx.max()) < 1024
    counts = np.bincount(idx.astype(np.int64), minlength=1024)
    assert counts.min() > 100 and counts.max() < 300   # expected ~195 per bin
    first = [splitmix_py(7, k + 1) >> 54 for k in range(5)]
    assert [int(v) for v in idx[:5]] == first


def test_read_checksum_and_write_result_by_loops():
    rng = np.random.default_rng(3)
    log2n, ops, seed = 12, 5000, 99
    M = rng.integers(0, 2 ** 32, size=1 << log2n, dtype=np.uint64).astype(np.uint32)
    want_sum, want_M = 0, [int(v) for v in M]
    for k in range(ops):
        i = splitmix_py(seed, k + 1) >> (64 - log2n)
        want_sum = (want_sum + int(M[i])) & MASK
        want_M[i] = ((i * 0x9E3779B1) & 0xFFFFFFFF) ^ 0x5A5A5A5A
    assert mbo.random_read_checksum(M, log2n, ops, seed) == want_sum
    np.testing.assert_array_equal(mbo.random_write_result(M, log2n, ops, seed), np.array(want_M, np.uint32))
