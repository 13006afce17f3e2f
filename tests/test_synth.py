"""Host-side checks of the seeded input generator (no reconstruction here)."""
import numpy as np

import synth


def test_deterministic_and_in_range():
    spec = synth.workload("single512").tiles[0]
    I1, J1 = synth.tile_pair(spec, 1)
    I2, J2 = synth.generate([spec], 1, nthreads=3)[0]
    assert np.array_equal(I1, I2) and np.array_equal(J1, J2)
    assert I1.min() >= 20 and I1.max() <= 255
    assert (I1 >= 120).sum() > 300 * 20          # the blobs are there
    I3, _ = synth.tile_pair(spec, 2)
    assert not np.array_equal(I1, I3)            # the seed matters


def test_markers():
    spec = synth.workload("single512").tiles[0]
    I, J = synth.tile_pair(spec, 1)
    assert np.array_equal(J, np.maximum(I.astype(int) - 10, 0).astype(np.uint8))
    I2, J2 = synth.tile_pair(synth.with_marker(spec, synth.FILLHOLES), 1)
    assert np.array_equal(I, I2)
    border = np.zeros_like(I, bool)
    border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
    assert np.array_equal(J2[border], I[border]) and (J2[~border] == 0).all()


def test_workload_shapes():
    w = synth.workload("single4096")
    assert len(w.tiles) == 4 and {(t.conn, t.marker) for t in w.tiles} == {(4, 0), (4, 1), (8, 0), (8, 1)}
    assert all(t.nblobs == 6711 for t in w.tiles)
    b = synth.workload("batch64")
    assert len(b.tiles) == 64 and b.pixels == 64 * 4096 * 4096
    assert 16 < sum(t.marker for t in b.tiles) < 48
    u = synth.workload("uneven1000")
    assert len(u.tiles) == 1000
    Hs = {t.H for t in u.tiles}
    assert Hs == set(range(256, 4097, 256))
    assert all(0 <= t.nblobs <= round(t.H * t.W / 1000) and t.rmin == 3 and t.rmax == 20 for t in u.tiles)
    assert 4.0e9 < u.pixels < 5.5e9


def test_pitch_and_ragged_sizes():
    spec = synth.TileSpec(37, 53, 5, 3, 6, synth.HDOME, 8, 9)
    I, J = synth.tile_pair(spec, 99)
    buf_i = np.zeros((37, 64), np.uint8)
    buf_j = np.zeros((37, 64), np.uint8)
    synth.generate_into([spec], 99, [buf_i.ctypes.data], [buf_j.ctypes.data], pitches=[64])
    assert np.array_equal(buf_i[:, :53], I) and np.array_equal(buf_j[:, :53], J)
    assert (buf_i[:, 53:] == 0).all()
