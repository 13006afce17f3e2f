"""Property-based pins for the oracle (hypothesis; skipped where it is not
installed): order-theoretic facts of reconstruction that hold for every input
and that a plausible mistake breaks.

* dilation: J <= R <= I; R is a fixed point of one more geodesic dilation;
  increasing in the marker and in the mask; R_I(J) = R_I(R_I(J)); the result
  for the union (pixel max) of two markers is the max of the two results;
* erosion: the dual statements (I <= R <= J, decreasing in the marker's
  complement, min over markers);
* FillHoles: F >= I, idempotent, equal to I on the image border, increasing in I;
* distance transform: zero exactly on the background, and adding background
  pixels never increases a distance.
"""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402
from hypothesis.extra import numpy as hnp  # noqa: E402

SETTINGS = dict(max_examples=60, deadline=None)


@st.composite
def mask_and_markers(draw):
    h = draw(st.integers(1, 12))
    w = draw(st.integers(1, 12))
    hi = draw(st.sampled_from([2, 4, 16, 256]))
    I = draw(hnp.arrays(np.uint8, (h, w), elements=st.integers(0, hi - 1)))
    A = draw(hnp.arrays(np.uint8, (h, w), elements=st.integers(0, hi - 1)))
    B = draw(hnp.arrays(np.uint8, (h, w), elements=st.integers(0, hi - 1)))
    conn = draw(st.sampled_from([4, 8]))
    return I, np.minimum(A, I), np.minimum(B, I), conn


@settings(**SETTINGS)
@given(mask_and_markers())
def test_dilation_order_properties(case):
    I, J1, J2, conn = case
    R1 = oracle.recon(I, J1, conn)
    R2 = oracle.recon(I, J2, conn)
    assert (J1 <= R1).all() and (R1 <= I).all()
    assert not oracle.dilate_step(I, R1, conn)[1]                       # fixed point
    np.testing.assert_array_equal(oracle.recon(I, R1, conn), R1)         # idempotent
    np.testing.assert_array_equal(oracle.recon(I, np.maximum(J1, J2), conn), np.maximum(R1, R2))
    Jlo = np.minimum(J1, J2)
    assert (oracle.recon(I, Jlo, conn) <= R1).all()                      # increasing in the marker
    I2 = np.maximum(I, (I.astype(int) + 3).clip(0, 255).astype(np.uint8) * (I % 2 == 0))
    assert (oracle.recon(I2, J1, conn) >= R1).all()                      # increasing in the mask


@settings(**SETTINGS)
@given(mask_and_markers())
def test_erosion_order_properties(case):
    I, J1, J2, conn = case
    Ic, K1, K2 = 255 - I, 255 - J1, 255 - J2      # erosion pairs: K >= Ic
    E1 = oracle.recon_erode(Ic, K1, conn)
    E2 = oracle.recon_erode(Ic, K2, conn)
    assert (Ic <= E1).all() and (E1 <= K1).all()
    assert not oracle.erode_step(Ic, E1, conn)[1]
    np.testing.assert_array_equal(oracle.recon_erode(Ic, np.minimum(K1, K2), conn), np.minimum(E1, E2))


@settings(**SETTINGS)
@given(mask_and_markers())
def test_fill_holes_properties(case):
    I, _, _, conn = case
    F = oracle.fill_holes(I, conn)
    assert (F >= I).all()
    np.testing.assert_array_equal(oracle.fill_holes(F, conn), F)
    np.testing.assert_array_equal(F[0, :], I[0, :])
    np.testing.assert_array_equal(F[-1, :], I[-1, :])
    np.testing.assert_array_equal(F[:, 0], I[:, 0])
    np.testing.assert_array_equal(F[:, -1], I[:, -1])
    Iup = np.maximum(I, np.roll(I, 1, axis=1))
    assert (oracle.fill_holes(Iup, conn) >= F).all()                     # increasing in I


@settings(**SETTINGS)
@given(hnp.arrays(np.uint8, st.tuples(st.integers(1, 14), st.integers(1, 14)), elements=st.integers(0, 1)),
       st.integers(0, 10 ** 6))
def test_distance_transform_properties(B, seed):
    site, d2 = oracle.distance_transform(B)
    if not (B == 0).any():
        assert (site == -1).all()
        return
    assert ((d2 == 0) == (B == 0)).all()
    rng = np.random.default_rng(seed)
    B2 = np.where(rng.random(B.shape) < 0.2, 0, B).astype(np.uint8)     # more background
    _, d2b = oracle.distance_transform(B2)
    # exact-up-to-bound distances can only shrink when background is added
    ex1 = np.sqrt(d2.astype(float))
    ex2 = np.sqrt(d2b.astype(float))
    assert (ex2 <= ex1 + 0.5).all()
