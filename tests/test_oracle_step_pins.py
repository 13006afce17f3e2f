"""Pins for the oracle's one-step operators and for Adam beyond its first step.

* ``oracle.dilate_step`` / ``oracle.erode_step`` (one whole-image geodesic
  dilation min(delta(X), I), and its dual max(eps(X), I); Table II after
  Vincent 1993) against scipy.ndimage's grey dilation / erosion with the
  4- or 8-connected closed structuring element, a library routine that shares
  nothing with the oracle. Pixels outside the image are absent: constant 0 for
  the dilation (the identity of max) and 255 for the erosion (that of min).
  Every shape class is covered, including 1 x 1, 1 x N and N x 1, and the
  "changed" flag must say whether any byte moved.
* Planted mistakes in a copy of the step functions' C source must fail those
  pins (the invariant tests call these steps to check stability, so a step
  that silently ignores a neighbour would hide a wrong R there).
* Adam (Kingma & Ba 2015, Algorithm 1) under a constant gradient g has the
  closed form m_hat_t = g and v_hat_t = g^2 for every t, so
  theta_t = theta_0 - t * lr * g / (|g| + eps); checked for t = 1 .. 10, and a
  bias correction that drops the power of t must fail it.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import mlp

FOOT = {4: ndimage.generate_binary_structure(2, 1), 8: ndimage.generate_binary_structure(2, 2)}

SHAPES = [(1, 1), (1, 2), (2, 1), (1, 17), (23, 1), (2, 2), (3, 3), (5, 64), (64, 5), (31, 47), (64, 97)]


def lib_dilate_step(I, X, conn):
    """min(delta(X), I) by scipy: grey dilation over the closed neighbourhood."""
    d = ndimage.grey_dilation(X, footprint=FOOT[conn], mode="constant", cval=0)
    return np.minimum(d, I).astype(np.uint8)


def lib_erode_step(I, X, conn):
    """max(eps(X), I) by scipy: grey erosion over the closed neighbourhood."""
    e = ndimage.grey_erosion(X, footprint=FOOT[conn], mode="constant", cval=255)
    return np.maximum(e, I).astype(np.uint8)


def cases(seed=11):
    """(I, X) pairs of every shape class: random bytes, few levels, and
    sparse markers (a step from a sparse X moves many pixels)."""
    rng = np.random.default_rng(seed)
    out = []
    for h, w in SHAPES:
        for hi in (4, 256):
            I = rng.integers(0, hi, size=(h, w)).astype(np.uint8)
            X = rng.integers(0, hi, size=(h, w)).astype(np.uint8)
            Xs = np.where(rng.random((h, w)) < 0.15, X, 0).astype(np.uint8)
            out += [(I, X), (I, Xs), (I, np.full((h, w), 255, np.uint8) - Xs)]
    return out


def step_failures(dstep, estep):
    """Names of the cases where a pair of step functions disagrees with the
    library definition (value or changed flag)."""
    fails = []
    for i, (I, X) in enumerate(cases()):
        for conn in (4, 8):
            for name, fn, ref in (("dilate", dstep, lib_dilate_step), ("erode", estep, lib_erode_step)):
                want = ref(I, X, conn)
                got, changed = fn(I, X, conn)
                if not np.array_equal(got, want):
                    fails.append("%s case %d %s conn %d" % (name, i, I.shape, conn))
                elif bool(changed) != bool((want != X).any()):
                    fails.append("%s flag case %d conn %d" % (name, i, conn))
    return fails


def test_steps_match_library_grey_morphology():
    assert step_failures(oracle.dilate_step, oracle.erode_step) == []


def test_step_leaves_input_untouched_and_is_not_in_place():
    """Each step is one Jacobi update of the whole image: a raised pixel must
    not feed its right / lower neighbours within the same step."""
    I = np.full((1, 6), 9, np.uint8)
    X = np.array([[7, 0, 0, 0, 0, 0]], np.uint8)
    Y, changed = oracle.dilate_step(I, X, 4)
    assert changed and Y.tolist() == [[7, 7, 0, 0, 0, 0]] and X.tolist() == [[7, 0, 0, 0, 0, 0]]
    Z, changed = oracle.erode_step(np.zeros((6, 1), np.uint8), (255 - X).T.copy(), 8)
    assert changed and Z.ravel().tolist() == [248, 248, 255, 255, 255, 255]


# ---------------------------------------------------------------------------
# planted mistakes in the step functions

STEP_MUTANTS = {
    "dilate: one diagonal dropped": ("oracle_dilate_step",
                                     "if (conn == 4 && dy != 0 && dx != 0) continue;",
                                     "if ((conn == 4 || dy + dx == 2) && dy != 0 && dx != 0) continue;"),
    "dilate: updated in place": ("oracle_dilate_step", "m = u8max(m, old[", "m = u8max(m, X["),
    "dilate: last column skipped": ("oracle_dilate_step", "xx >= W", "xx >= W - 1"),
    "dilate: no clamp by the mask": ("oracle_dilate_step", "uint8_t v = u8min(m, I[(size_t)y * W + x]);",
                                     "uint8_t v = m; (void)I;"),
    "dilate: open neighbourhood": ("oracle_dilate_step", "if (conn == 4 && dy != 0 && dx != 0) continue;",
                                   "if ((conn == 4 && dy != 0 && dx != 0) || (dy == 0 && dx == 0)) continue;"),
    "dilate: changed flag lost": ("oracle_dilate_step", "changed = 1;", "changed = 0;"),
    "erode: one diagonal dropped": ("oracle_erode_step",
                                    "if (conn == 4 && dy != 0 && dx != 0) continue;",
                                    "if ((conn == 4 || dy - dx == 2) && dy != 0 && dx != 0) continue;"),
    "erode: transposed row stride": ("oracle_erode_step", "old[(size_t)yy * W + xx]", "old[(size_t)xx * W + yy]"),
    "erode: first row skipped": ("oracle_erode_step", "yy < 0 ||", "yy < 1 ||"),
    "erode: min for max with the mask": ("oracle_erode_step", "uint8_t v = u8max(m, I[(size_t)y * W + x]);",
                                         "uint8_t v = u8min(m, I[(size_t)y * W + x]);"),
}


def _mutate(src, func, old, new):
    """Replaces `old` by `new` once, inside the body of C function `func` only."""
    start = src.index("int %s(" % func)
    end = src.index("\n}\n", start)
    body = src[start:end]
    assert old in body, "mutation site not found in %s: %s" % (func, old)
    return src[:start] + body.replace(old, new, 1) + src[end:]


def _load_steps(so):
    L = ctypes.CDLL(str(so))
    for f in (L.oracle_dilate_step, L.oracle_erode_step):
        f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        f.restype = ctypes.c_int

    def wrap(fn):
        def step(I, X, conn):
            I = np.ascontiguousarray(I, np.uint8)
            Y = np.array(X, np.uint8, order="C", copy=True)
            rc = fn(I.ctypes.data, Y.ctypes.data, I.shape[0], I.shape[1], conn)
            if rc < 0:
                raise ValueError("status %d" % -rc)
            return Y, bool(rc)
        return step

    return wrap(L.oracle_dilate_step), wrap(L.oracle_erode_step)


def test_unmutated_copy_passes(tmp_path):
    """The harness itself: an unedited copy compiled the same way passes."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "recon_oracle.c")).read()
    c, so = tmp_path / "same.c", tmp_path / "libsame.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(so), str(c)])
    assert step_failures(*_load_steps(so)) == []


@pytest.mark.parametrize("name", sorted(STEP_MUTANTS))
def test_planted_step_mistake_fails_pins(name, tmp_path):
    func, old, new = STEP_MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "recon_oracle.c")).read()
    bad = _mutate(src, func, old, new)
    c, so = tmp_path / "mut.c", tmp_path / "libmut.so"
    c.write_text(bad)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(so), str(c)])
    assert step_failures(*_load_steps(so)), "planted mistake not caught: " + name


# ---------------------------------------------------------------------------
# Adam beyond the first step

G_CONST = np.array([3.0, -0.5, 1e-3, -2e-2, 0.0])


def adam_closed_form_failures(step_fn, lr=0.01, eps=1e-8, steps=10):
    """Constant gradient g from theta_0 = 0: m_t = (1 - beta1^t) g and
    v_t = (1 - beta2^t) g^2, so both bias-corrected moments are exact and
    theta_t = -t * lr * g / (|g| + eps)."""
    th = np.zeros_like(G_CONST)
    m = np.zeros_like(G_CONST)
    v = np.zeros_like(G_CONST)
    fails = []
    for t in range(1, steps + 1):
        th, m, v = step_fn(th, G_CONST.copy(), m, v, t, lr=lr, eps=eps)
        want = -t * lr * G_CONST / (np.abs(G_CONST) + eps)
        if not np.allclose(th, want, rtol=1e-12, atol=1e-15):
            fails.append(t)
        if not np.allclose(m, (1 - 0.9 ** t) * G_CONST, rtol=1e-12, atol=0):
            fails.append(("m", t))
        if not np.allclose(v, (1 - 0.999 ** t) * G_CONST ** 2, rtol=1e-12, atol=0):
            fails.append(("v", t))
    return fails


def test_adam_constant_gradient_closed_form():
    assert adam_closed_form_failures(mlp.adam_step) == []


def test_adam_alternating_gradient_hand_worked():
    """g_1 = +1, g_2 = -1 (beta1 0.9, beta2 0.999): m_2 = 0.9 * 0.1 - 0.1 = -0.01,
    m_hat_2 = -0.01 / 0.19; v_2 = 0.999 * 0.001 + 0.001 = 0.001999,
    v_hat_2 = 1. theta_2 = -lr * 1 - lr * (-0.01 / 0.19) / 1 (eps -> 0)."""
    lr = 0.1
    th, m, v = mlp.adam_step(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, lr=lr, eps=0.0)
    th, m, v = mlp.adam_step(th, -np.ones(1), m, v, 2, lr=lr, eps=0.0)
    np.testing.assert_allclose(m, [-0.01], rtol=1e-12)
    np.testing.assert_allclose(v, [0.001999], rtol=1e-12)
    np.testing.assert_allclose(th, [-lr + lr * 0.01 / 0.19], rtol=1e-12)


ADAM_PLANTS = {
    "first moment bias correction without the power of t":
        lambda s: s.replace("mhat = m / (1 - beta1 ** t)", "mhat = m / (1 - beta1)"),
    "second moment bias correction without the power of t":
        lambda s: s.replace("vhat = v / (1 - beta2 ** t)", "vhat = v / (1 - beta2)"),
    "step count off by one":
        lambda s: s.replace("mhat = m / (1 - beta1 ** t)", "mhat = m / (1 - beta1 ** (t + 1))"),
    "gradient squared left out":
        lambda s: s.replace("(1 - beta2) * grad * grad", "(1 - beta2) * np.abs(grad)"),
}


@pytest.mark.parametrize("name", sorted(ADAM_PLANTS))
def test_planted_adam_mistake_fails_closed_form(name):
    import inspect
    import types
    src = inspect.getsource(mlp)
    bad = ADAM_PLANTS[name](src)
    assert bad != src
    mod = types.ModuleType("mlp_bad")
    exec(compile(bad, "mlp_bad", "exec"), mod.__dict__)
    assert adam_closed_form_failures(mod.adam_step) or _alternating_fails(mod.adam_step), \
        "planted mistake not caught: " + name


def _alternating_fails(step_fn):
    lr = 0.1
    th, m, v = step_fn(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, lr=lr, eps=0.0)
    th, m, v = step_fn(th, -np.ones(1), m, v, 2, lr=lr, eps=0.0)
    return not np.allclose(th, [-lr + lr * 0.01 / 0.19], rtol=1e-12)
