"""GPU checks of the cost-model kernels through the C ABI against the CPU
oracle (oracle/mlp.py, fp64) and against plain NumPy feature counts.

Tolerances (fp32 kernels vs fp64 oracle): every output is a sum of at most
K = 84 products (20 + 64 inputs on the longest path), each rounded once by an
FMA, so |error| <= K * 2^-24 * sum |terms| (plus the same again through the
previous layer). The tests use rtol 1e-4 and an absolute floor of 1e-5 times
the scale of the compared vector, well above that bound for these magnitudes
and far below any plausible mistake (a dropped term or a wrong index moves
values by O(1)).
"""
import numpy as np
import pytest

import synth
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    import paper_1311_0378_gb300.build as b
    b.build()
    c = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    yield c
    rc.recon_free(c)


def f32(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    torch.cuda.synchronize()
    return t


def close(got, want, rtol=1e-4):
    scale = max(1.0, float(np.abs(want).max()))
    np.testing.assert_allclose(got, want, rtol=rtol, atol=1e-5 * scale)


def numpy_features(I, J):
    I = I.astype(np.int32)
    J = J.astype(np.int32)
    px = np.float32(I.size)
    d = I - J
    f = np.zeros(20, np.float32)
    for k in range(16):
        f[k] = np.float32(np.count_nonzero((d >> 4) == k)) / px
    f[16] = np.float32(np.count_nonzero(I >= 100)) / px
    f[17] = np.float32(np.count_nonzero(J == 0)) / px
    f[18] = np.float32(np.log2(np.float32(I.shape[0])) / 12)
    f[19] = np.float32(np.log2(np.float32(I.shape[1])) / 12)
    return f


def test_features_match_numpy(ctx):
    specs = [synth.TileSpec(H, W, nb, 3, 20, m, 8, t) for t, (H, W, nb, m) in enumerate([
        (256, 256, 60, 0), (512, 768, 300, 1), (37, 1000, 20, 1), (700, 130, 50, 0), (1, 500, 0, 1)])]
    pairs = synth.generate(specs, 21)
    devs = [(torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()) for I, J in pairs]
    torch.cuda.synchronize()
    feat = torch.zeros((len(specs), 20), dtype=torch.float32, device="cuda")
    tiles = [(a.data_ptr(), b.data_ptr(), s.H, s.W, s.W, 8) for (a, b), s in zip(devs, specs)]
    rc.check(rc.recon_features(ctx, tiles, feat.data_ptr()), "features")
    got = feat.cpu().numpy()
    for t, (I, J) in enumerate(pairs):
        want = numpy_features(I, J)
        np.testing.assert_array_equal(got[t, :18], want[:18])     # exact integer counts / exact px
        np.testing.assert_allclose(got[t, 18:], want[18:], rtol=2e-7)


def test_features_of_erosion_fillholes_and_violations(ctx):
    """Erosion tiles are described by their complemented values, FillHoles tiles
    by the complemented mask with a zero marker; pixels with J > I take no
    histogram bin but count in the other features."""
    specs = [synth.TileSpec(H, W, nb, 3, 20, m, 8, t) for t, (H, W, nb, m) in enumerate([
        (256, 512, 80, 0), (300, 1024, 40, 1), (128, 256, 30, 0), (129, 257, 30, 1)])]
    pairs = synth.generate(specs, 22)
    viol = []
    for I, J in pairs[2:]:
        J = J.copy()
        J[5, :40] = np.minimum(255, I[5, :40].astype(np.int32) + 7).astype(np.uint8)   # J > I on part of a row
        viol.append((I, J, 0))
    cases = [(pairs[0][0], 255 - pairs[0][1], 1),          # erosion: J >= I
             (pairs[1][0], np.zeros_like(pairs[1][1]), 2)]  # FillHoles: J is output only
    cases += viol                                          # dilation with violations (16-byte and byte paths)
    devs = [(torch.from_numpy(np.ascontiguousarray(I)).cuda(), torch.from_numpy(np.ascontiguousarray(J)).cuda())
            for I, J, _ in cases]
    torch.cuda.synchronize()
    feat = torch.zeros((len(cases), 20), dtype=torch.float32, device="cuda")
    tiles = [(a.data_ptr(), b.data_ptr(), I.shape[0], I.shape[1], I.shape[1], 8, op)
             for (a, b), (I, _, op) in zip(devs, cases)]
    rc.check(rc.recon_features(ctx, tiles, feat.data_ptr()), "features")
    got = feat.cpu().numpy()
    for t, (I, J, op) in enumerate(cases):
        if op == 1:
            I, J = 255 - I, 255 - J
        elif op == 2:
            I, J = 255 - I, np.zeros_like(J)
        want = numpy_features(I, J)
        np.testing.assert_array_equal(got[t, :18], want[:18])
        np.testing.assert_allclose(got[t, 18:], want[18:], rtol=2e-7)
    assert all(np.count_nonzero(J.astype(np.int32) > I) > 0 for I, J, _ in viol)


def test_forward_matches_oracle(ctx):
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 1, size=(300, 20))
    theta = mlp.init(5)
    Y = torch.zeros((300, 2), dtype=torch.float32, device="cuda")
    dth, dX = f32(theta), f32(X)
    rc.check(rc.recon_mlp_forward(ctx, dth.data_ptr(), dX.data_ptr(), 300, Y.data_ptr()))
    close(Y.cpu().numpy(), mlp.forward(theta, X)[0])


@pytest.mark.parametrize("use_idx", [False, True])
def test_gradient_matches_oracle(ctx, use_idx):
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, size=(500, 20))
    T = rng.normal(size=(500, 2))
    theta = mlp.init(7)
    idx = rng.permutation(500)[:173] if use_idx else np.arange(173)
    g = torch.zeros(mlp.n_params(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    didx = torch.from_numpy(idx.astype(np.int32)).cuda()
    dth, dX, dT = f32(theta), f32(X), f32(T)
    rc.check(rc.recon_mlp_grad(ctx, dth.data_ptr(), dX.data_ptr(), dT.data_ptr(),
                               didx.data_ptr() if use_idx else 0, 173, g.data_ptr(), loss.data_ptr()))
    Y, cache = mlp.forward(theta, X[idx])
    close(g.cpu().numpy(), mlp.backward(theta, cache, Y, T[idx]))
    close(loss.cpu().numpy()[0], mlp.loss(Y, T[idx]))


def test_adam_matches_oracle(ctx):
    rng = np.random.default_rng(4)
    theta = mlp.init(1)
    m = rng.normal(size=theta.size) * 1e-2
    v = np.abs(rng.normal(size=theta.size)) * 1e-3
    grad = rng.normal(size=theta.size)
    want, wm, wv = mlp.adam_step(theta, grad, m, v, 5, lr=1e-3)
    dth, dg, dm, dv = f32(theta), f32(grad), f32(m), f32(v)
    rc.check(rc.recon_mlp_adam(ctx, dth.data_ptr(), dg.data_ptr(), dm.data_ptr(), dv.data_ptr(), 5, 1e-3))
    close(dth.cpu().numpy(), want)
    close(dm.cpu().numpy(), wm)
    close(dv.cpu().numpy(), wv)
    assert (dg.cpu().numpy() == 0).all()


def test_training_reduces_loss_like_oracle(ctx):
    rng = np.random.default_rng(6)
    X = rng.uniform(0, 1, size=(2048, 20))
    T = np.stack([X[:, :5].sum(1) - 2.5, 2 * X[:, 5] - X[:, 6]], axis=1)
    theta0 = mlp.init(9)
    l0 = mlp.loss(mlp.forward(theta0, X)[0], T)
    dth = f32(theta0)
    st, losses = rc.recon_mlp_train(ctx, dth.data_ptr(), f32(X).data_ptr(), f32(T).data_ptr(), 2048,
                                    40, 64, 3e-3, 1)
    rc.check(st, "train")
    l_gpu = mlp.loss(mlp.forward(dth.cpu().numpy().astype(np.float64), X)[0], T)
    l_cpu = mlp.loss(mlp.forward(mlp.train(theta0, X, T, 40, 3e-3, 64, 1), X)[0], T)
    assert l_gpu < 0.05 * l0 and l_cpu < 0.05 * l0
    assert losses[-1] < losses[0]


def test_training_checkpoint_resume(ctx, tmp_path):
    """Training 3 epochs, checkpointing (theta, Adam moments, step, epoch) to a
    file and resuming for 3 more follows the same update sequence as 6 epochs
    at once (the shuffle of epoch e depends only on (seed, e)); the two end
    points agree up to the summation order of the gradient reduction."""
    from paper_1311_0378_gb300 import cost_model
    rng = np.random.default_rng(8)
    n = 1500
    X = rng.uniform(0, 1, size=(n, 20))
    T = np.stack([X[:, :4].sum(1) - 2.0, X[:, 7] - 0.5], axis=1)
    theta0 = mlp.init(3)
    npar = rc.RECON_MLP_NPARAMS
    dX, dT = f32(X), f32(T)
    # straight: 6 epochs
    th_a, mv_a = f32(theta0), f32(np.zeros(2 * npar))
    st, step_a, _ = rc.recon_mlp_train_resume(ctx, th_a.data_ptr(), mv_a.data_ptr(), 0, 0, dX.data_ptr(),
                                              dT.data_ptr(), n, 6, 100, 2e-3, 5)
    rc.check(st, "straight")
    # 3 epochs, checkpoint through a file, resume 3
    th_b, mv_b = f32(theta0), f32(np.zeros(2 * npar))
    st, step_b, _ = rc.recon_mlp_train_resume(ctx, th_b.data_ptr(), mv_b.data_ptr(), 0, 0, dX.data_ptr(),
                                              dT.data_ptr(), n, 3, 100, 2e-3, 5)
    rc.check(st, "first half")
    p = str(tmp_path / "t.ckpt")
    cost_model.save_checkpoint(p, th_b.cpu().numpy(), mv_b.cpu().numpy(), {"step": step_b, "epoch": 3})
    th_l, mv_l, state = cost_model.load_checkpoint(p)
    th_c, mv_c = f32(th_l), f32(mv_l)
    st, step_c, _ = rc.recon_mlp_train_resume(ctx, th_c.data_ptr(), mv_c.data_ptr(), state["step"],
                                              state["epoch"], dX.data_ptr(), dT.data_ptr(), n, 3, 100, 2e-3, 5)
    rc.check(st, "resumed half")
    assert step_a == step_c == 6 * 15
    close(th_c.cpu().numpy(), th_a.cpu().numpy(), rtol=1e-3)
    assert not np.allclose(th_a.cpu().numpy(), theta0)   # it trained
