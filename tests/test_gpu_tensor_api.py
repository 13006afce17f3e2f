"""run() / batch() on tensors, against the CPU oracle byte for byte: dilation,
erosion and FillHoles through run(), and a batch of tiles of several sizes and
both markers through batch()."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402


def test_run_on_tensors_matches_oracle():
    import paper_1311_0378_gb300.build as b
    b.build()
    spec = synth.TileSpec(700, 515, 150, 3, 20, synth.FILLHOLES, 8, 2)
    I, J = synth.tile_pair(spec, 11)
    for conn in (4, 8):
        dI, dJ = torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()
        out = rc.run(dI, dJ, conn)
        assert out is dJ
        np.testing.assert_array_equal(dJ.cpu().numpy(), oracle.recon(I, J, conn))
        # erosion of the complemented pair, FillHoles of the mask
        cI, cJ = torch.from_numpy(255 - I).cuda(), torch.from_numpy(255 - J).cuda()
        rc.run(cI, cJ, conn, rc.RECON_OP_ERODE)
        np.testing.assert_array_equal(cJ.cpu().numpy(), oracle.recon_erode(255 - I, 255 - J, conn))
        F = torch.empty_like(dI)
        rc.run(dI, F, conn, rc.RECON_OP_FILL_HOLES)
        np.testing.assert_array_equal(F.cpu().numpy(), oracle.fill_holes(I, conn))


def test_batch_on_tensors_matches_oracle():
    specs = [synth.TileSpec(h, w, n, 3, 20, m, 8, t) for t, (h, w, n, m) in
             enumerate([(256, 512, 60, 0), (300, 129, 40, 1), (1024, 768, 500, 1), (64, 64, 5, 0)])]
    pairs = synth.generate(specs, 13)
    dev = [(torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()) for I, J in pairs]
    outs = rc.batch(dev, conn=8)
    for (I, J), R in zip(pairs, outs):
        np.testing.assert_array_equal(R.cpu().numpy(), oracle.recon(I, J, 8))


def test_batch_reports_failing_tile():
    I = torch.full((64, 64), 10, dtype=torch.uint8, device="cuda")
    good = torch.zeros_like(I)
    bad = torch.zeros_like(I)
    bad[5, 5] = 11
    with pytest.raises(rc.ReconError, match="first failing tile 1"):
        rc.batch([(I, good), (I, bad)])
