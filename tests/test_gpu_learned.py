"""The learned schedule (committed cost model, trained on the GPU by the
library's own MLP kernels on 20k generated tiles labelled with the work the
method reports) against the plain schedule on a fresh 1000-tile uneven batch:
identical output bytes, predicted work that tracks the measured work, and the
time the learned schedule saves."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402
from paper_1311_0378_gb300 import cost_model  # noqa: E402


def test_model_file_meta():
    theta, norm, variants, meta = cost_model.load()
    assert theta.shape == (rc.RECON_MLP_NPARAMS,) and np.isfinite(theta).all()
    assert meta["tiles"] == 20000 and variants == (1 + 256 * 32, 1)


def test_learned_schedule_gain_and_identity():
    import paper_1311_0378_gb300.build as b
    b.build()
    ctx = rc.recon_init(0, 0, 0)
    try:
        res = cost_model.evaluate(ctx, cost_model.MODEL_PATH, "eval1000", reps=3)
    finally:
        rc.recon_free(ctx)
    print("learned vs plain on eval1000:", res)
    assert res["outputs_identical"]
    assert res["gain"] > 1.0, res


def test_learned_outputs_match_oracle_and_predictions_rank_work():
    """On 40 tiles of the evaluation law: the learned batch equals the oracle
    byte for byte, and the model's predicted work ranks the tiles like the
    work the kernel measures (Spearman rank correlation)."""
    import paper_1311_0378_gb300.build as b
    b.build()
    specs = list(synth.workload("eval1000").tiles[:40])
    pairs = synth.generate(specs, 6)
    wants, _ = oracle.recon_tiles(pairs, [s.conn for s in specs], "sweep")
    ctx = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
    try:
        cost_model.install(ctx)
        devs = [(torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()) for I, J in pairs]
        torch.cuda.synchronize()
        tiles = [(a.data_ptr(), b_.data_ptr(), s.H, s.W, s.W, s.conn) for (a, b_), s in zip(devs, specs)]
        st, var, order, pred = rc.recon_sched_plan_batch(ctx, tiles)
        rc.check(st, "plan")
        measured = []
        for t in range(len(specs)):
            J0 = torch.from_numpy(pairs[t][1]).cuda()
            torch.cuda.synchronize()
            devs[t][1].copy_(J0)
            torch.cuda.synchronize()
            rc.check(rc.recon_batch_ex(ctx, [tiles[t]], [var[t]], None), "solo")
            measured.append(rc.recon_get_work(ctx, 1)[0]["busy_ns"])
            np.testing.assert_array_equal(devs[t][1].cpu().numpy(), wants[t])
        vb = cost_model.load()[2][1]
        chosen = [pred[2 * t + 1] if var[t] == vb else pred[2 * t] for t in range(len(specs))]
        rp = np.argsort(np.argsort(chosen))
        rm = np.argsort(np.argsort(measured))
        rho = np.corrcoef(rp, rm)[0, 1]
        print("Spearman(predicted, measured work) =", rho)
        assert rho > 0.8
    finally:
        rc.recon_free(ctx)
