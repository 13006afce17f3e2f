"""Host logic of the cost-model file (no GPU)."""
import numpy as np
import pytest

from paper_1311_0378_gb300 import cost_model
import paper_1311_0378_gb300 as rc


def test_roundtrip(tmp_path):
    theta = np.arange(rc.RECON_MLP_NPARAMS, dtype=np.float32) / 7
    p = tmp_path / "m.bin"
    cost_model.save(str(p), theta, [1.0, 2.0, 3.0, 4.0], (-1, 2), {"tiles": 5})
    th, norm, var, meta = cost_model.load(str(p))
    assert np.array_equal(th, theta) and list(norm) == [1, 2, 3, 4] and var == (-1, 2)
    assert meta == {"tiles": 5}


def test_bad_file(tmp_path):
    p = tmp_path / "x.bin"
    p.write_bytes(b"nope" + b"\0" * 64)
    with pytest.raises(ValueError):
        cost_model.load(str(p))


def test_init_params_layout():
    th = cost_model.init_params(np.random.default_rng(0))
    assert th.dtype == np.float32 and th.size == rc.RECON_MLP_NPARAMS
    assert np.all(th[20 * 64:20 * 64 + 64] == 0)   # b1 starts at zero


def test_checkpoint_roundtrip(tmp_path):
    n = rc.RECON_MLP_NPARAMS
    theta = np.linspace(-1, 1, n, dtype=np.float32)
    mv = np.arange(2 * n, dtype=np.float32) * 1e-3
    state = {"step": 123, "epoch": 4, "norm": [0.5, 2.0, 1.5, 3.0], "seed": 9, "lr": 2e-3, "batch": 256}
    p = tmp_path / "c.ckpt"
    cost_model.save_checkpoint(str(p), theta, mv, state)
    th, m2, st = cost_model.load_checkpoint(str(p))
    assert np.array_equal(th, theta) and np.array_equal(m2, mv) and st == state
    assert not (tmp_path / "c.ckpt.tmp").exists()


def test_checkpoint_rejects_bad_and_truncated(tmp_path):
    p = tmp_path / "bad.ckpt"
    p.write_bytes(b"RCM1" + b"\0" * 64)
    with pytest.raises(ValueError):
        cost_model.load_checkpoint(str(p))
    q = tmp_path / "short.ckpt"
    cost_model.save_checkpoint(str(q), np.zeros(rc.RECON_MLP_NPARAMS, np.float32),
                               np.zeros(2 * rc.RECON_MLP_NPARAMS, np.float32), {"step": 0})
    q.write_bytes(q.read_bytes()[:-100])
    with pytest.raises(ValueError):
        cost_model.load_checkpoint(str(q))


def test_tuning_cache_file_roundtrip(tmp_path):
    from paper_1311_0378_gb300 import tuning
    entries = [(18, 2, 0, 128, 4, 1, 512), (24, 3, 1, 64, 2, 0, 0)]
    p = str(tmp_path / "tune.json")
    tuning.write_entries(p, entries)
    assert tuning.read_entries(p) == entries
    (tmp_path / "bad.json").write_text('{"entries": [{"size_bucket": 1}]}')
    with pytest.raises(ValueError):
        tuning.read_entries(str(tmp_path / "bad.json"))
