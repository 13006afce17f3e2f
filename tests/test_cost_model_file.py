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
