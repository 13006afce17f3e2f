"""The tensor-level calls run() / batch() of the binding reject what the C ABI
cannot take (wrong dtype, device, rank, layout or mismatched shapes) before
any library call; this needs no GPU."""
import pytest

torch = pytest.importorskip("torch")

import paper_1311_0378_gb300 as rc  # noqa: E402


def _fake_cuda(monkeypatch):
    """Argument checks only: report every tensor as a CUDA tensor."""
    class Dev:
        type = "cuda"
        index = 0

        def __eq__(self, other):
            return True

        def __repr__(self):
            return "cuda:0"
    monkeypatch.setattr(torch.Tensor, "device", property(lambda self: Dev()))


def test_rejects_cpu_tensors():
    I = torch.zeros(4, 4, dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA"):
        rc.run(I, I.clone())


def test_rejects_wrong_dtype_rank_layout_shape(monkeypatch):
    _fake_cuda(monkeypatch)
    I = torch.zeros(4, 6, dtype=torch.uint8)
    with pytest.raises(TypeError, match="uint8"):
        rc.run(I.float(), I.clone())
    with pytest.raises(ValueError, match="2-D"):
        rc.run(I.view(-1), I.clone().view(-1))
    with pytest.raises(ValueError, match="contiguous"):
        rc.run(I.t(), I.clone().t())
    with pytest.raises(ValueError, match="shape"):
        rc.run(I, torch.zeros(4, 5, dtype=torch.uint8))
    with pytest.raises(TypeError, match="Tensor"):
        rc.run(I.numpy(), I.clone())
    with pytest.raises(ValueError, match="at least one"):
        rc.batch([])
