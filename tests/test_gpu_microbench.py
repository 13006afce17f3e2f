"""GPU parity for the device micro-benchmarks (Tables III and IV): the random
read checksum and the matrix after a random write run equal the oracle's, and
every atomic count is exact."""
import numpy as np
import pytest

from oracle import microbench as mbo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1311_0378_gb300.build as b
    b.build()
    torch.cuda.set_device(0)


def _matrix(log2n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 32, size=1 << log2n, dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("log2n,ops", [(12, 3), (20, 1_000_003), (24, 10_000_000)])
def test_random_read_checksum(log2n, ops):
    M = _matrix(log2n, log2n)
    d = torch.from_numpy(M.view(np.int32)).cuda()
    torch.cuda.synchronize()
    st, cs, ms = rc.recon_mb_random(d.data_ptr(), log2n, ops, False, 1234 + log2n)
    rc.check(st, "recon_mb_random")
    assert ms > 0
    assert cs == mbo.random_read_checksum(M, log2n, ops, 1234 + log2n)


@pytest.mark.parametrize("log2n,ops", [(10, 77), (18, 300_001)])
def test_random_write_result(log2n, ops):
    M = _matrix(log2n, 100 + log2n)
    d = torch.from_numpy(M.view(np.int32)).cuda()
    torch.cuda.synchronize()
    st, _, ms = rc.recon_mb_random(d.data_ptr(), log2n, ops, True, 77)
    rc.check(st, "recon_mb_random")
    got = d.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, mbo.random_write_result(M, log2n, ops, 77))


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_atomic_counts(mode):
    threads = rc.recon_mb_threads(0)
    assert threads > 0 and threads % 256 == 0
    ctas = threads // 256
    iters = 37
    C = torch.zeros(threads, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    st, ms = rc.recon_mb_atomic(C.data_ptr(), mode, iters)
    rc.check(st, "recon_mb_atomic")
    got = C.cpu().numpy().view(np.uint32)
    if mode == 0:
        assert got[0] == threads * iters and not got[1:].any()
    elif mode == 2:
        assert (got[:ctas] == 256 * iters).all() and not got[ctas:].any()
    else:
        assert (got == iters).all()


def test_bad_arguments():
    assert rc.recon_mb_random(0, 24, 10, False, 1)[0] == rc.RECON_EINVAL
    C = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert rc.recon_mb_atomic(C.data_ptr(), 4, 1)[0] == rc.RECON_EINVAL
