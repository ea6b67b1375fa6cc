"""GPU test of qst_probs_static, the allocation-free POVM map.

It exists for callers that cannot call cudaMalloc (a framework whose pool
allocator owns the device memory, a latency-bound loop that must not take an
allocation's synchronisation, a one-off evaluation without a context).  It
must give what qst_probs gives.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2207_05341_gb300 import qst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    if not os.path.exists(qst.LIB_PATH):
        from paper_2207_05341_gb300 import build
        build.build()
    qst.load()


def _reference_probs(N, rho_dev):
    ctx = qst.qst_init(N)
    try:
        p = torch.empty(4 ** N, device="cuda")
        qst.qst_probs(ctx, rho_dev, p)
        torch.cuda.synchronize()
        return p
    finally:
        qst.qst_destroy(ctx)


def test_static_probs_matches_qst_probs_on_two_calls():
    """Two calls in a row (a large problem, then a smaller one) through the C ABI."""
    for N, seed in ((10, 1), (6, 2)):
        rho = synth.ginibre_mixed(N, 3, seed)
        rho_dev = torch.from_numpy(rho.astype(np.complex64)).cuda()
        p = torch.full((4 ** N,), float("nan"), device="cuda")
        qst.qst_probs_static(N, rho_dev, p)
        torch.cuda.synchronize()
        want = _reference_probs(N, rho_dev)
        err = (p - want).abs().max().item() / want.abs().max().item()
        assert err <= 1e-4, (N, err)
        assert torch.isfinite(p).all()


def test_static_probs_rejects_sizes_beyond_its_array():
    rho = torch.zeros((1 << 11, 1 << 11), dtype=torch.complex64, device="cuda")
    p = torch.empty(4 ** 11, device="cuda")
    with pytest.raises(qst.QstError) as e:
        qst.qst_probs_static(11, rho, p)
    assert e.value.status == qst.QST_E_INVAL
