"""GPU test of qst_probs_static, the allocation-free POVM map.

It exists for callers that cannot call cudaMalloc (a framework whose pool
allocator owns the device memory, a latency-bound loop that must not take an
allocation's synchronisation, a one-off evaluation without a context).  It
must give what qst_probs gives, and a call must not allocate device memory.
The file name makes pytest collect it last.
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


def _rho(N, seed):
    return torch.from_numpy(synth.ginibre_mixed(N, max(1, (1 << N) // 3), seed).astype(np.complex64)).cuda()


def _err(p, want):
    return (p - want).abs().max().item() / want.abs().max().item()


def test_static_probs_matches_qst_probs_on_two_calls():
    """Two calls in a row (a large problem, then a smaller one) through the C ABI."""
    for N, seed in ((10, 1), (6, 2)):
        rho_dev = _rho(N, seed)
        p = torch.full((4 ** N,), float("nan"), device="cuda")
        qst.qst_probs_static(N, rho_dev, p)
        torch.cuda.synchronize()
        want = _reference_probs(N, rho_dev)
        assert _err(p, want) <= 1e-4, N
        assert torch.isfinite(p).all()


@pytest.mark.parametrize("N", [1, 2, 3, 6, 10])
def test_static_probs_all_sizes_on_a_side_stream(N):
    """Every tile shape of the two passes, down to the degenerate ones (N = 1..3), on a non-default
    stream whose handle is passed through the C ABI."""
    rho_dev = _rho(N, 10 + N)
    want = _reference_probs(N, rho_dev)
    s = torch.cuda.Stream()
    p = torch.full((4 ** N,), float("nan"), device="cuda")
    torch.cuda.current_stream().synchronize()
    qst.qst_probs_static(N, rho_dev, p, stream=s.cuda_stream)
    s.synchronize()
    assert _err(p, want) <= 1e-4, N


def test_static_probs_allocates_no_device_memory():
    """After one warm-up call (which may load the module that holds the array), further calls at
    several sizes change neither the device's free memory nor torch's reserved pool."""
    rho10, rho6 = _rho(10, 3), _rho(6, 4)
    p10 = torch.empty(4 ** 10, device="cuda")
    p6 = torch.empty(4 ** 6, device="cuda")
    qst.qst_probs_static(10, rho10, p10)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(3):
        qst.qst_probs_static(10, rho10, p10)
        qst.qst_probs_static(6, rho6, p6)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_static_probs_rejects_host_pointers():
    N = 3
    rho_h = np.zeros((8, 8), dtype=np.complex64)
    p_h = np.zeros(4 ** N, dtype=np.float32)
    p_d = torch.empty(4 ** N, device="cuda")
    for rho, p in ((rho_h, p_d), (_rho(N, 5), p_h)):
        with pytest.raises(qst.QstError) as e:
            qst.qst_probs_static(N, rho, p)
        assert e.value.status == qst.QST_E_INVAL


def test_static_probs_rejects_sizes_beyond_its_array():
    rho = torch.zeros((1 << 11, 1 << 11), dtype=torch.complex64, device="cuda")
    p = torch.empty(4 ** 11, device="cuda")
    with pytest.raises(qst.QstError) as e:
        qst.qst_probs_static(11, rho, p)
    assert e.value.status == qst.QST_E_INVAL
