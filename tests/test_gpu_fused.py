"""The one-CTA iteration of small tomographies (FP32, 3-layer network, Chol_H, N <= 7): one qst_step
against the FP64 oracle (loss, Rprop update of every parameter, the next hidden layer through the next
step's loss), against the phase-by-phase kernels of the same context type, and a ragged batch with
more tomographies than resident CTAs (each CTA then takes several from the work list) against the
same tomographies run one context at a time, bit for bit.

Tolerances as in test_gpu_parity.py: FP32 sums over at most 4^7 terms before an FP64 reduction,
1e-4 relative on the loss; Rprop moves every parameter by exactly 0 or +-lr, so the updated
parameters agree to rounding wherever the gradient is not near zero."""
import numpy as np
import pytest

import oracle as O
from paper_2207_05341_gb300 import qst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M = O.tetrahedral_povm()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    if not os.path.exists(qst.LIB_PATH):
        from paper_2207_05341_gb300 import build
        build.build()
    qst.load()


def _problem(N, seed):
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 2), 700 + seed)
    f = synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, 10**5 * N, 710 + seed))
    return f.astype(np.float32), synth.init_theta(N, 720 + seed).astype(np.float32)


def _opt(fused_max=7):
    o = qst.qst_default_options()
    o.fused_max_qubits = fused_max
    return o


def _steps(N, f, theta, steps, fused_max=7, timing=False):
    ctx = qst.qst_init(N, opt=_opt(fused_max))
    try:
        if timing:
            qst.qst_timing_enable(ctx, steps)
        qst.qst_set_params(ctx, torch.from_numpy(theta).cuda())
        fd = torch.from_numpy(f).cuda()
        losses = [qst.qst_step(ctx, fd) for _ in range(steps)]
        out = torch.empty(theta.size, device="cuda")
        qst.qst_get_params(ctx, out)
        qst.qst_sync(ctx)
        tm = qst.qst_timing_read(ctx) if timing else None
        return losses, out.cpu().numpy(), tm, qst.qst_kernel_launches(ctx)
    finally:
        qst.qst_destroy(ctx)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_fused_step_matches_oracle(N):
    f, th = _problem(N, N)
    losses, got, _, _ = _steps(N, f, th, 2)
    (L0, s0), (L1, _) = losses
    assert s0 == qst.QST_OK
    f64, th64 = f.astype(np.float64), th.astype(np.float64)
    L_ref, g_ref, _ = O.loss_and_grad(th64, f64, M, N)
    assert abs(L0 - L_ref) <= 1e-4 * abs(L_ref), (L0, L_ref)
    # after two steps: replay the oracle's Rprop on the first step's update, then check the second
    # step's loss at the parameters the GPU held after its first step (the next hidden layer)
    st = O.RpropState(th.size)
    want1 = O.rprop_update(th64, g_ref, st)
    ctx = qst.qst_init(N, opt=_opt())
    try:
        qst.qst_set_params(ctx, torch.from_numpy(th).cuda())
        qst.qst_step(ctx, torch.from_numpy(f).cuda())
        out = torch.empty(th.size, device="cuda")
        qst.qst_get_params(ctx, out)
        qst.qst_sync(ctx)
        p1 = out.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)
    big = np.abs(g_ref) > 1e-4 * np.abs(g_ref).max()
    np.testing.assert_allclose(p1[big], want1[big], rtol=0, atol=1e-6)
    moved = np.abs(p1 - th64)
    assert np.all((moved < 1e-7) | (np.abs(moved - 1e-3) < 1e-6))
    L1_ref, _, _ = O.loss_and_grad(p1, f64, M, N)
    assert abs(L1 - L1_ref) <= 1e-4 * abs(L1_ref), (L1, L1_ref)


@pytest.mark.parametrize("N", [3, 5, 7])
def test_fused_and_phase_by_phase_paths_agree(N):
    f, th = _problem(N, 20 + N)
    la, pa, _, ka = _steps(N, f, th, 6)
    lb, pb, _, kb = _steps(N, f, th, 6, fused_max=-1)
    assert ka < kb  # one kernel per steady-state iteration against one per phase
    for (a, _), (b, _) in zip(la, lb):
        assert abs(a - b) <= 1e-4 * abs(b), (a, b)
    # the same Rprop moves, except where a gradient near zero took another sign
    assert np.mean(np.abs(pa - pb) < 1e-6) > 0.99


def test_fused_step_is_timed_as_one_phase():
    N = 6
    f, th = _problem(N, 40)
    _, _, tm, _ = _steps(N, f, th, 4, timing=True)
    timed = {p for p in qst.PHASES if tm[p][1] > 0}
    assert timed == {"hidden", "fused"}
    assert tm["fused"][1] == 4 and tm["hidden"][1] == 1
    _, _, tm, _ = _steps(N, f, th, 2, fused_max=-1, timing=True)
    assert tm["fused"][1] == 0 and tm["w2"][1] == 2


def test_fused_limit_option():
    for bad in (-2, 8):
        with pytest.raises(qst.QstError) as e:
            qst.qst_init(3, opt=_opt(bad))
        assert e.value.status == qst.QST_E_INVAL
    # a limit below N: the phase-by-phase kernels (several launches per step)
    f, th = _problem(5, 41)
    _, _, _, k_on = _steps(5, f, th, 3)
    _, _, _, k_off = _steps(5, f, th, 3, fused_max=4)
    assert k_off > k_on
    # 0: the process-wide tuned limit
    lim = qst.qst_get_tuning()["fused_max_qubits"]
    for N in (lim, lim + 1):
        if 1 <= N <= 7:
            fN, thN = _problem(N, 42)
            _, _, _, k_def = _steps(N, fN, thN, 3, fused_max=0)
            _, _, _, k_fused = _steps(N, fN, thN, 3, fused_max=7)
            assert (k_def == k_fused) == (N <= lim), (N, lim, k_def, k_fused)


def test_ragged_batch_with_more_tomographies_than_ctas_is_bit_identical():
    """More tomographies than the persistent launch has CTAs (at most 2 per SM): every CTA takes
    several from the work list, and each result is the one its own context gives."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rng = np.random.default_rng(5)
    B = 2 * sms + 37
    Ns = [int(x) for x in rng.integers(1, 5, B)]
    Ns[:3] = [7, 6, 8]  # one large fused, one mid, one that runs its own kernel chain
    data = [_problem(N, 100 + b) for b, N in enumerate(Ns)]
    steps = 3
    stream = torch.cuda.Stream()
    bt = qst.qst_batch_init(Ns, opt=_opt(), stream=stream.cuda_stream)
    try:
        fds = [torch.from_numpy(f).cuda() for f, _ in data]
        for b, (_, th) in enumerate(data):
            qst.qst_batch_set_params(bt, b, th)
        torch.cuda.synchronize()
        losses = [qst.qst_batch_step(bt, fds, want_losses=True) for _ in range(steps)]
        got = []
        for b in range(B):
            out = torch.empty(data[b][1].size, device="cuda")
            qst.qst_get_params(qst.qst_batch_context(bt, b), out)
            got.append(out)
        qst.qst_batch_sync(bt)
        torch.cuda.synchronize()
        got = [g.cpu().numpy() for g in got]
    finally:
        qst.qst_batch_destroy(bt)
    for b in list(range(3)) + list(range(3, B, 17)):
        N = Ns[b]
        want_l, want_p, _, _ = _steps(N, data[b][0], data[b][1], steps)
        assert [l[b] for l in losses] == [l for l, _ in want_l], b
        assert np.array_equal(got[b], want_p), b
