"""GPU parity of the CNN mapping network of App. A (QST_NET_CNN) against the oracle.

The pooling argmax is decided in the context's precision on both sides (the oracle evaluates the
convolution in that precision, in the kernel's order); losses are then held to the same bars as
the FNN path (FP64 1e-9, FP32 1e-4 relative; the mixed path 1e-4), FP64 gradients to 1e-9 of the
largest entry and in norm.

FP32 gradients are checked per block.  The output layer's (W2^T, b2: products
h_j dL/dt_i) stay at 1e-4 of the block's largest entry.  The head's (W1, b1, the convolution) all
go through dL/dh_j = sum_i W2^T[j][i] dL/dt_i, and rho does not change when t is scaled, so
sum_i t_i dL/dt_i = 0 exactly: these sums cancel heavily (sum |terms| / |sum| has median about
2e3 and reaches 1e5 on these inputs at N = 10, 11), and an FP32 rounding of the trace
normalisation (relative 1e-7) comes out of them multiplied by that factor: perturbing that
normalisation by 1e-7 in the oracle moves dL/dh by 1e-3 in norm at N = 11.  The head block is held
to 2e-3 (largest entry and norm, relative to the block); FP64 at N = 10 (its largest size) checks
the same tiled path to 1e-9.
"""
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


def _opt(prec, mapping=qst.QST_MAP_CHOL_H):
    o = qst.qst_default_options()
    o.precision = prec
    o.mapping = mapping
    o.network = qst.QST_NET_CNN
    return o


def _problem(N, seed, shots=10**5):
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 2), 6000 + seed)
    P = O.born_probabilities(rho, M).real
    f = synth.frequencies(synth.multinomial_counts(P, shots, 6100 + seed)) if shots else P / P.sum()
    return f, synth.init_theta_cnn(N, 6200 + seed)


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _rel_norm(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _check_grad(g, g_ref, N, prec):
    if prec == qst.QST_FP64:
        rm, rn = _rel_max(g, g_ref), _rel_norm(g, g_ref)
        assert rm < 1e-9 and rn < 1e-9, (rm, rn)
        return
    # FP32: per block (module docstring)
    n, H = 4 ** N, 4 * N
    out, head = slice(0, H * n + n), slice(H * n + n, None)
    rm, rn = _rel_max(g[out], g_ref[out]), _rel_norm(g[out], g_ref[out])
    assert rm < 1e-4 and rn < 1e-4, ("output layer", rm, rn)
    rm, rn = _rel_max(g[head], g_ref[head]), _rel_norm(g[head], g_ref[head])
    assert rm < 2e-3 and rn < 2e-3, ("head", rm, rn)


def _dt(prec):
    return np.float64 if prec == qst.QST_FP64 else np.float32


def _gpu_loss_grad(N, theta, f, opt):
    dt = _dt(opt.precision)
    ctx = qst.qst_init(N, opt=opt)
    try:
        th = torch.from_numpy(theta.astype(dt)).cuda()
        g = torch.empty_like(th)
        L, _ = qst.qst_loss_grad(ctx, th, torch.from_numpy(f.astype(dt)).cuda(), g)
        return L, g.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)


# N >= 9 (pooling windows of 64 x 64 and up) takes the tiled convolution and the two-kernel pooling
CASES = [(qst.QST_FP64, N, shots) for N in (3, 4, 5) for shots in (0, 10**5)] + \
        [(qst.QST_FP32, N, shots) for N in (3, 5, 7) for shots in (0, 10**5)] + \
        [(qst.QST_FP64, 9, 10**5), (qst.QST_FP32, 9, 0), (qst.QST_FP32, 10, 10**6)]


@pytest.mark.parametrize("prec,N,shots", CASES)
def test_cnn_loss_grad_parity(prec, N, shots):
    f, theta = _problem(N, N + (1 if shots else 0), shots)
    dt = _dt(prec)
    th64 = theta.astype(dt).astype(np.float64)
    f64 = f.astype(dt).astype(np.float64)
    assert theta.size == qst.qst_theta_size_net(N, qst.QST_NET_CNN) == synth.theta_size_cnn(N)
    L_ref, g_ref, _ = O.loss_and_grad(th64, f64, M, N, network="cnn", decision=dt)
    L, g = _gpu_loss_grad(N, theta, f, _opt(prec))
    tol = 1e-9 if prec == qst.QST_FP64 else 1e-4
    assert abs(L - L_ref) <= tol * abs(L_ref)
    _check_grad(g, g_ref, N, prec)


@pytest.mark.parametrize("prec,N", [(qst.QST_FP64, 10), (qst.QST_FP32, 11)])
def test_cnn_loss_grad_full_size(prec, N):
    """N = 11 (a 2048 x 2048 input, 256 x 256 pooling windows; FP64 contexts stop at N = 10),
    10^7 shots: loss and gradient."""
    f, theta = _problem(N, 11, 10**7)
    dt = _dt(prec)
    f64 = f.astype(dt).astype(np.float64)
    th64 = theta.astype(dt).astype(np.float64)
    L_ref, g_ref, _ = O.loss_and_grad(th64, f64, M, N, network="cnn", decision=dt)
    L, g = _gpu_loss_grad(N, theta, f, _opt(prec))
    assert abs(L - L_ref) <= (1e-9 if prec == qst.QST_FP64 else 1e-4) * abs(L_ref)
    _check_grad(g, g_ref, N, prec)


@pytest.mark.parametrize("N", [3, 5, 9])
def test_cnn_single_step_matches_oracle_rprop(N):
    """One FP32 qst_step (N >= 4: the output layer through the bulk-copy W2 pass on two row halves)
    against one oracle Rprop update from the oracle's gradient."""
    f, theta = _problem(N, 70 + N)
    th32 = theta.astype(np.float32)
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP32))
    try:
        qst.qst_set_params(ctx, torch.from_numpy(th32).cuda())
        L, _ = qst.qst_step(ctx, torch.from_numpy(f.astype(np.float32)).cuda())
        out = torch.empty(th32.size, device="cuda")
        qst.qst_get_params(ctx, out)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)
    th64 = th32.astype(np.float64)
    L_ref, g_ref, _ = O.loss_and_grad(th64, f.astype(np.float32).astype(np.float64), M, N, network="cnn",
                                      decision=np.float32)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    want = O.rprop_update(th64, g_ref, O.RpropState(theta.size))
    big = np.abs(g_ref) > 1e-4 * np.abs(g_ref).max()
    np.testing.assert_allclose(got[big], want[big], rtol=0, atol=1e-6)
    # tiny gradients may differ in sign; every parameter still moved by 0 or +-lr
    moved = np.abs(got - th64)
    assert np.all((moved < 1e-7) | (np.abs(moved - 1e-3) < 1e-6))


def test_cnn_with_chol_delta_and_mixed():
    N = 4
    f, theta = _problem(N, 40, 0)
    L_ref, g_ref, _ = O.loss_and_grad(theta, f, M, N, mapping="chol_delta", network="cnn")
    L, g = _gpu_loss_grad(N, theta, f, _opt(qst.QST_FP64, qst.QST_MAP_CHOL_DELTA))
    assert abs(L - L_ref) <= 1e-9 * abs(L_ref)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-9
    N = 8
    f, theta = _problem(N, 41, 10**6)
    f32 = f.astype(np.float32).astype(np.float64)
    th32 = theta.astype(np.float32).astype(np.float64)
    L_ref, _, _ = O.loss_and_grad(th32, f32, M, N, network="cnn", decision=np.float32)
    L, g = _gpu_loss_grad(N, theta, f, _opt(qst.QST_MIXED))
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)


def test_cnn_reconstruction_matches_oracle():
    """300 Rprop steps in FP64 on the GPU against the oracle's loop from the same start."""
    N = 3
    psi = synth.haar_pure(N, 12)
    rho_t = synth.depolarized(psi, 0.1)
    f = np.ascontiguousarray(O.born_probabilities(rho_t, M).real)
    theta = synth.init_theta_cnn(N, 13)
    _, rho_ref, losses = O.reconstruct(theta, f, M, N, 300, network="cnn")
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP64))
    try:
        qst.qst_set_params(ctx, theta)
        rho = np.empty((8, 8), dtype=np.complex128)
        qst.qst_reconstruct(ctx, f, 300, rho)
    finally:
        qst.qst_destroy(ctx)
    F, F_ref = O.fidelity(rho, rho_t), O.fidelity(rho_ref, rho_t)
    assert F_ref > 0.9
    assert abs(F - F_ref) < 1e-6, (F, F_ref)


def test_cnn_graph_replay_and_checkpoint():
    N = 6
    f, theta = _problem(N, 60)
    out = []
    for graph in (False, True):
        stream = torch.cuda.Stream()
        ctx = qst.qst_init(N, opt=_opt(qst.QST_FP32), stream=stream.cuda_stream)
        try:
            if graph:
                qst.qst_graph_enable(ctx, True)
            qst.qst_set_params(ctx, theta.astype(np.float32))
            fd = torch.from_numpy(f.astype(np.float32)).cuda()
            torch.cuda.synchronize()
            losses = [qst.qst_step(ctx, fd)[0] for _ in range(3)]
            state = qst.qst_get_state(ctx)
            losses += [qst.qst_step(ctx, fd)[0] for _ in range(3)]
            th = torch.empty(theta.size, device="cuda")
            qst.qst_get_params(ctx, th)
            qst.qst_sync(ctx)
            out.append((losses, th.cpu().numpy(), state))
        finally:
            qst.qst_destroy(ctx)
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])
    # resume from the checkpoint taken after 3 steps
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP32))
    try:
        qst.qst_set_state(ctx, out[0][2])
        fd = torch.from_numpy(f.astype(np.float32)).cuda()
        again = [qst.qst_step(ctx, fd)[0] for _ in range(3)]
    finally:
        qst.qst_destroy(ctx)
    assert again == out[0][0][3:]


def test_cnn_needs_three_qubits():
    with pytest.raises(qst.QstError) as e:
        qst.qst_init(2, opt=_opt(qst.QST_FP32))
    assert e.value.status == qst.QST_E_INVAL
