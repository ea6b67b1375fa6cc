"""GPU parity of the CNN mapping network of App. A (QST_NET_CNN) against the oracle.

The pooling argmax is decided in the context's precision on both sides (the oracle evaluates the
convolution in that precision, in the kernel's order); losses and gradients are then held to the
same bars as the FNN path (FP64 1e-9, FP32 1e-4 relative on the loss and the gradient's largest
entry and norm; the mixed path 1e-4 on the loss).
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


CASES = [(qst.QST_FP64, N, shots) for N in (3, 4, 5) for shots in (0, 10**5)] + \
        [(qst.QST_FP32, N, shots) for N in (3, 5, 7) for shots in (0, 10**5)]


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
    assert _rel_max(g, g_ref) < tol
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < tol


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
