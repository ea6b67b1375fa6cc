"""GPU parity of the Cholesky decomposition map Chol_Delta (Sec. 2.2.1 eq. T_matrix) against the oracle.

T is the complex lower-triangular matrix of the network output and rho = T^dag T / Tr(T^dag T);
the backward pulls dL = 2 Re Tr[G T^dag dT] back to t through the lower tiles of T G.  Bars: the
same as for Chol_H (FP64 1e-10, FP32 1e-4 relative on the loss and on the gradient's largest
entry and norm).
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


def _opt(prec):
    o = qst.qst_default_options()
    o.precision = prec
    o.mapping = qst.QST_MAP_CHOL_DELTA
    return o


def _problem(N, seed, shots=10**5):
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 2), 3000 + seed)
    f = synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, shots, 3100 + seed))
    return rho, f, synth.init_theta(N, 3200 + seed)


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _gpu_loss_grad(N, theta, f, prec):
    dt = np.float64 if prec == qst.QST_FP64 else np.float32
    ctx = qst.qst_init(N, opt=_opt(prec))
    try:
        th = torch.from_numpy(theta.astype(dt)).cuda()
        g = torch.empty_like(th)
        L, _ = qst.qst_loss_grad(ctx, th, torch.from_numpy(f.astype(dt)).cuda(), g)
        return L, g.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)


# d = 2 .. 256: the small-matrix product, one tile with a ragged 32-wide T tile (d < 32), several tiles
CASES = [(qst.QST_FP64, N) for N in (1, 2, 3, 4, 5, 6)] + [(qst.QST_FP32, N) for N in (2, 3, 5, 6, 7, 8)]


@pytest.mark.parametrize("prec,N", CASES)
def test_chol_delta_loss_grad_parity(prec, N):
    _, f, theta = _problem(N, N)
    dt = np.float64 if prec == qst.QST_FP64 else np.float32
    th64 = theta.astype(dt).astype(np.float64)
    f64 = f.astype(dt).astype(np.float64)
    L_ref, g_ref, _ = O.loss_and_grad(th64, f64, M, N, mapping="chol_delta")
    L, g = _gpu_loss_grad(N, theta, f, prec)
    tol = 1e-10 if prec == qst.QST_FP64 else 1e-4
    assert abs(L - L_ref) <= tol * abs(L_ref)
    assert _rel_max(g, g_ref) < tol
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < tol


def test_chol_delta_differs_from_chol_h():
    """Same network output, different map: the losses must differ (the lower-triangular T is not Hermitian)."""
    N = 4
    _, f, theta = _problem(N, 40)
    Ld, _ = _gpu_loss_grad(N, theta, f, qst.QST_FP64)
    o = qst.qst_default_options()
    o.precision = qst.QST_FP64
    ctx = qst.qst_init(N, opt=o)
    try:
        g = torch.empty(theta.size, dtype=torch.float64, device="cuda")
        Lh, _ = qst.qst_loss_grad(ctx, torch.from_numpy(theta).cuda(), torch.from_numpy(f).cuda(), g)
    finally:
        qst.qst_destroy(ctx)
    Lh_ref = O.loss_and_grad(theta, f, M, N)[0]
    Ld_ref = O.loss_and_grad(theta, f, M, N, mapping="chol_delta")[0]
    assert abs(Lh - Lh_ref) < 1e-10 * abs(Lh_ref) and abs(Ld - Ld_ref) < 1e-10 * abs(Ld_ref)
    assert abs(Ld - Lh) > 1e-6 * abs(Lh)


def test_chol_delta_rho_is_the_oracle_state():
    N = 5
    _, f, theta = _problem(N, 50)
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP64))
    try:
        qst.qst_set_params(ctx, theta)
        rho = torch.empty((32, 32), dtype=torch.complex128, device="cuda")
        qst.qst_get_rho(ctx, torch.from_numpy(f).cuda(), rho)
        got = rho.cpu().numpy()
    finally:
        qst.qst_destroy(ctx)
    want = O.state_from_theta(theta, f, N, mapping="chol_delta")
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_chol_delta_reconstruction_matches_oracle():
    N = 3
    psi = synth.haar_pure(N, 8)
    rho_t = synth.depolarized(psi, 0.1)
    f = np.ascontiguousarray(O.born_probabilities(rho_t, M).real)
    theta = synth.init_theta(N, 9)
    _, rho_ref, _ = O.reconstruct(theta, f, M, N, 300, mapping="chol_delta")
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP64))
    try:
        qst.qst_set_params(ctx, theta)
        rho = np.empty((8, 8), dtype=np.complex128)
        qst.qst_reconstruct(ctx, f, 300, rho)
    finally:
        qst.qst_destroy(ctx)
    F, F_ref = O.fidelity(rho, rho_t), O.fidelity(rho_ref, rho_t)
    assert F_ref > 0.95
    assert abs(F - F_ref) < 1e-6, (F, F_ref)


def test_chol_delta_graph_replay_is_bit_identical():
    N = 7
    _, f, theta = _problem(N, 70)
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
            losses = [qst.qst_step(ctx, fd)[0] for _ in range(5)]
            th = torch.empty(theta.size, device="cuda")
            qst.qst_get_params(ctx, th)
            qst.qst_sync(ctx)
            out.append((losses, th.cpu().numpy()))
        finally:
            qst.qst_destroy(ctx)
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])


def test_chol_delta_mixed_is_unsupported():
    o = _opt(qst.QST_MIXED)
    with pytest.raises(qst.QstError) as e:
        qst.qst_init(8, opt=o)
    assert e.value.status == qst.QST_E_UNSUPPORTED
