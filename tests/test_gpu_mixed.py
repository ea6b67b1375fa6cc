"""GPU parity of the mixed-precision paths (tcgen05 products with 16-bit hi + lo operands).

Tolerances from the arithmetic.  QST_MIXED (FP16 hi + lo after power-of-two
scaling): ~22 significant bits per operand and a dropped lo*lo term <= 2^-22 of
a product term (together ~2^-21); the tensor core's FP32 accumulation then adds
up to one truncation (2^-23 relative) per K = 16 step, i.e. (2d / 16) 2^-23 for
K = 2d.  The bar is 1e-5 + (2d / 16) 2^-23 (4e-5 at d = 2048) on rho, the loss
and the gradient.  QST_MIXED_BF16 (BF16 hi + lo, ~16 bits): 1e-4 on rho and the
loss and 1e-3 on the gradient (normwise; the backward product adds its own split).
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


def _ctx(N, prec):
    o = qst.qst_default_options()
    o.precision = prec
    return qst.qst_init(N, opt=o)


def _problem(N, seed, shots=10**6):
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 4), 700 + seed)
    P = O.born_probabilities(rho, M).real
    f = synth.frequencies(synth.multinomial_counts(P, shots, 800 + seed))
    return rho, f, synth.init_theta(N, 900 + seed)


def TOLS(mode, N):
    """(rho, loss, gradient) tolerances; see the module docstring."""
    if mode == qst.QST_MIXED:
        t = 1e-5 + (2 * (1 << N) / 16) * 2.0 ** -23
        return t, t, t
    return 1e-4, 1e-4, 1e-3


@pytest.mark.parametrize("mode", [qst.QST_MIXED, qst.QST_MIXED_BF16])
@pytest.mark.parametrize("N", [7, 8, 9, 10, 11])
def test_mixed_rho_matches_fp32_path(N, mode):
    _, f, theta = _problem(N, N)
    th = torch.from_numpy(theta.astype(np.float32)).cuda()
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    out = {}
    for prec in (qst.QST_FP32, mode):
        ctx = _ctx(N, prec)
        try:
            qst.qst_set_params(ctx, th)
            rho = torch.empty((1 << N, 1 << N), dtype=torch.complex64, device="cuda")
            L, st = qst.qst_get_rho(ctx, fd, rho, want_loss=True)
            assert st == qst.QST_OK
            out[prec] = (rho.cpu().numpy().astype(np.complex128), L)
        finally:
            qst.qst_destroy(ctx)
    (r32, L32), (rmx, Lmx) = out[qst.QST_FP32], out[mode]
    t_rho, t_loss, _ = TOLS(mode, N)
    assert np.linalg.norm(rmx - r32) / np.linalg.norm(r32) < t_rho
    assert np.abs(rmx - r32).max() < t_rho * np.abs(r32).max()
    assert abs(Lmx - L32) < t_loss * abs(L32)


@pytest.mark.parametrize("mode", [qst.QST_MIXED, qst.QST_MIXED_BF16])
@pytest.mark.parametrize("N", [7, 9, 11])
def test_mixed_loss_grad_vs_oracle(N, mode):
    _, f, theta = _problem(N, 20 + N)
    th64 = theta.astype(np.float32).astype(np.float64)
    f64 = f.astype(np.float32).astype(np.float64)
    L_ref, g_ref, _ = O.loss_and_grad(th64, f64, M, N)
    ctx = _ctx(N, mode)
    try:
        th = torch.from_numpy(theta.astype(np.float32)).cuda()
        g = torch.empty_like(th)
        L, st = qst.qst_loss_grad(ctx, th, torch.from_numpy(f.astype(np.float32)).cuda(), g)
        g = g.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)
    assert st == qst.QST_OK
    _, t_loss, t_grad = TOLS(mode, N)
    assert abs(L - L_ref) <= t_loss * abs(L_ref)
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel < t_grad, rel


def test_mixed_reconstruction_reaches_oracle_fidelity():
    """N = 8 from exact probabilities of a pure state: mixed and oracle reconstructions both reach F ~ 1."""
    N = 8
    psi = synth.haar_pure(N, 31)
    f = O.born_probabilities(synth.pure_density(psi), M).real
    theta = synth.init_theta(N, 32)
    iters = 300
    _, rho_ref, _ = O.reconstruct(theta.astype(np.float32).astype(np.float64),
                                  f.astype(np.float32).astype(np.float64), M, N, iters)
    F_ref = O.fidelity_pure(rho_ref, psi)
    ctx = _ctx(N, qst.QST_MIXED)
    try:
        qst.qst_set_params(ctx, theta.astype(np.float32))
        rho = np.empty((1 << N, 1 << N), dtype=np.complex64)
        qst.qst_reconstruct(ctx, np.ascontiguousarray(f.astype(np.float32)), iters, rho)
    finally:
        qst.qst_destroy(ctx)
    F = O.fidelity_pure(rho.astype(np.complex128), psi)
    print(f"N=8 reconstruction: F mixed {F:.6f}, oracle {F_ref:.6f}")
    assert F_ref > 0.99
    assert abs(F - F_ref) < 1e-4, (F, F_ref)


def test_mixed_trajectory_tracks_fp32_n10():
    """N = 10, 10^6 shots, 60 Rprop steps: the mixed path follows the FP32 path's loss trajectory."""
    N = 10
    _, f, theta = _problem(N, 40, shots=10**6)
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    traj = {}
    for prec in (qst.QST_FP32, qst.QST_MIXED):
        ctx = _ctx(N, prec)
        try:
            qst.qst_set_params(ctx, theta.astype(np.float32))
            traj[prec] = np.array([qst.qst_step(ctx, fd)[0] for _ in range(60)])
        finally:
            qst.qst_destroy(ctx)
    rel = np.abs(traj[qst.QST_MIXED] - traj[qst.QST_FP32]) / np.abs(traj[qst.QST_FP32])
    assert rel.max() < 1e-5, rel.max()
