"""GPU parity of the P-order absolute projection (Sec. 3.2 eq. abs_P) against the oracle.

The eigendecomposition is a Jacobi method run for a fixed number of sweeps (the mixed-precision
path refines the previous eigenvectors on tensor cores from its second step on); after
12 sweeps it has converged to rounding level for these sizes, so the FP64 path
is held to 1e-8 and the FP32 path to 1e-4 on the loss and 2e-3 (normwise) on
the gradient, whose Daleckii-Krein factors divide by eigenvalue gaps.  N = 8 and
N = 10 (d = 256, 1024) run the sweeps as passes over cosets of 16 (N = 8) and of 16 and 8
indices (N = 10), N <= 5 as passes over cosets of 4 and 2.
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


def _opt(prec, mapping=qst.QST_MAP_ABS_P, P=2.0):
    o = qst.qst_default_options()
    o.precision = prec
    o.mapping = mapping
    o.P = P
    return o


def _problem(N, seed):
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 2), 1000 + seed)
    f = synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, 10**5, 1100 + seed))
    return f, synth.init_theta(N, 1200 + seed)


def _gpu(N, theta, f, opt):
    dt = np.float64 if opt.precision == qst.QST_FP64 else np.float32
    ctx = qst.qst_init(N, opt=opt)
    try:
        th = torch.from_numpy(theta.astype(dt)).cuda()
        g = torch.empty_like(th)
        L, _ = qst.qst_loss_grad(ctx, th, torch.from_numpy(f.astype(dt)).cuda(), g)
        return L, g.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)


CASES = [(qst.QST_FP64, N, P) for N in (1, 2, 4, 6) for P in (0.5, 1.5, 2.0, 4.0)] + \
        [(qst.QST_FP32, N, P) for N in (3, 6) for P in (1.0, 2.0, 3.0)] + \
        [(prec, N, 1.5) for prec in (qst.QST_FP64, qst.QST_FP32) for N in (8, 10)] + \
        [(qst.QST_MIXED, N, P) for N in (7, 9) for P in (1.5, 3.0)]


@pytest.mark.parametrize("prec,N,P", CASES)
def test_abs_p_loss_grad_parity(prec, N, P):
    f, theta = _problem(N, N + int(10 * P))
    dt = np.float64 if prec == qst.QST_FP64 else np.float32
    L_ref, g_ref, _ = O.loss_and_grad(theta.astype(dt).astype(np.float64), f.astype(dt).astype(np.float64), M, N,
                                      mapping="abs_p", P=P)
    L, g = _gpu(N, theta, f, _opt(prec, P=P))
    tl, tg = (1e-8, 1e-8) if prec == qst.QST_FP64 else (1e-4, 2e-3)  # mixed: products on tensor cores
    rl = abs(L - L_ref) / abs(L_ref)
    rg = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rl <= tl and rg < tg, (rl, rg)


@pytest.mark.parametrize("prec", [qst.QST_FP32, qst.QST_MIXED])
def test_abs_p_full_size_n11(prec):
    """N = 11 (d = 2048, 4^11 outcomes, 10^7 shots of a depolarised Haar state): the A_P loss and gradient
    of a cold start (12 FP32 sweeps, passes over cosets of 16 and 8 indices; on the mixed path the products
    and the Daleckii-Krein backward on tensor cores) against the oracle, at the FP32 bars above."""
    N, P = 11, 1.5
    rho = synth.depolarized(synth.haar_pure(N, 30), 0.1)
    f = synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, 10**7, 31))
    theta = synth.init_theta(N, 32)
    L_ref, g_ref, _ = O.loss_and_grad(theta.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64),
                                      M, N, mapping="abs_p", P=P)
    L, g = _gpu(N, theta, f, _opt(prec, P=P))
    rl = abs(L - L_ref) / abs(L_ref)
    rg = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rl <= 1e-4 and rg < 2e-3, (rl, rg)


def test_abs_p2_equals_chol_h():
    """Sec. 3.2: A_P with P = 2 is the unified Chol_H map."""
    N = 5
    f, theta = _problem(N, 77)
    La, ga = _gpu(N, theta, f, _opt(qst.QST_FP64, qst.QST_MAP_ABS_P, 2.0))
    Lc, gc = _gpu(N, theta, f, _opt(qst.QST_FP64, qst.QST_MAP_CHOL_H))
    assert abs(La - Lc) < 1e-10 * abs(Lc)
    assert np.linalg.norm(ga - gc) / np.linalg.norm(gc) < 1e-8


def test_abs_p_reconstruction_matches_oracle():
    N, P = 3, 1.5
    psi = synth.haar_pure(N, 5)
    rho_t = synth.depolarized(psi, 0.1)
    f = np.ascontiguousarray(O.born_probabilities(rho_t, M).real)
    theta = synth.init_theta(N, 6)
    _, rho_ref, _ = O.reconstruct(theta, f, M, N, 300, mapping="abs_p", P=P)
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP64, P=P))
    try:
        qst.qst_set_params(ctx, theta)
        rho = np.empty((8, 8), dtype=np.complex128)
        qst.qst_reconstruct(ctx, f, 300, rho)
    finally:
        qst.qst_destroy(ctx)
    F, F_ref = O.fidelity(rho, rho_t), O.fidelity(rho_ref, rho_t)
    assert F_ref > 0.99
    assert abs(F - F_ref) < 1e-6, (F, F_ref)


@pytest.mark.parametrize("N,P,k,lr", [(7, 1.5, 6, 1e-7), (8, 3.0, 6, 1e-7), (10, 1.5, 3, 1e-7),
                                      (7, 1.5, 4, 1e-3), (9, 1.5, 3, 1e-3)])
def test_mixed_warm_steps_follow_the_oracle(N, P, k, lr):
    """QST_MIXED: warm-started steps refine the previous eigenvectors on tensor cores.  Every step's loss is the oracle's
    (exact FP64 eigendecomposition) at the parameters the GPU held before it, and every parameter the
    step moved went against the sign of the oracle's gradient wherever that gradient is not small.
    With steps of 1e-7 T moves little and first-order refinements suffice; with the paper's 1e-3 T moves
    by more than the gaps of its near-degenerate eigenvalues, and the block passes over neighbours in the
    order of lambda resolve those couplings before the refinement is taken."""
    f, theta = _problem(N, 300 + N)
    opt = _opt(qst.QST_MIXED, P=P)
    opt.lr = lr
    opt.step_min = min(opt.step_min, lr)
    ctx = qst.qst_init(N, opt=opt)
    try:
        qst.qst_set_params(ctx, theta.astype(np.float32))
        fd = torch.from_numpy(f.astype(np.float32)).cuda()
        f64 = f.astype(np.float32).astype(np.float64)
        out = torch.empty(theta.size, device="cuda")
        qst.qst_get_params(ctx, out)
        th = out.cpu().numpy().astype(np.float64)
        for it in range(k):
            L, _ = qst.qst_step(ctx, fd)
            qst.qst_get_params(ctx, out)
            th1 = out.cpu().numpy().astype(np.float64)
            L_ref, g_ref, _ = O.loss_and_grad(th, f64, M, N, mapping="abs_p", P=P)
            assert abs(L - L_ref) <= 1e-4 * abs(L_ref), (it, L, L_ref)
            moved = th1 != th
            big = np.abs(g_ref) > 1e-2 * np.abs(g_ref).max()
            sel = moved & big
            assert sel.sum() > 0
            assert np.all(np.sign(th1[sel] - th[sel]) == -np.sign(g_ref[sel])), it
            th = th1
        refinements, fallbacks = qst.qst_eig_counts(ctx)
        # every warm step refined on tensor cores (with the block passes where T moved far), none handed
        # to the sweeps
        assert refinements >= k - 1 and fallbacks == 0, (refinements, fallbacks)
    finally:
        qst.qst_destroy(ctx)


@pytest.mark.parametrize("N", [8, 10])
def test_mixed_warm_steps_on_the_sweeps_follow_the_oracle(N):
    """QST_MIXED with eig_refine = 0: every warm step runs the Jacobi sweeps from the previous eigenvectors,
    with Q^dag T Q and X = Q |Lambda|^P Q^dag on tensor cores (the path the refinement hands its steps to).
    Each step's loss is the oracle's at the parameters the GPU held before it, every moved parameter went
    against the sign of the oracle's gradient where that gradient is not small, and no refinement ran."""
    P, k = 1.5, 4
    f, theta = _problem(N, 320 + N)
    opt = _opt(qst.QST_MIXED, P=P)
    opt.eig_refine = 0
    ctx = qst.qst_init(N, opt=opt)
    try:
        qst.qst_set_params(ctx, theta.astype(np.float32))
        fd = torch.from_numpy(f.astype(np.float32)).cuda()
        f64 = f.astype(np.float32).astype(np.float64)
        out = torch.empty(theta.size, device="cuda")
        qst.qst_get_params(ctx, out)
        th = out.cpu().numpy().astype(np.float64)
        for it in range(k):
            L, _ = qst.qst_step(ctx, fd)
            qst.qst_get_params(ctx, out)
            th1 = out.cpu().numpy().astype(np.float64)
            L_ref, g_ref, _ = O.loss_and_grad(th, f64, M, N, mapping="abs_p", P=P)
            assert abs(L - L_ref) <= 1e-4 * abs(L_ref), (it, L, L_ref)
            moved = th1 != th
            big = np.abs(g_ref) > 1e-2 * np.abs(g_ref).max()
            sel = moved & big
            assert sel.sum() > 0
            assert np.all(np.sign(th1[sel] - th[sel]) == -np.sign(g_ref[sel])), it
            th = th1
        assert qst.qst_eig_counts(ctx) == (0, 0)
    finally:
        qst.qst_destroy(ctx)


def _steps(N, theta, f, opt, k):
    ctx = qst.qst_init(N, opt=opt)
    try:
        qst.qst_set_params(ctx, theta)
        return [qst.qst_step(ctx, np.ascontiguousarray(f))[0] for _ in range(k)]
    finally:
        qst.qst_destroy(ctx)


def test_warm_start_follows_cold_start_trajectory():
    """Warm-started eigendecompositions (2 sweeps from the last eigenvectors) give the same
    iteration as a cold start every step (12 sweeps)."""
    N, P = 5, 1.5
    f, theta = _problem(N, 91)
    warm = _opt(qst.QST_FP64, P=P)
    cold = _opt(qst.QST_FP64, P=P)
    cold.eig_warm_sweeps = -1
    lw = np.array(_steps(N, theta, f, warm, 10))
    lc = np.array(_steps(N, theta, f, cold, 10))
    # both eigendecompositions are exact to rounding; Rprop's sign decisions can then differ only on
    # gradients at rounding level, so the losses agree far below any step's change
    rel = np.abs(lw - lc) / np.abs(lc)
    assert rel.max() < 1e-7, rel


def test_abs_p_checkpoint_resume_bit_identical():
    N, P = 4, 1.5
    f, theta = _problem(N, 92)
    f = np.ascontiguousarray(f)
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP64, P=P))
    try:
        qst.qst_set_params(ctx, theta)
        for _ in range(3):
            qst.qst_step(ctx, f)
        blob = qst.qst_get_state(ctx)
        la = [qst.qst_step(ctx, f)[0] for _ in range(4)]
        qst.qst_set_state(ctx, blob)
        lb = [qst.qst_step(ctx, f)[0] for _ in range(4)]
        assert la == lb
    finally:
        qst.qst_destroy(ctx)
