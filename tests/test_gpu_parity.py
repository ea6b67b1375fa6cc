"""GPU parity of libqst against the FP64 oracle, through the C ABI.

Tolerances (FP32 paths), from the arithmetic: every kernel accumulates in FP32
over at most a few thousand terms before an FP64 reduction, so relative
errors stay near 1e-6; the bar is 1e-4 relative on p, the loss and the
gradient (max error relative to the largest entry), and 1e-3 for central
finite differences with h = 1e-3.  FP64 paths are held to 1e-10.
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
    return o


def _np_dtype(prec):
    return np.float64 if prec == qst.QST_FP64 else np.float32


def _cplx(rho, prec):
    dt = np.complex128 if prec == qst.QST_FP64 else np.complex64
    return torch.from_numpy(np.ascontiguousarray(rho.astype(dt))).cuda()


def _rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ------------------------------------------------------------------ POVM map
@pytest.mark.parametrize("prec", [qst.QST_FP32, qst.QST_FP64])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_probs_parity(N, prec):
    ctx = qst.qst_init(N, opt=_opt(prec))
    try:
        for seed, rho in ((1, synth.ginibre_mixed(N, max(1, (1 << N) // 3), 100 + N)),
                          (2, synth.random_hermitian(1 << N, 200 + N))):
            want = O.born_probabilities(rho, M).real
            p = torch.empty(4 ** N, dtype=torch.float64 if prec == qst.QST_FP64 else torch.float32, device="cuda")
            qst.qst_probs(ctx, _cplx(rho, prec), p)
            got = p.cpu().numpy().astype(np.float64)
            n = 4 ** N
            den = np.maximum(np.abs(want), 1e-3 / n)
            tol = 1e-10 if prec == qst.QST_FP64 else 1e-4
            if seed == 1:
                assert np.max(np.abs(got - want) / den) < tol
            assert _rel_max(got, want) < tol
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol / 10
    finally:
        qst.qst_destroy(ctx)


def test_probs_only_reads_lower_triangle():
    N = 5
    rho = synth.ginibre_mixed(N, 4, 3)
    junk = rho.copy()
    iu = np.triu_indices(1 << N, 1)
    junk[iu] = 123.0 + 45.0j
    ctx = qst.qst_init(N)
    try:
        a = torch.empty(4 ** N, device="cuda")
        b = torch.empty(4 ** N, device="cuda")
        qst.qst_probs(ctx, _cplx(rho, qst.QST_FP32), a)
        qst.qst_probs(ctx, _cplx(junk, qst.QST_FP32), b)
        assert torch.equal(a, b)
    finally:
        qst.qst_destroy(ctx)


@pytest.mark.parametrize("N", [11, 12])
def test_probs_full_size_sampled(N):
    """Full-size POVM map: sampled outcomes against the oracle one by one, plus sum p = Tr rho."""
    rng = np.random.default_rng(N)
    psi = synth.haar_pure(N, 20)
    rho = synth.depolarized(psi, 0.1)
    ctx = qst.qst_init(N)
    try:
        p = torch.empty(4 ** N, device="cuda")
        qst.qst_probs(ctx, _cplx(rho, qst.QST_FP32), p)
        got = p.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)
    ks = np.concatenate([[0, 4 ** N - 1], rng.integers(0, 4 ** N, 30)])
    for k in ks:
        want = O.born_probability_at(rho, M, int(k)).real
        assert abs(got[k] - want) <= 1e-4 * max(abs(want), 1e-3 / 4 ** N), (k, got[k], want)
    assert abs(got.sum() - 1.0) < 1e-4
    assert got.min() > -1e-6 / 4 ** N


# ------------------------------------------------------------------ loss and gradient
def _problem(N, seed, shots=10**5, rank=None):
    rank = rank or max(1, (1 << N) // 2)
    rho = synth.ginibre_mixed(N, rank, 300 + seed)
    P = O.born_probabilities(rho, M).real
    f = synth.frequencies(synth.multinomial_counts(P, shots, 400 + seed))
    theta = synth.init_theta(N, 500 + seed)
    return rho, f, theta


def _gpu_loss_grad(N, theta, f, prec, ctx=None):
    dt = _np_dtype(prec)
    own = ctx is None
    if own:
        ctx = qst.qst_init(N, opt=_opt(prec))
    try:
        th = torch.from_numpy(theta.astype(dt)).cuda()
        fd = torch.from_numpy(f.astype(dt)).cuda()
        g = torch.empty_like(th)
        L, st = qst.qst_loss_grad(ctx, th, fd, g)
        return L, g.cpu().numpy().astype(np.float64), st
    finally:
        if own:
            qst.qst_destroy(ctx)


@pytest.mark.parametrize("prec", [qst.QST_FP32, qst.QST_FP64])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
def test_loss_grad_parity(N, prec):
    _, f, theta = _problem(N, N)
    dt = _np_dtype(prec)
    # the oracle sees exactly the values the GPU sees
    th64 = theta.astype(dt).astype(np.float64)
    f64 = f.astype(dt).astype(np.float64)
    L_ref, g_ref, _ = O.loss_and_grad(th64, f64, M, N)
    L, g, st = _gpu_loss_grad(N, theta, f, prec)
    tol = 1e-10 if prec == qst.QST_FP64 else 1e-4
    assert st == qst.QST_OK
    assert abs(L - L_ref) <= tol * abs(L_ref)
    assert _rel_max(g, g_ref) < tol
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < tol


@pytest.mark.parametrize("rank", [1, 4, 16, 256])
def test_gradient_central_fd_n8(rank):
    """N = 8, FP32: directional central differences (h = 1e-3) and the oracle's analytic gradient."""
    N = 8
    _, f, theta = _problem(N, 10 + rank, shots=10**6, rank=rank)
    ctx = qst.qst_init(N)
    try:
        L, g, _ = _gpu_loss_grad(N, theta, f, qst.QST_FP32, ctx)
        rng = np.random.default_rng(rank)
        gn = np.linalg.norm(g)
        # steepest direction, two directions correlated with g (v_i = g_i u_i, u_i ~ U(0.5, 1.5)),
        # and one unstructured direction; unit length, so |dL/dv| <= ||g||
        dirs = [g / gn]
        for _ in range(2):
            v = g * rng.uniform(0.5, 1.5, theta.size)
            dirs.append(v / np.linalg.norm(v))
        v = rng.standard_normal(theta.size)
        dirs.append(v / np.linalg.norm(v))
        h = 1e-3
        th64 = theta.astype(np.float32).astype(np.float64)
        f64 = f.astype(np.float32).astype(np.float64)
        _, g64, _ = O.loss_and_grad(th64, f64, M, N)
        for v in dirs:
            Lp = _gpu_loss_grad(N, theta + h * v, f, qst.QST_FP32, ctx)[0]
            Lm = _gpu_loss_grad(N, theta - h * v, f, qst.QST_FP32, ctx)[0]
            fd = (Lp - Lm) / (2 * h)
            an = float(np.dot(g, v))
            # the central difference's own O(h^2) error, measured noise-free by the FP64 oracle
            Lp64 = O.loss_and_grad(th64 + h * v, f64, M, N)[0]
            Lm64 = O.loss_and_grad(th64 - h * v, f64, M, N)[0]
            fd64 = (Lp64 - Lm64) / (2 * h)
            trunc = abs(fd64 - float(np.dot(g64, v)))
            # FP32 rounding of the two losses, measured against the FP64 oracle at the same points
            noise = (abs(Lp - Lp64) + abs(Lm - Lm64)) / (2 * h)
            assert abs(fd - an) <= 1e-3 * max(abs(an), 0.5 * gn) + trunc + noise, (fd, an, gn, trunc, noise)
            assert abs(fd - fd64) <= noise + 1e-4 * abs(fd64) + 1e-12
    finally:
        qst.qst_destroy(ctx)
    L_ref, g_ref, _ = O.loss_and_grad(theta.astype(np.float32).astype(np.float64),
                                      f.astype(np.float32).astype(np.float64), M, N)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-4


def test_loss_grad_full_size_n11():
    """N = 11 (4,194,304 outcomes), 10^7 shots: loss and gradient vs the oracle."""
    N = 11
    psi = synth.haar_pure(N, 20)
    rho = synth.depolarized(psi, 0.1)
    P = O.born_probabilities(rho, M).real
    f = synth.frequencies(synth.multinomial_counts(P, 10**7, 21))
    theta = synth.init_theta(N, 22)
    L, g, st = _gpu_loss_grad(N, theta, f, qst.QST_FP32)
    L_ref, g_ref, _ = O.loss_and_grad(theta.astype(np.float32).astype(np.float64),
                                      f.astype(np.float32).astype(np.float64), M, N)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    assert _rel_max(g, g_ref) < 1e-4
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-4


# ------------------------------------------------------------------ Rprop step and loop
def test_single_step_matches_oracle_rprop():
    N = 5
    _, f, theta = _problem(N, 7)
    th32 = theta.astype(np.float32)
    f32 = f.astype(np.float32)
    ctx = qst.qst_init(N)
    try:
        qst.qst_set_params(ctx, torch.from_numpy(th32).cuda())
        L, st = qst.qst_step(ctx, torch.from_numpy(f32).cuda())
        out = torch.empty(th32.size, device="cuda")
        qst.qst_get_params(ctx, out)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        qst.qst_destroy(ctx)
    L_ref, g_ref, _ = O.loss_and_grad(th32.astype(np.float64), f32.astype(np.float64), M, N)
    assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
    stt = O.RpropState(theta.size)
    want = O.rprop_update(th32.astype(np.float64), g_ref, stt)
    big = np.abs(g_ref) > 1e-4 * np.abs(g_ref).max()
    np.testing.assert_allclose(got[big], want[big], rtol=0, atol=1e-6)
    # tiny gradients may differ in sign; every parameter still moved by 0 or +-lr
    moved = np.abs(got - th32.astype(np.float64))
    assert np.all((moved < 1e-7) | (np.abs(moved - 1e-3) < 1e-6))


def test_checkpoint_resume_is_bit_identical():
    N = 4
    _, f, theta = _problem(N, 3)
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    ctx = qst.qst_init(N)
    try:
        qst.qst_set_params(ctx, torch.from_numpy(theta.astype(np.float32)).cuda())
        for _ in range(3):
            qst.qst_step(ctx, fd)
        blob = qst.qst_get_state(ctx)
        la = [qst.qst_step(ctx, fd)[0] for _ in range(4)]
        a = torch.empty(theta.size, device="cuda"); qst.qst_get_params(ctx, a)
        qst.qst_set_state(ctx, blob)
        assert qst.qst_iterations(ctx) == 3
        lb = [qst.qst_step(ctx, fd)[0] for _ in range(4)]
        b = torch.empty(theta.size, device="cuda"); qst.qst_get_params(ctx, b)
        assert la == lb
        assert torch.equal(a, b)
    finally:
        qst.qst_destroy(ctx)


def test_host_and_device_inputs_agree():
    N = 4
    _, f, theta = _problem(N, 4)
    f32 = np.ascontiguousarray(f.astype(np.float32))
    res = []
    for dev in (True, False):
        ctx = qst.qst_init(N)
        try:
            qst.qst_set_params(ctx, theta.astype(np.float32))
            fin = torch.from_numpy(f32).cuda() if dev else f32
            res.append([qst.qst_step(ctx, fin)[0] for _ in range(3)])
        finally:
            qst.qst_destroy(ctx)
    assert res[0] == res[1]


def test_invalid_inputs_are_rejected():
    with pytest.raises(qst.QstError) as e:
        qst.qst_init(13)
    assert e.value.status == qst.QST_E_INVAL
    bad = qst.tetrahedral_povm_flat().copy()
    bad[0] += 0.1
    with pytest.raises(qst.QstError) as e:
        qst.qst_init(3, povm=bad)
    assert e.value.status == qst.QST_E_INVAL
    N = 3
    _, f, theta = _problem(N, 5)
    ctx = qst.qst_init(N)
    try:
        with pytest.raises(qst.QstError) as e:
            qst.qst_step(ctx, f.astype(np.float32))
        assert e.value.status == qst.QST_E_STATE
        qst.qst_set_params(ctx, theta.astype(np.float32))
        for badf in (np.full(64, np.nan), -f, 2 * f):
            with pytest.raises(qst.QstError) as e:
                qst.qst_step(ctx, np.ascontiguousarray(badf.astype(np.float32)))
            assert e.value.status == qst.QST_E_INPUT
    finally:
        qst.qst_destroy(ctx)


def test_get_rho_is_physical_and_matches_oracle():
    N = 6
    _, f, theta = _problem(N, 6)
    th32 = theta.astype(np.float32)
    ctx = qst.qst_init(N)
    try:
        qst.qst_set_params(ctx, th32)
        rho = torch.empty((1 << N, 1 << N), dtype=torch.complex64, device="cuda")
        L, _ = qst.qst_get_rho(ctx, f.astype(np.float32), rho, want_loss=True)
        r = rho.cpu().numpy().astype(np.complex128)
    finally:
        qst.qst_destroy(ctx)
    assert np.abs(r - r.conj().T).max() < 1e-7
    assert abs(np.trace(r).real - 1) < 1e-5
    assert np.linalg.eigvalsh(r).min() > -1e-6
    want = O.state_from_theta(th32.astype(np.float64), f.astype(np.float32).astype(np.float64), N)
    assert np.abs(r - want).max() < 1e-4 * np.abs(want).max()
    L_ref = O.nll(O.born_probabilities(want, M).real, f.astype(np.float32).astype(np.float64))
    assert abs(L - L_ref) < 1e-4 * abs(L_ref)


def test_reconstruct_n2_fp64_matches_oracle():
    """N = 2, FP64, 10^4 shots, 1000 iterations: GPU and oracle reach the same state."""
    N = 2
    psi = synth.haar_pure(N, 1)
    P = O.born_probabilities(synth.pure_density(psi), M).real
    f = synth.frequencies(synth.multinomial_counts(P, 10**4, 2))
    theta = synth.init_theta(N, 3)
    _, rho_ref, losses = O.reconstruct(theta, f, M, N, 1000)
    ctx = qst.qst_init(N, opt=_opt(qst.QST_FP64))
    try:
        qst.qst_set_params(ctx, theta)
        rho = np.empty((4, 4), dtype=np.complex128)
        L, _ = qst.qst_reconstruct(ctx, f, 1000, rho)
    finally:
        qst.qst_destroy(ctx)
    F_gpu = O.fidelity_pure(rho, psi)
    F_ref = O.fidelity_pure(rho_ref, psi)
    assert abs(F_gpu - F_ref) < 1e-4
    assert F_gpu > 0.97
    assert abs(L - O.nll(O.born_probabilities(rho_ref, M).real, f)) < 1e-6


def test_reconstruct_exact_probabilities_reaches_target():
    N = 4
    psi = synth.haar_pure(N, 11)
    f = O.born_probabilities(synth.pure_density(psi), M).real
    theta = synth.init_theta(N, 12)
    ctx = qst.qst_init(N)
    try:
        qst.qst_set_params(ctx, theta.astype(np.float32))
        rho = np.empty((16, 16), dtype=np.complex64)
        qst.qst_reconstruct(ctx, np.ascontiguousarray(f.astype(np.float32)), 1000, rho)
    finally:
        qst.qst_destroy(ctx)
    assert O.fidelity_pure(rho.astype(np.complex128), psi) > 0.99
