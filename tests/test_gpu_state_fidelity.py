"""GPU state fidelity (Sec. 2.3 eq. F_QF through eq. fq_decom) against the oracle.

The oracle evaluates eq. F_QF by its singular-value route (`fidelity`) on its own rho^ from the same
parameters; for the pure target (w = 1) it uses <psi|rho^|psi> (Sec. 2.3), which is exact, whereas
the singular-value route carries ~1e-8 from the square roots of the zero eigenvalues of a rank-one
matrix.  Bars: FP64 1e-9.  FP32: the eigenvectors come out of 12 Jacobi sweeps, each entry the
product of about 12 d plane rotations rounded in FP32, so their error grows like sqrt(12 d) u
(u = 2^-24; 9e-6 at d = 2048), and F, a smooth function of them, is held to ten times that.
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


def _ctx(N, prec, mapping=qst.QST_MAP_CHOL_H, P=2.0, network=qst.QST_NET_FNN):
    o = qst.qst_default_options()
    o.precision = prec
    o.mapping = mapping
    o.P = P
    o.network = network
    return qst.qst_init(N, opt=o)


def _setup(N, lam, seed, network="fnn"):
    psi = synth.haar_pure(N, 300 + seed)
    P = O.born_probabilities(synth.depolarized(psi, lam), M).real
    f = synth.frequencies(synth.multinomial_counts(P, 10**5, 310 + seed))
    theta = (synth.init_theta_cnn if network == "cnn" else synth.init_theta)(N, 320 + seed)
    return psi, f, theta


def _tol32(N):
    return 10.0 * np.sqrt(12.0 * (1 << N)) * 2.0 ** -24


def _want(theta, f, N, psi, w, dt, mapping="chol_h", P=2.0, network="fnn"):
    th = theta.astype(dt).astype(np.float64)
    f64 = f.astype(dt).astype(np.float64)
    rh = O.state_from_theta(th, f64, N, mapping=mapping, P=P, network=network, decision=dt)
    if w == 1.0:
        return O.fidelity_pure(rh, psi)
    return O.fidelity(rh, O.noisy_target(psi, w))


def _gpu(N, prec, theta, f, psi, w, mapping=qst.QST_MAP_CHOL_H, P=2.0, network=qst.QST_NET_FNN, host=False):
    dt = np.float64 if prec == qst.QST_FP64 else np.float32
    ct = np.complex128 if prec == qst.QST_FP64 else np.complex64
    ctx = _ctx(N, prec, mapping, P, network)
    try:
        qst.qst_set_params(ctx, theta.astype(dt))
        fx = f.astype(dt)
        px = psi.astype(ct)
        if not host:
            fx = torch.from_numpy(fx).cuda()
            px = torch.from_numpy(px).cuda()
        F = qst.qst_state_fidelity(ctx, fx, px, w)
        F2 = qst.qst_state_fidelity(ctx, fx, px, w)
    finally:
        qst.qst_destroy(ctx)
    if mapping == qst.QST_MAP_ABS_P:  # the second forward starts from the first one's eigenvectors
        assert abs(F - F2) < 1e-12
    else:  # a cold eigensolver run and fixed-order reductions repeat exactly
        assert F == F2
    return F


@pytest.mark.parametrize("N,w", [(2, 1.0), (2, 0.3), (4, 0.9), (4, 0.0), (6, 0.9), (6, 1.0), (7, 0.5)])
def test_state_fidelity_fp64_chol_h(N, w):
    psi, f, theta = _setup(N, 0.1, N)
    got = _gpu(N, qst.QST_FP64, theta, f, psi, w, host=(N == 4))
    want = _want(theta, f, N, psi, w, np.float64)
    assert abs(got - want) < 1e-9, (got, want)


@pytest.mark.parametrize("P", [1.5, 3.0])
def test_state_fidelity_fp64_abs_p(P):
    N = 4
    psi, f, theta = _setup(N, 0.2, 40)
    got = _gpu(N, qst.QST_FP64, theta, f, psi, 0.8, mapping=qst.QST_MAP_ABS_P, P=P)
    want = _want(theta, f, N, psi, 0.8, np.float64, mapping="abs_p", P=P)
    assert abs(got - want) < 1e-9, (got, want)


@pytest.mark.parametrize("N,w,prec", [(5, 0.9, qst.QST_FP32), (8, 0.9, qst.QST_FP32), (8, 1.0, qst.QST_FP32),
                                      (8, 0.9, qst.QST_MIXED)])
def test_state_fidelity_fp32(N, w, prec):
    psi, f, theta = _setup(N, 0.1, 50 + N)
    got = _gpu(N, prec, theta, f, psi, w)
    want = _want(theta, f, N, psi, w, np.float32)
    assert abs(got - want) < _tol32(N), (got, want)


def test_state_fidelity_cnn():
    N = 5
    psi, f, theta = _setup(N, 0.1, 60, network="cnn")
    got = _gpu(N, qst.QST_FP64, theta, f, psi, 0.9, network=qst.QST_NET_CNN)
    want = _want(theta, f, N, psi, 0.9, np.float64, network="cnn")
    assert abs(got - want) < 1e-9, (got, want)


def test_state_fidelity_full_size_n11():
    """N = 11 (d = 2048), the benchmark's target family (depolarised Haar pure state, lambda = 0.1)."""
    N = 11
    psi, f, theta = _setup(N, 0.1, 70)
    got = _gpu(N, qst.QST_FP32, theta, f, psi, 0.9)
    want = _want(theta, f, N, psi, 0.9, np.float32)
    assert abs(got - want) < _tol32(N), (got, want)
    got1 = _gpu(N, qst.QST_FP32, theta, f, psi, 1.0)
    want1 = _want(theta, f, N, psi, 1.0, np.float32)
    assert abs(got1 - want1) < _tol32(N), (got1, want1)


def _theta_for_T(T, N):
    """Parameters whose network output is the R of a given Hermitian T (Sec. 3.1 readings: T_ii = R_ii,
    T_ij = R_ij + i R_ji for i > j): every weight and b1 zero, b2 = R, so t = b2 whatever f is."""
    d, n, H = 1 << N, 4 ** N, 2 * N
    R = np.diag(T.real.diagonal()).astype(np.float64)
    il = np.tril_indices(d, -1)
    R[il] = T.real[il]
    R[(il[1], il[0])] = T.imag[il]
    theta = np.zeros(2 * H * n + n + H)
    theta[2 * H * n:2 * H * n + n] = R.reshape(-1)
    return theta


@pytest.mark.parametrize("N,prec", [(6, qst.QST_FP64), (8, qst.QST_FP32), (11, qst.QST_FP32)])
def test_state_fidelity_near_the_target(N, prec):
    """rho^ close to the target (F ~ 0.99): T = sqrt of a depolarised state near the target, so that
    2^N - 1 eigenvalues of rho^ sit at ~lambda / d and their square roots carry a tenth of Tr sqrt."""
    d = 1 << N
    psi = synth.haar_pure(N, 400 + N)
    rng = np.random.default_rng(410 + N)
    near = psi + 0.03 * (rng.standard_normal(d) + 1j * rng.standard_normal(d)) / np.sqrt(2 * d)
    near /= np.linalg.norm(near)
    rho_near = synth.depolarized(near, 0.12)
    ev, V = np.linalg.eigh(rho_near)
    T = (V * np.sqrt(np.clip(ev, 0, None))) @ V.conj().T
    theta = _theta_for_T(0.5 * (T + T.conj().T), N)
    f = np.full(4 ** N, 1.0 / 4 ** N)
    dt = np.float64 if prec == qst.QST_FP64 else np.float32
    got = _gpu(N, prec, theta, f, psi, 0.9)
    want = _want(theta, f, N, psi, 0.9, dt)
    assert want > 0.95
    assert abs(got - want) < (1e-9 if prec == qst.QST_FP64 else _tol32(N)), (got, want)


def test_state_fidelity_bounded_by_classical_and_rejects():
    N = 4
    psi, f, theta = _setup(N, 0.1, 80)
    ctx = _ctx(N, qst.QST_FP64)
    try:
        qst.qst_set_params(ctx, theta)
        fd = torch.from_numpy(f).cuda()
        Pt = torch.from_numpy(np.ascontiguousarray(O.born_probabilities(O.noisy_target(psi, 0.7), M).real)).cuda()
        pd = torch.from_numpy(psi.astype(np.complex128)).cuda()
        Fq = qst.qst_state_fidelity(ctx, fd, pd, 0.7)
        Fc = qst.qst_classical_fidelity(ctx, fd, Pt)
        assert 0.0 < Fq <= Fc + 1e-12  # eq. F_CF bounds eq. F_QF
        with pytest.raises(qst.QstError) as e:
            qst.qst_state_fidelity(ctx, fd, pd, 1.5)
        assert e.value.status == qst.QST_E_INVAL
    finally:
        qst.qst_destroy(ctx)
    o = qst.qst_default_options()
    o.precision = qst.QST_FP64
    o.mapping = qst.QST_MAP_CHOL_DELTA
    ctx = qst.qst_init(N, opt=o)
    try:
        qst.qst_set_params(ctx, theta)
        with pytest.raises(qst.QstError) as e:
            qst.qst_state_fidelity(ctx, torch.from_numpy(f).cuda(), torch.from_numpy(psi).cuda(), 0.7)
        assert e.value.status == qst.QST_E_UNSUPPORTED
    finally:
        qst.qst_destroy(ctx)
