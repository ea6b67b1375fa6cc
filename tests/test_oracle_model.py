"""Pins of the oracle's network, state mapping, likelihood, gradient and Rprop (Sec. 3.1, 3.2, 4.1)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2207_05341_gb300 import synth


def test_hermitian_map_is_a_bijection():
    rng = np.random.default_rng(1)
    for d in (1, 2, 4, 8):
        t = rng.standard_normal(d * d)
        T = O.hermitian_from_output(t)
        assert np.allclose(T, T.conj().T)
        R = t.reshape(d, d)
        for i in range(d):
            assert T[i, i] == R[i, i]
            for j in range(i):
                assert T[i, j] == R[i, j] + 1j * R[j, i]
        # Frobenius norm: sum R_ii^2 + 2 sum_{i != j} R_ij^2
        want = np.sum(np.diag(R) ** 2) + 2 * (np.sum(R ** 2) - np.sum(np.diag(R) ** 2))
        assert abs(np.linalg.norm(T) ** 2 - want) < 1e-12 * want


@pytest.mark.parametrize("seed", [0, 1])
def test_state_maps_are_physical_and_agree(seed):
    d = 8
    T = synth.random_hermitian(d, seed)
    for rho in (O.chol_h(T), O.abs_p(T, 0.5), O.abs_p(T, 1.5), O.abs_p(T, 3.0)):
        assert np.allclose(rho, rho.conj().T, atol=1e-14)
        assert abs(np.trace(rho).real - 1) < 1e-13
        assert np.linalg.eigvalsh(rho).min() > -1e-14
    # Sec. 3.2: Chol_H is A_P with P = 2
    np.testing.assert_allclose(O.chol_h(T), O.abs_p(T, 2.0), atol=1e-13)
    # A_4 is T^4 / Tr T^4 (a matrix power), A_1 is |T| / Tr|T|
    T4 = np.linalg.matrix_power(T, 4)
    np.testing.assert_allclose(O.abs_p(T, 4.0), T4 / np.trace(T4).real, atol=1e-13)
    w, V = np.linalg.eigh(T)
    absT = (V * np.abs(w)) @ V.conj().T
    np.testing.assert_allclose(O.abs_p(T, 1.0), absT / np.trace(absT).real, atol=1e-13)
    # diagonal T maps to |lambda|^P / sum
    lam = np.array([0.3, -1.2, 2.0, 0.1])
    np.testing.assert_allclose(np.diag(O.abs_p(np.diag(lam).astype(complex), 1.5)).real,
                               np.abs(lam) ** 1.5 / np.sum(np.abs(lam) ** 1.5), atol=1e-15)


def test_loss_gibbs_inequality_and_one_qubit_closed_form():
    M = O.tetrahedral_povm()
    rng = np.random.default_rng(2)
    f = rng.dirichlet(np.ones(16))
    H = -np.sum(f * np.log(f))
    for s in range(5):
        p = O.born_probabilities(synth.ginibre_mixed(2, 2, s), M).real
        assert O.nll(p, f) >= H - 1e-14
    assert abs(O.nll(f, f) - H) < 1e-14
    # zero-frequency outcomes contribute nothing
    f0 = f.copy(); f0[3] = 0; f0 /= f0.sum()
    p = rng.dirichlet(np.ones(16))
    assert abs(O.nll(p, f0) + np.sum(np.delete(f0 * np.log(p), 3))) < 1e-14
    # N = 1: rho = (I + r.sigma)/2, L = -sum f_a log((1 + s_a.r)/4)
    s = np.array([[1, 1, 1], [-1, -1, 1], [-1, 1, -1], [1, -1, -1]]) / np.sqrt(3)
    r = np.array([0.2, -0.3, 0.5])
    sx = np.array([[0, 1], [1, 0]]); sy = np.array([[0, -1j], [1j, 0]]); sz = np.diag([1, -1])
    rho = (np.eye(2) + r[0] * sx + r[1] * sy + r[2] * sz) / 2
    fa = np.array([0.1, 0.2, 0.3, 0.4])
    assert abs(O.nll(O.born_probabilities(rho, M).real, fa) + np.sum(fa * np.log((1 + s @ r) / 4))) < 1e-15


def _fd_check(N, mapping, P, idx=None, seed=0, h=1e-6, rtol=2e-6):
    M = O.tetrahedral_povm()
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 2), 50 + seed)
    f = O.born_probabilities(rho, M).real
    theta = synth.init_theta(N, 60 + seed)
    L, g, _ = O.loss_and_grad(theta, f, M, N, mapping, P)
    if idx is None:
        idx = np.arange(theta.size)
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        Lp = O.loss_and_grad(tp, f, M, N, mapping, P)[0]
        Lm = O.loss_and_grad(tm, f, M, N, mapping, P)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= rtol * max(1.0, np.abs(g).max()), (i, fd, g[i])


@pytest.mark.parametrize("N", [1, 2])
def test_gradient_central_fd_chol_h_all_coordinates(N):
    _fd_check(N, "chol_h", 2.0)


def test_gradient_central_fd_chol_h_n3_sampled():
    idx = np.random.default_rng(0).choice(synth.theta_size(3), 80, replace=False)
    _fd_check(3, "chol_h", 2.0, idx=idx, seed=3)


@pytest.mark.parametrize("N", [1, 2])
def test_gradient_central_fd_chol_delta_all_coordinates(N):
    _fd_check(N, "chol_delta", 2.0, seed=7)


def test_gradient_central_fd_chol_delta_n3_sampled():
    idx = np.random.default_rng(1).choice(synth.theta_size(3), 80, replace=False)
    _fd_check(3, "chol_delta", 2.0, idx=idx, seed=4)


def test_chol_delta_reaches_every_state_via_numpy_cholesky():
    """Sec. 2.2.1 eq. T_matrix: every density matrix is T^dag T / Tr with T lower triangular.

    With the exchange matrix E, E rho E = C C^dag (numpy's Cholesky, C lower) gives
    rho = T^dag T for T = E C^dag E, which is lower triangular with a positive diagonal.
    Reading its entries back into R (T_ii = R_ii, T_ij = R_ij + i R_ji) and mapping
    forward must return rho; an orientation or index slip in the map fails here.
    """
    for N, r, seed in ((1, 1, 0), (2, 3, 1), (3, 8, 2), (3, 2, 3)):
        d = 1 << N
        rho = synth.ginibre_mixed(N, r, seed)
        rho = rho + 1e-9 * np.eye(d)  # full rank for the Cholesky factorisation
        rho /= np.trace(rho).real
        E = np.eye(d)[::-1]
        C = np.linalg.cholesky(E @ rho @ E)
        T = E @ C.conj().T @ E
        assert np.allclose(T, np.tril(T)) and np.all(np.diag(T).real > 0)
        R = np.zeros((d, d))
        for i in range(d):
            R[i, i] = T[i, i].real
            for j in range(i):
                R[i, j], R[j, i] = T[i, j].real, T[i, j].imag
        Tm = O.lower_from_output(R.ravel())
        np.testing.assert_allclose(O.chol_delta(Tm), rho, atol=1e-12)
        # upper triangle of the map is zero, and the state is physical for any t
        t = np.random.default_rng(seed).standard_normal(d * d)
        Tr_ = O.lower_from_output(t)
        assert np.all(np.triu(Tr_, 1) == 0)
        rho2 = O.chol_delta(Tr_)
        assert abs(np.trace(rho2).real - 1) < 1e-13 and np.linalg.eigvalsh(rho2).min() > -1e-14


@pytest.mark.parametrize("P", [0.5, 1.0, 1.5, 2.0, 3.0])
def test_gradient_central_fd_abs_p(P):
    _fd_check(2, "abs_p", P, seed=int(P * 10))


def test_gradient_identity_g_x_orthogonal_to_x():
    """dL/dX is orthogonal to X: scaling T leaves rho and hence L unchanged."""
    M = O.tetrahedral_povm()
    N = 3
    f = O.born_probabilities(synth.ginibre_mixed(N, 3, 1), M).real
    theta = synth.init_theta(N, 2)
    L, g, aux = O.loss_and_grad(theta, f, M, N)
    # dL/dT along T: Re Tr[Gam T] = 2 <G_X, X> = 0
    assert abs(np.real(np.trace(aux["Gam"] @ aux["T"]))) < 1e-10 * np.abs(aux["Gam"]).max()


def test_rprop_hand_computed_sequence():
    """A hand-worked Rprop sequence: grow by 1.2, shrink by 0.5 and skip on a sign flip."""
    st = O.RpropState(1, lr=0.1)
    x = np.zeros(1)
    seq = [(2.0, -0.1, 0.1), (3.0, -0.22, 0.12), (1.0, -0.364, 0.144),
           (-1.0, -0.364, 0.072), (-1.0, -0.292, 0.072), (0.0, -0.292, 0.072),
           (-5.0, -0.22, 0.072), (-5.0, -0.1336, 0.0864)]
    for g, want_x, want_step in seq:
        x = O.rprop_update(x, np.array([g]), st)
        assert abs(x[0] - want_x) < 1e-12 and abs(st.step[0] - want_step) < 1e-12, (g, x, st.step)
    # bounds
    st = O.RpropState(2, lr=40.0)
    x = np.zeros(2)
    for _ in range(3):
        x = O.rprop_update(x, np.array([1.0, 1.0]), st)
    assert st.step[0] == 50.0
    st = O.RpropState(1, lr=2e-6)
    x = np.zeros(1)
    for g in (1.0, -1.0, 0.0, 1.0, -1.0):
        x = O.rprop_update(x, np.array([g]), st)
    assert st.step[0] == 1e-6


def test_fidelity_properties_and_printed_formulas(golden_dir):
    rho = synth.ginibre_mixed(3, 3, 1)
    sig = synth.ginibre_mixed(3, 2, 2)
    # rank-deficient states: sqrt of ~1e-17 eigenvalues limits agreement to ~1e-8
    assert abs(O.fidelity(rho, sig) - O.fidelity(sig, rho)) < 1e-7
    assert abs(O.fidelity(rho, rho) - 1) < 1e-7
    psi = synth.haar_pure(3, 4)
    assert abs(O.fidelity(rho, synth.pure_density(psi)) - O.fidelity_pure(rho, psi)) < 1e-7
    M = O.tetrahedral_povm()
    Fc = O.classical_fidelity(O.born_probabilities(rho, M).real, O.born_probabilities(sig, M).real)
    assert O.fidelity(rho, sig) <= Fc + 1e-12
    # Fig. 6 caption: ideal fidelity of a depolarised 8-qubit pure state vs the pure state
    N = 8
    d = 1 << N
    psi = synth.haar_pure(N, 1)
    for lam in (0.0, 0.1, 0.3):
        rl = synth.depolarized(psi, lam)
        assert abs(O.fidelity_pure(rl, psi) - (1 - (1 - 1 / d) * lam)) < 1e-12
    # Fig. 3 caption: purity of the white-noise 10-qubit state
    N = 10
    d = 1 << N
    psi = synth.product_plus(N)
    for p in (0.0, 0.4, 1.0):
        r = synth.white_noise(psi, p)
        assert abs(np.sum(np.abs(r) ** 2) - ((1 - 1 / d) * p * p + 1 / d)) < 1e-12


def test_decomposed_fidelity_pins():
    """Sec. 2.3 eq. fq_decom (one decomposition) against eq. F_QF by the singular-value route, the
    pure-target form <psi|rho^|psi>, a closed form, and the network's own decomposition of T."""
    rng = np.random.default_rng(5)
    for N, r1, r2 in ((2, 1, 4), (3, 3, 2), (4, 16, 5)):
        rt = synth.ginibre_mixed(N, r1, 10 + N)
        rho = synth.ginibre_mixed(N, r2, 20 + N)
        ev, Q = np.linalg.eigh(rt)
        got = O.fidelity_decomposed(Q, ev, rho)
        assert abs(got - O.fidelity(rt, rho)) < 1e-7 * max(got, 1e-3), (N, got)
        # the roles swap (eq. F_QF is symmetric): decompose the other state
        ev2, Q2 = np.linalg.eigh(rho)
        assert abs(O.fidelity_decomposed(Q2, ev2, rt) - got) < 1e-7
    # closed form: a pure rho~ = |phi><phi| against w |psi><psi| + (1 - w) I / d
    N, d = 3, 8
    phi = synth.haar_pure(N, 3)
    psi = synth.haar_pure(N, 4)
    Q = np.linalg.qr(np.column_stack([phi] + [rng.standard_normal(d) + 1j * rng.standard_normal(d)
                                              for _ in range(d - 1)]))[0]
    sigma = np.zeros(d)
    sigma[0] = 1.0
    for w in (0.0, 0.35, 1.0):
        want = w * abs(np.vdot(phi, psi)) ** 2 + (1 - w) / d
        # the d - 1 zero eigenvalues come out at ~1e-17, their square roots at ~3e-9
        assert abs(O.fidelity_decomposed(Q, sigma, O.noisy_target(psi, w)) - want) < 1e-7
    # the network's state: Chol_H and A_P, mixed and pure targets
    M = O.tetrahedral_povm()
    N = 3
    psi = synth.haar_pure(N, 7)
    f = O.born_probabilities(synth.depolarized(psi, 0.2), M).real
    theta = synth.init_theta(N, 8)
    for mapping, P in (("chol_h", 2.0), ("abs_p", 1.5), ("abs_p", 1.0)):
        rh = O.state_from_theta(theta, f, N, mapping=mapping, P=P)
        for w in (1.0, 0.8, 0.1):
            got = O.state_fidelity_decomposed(theta, f, N, psi, w, mapping=mapping, P=P)
            assert abs(got - O.fidelity(rh, O.noisy_target(psi, w))) < 1e-7
        # w = 1: M is rank one, its other 7 eigenvalues come out at ~1e-17 (square roots ~3e-9)
        assert abs(O.state_fidelity_decomposed(theta, f, N, psi, 1.0, mapping=mapping, P=P)
                   - O.fidelity_pure(rh, psi)) < 1e-7
    with pytest.raises(ValueError):
        O.state_fidelity_decomposed(theta, f, N, psi, 0.5, mapping="chol_delta")


def test_reconstruction_from_exact_probabilities_reaches_target():
    """Sec. 4.2: Chol_H reaches fidelity ~1 from exact (noise-free) probabilities."""
    M = O.tetrahedral_povm()
    N = 2
    psi = synth.haar_pure(N, 1)
    rho_t = synth.pure_density(psi)
    f = O.born_probabilities(rho_t, M).real
    theta0 = synth.init_theta(N, 1)
    _, rho, losses = O.reconstruct(theta0, f, M, N, 1000)
    assert O.fidelity_pure(rho, psi) > 0.99
    assert losses[-1] < losses[0]


def test_splitmix64_matches_published_outputs(golden_dir):
    lines = [l.split() for l in open(os.path.join(golden_dir, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    seed = int(lines[0][1])
    want = np.array([int(l[0]) for l in lines[1:]], dtype=np.uint64)
    np.testing.assert_array_equal(O.splitmix64(seed, np.arange(want.size)), want)


def test_sampled_classical_fidelity_pins():
    """Sec. 2.3 eq. fc_sample: equal distributions give exactly 1; the estimate converges to eq. F_CF;
    the draws follow P_hat (chi-square against the expected counts)."""
    rng = np.random.default_rng(5)
    n = 256
    P = rng.dirichlet(np.ones(n))
    assert O.sampled_classical_fidelity(P, P, 1000, 7) == pytest.approx(1.0, abs=1e-15)
    Ph = rng.dirichlet(np.ones(n) * 3)
    exact = O.classical_fidelity(Ph, P)
    S = 400_000
    est = O.sampled_classical_fidelity(Ph, P, S, 11)
    r = np.sqrt(P / Ph)
    se = 2 * np.sqrt(exact) * np.sqrt(np.sum(Ph * r ** 2) - exact) / np.sqrt(S)  # delta method
    assert abs(est - exact) < 5 * se, (est, exact, se)
    # the inverse-CDF draws have the distribution P_hat
    c = np.cumsum(Ph)
    u = (O.splitmix64(3, np.arange(S)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    k = np.searchsorted(c, u * c[-1], side="right")
    counts = np.bincount(k, minlength=n)
    chi2 = np.sum((counts - S * Ph) ** 2 / (S * Ph))
    assert chi2 < n + 5 * np.sqrt(2 * n)
    # zero-probability outcomes are never drawn
    Pz = Ph.copy(); Pz[::3] = 0; Pz /= Pz.sum()
    c = np.cumsum(Pz)
    k = np.searchsorted(c, u * c[-1], side="right")
    assert np.all(Pz[k] > 0)


def test_integer_multinomial_sampler_pins():
    """Sec. 4 sampling: counts sum to the shots, never land on zero-probability outcomes, follow P
    (chi-square), and a one-outcome distribution takes every shot."""
    rng = np.random.default_rng(8)
    n = 64
    P = rng.dirichlet(np.ones(n))
    P[::5] = 0.0
    P /= P.sum()
    S = 200_000
    c = O.multinomial_counts_integer(P, S, 21)
    assert c.sum() == S and np.all(c[P == 0] == 0)
    m = P > 0
    chi2 = np.sum((c[m] - S * P[m]) ** 2 / (S * P[m]))
    dof = m.sum() - 1
    assert chi2 < dof + 5 * np.sqrt(2 * dof)
    one = np.zeros(n); one[17] = 1.0
    assert np.array_equal(O.multinomial_counts_integer(one, 1000, 3), 1000 * (np.arange(n) == 17))
    # same seed, same counts; another seed, other counts
    assert np.array_equal(O.multinomial_counts_integer(P, 5000, 4), O.multinomial_counts_integer(P, 5000, 4))
    assert not np.array_equal(O.multinomial_counts_integer(P, 5000, 4), O.multinomial_counts_integer(P, 5000, 5))


def test_cnn_conv_and_pool_match_library_routines():
    """App. A: the 3 x 3 convolution with zero padding is scipy's 2-D correlation plus the bias; the
    pooled features are the maxima of ReLU(conv) over 2^(N-3)-square windows (block-reshape max)."""
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(12)
    for N in (3, 4, 5):
        d = 1 << N
        f = rng.dirichlet(np.ones(d * d))
        th = synth.init_theta_cnn(N, 13 + N)
        W2T, b2, W1, b1, cW, cB = O.unpack_theta_cnn(th, N)
        conv = O.conv3x3(f.reshape(d, d), cW, cB)
        for c in range(O.CNN_MAPS):
            want = scipy_signal.correlate2d(f.reshape(d, d), cW[c], mode="same", boundary="fill") + cB[c]
            np.testing.assert_allclose(conv[c], want, atol=1e-15)
        feats, pos, vals = O.cnn_features(f, cW, cB, N)
        p = d // O.CNN_GRID
        blocks = np.maximum(conv, 0).reshape(O.CNN_MAPS, O.CNN_GRID, p, O.CNN_GRID, p).max(axis=(2, 4))
        np.testing.assert_allclose(feats, blocks.ravel(), atol=1e-15)
        assert feats.size == 640 and th.size == synth.theta_size_cnn(N)


def test_gradient_central_fd_cnn_sampled():
    """The CNN network's backward (dense layers, max-pool routing, convolution) against central differences:
    every convolution parameter and a sample of the dense ones."""
    M = O.tetrahedral_povm()
    N = 3
    rho = synth.ginibre_mixed(N, 4, 70)
    f = O.born_probabilities(rho, M).real  # distinct entries: no pooling ties
    theta = synth.init_theta_cnn(N, 71)
    L, g, _ = O.loss_and_grad(theta, f, M, N, network="cnn")
    rng = np.random.default_rng(3)
    n_conv = 100
    idx = np.r_[np.arange(theta.size - n_conv, theta.size), rng.choice(theta.size - n_conv, 60, replace=False)]
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (O.loss_and_grad(tp, f, M, N, network="cnn")[0] - O.loss_and_grad(tm, f, M, N, network="cnn")[0]) / (2 * h)
        assert abs(fd - g[i]) <= 2e-6 * max(1.0, np.abs(g).max()), (i, fd, g[i])
    assert np.abs(g[-n_conv:]).max() > 0  # the convolution does receive gradient


def test_network_forward_hand_values():
    """Sec. 3.1 at N = 1 (4 inputs, 2 hidden units, 4 outputs), values worked out by hand.

    One hidden pre-activation is negative, so the LeakyReLU slope (0.01, Sec. 4.1 reading) is
    hit: with ReLU, slope 0.1 or an untransposed output layer the outputs differ.
      pre = W1 f + b1 = (3 + 0.5, -0.1 - 0.4) = (3.5, -0.5),  h = (3.5, -0.005)
      t_i = sum_j W2^T[j][i] h_j + b2_i = (3.5 - 0.5 + 0.25, -1 + 0.5, -3.5 + 1, 7 + 0.5 - 2)
    """
    f = np.array([0.1, 0.2, 0.3, 0.4])
    W1 = np.array([[1.0, 2.0, 3.0, 4.0], [-1.0, 0.0, 0.0, 0.0]])
    b1 = np.array([0.5, -0.4])
    W2T = np.array([[1.0, 0.0, -1.0, 2.0], [100.0, 200.0, 0.0, -100.0]])
    b2 = np.array([0.25, 0.5, 1.0, -2.0])
    theta = np.concatenate([W1.ravel(), W2T.ravel(), b2, b1])
    pre, h, t = O.network_forward(theta, f, 1)
    np.testing.assert_allclose(pre, [3.5, -0.5], rtol=0, atol=1e-14)
    np.testing.assert_allclose(h, [3.5, -0.005], rtol=0, atol=1e-14)
    np.testing.assert_allclose(t, [3.25, -0.5, -2.5, 5.5], rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.leaky_relu(np.array([-2.0, 0.0, 3.0])), [-0.02, 0.0, 3.0], rtol=0, atol=1e-15)


def test_theta_layout_markers():
    """theta = [W1 (H x n) | W2^T (H x n) | b2 (n) | b1 (H)], both matrices row-major."""
    N, n, H = 1, 4, 2
    theta = np.concatenate([1000 + np.arange(H * n), 2000 + np.arange(H * n), 3000 + np.arange(n),
                            4000 + np.arange(H)]).astype(float)
    W1, W2T, b2, b1 = O.unpack_theta(theta, N)
    assert W1.shape == (H, n) and W2T.shape == (H, n)
    assert W1[1, 2] == 1000 + 1 * n + 2 and W2T[0, 3] == 2003 and W2T[1, 0] == 2000 + n
    assert b2[2] == 3002 and b1[1] == 4001
    np.testing.assert_array_equal(O.pack_theta(W1, W2T, b2, b1), theta)
    assert theta.size == synth.theta_size(N) == 2 * H * n + n + H


def _zero_one_plus_minus_povm():
    """{|0><0|, |1><1|, |+><+|, |-><-|} / 2: a valid POVM (sums to I) whose |1><1| outcome has
    probability exactly 0 on |0><0|."""
    kets = [np.array([1, 0]), np.array([0, 1]), np.array([1, 1]) / np.sqrt(2), np.array([1, -1]) / np.sqrt(2)]
    return np.stack([np.outer(k, k.conj()).astype(complex) / 2 for k in kets])


def test_likelihood_clamp_terms_by_hand():
    """Clamp reading of the likelihood (q_k < q_min with f_k > 0 becomes the constant -f_k log q_min):
    q = (2, 0, 1, 1), t = 4, f = 1/4 each:
      L = -(1/4)(log 2 + log q_min + 0 + 0) + log 4 = (7 log 2 - log q_min) / 4
      g = -f/q + 1/t on the live terms, 1/t on the clamped one: (1/8, 1/4, 0, 0)."""
    for qmin in (O.Q_MIN_FP64, O.Q_MIN_FP32):
        L, g, nc = O.likelihood_terms(np.array([2.0, 0.0, 1.0, 1.0]), np.full(4, 0.25), 4.0, qmin)
        assert nc == 1
        assert abs(L - (7 * np.log(2) - np.log(qmin)) / 4) < 1e-13 * abs(L)
        np.testing.assert_allclose(g, [0.125, 0.25, 0.0, 0.0], rtol=0, atol=1e-15)
    # negative values are clamped too; f_k = 0 terms are never counted
    L, g, nc = O.likelihood_terms(np.array([-1e-30, 0.0, 1.0]), np.array([0.5, 0.0, 0.5]), 1.0, 1e-20)
    assert nc == 1 and abs(L - (-0.5 * np.log(1e-20))) < 1e-12
    np.testing.assert_allclose(g, [1.0, 1.0, 0.5], rtol=0, atol=1e-15)
    # without clamps it is the paper's L = -sum f log p with p = q / t
    rng = np.random.default_rng(5)
    q = rng.uniform(0.1, 1, 16); f = rng.dirichlet(np.ones(16)); t = q.sum() * 1.7
    assert abs(O.likelihood_terms(q, f, t)[0] - O.nll(q / t, f)) < 1e-13


def test_loss_and_grad_clamp_case_by_hand():
    """N = 1 with the |0>, |1>, |+>, |-> POVM and theta giving t = (2, 0, 0, 0): T = diag(2, 0),
    X = diag(4, 0), t_X = 4, q = (2, 0, 1, 1); the |1><1| outcome is clamped.
      L = (7 log 2 - log q_min) / 4
      G_X = (1/8) |0><0|/2 + (1/4) |1><1|/2 = diag(1/16, 1/8);  Gam = T G_X + G_X T = diag(1/4, 0)
      dL/dt = (1/4, 0, 0, 0) = dL/db2; h = LeakyReLU(0) = 0, so every other gradient is 0."""
    M = _zero_one_plus_minus_povm()
    n, H = 4, 2
    theta = np.zeros(2 * H * n + n + H)
    theta[2 * H * n] = 2.0  # b2[0]
    f = np.full(4, 0.25)
    for qmin in (O.Q_MIN_FP64, O.Q_MIN_FP32):
        L, g, aux = O.loss_and_grad(theta, f, M, 1, q_min=qmin)
        assert aux["clamped"] == 1
        assert abs(L - (7 * np.log(2) - np.log(qmin)) / 4) < 1e-13 * abs(L)
        want = np.zeros_like(theta)
        want[2 * H * n] = 0.25
        np.testing.assert_allclose(g, want, rtol=0, atol=1e-15)
