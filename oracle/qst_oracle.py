"""Plain FP64 CPU oracle of the NN-QST maximum-likelihood iteration (arXiv:2207.05341).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library.

Everything is NumPy in float64 / complex128, written for clarity and checked
against the paper's mathematics by the tests in ``tests/test_oracle_*.py``:
a brute-force Kronecker expansion of the POVM map, closed forms, invariants,
central finite differences of the loss and a hand-computed Rprop sequence.

The steps follow the paper in this order:
  Sec. 3.1  network: input f (the measured frequencies, length K^N), hidden
            width 2N with LeakyReLU, linear output of 4^N reals;
  Sec. 3.2  the 4^N reals become a Hermitian T, then either the unified
            decomposition rho = T^dag T / Tr(T^dag T)   (eq. unified_DP, "Chol_H")
            or the P-order absolute projection
            rho = Q |Lambda|^P Q^dag / Tr|Lambda|^P     (eq. abs_P, "A_P");
  Sec. 2.2.1 alternatively a complex lower-triangular T and
            rho = T^dag T / Tr(T^dag T)                 (eq. T_matrix, "Chol_Delta");
  Sec. 3.3  probabilities P_k = Tr[(M_k1 x ... x M_kN) rho]  (eq. PS);
  Sec. 3.1  loss L = -sum_k f_k log P_k;
  Sec. 4.1  LeakyReLU hidden layer, Rprop with learning rate 0.001.

Readings where the paper is silent (each also listed in the design notes):
  * the 4^N outputs t become R = t reshaped row-major to d x d, and
    T_ii = R_ii, T_ij = R_ij + i R_ji (i > j), T_ji = conj(T_ij);
    for Chol_Delta the same lower triangle with T_ji = 0 (i > j);
  * the output layer is linear; the LeakyReLU negative slope is 0.01;
  * Rprop: initial step lr, factors (0.5, 1.2), step bounds [1e-6, 50],
    sign(g * g_prev) decides the factor, and the gradient is zeroed where the
    sign flipped;
  * qubit 1 is the most significant factor of the Kronecker product and the
    most significant base-K digit of the outcome index k;
  * eq. PS writes b_i Tr[M_j B] for the second term; the Born rule of Sec. 2.1
    gives the coefficient (M_i)_{21} = c_i there, which is what is used;
  * terms with f_k = 0 contribute nothing to L; for A_P with P <= 1 the
    eigenvalue magnitudes are floored at eps * max|lambda| (eps = 1e-15);
  * a term with f_k > 0 whose unnormalised Born value q_k = Tr[M_k X] lies
    below q_min (the smallest normal number of the precision compared with;
    for the PSD X of the state maps only rounding can bring q_k to 0 or
    below) is clamped: it adds the constant -f_k log q_min to L, nothing to
    dL/dq_k, and is counted.

Parity unpinned: long multi-step Rprop trajectories (a sign-driven optimiser
amplifies rounding); single steps, gradients and final fidelities are pinned.
"""
from __future__ import annotations

import numpy as np

LEAKY_SLOPE = 0.01
RPROP_LR = 1e-3
RPROP_ETAS = (0.5, 1.2)
RPROP_STEP_BOUNDS = (1e-6, 50.0)
ABS_P_EPS = 1e-15

_I2 = np.eye(2, dtype=complex)
_SX = np.array([[0, 1], [1, 0]], dtype=complex)
_SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
_SZ = np.array([[1, 0], [0, -1]], dtype=complex)


# --------------------------------------------------------------------------
# Measurement model (Sec. 2.1, Sec. 3.3, Sec. 4.1)
# --------------------------------------------------------------------------

def tetrahedral_povm() -> np.ndarray:
    """Sec. 4.1: M_a = (I + s_a . sigma) / 4 with the four listed tetrahedron vectors s_a.

    Returns a (4, 2, 2) complex array.
    """
    s = np.array([[1, 1, 1], [-1, -1, 1], [-1, 1, -1], [1, -1, -1]], dtype=float) / np.sqrt(3.0)
    return np.stack([(_I2 + s[a, 0] * _SX + s[a, 1] * _SY + s[a, 2] * _SZ) / 4.0 for a in range(4)])


def _pair_axes(N: int) -> list[int]:
    # rho reshaped to (2,)*2N has axes i_1..i_N, j_1..j_N; this order puts (i_q, j_q) side by side.
    return [ax for q in range(N) for ax in (q, N + q)]


def born_probabilities(rho: np.ndarray, povm: np.ndarray) -> np.ndarray:
    """Sec. 3.3 eq. PS for N qubits: P_k = Tr[(M_k1 x ... x M_kN) rho], complex result.

    The trace against a product operator factorises over qubits: for qubit q the
    pair of indices (i_q, j_q) of rho is contracted with (M_{k_q})_{j_q i_q}
    (Born rule of Sec. 2.1, Tr[M X] = sum_ij M_ji X_ij).  The contraction is
    applied one qubit at a time, so the cost is N * K * 4^N instead of K^N 4^N.
    The imaginary part is returned too; it vanishes for Hermitian rho.
    """
    d = rho.shape[0]
    N = d.bit_length() - 1
    K = povm.shape[0]
    A = np.empty((K, 4), dtype=complex)
    for a in range(K):
        for i in range(2):
            for j in range(2):
                A[a, 2 * i + j] = povm[a][j, i]
    t = rho.reshape((2,) * (2 * N)).transpose(_pair_axes(N)).reshape((4,) * N)
    for q in range(N):
        t = np.moveaxis(np.tensordot(A, t, axes=([1], [q])), 0, q)
    return t.reshape(-1)


def born_probability_at(rho: np.ndarray, povm: np.ndarray, k: int) -> complex:
    """One outcome of eq. PS: Tr[(M_k1 x ... x M_kN) rho] for a single index k.

    Contracts each qubit's index pair of rho with its own M_{k_q}, one qubit at
    a time (cost O(d^2) per outcome), for spot checks of large problems.
    """
    d = rho.shape[0]
    N = d.bit_length() - 1
    K = povm.shape[0]
    digits = [(k // K ** (N - 1 - q)) % K for q in range(N)]
    t = rho.reshape((2,) * (2 * N)).transpose(_pair_axes(N)).reshape((4,) * N)
    for q in range(N):
        m = povm[digits[q]]
        a = np.array([m[j, i] for i in range(2) for j in range(2)])
        t = np.tensordot(a, t, axes=([0], [0]))
    return complex(t)


def povm_adjoint(g: np.ndarray, povm: np.ndarray) -> np.ndarray:
    """G = sum_k g_k (M_k1 x ... x M_kN): the adjoint of the real-linear map rho -> Re P.

    With <A, B> = Re Tr(A^dag B) on Hermitian matrices, sum_k g_k P_k = <G, rho>.
    Applied one qubit at a time like born_probabilities.
    """
    K = povm.shape[0]
    N = round(np.log(g.size) / np.log(K))
    B = np.empty((4, K), dtype=complex)
    for a in range(K):
        for i in range(2):
            for j in range(2):
                B[2 * i + j, a] = povm[a][i, j]
    t = np.asarray(g, dtype=complex).reshape((K,) * N)
    for q in range(N):
        t = np.moveaxis(np.tensordot(B, t, axes=([1], [q])), 0, q)
    inv = np.argsort(_pair_axes(N))
    d = 1 << N
    return t.reshape((2,) * (2 * N)).transpose(inv).reshape(d, d)


# --------------------------------------------------------------------------
# Network (Sec. 3.1, Sec. 4.1)
# --------------------------------------------------------------------------

def unpack_theta(theta: np.ndarray, N: int):
    """Split the flat parameter vector [W1 (H x n) | W2^T (H x n) | b2 (n) | b1 (H)]."""
    n, H = 4 ** N, 2 * N
    o = 0
    W1 = theta[o:o + H * n].reshape(H, n); o += H * n
    W2T = theta[o:o + H * n].reshape(H, n); o += H * n
    b2 = theta[o:o + n]; o += n
    b1 = theta[o:o + H]; o += H
    assert o == theta.size
    return W1, W2T, b2, b1


def pack_theta(W1, W2T, b2, b1) -> np.ndarray:
    return np.concatenate([np.ravel(W1), np.ravel(W2T), np.ravel(b2), np.ravel(b1)])


def leaky_relu(x: np.ndarray) -> np.ndarray:
    return np.where(x > 0, x, LEAKY_SLOPE * x)


def network_forward(theta: np.ndarray, f: np.ndarray, N: int):
    """Sec. 3.1: K^N inputs -> 2N hidden (LeakyReLU) -> 4^N linear outputs.

    Returns (pre, h, t): hidden pre-activation, hidden activation, output.
    """
    W1, W2T, b2, b1 = unpack_theta(theta, N)
    pre = W1 @ f + b1
    h = leaky_relu(pre)
    t = W2T.T @ h + b2
    return pre, h, t


# --------------------------------------------------------------------------
# The CNN mapping network of App. A
# --------------------------------------------------------------------------

CNN_MAPS = 10  # feature maps of the 3 x 3 convolution
CNN_GRID = 8   # pooled grid per map (the pooling window is 2^(N-3) square): 10 x 8 x 8 = 640 features


def cnn_sizes(N: int):
    """(n, H, F): outputs 4^N, hidden width 4N, pooled features 640."""
    return 4 ** N, 4 * N, CNN_MAPS * CNN_GRID ** 2


def unpack_theta_cnn(theta: np.ndarray, N: int):
    """[W2^T (H x n) | b2 (n) | W1 (H x F) | b1 (H) | conv W (10 x 3 x 3) | conv b (10)]."""
    n, H, F = cnn_sizes(N)
    o = 0
    W2T = theta[o:o + H * n].reshape(H, n); o += H * n
    b2 = theta[o:o + n]; o += n
    W1 = theta[o:o + H * F].reshape(H, F); o += H * F
    b1 = theta[o:o + H]; o += H
    cW = theta[o:o + CNN_MAPS * 9].reshape(CNN_MAPS, 3, 3); o += CNN_MAPS * 9
    cB = theta[o:o + CNN_MAPS]; o += CNN_MAPS
    assert o == theta.size
    return W2T, b2, W1, b1, cW, cB


def pack_theta_cnn(W2T, b2, W1, b1, cW, cB) -> np.ndarray:
    return np.concatenate([np.ravel(W2T), np.ravel(b2), np.ravel(W1), np.ravel(b1), np.ravel(cW), np.ravel(cB)])


def conv3x3(img: np.ndarray, cW: np.ndarray, cB: np.ndarray, dtype=np.float64) -> np.ndarray:
    """App. A: 3 x 3 convolution, stride 1, zero padding 1, 10 maps with bias.

    out[c, y, x] = b_c + sum_{ky, kx} W[c, ky, kx] img[y + ky - 1, x + kx - 1], accumulated in `dtype`
    in the order bias, then (ky, kx) row-major, each product and sum rounded to `dtype` (so a float32
    evaluation decides the pooling argmax exactly as a float32 kernel that accumulates in this order).
    """
    d = img.shape[0]
    pad = np.zeros((d + 2, d + 2), dtype=dtype)
    pad[1:-1, 1:-1] = img.astype(dtype)
    out = np.empty((cW.shape[0], d, d), dtype=dtype)
    for c in range(cW.shape[0]):
        acc = np.full((d, d), dtype(cB[c]), dtype=dtype)
        for ky in range(3):
            for kx in range(3):
                acc = acc + dtype(cW[c, ky, kx]) * pad[ky:ky + d, kx:kx + d]
        out[c] = acc
    return out


def cnn_features(f: np.ndarray, cW, cB, N: int, decision=np.float64):
    """App. A: f as a d x d matrix (row-major) -> conv -> ReLU -> max-pool (window 2^(N-3), stride the
    same) -> 640 features.  The argmax of each window is taken on the `decision`-precision convolution
    (first row-major index on ties); the feature is ReLU of the FP64 convolution there.
    Returns (features (640,), argmax positions (640, 2), FP64 convolution at them)."""
    d = 1 << N
    p = d // CNN_GRID
    img = np.asarray(f, dtype=np.float64).reshape(d, d)
    conv_dec = conv3x3(img, cW, cB, decision)
    conv64 = conv3x3(img, cW, cB, np.float64)
    feats, pos, vals = [], [], []
    for c in range(CNN_MAPS):
        for I in range(CNN_GRID):
            for J in range(CNN_GRID):
                win = conv_dec[c, I * p:(I + 1) * p, J * p:(J + 1) * p]
                a = int(np.argmax(win))
                y, x = I * p + a // p, J * p + a % p
                v = conv64[c, y, x]
                feats.append(max(v, 0.0)); pos.append((y, x)); vals.append(v)
    return np.array(feats), np.array(pos), np.array(vals)


def network_forward_cnn(theta: np.ndarray, f: np.ndarray, N: int, decision=np.float64):
    """App. A network: features (640) -> 4N hidden (LeakyReLU) -> 4^N linear outputs."""
    W2T, b2, W1, b1, cW, cB = unpack_theta_cnn(theta, N)
    feats, pos, vals = cnn_features(f, cW, cB, N, decision)
    pre = W1 @ feats + b1
    h = leaky_relu(pre)
    t = W2T.T @ h + b2
    return pre, h, t, feats, pos, vals


def network_backward_cnn(theta, f, N, dt, pre, h, feats, pos, vals):
    """Chain rule of the App. A network back from dL/dt to dL/dtheta (CNN layout)."""
    W2T, b2, W1, b1, cW, cB = unpack_theta_cnn(theta, N)
    d = 1 << N
    dW2T = np.outer(h, dt)
    db2 = dt
    dh = W2T @ dt
    dpre = dh * np.where(pre > 0, 1.0, LEAKY_SLOPE)
    dW1 = np.outer(dpre, feats)
    db1 = dpre
    dfeat = W1.T @ dpre
    pad = np.zeros((d + 2, d + 2))
    pad[1:-1, 1:-1] = np.asarray(f, dtype=np.float64).reshape(d, d)
    dcW = np.zeros((CNN_MAPS, 3, 3))
    dcB = np.zeros(CNN_MAPS)
    for i in range(CNN_MAPS * CNN_GRID ** 2):
        if vals[i] <= 0:
            continue  # ReLU'(conv) = 0 at the pooled position
        c = i // CNN_GRID ** 2
        y, x = pos[i]
        dcW[c] += dfeat[i] * pad[y:y + 3, x:x + 3]
        dcB[c] += dfeat[i]
    return pack_theta_cnn(dW2T, db2, dW1, db1, dcW, dcB)


def hermitian_from_output(t: np.ndarray) -> np.ndarray:
    """Sec. 3.1/3.2: the 4^N real outputs become a Hermitian d x d matrix T.

    R = t reshaped row-major to d x d; the diagonal of T is R's diagonal, the
    strict lower triangle is R_ij + i R_ji and the upper triangle its conjugate.
    """
    d = int(round(np.sqrt(t.size)))
    R = t.reshape(d, d)
    L = np.tril(R, -1) + 1j * np.tril(R.T, -1)
    return L + L.conj().T + np.diag(np.diag(R))


def lower_from_output(t: np.ndarray) -> np.ndarray:
    """Sec. 2.2.1 eq. T_matrix: the 4^N real outputs become a complex lower-triangular T.

    The same R = t reshaped row-major as for the Hermitian T: the diagonal of T is
    R's diagonal, the strict lower triangle is R_ij + i R_ji, the upper triangle is 0.
    """
    d = int(round(np.sqrt(t.size)))
    R = t.reshape(d, d)
    return np.tril(R, -1) + 1j * np.tril(R.T, -1) + np.diag(np.diag(R))


def output_grad_from_lower(Gam: np.ndarray) -> np.ndarray:
    """Pull a gradient back through lower_from_output.

    Gam is any complex matrix with dL = Re Tr[Gam dT] for lower-triangular dT.
    dT_ii = dR_ii, and for i > j dT_ij = dR_ij + i dR_ji, so
    dL/dR_ii = Re Gam_ii, dL/dR_ij = Re Gam_ji and dL/dR_ji = -Im Gam_ji.
    Returned flat, row-major, like t.
    """
    d = Gam.shape[0]
    dR = np.zeros((d, d))
    il = np.tril_indices(d, -1)
    GT = Gam.T
    dR[il] = GT[il].real
    dR[(il[1], il[0])] = -GT[il].imag
    dR[np.diag_indices(d)] = np.diag(Gam).real
    return dR.ravel()


def output_grad_from_hermitian(Gam: np.ndarray) -> np.ndarray:
    """Pull a gradient back through hermitian_from_output.

    Gam is the Hermitian matrix with dL = Re Tr[Gam dT] for Hermitian dT.
    Then dL/dR_ii = Gam_ii, and for i > j: dL/dR_ij = 2 Re Gam_ij and
    dL/dR_ji = 2 Im Gam_ij.  Returned flat, row-major, like t.
    """
    d = Gam.shape[0]
    dR = np.zeros((d, d))
    il = np.tril_indices(d, -1)
    dR[il] = 2.0 * Gam[il].real
    dR[(il[1], il[0])] = 2.0 * Gam[il].imag
    dR[np.diag_indices(d)] = np.diag(Gam).real
    return dR.ravel()


# --------------------------------------------------------------------------
# State mapping (Sec. 3.2)
# --------------------------------------------------------------------------

def chol_delta(T: np.ndarray) -> np.ndarray:
    """Sec. 2.2.1 eq. T_matrix: rho = T^dag T / Tr(T^dag T) for lower-triangular T."""
    X = T.conj().T @ T
    return X / np.trace(X).real


def chol_h(T: np.ndarray) -> np.ndarray:
    """Sec. 3.2 eq. unified_DP: rho = T^dag T / Tr(T^dag T) for Hermitian T."""
    X = T.conj().T @ T
    return X / np.trace(X).real


def _abs_p_spectrum(T: np.ndarray, P: float):
    """Sec. 3.2 eq. abs_P on T = Q Lambda Q^dag: returns (lam, Q, g, g') with g = |lambda|^P
    (magnitudes floored at ABS_P_EPS * max|lambda| for P <= 1) and g' = dg/dlambda (0 below the floor)."""
    lam, Q = np.linalg.eigh(T)
    a = np.abs(lam)
    floor = ABS_P_EPS * a.max() if P <= 1.0 else 0.0
    a_used = np.maximum(a, floor)
    g = a_used ** P
    gp = np.where(a > floor, P * a_used ** (P - 1.0) * np.sign(lam), 0.0)
    return lam, Q, g, gp


def abs_p_unnormalised(T: np.ndarray, P: float) -> np.ndarray:
    """S = Q |Lambda|^P Q^dag, so that eq. abs_P reads rho = S / Tr S."""
    lam, Q, g, _ = _abs_p_spectrum(T, P)
    return (Q * g) @ Q.conj().T


def abs_p(T: np.ndarray, P: float) -> np.ndarray:
    """Sec. 3.2 eq. abs_P: T = Q Lambda Q^dag, rho = Q |Lambda|^P Q^dag / Tr |Lambda|^P."""
    lam, Q, g, _ = _abs_p_spectrum(T, P)
    return (Q * (g / g.sum())) @ Q.conj().T


def _abs_p_backward(T: np.ndarray, P: float, G_S: np.ndarray) -> np.ndarray:
    """Gradient of L through S = Q g(Lambda) Q^dag, g = |lambda|^P: returns Gam with dL = Re Tr[Gam dT].

    G_S = dL/dS.  Through the spectral function the Daleckii-Krein formula gives
    Gam = Q (D o (Q^dag G_S Q)) Q^dag with D_ij = (g_i - g_j) / (lambda_i - lambda_j),
    or g'(lambda_i) when equal (the mean of the two derivatives).
    """
    lam, Q, g, gp = _abs_p_spectrum(T, P)
    C = Q.conj().T @ G_S @ Q
    li, lj = np.meshgrid(lam, lam, indexing="ij")
    gi, gj = np.meshgrid(g, g, indexing="ij")
    dl = li - lj
    same = np.abs(dl) <= 1e-13 * max(1.0, np.abs(lam).max())
    D = np.where(same, np.add.outer(gp, gp) / 2.0, (gi - gj) / np.where(same, 1.0, dl))
    Gam = Q @ (D * C) @ Q.conj().T
    return 0.5 * (Gam + Gam.conj().T)


# --------------------------------------------------------------------------
# Likelihood and its gradient (Sec. 2.1 eq. MLE, Sec. 3.1)
# --------------------------------------------------------------------------

def nll(p: np.ndarray, f: np.ndarray) -> float:
    """Sec. 3.1 loss L = -sum_k f_k log p_k, terms with f_k = 0 omitted."""
    m = f > 0
    return float(-np.sum(f[m] * np.log(p[m])))


Q_MIN_FP64 = float(np.finfo(np.float64).tiny)
Q_MIN_FP32 = float(np.finfo(np.float32).tiny)


def likelihood_terms(q: np.ndarray, f: np.ndarray, t: float, q_min: float = Q_MIN_FP64):
    """Sec. 3.1 / Sec. 2.1 eq. MLE on the unnormalised Born values q_k = Tr[M_k X] of X = t rho.

    With p_k = q_k / t:  L = -sum_k f_k log p_k = -sum_k f_k log q_k + (sum_k f_k) log t, and
    g_k = dL/dq_k = -f_k / q_k + (sum_k f_k) / t.  Terms with f_k = 0 are omitted from the sum (they
    keep g_k = sum f / t).  A term with f_k > 0 and q_k < q_min is clamped: it contributes the
    constant -f_k log q_min to L and its g_k keeps only sum f / t.
    Returns (L, g, number of clamped terms).
    """
    q = np.asarray(q, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    sumf = float(np.sum(f))
    pos = f > 0
    clamp = pos & ~(q >= q_min)
    live = pos & ~clamp
    L = -np.sum(f[live] * np.log(q[live])) - np.sum(f[clamp]) * np.log(q_min) + sumf * np.log(t)
    g = np.full(q.shape, sumf / t)
    g[live] -= f[live] / q[live]
    return float(L), g, int(np.count_nonzero(clamp))


def state_from_theta(theta, f, N, mapping="chol_h", P=2.0, network="fnn", decision=np.float64):
    if network == "cnn":
        t = network_forward_cnn(theta, f, N, decision)[2]
    else:
        pre, h, t = network_forward(theta, f, N)
    if mapping == "chol_delta":
        return chol_delta(lower_from_output(t))
    T = hermitian_from_output(t)
    rho = chol_h(T) if mapping == "chol_h" else abs_p(T, P)
    return rho


def loss_and_grad(theta, f, povm, N, mapping="chol_h", P=2.0, network="fnn", decision=np.float64,
                  q_min=Q_MIN_FP64):
    """One forward and backward pass of the Sec. 3 network through the likelihood.

    Returns (L, dL/dtheta, aux) with aux holding rho, p and the intermediates
    (and "clamped", the number of terms clamped at q_min; see likelihood_terms).
    The state map gives an unnormalised S with rho = S / t, t = Tr S
    (Chol_H / Chol_Delta: S = X = T^dag T; A_P: S = Q |Lambda|^P Q^dag); then
      q_k       = Tr[M_k S]                               (eq. PS on S; p = q / t)
      L, g_k    = likelihood_terms(q, f, t):  L = -sum f log q + (sum f) log t,
                  g_k = dL/dq_k = -f_k / q_k + (sum f) / t
      G_S       = sum_k g_k M_k                           (POVM adjoint; dL/dS)
      Chol_H:   Gam = T G_S + G_S T            (dS = dT T + T dT for Hermitian T)
      Chol_Delta: dS = dT^dag T + T^dag dT gives dL = 2 Re Tr[G_S T^dag dT], Gam = 2 G_S T^dag
      A_P:      Daleckii-Krein (see _abs_p_backward)
      t         <- Gam (output_grad_from_hermitian, or output_grad_from_lower)
      W2^T, b2, h <- t;  pre <- h (LeakyReLU');  W1, b1 <- pre.
    """
    if network == "cnn":
        pre, h, t, feats, pos, vals = network_forward_cnn(theta, f, N, decision)
    else:
        W1, W2T, b2, b1 = unpack_theta(theta, N)
        pre, h, t = network_forward(theta, f, N)
    T = lower_from_output(t) if mapping == "chol_delta" else hermitian_from_output(t)
    if mapping in ("chol_h", "chol_delta"):
        S = T.conj().T @ T
    else:
        S = abs_p_unnormalised(T, P)
    tS = np.trace(S).real
    rho = S / tS
    q = born_probabilities(S, povm).real
    L, gq, nclamp = likelihood_terms(q, f, tS, q_min)
    G_S = povm_adjoint(gq, povm)
    if mapping == "chol_h":
        Gam = T @ G_S + G_S @ T
    elif mapping == "chol_delta":
        Gam = 2.0 * G_S @ T.conj().T
    else:
        Gam = _abs_p_backward(T, P, G_S)
    dt = output_grad_from_lower(Gam) if mapping == "chol_delta" else output_grad_from_hermitian(Gam)
    aux = dict(rho=rho, p=q / tS, T=T, t=t, h=h, pre=pre, Gam=Gam, dt=dt, clamped=nclamp)
    if network == "cnn":
        grad = network_backward_cnn(theta, f, N, dt, pre, h, feats, pos, vals)
        return L, grad, aux

    db2 = dt
    dW2T = np.outer(h, dt)
    dh = W2T @ dt
    dpre = dh * np.where(pre > 0, 1.0, LEAKY_SLOPE)
    db1 = dpre
    dW1 = np.outer(dpre, f)
    grad = pack_theta(dW1, dW2T, db2, db1)
    return L, grad, aux


# --------------------------------------------------------------------------
# Optimiser (Sec. 4.1: Rprop, learning rate 0.001)
# --------------------------------------------------------------------------

class RpropState:
    """Per-parameter Rprop state: the step sizes and the previous (masked) gradient's sign."""

    def __init__(self, size: int, lr: float = RPROP_LR):
        self.step = np.full(size, lr, dtype=np.float64)
        self.prev_sign = np.zeros(size, dtype=np.int8)


def rprop_update(theta, grad, state: RpropState,
                 etas=RPROP_ETAS, bounds=RPROP_STEP_BOUNDS):
    """One Rprop update (sign-based step adaptation).

    For each parameter: c = sign(g) * sign(g_prev); the step grows by etas[1]
    when c > 0, shrinks by etas[0] when c < 0, and stays otherwise; it is then
    clamped to ``bounds``.  Where c < 0 the gradient is treated as 0 (no move
    this time, and it is remembered as 0).  The parameter moves by
    -sign(g) * step.  Returns the new theta; ``state`` is updated in place.
    """
    sg = np.sign(grad).astype(np.int8)
    c = sg * state.prev_sign
    factor = np.where(c > 0, etas[1], np.where(c < 0, etas[0], 1.0))
    state.step = np.clip(state.step * factor, bounds[0], bounds[1])
    sg = np.where(c < 0, 0, sg).astype(np.int8)
    state.prev_sign = sg
    return theta - sg * state.step


def reconstruct(theta0, f, povm, N, iters, mapping="chol_h", P=2.0, callback=None, network="fnn",
                decision=np.float64):
    """The NN-QST loop of Fig. 1: forward, likelihood, backward, Rprop, repeated.

    Returns (theta, rho, losses).  ``callback(it, rho)`` runs after each step
    if given (for fidelity tracking).
    """
    theta = np.array(theta0, dtype=np.float64)
    st = RpropState(theta.size)
    losses = []
    for it in range(iters):
        L, g, aux = loss_and_grad(theta, f, povm, N, mapping, P, network, decision)
        losses.append(L)
        theta = rprop_update(theta, g, st)
        if callback is not None:
            callback(it, aux["rho"])
    rho = state_from_theta(theta, f, N, mapping, P, network, decision)
    return theta, rho, np.array(losses)


# --------------------------------------------------------------------------
# Evaluation (Sec. 2.3)
# --------------------------------------------------------------------------

def _psd_sqrt(A: np.ndarray) -> np.ndarray:
    w, V = np.linalg.eigh(0.5 * (A + A.conj().T))
    return (V * np.sqrt(np.clip(w, 0.0, None))) @ V.conj().T


def fidelity(rho_hat: np.ndarray, rho: np.ndarray) -> float:
    """Sec. 2.3 eq. F_QF: (Tr sqrt(sqrt(rho_hat) rho sqrt(rho_hat)))^2.

    Evaluated as the squared sum of singular values of sqrt(rho_hat) sqrt(rho),
    which equals the trace in eq. F_QF and avoids a second matrix square root.
    """
    s = np.linalg.svd(_psd_sqrt(rho_hat) @ _psd_sqrt(rho), compute_uv=False)
    return float(np.sum(s) ** 2)


def fidelity_pure(rho_hat: np.ndarray, psi: np.ndarray) -> float:
    """Sec. 2.3: for a pure target the fidelity reduces to <psi| rho_hat |psi>."""
    return float(np.real(np.vdot(psi, rho_hat @ psi)))


def fidelity_decomposed(Q: np.ndarray, sigma: np.ndarray, rho: np.ndarray) -> float:
    """Sec. 2.3 eq. fq_decom: with rho~ = Q diag(sigma) Q^dag known, F_q(rho~, rho) = (sum_i sqrt(s'_i))^2,
    s' the eigenvalues of Q sqrt(Sigma) Q^dag rho Q sqrt(Sigma) Q^dag (clamped at 0): one decomposition."""
    S = (Q * np.sqrt(np.clip(sigma, 0.0, None))) @ Q.conj().T
    M = S @ rho @ S
    ev = np.linalg.eigvalsh(0.5 * (M + M.conj().T))
    return float(np.sum(np.sqrt(np.clip(ev, 0.0, None))) ** 2)


def noisy_target(psi: np.ndarray, w: float) -> np.ndarray:
    """The targets of the Sec. 4 sweeps: w |psi><psi| / <psi|psi> + (1 - w) I / d (white noise with
    p = w, the depolarising channel with lambda = 1 - w, the pure state with w = 1)."""
    u = np.asarray(psi, dtype=np.complex128)
    u = u / np.linalg.norm(u)
    d = u.size
    return w * np.outer(u, u.conj()) + (1.0 - w) * np.eye(d) / d


def state_fidelity_decomposed(theta, f, N, psi, w, mapping="chol_h", P=2.0, network="fnn",
                              decision=np.float64) -> float:
    """F_q of the network's state against noisy_target(psi, w) through eq. fq_decom, with the
    decomposition of rho^ taken from that of T (Sec. 3.2): T = Q Lambda Q^dag gives
    rho^ = Q diag(g) Q^dag / sum g, g = lambda^2 for Chol_H (T^dag T = T^2 for Hermitian T) and
    g = |lambda|^P for A_P (with its floor for P <= 1)."""
    if mapping not in ("chol_h", "abs_p"):
        raise ValueError("eq. fq_decom needs the decomposition of a Hermitian T")
    t = network_forward_cnn(theta, f, N, decision)[2] if network == "cnn" else network_forward(theta, f, N)[2]
    lam, Q = np.linalg.eigh(hermitian_from_output(t))
    if mapping == "chol_h":
        g = lam ** 2
    else:
        a = np.abs(lam)
        if P <= 1.0:
            a = np.maximum(a, ABS_P_EPS * a.max())
        g = a ** P
    return fidelity_decomposed(Q, g / g.sum(), noisy_target(psi, w))


def classical_fidelity(P_hat: np.ndarray, P: np.ndarray) -> float:
    """Sec. 2.3 eq. F_CF: (sum_k sqrt(P_hat_k P_k))^2, an upper bound on F_q."""
    return float(np.sum(np.sqrt(np.clip(P_hat, 0, None) * np.clip(P, 0, None))) ** 2)


_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB


def splitmix64(seed: int, s: np.ndarray) -> np.ndarray:
    """Output s (0-based) of the SplitMix64 generator started at `seed` (Steele, Lea and Flood,
    OOPSLA 2014): x = seed + (s + 1) * gamma, then the published two-round mix of x."""
    s = np.asarray(s, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (s + np.uint64(1)) * np.uint64(_SM_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_M2)
    return z ^ (z >> np.uint64(31))


def multinomial_counts_integer(P: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Seeded multinomial counts by integer inverse CDF (the sampler of the synthetic sweeps, Sec. 4).

    Weights w_k = floor(max(P_k, 0) 2^52), exact running sums C, W = C[-1]; draw s takes
    t_s = floor((splitmix64(seed, s) >> 11) W / 2^53) and counts k_s = the smallest k with C_k > t_s.
    """
    w = np.floor(np.clip(np.asarray(P, dtype=np.float64), 0, None) * 2.0 ** 52).astype(np.uint64)
    C = np.cumsum(w, dtype=np.uint64)
    W = int(C[-1])
    a = (splitmix64(seed, np.arange(shots)) >> np.uint64(11)).astype(object)
    t = np.array([(int(x) * W) >> 53 for x in a], dtype=np.uint64)
    k = np.searchsorted(C, t, side="right")
    return np.bincount(k, minlength=w.size).astype(np.int64)


def sampled_classical_fidelity(P_hat: np.ndarray, P: np.ndarray, samples: int, seed: int) -> float:
    """Sec. 2.3 eq. fc_sample: F_c ~ (E_{k ~ P_hat}[sqrt(P_k / P_hat_k)])^2 from `samples` draws.

    Draw s takes u_s = (splitmix64(seed, s) >> 11) 2^-53 in [0, 1) and k_s, the smallest k with
    c_k > u_s c_{n-1}, where c is the running sum of max(P_hat, 0) (inverse CDF).
    """
    ph = np.clip(P_hat, 0, None)
    c = np.cumsum(ph)
    u = (splitmix64(seed, np.arange(samples)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    k = np.searchsorted(c, u * c[-1], side="right")
    return float(np.mean(np.sqrt(np.clip(P[k], 0, None) / ph[k])) ** 2)
