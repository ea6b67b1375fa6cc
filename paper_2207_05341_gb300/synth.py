"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle's tests.

This module draws random numbers and builds the target states of Sec. 4
(Haar pure states, rank-r Ginibre mixtures, the depolarising channel and
white-noise mixtures of eq. "white noise", the product, GHZi and W states).
It holds none of the tomography method's arithmetic: no POVM map, no network,
no state mapping, no likelihood.  Measurement counts are drawn from
probabilities that the caller computes and passes in.

Everything here is NumPy on the host and never touches a GPU.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def haar_pure(N: int, seed: int) -> np.ndarray:
    """Haar-random pure state vector of N qubits (complex128, length 2^N).

    Drawn as a vector of i.i.d. standard complex normals, normalised.
    """
    d = 1 << N
    r = _rng(seed)
    z = r.standard_normal(d) + 1j * r.standard_normal(d)
    return z / np.linalg.norm(z)


def ginibre_mixed(N: int, rank: int, seed: int) -> np.ndarray:
    """Rank-r Ginibre mixed state rho = G G^dag / Tr(G G^dag), G a d x r complex normal matrix."""
    d = 1 << N
    if not 1 <= rank <= d:
        raise ValueError("rank must lie in [1, 2^N]")
    r = _rng(seed)
    g = r.standard_normal((d, rank)) + 1j * r.standard_normal((d, rank))
    rho = g @ g.conj().T
    rho /= np.trace(rho).real
    return 0.5 * (rho + rho.conj().T)


def pure_density(psi: np.ndarray) -> np.ndarray:
    """|psi><psi| as a dense matrix."""
    return np.outer(psi, psi.conj())


def depolarized(psi: np.ndarray, lam: float) -> np.ndarray:
    """Sec. 4, depolarising channel: (1 - lam)|psi><psi| + lam I / d."""
    d = psi.shape[0]
    return (1.0 - lam) * pure_density(psi) + (lam / d) * np.eye(d)


def white_noise(psi: np.ndarray, p: float) -> np.ndarray:
    """Sec. 4, eq. "white noise": p|psi><psi| + (1 - p) I / d."""
    d = psi.shape[0]
    return p * pure_density(psi) + ((1.0 - p) / d) * np.eye(d)


def product_plus(N: int) -> np.ndarray:
    """Sec. 4 product state ((|0> + |1>)/sqrt 2)^{(x)N}."""
    d = 1 << N
    return np.full(d, d ** -0.5, dtype=complex)


def ghzi(N: int) -> np.ndarray:
    """Sec. 4 GHZi state (|0...0> + i|1...1>)/sqrt 2."""
    d = 1 << N
    v = np.zeros(d, dtype=complex)
    v[0] = 2 ** -0.5
    v[d - 1] = 1j * 2 ** -0.5
    return v


def w_state(N: int) -> np.ndarray:
    """Sec. 4 W state: equal superposition of the N one-excitation basis states."""
    d = 1 << N
    v = np.zeros(d, dtype=complex)
    for q in range(N):
        v[1 << q] = N ** -0.5
    return v


def multinomial_counts(P: np.ndarray, shots: int, seed: int) -> np.ndarray:
    """Seeded multinomial outcome counts for the probability vector P (Sec. 4.5.1).

    P is taken as given (clipped at 0 and renormalised in FP64 so that the
    sampler accepts it); the counts are int64 and sum to ``shots``.
    """
    p = np.clip(np.asarray(P, dtype=np.float64), 0.0, None)
    p = p / p.sum()
    return _rng(seed).multinomial(int(shots), p).astype(np.int64)


def frequencies(counts: np.ndarray, dtype=np.float64) -> np.ndarray:
    """f_k = counts_k / shots, formed in the requested precision from the integer counts."""
    c = np.asarray(counts)
    shots = int(c.sum())
    return (c.astype(np.float64) / shots).astype(dtype)


def fnn_sizes(N: int) -> tuple[int, int]:
    """(n, H): input/output width 4^N and hidden width 2N of the Sec. 3.1 network."""
    return 4 ** N, 2 * N


def theta_size(N: int) -> int:
    """Number of network parameters: W1 (H x n), W2^T (H x n), b2 (n), b1 (H)."""
    n, H = fnn_sizes(N)
    return 2 * H * n + n + H


def theta_size_cnn(N: int) -> int:
    """Parameters of the CNN mapping network: W2^T (4N x n), b2, W1 (4N x 640), b1, conv (10 x 9), conv bias."""
    n, H = 4 ** N, 4 * N
    return H * n + n + H * 640 + H + 90 + 10


def init_theta_cnn(N: int, seed: int) -> np.ndarray:
    """Seeded initial CNN parameters (FP64, flat, the library's CNN layout
    [W2^T | b2 | W1 | b1 | conv W | conv b]); each layer uniform in +-1/sqrt(fan_in):
    the convolution has fan_in 9, the first dense layer 640, the output layer 4N."""
    n, H = 4 ** N, 4 * N
    r = _rng(seed)
    ac, a1, a2 = 1.0 / 3.0, 1.0 / np.sqrt(640.0), 1.0 / np.sqrt(H)
    cW = r.uniform(-ac, ac, size=90)
    cB = r.uniform(-ac, ac, size=10)
    W1 = r.uniform(-a1, a1, size=H * 640)
    b1 = r.uniform(-a1, a1, size=H)
    W2T = r.uniform(-a2, a2, size=H * n)
    b2 = r.uniform(-a2, a2, size=n)
    return np.concatenate([W2T, b2, W1, b1, cW, cB])


def init_theta(N: int, seed: int) -> np.ndarray:
    """Seeded initial network parameters in FP64, flat, in the library's theta layout.

    Each layer is drawn like a default fully-connected layer: weights and bias
    uniform in +-1/sqrt(fan_in).  Layer 1 has fan_in n, layer 2 fan_in H.
    Layout: [W1 (H x n, row-major) | W2^T (H x n, row-major) | b2 (n) | b1 (H)].
    """
    n, H = fnn_sizes(N)
    r = _rng(seed)
    a1 = 1.0 / np.sqrt(n)
    a2 = 1.0 / np.sqrt(H)
    W1 = r.uniform(-a1, a1, size=(H, n))
    b1 = r.uniform(-a1, a1, size=H)
    W2T = r.uniform(-a2, a2, size=(H, n))
    b2 = r.uniform(-a2, a2, size=n)
    return np.concatenate([W1.ravel(), W2T.ravel(), b2, b1])


def random_hermitian(d: int, seed: int) -> np.ndarray:
    """Random (not necessarily positive) Hermitian matrix with complex normal entries."""
    r = _rng(seed)
    a = r.standard_normal((d, d)) + 1j * r.standard_normal((d, d))
    return 0.5 * (a + a.conj().T)
