"""Host-side checks of the Jacobi eigensolver's ordering (Sec. 3.2, eq. abs_P needs T = Q Lambda Q^dag every
iteration).  No GPU: qst_jacobi_schedule is host-only.

A sweep is the d - 1 rounds m = 1 .. d - 1 of the XOR ordering (round m rotates the pairs {x, x ^ m}); a
pass applies the 2^k - 1 rounds of one k-dimensional subspace of GF(2)^N (k = 1, 2 for N <= 5; 3, 4 for
N >= 6).  Checked here: every round appears exactly once per sweep, the passes are in the reduced form the
kernels' coset numbering assumes, the cosets that numbering gives (pivot bits inserted as zeros) partition
0 .. d - 1 within bounds, and a NumPy run of the pass algorithm (each coset's unitary built from the
subspace's rounds in order, then U^dag A U on every block) diagonalises a random Hermitian matrix to the
eigenvalues numpy.linalg.eigvalsh gives.
"""
import os

import numpy as np
import pytest

from paper_2207_05341_gb300 import qst


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(qst.LIB_PATH):
        from paper_2207_05341_gb300 import build
        build.build()
    qst.load()


def _top(x):
    return int(x).bit_length() - 1


def _insert_zero(x, p):
    return ((x >> p) << (p + 1)) | (x & ((1 << p) - 1))


def _span(basis):
    out = [0]
    for v in basis:
        out = out + [x ^ v for x in out]
    return out  # local index j -> XOR of basis[i] over the bits i of j


def _cosets(N, basis):
    """The kernels' numbering: coset c -> its 2^k elements (pivot bits of the representative clear)."""
    d = 1 << N
    piv = sorted(_top(v) for v in basis)
    x = np.arange(d >> len(basis))
    for p in piv:
        x = _insert_zero(x, p)
    return np.stack([x ^ s for s in _span(basis)], 1)


PASSES = {1: 1, 2: 1, 3: 5, 4: 5, 5: 13, 6: 9, 7: 17, 8: 17, 9: 73, 10: 145, 11: 273, 12: 273}


@pytest.mark.parametrize("N", list(range(1, 13)))
def test_every_round_once_per_sweep(N):
    d = 1 << N
    sched = qst.qst_jacobi_schedule(N)
    assert len(sched) == PASSES[N]
    assert len(sched) % 2 == 1  # an even number of sweeps returns the ping-pong buffers to the first pair
    seen = np.zeros(d, dtype=int)
    for basis in sched:
        k = len(basis)
        assert (1 <= k <= 2) if N <= 5 else (3 <= k <= 4), basis
        tops = [_top(v) for v in basis]
        assert tops == sorted(set(tops)), basis  # reduced form: distinct pivots, ascending
        for i, v in enumerate(basis):
            assert 0 < v < d
            assert all(not (v >> t) & 1 for jj, t in enumerate(tops) if jj != i), basis
        for m in _span(basis)[1:]:
            seen[m] += 1
    assert seen[0] == 0 and np.all(seen[1:] == 1)


def test_schedule_arguments():
    with pytest.raises(qst.QstError):
        qst.qst_jacobi_schedule(0)
    with pytest.raises(qst.QstError):
        qst.qst_jacobi_schedule(13)


@pytest.mark.parametrize("N", list(range(1, 13)))
def test_coset_numbering_partitions_the_indices(N):
    d = 1 << N
    for basis in qst.qst_jacobi_schedule(N):
        e = _cosets(N, basis)
        assert e.min() >= 0 and e.max() < d
        assert np.array_equal(np.sort(e.ravel()), np.arange(d)), basis
        # local index j of every coset differs from its representative by the subspace element j
        assert np.all((e ^ e[:, :1]) == np.array(_span(basis))[None, :])


def _rotation(a, b, c):
    r = abs(c)
    if r <= 1e-300:
        return 1.0, 0.0, 1.0 + 0j
    tau = (b - a) / (2 * r)
    t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + np.sqrt(1 + tau * tau))
    cs = 1 / np.sqrt(1 + t * t)
    return cs, t * cs, np.conj(c / r)


def _coset_unitary(B):
    G = B.shape[0]
    B = B.copy()
    U = np.eye(G, dtype=complex)
    for s in range(1, G):
        for p in range(G):
            q = p ^ s
            if q < p:
                continue
            cs, sn, emph = _rotation(B[p, p].real, B[q, q].real, B[p, q])
            R = np.eye(G, dtype=complex)
            R[p, p], R[p, q], R[q, p], R[q, q] = cs, sn, -emph * sn, emph * cs
            B = R.conj().T @ B @ R
            U = U @ R
    return U


@pytest.mark.parametrize("N", [3, 4, 5, 6, 7])
def test_pass_algorithm_diagonalises(N):
    d = 1 << N
    rng = np.random.default_rng(N)
    Z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    T = (Z + Z.conj().T) / 2
    A, V = T.copy(), np.eye(d, dtype=complex)
    sched = qst.qst_jacobi_schedule(N)
    for _ in range(10):
        for basis in sched:
            U = np.zeros((d, d), dtype=complex)
            for row in _cosets(N, basis):
                U[np.ix_(row, row)] = _coset_unitary(A[np.ix_(row, row)])
            A = U.conj().T @ A @ U
            V = V @ U
    off = np.linalg.norm(A - np.diag(np.diag(A))) / np.linalg.norm(T)
    assert off < 1e-13, off
    np.testing.assert_allclose(np.sort(np.diag(A).real), np.linalg.eigvalsh(T), rtol=0, atol=1e-12)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(d), rtol=0, atol=1e-12)
    np.testing.assert_allclose(V @ np.diag(np.diag(A)) @ V.conj().T, T, rtol=0, atol=1e-11)
