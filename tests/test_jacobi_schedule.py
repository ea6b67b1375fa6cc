"""Host-side checks of the Jacobi eigensolver's ordering (Sec. 3.2, eq. abs_P needs T = Q Lambda Q^dag every
iteration).  No GPU: qst_jacobi_schedule is host-only.

A sweep is the d - 1 rounds m = 1 .. d - 1 of the XOR ordering (round m rotates the pairs {x, x ^ m}); a
pass applies the three rounds {a, b, a ^ b} of one 2-dimensional subspace of GF(2)^N, or a single round.
Checked here: every round appears exactly once per sweep, the passes are in the reduced form the kernel's
coset numbering assumes, the cosets that numbering gives (pivot bits inserted as zeros) partition
0 .. d - 1 within bounds, and a NumPy run of the pass algorithm (each coset's 4 x 4 unitary built from the
rounds in order, then U^dag A U on every block) diagonalises a random Hermitian matrix to the eigenvalues
numpy.linalg.eigvalsh gives.
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


def _cosets(N, a, b):
    """The kernel's numbering: coset c of the pass -> its G elements (local index bit 0: a, bit 1: b)."""
    d = 1 << N
    if b == 0:
        c = np.arange(d // 2)
        x = _insert_zero(c, _top(a))
        return np.stack([x, x ^ a], 1)
    c = np.arange(d // 4)
    x = _insert_zero(_insert_zero(c, _top(b)), _top(a))
    return np.stack([x, x ^ a, x ^ b, x ^ a ^ b], 1)


@pytest.mark.parametrize("N", list(range(1, 13)))
def test_every_round_once_per_sweep(N):
    d = 1 << N
    sched = qst.qst_jacobi_schedule(N)
    assert len(sched) % 2 == 1  # an even number of sweeps returns the ping-pong buffers to the first pair
    seen = np.zeros(d, dtype=int)
    for a, b in sched:
        assert 0 < a < d and 0 <= b < d
        if b == 0:
            seen[a] += 1
            continue
        assert _top(b) < _top(a) and not (a >> _top(b)) & 1, (a, b)
        for m in (a, b, a ^ b):
            seen[m] += 1
    assert seen[0] == 0 and np.all(seen[1:] == 1)
    lines = sum(1 for _, b in sched if b)
    # even N: a partition into lines; odd N >= 3: (d - 8) / 3 lines, and a plane as one line and 4 rounds
    assert lines == ((d - 1) // 3 if N % 2 == 0 else ((d - 8) // 3 + 1 if N > 1 else 0))


def test_passes_per_sweep():
    assert [len(qst.qst_jacobi_schedule(N)) for N in (1, 2, 3, 10, 11, 12)] == [1, 1, 5, 341, 685, 1365]
    with pytest.raises(qst.QstError):
        qst.qst_jacobi_schedule(0)
    with pytest.raises(qst.QstError):
        qst.qst_jacobi_schedule(13)


@pytest.mark.parametrize("N", list(range(1, 13)))
def test_coset_numbering_partitions_the_indices(N):
    d = 1 << N
    for a, b in qst.qst_jacobi_schedule(N):
        e = _cosets(N, a, b)
        assert e.min() >= 0 and e.max() < d
        assert np.array_equal(np.sort(e.ravel()), np.arange(d)), (a, b)
        # the local pairs of each round are the round's pairs {x, x ^ m}
        if b:
            assert np.all(e[:, 1] ^ e[:, 0] == a) and np.all(e[:, 2] ^ e[:, 0] == b)
            assert np.all(e[:, 3] ^ e[:, 0] == a ^ b)


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


@pytest.mark.parametrize("N", [3, 4, 5])
def test_pass_algorithm_diagonalises(N):
    d = 1 << N
    rng = np.random.default_rng(N)
    Z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    T = (Z + Z.conj().T) / 2
    A, V = T.copy(), np.eye(d, dtype=complex)
    sched = qst.qst_jacobi_schedule(N)
    for _ in range(10):
        for a, b in sched:
            e = _cosets(N, a, b)
            U = np.zeros((d, d), dtype=complex)
            for row in e:
                U[np.ix_(row, row)] = _coset_unitary(A[np.ix_(row, row)])
            A = U.conj().T @ A @ U
            V = V @ U
    off = np.linalg.norm(A - np.diag(np.diag(A))) / np.linalg.norm(T)
    assert off < 1e-13, off
    np.testing.assert_allclose(np.sort(np.diag(A).real), np.linalg.eigvalsh(T), rtol=0, atol=1e-12)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(d), rtol=0, atol=1e-12)
    np.testing.assert_allclose(V @ np.diag(np.diag(A)) @ V.conj().T, T, rtol=0, atol=1e-11)
