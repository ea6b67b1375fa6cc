"""Pins of the oracle's measurement model (Sec. 2.1, Sec. 3.3 eq. PS, Sec. 4.1) against the mathematics.

These tests check the oracle against things other than itself: the paper's
printed POVM vectors, explicit Kronecker products (brute force), the closed
single-qubit Born probabilities, the 2-qubit block formula and invariants.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_2207_05341_gb300 import synth


def _golden(golden_dir):
    vals = {}
    with open(os.path.join(golden_dir, "paper_constants.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = (s.strip() for s in line.split("="))
                vals[k] = [float(x) for x in v.split()]
    return vals


def _pauli():
    return (np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
            np.array([[1, 0], [0, -1]], complex))


def test_povm_matches_printed_vectors(golden_dir):
    g = _golden(golden_dir)
    M = O.tetrahedral_povm()
    assert M.shape == (int(g["K"][0]), 2, 2)
    sx, sy, sz = _pauli()
    for a in range(4):
        s = np.array(g[f"s{a}"]) / np.sqrt(3.0)
        # recover the Bloch vector of 4 M_a - I from Pauli traces
        rec = np.array([np.trace(4 * M[a] @ P).real / 2 for P in (sx, sy, sz)])
        np.testing.assert_allclose(rec, s, atol=1e-15)
        np.testing.assert_allclose(np.trace(M[a]).real, 0.5, atol=1e-15)


def test_povm_is_informationally_complete_sic():
    M = O.tetrahedral_povm()
    np.testing.assert_allclose(M.sum(0), np.eye(2), atol=1e-15)
    for a in range(4):
        w = np.linalg.eigvalsh(M[a])
        np.testing.assert_allclose(w, [0.0, 0.5], atol=1e-15)
        for b in range(4):
            # Tr(M_a M_b) = (1 + s_a.s_b)/8: 1/4 on the diagonal, 1/12 off it (tetrahedron)
            want = 0.25 if a == b else 1.0 / 12.0
            assert abs(np.trace(M[a] @ M[b]).real - want) < 1e-15
    # informational completeness: the 4 elements span all 2x2 Hermitian matrices
    assert np.linalg.matrix_rank(M.reshape(4, 4)) == 4


def test_single_qubit_closed_form():
    """For rho = (I + r.sigma)/2 the tetrahedral POVM gives p_a = (1 + s_a.r)/4."""
    sx, sy, sz = _pauli()
    s = np.array([[1, 1, 1], [-1, -1, 1], [-1, 1, -1], [1, -1, -1]]) / np.sqrt(3)
    rng = np.random.default_rng(5)
    for _ in range(5):
        r = rng.standard_normal(3)
        r *= rng.uniform(0, 1) / np.linalg.norm(r)
        rho = (np.eye(2) + r[0] * sx + r[1] * sy + r[2] * sz) / 2
        p = O.born_probabilities(rho, O.tetrahedral_povm())
        np.testing.assert_allclose(p.real, (1 + s @ r) / 4, atol=1e-15)
        assert np.abs(p.imag).max() < 1e-16


def _kron_probs(rho, M):
    N = rho.shape[0].bit_length() - 1
    out = []
    for ks in itertools.product(range(M.shape[0]), repeat=N):
        op = np.array([[1.0 + 0j]])
        for k in ks:
            op = np.kron(op, M[k])
        out.append(np.trace(op @ rho))
    return np.array(out)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_born_map_matches_explicit_kron(N):
    """Brute force: explicit Kronecker products, on non-Hermitian complex matrices too."""
    M = O.tetrahedral_povm()
    rng = np.random.default_rng(100 + N)
    d = 1 << N
    A = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    np.testing.assert_allclose(O.born_probabilities(A, M), _kron_probs(A, M), atol=1e-12)
    H = synth.random_hermitian(d, 7 + N)
    np.testing.assert_allclose(O.born_probabilities(H, M), _kron_probs(H, M), atol=1e-12)


def test_two_qubit_block_formula():
    """Sec. 3.3 eq. PS: P_(i,j) from the four blocks A, B, C, D of rho.

    Born rule: Tr[(M_i x M_j)(E_kl x Blk)] = (M_i)_lk Tr[M_j Blk], so the block B
    (upper right, E_12) pairs with c_i = (M_i)_21 and C with b_i.
    """
    M = O.tetrahedral_povm()
    rho = synth.ginibre_mixed(2, 3, 11)
    A, B, C, D = rho[:2, :2], rho[:2, 2:], rho[2:, :2], rho[2:, 2:]
    p = O.born_probabilities(rho, M).real
    for i in range(4):
        a, b, c, dd = M[i][0, 0], M[i][0, 1], M[i][1, 0], M[i][1, 1]
        for j in range(4):
            want = (a * np.trace(M[j] @ A) + c * np.trace(M[j] @ B)
                    + b * np.trace(M[j] @ C) + dd * np.trace(M[j] @ D))
            assert abs(p[4 * i + j] - want.real) < 1e-15
    # the printed coefficient order (b with B) differs for this POVM, whose off-diagonals are complex
    i = 0
    a, b, c, dd = M[i][0, 0], M[i][0, 1], M[i][1, 0], M[i][1, 1]
    printed = (a * np.trace(M[0] @ A) + b * np.trace(M[0] @ B) + c * np.trace(M[0] @ C)
               + dd * np.trace(M[0] @ D))
    assert abs(printed - p[0]) > 1e-6


@pytest.mark.parametrize("N", [1, 3, 5])
def test_probabilities_sum_to_trace_and_are_nonnegative(N):
    M = O.tetrahedral_povm()
    for rank in (1, 2):
        rho = synth.ginibre_mixed(N, min(rank, 1 << N), 20 + N + rank)
        p = O.born_probabilities(rho, M)
        assert abs(p.real.sum() - 1.0) < 1e-12
        assert p.real.min() > -1e-15
        assert np.abs(p.imag).max() < 1e-14
    H = synth.random_hermitian(1 << N, 3)
    assert abs(O.born_probabilities(H, M).real.sum() - np.trace(H).real) < 1e-10


def test_maximally_mixed_and_product_states():
    M = O.tetrahedral_povm()
    N = 4
    d = 1 << N
    p = O.born_probabilities(np.eye(d) / d, M).real
    np.testing.assert_allclose(p, np.full(4 ** N, 4.0 ** -N), atol=1e-15)
    # a product state gives a product distribution
    rng = np.random.default_rng(3)
    singles, rho = [], np.array([[1.0 + 0j]])
    for q in range(N):
        r = synth.ginibre_mixed(1, 1 + q % 2, 40 + q)
        singles.append(O.born_probabilities(r, M).real)
        rho = np.kron(rho, r)
    want = singles[0]
    for s in singles[1:]:
        want = np.kron(want, s)
    np.testing.assert_allclose(O.born_probabilities(rho, M).real, want, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_adjoint_bruteforce_and_identity(N):
    M = O.tetrahedral_povm()
    rng = np.random.default_rng(N)
    g = rng.standard_normal(4 ** N)
    G = O.povm_adjoint(g, M)
    want = np.zeros((1 << N, 1 << N), complex)
    for k, ks in enumerate(itertools.product(range(4), repeat=N)):
        op = np.array([[1.0 + 0j]])
        for a in ks:
            op = np.kron(op, M[a])
        want += g[k] * op
    np.testing.assert_allclose(G, want, atol=1e-13)
    X = synth.random_hermitian(1 << N, 9)
    lhs = np.dot(g, O.born_probabilities(X, M).real)
    rhs = np.real(np.trace(G @ X))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_single_outcome_helper_matches_full_map():
    M = O.tetrahedral_povm()
    rho = synth.ginibre_mixed(4, 5, 77)
    p = O.born_probabilities(rho, M)
    for k in (0, 1, 17, 100, 255):
        assert abs(O.born_probability_at(rho, M, k) - p[k]) < 1e-15
