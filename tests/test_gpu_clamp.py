"""GPU parity of the likelihood's clamp (QST_W_CLAMP) against the oracle.

The POVM {|0><0|, |1><1|, |+><+|, |-><-|} / 2 (a valid POVM: it sums to I) and parameters whose
output is t = (2, 0, ..., 0) give T = 2 |0...0><0...0|, X = 4 |0...0><0...0|: every outcome with a
|1><1| factor has q_k = 0 exactly (all the arithmetic is on dyadic numbers, in every precision),
and with uniform f those terms are clamped.  Reading of the likelihood: a clamped term adds the
constant -f_k log q_min (q_min the smallest normal number of the precision) to L and nothing to
dL/dq_k, and the call returns QST_W_CLAMP.  N = 1 runs the generic high-qubit pass, N = 7 the
Pauli-basis one; the mixed path's tensor-core products see the same exact operands.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_05341_gb300 import qst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    if not os.path.exists(qst.LIB_PATH):
        from paper_2207_05341_gb300 import build
        build.build()
    qst.load()


def _povm():
    kets = [np.array([1, 0]), np.array([0, 1]), np.array([1, 1]) / np.sqrt(2), np.array([1, -1]) / np.sqrt(2)]
    M = np.stack([np.outer(k, k.conj()).astype(complex) / 2 for k in kets])
    flat = np.empty((4, 2, 2, 2))
    flat[..., 0] = M.real
    flat[..., 1] = M.imag
    return M, np.ascontiguousarray(flat.reshape(-1))


def _inputs(N):
    n, H = 4 ** N, 2 * N
    theta = np.zeros(synth.theta_size(N))
    theta[2 * H * n] = 2.0  # b2[0]: t = (2, 0, ..., 0)
    f = np.full(n, 1.0 / n)
    return theta, f


CASES = [(qst.QST_FP64, 1), (qst.QST_FP32, 1), (qst.QST_FP64, 7), (qst.QST_FP32, 7), (qst.QST_MIXED, 7)]


@pytest.mark.parametrize("prec,N", CASES)
def test_clamped_likelihood_matches_oracle(prec, N):
    M, flat = _povm()
    theta, f = _inputs(N)
    fp64 = prec == qst.QST_FP64
    qmin = O.Q_MIN_FP64 if fp64 else O.Q_MIN_FP32
    L_ref, g_ref, aux = O.loss_and_grad(theta, f, M, N, q_min=qmin)
    assert aux["clamped"] == 4 ** N - 3 ** N
    dt = torch.float64 if fp64 else torch.float32
    opt = qst.qst_default_options()
    opt.precision = prec
    ctx = qst.qst_init(N, povm=flat, opt=opt)
    try:
        th = torch.tensor(theta, dtype=dt, device="cuda")
        fd = torch.tensor(f, dtype=dt, device="cuda")
        g = torch.empty_like(th)
        L, st = qst.qst_loss_grad(ctx, th, fd, g)
        assert st == qst.QST_W_CLAMP
        g = g.cpu().numpy().astype(np.float64)
        tol = 1e-10 if fp64 else 1e-4
        assert abs(L - L_ref) <= tol * abs(L_ref), (L, L_ref)
        assert np.abs(g - g_ref).max() <= tol * np.abs(g_ref).max(), np.abs(g - g_ref).max()
        assert np.linalg.norm(g - g_ref) <= tol * np.linalg.norm(g_ref)
        # the training step reports the same warning, and the next call without a clamp clears it
        qst.qst_set_params(ctx, th)
        L1, st1 = qst.qst_step(ctx, fd)
        assert st1 == qst.QST_W_CLAMP
        assert abs(L1 - L_ref) <= tol * abs(L_ref)
    finally:
        qst.qst_destroy(ctx)


def test_no_clamp_without_zero_probabilities():
    """The same POVM on a full-rank state: no term is clamped and the status is QST_OK."""
    M, flat = _povm()
    N = 3
    rho = synth.ginibre_mixed(N, 8, 4)
    f = synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, 10**5, 5))
    theta = synth.init_theta(N, 6)
    L_ref, g_ref, aux = O.loss_and_grad(theta.astype(np.float32).astype(np.float64),
                                        f.astype(np.float32).astype(np.float64), M, N, q_min=O.Q_MIN_FP32)
    assert aux["clamped"] == 0
    ctx = qst.qst_init(N, povm=flat)
    try:
        th = torch.tensor(theta, dtype=torch.float32, device="cuda")
        g = torch.empty_like(th)
        L, st = qst.qst_loss_grad(ctx, th, torch.tensor(f, dtype=torch.float32, device="cuda"), g)
        assert st == qst.QST_OK
        assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
        g = g.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    finally:
        qst.qst_destroy(ctx)
