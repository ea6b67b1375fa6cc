"""GPU synthetic data (Sec. 4): the sweep test states and the seeded multinomial counts.

The counts are integer arithmetic end to end, so they must equal the oracle's bit for bit.
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


def _ctx(N, prec=qst.QST_FP64):
    o = qst.qst_default_options()
    o.precision = prec
    return qst.qst_init(N, opt=o)


@pytest.mark.parametrize("N,shots,seed", [(1, 1000, 1), (2, 10**5, 2), (5, 10**5, 3), (8, 3 * 10**5, 4)])
def test_counts_bit_exact_with_oracle(N, shots, seed):
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 2), 5000 + N)
    P = np.ascontiguousarray(O.born_probabilities(rho, M).real)
    P[::7] = 0.0  # outcomes of zero probability must never be drawn
    ctx = _ctx(N)
    try:
        Pd = torch.from_numpy(P).cuda()
        counts = torch.empty(4 ** N, dtype=torch.int64, device="cuda")
        f = torch.empty(4 ** N, dtype=torch.float64, device="cuda")
        qst.qst_sample_counts(ctx, Pd, shots, seed, counts, f)
        got = counts.cpu().numpy()
        fg = f.cpu().numpy()
        qst.qst_sample_counts(ctx, Pd, shots, seed, counts)
        again = counts.cpu().numpy()
    finally:
        qst.qst_destroy(ctx)
    want = O.multinomial_counts_integer(P, shots, seed)
    assert np.array_equal(got, want)
    assert np.array_equal(again, want)
    np.testing.assert_array_equal(fg, want / shots)


def test_counts_reject_bad_probabilities():
    ctx = _ctx(2)
    try:
        counts = torch.empty(16, dtype=torch.int64, device="cuda")
        for bad in (np.full(16, 2.0), np.zeros(16), np.r_[np.nan, np.ones(15) / 15]):
            with pytest.raises(qst.QstError) as e:
                qst.qst_sample_counts(ctx, torch.from_numpy(bad).cuda(), 100, 1, counts)
            assert e.value.status == qst.QST_E_INPUT
    finally:
        qst.qst_destroy(ctx)


@pytest.mark.parametrize("prec", [qst.QST_FP64, qst.QST_FP32])
@pytest.mark.parametrize("kind,make", [(qst.QST_STATE_PRODUCT, synth.product_plus), (qst.QST_STATE_GHZI, synth.ghzi),
                                       (qst.QST_STATE_W, synth.w_state)])
def test_test_states_match_generators(prec, kind, make):
    N = 6
    ctx = _ctx(N, prec)
    try:
        for w in (1.0, 0.7, 0.0):
            dt = torch.complex128 if prec == qst.QST_FP64 else torch.complex64
            rho = torch.empty((64, 64), dtype=dt, device="cuda")
            qst.qst_test_state(ctx, kind, w, rho)
            want = synth.white_noise(make(N), w)  # w |psi><psi| + (1 - w) I / d
            tol = 1e-15 if prec == qst.QST_FP64 else 1e-7
            np.testing.assert_allclose(rho.cpu().numpy(), want, atol=tol)
    finally:
        qst.qst_destroy(ctx)


def test_depolarized_ghzi_sweep_end_to_end_on_device():
    """State -> probabilities -> counts -> frequencies, all on the GPU, equal to the host pipeline
    run with the same generator definitions (the oracle's sampler)."""
    N, lam, shots, seed = 8, 0.2, 10**5, 9
    ctx = _ctx(N)
    try:
        rho = torch.empty((256, 256), dtype=torch.complex128, device="cuda")
        qst.qst_test_state(ctx, qst.QST_STATE_GHZI, 1.0 - lam, rho)
        P = torch.empty(4 ** N, dtype=torch.float64, device="cuda")
        qst.qst_probs(ctx, rho, P)
        counts = torch.empty(4 ** N, dtype=torch.int64, device="cuda")
        qst.qst_sample_counts(ctx, P, shots, seed, counts)
        got = counts.cpu().numpy()
        Pg = P.cpu().numpy()
    finally:
        qst.qst_destroy(ctx)
    P_host = O.born_probabilities(synth.depolarized(synth.ghzi(N), lam), M).real
    np.testing.assert_allclose(Pg, P_host, atol=1e-15)
    assert np.array_equal(got, O.multinomial_counts_integer(Pg, shots, seed))
    assert got.sum() == shots
