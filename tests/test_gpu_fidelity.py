"""GPU classical fidelity (Sec. 2.3 eq. F_CF and the sampled eq. fc_sample) against the oracle.

Exact F_c: FP64 within 1e-10, FP32 within 1e-5 relative.  Sampled: FP64 uses the oracle's sampler on
the oracle's P^ with the same SplitMix64 draws and must agree to rounding (a draw moves to another
outcome only if u_s c_{n-1} falls within rounding of a running-sum boundary); FP32 probabilities
differ from the oracle's at the 1e-7 level, so there the estimate is compared with the exact value
within its sampling error.
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


def _setup(N, prec, mapping, seed):
    rho_t = synth.ginibre_mixed(N, max(1, (1 << N) // 4), 4000 + seed)
    P = O.born_probabilities(rho_t, M).real
    f = synth.frequencies(synth.multinomial_counts(P, 10**5, 4100 + seed))
    theta = synth.init_theta(N, 4200 + seed)
    dt = np.float64 if prec == qst.QST_FP64 else np.float32
    o = qst.qst_default_options()
    o.precision = prec
    o.mapping = mapping
    ctx = qst.qst_init(N, opt=o)
    qst.qst_set_params(ctx, theta.astype(dt))
    th64 = theta.astype(dt).astype(np.float64)
    f64 = f.astype(dt).astype(np.float64)
    P_hat = O.born_probabilities(O.state_from_theta(th64, f64, N, mapping=_oracle_map(mapping)), M).real
    return ctx, torch.from_numpy(f.astype(dt)).cuda(), torch.from_numpy(P.astype(dt)).cuda(), P_hat, P


def _oracle_map(m):
    return {qst.QST_MAP_CHOL_H: "chol_h", qst.QST_MAP_CHOL_DELTA: "chol_delta", qst.QST_MAP_ABS_P: "abs_p"}[m]


@pytest.mark.parametrize("prec,N,mapping", [(qst.QST_FP64, 2, qst.QST_MAP_CHOL_H), (qst.QST_FP64, 5, qst.QST_MAP_CHOL_H),
                                            (qst.QST_FP64, 4, qst.QST_MAP_CHOL_DELTA), (qst.QST_FP32, 3, qst.QST_MAP_CHOL_H),
                                            (qst.QST_FP32, 7, qst.QST_MAP_CHOL_H), (qst.QST_MIXED, 8, qst.QST_MAP_CHOL_H)])
def test_exact_classical_fidelity(prec, N, mapping):
    ctx, f, P, P_hat, P64 = _setup(N, prec, mapping, N)
    try:
        got = qst.qst_classical_fidelity(ctx, f, P)
        got2 = qst.qst_classical_fidelity(ctx, f, P)
    finally:
        qst.qst_destroy(ctx)
    want = O.classical_fidelity(P_hat, P.cpu().numpy().astype(np.float64))
    tol = 1e-10 if prec == qst.QST_FP64 else 1e-5
    assert abs(got - want) <= tol * want, (got, want)
    assert got == got2  # fixed-order reductions repeat exactly
    assert 0.0 < got <= 1.0 + 1e-6


@pytest.mark.parametrize("N,samples,seed", [(2, 1000, 1), (4, 20000, 2), (6, 50000, 3)])
def test_sampled_classical_fidelity_fp64_matches_oracle_draws(N, samples, seed):
    ctx, f, P, P_hat, _ = _setup(N, qst.QST_FP64, qst.QST_MAP_CHOL_H, 10 + N)
    try:
        got = qst.qst_classical_fidelity(ctx, f, P, samples=samples, seed=seed)
    finally:
        qst.qst_destroy(ctx)
    want = O.sampled_classical_fidelity(P_hat, P.cpu().numpy(), samples, seed)
    assert abs(got - want) <= 1e-9 * want, (got, want)


def test_sampled_classical_fidelity_fp32_within_sampling_error():
    N, S = 8, 200_000
    ctx, f, P, P_hat, _ = _setup(N, qst.QST_FP32, qst.QST_MAP_CHOL_H, 30)
    try:
        exact = qst.qst_classical_fidelity(ctx, f, P)
        est = qst.qst_classical_fidelity(ctx, f, P, samples=S, seed=77)
        est2 = qst.qst_classical_fidelity(ctx, f, P, samples=S, seed=77)
    finally:
        qst.qst_destroy(ctx)
    Pn = P.cpu().numpy().astype(np.float64)
    r = np.sqrt(np.clip(Pn, 0, None) / np.clip(P_hat, 1e-300, None))
    se = 2 * np.sqrt(exact) * np.sqrt(max(np.sum(P_hat * r ** 2) - exact, 0.0)) / np.sqrt(S)
    assert abs(est - exact) < 6 * se + 1e-6, (est, exact, se)
    assert est == est2


def test_classical_fidelity_of_the_target_itself_is_one():
    """With the state's own distribution as target, eq. F_CF is 1 and every sampled ratio is 1."""
    N = 5
    ctx, f, _, P_hat, _ = _setup(N, qst.QST_FP64, qst.QST_MAP_CHOL_H, 50)
    try:
        Pself = torch.from_numpy(np.ascontiguousarray(P_hat)).cuda()
        assert abs(qst.qst_classical_fidelity(ctx, f, Pself) - 1.0) < 1e-12
        assert abs(qst.qst_classical_fidelity(ctx, f, Pself, samples=5000, seed=9) - 1.0) < 1e-12
    finally:
        qst.qst_destroy(ctx)
