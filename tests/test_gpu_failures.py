"""Failure paths of the C ABI that can be reached without a GPU fault (host-side injection).

* QST_E_NOMEM from the context's device-memory budget (qst_options.device_memory_limit): qst_init
  refuses before cudaMalloc and frees what it had allocated.
* QST_E_INPUT for frequencies that are not a distribution (sum != 1, NaN, negative) in qst_loss_grad,
  qst_step and the batch step; a refused batch step advances none of its tomographies.
* QST_E_TIMEOUT from a bounded device-side wait that runs out: the tensor-core products or the bulk
  weight passes are told to issue none of their operand copies (qst_inject_wait_timeout), so the waits
  for those copies end at their limit (about 2 s) and the kernels return; the context is usable again.
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


def _f(N, seed=3):
    rho = synth.ginibre_mixed(N, 2, seed)
    return synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, 10**4, seed + 1))


def test_memory_budget_refuses_a_context_that_does_not_fit():
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    o = qst.qst_default_options()
    o.device_memory_limit = 1 << 20  # 1 MiB: N = 8 needs about 40 MiB
    with pytest.raises(qst.QstError) as e:
        qst.qst_init(8, opt=o)
    assert e.value.status == qst.QST_E_NOMEM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # nothing kept
    o.device_memory_limit = 1 << 30
    ctx = qst.qst_init(8, opt=o)  # a budget that fits
    qst.qst_destroy(ctx)


def test_memory_budget_applies_to_first_use_scratch():
    """Scratch allocated on first use counts against the budget too: a context that fits exactly
    refuses the sampler's scratch with QST_E_NOMEM and stays usable."""
    N = 6
    o = qst.qst_default_options()
    ctx = qst.qst_init(N, opt=o)
    qst.qst_destroy(ctx)
    # find the context's own footprint: the smallest budget that qst_init accepts, by bisection
    lo, hi = 1 << 16, 1 << 30
    while hi - lo > 4096:
        mid = (lo + hi) // 2
        o.device_memory_limit = mid
        try:
            c = qst.qst_init(N, opt=o)
            qst.qst_destroy(c)
            hi = mid
        except qst.QstError as err:
            assert err.status == qst.QST_E_NOMEM
            lo = mid
    o.device_memory_limit = hi
    ctx = qst.qst_init(N, opt=o)
    try:
        P = torch.full((4 ** N,), 1.0 / 4 ** N, dtype=torch.float64, device="cuda")
        counts = torch.empty(4 ** N, dtype=torch.int64, device="cuda")
        with pytest.raises(qst.QstError) as e:
            qst.qst_sample_counts(ctx, P, 1000, 1, counts)
        assert e.value.status == qst.QST_E_NOMEM
        qst.qst_set_params(ctx, synth.init_theta(N, 1).astype(np.float32))
        L, st = qst.qst_step(ctx, torch.from_numpy(_f(N).astype(np.float32)).cuda())
        assert st == qst.QST_OK and np.isfinite(L)
    finally:
        qst.qst_destroy(ctx)


def _bad_inputs(f):
    yield "sum 2", 2.0 * f
    g = f.copy(); g[5] = np.nan
    yield "nan", g
    g = f.copy(); g[1] = -g[1] - 1e-3; g /= g.sum()
    yield "negative", g


@pytest.mark.parametrize("prec", [qst.QST_FP32, qst.QST_FP64])
def test_loss_grad_and_step_refuse_bad_frequencies(prec):
    N = 4
    dt = np.float64 if prec == qst.QST_FP64 else np.float32
    o = qst.qst_default_options()
    o.precision = prec
    ctx = qst.qst_init(N, opt=o)
    try:
        theta = torch.from_numpy(synth.init_theta(N, 2).astype(dt)).cuda()
        qst.qst_set_params(ctx, theta)
        good = _f(N)
        for what, bad in _bad_inputs(good):
            g = torch.full_like(theta, 7.0)
            with pytest.raises(qst.QstError) as e:
                qst.qst_loss_grad(ctx, theta, torch.from_numpy(bad.astype(dt)).cuda(), g)
            assert e.value.status == qst.QST_E_INPUT, what
            assert bool((g == 7.0).all()), what  # nothing written
            with pytest.raises(qst.QstError) as e:
                qst.qst_step(ctx, torch.from_numpy(bad.astype(dt)).cuda())
            assert e.value.status == qst.QST_E_INPUT, what
        assert qst.qst_iterations(ctx) == 0
        L, st = qst.qst_step(ctx, torch.from_numpy(good.astype(dt)).cuda())
        assert st == qst.QST_OK and qst.qst_iterations(ctx) == 1
    finally:
        qst.qst_destroy(ctx)


def test_batch_step_refuses_bad_frequencies_before_any_step():
    Ns = [3, 4, 5]
    bt = qst.qst_batch_init(Ns)
    try:
        fs = []
        for b, N in enumerate(Ns):
            qst.qst_batch_set_params(bt, b, synth.init_theta(N, 10 + b).astype(np.float32))
            fs.append(torch.from_numpy(_f(N, 20 + b).astype(np.float32)).cuda())
        for what, bad in _bad_inputs(_f(Ns[2], 22)):
            inputs = fs[:2] + [torch.from_numpy(bad.astype(np.float32)).cuda()]
            with pytest.raises(qst.QstError) as e:
                qst.qst_batch_step(bt, inputs)
            assert e.value.status == qst.QST_E_INPUT, what
            for b in range(3):
                assert qst.qst_iterations(qst.qst_batch_context(bt, b)) == 0, (what, b)
        qst.qst_batch_step(bt, fs)
        for b in range(3):
            assert qst.qst_iterations(qst.qst_batch_context(bt, b)) == 1
    finally:
        qst.qst_batch_destroy(bt)


@pytest.mark.parametrize("what,N,prec", [(qst.QST_INJECT_TC_LOADS, 7, qst.QST_MIXED),
                                         (qst.QST_INJECT_WPASS_LOADS, 8, qst.QST_FP32)])
def test_wait_that_runs_out_is_reported_and_the_context_recovers(what, N, prec):
    f = torch.from_numpy(_f(N).astype(np.float32)).cuda()
    theta = torch.from_numpy(synth.init_theta(N, 5).astype(np.float32)).cuda()
    o = qst.qst_default_options()
    o.precision = prec
    ctx = qst.qst_init(N, opt=o)
    try:
        qst.qst_set_params(ctx, theta)
        want = [qst.qst_step(ctx, f)[0] for _ in range(2)]
        qst.qst_set_params(ctx, theta)
        qst.qst_inject_wait_timeout(what, 1)
        try:
            with pytest.raises(qst.QstError) as e:
                qst.qst_step(ctx, f)
            assert e.value.status == qst.QST_E_TIMEOUT
        finally:
            qst.qst_inject_wait_timeout(what, 0)
        # the context works again, bit for bit as before the timeout
        qst.qst_set_params(ctx, theta)
        got = [qst.qst_step(ctx, f)[0] for _ in range(2)]
        assert got == want
    finally:
        qst.qst_destroy(ctx)


def test_injection_hook_validates_its_arguments():
    for what, count in ((0, 1), (3, 1), (qst.QST_INJECT_TC_LOADS, -1)):
        with pytest.raises(qst.QstError) as e:
            qst.qst_inject_wait_timeout(what, count)
        assert e.value.status == qst.QST_E_INVAL
