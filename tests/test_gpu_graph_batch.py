"""CUDA-graph replay of qst_step and batches of tomographies: both must reproduce the
launch-by-launch path bit for bit (all reductions in the library have a fixed order)."""
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


def _inputs(N, seed):
    M = O.tetrahedral_povm()
    rho = synth.ginibre_mixed(N, max(1, (1 << N) // 3), 40 + seed)
    f = synth.frequencies(synth.multinomial_counts(O.born_probabilities(rho, M).real, 10**5 * N, 50 + seed))
    return f.astype(np.float32), synth.init_theta(N, 60 + seed).astype(np.float32)


def _run(N, f, theta, steps, prec, graph, timing=False, extra=None, host=False, network=qst.QST_NET_FNN,
         fused_max=0):
    stream = torch.cuda.Stream()
    o = qst.qst_default_options()
    o.precision = prec
    o.network = network
    o.fused_max_qubits = fused_max
    ctx = qst.qst_init(N, opt=o, stream=stream.cuda_stream)
    try:
        if graph:
            qst.qst_graph_enable(ctx, True)
        if timing:
            qst.qst_timing_enable(ctx, steps)
        qst.qst_set_params(ctx, theta)
        fd = torch.from_numpy(f).pin_memory() if host else torch.from_numpy(f).cuda()
        torch.cuda.synchronize()
        losses = [qst.qst_step(ctx, fd)[0] for _ in range(steps)]
        out = torch.empty(theta.size, device="cuda")
        qst.qst_get_params(ctx, out)
        qst.qst_sync(ctx)
        if extra is not None:
            extra["launches"] = qst.qst_kernel_launches(ctx)
            if timing:
                extra["timing"] = qst.qst_timing_read(ctx)
        return losses, out.cpu().numpy(), qst.qst_iterations(ctx)
    finally:
        qst.qst_destroy(ctx)


@pytest.mark.parametrize("N,prec", [(5, qst.QST_FP32), (8, qst.QST_MIXED)])
def test_graph_replay_is_bit_identical(N, prec):
    f, theta = _inputs(N, N)
    la, ta, ia = _run(N, f, theta, 6, prec, graph=False)
    lb, tb, ib = _run(N, f, theta, 6, prec, graph=True)
    assert la == lb and ia == ib == 6
    assert np.array_equal(ta, tb)


@pytest.mark.parametrize("prec,fused_max", [(qst.QST_FP32, -1), (qst.QST_FP32, 7), (qst.QST_MIXED, 0)])
def test_timed_graph_replay(prec, fused_max):
    """Phase events captured as graph nodes: same results and launch count as the
    launch-by-launch path, and every phase of the latest replay is timed once (an FP32
    N = 7 iteration is one fused kernel by default, timed as one phase)."""
    N = 7
    f, theta = _inputs(N, 3)
    xa, xb = {}, {}
    la, ta, _ = _run(N, f, theta, 5, prec, graph=False, timing=True, extra=xa, fused_max=fused_max)
    lb, tb, _ = _run(N, f, theta, 5, prec, graph=True, timing=True, extra=xb, fused_max=fused_max)
    assert la == lb and np.array_equal(ta, tb)
    assert xa["launches"] == xb["launches"] > 0
    tm = xb["timing"]
    timed = [p for p in qst.PHASES if tm[p][1] > 0]
    assert "hidden" not in timed  # a replay does not recompute the f-dependent activation
    fused = prec == qst.QST_FP32 and fused_max == 7
    last = "fused" if fused else "w2"
    if fused:
        assert timed == ["fused"]
    else:
        assert {"build_T", "povm_lo", "povm_hi", "w2", "w1"} <= set(timed)
    assert all(tm[p][1] == 1 and tm[p][0] > 0 for p in timed)
    # the launch-by-launch path recorded all five steps
    assert xa["timing"][last][1] == 5 and xa["timing"]["hidden"][1] == 1


@pytest.mark.parametrize("N,prec,network", [(6, qst.QST_FP32, qst.QST_NET_FNN), (8, qst.QST_MIXED, qst.QST_NET_FNN),
                                            (6, qst.QST_FP32, qst.QST_NET_CNN)])
def test_graph_replay_with_page_locked_host_f(N, prec, network):
    """A captured step copies a page-locked host f on a side stream beside its first kernels (the FNN
    reads f first in the likelihood, the CNN at once): same losses and parameters as device f."""
    f, theta = _inputs(N, 20 + N)
    if network == qst.QST_NET_CNN:
        theta = synth.init_theta_cnn(N, 70 + N).astype(np.float32)
    la, ta, _ = _run(N, f, theta, 6, prec, graph=False, network=network)
    lb, tb, ib = _run(N, f, theta, 6, prec, graph=True, host=True, network=network)
    xc = {}
    lc, tc, _ = _run(N, f, theta, 6, prec, graph=True, host=True, timing=True, extra=xc, network=network)
    assert la == lb == lc and ib == 6
    assert np.array_equal(ta, tb) and np.array_equal(ta, tc)
    fused = prec == qst.QST_FP32 and network == qst.QST_NET_FNN  # N = 6: one fused kernel per iteration
    assert xc["timing"]["fused" if fused else "w2"][1] == 1


def test_graph_needs_a_stream():
    ctx = qst.qst_init(3)
    try:
        with pytest.raises(qst.QstError) as e:
            qst.qst_graph_enable(ctx, True)
        assert e.value.status == qst.QST_E_UNSUPPORTED
    finally:
        qst.qst_destroy(ctx)


def test_batch_matches_individual_contexts():
    Ns = [3, 5, 7, 4, 6, 8, 3]
    data = [_inputs(N, 10 + b) for b, N in enumerate(Ns)]
    steps = 5
    want = [_run(N, f, th, steps, qst.QST_FP32, graph=False) for N, (f, th) in zip(Ns, data)]
    stream = torch.cuda.Stream()
    bt = qst.qst_batch_init(Ns, stream=stream.cuda_stream)
    try:
        fds = [torch.from_numpy(f).cuda() for f, _ in data]
        for b, (_, th) in enumerate(data):
            qst.qst_batch_set_params(bt, b, th)
        torch.cuda.synchronize()
        losses = [qst.qst_batch_step(bt, fds, want_losses=True) for _ in range(steps)]
        for b, N in enumerate(Ns):
            out = torch.empty(data[b][1].size, device="cuda")
            qst.qst_get_params(qst.qst_batch_context(bt, b), out)
            qst.qst_batch_sync(bt)
            torch.cuda.synchronize()
            assert [l[b] for l in losses] == want[b][0], b
            assert np.array_equal(out.cpu().numpy(), want[b][1]), b
        assert qst.qst_batch_kernel_launches(bt) > 0
    finally:
        qst.qst_batch_destroy(bt)


@pytest.mark.parametrize("prec,fused_max,conc", [(qst.QST_FP32, 6, 0), (qst.QST_MIXED, 0, 1), (qst.QST_MIXED_BF16, 0, 0),
                                                  (qst.QST_FP32, 6, 1)])
def test_grouped_batch_matches_individual_contexts(prec, fused_max, conc):
    """Runs of tomographies of one size (N = 7, 8, 9) launch each kernel of their iteration once for the
    whole run: losses and parameters bit-identical to each tomography run on its own context, and far
    fewer launches per iteration than one chain per tomography."""
    Ns = [9, 7, 8, 9, 8, 7, 7]
    data = [_inputs(N, 30 + b) for b, N in enumerate(Ns)]
    steps = 4
    want = [_run(N, f, th, steps, prec, graph=False, fused_max=fused_max) for N, (f, th) in zip(Ns, data)]
    stream = torch.cuda.Stream()
    o = qst.qst_default_options()
    o.precision = prec
    o.fused_max_qubits = fused_max
    tuning = qst.qst_get_tuning()
    qst.qst_set_tuning(batch_concurrent_runs=conc)  # the runs one after another, or all at once
    bt = qst.qst_batch_init(Ns, opt=o, stream=stream.cuda_stream)
    try:
        fds = [torch.from_numpy(f).cuda() for f, _ in data]
        for b, (_, th) in enumerate(data):
            qst.qst_batch_set_params(bt, b, th)
        torch.cuda.synchronize()
        losses = [qst.qst_batch_step(bt, fds, want_losses=True)]
        l0 = qst.qst_batch_kernel_launches(bt)
        losses += [qst.qst_batch_step(bt, fds, want_losses=True) for _ in range(steps - 1)]
        per_iter = (qst.qst_batch_kernel_launches(bt) - l0) / (steps - 1)
        for b, N in enumerate(Ns):
            out = torch.empty(data[b][1].size, device="cuda")
            qst.qst_get_params(qst.qst_batch_context(bt, b), out)
            qst.qst_batch_sync(bt)
            torch.cuda.synchronize()
            assert [l[b] for l in losses] == want[b][0], b
            assert np.array_equal(out.cpu().numpy(), want[b][1]), b
        # three runs of about a dozen launches each, against 7 chains of about a dozen
        assert per_iter <= 3 * 16, per_iter
    finally:
        qst.qst_batch_destroy(bt)
        qst.qst_set_tuning(**tuning)
