"""Benchmark of the NN-QST maximum-likelihood iteration on one GB300 (N = 11 qubits).

One step = one full iteration of the hot path (network forward, Hermitian T,
X = T T, POVM map, likelihood, adjoint, G T, backward, Rprop) through the C ABI
(qst_step).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (synthetic, seeded): N = 11, a Haar-random pure state mixed with
depolarising noise, 10^7 multinomial shots of the tetrahedral product POVM, the
3-layer network (4^11 -> 22 -> 4^11) from a seeded default initialisation.
Under torchrun (N > 1 GPUs) every rank runs its own independent tomography
(replicas; there is no collective in the method's data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "11-qubit QST MLE iters/s & time-to-fidelity 0.99: mixed vs plain FP32, 1 GB300"
UNIT = "iters/s"
NQ = 11
SHOTS = 10**7
LAMBDAS = (0.0, 0.1, 0.2)
STATE_SEEDS = (20, 21, 22)
THETA_SEED = 23
COUNT_SEED = 24
FID_TARGET = 0.99
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP32_LANES_PER_SM = 128
NUM_SMS = 152


def workload_name(lam):
    return (f"N=11 qubits (rho 2048x2048, 4^11 outcomes), Haar pure state + depolarizing lambda={lam}, "
            f"10^7 shots, Chol_H, FNN 4^11->22->4^11, Rprop")


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(dist, ws, ms_local):
    """The timed region's length as the job sees it: the max over the ranks (one float64 all-reduced on
    the host; the replicas exchange nothing else)."""
    if ws <= 1:
        return ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, steps, ms_max):
    """Whole-job iterations per second: every rank ran `steps` iterations within ms_max."""
    return ws * steps / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clocks sampled every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"qst_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            out = {}
            for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
                for kk, vv in d.items():
                    if kk.startswith(k) and isinstance(vv, (int, float)):
                        out.setdefault(k, float(vv))
            if "hbm_gbs" in out:
                return out, "measured"
        except Exception:
            pass
    return dict(FALLBACK_PEAKS), "fallback"


def sources_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2207_05341_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded(phase, key):
    """A per-launch ncu figure of the phase's kernel from profiles/traffic.json (DRAM bytes, tensor-pipe
    share), or None once that kernel's sources have changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        e = json.load(open(p))["entries"][phase]
        if sources_hash(e["sources"]) != e["sha"]:
            return None
        return e.get(key)
    except Exception:
        return None


def recorded_traffic(phase):
    return recorded(phase, "bytes_per_launch")


# ------------------------------------------------------------------ algorithmic work per phase (N = 11)
def phase_work(phase, N, mixed):
    """(bound, algorithmic amount per launch, unit) of each phase, as stated in the design notes."""
    n = 4 ** N
    d = 2 ** N
    H = 2 * N
    if phase == "build_T":
        return "hbm", (H + 1) * 4 * n + (12 if mixed else 8) * n, "B"
    if phase == "x_fwd":
        return ("tensor" if mixed else "alu"), 4 * d ** 3, "FLOP"
    if phase == "gt":
        return ("tensor" if mixed else "alu"), 8 * d ** 3, "FLOP"
    if phase == "povm_lo":    # lower half of X read, packed intermediate written
        return "hbm", 4 * n + 4 * n, "B"
    if phase == "povm_hi":    # intermediate and f read, packed adjoint written
        return "hbm", 4 * n + 4 * n + 4 * n, "B"
    if phase == "povm_adj":   # packed adjoint read, G written
        return "hbm", 4 * n + 8 * n, "B"
    if phase == "povm_map":   # qst_probs: lower half of rho read, p written (8 n B, the map's algorithmic bytes)
        return "hbm", 8 * n, "B"
    if phase == "sym":
        return "hbm", 8 * n + 4 * n, "B"
    if phase == "w2":
        return "hbm", 16 * H * n + 20 * n, "B"
    if phase == "w1":
        return "hbm", 16 * H * n + 4 * n, "B"
    if phase == "hidden":
        return "hbm", 4 * H * n + 4 * n, "B"
    return "hbm", 0, "B"


# ------------------------------------------------------------------ evaluation (off the clock)
def fidelity_depolarized(torch, rho_hat, psi, lam):
    """F_q of Sec. 2.3 between rho_hat and (1-lam)|psi><psi| + lam I/d, evaluated on the GPU.

    sqrt(rho) = b I + (sqrt(1 - lam + lam/d) - b)|psi><psi| with b = sqrt(lam/d), then
    F = (sum_i sqrt(w_i))^2 over the eigenvalues w of sqrt(rho) rho_hat sqrt(rho).
    Measurement harness only (not part of the hot path).
    """
    d = rho_hat.shape[0]
    if lam == 0.0:
        return float(torch.real(torch.vdot(psi, rho_hat @ psi)))
    # complex128: the spectrum spans (1 - lam)^2 down to (lam / d)^2 ~ 1e-9, below FP32 resolution
    rho_hat = rho_hat.to(torch.complex128)
    psi = psi.to(torch.complex128)
    b = (lam / d) ** 0.5
    a = (1 - lam + lam / d) ** 0.5 - b
    S = a * torch.outer(psi, psi.conj())
    S.diagonal().add_(b)
    Mx = S @ rho_hat @ S
    Mx = 0.5 * (Mx + Mx.conj().T)
    w = torch.linalg.eigvalsh(Mx).clamp_min(0)
    return float(torch.sqrt(w).sum() ** 2)


# ------------------------------------------------------------------ our arm
def make_inputs(torch, qst, synth, dev, lam, seed, exact=False):
    """Target state, exact probabilities (by the library's own POVM map) and seeded counts.

    exact=True returns the noise-free probabilities themselves as f (the setting of
    the paper's Fig. 2-4 timings); otherwise f = counts / shots with 10^7 shots.
    """
    psi = synth.haar_pure(NQ, seed)
    rho = synth.depolarized(psi, lam)
    # the library works on the stream it is given: use torch's current stream so that the
    # copies below are ordered after qst_probs (torch streams do not sync with the legacy one)
    ctx = qst.qst_init(NQ, stream=torch.cuda.current_stream(dev).cuda_stream)
    try:
        rho_t = torch.from_numpy(rho.astype(np.complex64)).to(dev)
        P = torch.empty(4 ** NQ, device=dev)
        qst.qst_probs(ctx, rho_t, P)
        P = P.double().cpu().numpy()
    finally:
        qst.qst_destroy(ctx)
    if exact:
        P = np.clip(P, 0.0, None)
        return psi, (P / P.sum()).astype(np.float32)
    f = synth.frequencies(synth.multinomial_counts(P, SHOTS, COUNT_SEED + seed), np.float32)
    return psi, f


def time_steps(torch, qst, ctx, f_dev, K, stream):
    l0 = qst.qst_kernel_launches(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        qst.qst_step(ctx, f_dev, want_loss=False)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), qst.qst_kernel_launches(ctx) - l0


def run_precision(torch, qst, synth, dev, stream, prec, theta0, f, K, W, dist, mapping=None, network=None):
    """K timed iterations replayed from the captured CUDA graph (the headline), the same
    K launched kernel by kernel, per-phase device times from timed graph replays, and the
    end-to-end rate through qst_step with a page-locked host f and the loss read back."""
    opt = qst.qst_default_options()
    opt.precision = prec
    if mapping is not None:
        opt.mapping = mapping
    if network is not None:
        opt.network = network
    ctx = qst.qst_init(NQ, opt=opt, stream=stream.cuda_stream)
    try:
        qst.qst_set_params(ctx, theta0)
        f_dev = torch.from_numpy(f).to(dev)
        qst.qst_graph_enable(ctx, True)
        for _ in range(max(W, 3)):
            qst.qst_step(ctx, f_dev, want_loss=False)
        torch.cuda.synchronize()
        dist.barrier()
        with ClockSampler(torch.cuda.current_device()) as clk:
            ms, launches = time_steps(torch, qst, ctx, f_dev, K, stream)
        torch.cuda.synchronize()
        dist.barrier()
        # launch by launch, for comparison (same kernels, host launch gaps included)
        qst.qst_graph_enable(ctx, False)
        for _ in range(2):
            qst.qst_step(ctx, f_dev, want_loss=False)
        ms_nograph, _ = time_steps(torch, qst, ctx, f_dev, K, stream)
        # per phase: events captured in the graph, read after each replay
        qst.qst_graph_enable(ctx, True)
        qst.qst_timing_enable(ctx, 1)
        qst.qst_step(ctx, f_dev, want_loss=False)
        reps = min(K, 20)
        acc = {p: [0.0, 0] for p in qst.PHASES}
        for _ in range(reps):
            qst.qst_step(ctx, f_dev, want_loss=False)
            for p, (t, n) in qst.qst_timing_read(ctx).items():
                acc[p][0] += t
                acc[p][1] += n
        phases = {p: (t, n) for p, (t, n) in acc.items()}
        qst.qst_timing_enable(ctx, 0)
        # end to end: page-locked host f copied in (a node of the graph) and the loss read back every step
        f_pin = torch.from_numpy(f).pin_memory()
        qst.qst_step(ctx, f_pin, want_loss=True)
        qst.qst_step(ctx, f_pin, want_loss=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            qst.qst_step(ctx, f_pin, want_loss=True)
        e2e_s = time.perf_counter() - t0
        return {"ms": ms, "ms_nograph": ms_nograph, "launches": launches, "phases": phases,
                "clocks": clk.summary(), "e2e_s": e2e_s}
    finally:
        qst.qst_destroy(ctx)


def povm_map_time(torch, qst, dev, stream, reps=10, calls=16, buffers=8):
    """GPU time of one qst_probs call (Sec. 3.3 eq. PS) at N = 11: `calls` calls over `buffers` different
    rho (8 x 33.5 MB, larger than L2) captured in one CUDA graph and replayed `reps` times (replay
    launches the kernels back to back: what is timed is GPU work, not the host's launch rate)."""
    d, n = 2 ** NQ, 4 ** NQ
    ctx = qst.qst_init(NQ, stream=stream.cuda_stream)
    try:
        g = torch.Generator(device=dev).manual_seed(5)
        rhos = [torch.randn(d, d, dtype=torch.complex64, device=dev, generator=g) for _ in range(buffers)]
        ps = [torch.empty(n, device=dev) for _ in range(buffers)]
        for k in range(buffers):
            qst.qst_probs(ctx, rhos[k], ps[k])  # first calls outside the capture (one-time set-up)
        stream.synchronize()
        G = torch.cuda.CUDAGraph()
        with torch.cuda.graph(G, stream=stream):
            for i in range(calls):
                qst.qst_probs(ctx, rhos[i % buffers], ps[i % buffers])
        G.replay()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            G.replay()
        e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / (reps * calls)
        return {"workload": f"qst_probs at N=11 (rho 2048x2048 complex64, 4^11 outcomes), {buffers} inputs of "
                            f"33.5 MB rotated (268 MB, larger than L2), {calls} calls per graph replay",
                "us_per_call": us, "kernels_per_call": 2}
    finally:
        qst.qst_destroy(ctx)


def fidelity_run(torch, qst, dev, stream, prec, theta0, f, psi, lam, max_iters, every, stop_at_target):
    """Iterate qst_step from theta0; every `every` steps evaluate F (off the clock).

    Returns GPU seconds of the steps only, the first iteration with F >= 0.99 (or
    None), and the peak F with its iteration and time.
    """
    opt = qst.qst_default_options()
    opt.precision = prec
    ctx = qst.qst_init(NQ, opt=opt, stream=stream.cuda_stream)
    d = 2 ** NQ
    try:
        qst.qst_set_params(ctx, theta0)
        qst.qst_graph_enable(ctx, True)
        f_dev = torch.from_numpy(f).to(dev)
        psi_t = torch.from_numpy(psi.astype(np.complex64)).to(dev)
        rho = torch.empty((d, d), dtype=torch.complex64, device=dev)
        gpu_ms, it = 0.0, 0
        hit = None
        peak = (-1.0, 0, 0.0)
        F = None
        traj = []
        while it < max_iters:
            chunk = every if it < 100 else 5 * every
            ms, _ = time_steps(torch, qst, ctx, f_dev, chunk, stream)
            gpu_ms += ms
            it += chunk
            qst.qst_get_rho(ctx, f_dev, rho)
            F = fidelity_depolarized(torch, rho, psi_t, lam)
            traj.append((it, gpu_ms / 1e3, F))
            if F > peak[0]:
                peak = (F, it, gpu_ms / 1e3)
            if hit is None and F >= FID_TARGET:
                hit = {"iters": it, "seconds": gpu_ms / 1e3}
                if stop_at_target:
                    break
        return {"lambda": lam, "reached": hit is not None, "iters": hit["iters"] if hit else None,
                "seconds": hit["seconds"] if hit else None, "F_last": F, "iters_run": it,
                "F_peak": peak[0], "peak_iter": peak[1], "peak_seconds": peak[2], "trajectory": traj}
    finally:
        qst.qst_destroy(ctx)


def fidelity_eval(torch, qst, dev, stream, theta0, lam, seed, steps=200, samples=10**6):
    """On-device classical fidelity (Sec. 2.3 eq. F_CF and the sampled eq. fc_sample, qst_classical_fidelity)
    beside the state fidelity F_q of the harness (torch, complex128), after `steps` mixed iterations at
    N = 11 from exact probabilities (the target distribution is then the input itself)."""
    from paper_2207_05341_gb300 import synth
    psi, P = make_inputs(torch, qst, synth, dev, lam, seed, exact=True)
    opt = qst.qst_default_options()
    opt.precision = qst.QST_MIXED
    ctx = qst.qst_init(NQ, opt=opt, stream=stream.cuda_stream)
    try:
        qst.qst_set_params(ctx, theta0)
        qst.qst_graph_enable(ctx, True)
        P_dev = torch.from_numpy(P).to(dev)
        time_steps(torch, qst, ctx, P_dev, steps, stream)
        out = {"workload": f"N=11, depolarizing lambda={lam}, exact probabilities, {steps} mixed iterations"}
        for name, S in (("exact", 0), ("sampled", samples)):
            best, val = None, None
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                val = qst.qst_classical_fidelity(ctx, P_dev, P_dev, samples=S, seed=1)
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            out[f"Fc_{name}"] = val
            out[f"Fc_{name}_ms"] = best * 1e3
        out["samples"] = samples
        d = 2 ** NQ
        rho = torch.empty((d, d), dtype=torch.complex64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qst.qst_get_rho(ctx, P_dev, rho)
        Fq = fidelity_depolarized(torch, rho, torch.from_numpy(psi.astype(np.complex64)).to(dev), lam)
        torch.cuda.synchronize()
        out["Fq_harness"] = Fq
        out["Fq_harness_ms"] = (time.perf_counter() - t0) * 1e3
        # the library's own F_q (eq. fq_decom: Jacobi decomposition of T, secular equation of the target)
        psi_dev = torch.from_numpy(psi.astype(np.complex64)).to(dev)
        best = None
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            val = qst.qst_state_fidelity(ctx, P_dev, psi_dev, 1.0 - lam)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        out["Fq_gpu"] = val
        out["Fq_gpu_ms"] = best * 1e3
        out["note"] = ("F_c >= F_q (eq. F_CF is an upper bound); Fq_harness is the harness's complex128 "
                       "evaluation, Fq_gpu the library's (qst_state_fidelity, 12 FP32 Jacobi sweeps on T)")
        return out
    finally:
        qst.qst_destroy(ctx)


def sampler_eval(torch, qst, synth, dev, stream, lam, seed):
    """Synthetic data on the GPU (qst_test_state, qst_probs, qst_sample_counts) against the host
    generator (numpy multinomial) for the headline workload's 10^7 shots at N = 11."""
    opt = qst.qst_default_options()
    ctx = qst.qst_init(NQ, opt=opt, stream=stream.cuda_stream)
    try:
        d, n = 2 ** NQ, 4 ** NQ
        rho = torch.empty((d, d), dtype=torch.complex64, device=dev)
        P32 = torch.empty(n, dtype=torch.float32, device=dev)
        counts = torch.empty(n, dtype=torch.int64, device=dev)
        f = torch.empty(n, dtype=torch.float32, device=dev)
        qst.qst_test_state(ctx, qst.QST_STATE_GHZI, 1.0 - lam, rho)
        qst.qst_probs(ctx, rho, P32)
        P = P32.double()
        qst.qst_sample_counts(ctx, P, SHOTS, seed, counts, f)  # warm-up (allocates the scratch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qst.qst_sample_counts(ctx, P, SHOTS, seed, counts, f)
        torch.cuda.synchronize()
        gpu_ms = (time.perf_counter() - t0) * 1e3
        Ph = P.cpu().numpy()
        t0 = time.perf_counter()
        synth.multinomial_counts(Ph, SHOTS, seed)
        host_ms = (time.perf_counter() - t0) * 1e3
        return {"workload": f"N=11 GHZi state, depolarizing lambda={lam}, {SHOTS} shots",
                "gpu_counts_ms": gpu_ms, "host_numpy_multinomial_ms": host_ms,
                "counts_sum": int(counts.sum().item())}
    finally:
        qst.qst_destroy(ctx)


def cpu_baseline(f, theta0, seconds=12.0):
    """The FP64 oracle, as it stands, on the host cores: full N = 11 iterations."""
    import oracle as O
    M = O.tetrahedral_povm()
    theta = theta0.astype(np.float64)
    f64 = f.astype(np.float64)
    st = O.RpropState(theta.size)
    t0 = time.perf_counter()
    n = 0
    while True:
        _, g, _ = O.loss_and_grad(theta, f64, M, NQ)
        theta = O.rprop_update(theta, g, st)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 8:
            break
    return {"value": n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} full N=11 iterations (loss, analytic gradient, Rprop) in FP64 NumPy, {el:.1f} s"}


def batch_c4(torch, qst, synth, dev, steps, warmup, seed=30, B=512, prec=None):
    """512 independent tomographies, N ~ U{3..9}, rank-r Ginibre states (r ~ U{1..2^N}),
    10^5 N shots each; one graph launch per iteration of all of them.  prec: None = FP32; QST_MIXED
    runs the tomographies with N >= 7 on the tensor-core path."""
    rng = np.random.default_rng(seed)
    Ns = [int(x) for x in rng.integers(3, 10, B)]
    stream = torch.cuda.Stream(device=dev)
    o = None
    if prec is not None:
        o = qst.qst_default_options()
        o.precision = prec
    bt = qst.qst_batch_init(Ns, opt=o, stream=stream.cuda_stream)
    try:
        fds = []
        with torch.cuda.stream(stream):
            for b, N in enumerate(Ns):
                r = int(rng.integers(1, 2 ** N + 1))
                rho = synth.ginibre_mixed(N, r, seed * 100000 + b)
                rho_t = torch.from_numpy(rho.astype(np.complex64)).to(dev)
                P = torch.empty(4 ** N, device=dev)
                cb = qst.qst_batch_context(bt, b)
                torch.cuda.current_stream(dev).synchronize()
                qst.qst_probs(cb, rho_t, P)
                qst.qst_sync(cb)  # the context runs on its own stream
                P = P.double().cpu().numpy()
                f = synth.frequencies(synth.multinomial_counts(P, 10**5 * N, seed * 100000 + B + b), np.float32)
                fds.append(torch.from_numpy(f).to(dev))
                qst.qst_batch_set_params(bt, b, synth.init_theta(N, seed * 100000 + 2 * B + b).astype(np.float32))
            for _ in range(max(warmup, 2)):
                qst.qst_batch_step(bt, fds)
            torch.cuda.synchronize()
            l0 = qst.qst_batch_kernel_launches(bt)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                qst.qst_batch_step(bt, fds)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            launches = qst.qst_batch_kernel_launches(bt) - l0
            losses = qst.qst_batch_step(bt, fds, want_losses=True)
        it_s = B * steps / (ms / 1e3)
        # algorithmic HBM bytes of one iteration of all B (the per-phase bytes of the single-context
        # rooflines, summed over the memory phases of each tomography)
        mem_phases = ("build_T", "povm_lo", "povm_hi", "povm_adj", "sym", "w2", "w1")
        hbm_bytes = sum(phase_work(ph, N, prec is not None and N >= 7)[1] for N in Ns for ph in mem_phases)
        floor_ms = hbm_bytes / (load_peaks()[0]["hbm_gbs"] * 1e9) * 1e3
        return {"workload": "512 tomographies, N ~ U{3..9}, rank-r Ginibre (r ~ U{1..2^N}), 10^5 N shots, "
                            + ("FP32" if prec is None else "mixed FP16x3 for N >= 7, FP32 below"),
                "Ns_hist": {str(k): Ns.count(k) for k in range(3, 10)},
                "ms_per_batch_iteration": ms / steps, "aggregate_iters_per_s": it_s,
                "tomographies_per_s_at_1000_iters": it_s / 1000.0,
                "graph_nodes_per_iteration": launches // max(steps, 1),
                "hbm_bytes_per_iteration": hbm_bytes,
                "hbm_floor_ms": floor_ms,
                "frac_of_hbm_floor": floor_ms / (ms / steps),
                "all_losses_finite": bool(np.all(np.isfinite(losses)))}
    finally:
        qst.qst_batch_destroy(bt)


def c5_leg(torch, qst, synth, dev, steps, seed=40):
    """N = 12 (rho 4096 x 4096, 4^12 outcomes), 10^8 shots, depolarised rank-r Ginibre state:
    Chol_H (= A_2, Sec. 3.2) on the mixed tensor-core path, and A_P with P = 1.5: mixed (cold Jacobi
    first step, then tensor-core refinements of the previous eigenvectors, handed to the sweeps when they
    do not converge), mixed with every warm step on the sweeps (eig_refine = 0), and FP32 (cold first
    step, then warm-started Jacobi sweeps)."""
    N = 12
    rng = np.random.default_rng(seed)
    r = int(np.exp(rng.uniform(0, np.log(64))))
    lam = float(rng.uniform(0, 0.3))
    g = synth.ginibre_mixed(N, r, seed)
    rho = (1 - lam) * g + lam * np.eye(2 ** N) / 2 ** N
    stream = torch.cuda.Stream(device=dev)
    out = {"workload": f"N=12, rank-{r} Ginibre mixed with depolarizing lambda={lam:.3f}, 10^8 shots"}
    with torch.cuda.stream(stream):
        ctx = qst.qst_init(N, stream=stream.cuda_stream)
        try:
            P = torch.empty(4 ** N, device=dev)
            qst.qst_probs(ctx, torch.from_numpy(rho.astype(np.complex64)).to(dev), P)
            P = P.double().cpu().numpy()
        finally:
            qst.qst_destroy(ctx)
        del rho, g
        f = torch.from_numpy(synth.frequencies(synth.multinomial_counts(P, 10**8, seed + 1), np.float32)).to(dev)
        theta = synth.init_theta(N, seed + 2).astype(np.float32)
        for name, prec, mapping, p_ord in (("chol_h_mixed_fp16x3", qst.QST_MIXED, qst.QST_MAP_CHOL_H, 2.0),
                                           ("abs_p1.5_mixed_tc_refinement", qst.QST_MIXED, qst.QST_MAP_ABS_P, 1.5),
                                           ("abs_p1.5_mixed_sweeps", qst.QST_MIXED, qst.QST_MAP_ABS_P, 1.5),
                                           ("abs_p1.5_fp32_jacobi", qst.QST_FP32, qst.QST_MAP_ABS_P, 1.5)):
            o = qst.qst_default_options()
            o.precision, o.mapping, o.P = prec, mapping, p_ord
            if name.endswith("_sweeps"):
                o.eig_refine = 0  # warm steps straight to the sweeps (products on tensor cores)
            ctx = qst.qst_init(N, opt=o, stream=stream.cuda_stream)
            try:
                qst.qst_set_params(ctx, theta)
                L0, _ = qst.qst_step(ctx, f)  # first step: input validation, hidden layer, cold eigensolver
                k = 2 if prec == qst.QST_FP32 else steps  # the FP32 Jacobi path takes about a second per step
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(k):
                    qst.qst_step(ctx, f, want_loss=False)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / k
                L1, _ = qst.qst_step(ctx, f)
                out[name] = {"ms_per_iter": ms, "iters_per_s": 1e3 / ms, "steps_timed": k,
                             "loss_first": L0, "loss_after": L1}
                if mapping == qst.QST_MAP_ABS_P and prec != qst.QST_FP32:
                    ref, fb = qst.qst_eig_counts(ctx)
                    out[name]["tc_refinements"], out[name]["steps_on_jacobi_sweeps"] = ref, fb
            finally:
                qst.qst_destroy(ctx)
    out["note"] = "A_P with P = 2 is Chol_H (Sec. 3.2), so the P = 2 runs of this config use the T T path"
    return out


class _NoDist:
    def barrier(self):
        pass


def profile_only(args):
    """Short, fixed launch sequence for ncu: inputs, then a few steps of each available path."""
    import torch

    from paper_2207_05341_gb300 import qst, synth
    qst.load()
    dev = torch.device("cuda", 0)
    psi, f = make_inputs(torch, qst, synth, dev, LAMBDAS[1], STATE_SEEDS[1])
    cnn = args.profile_net == "cnn"
    theta0 = (synth.init_theta_cnn if cnn else synth.init_theta)(NQ, THETA_SEED).astype(np.float32)
    f_dev = torch.from_numpy(f).to(dev)
    for prec in (qst.QST_MIXED,) if cnn else (qst.QST_FP32, qst.QST_MIXED, qst.QST_MIXED_BF16):
        o = qst.qst_default_options()
        o.precision = prec
        if cnn:
            o.network = qst.QST_NET_CNN
        try:
            ctx = qst.qst_init(NQ, opt=o)
        except qst.QstError:
            continue
        try:
            qst.qst_set_params(ctx, theta0)
            for _ in range(args.profile_steps):
                qst.qst_step(ctx, f_dev, want_loss=False)
            qst.qst_sync(ctx)
        finally:
            qst.qst_destroy(ctx)
    torch.cuda.synchronize()


def profile_batch(args):
    """Profiling aid: the 512-tomography batch of batch_c4 (uniform random frequencies instead of sampled
    counts, which do not change the kernels), 3 warm-up iterations, then args.profile_batch_steps
    iterations inside the NVTX range "timed" (for ncu --nvtx --nvtx-include "timed/")."""
    import torch

    from paper_2207_05341_gb300 import qst, synth
    qst.load()
    dev = torch.device("cuda", 0)
    Ns = [int(x) for x in np.random.default_rng(30).integers(args.profile_batch_min_n, args.profile_batch_max_n + 1,
                                                             args.profile_batch_count)]
    stream = torch.cuda.Stream(device=dev)
    o = qst.qst_default_options()
    if args.profile_batch == "mixed":
        o.precision = qst.QST_MIXED
    bt = qst.qst_batch_init(Ns, opt=o, stream=stream.cuda_stream)
    try:
        fds = []
        for b, N in enumerate(Ns):
            f = np.random.default_rng(1000 + b).random(4 ** N).astype(np.float32)
            fds.append(torch.from_numpy(f / f.sum()).to(dev))
            qst.qst_batch_set_params(bt, b, synth.init_theta(N, 2000 + b).astype(np.float32))
        torch.cuda.synchronize()
        for _ in range(3):
            qst.qst_batch_step(bt, fds)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        for _ in range(args.profile_batch_steps):
            qst.qst_batch_step(bt, fds)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    finally:
        qst.qst_batch_destroy(bt)


def profile_absp(args):
    """Profiling aid: one A_P (P = 1.5) context at N = args.profile_absp on the mixed path, its cold first
    step and one warm-started step, with uniform random frequencies."""
    import torch

    from paper_2207_05341_gb300 import qst, synth
    qst.load()
    N = args.profile_absp
    o = qst.qst_default_options()
    o.precision, o.mapping, o.P = qst.QST_MIXED, qst.QST_MAP_ABS_P, 1.5
    ctx = qst.qst_init(N, opt=o)
    try:
        f = np.random.default_rng(N).random(4 ** N).astype(np.float32)
        fd = torch.from_numpy(f / f.sum()).cuda()
        qst.qst_set_params(ctx, synth.init_theta(N, 3).astype(np.float32))
        for _ in range(2):
            qst.qst_step(ctx, fd)
        qst.qst_sync(ctx)
    finally:
        qst.qst_destroy(ctx)


def main_ours(args):
    import torch

    from paper_2207_05341_gb300 import qst, synth
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = _NoDist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
        dist = tdist
    qst.load()
    stream = torch.cuda.Stream(device=dev)
    lam = LAMBDAS[1]
    psi, f = make_inputs(torch, qst, synth, dev, lam, STATE_SEEDS[1])
    theta0 = synth.init_theta(NQ, THETA_SEED).astype(np.float32)

    mixed_ok = True
    try:
        o = qst.qst_default_options(); o.precision = qst.QST_MIXED
        c = qst.qst_init(NQ, opt=o); qst.qst_destroy(c)
    except qst.QstError:
        mixed_ok = False
    precs = [("plain_fp32", qst.QST_FP32)]
    if mixed_ok:
        precs += [("mixed_fp16x3", qst.QST_MIXED), ("mixed_bf16x3", qst.QST_MIXED_BF16)]
    res = {}
    with torch.cuda.stream(stream):
        for name, prec in precs:
            res[name] = run_precision(torch, qst, synth, dev, stream, prec, theta0, f, args.steps, args.warmup, dist)
        # Chol_Delta (Sec. 2.2.1 eq. T_matrix), FP32: not this metric's map, reported beside it
        res["chol_delta_fp32"] = run_precision(torch, qst, synth, dev, stream, qst.QST_FP32, theta0, f, args.steps,
                                               args.warmup, dist, mapping=qst.QST_MAP_CHOL_DELTA)
        # the CNN mapping network of App. A (4N hidden units, about the FNN's parameter count), mixed
        theta_cnn = synth.init_theta_cnn(NQ, THETA_SEED).astype(np.float32)
        res["cnn_mixed_fp16x3"] = run_precision(torch, qst, synth, dev, stream, qst.QST_MIXED, theta_cnn, f, args.steps,
                                                args.warmup, dist, network=qst.QST_NET_CNN)

    head = "mixed_fp16x3" if mixed_ok else "plain_fp32"
    # max over ranks of the timed region
    ms_max = max_over_ranks(dist, ws, res[head]["ms"])
    value = job_rate(ws, args.steps, ms_max)

    ttf = {}
    if args.ttf and rank == 0:
        with torch.cuda.stream(stream):
            inputs = {}
            for lam_i, seed in zip(LAMBDAS, STATE_SEEDS):
                inputs[("exact", lam_i)] = make_inputs(torch, qst, synth, dev, lam_i, seed, exact=True)
                inputs[("shots", lam_i)] = (psi, f) if lam_i == lam else make_inputs(torch, qst, synth, dev, lam_i, seed)
            for name, prec in precs:
                ttf[name] = {"exact_probabilities": [], "shots_1e7": []}
                for lam_i in LAMBDAS:
                    psi_i, f_i = inputs[("exact", lam_i)]
                    ttf[name]["exact_probabilities"].append(
                        fidelity_run(torch, qst, dev, stream, prec, theta0, f_i, psi_i, lam_i, args.max_iters,
                                     args.fid_every, True))
                    psi_i, f_i = inputs[("shots", lam_i)]
                    ttf[name]["shots_1e7"].append(
                        fidelity_run(torch, qst, dev, stream, prec, theta0, f_i, psi_i, lam_i, args.shots_iters,
                                     args.fid_every, False))
    # 10^7 shots: F peaks below 0.99 for lambda > 0 (the statistical limit of 2.4 counts per outcome), so these
    # runs are timed to 0.99 F_ref,final, F_ref,final the plain FP32 path's fidelity after the same iteration
    # budget (its trajectory follows the FP64 oracle's within 1e-4 at N = 11; tests/test_gpu_n11_fidelity.py)
    q17 = None
    if ttf:
        q17 = {"rule": "time to 0.99 F_ref,final; F_ref,final = plain FP32 path's F after the shots_1e7 budget",
               "per_lambda": []}
        for j, lam_j in enumerate(LAMBDAS):
            F_ref = ttf["plain_fp32"]["shots_1e7"][j]["F_last"]
            row = {"lambda": lam_j, "F_ref_final": F_ref, "threshold": 0.99 * F_ref}
            for name in ttf:
                tr = ttf[name]["shots_1e7"][j]["trajectory"]
                hit = next(((it, sec) for it, sec, F in tr if F >= 0.99 * F_ref), None)
                row[name] = {"iters": hit[0], "seconds": hit[1]} if hit else None
            q17["per_lambda"].append(row)
        for name in ttf:
            for kind in ttf[name]:
                for e in ttf[name][kind]:
                    e.pop("trajectory", None)
    if ws > 1:
        dist.barrier()
    if rank != 0:
        return

    peaks, peak_src = load_peaks()
    r = res[head]
    per = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in r["phases"].items()}
    dom = max((k for k in per if per[k] > 0), key=lambda k: per[k])
    clk = r["clocks"]
    mixed = head != "plain_fp32"

    def roof(phase, ms):
        """(bound, achieved, peak, unit, frac) of one phase from its algorithmic work and its time."""
        bound, amount, unit = phase_work(phase, NQ, mixed)
        sec = ms / 1e3
        if bound == "hbm":
            achieved, peak, runit = amount / sec / 1e9, peaks["hbm_gbs"], "GB/s"
        elif bound == "tensor":
            achieved, peak, runit = amount / sec / 1e12, peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]), "TFLOP/s"
        else:
            mhz = clk.get("sm_max_mhz") or 2070.0
            achieved = amount / sec / 1e12
            peak = NUM_SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
            runit = "TFLOP/s"
        return bound, achieved, peak, runit, achieved / peak

    bound, achieved, peak, runit, _ = roof(dom, per[dom])
    # every phase of the headline step, and the POVM map on its own (qst_probs, graph replay)
    rooflines = {}
    for ph, ms in per.items():
        if ms <= 0:
            continue
        b, a, pk, u, fr = roof(ph, ms)
        e = {"bound": b, "ms": round(ms, 4), "achieved": round(a, 2), "peak": pk, "unit": u, "frac": round(fr, 4)}
        if b == "tensor":  # useful FLOP (4 d^3 lower-tile T T, 8 d^3 G T) against both BF16 peaks
            e["frac_of_burst"] = round(a / peaks["bf16_tflops"], 4)
            e["frac_of_sustained"] = round(a / peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]), 4)
            e["tensor_pipe_active_pct_ncu"] = recorded(ph, "tensor_pipe_pct")
        tr = recorded_traffic(ph)
        if tr is not None:
            e["traffic"] = tr
        rooflines[ph] = e
    if rank == 0:
        with torch.cuda.stream(stream):
            pm = povm_map_time(torch, qst, dev, stream)
        b, a, pk, u, fr = roof("povm_map", pm["us_per_call"] / 1e3)
        rooflines["povm_map"] = {"bound": b, "us_per_call": round(pm["us_per_call"], 2), "achieved": round(a, 2),
                                 "peak": pk, "unit": u, "frac": round(fr, 4), "workload": pm["workload"],
                                 "bytes_per_call": 8 * 4 ** NQ,
                                 "note": "algorithmic bytes 8 n (the lower half of rho read, p written); two kernels"}
    e2e_rate = args.steps / res[head]["e2e_s"]
    n = 4 ** NQ
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp16x3+f32" if head == "mixed_fp16x3" else "f32", "data": "synthetic",
        "config": {"workload": workload_name(lam)},
        "setup": {"path": head, "parallelism": "replicas" if ws > 1 else "single",
                  "launch": "one CUDA graph replay per iteration (qst_graph_enable)",
                  "l2": "inputs larger than L2: 1.5 GB of parameters and Rprop state (3.3 GB of traffic) per step, no flush",
                  "counts": "10^7 multinomial shots (numpy, seed 45) from the Born probabilities of the library's "
                            "own FP32 POVM map; the reference arm draws with the same seed from the oracle's FP64 "
                            "probabilities (the two count vectors agree except where rounding-level differences of "
                            "P move a draw)"},
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons")},
        "e2e": {"value": ws * e2e_rate, "unit": UNIT, "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 12},
        "gpu_launches": int(res[head]["launches"]),
        "roofline": {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": runit,
                     "frac": achieved / peak, "peak_source": peak_src if bound != "alu" else "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                     "traffic": recorded_traffic(dom)},
        "rooflines": rooflines,
        "paths": {name: {"iters_per_s": ws * args.steps / (v["ms"] / 1e3), "ms_per_step": v["ms"] / args.steps,
                         "ms_per_step_launch_by_launch": v["ms_nograph"] / args.steps,
                         "phase_ms": {k: round(pm[0] / pm[1], 4) for k, pm in v["phases"].items() if pm[1]}}
                  for name, v in res.items()},
        "time_to_fidelity": ({"target": FID_TARGET, "note": "GPU time of the steps only; F evaluated off the clock every "
                              f"{args.fid_every} steps up to 100, then every {5 * args.fid_every}; exact_probabilities = noise-free f (paper Fig. 4 setting), "
                              "shots_1e7 = 10^7-shot counts (F peaks, then decays as the fit follows shot noise)",
                              **ttf, "shots_1e7_to_0.99_of_F_ref": q17} if ttf else None),
        "paper_context": "11-qubit tomography within 2 minutes on a laptop (GTX 1070); not this metric's baseline",
    }
    if args.ttf:
        with torch.cuda.stream(stream):
            line["fidelity_on_device"] = fidelity_eval(torch, qst, dev, stream, theta0, LAMBDAS[1], STATE_SEEDS[1])
            line["synthetic_data_on_device"] = sampler_eval(torch, qst, synth, dev, stream, LAMBDAS[1], 5)
    if args.batch:
        line["batch_c4"] = batch_c4(torch, qst, synth, dev, args.steps, args.warmup)
        line["batch_c4_mixed"] = batch_c4(torch, qst, synth, dev, args.steps, args.warmup, prec=qst.QST_MIXED)
    if args.c5:
        line["n12_c5"] = c5_leg(torch, qst, synth, dev, min(args.steps, 10))
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(f, theta0, args.cpu_seconds)
    print(json.dumps(line), flush=True)


def main_reference(args):
    """The reference arm: the FP64 NumPy oracle on the host cores, same metric and workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2207_05341_gb300 import synth
    import oracle as O
    lam = LAMBDAS[1]
    psi = synth.haar_pure(NQ, STATE_SEEDS[1])
    rho = synth.depolarized(psi, lam)
    M = O.tetrahedral_povm()
    P = O.born_probabilities(rho, M).real
    f = synth.frequencies(synth.multinomial_counts(P, SHOTS, COUNT_SEED + STATE_SEEDS[1]), np.float32)
    theta = synth.init_theta(NQ, THETA_SEED).astype(np.float32).astype(np.float64)
    f64 = f.astype(np.float64)
    st = O.RpropState(theta.size)
    for _ in range(args.warmup):
        _, g, _ = O.loss_and_grad(theta, f64, M, NQ)
        theta = O.rprop_update(theta, g, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, g, _ = O.loss_and_grad(theta, f64, M, NQ)
        theta = O.rprop_update(theta, g, st)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(lam)},
            "setup": {"path": "oracle (FP64 NumPy, host)",
                      "counts": "10^7 multinomial shots (numpy, seed 45) from the oracle's FP64 Born probabilities"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} full N=11 iterations after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-ttf", dest="ttf", action="store_false")
    ap.add_argument("--max-iters", type=int, default=2000)
    ap.add_argument("--shots-iters", type=int, default=200)
    ap.add_argument("--fid-every", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-c5", dest="c5", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="profiling aid: only run this many plain and mixed steps at N=11 and exit (no JSON line)")
    ap.add_argument("--profile-net", choices=["fnn", "cnn"], default="fnn",
                    help="with --profile-steps: the FNN in FP32, mixed FP16x3 and BF16x3, or the CNN (mixed)")
    ap.add_argument("--profile-batch", choices=["mixed", "fp32"], default=None,
                    help="profiling aid: only run the 512-tomography batch, its timed iterations in the NVTX "
                         "range 'timed', and exit (no JSON line)")
    ap.add_argument("--profile-batch-steps", type=int, default=2)
    ap.add_argument("--profile-absp", type=int, default=0,
                    help="profiling aid: one mixed A_P context at this N, a cold and a warm step, and exit")
    ap.add_argument("--profile-batch-max-n", type=int, default=9,
                    help="with --profile-batch: N ~ U{min..this} (a smaller case for full ncu captures)")
    ap.add_argument("--profile-batch-min-n", type=int, default=3)
    ap.add_argument("--profile-batch-count", type=int, default=512)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        main_reference(args)
    elif args.profile_steps > 0:
        profile_only(args)
    elif args.profile_batch:
        profile_batch(args)
    elif args.profile_absp:
        profile_absp(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
