"""Autotuner for the launch parameters of libqst (qst_tuning): times candidates on the GPU it runs on
and, with --write, stores the best in csrc/tuned.h (the defaults of the next build).

Workload: a batch of B independent tomographies with N ~ U{3..9} (the many-states setting of Sec. 4,
one graph launch per iteration of all of them), FP32 and mixed precision, with synthetic frequencies
and network parameters; and, as a guard, single-context mixed steps at N = 10 and 11 (the 11-qubit
step is the headline workload), which the chunk parameter of the weight passes also reaches.

    python -m paper_2207_05341_gb300.autotune [--batch 512] [--steps 10] [--out log.json] [--write]
    python -m paper_2207_05341_gb300.autotune --apply log.json    # store a log's best values (no GPU)

Stage 1 picks bulk_chunks_per_cta (least 256-column chunks per CTA of a weight pass) by the mixed
batch's time, among the values that keep every guard step within 5 % of its time at the smallest
value (smaller tomographies run mostly in batches, where few CTAs per tomography pay off); stage 2
picks fused_max_qubits and fused_ctas_per_sm, stage 3 batch_concurrent_runs, each by the sum of the
FP32 and mixed batch times.  Every candidate is timed with CUDA events on the batch's stream after warm-up iterations.
"""
import argparse
import json
import os
import re
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

CHUNKS = [1, 2, 4, 8, 16, 32, 64]
FUSED_MAX = [5, 6, 7]
FUSED_CTAS = [1, 2]


def _frequencies(N, seed):
    f = np.random.default_rng(seed).random(4 ** N).astype(np.float32)
    return f / f.sum()


def time_batch(torch, qst, synth, Ns, prec, steps, warmup=3):
    """ms per iteration of one batch step over all tomographies."""
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(device=dev)
    o = qst.qst_default_options()
    o.precision = prec
    bt = qst.qst_batch_init(Ns, opt=o, stream=stream.cuda_stream)
    try:
        fds = []
        for b, N in enumerate(Ns):
            fds.append(torch.from_numpy(_frequencies(N, 1000 + b)).to(dev))
            qst.qst_batch_set_params(bt, b, synth.init_theta(N, 2000 + b).astype(np.float32))
        torch.cuda.synchronize()
        for _ in range(warmup):
            qst.qst_batch_step(bt, fds)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            qst.qst_batch_step(bt, fds)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        qst.qst_batch_destroy(bt)


def time_single(torch, qst, synth, N, prec, steps, warmup=3, repeats=3):
    """ms per qst_step of one context (graph replay, device-resident f; the best of `repeats` runs of
    `steps` steps)."""
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(device=dev)
    o = qst.qst_default_options()
    o.precision = prec
    ctx = qst.qst_init(N, opt=o, stream=stream.cuda_stream)
    try:
        qst.qst_graph_enable(ctx, True)
        qst.qst_set_params(ctx, synth.init_theta(N, 3).astype(np.float32))
        fd = torch.from_numpy(_frequencies(N, 7)).to(dev)
        for _ in range(warmup):
            qst.qst_step(ctx, fd)
        qst.qst_sync(ctx)
        best = None
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                qst.qst_step(ctx, fd)
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1) / steps
            best = t if best is None else min(best, t)
        return best
    finally:
        qst.qst_destroy(ctx)


def write_tuned(best):
    path = os.path.join(HERE, "csrc", "tuned.h")
    src = open(path).read()
    names = {"bulk_chunks_per_cta": "kTunedBulkChunksPerCta", "fused_ctas_per_sm": "kTunedFusedCtasPerSm",
             "fused_max_qubits": "kTunedFusedMaxQubits", "batch_concurrent_runs": "kTunedBatchConcurrentRuns"}
    for key, const in names.items():
        if key not in best:
            continue
        src, k = re.subn(r"(constexpr int %s = )\d+;" % const, r"\g<1>%d;" % best[key], src)
        if k != 1:
            raise RuntimeError(f"{const} not found in {path}")
    open(path, "w").write(src)
    return path


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--seed", type=int, default=30)
    ap.add_argument("--write", action="store_true", help="store the best values in csrc/tuned.h")
    ap.add_argument("--out", help="write the timings and the choice to this JSON file")
    ap.add_argument("--apply", help="store the best values of an earlier --out log in csrc/tuned.h and exit")
    args = ap.parse_args(argv)
    if args.apply:
        best = json.load(open(args.apply))["best"]
        print(write_tuned(best), best)
        return best

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("autotune needs a CUDA device")
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2207_05341_gb300 import qst, synth
    qst.load()

    Ns = [int(x) for x in np.random.default_rng(args.seed).integers(3, 10, args.batch)]
    start = qst.qst_get_tuning()
    log = {"workload": f"{args.batch} tomographies, N ~ U{{3..9}}", "start": start, "stage1": [], "stage2": []}

    # stage 1: chunks per CTA of the weight passes
    guard_N = [10, 11]
    guard_ref = None
    best1 = None
    for ch in CHUNKS:
        qst.qst_set_tuning(bulk_chunks_per_cta=ch)
        guard = {N: time_single(torch, qst, synth, N, qst.QST_MIXED, args.steps) for N in guard_N}
        if guard_ref is None:
            guard_ref = guard
        ok = all(guard[N] <= 1.05 * guard_ref[N] for N in guard_N)
        mixed = time_batch(torch, qst, synth, Ns, qst.QST_MIXED, args.steps)
        row = {"bulk_chunks_per_cta": ch, "batch_mixed_ms": mixed,
               "single_mixed_ms": {str(N): guard[N] for N in guard_N}, "guard_ok": ok}
        log["stage1"].append(row)
        print(json.dumps(row), flush=True)
        if ok and (best1 is None or mixed < best1[1]):
            best1 = (ch, mixed)
    qst.qst_set_tuning(bulk_chunks_per_cta=best1[0])

    # stage 2: the fused batch launch
    best2 = None
    for fm in FUSED_MAX:
        for fc in FUSED_CTAS:
            qst.qst_set_tuning(fused_max_qubits=fm, fused_ctas_per_sm=fc)
            fp32 = time_batch(torch, qst, synth, Ns, qst.QST_FP32, args.steps)
            mixed = time_batch(torch, qst, synth, Ns, qst.QST_MIXED, args.steps)
            row = {"fused_max_qubits": fm, "fused_ctas_per_sm": fc, "batch_fp32_ms": fp32, "batch_mixed_ms": mixed}
            log["stage2"].append(row)
            print(json.dumps(row), flush=True)
            if best2 is None or fp32 + mixed < best2[2]:
                best2 = (fm, fc, fp32 + mixed)
    best = {"bulk_chunks_per_cta": best1[0], "fused_max_qubits": best2[0], "fused_ctas_per_sm": best2[1]}
    qst.qst_set_tuning(**best)

    # stage 3: runs of one size one after another, or all at once
    best3 = None
    log["stage3"] = []
    for conc in (0, 1):
        qst.qst_set_tuning(batch_concurrent_runs=conc)
        fp32 = time_batch(torch, qst, synth, Ns, qst.QST_FP32, args.steps)
        mixed = time_batch(torch, qst, synth, Ns, qst.QST_MIXED, args.steps)
        row = {"batch_concurrent_runs": conc, "batch_fp32_ms": fp32, "batch_mixed_ms": mixed}
        log["stage3"].append(row)
        print(json.dumps(row), flush=True)
        if best3 is None or fp32 + mixed < best3[1]:
            best3 = (conc, fp32 + mixed)
    best["batch_concurrent_runs"] = best3[0]
    qst.qst_set_tuning(**best)
    log["best"] = best
    print(json.dumps({"best": best}), flush=True)
    if args.write:
        log["written"] = write_tuned(best)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(log, fh, indent=1)
    return log


if __name__ == "__main__":
    main()
