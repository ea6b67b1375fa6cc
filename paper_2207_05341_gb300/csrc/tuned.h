// Launch parameters chosen by autotune.py from timings on the target GPU (the defaults of qst_tuning).
// kFusedThreads fixes the order of the one-CTA iteration's sums, and the chunks per CTA of the bulk
// weight passes fix the partition of theirs: a batch and a single context use the same values, so their
// iterations stay bit-identical.
#pragma once

namespace qst {
constexpr int kFusedThreads = 512;          // threads of the CTA that runs one tomography's iteration
constexpr int kFusedCtasPerSmMax = 2;       // register budget of that kernel: resident CTAs per SM at most
constexpr int kTunedFusedCtasPerSm = 2;     // resident CTAs per SM of the persistent batch launch
constexpr int kTunedFusedMaxQubits = 6;     // largest N run as one fused iteration by default
constexpr int kTunedBulkChunksPerCta = 32;  // least 256-column chunks per CTA of a bulk weight pass
constexpr int kTunedBatchConcurrentRuns = 1;  // 1: a batch's runs of one size start together
}  // namespace qst
