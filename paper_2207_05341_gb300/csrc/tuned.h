// Launch parameters of the one-CTA iteration (tomo_fused.cu), written by autotune.py from timings on the
// target GPU.  The thread count fixes the order of the step's sums: a batch and a single context use the
// same value, so their iterations stay bit-identical.
#pragma once

namespace qst {
constexpr int kFusedThreads = 512;          // threads of the CTA that runs one tomography's iteration
constexpr int kFusedCtasPerSm = 2;          // resident CTAs per SM of the persistent batch launch (at most)
constexpr int kFusedMaxQubitsDefault = 7;   // largest N run as one fused iteration by default
}  // namespace qst
