// Counter-based random numbers shared by the samplers (fidelity.cu, sampler.cu).
#pragma once

namespace qst {

// Output s (0-based) of the SplitMix64 generator started at `seed` (Steele, Lea and Flood, OOPSLA 2014):
// x = seed + (s + 1) 0x9E3779B97F4A7C15, then its published two-round mix.  Any draw is computed on its
// own, so every thread takes its draws without shared state.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long s) {
  unsigned long long z = seed + (s + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace qst
