// Classical fidelity of Sec. 2.3 between the reconstructed state and a target distribution, on the GPU:
//   exact   (eq. F_CF)     F_c = (sum_k sqrt(P^_k P_k))^2,
//   sampled (eq. fc_sample) F_c ~ (mean_s sqrt(P_{k_s} / P^_{k_s}))^2 with k_s ~ P^,
// where P^_k = q_k / Tr X are the Born probabilities of rho^ = X / Tr X (q from the POVM map of X).
// The draws use the inverse CDF of P^: u_s = (splitmix64(seed, s) >> 11) 2^-53 and k_s = the smallest k
// with c_k > u_s c_{n-1}, c the running sum of max(P^, 0) in FP64 (a three-kernel scan).  SplitMix64 is
// the published counter-based generator (Steele, Lea and Flood, OOPSLA 2014): x = seed + (s + 1) gamma,
// then its two-round mix.  Every sum has a fixed order (block partials, last block), so results repeat.
#include "impl.h"
#include "rng.cuh"

namespace qst {

namespace {

constexpr int kScanPer = 8;                   // elements per thread in the block scan
constexpr int kScanBlock = 256 * kScanPer;    // elements per block

// Sum of one double per thread over the block (warp shuffles, then warps in order); valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Last block: out = (sum of partials[0 .. gridDim.x) * scale)^2, in a fixed order.
__device__ __forceinline__ void finish_square(double* partials, unsigned int* counter, double scale, double* out) {
  if (last_block_arrived(counter)) {
    if (threadIdx.x < 32) {
      double v = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) v += partials[b];
      v = warp_sum(v);
      if (threadIdx.x == 0) {
        v *= scale;
        *out = v * v;
        *counter = 0u;
      }
    }
  }
}

// eq. F_CF: sum_k sqrt(max(q_k, 0) max(P_k, 0)) / sqrt(Tr X), squared -> *out.
template <class R>
__global__ void __launch_bounds__(256) k_fc_exact(const R* __restrict__ q, const R* __restrict__ P, long long n,
                                                   const double* scal, double* partials, unsigned int* counter,
                                                   double* out) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const R a = q[i] > R(0) ? q[i] : R(0), b = P[i] > R(0) ? P[i] : R(0);
    acc += (double)sqrt(a * b);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  finish_square(partials, counter, 1.0 / sqrt(scal[0]), out);
}

// Block-local inclusive scan of P^_k = max(q_k, 0) / Tr X (FP64) into cdf; block totals into tops.
template <class R>
__global__ void __launch_bounds__(256) k_scan_local(const R* __restrict__ q, long long n, const double* scal,
                                                     double* __restrict__ cdf, double* __restrict__ tops) {
  __shared__ double wsum[8];
  const double inv = 1.0 / scal[0];
  const long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanPer;
  double v[kScanPer];
  double run = 0.0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const long long i = base + k;
    const R a = i < n && q[i] > R(0) ? q[i] : R(0);
    run += (double)a * inv;
    v[k] = run;
  }
  // exclusive scan of the thread totals across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  double woff = 0.0;
  for (int w = 0; w < warp; ++w) woff += wsum[w];
  const double off = woff + x - run;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const long long i = base + k;
    if (i < n) cdf[i] = v[k] + off;
  }
  if (threadIdx.x == 255) tops[blockIdx.x] = off + run;
}

// In place: tops[b] <- sum of tops[0 .. b) (one block of 1024 threads, each a contiguous run).
__global__ void __launch_bounds__(1024) k_scan_tops(double* tops, int nb) {
  __shared__ double wsum[32];
  const int per = (nb + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  double run = 0.0;
  for (int b = b0; b < b0 + per && b < nb; ++b) run += tops[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  double off = x - run;
  for (int w = 0; w < warp; ++w) off += wsum[w];
  for (int b = b0; b < b0 + per && b < nb; ++b) {
    const double t = tops[b];
    tops[b] = off;
    off += t;
  }
}

__global__ void __launch_bounds__(256) k_scan_add(double* __restrict__ cdf, long long n, const double* __restrict__ tops) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    cdf[i] += tops[i / kScanBlock];
}

// eq. fc_sample: draws k_s by inverse CDF, accumulates sqrt(P_k / P^_k); (mean)^2 -> *out.
template <class R>
__global__ void __launch_bounds__(256) k_fc_sample(const double* __restrict__ cdf, const R* __restrict__ q,
                                                    const R* __restrict__ P, long long n, long long samples,
                                                    unsigned long long seed, const double* scal, double* partials,
                                                    unsigned int* counter, double* out) {
  const double inv = 1.0 / scal[0];
  const double total = cdf[n - 1];
  double acc = 0.0;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < samples;
       s += (long long)gridDim.x * blockDim.x) {
    const double u = (double)(splitmix64(seed, (unsigned long long)s) >> 11) * 0x1.0p-53;
    const double t = u * total;
    long long lo = 0, hi = n - 1;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (cdf[mid] > t) hi = mid;
      else lo = mid + 1;
    }
    const double ph = (double)q[lo] * inv;  // > 0: a draw never lands on an outcome of zero mass
    const double pk = P[lo] > R(0) ? (double)P[lo] : 0.0;
    acc += sqrt(pk / ph);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  finish_square(partials, counter, 1.0 / (double)samples, out);
}

int grid_for(long long work) {
  long long g = (work + 255) / 256;
  if (g > kPartialBlocks) g = kPartialBlocks;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

long long fidelity_cdf_len(long long n) { return n + (n + kScanBlock - 1) / kScanBlock; }

template <class R>
cudaError_t classical_fidelity_exact(long long n, const R* q, const R* P, const double* scal, double* partials,
                                     unsigned int* counter, double* out, cudaStream_t s) {
  k_fc_exact<R><<<grid_for(n), 256, 0, s>>>(q, P, n, scal, partials, counter, out);
  return cudaGetLastError();
}

template <class R>
cudaError_t classical_fidelity_sampled(long long n, const R* q, const R* P, long long samples,
                                       unsigned long long seed, const double* scal, double* cdf, double* partials,
                                       unsigned int* counter, double* out, cudaStream_t s) {
  const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
  double* tops = cdf + n;
  k_scan_local<R><<<nb, 256, 0, s>>>(q, n, scal, cdf, tops);
  k_scan_tops<<<1, 1024, 0, s>>>(tops, nb);
  k_scan_add<<<grid_for(n), 256, 0, s>>>(cdf, n, tops);
  k_fc_sample<R><<<grid_for(samples), 256, 0, s>>>(cdf, q, P, n, samples, seed, scal, partials, counter, out);
  return cudaGetLastError();
}

template cudaError_t classical_fidelity_exact<float>(long long, const float*, const float*, const double*, double*,
                                                     unsigned int*, double*, cudaStream_t);
template cudaError_t classical_fidelity_exact<double>(long long, const double*, const double*, const double*, double*,
                                                      unsigned int*, double*, cudaStream_t);
template cudaError_t classical_fidelity_sampled<float>(long long, const float*, const float*, long long,
                                                       unsigned long long, const double*, double*, double*,
                                                       unsigned int*, double*, cudaStream_t);
template cudaError_t classical_fidelity_sampled<double>(long long, const double*, const double*, long long,
                                                        unsigned long long, const double*, double*, double*,
                                                        unsigned int*, double*, cudaStream_t);

}  // namespace qst
