// Synthetic measurement data on the GPU (Sec. 4): the test states of the paper's sweeps and seeded
// multinomial counts of a probability vector (Sec. 4.5.1: "a certain number of samples from sampling a
// multinomial distribution of measurement probabilities").
//
// States: rho = w |psi><psi| + (1 - w) I / d for the product state ((|0> + |1>)/sqrt 2)^N, the GHZi state
// (|0..0> + i |1..1>)/sqrt 2 and the W state (equal superposition of the N one-excitation states); white
// noise uses w = p, the depolarising channel w = 1 - lambda.
//
// Counts: each probability becomes an integer weight w_k = floor(max(P_k, 0) 2^52) (P_k <= 1), so the
// running sums C_k are exact whatever the order of the scan.  Shot s takes z_s = splitmix64(seed, s)
// (SplitMix64, Steele, Lea and Flood, OOPSLA 2014: x = seed + (s + 1) 0x9E3779B97F4A7C15, then its
// published mix), t_s = floor((z_s >> 11) W / 2^53) with W = C_{n-1} (exact 128-bit product), and the
// outcome k_s = the smallest k with C_k > t_s; counts[k_s] += 1 (integer atomics: the counts do not depend
// on the order).  Every decision is integer arithmetic, so the counts are bit-exact and reproducible.
#include "../../include/qst.h"
#include "impl.h"
#include "rng.cuh"

namespace qst {

namespace {

constexpr int kPer = 8;
constexpr int kBlockElems = 256 * kPer;

template <class R>
__global__ void __launch_bounds__(256) k_test_state(cx_t<R>* __restrict__ rho, int N, int kind, double w) {
  const int d = 1 << N;
  const long long nn = (long long)d * d;
  const R s2 = (R)0.70710678118654752440;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    auto amp = [&](int k, R& re, R& im) {  // psi_k
      re = R(0);
      im = R(0);
      if (kind == QST_STATE_PRODUCT) {
        re = (R)(1.0 / sqrt((double)d));
      } else if (kind == QST_STATE_GHZI) {
        if (k == 0) re = s2;
        if (k == d - 1) im = s2;
      } else if (__popc(k) == 1) {  // W
        re = (R)(1.0 / sqrt((double)N));
      }
    };
    R ar, ai, br, bi;
    amp(i, ar, ai);
    amp(j, br, bi);
    // w psi_i conj(psi_j) + (1 - w) delta_ij / d
    R re = (R)w * (ar * br + ai * bi), im = (R)w * (ai * br - ar * bi);
    if (i == j) re += (R)((1.0 - w) / d);
    rho[e] = cmake<cx_t<R>>(re, im);
  }
}

// Integer weights and a block-local inclusive scan; block totals to tops.  A bad probability
// (not finite, or above 1) raises *bad.
__global__ void __launch_bounds__(256) k_weights_scan(const double* __restrict__ P, long long n,
                                                       unsigned long long* __restrict__ C,
                                                       unsigned long long* __restrict__ tops, unsigned int* bad) {
  __shared__ unsigned long long wsum[8];
  const long long base = (long long)blockIdx.x * kBlockElems + (long long)threadIdx.x * kPer;
  unsigned long long v[kPer];
  unsigned long long run = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const long long i = base + k;
    unsigned long long wk = 0;
    if (i < n) {
      const double p = P[i];
      if (!(p <= 1.0) || !isfinite(p)) atomicOr(bad, 1u);
      else if (p > 0.0) wk = (unsigned long long)(p * 4503599627370496.0);  // floor(p 2^52)
    }
    run += wk;
    v[k] = run;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  unsigned long long off = x - run;
  for (int w = 0; w < warp; ++w) off += wsum[w];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const long long i = base + k;
    if (i < n) C[i] = v[k] + off;
  }
  if (threadIdx.x == 255) tops[blockIdx.x] = off + run;
}

__global__ void __launch_bounds__(1024) k_tops_scan(unsigned long long* tops, int nb) {
  __shared__ unsigned long long wsum[32];
  const int per = (nb + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  unsigned long long run = 0;
  for (int b = b0; b < b0 + per && b < nb; ++b) run += tops[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  unsigned long long off = x - run;
  for (int w = 0; w < warp; ++w) off += wsum[w];
  for (int b = b0; b < b0 + per && b < nb; ++b) {
    const unsigned long long t = tops[b];
    tops[b] = off;
    off += t;
  }
}

__global__ void __launch_bounds__(256) k_add_tops(unsigned long long* __restrict__ C, long long n,
                                                   const unsigned long long* __restrict__ tops,
                                                   long long* __restrict__ counts) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    C[i] += tops[i / kBlockElems];
    counts[i] = 0;
  }
}

__global__ void __launch_bounds__(256) k_draw(const unsigned long long* __restrict__ C, long long n, long long shots,
                                               unsigned long long seed, long long* __restrict__ counts) {
  const unsigned long long W = C[n - 1];
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < shots; s += (long long)gridDim.x * blockDim.x) {
    const unsigned long long a = splitmix64(seed, (unsigned long long)s) >> 11;  // < 2^53
    const unsigned long long hi = __umul64hi(a, W), lo = a * W;
    const unsigned long long t = (hi << 11) | (lo >> 53);                         // floor(a W / 2^53) < W
    long long l = 0, h = n - 1;
    while (l < h) {
      const long long m = (l + h) >> 1;
      if (C[m] > t) h = m;
      else l = m + 1;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(counts + l), 1ull);
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_freq(const long long* __restrict__ counts, long long n, long long shots,
                                               R* __restrict__ f) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    f[i] = (R)((double)counts[i] / (double)shots);  // correctly rounded, as counts / shots on the host
}

int grid_of(long long work, int sms_mult = 8) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long g = (work + 255) / 256;
  const long long cap = (long long)sms * sms_mult;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

long long sampler_scratch_words(long long n) { return n + (n + kBlockElems - 1) / kBlockElems; }

template <class R> cudaError_t make_test_state(int N, int kind, double w, cx_t<R>* rho, cudaStream_t s) {
  const long long nn = 1LL << (2 * N);
  k_test_state<R><<<grid_of(nn), 256, 0, s>>>(rho, N, kind, w);
  return cudaGetLastError();
}

cudaError_t multinomial_prepare(long long n, const double* P, unsigned long long* scratch, long long* counts,
                                unsigned int* bad, cudaStream_t s) {
  const int nb = (int)((n + kBlockElems - 1) / kBlockElems);
  unsigned long long* C = scratch;
  unsigned long long* tops = scratch + n;
  k_weights_scan<<<nb, 256, 0, s>>>(P, n, C, tops, bad);
  k_tops_scan<<<1, 1024, 0, s>>>(tops, nb);
  k_add_tops<<<grid_of(n), 256, 0, s>>>(C, n, tops, counts);
  return cudaGetLastError();
}

cudaError_t multinomial_draw(long long n, long long shots, unsigned long long seed, const unsigned long long* scratch,
                             long long* counts, cudaStream_t s) {
  if (shots > 0) k_draw<<<grid_of(shots), 256, 0, s>>>(scratch, n, shots, seed, counts);
  return cudaGetLastError();
}

template <class R> cudaError_t counts_to_frequencies(long long n, const long long* counts, long long shots, R* f,
                                                     cudaStream_t s) {
  k_freq<R><<<grid_of(n), 256, 0, s>>>(counts, n, shots, f);
  return cudaGetLastError();
}

template cudaError_t make_test_state<float>(int, int, double, cx_t<float>*, cudaStream_t);
template cudaError_t make_test_state<double>(int, int, double, cx_t<double>*, cudaStream_t);
template cudaError_t counts_to_frequencies<float>(long long, const long long*, long long, float*, cudaStream_t);
template cudaError_t counts_to_frequencies<double>(long long, const long long*, long long, double*, cudaStream_t);

}  // namespace qst
