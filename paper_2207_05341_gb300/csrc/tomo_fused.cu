// One whole iteration of the Fig. 1 loop for a small tomography in one CTA, and many tomographies of
// uneven sizes in one persistent launch (FP32, Chol_H state map, the 3-layer network of Sec. 3.1).
//
// For N <= 7 every step of an iteration is too small to fill the GPU on its own: a CTA takes one
// tomography and runs, separated by block barriers,
//   S2  t = W2 h + b2                                   (Sec. 3.1, linear output layer)
//   S3  T from t (R = t as d x d: T_ii = R_ii, T_ij = R_ij + i R_ji (i > j), T_ji = conj T_ij)
//   S4  X = T T, Tr X                                   (Sec. 3.2 eq. unified_DP)
//   S5  q = the product-POVM map of X, in place         (Sec. 3.3 eq. PS, one 4 x 4 mode map per qubit)
//   S6  L = -sum f log q + (sum f) log Tr X, g = dL/dq  (Sec. 3.1; the clamp of q below the smallest
//                                                        normal number as in povm.cu)
//   S7  G = sum_k g_k M_k, in place                     (the transposed mode maps)
//   S8  Y = G T, dL/dt from Y + Y^dag
//   S9  Rprop on W2^T, b2 (dh from the old weights), b1; Rprop on W1 and the next hidden layer
//       pre = W1' f + b1', h = LeakyReLU(pre), sum f    (Sec. 4.1)
// on the context's own buffers (T, X, G, Y, t = dt), with the same arithmetic for every placement of
// the tomography, so that a batch and a single context give bit-identical iterations.  The persistent
// kernel takes tomographies from a work list (largest first) through an atomic counter: ragged sizes in
// one launch.  Every sum runs in a fixed order (per-thread partial sums, then a fixed tree).
#include <float.h>

#include "impl.h"
#include "tuned.h"

namespace qst {

namespace {

constexpr int kFT = 32;          // GEMM tile (complex elements)
constexpr int kGroup = 256;      // threads per GEMM group
static_assert(kFusedThreads % kGroup == 0 && kFusedThreads <= 512, "fused step: 256 or 512 threads");

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

struct Smem {
  float2 A[2][kFT][kFT + 1];  // one A and B tile per GEMM group (blockDim <= 512)
  float2 B[2][kFT][kFT + 1];
  float vec[64];              // hidden layer / dh / dpre (H <= 14)
  double red[32 * 16];        // block reductions: 32 warps x up to 16 values
};

// Sums of the per-thread values v[0 .. M) over the block, in a fixed order; the totals are left in
// red[kTot + j] (read them before the next reduction).
constexpr int kTot = 31 * 16;
template <int M> __device__ void block_sum(const float (&v)[M], double* red) {
  static_assert(M <= 16, "at most 16 values per reduction");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const double s = warp_sum((double)v[j]);
    if (lane == 0) red[warp * 16 + j] = s;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * 16 + threadIdx.x];
    red[kTot + threadIdx.x] = s;  // warps <= 16 leave the last row free
  }
  __syncthreads();
}

__device__ double block_sum1(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

// C = A B, d x d complex row-major (global), by the whole block: groups of 256 threads take 32 x 32
// output tiles in turn, each thread a 2 x 2 block of one; tiles of TS = min(d, 32).
__device__ void block_cgemm(const float2* A, const float2* B, float2* C, int d, Smem& sm) {
  const int grp = threadIdx.x / kGroup, gt = threadIdx.x % kGroup, ngrp = (int)(blockDim.x / kGroup);
  const int TS = d < kFT ? d : kFT, nt = d / TS, tiles = nt * nt;
  const int ty = gt >> 4, tx = gt & 15;
  const bool act = 2 * ty < TS && 2 * tx < TS;
  const int rounds = (tiles + ngrp - 1) / ngrp;
  for (int rd = 0; rd < rounds; ++rd) {
    const int tile = rd * ngrp + grp;
    const bool have = tile < tiles;
    const int I = have ? tile / nt : 0, J = have ? tile % nt : 0;
    float2 acc[2][2] = {{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}};
    for (int k0 = 0; k0 < d; k0 += TS) {
      if (have) {
        for (int e = gt; e < TS * TS; e += kGroup) {
          const int r = e / TS, c = e % TS;
          sm.A[grp][r][c] = A[(long long)(I * TS + r) * d + k0 + c];
          sm.B[grp][r][c] = B[(long long)(k0 + r) * d + J * TS + c];
        }
      }
      __syncthreads();
      if (have && act) {
        for (int kk = 0; kk < TS; ++kk) {
          const float2 a0 = sm.A[grp][2 * ty][kk], a1 = sm.A[grp][2 * ty + 1][kk];
          const float2 b0 = sm.B[grp][kk][2 * tx], b1 = sm.B[grp][kk][2 * tx + 1];
          cmac(acc[0][0], a0, b0);
          cmac(acc[0][1], a0, b1);
          cmac(acc[1][0], a1, b0);
          cmac(acc[1][1], a1, b1);
        }
      }
      __syncthreads();
    }
    if (have && act) {
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) C[(long long)(I * TS + 2 * ty + u) * d + J * TS + 2 * tx + v] = acc[u][v];
    }
  }
  __syncthreads();
}

// The 4 x 4 mode maps of every qubit on a d x d complex matrix in place (global, whole block).
template <bool ADJ> __device__ void block_modes(float2* X, int N, const PovmB<float>& Bm) {
  const int d = 1 << N, half = d >> 1;
  for (int b = 0; b < N; ++b) {
    const int bit = 1 << b, low = bit - 1;
    for (int blk = threadIdx.x; blk < half * half; blk += blockDim.x) {
      const int rr = blk / half, cc = blk % half;
      const int r0 = ((rr & ~low) << 1) | (rr & low), c0 = ((cc & ~low) << 1) | (cc & low);
      float2* p00 = X + (long long)r0 * d + c0;
      float2 x00 = p00[0], x01 = p00[bit], x10 = p00[(long long)bit * d], x11 = p00[(long long)bit * d + bit];
      if (ADJ) mode_adj(Bm, x00, x01, x10, x11);
      else mode_fwd(Bm, x00, x01, x10, x11);
      p00[0] = x00; p00[bit] = x01; p00[(long long)bit * d] = x10; p00[(long long)bit * d + bit] = x11;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ float leaky_f(float p, float slope) { return p > 0.f ? p : slope * p; }

// One iteration for tomography `td`.
__device__ void tomo_iteration(const TomoDesc& td, const PovmB<float>& Bm, const NetCfg& cfg, Smem& sm) {
  const int N = td.N, d = 1 << N, H = 2 * N;
  const long long n = 1LL << (2 * N);
  const long long o2 = (long long)H * n, ob2 = 2LL * H * n, ob1 = 2LL * H * n + n;
  float* theta = td.theta;
  float* step = td.step;
  const float* f = td.f;
  float* t = td.t;
  float2 *T = td.T, *X = td.X, *G = td.G, *Y = td.Y;
  const RpropCfg<float> rc{(float)cfg.eta_minus, (float)cfg.eta_plus, (float)cfg.step_min, (float)cfg.step_max};
  const float slope = (float)cfg.slope;
  const int tid = threadIdx.x, nth = blockDim.x;

  if (tid < H) sm.vec[tid] = td.hid[tid];
  __syncthreads();
  // S2: t = W2 h + b2
  for (long long i = tid; i < n; i += nth) {
    float a = theta[ob2 + i];
    for (int j = 0; j < H; ++j) a = fmaf(theta[o2 + (long long)j * n + i], sm.vec[j], a);
    t[i] = a;
  }
  __syncthreads();
  // S3: the Hermitian T of R = t
  for (long long e = tid; e < n; e += nth) {
    const int i = (int)(e >> N), j = (int)(e & (d - 1));
    float re, im;
    if (i > j) { re = t[e]; im = t[(long long)j * d + i]; }
    else if (i < j) { re = t[(long long)j * d + i]; im = -t[e]; }
    else { re = t[e]; im = 0.f; }
    T[e] = make_float2(re, im);
  }
  __syncthreads();
  // S4: X = T T and its trace
  block_cgemm(T, T, X, d, sm);
  double tr = 0.0;
  for (int i = tid; i < d; i += nth) tr += (double)X[(long long)i * d + i].x;
  const double tX = block_sum1(tr, sm.red);
  // S5: q in place; slot (i, j) then holds the outcome k = interleave(i, j)
  block_modes<false>(X, N, Bm);
  // S6: likelihood, and g = dL/dq into G
  const double sumf = td.scal[1];
  const float gconst = (float)(sumf / tX);
  double acc = 0.0;
  unsigned int nclamp = 0;
  for (long long e = tid; e < n; e += nth) {
    const uint32_t i = (uint32_t)(e >> N), j = (uint32_t)(e & (d - 1));
    const float q = X[e].x;
    const float fk = f[interleave_ij(i, j)];
    float gk = gconst;
    if (fk > 0.f) {
      if (!(q >= FLT_MIN)) {  // clamped: the constant -f_k log q_min, nothing added to dL/dq_k
        ++nclamp;
        acc += (double)fk * (double)logf(FLT_MIN);
      } else {
        acc += (double)fk * (double)logf(q);
        gk -= fk / q;
      }
    }
    G[e] = make_float2(gk, 0.f);
  }
  if (nclamp) atomicAdd(td.flags, nclamp);
  const double ll = block_sum1(acc, sm.red);
  if (tid == 0) {
    td.scal[0] = tX;
    td.scal[2] = -ll + sumf * log(tX);
  }
  __syncthreads();
  // S7: G = sum_k g_k M_k in place
  block_modes<true>(G, N, Bm);
  // S8: Y = G T, then dL/dt: (a, b) below the diagonal 2 (Re Y_ab + Re Y_ba), above 2 (Im Y_ba - Im Y_ab)
  block_cgemm(G, T, Y, d, sm);
  for (long long e = tid; e < n; e += nth) {
    const int a = (int)(e >> N), b = (int)(e & (d - 1));
    const float2 yab = Y[e], yba = Y[(long long)b * d + a];
    t[e] = a > b ? 2.f * (yab.x + yba.x) : (a < b ? 2.f * (yba.y - yab.y) : 2.f * yab.x);
  }
  __syncthreads();
  // S9, layer 2: Rprop on b2 (g = dt) and W2^T (g = h_j dt_i); dh_j from the old weights
  float dh[14];
#pragma unroll
  for (int j = 0; j < 14; ++j) dh[j] = 0.f;
  for (long long i = tid; i < n; i += nth) {
    const float dv = t[i];
    {
      float st = step[ob2 + i];
      theta[ob2 + i] = rprop1(theta[ob2 + i], dv, st, rc);
      step[ob2 + i] = st;
    }
#pragma unroll
    for (int j = 0; j < 14; ++j) {
      if (j >= H) break;
      const long long o = o2 + (long long)j * n + i;
      const float w = theta[o];
      dh[j] = fmaf(w, dv, dh[j]);
      float st = step[o];
      theta[o] = rprop1(w, sm.vec[j] * dv, st, rc);
      step[o] = st;
    }
  }
  block_sum<14>(dh, sm.red);
  // dpre = dh LeakyReLU'(pre); Rprop on b1 (g = dpre)
  if (tid < H) {
    const float p = td.pre[tid];
    const float dp = (float)sm.red[kTot + tid] * (p > 0.f ? 1.f : slope);
    sm.vec[32 + tid] = dp;
    float st = step[ob1 + tid];
    theta[ob1 + tid] = rprop1(theta[ob1 + tid], dp, st, rc);
    step[ob1 + tid] = st;
  }
  __syncthreads();
  // S9, layer 1: Rprop on W1 (g = dpre_j f_i), then the next hidden layer from the new W1 and b1
  float pa[15];
#pragma unroll
  for (int j = 0; j < 15; ++j) pa[j] = 0.f;
  for (long long i = tid; i < n; i += nth) {
    const float fv = f[i];
    pa[14] += fv;
#pragma unroll
    for (int j = 0; j < 14; ++j) {
      if (j >= H) break;
      const long long o = (long long)j * n + i;
      float st = step[o];
      const float w = rprop1(theta[o], sm.vec[32 + j] * fv, st, rc);
      theta[o] = w;
      step[o] = st;
      pa[j] = fmaf(w, fv, pa[j]);
    }
  }
  // the sum of f rides as value 14 of the reduction
  block_sum<15>(pa, sm.red);
  if (tid < H) {
    const float p = (float)(sm.red[kTot + tid] + (double)theta[ob1 + tid]);
    td.pre[tid] = p;
    td.hid[tid] = leaky_f(p, slope);
  }
  if (tid == 0) td.scal[1] = sm.red[kTot + 14];
  __syncthreads();
}

// Persistent CTAs over a work list (list != NULL: count entries, taken in turn through *next), or the
// single tomography `one`.  Both run the same code on a shared-memory copy of the descriptor.
__global__ void __launch_bounds__(kFusedThreads, kFusedCtasPerSmMax) k_tomo(const TomoDesc* __restrict__ list, int count, TomoDesc one,
                                                         PovmB<float> Bm, NetCfg cfg, unsigned int* next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  __shared__ TomoDesc s_td;
  __shared__ int s_item;
  for (int round = 0;; ++round) {
    if (threadIdx.x == 0) {
      const int item = list ? (int)atomicAdd(next, 1u) : round;
      s_item = item;
      if (item < count) s_td = list ? list[item] : one;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= count) break;
    tomo_iteration(s_td, Bm, cfg, sm);
  }
}

}  // namespace

bool tomo_fused_ok(int N, int max_qubits) {
  const int m = max_qubits == 0 ? tuning().fused_max_qubits : max_qubits;
  return N >= 1 && N <= m && N <= kFusedMaxQubits;
}

cudaError_t tomo_fused_one(const TomoDesc& td, const PovmB<float>& B, const NetCfg& cfg, cudaStream_t s) {
  const size_t smem = sizeof(Smem);
  cudaError_t e = ensure_dynamic_smem((const void*)k_tomo, smem);
  if (e != cudaSuccess) return e;
  k_tomo<<<1, kFusedThreads, smem, s>>>(nullptr, 1, td, B, cfg, nullptr);
  return cudaGetLastError();
}

cudaError_t tomo_fused_list(const TomoDesc* list, int count, const PovmB<float>& B, const NetCfg& cfg,
                            unsigned int* next, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = sizeof(Smem);
  cudaError_t e = ensure_dynamic_smem((const void*)k_tomo, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tomo, kFusedThreads, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) per_sm = 1;
  const int cap = tuning().fused_ctas_per_sm;
  if (per_sm > cap) per_sm = cap;
  const int ctas = count < sms * per_sm ? count : sms * per_sm;
  if ((e = cudaMemsetAsync(next, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
  k_tomo<<<ctas, kFusedThreads, smem, s>>>(list, count, TomoDesc{}, B, cfg, next);
  return cudaGetLastError();
}

}  // namespace qst
