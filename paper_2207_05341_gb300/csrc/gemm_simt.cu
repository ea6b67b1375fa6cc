// Complex d x d products on the CUDA cores (the plain FP32 and FP64 paths):
//   X = T T   (Sec. 3.2 eq. unified_DP, Hermitian: only tiles I >= J are computed)
//   Y = G T   (backward of X = T T)
// Row-major complex operands.  Classic register-blocked tiling: a CTA computes a
// BM x BN tile, each thread a TM x TN block; the next K slice is prefetched into
// registers while the current one is multiplied.  Shared-memory layout: A is
// stored transposed with rows of BM + 4 entries, so that the stores of a warp
// (8 k by 4 m) fall in distinct bank groups; a thread's TN columns of B are
// 16-byte chunks (CW complex each) spaced by the chunks of the other threads of
// its row, so that the 16 threads of a row read consecutive chunks.
#include "impl.h"

namespace qst {

template <class R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_cgemm(int d, const cx_t<R>* __restrict__ A,
                                                                 const cx_t<R>* __restrict__ B,
                                                                 cx_t<R>* __restrict__ C, int lower,
                                                                 const void* const* tab) {
  using V = cx_t<R>;
  rebind(tab, A, B, C);
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  constexpr int LA = BM * BK / NT, LB = BK * BN / NT;
  constexpr int PAD = 4;
  constexpr int CW = 16 / (int)sizeof(V);  // complex entries per 16-byte chunk
  static_assert(TN % CW == 0, "a thread's columns are whole 16-byte chunks");
  static_assert(LA >= 1 && LB >= 1, "tile too small for the thread count");
  __shared__ __align__(16) V As[2][BK][BM + PAD];
  __shared__ __align__(16) V Bs[2][BK][BN + PAD];

  int I, J;
  if (lower) tri_decode(blockIdx.x, I, J);
  else { I = blockIdx.y; J = blockIdx.x; }
  const int m0 = I * BM, n0 = J * BN;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;

  V ra[LA], rb[LB];
  auto gload = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      const int m = e / BK, kk = e % BK;
      ra[l] = A[(long long)(m0 + m) * d + k0 + kk];
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      const int kk = e / BN, nn = e % BN;
      rb[l] = B[(long long)(k0 + kk) * d + n0 + nn];
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      As[buf][e % BK][e / BK] = ra[l];
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      Bs[buf][e / BN][e % BN] = rb[l];
    }
  };

  R accr[TM][TN], acci[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) { accr[i][j] = R(0); acci[i][j] = R(0); }

  const int nk = d / BK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) gload((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      V a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM / 2; ++i) {
        a[i] = As[buf][k][ty * (TM / 2) + i];
        a[TM / 2 + i] = As[buf][k][BM / 2 + ty * (TM / 2) + i];
      }
#pragma unroll
      for (int g = 0; g < TN / CW; ++g)
#pragma unroll
        for (int j = 0; j < CW; ++j) b[g * CW + j] = Bs[buf][k][g * (NTX * CW) + tx * CW + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          accr[i][j] = fma(a[i].x, b[j].x, accr[i][j]);
          accr[i][j] = fma(-a[i].y, b[j].y, accr[i][j]);
          acci[i][j] = fma(a[i].x, b[j].y, acci[i][j]);
          acci[i][j] = fma(a[i].y, b[j].x, acci[i][j]);
        }
    }
    if (kt + 1 < nk) {
      sstore(buf ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + (i < TM / 2 ? ty * (TM / 2) + i : BM / 2 + ty * (TM / 2) + (i - TM / 2));
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int nn = n0 + (j / CW) * (NTX * CW) + tx * CW + j % CW;
      C[(long long)m * d + nn] = cmake<V>(accr[i][j], acci[i][j]);
    }
  }
}

// Small matrices (d <= 16): one thread per output element.
template <class R>
__global__ void k_cgemm_small(int d, const cx_t<R>* A, const cx_t<R>* B, cx_t<R>* C, int lower) {
  using V = cx_t<R>;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < d * d; e += blockDim.x * gridDim.x) {
    const int m = e / d, nn = e % d;
    R sr = R(0), si = R(0);
    for (int k = 0; k < d; ++k) {
      const V a = A[m * d + k], b = B[k * d + nn];
      sr = fma(a.x, b.x, sr); sr = fma(-a.y, b.y, sr);
      si = fma(a.x, b.y, si); si = fma(a.y, b.x, si);
    }
    C[e] = cmake<V>(sr, si);
  }
}

template <class R, int BM, int BN, int BK, int TM, int TN>
static cudaError_t run_tiled(int d, const cx_t<R>* A, const cx_t<R>* B, cx_t<R>* C, bool lower, cudaStream_t s) {
  constexpr int NT = (BM / TM) * (BN / TN);
  const int nt = d / BM;
  BatchArgs ba;
  if (batch_take(ba, {A, B, C})) return cudaSuccess;
  if (lower) {
    k_cgemm<R, BM, BN, BK, TM, TN><<<dim3((unsigned)(nt * (nt + 1) / 2), 1, ba.nz), NT, 0, s>>>(d, A, B, C, 1, ba.tab);
  } else {
    k_cgemm<R, BM, BN, BK, TM, TN><<<dim3(d / BN, d / BM, ba.nz), NT, 0, s>>>(d, A, B, C, 0, ba.tab);
  }
  return cudaGetLastError();
}

template <>
cudaError_t cgemm_simt<float>(int d, const float2* A, const float2* B, float2* C, bool lower, cudaStream_t s) {
  if (d >= 128) return run_tiled<float, 128, 128, 8, 8, 8>(d, A, B, C, lower, s);
  if (d == 64) return run_tiled<float, 64, 64, 8, 4, 4>(d, A, B, C, lower, s);
  if (d == 32) return run_tiled<float, 32, 32, 8, 2, 2>(d, A, B, C, lower, s);
  k_cgemm_small<float><<<1, 256, 0, s>>>(d, A, B, C, lower ? 1 : 0);
  return cudaGetLastError();
}

template <>
cudaError_t cgemm_simt<double>(int d, const double2* A, const double2* B, double2* C, bool lower, cudaStream_t s) {
  if (d >= 64) return run_tiled<double, 64, 64, 8, 4, 4>(d, A, B, C, lower, s);
  if (d == 32) return run_tiled<double, 32, 32, 8, 2, 2>(d, A, B, C, lower, s);
  k_cgemm_small<double><<<1, 256, 0, s>>>(d, A, B, C, lower ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace qst
