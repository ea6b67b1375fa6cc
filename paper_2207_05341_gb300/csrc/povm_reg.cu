// Second pass of the product-POVM map (Sec. 3.3 eq. PS) over the high h qubits, with the
// likelihood and the adjoint fused in (see povm.cu for the two-pass scheme).
//
// For a fixed low outcome a_lo the packed intermediate is an nb x nb Hermitian matrix
// (nb = 2^h <= 32).  Here one warp holds G = 32 / nb such matrices, one row per lane
// (lane = sub * nb + i_h), as nb complex registers.  A qubit's mode map mixes the
// index pair (i_b, j_b): the column bit j_b pairs registers of a lane, the row bit
// i_b pairs lanes i_h and i_h ^ 2^b, which exchange the two values with a warp
// shuffle; each lane then computes only the two outputs of its own row.  Shared
// memory is used only to turn the strided global accesses (one float per
// (pair, a_lo)) into coalesced 32-byte segments: W and f are staged in, q or the
// packed adjoint are staged out.
#include <float.h>

#include "impl.h"

namespace qst {

namespace {

template <class T> __device__ __forceinline__ T min_norm();
template <> __device__ __forceinline__ float min_norm<float>() { return FLT_MIN; }
template <> __device__ __forceinline__ double min_norm<double>() { return DBL_MIN; }

template <class V> __device__ __forceinline__ V shfl_x(V v, int m) {
  V r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return r;
}

// Forward mode map of qubit BIT on register rows (see mode_fwd in common.cuh).
template <class R, int NB, int BIT>
__device__ __forceinline__ void fwd_bit(cx_t<R> (&x)[NB], const PovmB<R>& B, int ih) {
  using V = cx_t<R>;
  const bool up = (ih >> BIT) & 1;
  R p0[4], p1[4];  // coefficients of this row's two outputs a = 2 up and 2 up + 1
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    p0[m] = up ? B.b[2][m] : B.b[0][m];
    p1[m] = up ? B.b[3][m] : B.b[1][m];
  }
#pragma unroll
  for (int j0 = 0; j0 < NB; ++j0) {
    if (j0 & (1 << BIT)) continue;
    const int j1 = j0 | (1 << BIT);
    const V m0 = x[j0], m1 = x[j1];
    const V o0 = shfl_x(m0, 1 << BIT), o1 = shfl_x(m1, 1 << BIT);
    const V x00 = up ? o0 : m0, x01 = up ? o1 : m1, x10 = up ? m0 : o0, x11 = up ? m1 : o1;
    const V c0 = cadd(x00, x11), c3 = csub(x00, x11), c1 = cadd(x01, x10), c2 = cmuli(csub(x01, x10));
    x[j0].x = p0[0] * c0.x + p0[1] * c1.x + p0[2] * c2.x + p0[3] * c3.x;
    x[j0].y = p0[0] * c0.y + p0[1] * c1.y + p0[2] * c2.y + p0[3] * c3.y;
    x[j1].x = p1[0] * c0.x + p1[1] * c1.x + p1[2] * c2.x + p1[3] * c3.x;
    x[j1].y = p1[0] * c0.y + p1[1] * c1.y + p1[2] * c2.y + p1[3] * c3.y;
  }
}

// Adjoint mode map of qubit BIT (see mode_adj in common.cuh).
template <class R, int NB, int BIT>
__device__ __forceinline__ void adj_bit(cx_t<R> (&x)[NB], const PovmB<R>& B, int ih) {
  using V = cx_t<R>;
  const bool up = (ih >> BIT) & 1;
#pragma unroll
  for (int j0 = 0; j0 < NB; ++j0) {
    if (j0 & (1 << BIT)) continue;
    const int j1 = j0 | (1 << BIT);
    const V m0 = x[j0], m1 = x[j1];
    const V o0 = shfl_x(m0, 1 << BIT), o1 = shfl_x(m1, 1 << BIT);
    V g[4];
    g[0] = up ? o0 : m0; g[1] = up ? o1 : m1; g[2] = up ? m0 : o0; g[3] = up ? m1 : o1;
    V c[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      c[mu].x = B.b[0][mu] * g[0].x + B.b[1][mu] * g[1].x + B.b[2][mu] * g[2].x + B.b[3][mu] * g[3].x;
      c[mu].y = B.b[0][mu] * g[0].y + B.b[1][mu] * g[1].y + B.b[2][mu] * g[2].y + B.b[3][mu] * g[3].y;
    }
    const V ic2 = cmuli(c[2]);
    if (up) {  // row 1: x10 = c1 + i c2, x11 = c0 - c3
      x[j0] = cadd(c[1], ic2);
      x[j1] = csub(c[0], c[3]);
    } else {   // row 0: x00 = c0 + c3, x01 = c1 - i c2
      x[j0] = cadd(c[0], c[3]);
      x[j1] = csub(c[1], ic2);
    }
  }
}

template <class R, int NB>
__device__ __forceinline__ void fwd_all(cx_t<R> (&x)[NB], const PovmB<R>& B, int ih) {
  if constexpr (NB > 1) fwd_bit<R, NB, 0>(x, B, ih);
  if constexpr (NB > 2) fwd_bit<R, NB, 1>(x, B, ih);
  if constexpr (NB > 4) fwd_bit<R, NB, 2>(x, B, ih);
  if constexpr (NB > 8) fwd_bit<R, NB, 3>(x, B, ih);
  if constexpr (NB > 16) fwd_bit<R, NB, 4>(x, B, ih);
}

template <class R, int NB>
__device__ __forceinline__ void adj_all(cx_t<R> (&x)[NB], const PovmB<R>& B, int ih) {
  if constexpr (NB > 1) adj_bit<R, NB, 0>(x, B, ih);
  if constexpr (NB > 2) adj_bit<R, NB, 1>(x, B, ih);
  if constexpr (NB > 4) adj_bit<R, NB, 2>(x, B, ih);
  if constexpr (NB > 8) adj_bit<R, NB, 3>(x, B, ih);
  if constexpr (NB > 16) adj_bit<R, NB, 4>(x, B, ih);
}

template <int NB> struct Geo {
  static constexpr int G = 32 / NB;           // low outcomes per warp
  static constexpr int CB = 8 * G;            // low outcomes per block (8 warps)
  static constexpr int PITCH = NB * CB + 1;   // padded row pitch of the staging array
  static constexpr int RAW = NB * PITCH;      // staging array (reals)
  static constexpr int FS = NB * NB * CB;     // staged f (reals)
};

// MODE 0: forward only, write q to p.  MODE 1: likelihood (+ adjoint when adjoint != 0).
template <class R, int NB, int MODE>
__global__ void __launch_bounds__(256) k_povm_hi_reg(const R* __restrict__ W, R* __restrict__ p,
                                                      const R* __restrict__ f, double* scal, R* __restrict__ Wadj,
                                                      double* partials, unsigned int* counter, unsigned int* flags,
                                                      int g, PovmB<R> B, int adjoint) {
  using V = cx_t<R>;
  using Gm = Geo<NB>;
  constexpr int CB = Gm::CB, PITCH = Gm::PITCH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* raw = reinterpret_cast<R*>(smem_raw);
  R* fs = raw + Gm::RAW;
  __shared__ double red[8];
  const long long SS = 1LL << (2 * g);
  const long long al0 = (long long)blockIdx.x * CB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ih = lane % NB, c = warp * Gm::G + lane / NB;

  for (int t = tid; t < NB * NB * CB; t += blockDim.x) {
    const int cc = t % CB, pair = t / CB;
    raw[(pair / NB) * PITCH + (pair % NB) * CB + cc] = W[(long long)pair * SS + al0 + cc];
    if (MODE == 1) fs[t] = f[(long long)pair * SS + al0 + cc];  // ah == pair here
  }
  __syncthreads();
  V x[NB];
#pragma unroll
  for (int jh = 0; jh < NB; ++jh) {
    const R a = raw[ih * PITCH + jh * CB + c];
    const R b = raw[jh * PITCH + ih * CB + c];
    x[jh] = ih == jh ? cmake<V>(a, R(0)) : (ih > jh ? cmake<V>(a, b) : cmake<V>(b, -a));
  }
  fwd_all<R, NB>(x, B, ih);
  __syncthreads();  // staging array reused below

  if (MODE == 0) {
#pragma unroll
    for (int jh = 0; jh < NB; ++jh) raw[interleave_ij(ih, jh) * CB + c] = x[jh].x;
    __syncthreads();
    for (int t = tid; t < NB * NB * CB; t += blockDim.x) {
      const int cc = t % CB, ah = t / CB;
      p[(long long)ah * SS + al0 + cc] = raw[t];
    }
    return;
  }

  // L = -sum f log q + (sum f) log Tr X;  g_k = -f_k / q_k + sum f / Tr X
  const double tX = scal[0], sumf = scal[1];
  const R gconst = (R)(sumf / tX);
  const R qmin = min_norm<R>();
  R accr = R(0);  // a lane's NB terms in R (FP64 arithmetic is a slow pipe on this part); lanes and blocks in FP64
  unsigned int nclamp = 0;
#pragma unroll
  for (int jh = 0; jh < NB; ++jh) {
    R q = x[jh].x;
    const R fk = fs[interleave_ij(ih, jh) * CB + c];
    R gk = gconst;
    if (fk > R(0)) {
      if (!(q >= qmin)) { q = qmin; ++nclamp; }
      accr += fk * log(q);
      gk -= fk / q;
    }
    x[jh] = cmake<V>(gk, R(0));
  }
  if (nclamp) atomicAdd(flags, nclamp);
  double acc = warp_sum((double)accr);
  if (lane == 0) red[warp] = acc;
  if (adjoint) {
    adj_all<R, NB>(x, B, ih);
    // packed Hermitian output: Re at [i][j], Im at [j][i] for i > j, Re on the diagonal
#pragma unroll
    for (int jh = 0; jh < NB; ++jh) {
      if (jh <= ih) raw[ih * PITCH + jh * CB + c] = x[jh].x;
      if (jh < ih) raw[jh * PITCH + ih * CB + c] = x[jh].y;
    }
  }
  __syncthreads();
  if (tid < 32) {
    double v = tid < 8 ? red[tid] : 0.0;
    v = warp_sum(v);
    if (tid == 0) partials[blockIdx.x] = v;
  }
  if (adjoint) {
    for (int t = tid; t < NB * NB * CB; t += blockDim.x) {
      const int cc = t % CB, pair = t / CB;
      Wadj[(long long)pair * SS + al0 + cc] = raw[(pair / NB) * PITCH + (pair % NB) * CB + cc];
    }
  }
  if (last_block_arrived(counter)) {
    if (threadIdx.x < 32) {
      double v = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) v += partials[b];
      v = warp_sum(v);
      if (threadIdx.x == 0) {
        scal[2] = -v + sumf * log(tX);
        *counter = 0u;
      }
    }
  }
}

template <class R, int NB, int MODE>
cudaError_t launch_reg(const Dims& D, const R* W, R* p, const R* f, double* scal, R* Wadj, double* partials,
                       unsigned int* counter, unsigned int* flags, const PovmB<R>& B, bool adjoint, cudaStream_t s) {
  using Gm = Geo<NB>;
  const size_t sm = (size_t)(Gm::RAW + (MODE == 1 ? Gm::FS : 0)) * sizeof(R);
  cudaError_t e = ensure_dynamic_smem((const void*)k_povm_hi_reg<R, NB, MODE>, sm);
  if (e != cudaSuccess) return e;
  const long long SS = 1LL << (2 * D.g);
  const unsigned blocks = (unsigned)(SS / Gm::CB);
  k_povm_hi_reg<R, NB, MODE><<<blocks, 256, sm, s>>>(W, p, f, scal, Wadj, partials, counter, flags, D.g, B,
                                                     adjoint ? 1 : 0);
  return cudaGetLastError();
}

template <class R, int MODE>
cudaError_t dispatch_reg(const Dims& D, const R* W, R* p, const R* f, double* scal, R* Wadj, double* partials,
                         unsigned int* counter, unsigned int* flags, const PovmB<R>& B, bool adjoint, cudaStream_t s) {
  switch (D.nb) {
    case 2: return launch_reg<R, 2, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 4: return launch_reg<R, 4, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 8: return launch_reg<R, 8, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 16: return launch_reg<R, 16, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 32: return launch_reg<R, 32, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool povm_hi_reg_ok(const Dims& D) { return D.nb >= 2 && D.nb <= 32 && D.g >= 6; }

template <class R>
cudaError_t povm_hi_fwd_reg(const Dims& D, const R* W, R* p, const PovmB<R>& B, cudaStream_t s) {
  return dispatch_reg<R, 0>(D, W, p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, B, false, s);
}

template <class R>
cudaError_t povm_hi_nll_reg(const Dims& D, const R* W, const R* f, double* scal, R* Wadj, double* partials,
                            unsigned int* counter, unsigned int* flags, const PovmB<R>& B, bool adjoint,
                            cudaStream_t s) {
  return dispatch_reg<R, 1>(D, W, nullptr, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
}

template cudaError_t povm_hi_fwd_reg<float>(const Dims&, const float*, float*, const PovmB<float>&, cudaStream_t);
template cudaError_t povm_hi_fwd_reg<double>(const Dims&, const double*, double*, const PovmB<double>&, cudaStream_t);
template cudaError_t povm_hi_nll_reg<float>(const Dims&, const float*, const float*, double*, float*, double*,
                                            unsigned int*, unsigned int*, const PovmB<float>&, bool, cudaStream_t);
template cudaError_t povm_hi_nll_reg<double>(const Dims&, const double*, const double*, double*, double*, double*,
                                             unsigned int*, unsigned int*, const PovmB<double>&, bool, cudaStream_t);

}  // namespace qst
