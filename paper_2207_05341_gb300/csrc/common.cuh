// Shared device helpers of libqst: complex arithmetic, the single-qubit POVM
// mode maps, Rprop, block reductions.  Included by every .cu of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qst {

template <class R> struct Cx;
template <> struct Cx<float>  { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <class R> using cx_t = typename Cx<R>::T;

template <class V> __host__ __device__ __forceinline__ V cmake(decltype(V::x) re, decltype(V::x) im) {
  V v; v.x = re; v.y = im; return v;
}
template <class V> __device__ __forceinline__ V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <class V> __device__ __forceinline__ V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }
template <class V> __device__ __forceinline__ V cconj(V a) { return cmake<V>(a.x, -a.y); }
// i * a
template <class V> __device__ __forceinline__ V cmuli(V a) { return cmake<V>(-a.y, a.x); }
template <class V, class R> __device__ __forceinline__ V cscale(V a, R s) { return cmake<V>(a.x * s, a.y * s); }

// Single-qubit POVM in Pauli form: M_a = b[a][0] I + b[a][1] X + b[a][2] Y + b[a][3] Z
// (every Hermitian 2x2 matrix has real coefficients in this basis).
template <class R> struct PovmB { R b[4][4]; };

// Forward mode map on one qubit (Sec. 3.3 eq. PS, Born rule of Sec. 2.1):
//   y_a = sum_{ij} (M_a)_{ji} x_{ij} = sum_mu b[a][mu] c_mu
// with the Pauli components c = (x00 + x11, x01 + x10, i(x01 - x10), x00 - x11).
// Output a is written back to the slot of (i, j) = (a >> 1, a & 1).
template <class R, class V>
__device__ __forceinline__ void mode_fwd(const PovmB<R>& B, V& x00, V& x01, V& x10, V& x11) {
  V c0 = cadd(x00, x11), c3 = csub(x00, x11), c1 = cadd(x01, x10), c2 = cmuli(csub(x01, x10));
  V y[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    y[a].x = B.b[a][0] * c0.x + B.b[a][1] * c1.x + B.b[a][2] * c2.x + B.b[a][3] * c3.x;
    y[a].y = B.b[a][0] * c0.y + B.b[a][1] * c1.y + B.b[a][2] * c2.y + B.b[a][3] * c3.y;
  }
  x00 = y[0]; x01 = y[1]; x10 = y[2]; x11 = y[3];
}

// Adjoint mode map: from g_a in the slots of a, write G = sum_a g_a M_a:
//   c_mu = sum_a b[a][mu] g_a;  G00 = c0 + c3, G11 = c0 - c3, G10 = c1 + i c2, G01 = c1 - i c2.
template <class R, class V>
__device__ __forceinline__ void mode_adj(const PovmB<R>& B, V& x00, V& x01, V& x10, V& x11) {
  V g[4] = {x00, x01, x10, x11};
  V c[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    c[mu].x = B.b[0][mu] * g[0].x + B.b[1][mu] * g[1].x + B.b[2][mu] * g[2].x + B.b[3][mu] * g[3].x;
    c[mu].y = B.b[0][mu] * g[0].y + B.b[1][mu] * g[1].y + B.b[2][mu] * g[2].y + B.b[3][mu] * g[3].y;
  }
  V ic2 = cmuli(c[2]);
  x00 = cadd(c[0], c[3]);
  x11 = csub(c[0], c[3]);
  x10 = cadd(c[1], ic2);
  x01 = csub(c[1], ic2);
}

// Bit interleave: a_b = 2 i_b + j_b  <->  k = sum_b a_b 4^b.
__host__ __device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
__host__ __device__ __forceinline__ uint32_t compact_bits(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}
__host__ __device__ __forceinline__ uint32_t interleave_ij(uint32_t i, uint32_t j) {
  return (spread_bits(i) << 1) | spread_bits(j);
}
__host__ __device__ __forceinline__ uint32_t row_of(uint32_t a) { return compact_bits(a >> 1); }
__host__ __device__ __forceinline__ uint32_t col_of(uint32_t a) { return compact_bits(a); }

// Row index I of the t-th lower-triangular tile pair (I >= J), t = I(I+1)/2 + J.
__device__ __forceinline__ void tri_decode(uint32_t t, int& I, int& J) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((uint32_t)((i + 1) * (i + 2) / 2) <= t) ++i;
  while ((uint32_t)(i * (i + 1) / 2) > t) --i;
  I = i;
  J = (int)(t - (uint32_t)(i * (i + 1) / 2));
}

// Rprop on one parameter (Sec. 4.1): c = sign(g) sign(g_prev); the step is scaled
// by eta_plus / eta_minus / 1 for c > 0 / c < 0 / c == 0 and clamped; where c < 0
// the gradient counts as zero; the parameter moves by -sign(g) step.
template <class R> struct RpropCfg { R eta_minus, eta_plus, step_min, step_max; };

// One word of Rprop state per parameter holds the step and the previous gradient sign:
// +step (sign +1), -step (sign -1), or step * 2^64 (sign 0).  Steps stay within [2^-33, 2^30]
// (the options are checked), so |state| >= 2^31 marks sign 0, and the power-of-two scaling is
// exact: the arithmetic is the same as with a separate sign array, with 2 fewer bytes to stream
// per parameter and iteration.
template <class R> struct RpropCode {
  static constexpr R kZero = R(18446744073709551616.0);          // 2^64
  static constexpr R kInvZero = R(5.42101086242752217003726e-20);  // 2^-64
  static constexpr R kThreshold = R(2147483648.0);                 // 2^31
};

template <class R> __host__ __device__ __forceinline__ R rprop_encode(R step, int prev) {
  return prev == 0 ? step * RpropCode<R>::kZero : (prev < 0 ? -step : step);
}

template <class R>
__device__ __forceinline__ R rprop1(R w, R g, R& state, const RpropCfg<R>& c) {
  const R a = state < R(0) ? -state : state;
  const bool zero = a >= RpropCode<R>::kThreshold;
  const int prev = zero ? 0 : (state < R(0) ? -1 : 1);
  const R step = zero ? a * RpropCode<R>::kInvZero : a;
  int s = (g > R(0)) - (g < R(0));
  int cs = s * prev;
  R fac = cs > 0 ? c.eta_plus : (cs < 0 ? c.eta_minus : R(1));
  R st = step * fac;
  st = st < c.step_min ? c.step_min : (st > c.step_max ? c.step_max : st);
  if (cs < 0) s = 0;
  state = rprop_encode(st, s);
  return s > 0 ? w - st : (s < 0 ? w + st : w);
}

// Warp / block sum reduction of double values.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// "Last block done": every block has written its partial; the last one to arrive
// returns true (for all its threads).  The counter is reset by the caller's last block.
__device__ __forceinline__ bool last_block_arrived(unsigned int* counter) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// Fold a block's largest magnitude m >= 0 into *amax (float bits: non-negative floats
// order like their bit patterns).  Called by every thread of the block.
__device__ __forceinline__ void block_absmax_to(float m, unsigned int* amax) {
  __shared__ float s_red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) b = fmaxf(b, s_red[w]);
    atomicMax(amax, __float_as_uint(b));
  }
}

// Programmatic dependent launch: wait until the previous kernel on the stream has completed and its
// writes are visible (a no-op when the kernel was launched without the attribute).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// After grid_dep_wait(): the pointers pass through an empty asm that the compiler must take as changing them,
// so that no load through them is moved above the wait (a load through a const __restrict__ pointer may be).
template <class P> __device__ __forceinline__ int opaque_ptr(P& p) {
  asm volatile("" : "+l"(p));
  return 0;
}
template <class... P> __device__ __forceinline__ void after_wait(P&... ps) {
  const int unused[] = {0, opaque_ptr(ps)...};
  (void)unused;
}

// A tensor map that host code copied into global memory: order the copy before this thread's next use
// of the map by the tensor-map proxy (TMA).
__device__ __forceinline__ void tensormap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(map) : "memory");
}

// Launches of one kernel for a group of tomographies of one size (grid z = the tomography): row z of
// the device table `tab` holds that tomography's pointer arguments, in the order given here, and
// replaces the kernel's own (which are those of a single tomography when tab is NULL).
template <class... P> __device__ __forceinline__ void rebind(const void* const* tab, P&... ps) {
  if (tab == nullptr) return;
  const void* const* row = tab + (size_t)blockIdx.z * sizeof...(P);
  int k = 0;
  ((ps = (P)(const_cast<void*>(row[k++]))), ...);  // P: a (possibly restrict-qualified) pointer type
}

}  // namespace qst
