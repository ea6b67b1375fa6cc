// Product-POVM map of Sec. 3.3 (eq. PS), its adjoint, and the likelihood of Sec. 3.1.
//
//   q_k = Tr[(M_k1 (x) ... (x) M_kN) X],   k = sum_b a_b 4^b,  qubit b <-> row/col bit b.
//
// The map is a chain of per-qubit 4 x 4 mode contractions on the index pair
// (i_b, j_b) of X.  It runs in two passes:
//   pass 1 (povm_lo_*): one CTA per lower S x S tile (I >= J) of the d x d matrix
//     applies the g low qubits in shared memory.  For fixed low outcomes a_lo the
//     result Z[I, J, a_lo] is Hermitian in (I, J), so only lower tiles are read and
//     the result is stored packed as reals: Re at [I][J], Im at [J][I]
//     (W[(I nb + J) S^2 + a_lo]).
//   pass 2 (povm_hi_*): one CTA per chunk of C low outcomes loads the nb x nb
//     Hermitian matrices of its chunk, applies the h high qubits, and writes q
//     (forward), or evaluates the likelihood, forms g_k = dL/dq_k and applies the
//     adjoint high-qubit maps (training step).
// The adjoint pass 1 (povm_lo_adj) maps the packed adjoint back to the full
// Hermitian d x d matrix G = sum_k g_k M_k.
#include <float.h>

#include <mutex>
#include <unordered_map>

#include "impl.h"

namespace qst {

// cudaFuncSetAttribute once per kernel and size (host calls between launches leave the GPU idle).
cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(fn);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[fn] = bytes;
  return e;
}

Dims make_dims(int N, bool fp64) {
  Dims D;
  D.N = N;
  D.d = 1 << N;
  D.n = 1LL << (2 * N);
  D.H = 2 * N;
  int g = N < 6 ? N : 6;
  if (!fp64 && N >= 12) g = 7;
  D.g = g;
  D.h = N - g;
  D.S = 1 << g;
  D.nb = 1 << D.h;
  const long long SS = 1LL << (2 * g);
  const int vbytes = fp64 ? 16 : 8;
  long long budget = 96 * 1024;
  long long C = 1;
  while (C * 2 <= SS && (long long)D.nb * D.nb * (C * 2) * vbytes <= budget) C *= 2;
  D.C = (int)C;
  return D;
}

template <class T> __device__ __forceinline__ T min_normal();
template <> __device__ __forceinline__ float min_normal<float>() { return FLT_MIN; }
template <> __device__ __forceinline__ double min_normal<double>() { return DBL_MIN; }

// Apply per-qubit mode maps on bits [0, bits) of (row, col) of an array
// Z[(r * pitch + c) * C + cc], r, c < 2^side_log2, cc < C = 2^logC.
template <class R, bool ADJ>
__device__ void apply_modes(cx_t<R>* Z, int side_log2, int pitch, int logC, int bits, const PovmB<R>& B) {
  using V = cx_t<R>;
  if (bits <= 0) return;
  const int C = 1 << logC;
  const int half_log2 = side_log2 - 1;
  const int groups = 1 << (2 * half_log2 + logC);
  for (int b = 0; b < bits; ++b) {
    const int bit = 1 << b;
    const int lowmask = bit - 1;
    for (int t = threadIdx.x; t < groups; t += blockDim.x) {
      const int cc = t & (C - 1);
      const int gi = t >> logC;
      const int rr = gi >> half_log2;
      const int c2 = gi & ((1 << half_log2) - 1);
      const int r0 = ((rr & ~lowmask) << 1) | (rr & lowmask);
      const int c0 = ((c2 & ~lowmask) << 1) | (c2 & lowmask);
      V* p00 = Z + ((size_t)(r0 * pitch + c0) << logC) + cc;
      V* p01 = p00 + ((size_t)bit << logC);
      V* p10 = p00 + ((size_t)(bit * pitch) << logC);
      V* p11 = p10 + ((size_t)bit << logC);
      V x00 = *p00, x01 = *p01, x10 = *p10, x11 = *p11;
      if (ADJ) mode_adj(B, x00, x01, x10, x11);
      else mode_fwd(B, x00, x01, x10, x11);
      *p00 = x00; *p01 = x01; *p10 = x10; *p11 = x11;
    }
    __syncthreads();
  }
}

// The mode maps of all g qubits of an S x S tile (S = 2^g), two qubits per sweep: a thread takes
// the 4 x 4 elements that bits (b, b+1) of the row and column index span, applies qubit b and
// then qubit b + 1 in registers and stores them back (each element sees the same operations in
// the same order as with one qubit per sweep, so the result is bit-identical, with half the
// shared-memory traffic and barriers).
template <class R, bool ADJ>
__device__ void apply_modes_tile(cx_t<R>* Z, int g, int pitch, const PovmB<R>& B) {
  using V = cx_t<R>;
  int b = 0;
  for (; b + 1 < g; b += 2) {
    const int gh = g - 2;
    const int groups = 1 << (2 * gh);
    const int low = (1 << b) - 1;
    for (int t = threadIdx.x; t < groups; t += blockDim.x) {
      const int rr = t >> gh, cc = t & ((1 << gh) - 1);
      const int r0 = ((rr & ~low) << 2) | (rr & low);
      const int c0 = ((cc & ~low) << 2) | (cc & low);
      V x[4][4];  // [k][l]: row offset (k >> 1) << (b + 1) | (k & 1) << b, column offset likewise
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l)
          x[k][l] = Z[(r0 + (((k >> 1) << (b + 1)) | ((k & 1) << b))) * pitch + c0 + (((l >> 1) << (b + 1)) | ((l & 1) << b))];
#pragma unroll
      for (int hk = 0; hk < 2; ++hk)
#pragma unroll
        for (int hl = 0; hl < 2; ++hl) {  // qubit b: row bit k & 1, column bit l & 1
          if (ADJ) mode_adj(B, x[2 * hk][2 * hl], x[2 * hk][2 * hl + 1], x[2 * hk + 1][2 * hl], x[2 * hk + 1][2 * hl + 1]);
          else mode_fwd(B, x[2 * hk][2 * hl], x[2 * hk][2 * hl + 1], x[2 * hk + 1][2 * hl], x[2 * hk + 1][2 * hl + 1]);
        }
#pragma unroll
      for (int lk = 0; lk < 2; ++lk)
#pragma unroll
        for (int ll = 0; ll < 2; ++ll) {  // qubit b + 1: row bit k >> 1, column bit l >> 1
          if (ADJ) mode_adj(B, x[lk][ll], x[lk][2 + ll], x[2 + lk][ll], x[2 + lk][2 + ll]);
          else mode_fwd(B, x[lk][ll], x[lk][2 + ll], x[2 + lk][ll], x[2 + lk][2 + ll]);
        }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l)
          Z[(r0 + (((k >> 1) << (b + 1)) | ((k & 1) << b))) * pitch + c0 + (((l >> 1) << (b + 1)) | ((l & 1) << b))] = x[k][l];
    }
    __syncthreads();
  }
  if (b < g) {  // odd g: the last qubit alone
    const int half = g - 1;
    const int groups = 1 << (2 * half);
    const int bit = 1 << b, low = bit - 1;
    for (int t = threadIdx.x; t < groups; t += blockDim.x) {
      const int rr = t >> half, cc = t & ((1 << half) - 1);
      const int r0 = ((rr & ~low) << 1) | (rr & low);
      const int c0 = ((cc & ~low) << 1) | (cc & low);
      V* p00 = Z + r0 * pitch + c0;
      V x00 = p00[0], x01 = p00[bit], x10 = p00[bit * pitch], x11 = p00[bit * pitch + bit];
      if (ADJ) mode_adj(B, x00, x01, x10, x11);
      else mode_fwd(B, x00, x01, x10, x11);
      p00[0] = x00; p00[bit] = x01; p00[bit * pitch] = x10; p00[bit * pitch + bit] = x11;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- pass 1
template <class R>
__global__ void __launch_bounds__(256) k_povm_lo_fwd(const cx_t<R>* __restrict__ X, R* __restrict__ W,
                                                      int N, int g, PovmB<R> B) {
  using V = cx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Z = reinterpret_cast<V*>(smem_raw);
  const int S = 1 << g, pitch = S + 1, nb = 1 << (N - g);
  const long long d = 1LL << N;
  int I, J;
  tri_decode(blockIdx.x, I, J);
  const V* src = X + (long long)I * S * d + (long long)J * S;
  if (S * S == 16 * 256 && blockDim.x == 256) {  // 64 x 64 tiles: all 16 loads of a thread in flight at once
    V v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int e = threadIdx.x + k * 256;
      v[k] = src[(long long)(e >> 6) * d + (e & 63)];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int e = threadIdx.x + k * 256;
      Z[(e >> 6) * pitch + (e & 63)] = v[k];
    }
  } else {
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
      const int il = e >> g, jl = e & (S - 1);
      Z[il * pitch + jl] = src[il * d + jl];
    }
  }
  __syncthreads();
  if (I == J) {  // diagonal tile: rebuild the upper triangle from the lower one
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
      const int il = e >> g, jl = e & (S - 1);
      if (il < jl) Z[il * pitch + jl] = cconj(Z[jl * pitch + il]);
    }
    __syncthreads();
  }
  apply_modes_tile<R, false>(Z, g, pitch, B);
  const long long SS = (long long)S * S;
  R* wlo = W + ((long long)I * nb + J) * SS;
  R* whi = W + ((long long)J * nb + I) * SS;
  for (int al = threadIdx.x; al < S * S; al += blockDim.x) {
    const V v = Z[row_of(al) * pitch + col_of(al)];
    wlo[al] = v.x;
    if (I != J) whi[al] = v.y;
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_povm_lo_adj(const R* __restrict__ W, cx_t<R>* __restrict__ G,
                                                      int N, int g, PovmB<R> B, unsigned int* amax) {
  using V = cx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Z = reinterpret_cast<V*>(smem_raw);
  const int S = 1 << g, pitch = S + 1, nb = 1 << (N - g);
  const long long d = 1LL << N;
  int I, J;
  tri_decode(blockIdx.x, I, J);
  const long long SS = (long long)S * S;
  const R* wlo = W + ((long long)I * nb + J) * SS;
  const R* whi = W + ((long long)J * nb + I) * SS;
  if (S * S == 16 * 256 && blockDim.x == 256) {  // 64 x 64 tiles: all loads of a thread in flight at once
    R re[16], im[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int al = threadIdx.x + k * 256;
      re[k] = wlo[al];
      im[k] = (I != J) ? whi[al] : R(0);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int al = threadIdx.x + k * 256;
      Z[row_of(al) * pitch + col_of(al)] = cmake<V>(re[k], im[k]);
    }
  } else {
    for (int al = threadIdx.x; al < S * S; al += blockDim.x) {
      const R re = wlo[al];
      const R im = (I != J) ? whi[al] : R(0);
      Z[row_of(al) * pitch + col_of(al)] = cmake<V>(re, im);
    }
  }
  __syncthreads();
  apply_modes_tile<R, true>(Z, g, pitch, B);
  V* dst = G + (long long)I * S * d + (long long)J * S;
  float m = 0.f;
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    const int il = e >> g, jl = e & (S - 1);
    const V z = Z[il * pitch + jl];
    dst[il * d + jl] = z;
    m = fmaxf(m, fmaxf(fabsf((float)z.x), fabsf((float)z.y)));
  }
  if (amax) block_absmax_to(m, amax);  // the mirrored tile holds the same magnitudes
  if (I != J) {
    V* mir = G + (long long)J * S * d + (long long)I * S;
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
      const int r = e >> g, c = e & (S - 1);
      mir[r * d + c] = cconj(Z[c * pitch + r]);
    }
  }
}

// ---------------------------------------------------------------- pass 2
template <class R>
__device__ __forceinline__ void load_hermitian_chunk(cx_t<R>* Z, const R* __restrict__ W, int h, int logC,
                                                     long long SS, long long al0) {
  using V = cx_t<R>;
  const int nb = 1 << h, C = 1 << logC;
  const int tot = nb * nb * C;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int c = t & (C - 1);
    const int pidx = t >> logC;
    const int ih = pidx >> h, jh = pidx & (nb - 1);
    const R a = W[((long long)ih * nb + jh) * SS + al0 + c];
    V v;
    if (ih == jh) {
      v = cmake<V>(a, R(0));
    } else {
      const R b = W[((long long)jh * nb + ih) * SS + al0 + c];
      v = ih > jh ? cmake<V>(a, b) : cmake<V>(b, -a);
    }
    Z[t] = v;
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(256) k_povm_hi_fwd(const R* __restrict__ W, R* __restrict__ p, int N, int g,
                                                      int logC, PovmB<R> B) {
  using V = cx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Z = reinterpret_cast<V*>(smem_raw);
  const int h = N - g, nb = 1 << h, C = 1 << logC;
  const long long SS = 1LL << (2 * g);
  const long long al0 = (long long)blockIdx.x * C;
  load_hermitian_chunk<R>(Z, W, h, logC, SS, al0);
  apply_modes<R, false>(Z, h, nb, logC, h, B);
  const int tot = nb * nb * C;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int c = t & (C - 1);
    const uint32_t ah = (uint32_t)(t >> logC);
    p[(long long)ah * SS + al0 + c] = Z[((row_of(ah) * nb + col_of(ah)) << logC) + c].x;
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_povm_hi_nll(const R* __restrict__ W, const R* __restrict__ f,
                                                      double* scal, R* __restrict__ Wadj, double* partials,
                                                      unsigned int* counter, unsigned int* flags, int N, int g,
                                                      int logC, PovmB<R> B, int adjoint) {
  using V = cx_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Z = reinterpret_cast<V*>(smem_raw);
  __shared__ double red[32];
  const int h = N - g, nb = 1 << h, C = 1 << logC;
  const long long SS = 1LL << (2 * g);
  const long long al0 = (long long)blockIdx.x * C;
  load_hermitian_chunk<R>(Z, W, h, logC, SS, al0);
  apply_modes<R, false>(Z, h, nb, logC, h, B);

  // L = -sum_k f_k log q_k + (sum_k f_k) log Tr X;  g_k = dL/dq_k = -f_k / q_k + sum f / Tr X
  const double tX = scal[0], sumf = scal[1];
  const R gconst = (R)(sumf / tX);
  const R qmin = min_normal<R>();
  double acc = 0.0;
  unsigned int nclamp = 0;
  const int tot = nb * nb * C;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int c = t & (C - 1);
    const uint32_t ah = (uint32_t)(t >> logC);
    const int zi = ((row_of(ah) * nb + col_of(ah)) << logC) + c;
    R q = Z[zi].x;
    const R fk = f[(long long)ah * SS + al0 + c];
    R gk = gconst;
    if (fk > R(0)) {
      if (!(q >= qmin)) {  // clamped: the constant -f_k log q_min, nothing added to dL/dq_k
        ++nclamp;
        acc += (double)fk * (double)log(qmin);
      } else {
        acc += (double)fk * (double)log(q);
        gk -= fk / q;
      }
    }
    Z[zi] = cmake<V>(gk, R(0));
  }
  if (nclamp) atomicAdd(flags, nclamp);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
  if (adjoint) {
    apply_modes<R, true>(Z, h, nb, logC, h, B);
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int c = t & (C - 1);
      const int pidx = t >> logC;
      const int ih = pidx >> h, jh = pidx & (nb - 1);
      if (ih < jh) continue;
      const V v = Z[t];
      Wadj[((long long)ih * nb + jh) * SS + al0 + c] = v.x;
      if (ih > jh) Wadj[((long long)jh * nb + ih) * SS + al0 + c] = v.y;
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

// ---------------------------------------------------------------- Tr X of the computed X
// The likelihood and rho = X / Tr X use the trace of X as computed (not ||T||_F^2), so the
// normalisation carries the same rounding as q and the loss stays invariant to the scale of T.
template <class R>
__global__ void __launch_bounds__(256) k_trace(const cx_t<R>* __restrict__ X, int d, double* scal,
                                                const void* const* tab) {
  __shared__ double red[8];
  rebind(tab, X, scal);
  grid_dep_wait();
  after_wait(X, scal);
  // every diagonal load of a thread is issued before the first add (one memory latency, not d / 256)
  constexpr int kPer = 16;  // d <= 4096 = 16 x 256
  R v[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int i = threadIdx.x + k * 256;
    v[k] = i < d ? X[(long long)i * d + i].x : R(0);
  }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kPer; ++k)
    if (threadIdx.x + k * 256 < d) acc += (double)v[k];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    scal[0] = t;
  }
}

// ---------------------------------------------------------------- rho = X / Tr X from lower tiles
template <class R>
__global__ void __launch_bounds__(256) k_herm_complete(const cx_t<R>* __restrict__ X, cx_t<R>* __restrict__ rho,
                                                        int d, const double* scal) {
  using V = cx_t<R>;
  __shared__ V tile[32][33];
  const int TS = d < 32 ? d : 32;
  const int bi = blockIdx.y, bj = blockIdx.x;  // output tile (row block, col block)
  const R s = (R)(1.0 / scal[0]);
  // load the tile of the lower triangle that covers this output tile
  const int lr = bi >= bj ? bi : bj, lc = bi >= bj ? bj : bi;
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    tile[r][c] = X[(long long)(lr * TS + r) * d + lc * TS + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    const int gi = bi * TS + r, gj = bj * TS + c;
    V v;
    if (bi > bj) v = tile[r][c];
    else if (bi < bj) v = cconj(tile[c][r]);
    else v = gi >= gj ? tile[r][c] : cconj(tile[c][r]);
    rho[(long long)gi * d + gj] = cscale(v, s);
  }
}

// ---------------------------------------------------------------- launchers
static int ilog2i(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

template <class R> static cudaError_t set_smem(const void* fn, size_t bytes) { return ensure_dynamic_smem(fn, bytes); }

template <class R>
cudaError_t povm_lo_fwd(const Dims& D, const cx_t<R>* X, R* W, const PovmB<R>& B, cudaStream_t s) {
  const size_t sm = (size_t)D.S * (D.S + 1) * sizeof(cx_t<R>);
  cudaError_t e = set_smem<R>((const void*)k_povm_lo_fwd<R>, sm);
  if (e != cudaSuccess) return e;
  const unsigned tiles = (unsigned)(D.nb * (D.nb + 1) / 2);
  k_povm_lo_fwd<R><<<tiles, 256, sm, s>>>(X, W, D.N, D.g, B);
  return cudaGetLastError();
}

template <class R>
cudaError_t povm_lo_adj(const Dims& D, const R* Wadj, cx_t<R>* G, const PovmB<R>& B, unsigned int* amax,
                        cudaStream_t s) {
  const size_t sm = (size_t)D.S * (D.S + 1) * sizeof(cx_t<R>);
  cudaError_t e = set_smem<R>((const void*)k_povm_lo_adj<R>, sm);
  if (e != cudaSuccess) return e;
  const unsigned tiles = (unsigned)(D.nb * (D.nb + 1) / 2);
  k_povm_lo_adj<R><<<tiles, 256, sm, s>>>(Wadj, G, D.N, D.g, B, amax);
  return cudaGetLastError();
}

template <class R>
cudaError_t povm_hi_fwd(const Dims& D, const R* W, R* p, const PovmB<R>& B, cudaStream_t s) {
  if (povm_hi_pauli_ok(D)) return povm_hi_fwd_pauli<R>(D, W, p, B, s);
  const size_t sm = (size_t)D.nb * D.nb * D.C * sizeof(cx_t<R>);
  cudaError_t e = set_smem<R>((const void*)k_povm_hi_fwd<R>, sm);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((1LL << (2 * D.g)) / D.C);
  k_povm_hi_fwd<R><<<blocks, 256, sm, s>>>(W, p, D.N, D.g, ilog2i(D.C), B);
  return cudaGetLastError();
}

template <class R>
cudaError_t povm_hi_nll(const Dims& D, const R* W, const R* f, double* scal, R* Wadj, double* partials,
                        unsigned int* counter, unsigned int* flags, const PovmB<R>& B, bool adjoint,
                        cudaStream_t s) {
  if (povm_hi_pauli_ok(D)) return povm_hi_nll_pauli<R>(D, W, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
  const size_t sm = (size_t)D.nb * D.nb * D.C * sizeof(cx_t<R>);
  cudaError_t e = set_smem<R>((const void*)k_povm_hi_nll<R>, sm);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((1LL << (2 * D.g)) / D.C);
  if (blocks > (unsigned)kPartialBlocks * kPartialStride) return cudaErrorInvalidConfiguration;
  k_povm_hi_nll<R><<<blocks, 256, sm, s>>>(W, f, scal, Wadj, partials, counter, flags, D.N, D.g,
                                          ilog2i(D.C), B, adjoint ? 1 : 0);
  return cudaGetLastError();
}

template <class R> cudaError_t trace_X(const Dims& D, const cx_t<R>* X, double* scal, cudaStream_t s) {
  if (D.d > 4096) return cudaErrorInvalidValue;
  BatchArgs ba;
  if (batch_take(ba, {X, scal})) return cudaSuccess;
  return launch_dep(k_trace<R>, dim3(1, 1, ba.nz), dim3(256), 0, s, X, D.d, scal, ba.tab);
}

template <class R>
cudaError_t hermitian_complete(const Dims& D, const cx_t<R>* Xlow, cx_t<R>* rho, const double* scal,
                               cudaStream_t s) {
  const int TS = D.d < 32 ? D.d : 32;
  dim3 grid(D.d / TS, D.d / TS);
  k_herm_complete<R><<<grid, 256, 0, s>>>(Xlow, rho, D.d, scal);
  return cudaGetLastError();
}

#define QST_INST(R)                                                                                        \
  template cudaError_t povm_lo_fwd<R>(const Dims&, const cx_t<R>*, R*, const PovmB<R>&, cudaStream_t);       \
  template cudaError_t povm_lo_adj<R>(const Dims&, const R*, cx_t<R>*, const PovmB<R>&, unsigned int*,      \
                                      cudaStream_t);                                                         \
  template cudaError_t povm_hi_fwd<R>(const Dims&, const R*, R*, const PovmB<R>&, cudaStream_t);             \
  template cudaError_t povm_hi_nll<R>(const Dims&, const R*, const R*, double*, R*, double*, unsigned int*,  \
                                      unsigned int*, const PovmB<R>&, bool, cudaStream_t);                   \
  template cudaError_t hermitian_complete<R>(const Dims&, const cx_t<R>*, cx_t<R>*, const double*, cudaStream_t); \
  template cudaError_t trace_X<R>(const Dims&, const cx_t<R>*, double*, cudaStream_t);
QST_INST(float)
QST_INST(double)
#undef QST_INST

}  // namespace qst
