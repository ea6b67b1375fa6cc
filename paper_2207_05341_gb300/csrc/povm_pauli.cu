// Second pass of the product-POVM map (Sec. 3.3 eq. PS) over the high h qubits, with the
// likelihood and the adjoint fused in, computed in the Pauli basis (see povm.cu for the
// two-pass scheme).
//
// For a fixed low outcome a_lo the packed intermediate is an nb x nb Hermitian matrix W
// (nb = 2^h <= 32).  Its Pauli coefficients w_(x,z) = Tr(sigma_(x,z) W) (x: the flip part,
// z: the phase part of the Pauli string; per qubit (0,0) = I, (1,0) = X, (1,1) = Y,
// (0,1) = Z) are real, and they come from one Walsh-Hadamard transform per flip pattern
// x: with D_x(r) = W_(r^x, r), w_(x,z) = (-i)^|x&z| sum_r (-1)^(z.r) D_x(r).  Because
// D_x(r^x) = conj D_x(r), Re D_x is even and Im D_x odd under r -> r^x, so their
// transforms live on z with x.z even and odd respectively: a single real transform of
// Re D_x + Im D_x gives both, and w is that up to the sign of (-i)^|x&z|.
// Each qubit's POVM then acts on the 2 index bits (x_k, z_k) of w as the real 4 x 4 matrix
// b[a][mu] (M_a = sum_mu b[a][mu] sigma_mu): q = (b x ... x b) w.  The adjoint runs the
// same steps transposed: gamma = (b^T x ... x b^T) g, and G = sum gamma_mu sigma_mu is
// rebuilt per flip pattern by two transforms (the even and the odd parts give Re and Im).
//
// Layout: lanes of a warp are the flip patterns x of G = 32 / nb matrices, registers
// the nb values of z (or r); a qubit's map pairs registers (bit k of z) and lanes (bit k
// of x, one shuffle per value).  Everything is real: 5 qubits cost 32 x 4 FMAs per lane
// and map, where the complex register-row form needs about four times that.  Shared
// memory stages W and f in, q or the packed adjoint out, in coalesced 32-byte segments.
#include <float.h>

#include "impl.h"

namespace qst {

namespace {

template <class T> __device__ __forceinline__ T min_norm();
template <> __device__ __forceinline__ float min_norm<float>() { return FLT_MIN; }
template <> __device__ __forceinline__ double min_norm<double>() { return DBL_MIN; }

template <int NB> struct PGeo {
  static constexpr int G = 32 / NB;          // matrices (low outcomes) per warp
  static constexpr int CB = 8 * G;           // low outcomes per block (8 warps)
  static constexpr int LD = NB + 1;          // padded row of one staged matrix
  // pitch of one staged matrix: NB * LD rounded up to 32 / CB (mod 32), so that the
  // staging loop's 32 consecutive threads (CB low outcomes x 32 / CB entries) hit 32 banks
  static constexpr int SH = CB >= 32 ? 1 : 32 / CB;
  static constexpr int CP = (NB * LD + 31 - SH) / 32 * 32 + SH;
  static constexpr int MAT = CB * CP;        // staged matrices (reals); also q / packed adjoint out
  static constexpr int FS = NB * NB * CB;    // staged f (reals)
  static_assert(MAT >= FS, "the matrix staging area also holds one value per outcome");
};

// In-register Walsh-Hadamard transform of v[0..NB): v_z <- sum_r (-1)^(z.r) v_r.
template <class R, int NB> __device__ __forceinline__ void wht(R (&v)[NB]) {
#pragma unroll
  for (int hb = 1; hb < NB; hb <<= 1) {
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      if (r & hb) continue;
      const R a = v[r], b = v[r | hb];
      v[r] = a + b;
      v[r | hb] = a - b;
    }
  }
}

// Forward map of qubit K: (x_K, z_K) -> outcome a_K = 2 x_K + z_K (lane bit, register bit).
template <class R, int NB, int K> __device__ __forceinline__ void fwd_qubit(R (&w)[NB], const PovmB<R>& B, int x) {
  const bool L = (x >> K) & 1;
  R co0[2], cp0[2], co1[2], cp1[2];  // coefficients of own (o) and partner (p) values, per output
#pragma unroll
  for (int rp = 0; rp < 2; ++rp) {
    const int a0 = rp, a1 = 2 + rp;  // the output a = 2 L + rp
    co0[rp] = L ? B.b[a1][1] : B.b[a0][0];
    cp0[rp] = L ? B.b[a1][0] : B.b[a0][1];
    co1[rp] = L ? B.b[a1][2] : B.b[a0][3];
    cp1[rp] = L ? B.b[a1][3] : B.b[a0][2];
  }
#pragma unroll
  for (int r0 = 0; r0 < NB; ++r0) {
    if (r0 & (1 << K)) continue;
    const int r1 = r0 | (1 << K);
    const R o0 = w[r0], o1 = w[r1];
    const R p0 = __shfl_xor_sync(0xffffffffu, o0, 1 << K);
    const R p1 = __shfl_xor_sync(0xffffffffu, o1, 1 << K);
    w[r0] = co0[0] * o0 + cp0[0] * p0 + co1[0] * o1 + cp1[0] * p1;
    w[r1] = co0[1] * o0 + cp0[1] * p0 + co1[1] * o1 + cp1[1] * p1;
  }
}

// Adjoint map of qubit K: outcome a_K = 2 L + z_K -> Pauli index mu at (x_K, z_K).
template <class R, int NB, int K> __device__ __forceinline__ void adj_qubit(R (&w)[NB], const PovmB<R>& B, int x) {
  const bool L = (x >> K) & 1;
  // per output register bit rp: gamma_mu with mu = (L ? X : I) for rp = 0, (L ? Y : Z) for rp = 1, from
  // own values o0, o1 (outcomes 2L, 2L + 1) and the partner's p0, p1 (outcomes 2 - 2L, 3 - 2L)
  R c[2][4];
  c[0][0] = L ? B.b[2][1] : B.b[0][0];
  c[0][1] = L ? B.b[3][1] : B.b[1][0];
  c[0][2] = L ? B.b[0][1] : B.b[2][0];
  c[0][3] = L ? B.b[1][1] : B.b[3][0];
  c[1][0] = L ? B.b[2][2] : B.b[0][3];
  c[1][1] = L ? B.b[3][2] : B.b[1][3];
  c[1][2] = L ? B.b[0][2] : B.b[2][3];
  c[1][3] = L ? B.b[1][2] : B.b[3][3];
#pragma unroll
  for (int r0 = 0; r0 < NB; ++r0) {
    if (r0 & (1 << K)) continue;
    const int r1 = r0 | (1 << K);
    const R o0 = w[r0], o1 = w[r1];
    const R p0 = __shfl_xor_sync(0xffffffffu, o0, 1 << K);
    const R p1 = __shfl_xor_sync(0xffffffffu, o1, 1 << K);
    w[r0] = c[0][0] * o0 + c[0][1] * o1 + c[0][2] * p0 + c[0][3] * p1;
    w[r1] = c[1][0] * o0 + c[1][1] * o1 + c[1][2] * p0 + c[1][3] * p1;
  }
}

template <class R, int NB> __device__ __forceinline__ void fwd_all(R (&w)[NB], const PovmB<R>& B, int x) {
  if constexpr (NB > 1) fwd_qubit<R, NB, 0>(w, B, x);
  if constexpr (NB > 2) fwd_qubit<R, NB, 1>(w, B, x);
  if constexpr (NB > 4) fwd_qubit<R, NB, 2>(w, B, x);
  if constexpr (NB > 8) fwd_qubit<R, NB, 3>(w, B, x);
  if constexpr (NB > 16) fwd_qubit<R, NB, 4>(w, B, x);
}
template <class R, int NB> __device__ __forceinline__ void adj_all(R (&w)[NB], const PovmB<R>& B, int x) {
  if constexpr (NB > 1) adj_qubit<R, NB, 0>(w, B, x);
  if constexpr (NB > 2) adj_qubit<R, NB, 1>(w, B, x);
  if constexpr (NB > 4) adj_qubit<R, NB, 2>(w, B, x);
  if constexpr (NB > 8) adj_qubit<R, NB, 3>(w, B, x);
  if constexpr (NB > 16) adj_qubit<R, NB, 4>(w, B, x);
}

// sign of (-i)^|x&z| (forward) and of i^|x&z| after Re + Im (adjoint): - for |x&z| = 2, 3 mod 4
__device__ __forceinline__ bool neg_phase(int x, int z) { return (__popc(x & z) & 2) != 0; }

// MODE 0: forward only, write q to p.  MODE 1: likelihood (+ adjoint when adjoint != 0).
template <class R, int NB, int MODE>
__global__ void __launch_bounds__(256) k_povm_hi_pauli(const R* __restrict__ W, R* __restrict__ p,
                                                        const R* __restrict__ f, double* scal, R* __restrict__ Wadj,
                                                        double* partials, unsigned int* counter, unsigned int* flags,
                                                        int g, PovmB<R> B, int adjoint) {
  using Gm = PGeo<NB>;
  constexpr int CB = Gm::CB, LD = Gm::LD, CP = Gm::CP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* mat = reinterpret_cast<R*>(smem_raw);
  R* fs = mat + Gm::MAT;
  __shared__ double red[8];
  const long long SS = 1LL << (2 * g);
  const long long al0 = (long long)blockIdx.x * CB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x = lane % NB, c = warp * Gm::G + lane / NB;

  for (int t = tid; t < NB * NB * CB; t += blockDim.x) {
    const int cc = t % CB, pair = t / CB;
    mat[cc * CP + (pair / NB) * LD + (pair % NB)] = W[(long long)pair * SS + al0 + cc];
    if (MODE == 1) fs[t] = f[(long long)pair * SS + al0 + cc];  // here pair is the high outcome
  }
  __syncthreads();

  // Pauli coefficients of this lane's flip pattern x: transform of Re D_x + Im D_x
  R w[NB];
  {
    const R* m = mat + c * CP;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int rx = r ^ x;
      const R a = m[rx * LD + r], b = m[r * LD + rx];  // packed: Re W_ij at [i][j], Im W_ij at [j][i], i > j
      w[r] = x == 0 ? a : (rx > r ? a + b : b - a);
    }
  }
  wht<R, NB>(w);
#pragma unroll
  for (int z = 0; z < NB; ++z)
    if (neg_phase(x, z)) w[z] = -w[z];
  fwd_all<R, NB>(w, B, x);  // w[z] is now q at the outcome interleave_ij(x, z)
  __syncthreads();          // the staging area is reused below

  if (MODE == 0) {
#pragma unroll
    for (int z = 0; z < NB; ++z) mat[interleave_ij(x, z) * CB + c] = w[z];
    __syncthreads();
    for (int t = tid; t < NB * NB * CB; t += blockDim.x) {
      const int cc = t % CB, ah = t / CB;
      p[(long long)ah * SS + al0 + cc] = mat[t];
    }
    return;
  }

  // L = -sum f log q + (sum f) log Tr X;  g_k = -f_k / q_k + sum f / Tr X
  const double tX = scal[0], sumf = scal[1];
  const R gconst = (R)(sumf / tX);
  const R qmin = min_norm<R>();
  R accr = R(0);  // a lane's terms in R (FP64 arithmetic is a slow pipe on this part); lanes, blocks in FP64
  unsigned int nclamp = 0;
#pragma unroll
  for (int z = 0; z < NB; ++z) {
    R q = w[z];
    const R fk = fs[interleave_ij(x, z) * CB + c];
    R gk = gconst;
    if (fk > R(0)) {
      if (!(q >= qmin)) {  // clamped: the constant -f_k log q_min, nothing added to dL/dq_k
        ++nclamp;
        accr += fk * log(qmin);
      } else {
        accr += fk * log(q);
        gk -= fk / q;
      }
    }
    w[z] = gk;
  }
  if (nclamp) atomicAdd(flags, nclamp);
  double acc = warp_sum((double)accr);
  if (lane == 0) red[warp] = acc;
  if (adjoint) {
    adj_all<R, NB>(w, B, x);  // w[z] = gamma_(x,z)
    R re[NB], im[NB];
#pragma unroll
    for (int z = 0; z < NB; ++z) {
      const R v = neg_phase(x, z) ? -w[z] : w[z];
      const bool odd = __popc(x & z) & 1;
      re[z] = odd ? R(0) : v;
      im[z] = odd ? v : R(0);
    }
    wht<R, NB>(re);  // Re G_(r^x, r)
    wht<R, NB>(im);  // Im G_(r^x, r)
    R* m = mat + c * CP;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int rx = r ^ x;
      if (x == 0) {
        m[r * LD + r] = re[r];
      } else if (rx > r) {
        m[rx * LD + r] = re[r];
        m[r * LD + rx] = im[r];
      }
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
      Wadj[(long long)pair * SS + al0 + cc] = mat[cc * CP + (pair / NB) * LD + (pair % NB)];
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
cudaError_t launch_pauli(const Dims& D, const R* W, R* p, const R* f, double* scal, R* Wadj, double* partials,
                         unsigned int* counter, unsigned int* flags, const PovmB<R>& B, bool adjoint,
                         cudaStream_t s) {
  using Gm = PGeo<NB>;
  const size_t sm = (size_t)(Gm::MAT + (MODE == 1 ? Gm::FS : 0)) * sizeof(R);
  cudaError_t e = ensure_dynamic_smem((const void*)k_povm_hi_pauli<R, NB, MODE>, sm);
  if (e != cudaSuccess) return e;
  const long long SS = 1LL << (2 * D.g);
  const unsigned blocks = (unsigned)(SS / Gm::CB);
  if (MODE == 1 && blocks > (unsigned)kPartialBlocks * kPartialStride) return cudaErrorInvalidConfiguration;
  k_povm_hi_pauli<R, NB, MODE><<<blocks, 256, sm, s>>>(W, p, f, scal, Wadj, partials, counter, flags, D.g, B,
                                                       adjoint ? 1 : 0);
  return cudaGetLastError();
}

template <class R, int MODE>
cudaError_t dispatch_pauli(const Dims& D, const R* W, R* p, const R* f, double* scal, R* Wadj, double* partials,
                           unsigned int* counter, unsigned int* flags, const PovmB<R>& B, bool adjoint,
                           cudaStream_t s) {
  switch (D.nb) {
    case 2: return launch_pauli<R, 2, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 4: return launch_pauli<R, 4, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 8: return launch_pauli<R, 8, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 16: return launch_pauli<R, 16, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
    case 32: return launch_pauli<R, 32, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool povm_hi_pauli_ok(const Dims& D) { return D.nb >= 2 && D.nb <= 32 && D.g >= 6; }

template <class R>
cudaError_t povm_hi_fwd_pauli(const Dims& D, const R* W, R* p, const PovmB<R>& B, cudaStream_t s) {
  return dispatch_pauli<R, 0>(D, W, p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, B, false, s);
}

template <class R>
cudaError_t povm_hi_nll_pauli(const Dims& D, const R* W, const R* f, double* scal, R* Wadj, double* partials,
                              unsigned int* counter, unsigned int* flags, const PovmB<R>& B, bool adjoint,
                              cudaStream_t s) {
  return dispatch_pauli<R, 1>(D, W, nullptr, f, scal, Wadj, partials, counter, flags, B, adjoint, s);
}

template cudaError_t povm_hi_fwd_pauli<float>(const Dims&, const float*, float*, const PovmB<float>&, cudaStream_t);
template cudaError_t povm_hi_fwd_pauli<double>(const Dims&, const double*, double*, const PovmB<double>&,
                                               cudaStream_t);
template cudaError_t povm_hi_nll_pauli<float>(const Dims&, const float*, const float*, double*, float*, double*,
                                              unsigned int*, unsigned int*, const PovmB<float>&, bool, cudaStream_t);
template cudaError_t povm_hi_nll_pauli<double>(const Dims&, const double*, const double*, double*, double*, double*,
                                               unsigned int*, unsigned int*, const PovmB<double>&, bool,
                                               cudaStream_t);

}  // namespace qst
