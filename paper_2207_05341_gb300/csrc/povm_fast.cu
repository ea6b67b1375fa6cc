// Product-POVM map of Sec. 3.3 (eq. PS), its likelihood (Sec. 3.1) and adjoint for FP32 contexts
// with N = 7..11: the two passes of povm.cu (low g = 6 qubits in 64 x 64 tiles, then the h = N - 6
// high qubits per low outcome), rebuilt around registers.
//
// Pass 1, one CTA (256 threads) per lower tile pair (I >= J).  A thread holds a 4 x 4 block of the
// tile in registers, which spans the row and column bits of two qubits: three sweeps (qubits 0-1,
// 2-3, 4-5) with two transposes through shared memory in between.  The first sweep's block is read
// straight from HBM (two 16-byte loads per row), the last sweep's outputs are written straight to the
// packed intermediate, 32 consecutive outcomes per warp and register.  The shared-memory index
// swizzle (sw_idx) makes every transpose access conflict-free (16 distinct 8-byte bank pairs per
// half-warp for all three thread maps).
//
// Pass 2 (structured POVMs), one CTA per 32 consecutive low outcomes: thread (c, x) of 32 x nb
// reads the XOR diagonal x of the nb x nb Hermitian matrix of low outcome c (W_(r^x, r) for all r:
// with the XOR-diagonal slot layout these are nb coalesced loads), forms its Pauli coefficients with
// one Walsh-Hadamard transform over r, scales them by beta (and the sign of (-i)^|x & z|, one table
// entry per (x, z)), transforms over z, and hands the values over through one shared-memory
// transpose to thread (c, zeta), which transforms over x and writes 32 consecutive outcomes per
// register.  The likelihood and the adjoint (the same steps in reverse) follow in the same kernel.
// Per real value this costs about 3 FP32 operations per qubit (generic 4 x 4 maps: 5).
//
// Structured POVMs: per qubit the map from the 2 x 2 block (x00, x01, x10, x11) of X to the four
// outcomes is  c = (x00 + x11, x01 + x10, i (x01 - x10), x00 - x11)  (the Pauli components I, X, Y,
// Z), u_mu = beta_mu c_mu, then y(alpha, zeta) = sum_mu (-1)^(alpha x_mu + zeta z_mu) u_mu (a 2 x 2
// Walsh-Hadamard transform), and outcome a = out[2 alpha + zeta].
#include <float.h>

#include "impl.h"

namespace qst {

namespace {

constexpr int kTile = 64;            // S = 2^g, g = 6
constexpr int kLogSS = 12;           // S^2 = 4096 low outcomes
constexpr int kLoThreads = 256;

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Packed pairs of FP32 values (f32x2 arithmetic of sm_100 and later): a complex number (re, im), or the
// same value of two neighbouring low outcomes.
union P2 {
  float2 f;
  unsigned long long u;
};
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  P2 x{a}, y{b}, r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
  return r.f;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  P2 x{a}, y{b}, r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
  return r.f;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  P2 x{a}, y{b}, r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
  return r.f;
}
// a * b + c
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  P2 x{a}, y{b}, z{c}, r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(x.u), "l"(y.u), "l"(z.u));
  return r.f;
}
__device__ __forceinline__ float2 swap2(float2 a) { return f2(a.y, a.x); }

// Loads of data written by the kernel launched just before (programmatic dependent launch): volatile,
// so that they stay after the grid-dependency wait, and through L2 only.
__device__ __forceinline__ float ld_dep(const float* p) {
  float v;
  asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ float2 ld_dep2(const float* p) {
  float2 v;
  asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------- per-qubit 2 x 2 block maps
struct MapGeneric {
  float2 b[4][4];  // (b[a][mu], b[a][mu])
  __device__ __forceinline__ void fwd(float2& x00, float2& x01, float2& x10, float2& x11) const {
    // c = (x00 + x11, x01 + x10, i (x01 - x10), x00 - x11);  y_a = sum_mu b[a][mu] c_mu into slot a
    const float2 c0 = add2(x00, x11), c3 = sub2(x00, x11), c1 = add2(x01, x10);
    const float2 c2 = mul2(swap2(sub2(x01, x10)), f2(-1.f, 1.f));
    float2 y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) y[a] = fma2(b[a][3], c3, fma2(b[a][2], c2, fma2(b[a][1], c1, mul2(b[a][0], c0))));
    x00 = y[0]; x01 = y[1]; x10 = y[2]; x11 = y[3];
  }
  __device__ __forceinline__ void adj(float2& x00, float2& x01, float2& x10, float2& x11) const {
    // c_mu = sum_a b[a][mu] g_a;  G00 = c0 + c3, G11 = c0 - c3, G10 = c1 + i c2, G01 = c1 - i c2
    float2 c[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) c[m] = fma2(b[3][m], x11, fma2(b[2][m], x10, fma2(b[1][m], x01, mul2(b[0][m], x00))));
    const float2 ic2 = mul2(swap2(c[2]), f2(-1.f, 1.f));
    x00 = add2(c[0], c[3]);
    x11 = sub2(c[0], c[3]);
    x10 = add2(c[1], ic2);
    x01 = sub2(c[1], ic2);
  }
};

struct MapStruct {
  float2 bI, bZ, nbZ, bX, mbY, pbY;  // (bI, bI), (bZ, bZ), (-bZ, -bZ), (bX, bX), (-bY, bY), (bY, -bY)
  // forward: slots (row bit, column bit) = (alpha, zeta) afterwards
  __device__ __forceinline__ void fwd(float2& x00, float2& x01, float2& x10, float2& x11) const {
    const float2 cI = add2(x00, x11), cZ = sub2(x00, x11), cX = add2(x01, x10), v = sub2(x01, x10);  // c_Y = i v
    const float2 t = mul2(bI, cI), s = mul2(bX, cX), sv = swap2(v);
    const float2 e0 = fma2(bZ, cZ, t), e1 = fma2(nbZ, cZ, t);     // bI cI +- bZ cZ
    const float2 o0 = fma2(mbY, sv, s), o1 = fma2(pbY, sv, s);    // bX cX +- i bY v
    x00 = add2(e0, o0);
    x01 = add2(e1, o1);
    x10 = sub2(e0, o0);
    x11 = sub2(e1, o1);
  }
  // adjoint: from g in slots (alpha, zeta) to G = sum_a g_a M_a (the transpose of fwd, as mode_adj)
  __device__ __forceinline__ void adj(float2& x00, float2& x01, float2& x10, float2& x11) const {
    const float2 s0 = add2(x00, x10), s1 = add2(x01, x11), d0 = sub2(x00, x10), d1 = sub2(x01, x11);
    const float2 t = mul2(bI, add2(s0, s1)), s = mul2(bX, add2(d0, d1)), sv = swap2(sub2(d0, d1));
    const float2 cZ = sub2(s0, s1);
    const float2 icY = mul2(mbY, sv);  // i bY (d0 - d1)
    x00 = fma2(bZ, cZ, t);
    x11 = fma2(nbZ, cZ, t);
    x10 = add2(s, icY);
    x01 = sub2(s, icY);
  }
};

// Both qubits of a register block: k = (row bit b, row bit b+1), l = (column bit b, column bit b+1).
template <bool ADJ, class MAP> __device__ __forceinline__ void apply_pair(const MAP& m, float2 (&x)[4][4]) {
#pragma unroll
  for (int hk = 0; hk < 2; ++hk)
#pragma unroll
    for (int hl = 0; hl < 2; ++hl) {
      if (ADJ) m.adj(x[2 * hk][2 * hl], x[2 * hk][2 * hl + 1], x[2 * hk + 1][2 * hl], x[2 * hk + 1][2 * hl + 1]);
      else m.fwd(x[2 * hk][2 * hl], x[2 * hk][2 * hl + 1], x[2 * hk + 1][2 * hl], x[2 * hk + 1][2 * hl + 1]);
    }
#pragma unroll
  for (int lk = 0; lk < 2; ++lk)
#pragma unroll
    for (int ll = 0; ll < 2; ++ll) {
      if (ADJ) m.adj(x[lk][ll], x[lk][ll + 2], x[lk + 2][ll], x[lk + 2][ll + 2]);
      else m.fwd(x[lk][ll], x[lk][ll + 2], x[lk + 2][ll], x[lk + 2][ll + 2]);
    }
}

// Swizzled shared-memory index of complex element (i, j) of a 64 x 64 tile: column bits 4, 5 are
// folded onto bits 0, 1 and row bits 0, 1 onto bits 2, 3 (conflict-free for the three thread maps).
__device__ __forceinline__ int sw_idx(int i, int j) { return i * kTile + (j ^ ((j >> 4) & 3) ^ ((i & 3) << 2)); }

// Thread maps of the three sweeps (rows i, columns j of register (k, l)):
//   A: t = kappa + 16 rho:                        i = 4 rho + k,               j = 4 kappa + l
//   B: t = j01 + 4 i01 + 16 j45 + 64 i45:         i = i01 + 4 k + 16 i45,      j = j01 + 4 l + 16 j45
//   C: t = interleave(i03, j03):                  i = i03 + 16 k,              j = j03 + 16 l
__device__ __forceinline__ void map_B(int t, int& i0, int& j0) {
  i0 = ((t >> 2) & 3) + 16 * ((t >> 6) & 3);
  j0 = (t & 3) + 16 * ((t >> 4) & 3);
}

template <bool XOR> __device__ __forceinline__ long long slot(int I, int J, int nb) {
  return XOR ? (long long)((I ^ J) * nb + J) : (long long)(I * nb + J);
}

// Outcome digit of qubit b from its canonical slot bits (i_b, j_b): out[2 i + j], the four 2-bit
// outcomes packed in one word.
__device__ __forceinline__ int digit(unsigned out, int i, int j) { return (int)(out >> (2 * (2 * i + j))) & 3; }

struct Out4 { unsigned bits; };

// 16-byte load of two complex values (data read once: cached in L2 only).
__device__ __forceinline__ float4 ld4(const float2* p) {
  float4 v;
  asm("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

// ---------------------------------------------------------------- pass 1, forward
template <class MAP, bool XOR>
__global__ void __launch_bounds__(kLoThreads, 4) k_lo_fwd_fast(const float2* __restrict__ X, float* __restrict__ W,
                                                                 int N, MAP m, Out4 outmap, const void* const* tab) {
  __shared__ float2 Z[kTile * kTile];
  rebind(tab, X, W);
  pdl_trigger();
  const long long d = 1LL << N;
  const int nb = (int)(d >> 6);
  int I, J;
  tri_decode(blockIdx.x, I, J);
  const int t = threadIdx.x;
  float2 x[4][4];
  pdl_wait();
  after_wait(X, W);
  {  // sweep A: the 4 x 4 block straight from X (rows 4 rho + k, columns 4 kappa + l)
    const int kap = t & 15, rho = t >> 4;
    const float2* src = X + ((long long)I * kTile + 4 * rho) * d + (long long)J * kTile + 4 * kap;
    float4 a[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k][0] = ld4(src + k * d);
      a[k][1] = ld4(src + k * d + 2);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      x[k][0] = f2(a[k][0].x, a[k][0].y);
      x[k][1] = f2(a[k][0].z, a[k][0].w);
      x[k][2] = f2(a[k][1].x, a[k][1].y);
      x[k][3] = f2(a[k][1].z, a[k][1].w);
    }
    if (I == J && kap >= rho) {  // diagonal tile: entries above the diagonal from the conjugate of the mirror
      const float2* mir = X + ((long long)I * kTile + 4 * kap) * d + (long long)I * kTile + 4 * rho;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float4 b0 = ld4(mir + l * d);
        const float4 b1 = ld4(mir + l * d + 2);
        const float2 row[4] = {f2(b0.x, b0.y), f2(b0.z, b0.w), f2(b1.x, b1.y), f2(b1.z, b1.w)};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (4 * rho + k < 4 * kap + l) x[k][l] = f2(row[k].x, -row[k].y);
      }
    }
    apply_pair<false>(m, x);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) Z[sw_idx(4 * rho + k, 4 * kap + l)] = x[k][l];
  }
  __syncthreads();
  {  // sweep B: qubits 2, 3
    int i0, j0;
    map_B(t, i0, j0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) x[k][l] = Z[sw_idx(i0 + 4 * k, j0 + 4 * l)];
    apply_pair<false>(m, x);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) Z[sw_idx(i0 + 4 * k, j0 + 4 * l)] = x[k][l];
  }
  __syncthreads();
  // sweep C: qubits 4, 5, then the outputs: 32 consecutive outcomes per warp and register
  const int i03 = (int)compact_bits((uint32_t)t >> 1), j03 = (int)compact_bits((uint32_t)t);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) x[k][l] = Z[sw_idx(i03 + 16 * k, j03 + 16 * l)];
  apply_pair<false>(m, x);
  const unsigned out = outmap.bits;
  int base = 0;
#pragma unroll
  for (int b = 0; b < 4; ++b) base += digit(out, (i03 >> b) & 1, (j03 >> b) & 1) << (2 * b);
  float* wre = W + (slot<XOR>(I, J, nb) << kLogSS);
  float* wim = W + (slot<XOR>(J, I, nb) << kLogSS);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int al = base + (digit(out, k & 1, l & 1) << 8) + (digit(out, k >> 1, l >> 1) << 10);
      if (I == J) {
        wre[al] = x[k][l].x;
      } else if (XOR) {  // the pair slots hold Re + Im and Re - Im
        wre[al] = x[k][l].x + x[k][l].y;
        wim[al] = x[k][l].x - x[k][l].y;
      } else {
        wre[al] = x[k][l].x;
        wim[al] = x[k][l].y;
      }
    }
}

// ---------------------------------------------------------------- pass 1, adjoint
template <class MAP, bool XOR>
__global__ void __launch_bounds__(kLoThreads, 4) k_lo_adj_fast(const float* Wadj, float2* __restrict__ G,
                                                                 int N, MAP m, Out4 outmap, unsigned int* amax,
                                                                 const void* const* tab) {
  __shared__ float2 Z[kTile * kTile];
  rebind(tab, Wadj, G, amax);
  const long long d = 1LL << N;
  const int nb = (int)(d >> 6);
  int I, J;
  tri_decode(blockIdx.x, I, J);
  const int t = threadIdx.x;
  float2 x[4][4];
  pdl_wait();
  after_wait(Wadj, G, amax);
  const int i03 = (int)compact_bits((uint32_t)t >> 1), j03 = (int)compact_bits((uint32_t)t);
  {  // sweep C: the packed adjoint of the tile pair, then qubits 4, 5
    const unsigned out = outmap.bits;
    int base = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) base += digit(out, (i03 >> b) & 1, (j03 >> b) & 1) << (2 * b);
    const float* wre = Wadj + (slot<XOR>(I, J, nb) << kLogSS);
    const float* wim = Wadj + (slot<XOR>(J, I, nb) << kLogSS);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int al = base + (digit(out, k & 1, l & 1) << 8) + (digit(out, k >> 1, l >> 1) << 10);
        const float a = ld_dep(wre + al), b = I != J ? ld_dep(wim + al) : 0.f;
        x[k][l] = (I != J && XOR) ? f2(0.5f * (a + b), 0.5f * (a - b)) : f2(a, b);
      }
    apply_pair<true>(m, x);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) Z[sw_idx(i03 + 16 * k, j03 + 16 * l)] = x[k][l];
  }
  __syncthreads();
  {  // sweep B: qubits 2, 3
    int i0, j0;
    map_B(t, i0, j0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) x[k][l] = Z[sw_idx(i0 + 4 * k, j0 + 4 * l)];
    apply_pair<true>(m, x);
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int l = 0; l < 4; ++l) Z[sw_idx(i0 + 4 * k, j0 + 4 * l)] = x[k][l];
  }
  __syncthreads();
  // sweep A: qubits 0, 1, then the tile of G (and its conjugate transpose in the mirrored tile)
  const int kap = t & 15, rho = t >> 4;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) x[k][l] = Z[sw_idx(4 * rho + k, 4 * kap + l)];
  apply_pair<true>(m, x);
  float mx = 0.f;
  float2* dst = G + ((long long)I * kTile + 4 * rho) * d + (long long)J * kTile + 4 * kap;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    *reinterpret_cast<float4*>(dst + k * d) = make_float4(x[k][0].x, x[k][0].y, x[k][1].x, x[k][1].y);
    *reinterpret_cast<float4*>(dst + k * d + 2) = make_float4(x[k][2].x, x[k][2].y, x[k][3].x, x[k][3].y);
#pragma unroll
    for (int l = 0; l < 4; ++l) mx = fmaxf(mx, fmaxf(fabsf(x[k][l].x), fabsf(x[k][l].y)));
  }
  if (I != J) {
    float2* mir = G + ((long long)J * kTile + 4 * kap) * d + (long long)I * kTile + 4 * rho;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      *reinterpret_cast<float4*>(mir + l * d) = make_float4(x[0][l].x, -x[0][l].y, x[1][l].x, -x[1][l].y);
      *reinterpret_cast<float4*>(mir + l * d + 2) = make_float4(x[2][l].x, -x[2][l].y, x[3][l].x, -x[3][l].y);
    }
  }
  if (amax) block_absmax_to(mx, amax);  // the mirrored tile holds the same magnitudes
}

// ---------------------------------------------------------------- pass 2 (structured POVMs)
// Walsh-Hadamard transform over the register index, on packed pairs (two low outcomes at once).
template <int NB> __device__ __forceinline__ void wht2(float2 (&v)[NB]) {
#pragma unroll
  for (int hb = 1; hb < NB; hb <<= 1) {
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      if (r & hb) continue;
      const float2 a = v[r], b = v[r | hb];
      v[r] = add2(a, b);
      v[r | hb] = sub2(a, b);
    }
  }
}

__host__ __device__ constexpr int msb_c(int x) { return x <= 1 ? 0 : 1 + msb_c(x >> 1); }
__host__ __device__ constexpr int ctz_c(int x) { return (x & 1) ? 0 : 1 + ctz_c(x >> 1); }

struct HiParams {
  float beta[4];
  unsigned out;  // out[s] at bits 2s, 2s + 1
};

// Likelihood term of one outcome (Sec. 3.1), branch-free: acc += f log2 q (the caller scales by ln 2),
// returns g = dL/dq.  A term with q below the smallest normal number and f > 0 is clamped: the constant
// -f log q_min, nothing added to g (f = 0 terms add 0 to both).
__device__ __forceinline__ float nll_term(float q, float fk, float gconst, float& acc, unsigned int& nclamp) {
  const bool ok = q >= FLT_MIN;
  const float qs = ok ? q : FLT_MIN;
  acc = fmaf(fk, __log2f(qs), acc);
  nclamp += (!ok && fk > 0.f) ? 1u : 0u;
  return ok ? gconst - __fdividef(fk, q) : gconst;
}

// One CTA per 2 kCP consecutive low outcomes; thread (cp, v) handles the outcome pair a0 + 2 cp,
// a0 + 2 cp + 1 (packed pairs) and the index v (the diagonal x, later zeta) of NB.
// Pass-1 layout: slot (x, r) = W_(r^x, r) holds Re + Im of the lower entry of the pair (r < r^x),
// Re - Im of it (r > r^x), the real diagonal (x = 0): the real sequence whose transform over r gives
// the Pauli coefficients up to the sign of (-i)^|x & z| (see povm_pauli.cu).
// MODE 0: q into p.  MODE 1: likelihood (loss -> scal[2]) and, with adjoint, the transformed adjoint
// of the high qubits into Wadj (slot (x, r) = the transform over z back to r; pass-1 adjoint splits it
// into Re = (a + b) / 2 and Im = (a - b) / 2 of the pair).
// Outcome pairs per CTA: 8 (two CTAs per SM at NB = 32, so that one CTA's loads overlap the other's
// arithmetic, and the forward map's 256 CTAs cover every SM where 16 pairs left 24 of 152 idle); at
// least 16 when NB = 2 so that a CTA is a whole warp.
template <int NB, int MODE> constexpr int cta_pairs() { return NB < 4 ? 16 : 8; }

// BATCH: the grouped variant (a separate instantiation, so that the single-tomography kernel keeps its
// register allocation)
template <int NB, int MODE, int kCP = cta_pairs<NB, MODE>(), bool BATCH = false>
__global__ void __launch_bounds__(kCP * NB, (NB == 32 && kCP == 8) ? 2 : 1) k_hi_fast(const float* W, float* __restrict__ p,
                                                      const float* __restrict__ f, double* scal, float* __restrict__ Wadj,
                                                      double* partials, unsigned int* counter, unsigned int* flags,
                                                      HiParams P, int adjoint, const void* const* tab) {
  constexpr int H = msb_c(NB);
  if constexpr (BATCH) rebind(tab, W, p, f, scal, Wadj, partials, counter, flags);
  extern __shared__ __align__(16) float2 smp[];
  float2* fac = smp;            // [x][z]: the sign of (-i)^|x & z| times prod_k beta_(x_k, z_k), twice
  float2* buf = smp + NB * NB;  // [x][zeta][cp]: the transpose between the two halves
  __shared__ double red[32];
  pdl_trigger();
  static_assert((kCP * NB) % 32 == 0, "a CTA is a whole number of warps");
  // transpose buffer: [x][zeta][cp] with the x stride padded by 64 bytes when a half-warp spans two x
  constexpr int XS = NB * kCP + (kCP < 16 ? kCP : 0);
  const int t = threadIdx.x, cp = t % kCP, wv = t / kCP;
  const long long a0 = (long long)blockIdx.x * (2 * kCP) + 2 * cp;
  for (int e = t; e < NB * NB; e += blockDim.x) {
    const int xx = e / NB, zz = e % NB;
    float v = (__popc(xx & zz) & 2) ? -1.f : 1.f;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int xk = (xx >> k) & 1, zk = (zz >> k) & 1;
      v *= P.beta[xk ? (zk ? 2 : 1) : (zk ? 3 : 0)];
    }
    fac[e] = f2(v, v);
  }
  __syncthreads();
  pdl_wait();
  after_wait(f);
  // ---- thread (cp, x = wv): the sequence of the diagonal x, transformed r -> z -> zeta
  float2 w[NB];
  {
    const float* src = W + ((long long)(wv * NB) << kLogSS) + a0;
#pragma unroll
    for (int r = 0; r < NB; ++r) w[r] = ld_dep2(src + ((long long)r << kLogSS));
  }
  wht2<NB>(w);
#pragma unroll
  for (int z = 0; z < NB; ++z) w[z] = mul2(w[z], fac[wv * NB + z]);
  wht2<NB>(w);
#pragma unroll
  for (int z = 0; z < NB; ++z) buf[wv * XS + z * kCP + cp] = w[z];
  __syncthreads();
  // ---- thread (cp, zeta = wv): transform over x
  // outcome of (alpha, zeta): digits out[2 alpha_k + zeta_k]
  // base: the outcome of alpha = 0; dk: the change of the outcome when alpha_k flips to 1 (scalars, not
  // an array, so that they stay in registers when indexed by unrolled loop counters)
  int base = 0, d0 = 0, d1 = 0, d2 = 0, d3 = 0, d4 = 0;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const int zk = (wv >> k) & 1;
    const int o0 = digit(P.out, 0, zk), o1 = digit(P.out, 1, zk);
    base += o0 << (2 * k);
    const int dk = (o1 - o0) << (2 * k);
    if (k == 0) d0 = dk;
    if (k == 1) d1 = dk;
    if (k == 2) d2 = dk;
    if (k == 3) d3 = dk;
    if (k == 4) d4 = dk;
  }
  auto delta = [&](int k) { return k == 0 ? d0 : k == 1 ? d1 : k == 2 ? d2 : k == 3 ? d3 : d4; };
  // The outcomes of registers alpha are visited in Gray-code order g(i) = i ^ (i >> 1): consecutive ones
  // differ in one digit, so each offset is one addition away from the previous one.
  // MODE 1: the frequencies of this thread's outcomes; the first NPF of them are in flight during the
  // transform over x (all of them would not fit in the register budget at NB = 32)
  constexpr int NF = MODE == 1 ? NB : 1, NPF = NB >= 32 ? NB / 4 : NB;
  float2 fv[NF];
  // f arrives permuted (povm_permute_f): the pair of Gray step i of thread t of CTA b at float2 index
  // (b NB + i) (kCP NB) + t, so that a CTA reads one contiguous block.
  const float2* fp = reinterpret_cast<const float2*>(f) + (long long)blockIdx.x * NB * (kCP * NB) + t;
  auto load_f = [&](int i) { fv[i ^ (i >> 1)] = __ldg(fp + (long long)i * (kCP * NB)); };
  if (MODE == 1) {
#pragma unroll
    for (int i = 0; i < NPF; ++i) load_f(i);
  }
#pragma unroll
  for (int x = 0; x < NB; ++x) w[x] = buf[x * XS + wv * kCP + cp];
  wht2<NB>(w);
  if (MODE == 1) {
#pragma unroll
    for (int i = NPF; i < NB; ++i) load_f(i);
  }
  if (MODE == 0) {
    int off = base;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      *reinterpret_cast<float2*>(p + ((long long)off << kLogSS) + a0) = w[i ^ (i >> 1)];
      if (i + 1 < NB) {
        const int k = ctz_c(i + 1);
        off += ((((i + 1) ^ ((i + 1) >> 1)) >> k) & 1) ? delta(k) : -delta(k);
      }
    }
    return;
  }
  // L = -sum f log q + (sum f) log Tr X;  g_k = -f_k / q_k + sum f / Tr X
  const double tX = scal[0], sumf = scal[1];
  const float gconst = (float)(sumf / tX);
  float acc = 0.f;
  unsigned int nclamp = 0;
#pragma unroll
  for (int al = 0; al < NB; ++al)
    w[al] = f2(nll_term(w[al].x, fv[al].x, gconst, acc, nclamp), nll_term(w[al].y, fv[al].y, gconst, acc, nclamp));
  if (nclamp) atomicAdd(flags, nclamp);
  const double accd = warp_sum((double)acc * 0.69314718055994530942);  // log2 -> natural log
  if ((t & 31) == 0) red[t >> 5] = accd;
  if (adjoint) {
    wht2<NB>(w);      // alpha -> x
    __syncthreads();  // every thread has read buf
#pragma unroll
    for (int x = 0; x < NB; ++x) buf[x * XS + wv * kCP + cp] = w[x];
    __syncthreads();
    // ---- thread (cp, x = wv) again: zeta -> z, scale, z -> r
#pragma unroll
    for (int z = 0; z < NB; ++z) w[z] = buf[wv * XS + z * kCP + cp];
    wht2<NB>(w);
#pragma unroll
    for (int z = 0; z < NB; ++z) w[z] = mul2(w[z], fac[wv * NB + z]);
    wht2<NB>(w);
    float* dst = Wadj + ((long long)(wv * NB) << kLogSS) + a0;
#pragma unroll
    for (int r = 0; r < NB; ++r) *reinterpret_cast<float2*>(dst + ((long long)r << kLogSS)) = w[r];
  }
  __syncthreads();
  const int nwarps = (int)(blockDim.x >> 5);
  if (t < 32) {
    double v = t < nwarps ? red[t] : 0.0;
    v = warp_sum(v);
    if (t == 0) partials[blockIdx.x] = v;
  }
  if (last_block_arrived(counter)) {
    if (t < 32) {
      double v = 0.0;
      for (int b = t; b < (int)gridDim.x; b += 32) v += partials[b];
      v = warp_sum(v);
      if (t == 0) {
        scal[2] = -v + sumf * log(tX);
        *counter = 0u;
      }
    }
  }
}

// f in the order of the likelihood pass: one thread per pair of outcomes (a_hi, a_lo, a_lo + 1) of f,
// read contiguously, written to the slot (b NB + i) (kCP NB) + t of the pass-2 thread t = cp + kCP zeta of
// CTA b = a_lo / (2 kCP) that loads it at Gray step i (alpha = i ^ (i >> 1)).
template <int NB, int kCP>
__global__ void __launch_bounds__(256) k_permute_f(const float2* __restrict__ f, float2* __restrict__ fp,
                                                    unsigned inv_out, long long pairs) {
  constexpr int H = msb_c(NB);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < pairs; e += (long long)gridDim.x * blockDim.x) {
    const int a_hi = (int)(e >> (kLogSS - 1));
    const int alo2 = (int)(e & ((1 << (kLogSS - 1)) - 1));  // a_lo / 2
    const int b = alo2 / kCP, cp = alo2 % kCP;
    int al = 0, ze = 0;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int s = (int)(inv_out >> (2 * ((a_hi >> (2 * k)) & 3))) & 3;  // canonical slot 2 alpha + zeta of digit k
      al |= (s >> 1) << k;
      ze |= (s & 1) << k;
    }
    int i = al;  // inverse Gray code
#pragma unroll
    for (int sh = 1; sh < NB; sh <<= 1) i ^= i >> sh;
    fp[((long long)b * NB + i) * (kCP * NB) + cp + kCP * ze] = f[e];
  }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, size_t smem, cudaStream_t s, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

MapStruct map_struct(const PovmPlan& P) {
  const float bI = P.beta[0], bX = P.beta[1], bY = P.beta[2], bZ = P.beta[3];
  MapStruct m;
  m.bI = make_float2(bI, bI);
  m.bZ = make_float2(bZ, bZ);
  m.nbZ = make_float2(-bZ, -bZ);
  m.bX = make_float2(bX, bX);
  m.mbY = make_float2(-bY, bY);
  m.pbY = make_float2(bY, -bY);
  return m;
}

MapGeneric map_generic(const PovmPlan& P) {
  MapGeneric m;
  for (int a = 0; a < 4; ++a)
    for (int mu = 0; mu < 4; ++mu) m.b[a][mu] = make_float2(P.B.b[a][mu], P.B.b[a][mu]);
  return m;
}

Out4 out_of(const PovmPlan& P) {
  Out4 o{0u};
  for (int i = 0; i < 4; ++i) o.bits |= (unsigned)P.out[i] << (2 * i);
  return o;
}

template <int NB, int MODE>
cudaError_t launch_hi(const Dims& D, const float* W, float* p, const float* f, double* scal, float* Wadj,
                      double* partials, unsigned int* counter, unsigned int* flags, const PovmPlan& P, bool adjoint,
                      cudaStream_t s) {
  constexpr int kCP = cta_pairs<NB, MODE>();
  const size_t sm = (size_t)(NB * NB + NB * (NB * kCP + (kCP < 16 ? kCP : 0))) * sizeof(float2);
  BatchArgs ba;
  if (batch_take(ba, {W, p, f, scal, Wadj, partials, counter, flags})) return cudaSuccess;
  const void* fn = ba.tab ? (const void*)k_hi_fast<NB, MODE, kCP, true> : (const void*)k_hi_fast<NB, MODE, kCP, false>;
  cudaError_t e = ensure_dynamic_smem(fn, sm);
  if (e != cudaSuccess) return e;
  HiParams hp;
  for (int i = 0; i < 4; ++i) hp.beta[i] = P.beta[i];
  hp.out = out_of(P).bits;
  int adj = adjoint ? 1 : 0;
  const unsigned blocks = (unsigned)((1LL << kLogSS) / (2 * kCP));
  if (MODE == 1 && blocks > (unsigned)kPartialBlocks * kPartialStride) return cudaErrorInvalidConfiguration;
  void* args[] = {(void*)&W, (void*)&p, (void*)&f, (void*)&scal, (void*)&Wadj, (void*)&partials, (void*)&counter,
                  (void*)&flags, (void*)&hp, (void*)&adj, (void*)&ba.tab};
  return launch_pdl(fn, dim3(blocks, 1, ba.nz), dim3(kCP * NB), sm, s, args);
}

template <int MODE>
cudaError_t dispatch_hi(const Dims& D, const float* W, float* p, const float* f, double* scal, float* Wadj,
                        double* partials, unsigned int* counter, unsigned int* flags, const PovmPlan& P, bool adjoint,
                        cudaStream_t s) {
  switch (D.nb) {
    case 2: return launch_hi<2, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, P, adjoint, s);
    case 4: return launch_hi<4, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, P, adjoint, s);
    case 8: return launch_hi<8, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, P, adjoint, s);
    case 16: return launch_hi<16, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, P, adjoint, s);
    case 32: return launch_hi<32, MODE>(D, W, p, f, scal, Wadj, partials, counter, flags, P, adjoint, s);
  }
  return cudaErrorInvalidValue;
}

template <int NB>
cudaError_t launch_permute(const float* f, float* fperm, const PovmPlan& P, long long n, cudaStream_t s) {
  constexpr int kCP = cta_pairs<NB, 1>();
  unsigned inv = 0;  // canonical slot of outcome a at bits 2a, 2a + 1
  for (int sl = 0; sl < 4; ++sl) inv |= (unsigned)sl << (2 * P.out[sl]);
  const long long pairs = n / 2;
  long long blocks = (pairs + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_permute_f<NB, kCP><<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float2*>(f),
                                                        reinterpret_cast<float2*>(fperm), inv, pairs);
  return cudaGetLastError();
}

}  // namespace

bool povm_needs_fperm(const PovmPlan& P) { return P.structured != 0; }

cudaError_t povm_permute_f(const Dims& D, const float* f, float* fperm, const PovmPlan& P, cudaStream_t s) {
  switch (D.nb) {
    case 2: return launch_permute<2>(f, fperm, P, D.n, s);
    case 4: return launch_permute<4>(f, fperm, P, D.n, s);
    case 8: return launch_permute<8>(f, fperm, P, D.n, s);
    case 16: return launch_permute<16>(f, fperm, P, D.n, s);
    case 32: return launch_permute<32>(f, fperm, P, D.n, s);
  }
  return cudaErrorInvalidValue;
}

PovmPlan make_povm_plan(const PovmB<double>& Bd) {
  PovmPlan P;
  for (int a = 0; a < 4; ++a)
    for (int m = 0; m < 4; ++m) P.B.b[a][m] = (float)Bd.b[a][m];
  for (int s = 0; s < 4; ++s) P.out[s] = s;
  P.structured = 0;
  double beta[4];
  for (int m = 0; m < 4; ++m) beta[m] = fabs(Bd.b[0][m]);
  for (int m = 0; m < 4; ++m)
    if (!(beta[m] > 0.0)) return P;
  int out[4] = {-1, -1, -1, -1};
  for (int a = 0; a < 4; ++a) {
    for (int m = 0; m < 4; ++m)
      if (fabs(fabs(Bd.b[a][m]) - beta[m]) > 1e-12 * beta[m]) return P;
    if (!(Bd.b[a][0] > 0.0)) return P;
    const int al = Bd.b[a][1] < 0.0 ? 1 : 0;  // mu = X: (x, z) = (1, 0)
    const int ze = Bd.b[a][3] < 0.0 ? 1 : 0;  // mu = Z: (0, 1)
    if ((Bd.b[a][2] < 0.0) != ((al ^ ze) == 1)) return P;  // mu = Y: (1, 1)
    if (out[2 * al + ze] != -1) return P;
    out[2 * al + ze] = a;
  }
  P.structured = 1;
  for (int m = 0; m < 4; ++m) P.beta[m] = (float)beta[m];
  for (int s = 0; s < 4; ++s) P.out[s] = out[s];
  return P;
}

bool povm_fast_ok(const Dims& D) { return D.g == 6 && D.N >= 7 && D.N <= 11 && D.C > 0; }

cudaError_t povm_lo_fwd_fast(const Dims& D, const float2* X, float* W, const PovmPlan& P, cudaStream_t s) {
  const unsigned tiles = (unsigned)(D.nb * (D.nb + 1) / 2);
  const Out4 o = out_of(P);
  BatchArgs ba;
  if (batch_take(ba, {X, W})) return cudaSuccess;
  if (P.structured) {
    const MapStruct m = map_struct(P);
    return launch_dep(k_lo_fwd_fast<MapStruct, true>, dim3(tiles, 1, ba.nz), dim3(kLoThreads), 0, s, X, W, D.N, m, o,
                      ba.tab);
  } else {
    const MapGeneric m = map_generic(P);
    return launch_dep(k_lo_fwd_fast<MapGeneric, false>, dim3(tiles, 1, ba.nz), dim3(kLoThreads), 0, s, X, W, D.N, m,
                      o, ba.tab);
  }
}

cudaError_t povm_fwd_fast(const Dims& D, const float2* X, float* W, float* p, const PovmPlan& P, cudaStream_t s) {
  cudaError_t e = povm_lo_fwd_fast(D, X, W, P, s);
  if (e != cudaSuccess) return e;
  if (P.structured)
    return dispatch_hi<0>(D, W, p, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, P, false, s);
  return povm_hi_fwd_pauli<float>(D, W, p, P.B, s);
}

cudaError_t povm_hi_nll_fast(const Dims& D, const float* W, const float* f, double* scal, float* Wadj,
                             double* partials, unsigned int* counter, unsigned int* flags, const PovmPlan& P,
                             bool adjoint, cudaStream_t s) {
  if (P.structured)
    return dispatch_hi<1>(D, W, nullptr, f, scal, Wadj, partials, counter, flags, P, adjoint, s);
  return povm_hi_nll_pauli<float>(D, W, f, scal, Wadj, partials, counter, flags, P.B, adjoint, s);
}

cudaError_t povm_lo_adj_fast(const Dims& D, const float* Wadj, float2* G, const PovmPlan& P, unsigned int* amax,
                             cudaStream_t s) {
  const unsigned tiles = (unsigned)(D.nb * (D.nb + 1) / 2);
  const Out4 o = out_of(P);
  BatchArgs ba;
  if (batch_take(ba, {Wadj, G, amax})) return cudaSuccess;
  if (P.structured) {
    const MapStruct m = map_struct(P);
    void* args[] = {(void*)&Wadj, (void*)&G, (void*)&D.N, (void*)&m, (void*)&o, (void*)&amax, (void*)&ba.tab};
    return launch_pdl((const void*)k_lo_adj_fast<MapStruct, true>, dim3(tiles, 1, ba.nz), dim3(kLoThreads), 0, s,
                      args);
  }
  const MapGeneric m = map_generic(P);
  k_lo_adj_fast<MapGeneric, false><<<dim3(tiles, 1, ba.nz), kLoThreads, 0, s>>>(Wadj, G, D.N, m, o, amax, ba.tab);
  return cudaGetLastError();
}

}  // namespace qst
