// P-order absolute projection of Sec. 3.2 (eq. abs_P):
//   T = Q Lambda Q^dag,   X = Q |Lambda|^P Q^dag,   rho = X / Tr X,
// and its backward (Daleckii-Krein): with s_i = |lambda_i|^P,
//   dL/dT = Q (D o (Q^dag G Q)) Q^dag,  D_ij = (s_i - s_j) / (lambda_i - lambda_j),  D_ii = s'(lambda_i),
// where G = dL/dX comes from the adjoint POVM map.
//
// The eigendecomposition is a cyclic two-sided Jacobi method for complex Hermitian matrices (d = 2^N) in the
// XOR ordering: a sweep is the d - 1 rounds m = 1 .. d - 1, round m rotating the d / 2 disjoint pairs
// {x, x ^ m} at once.  For a pair (p, q) with c = A_pq = |c| e^{i phi}, the 2 x 2 block is first made real by
// diag(1, e^{-i phi}) and then zeroed by the real rotation of Golub and Van Loan (tan theta =
// sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / 2|c|).  The three rounds a, b, a ^ b of a
// 2-dimensional subspace of GF(2)^N all act within its cosets {x, x ^ a, x ^ b, x ^ a ^ b}, so the rounds of a
// sweep are grouped by a partition of the nonzero vectors of GF(2)^N into such subspaces (for odd N, all but
// four single rounds), and one kernel applies the three rounds of a subspace at once: each thread owns the
// 4 x 4 block (rows of one coset) x (columns of another) of A and of V, multiplies it by the cosets' 4 x 4
// unitaries, and every entry is read and written once per pass (double-buffered); V accumulates the
// rotations, V <- V U.  At N = 11 a sweep is 685 passes (2047 rounds), at N = 12 1365 (4095).
#include <float.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "impl.h"

namespace qst {

namespace {

template <class R> __device__ __forceinline__ R tiny_normal();
template <> __device__ __forceinline__ float tiny_normal<float>() { return FLT_MIN; }
template <> __device__ __forceinline__ double tiny_normal<double>() { return DBL_MIN; }
template <class R> __device__ __forceinline__ R eps_of();
template <> __device__ __forceinline__ float eps_of<float>() { return FLT_EPSILON; }
template <> __device__ __forceinline__ double eps_of<double>() { return DBL_EPSILON; }

// Rotation zeroing entry (p, q) of the Hermitian 2 x 2 block [[a, c], [conj c, b]] (a, b real, c = |c| e^{i phi}):
// R = [[cs, sn], [-e^{-i phi} sn, e^{-i phi} cs]] in the order (p, q).
template <class R> struct Rot2 {
  R cs, sn;
  cx_t<R> emph;  // e^{-i phi}
};

template <class R> __device__ __forceinline__ Rot2<R> rotation_for(R a, R b, cx_t<R> c) {
  Rot2<R> o;
  o.cs = R(1);
  o.sn = R(0);
  o.emph = cmake<cx_t<R>>(R(1), R(0));
  // |c| by hypot (no underflow of c.x^2 once the entry is tiny), and no rotation for entries that are
  // negligible against the diagonal: otherwise e^{i phi} = c / |c| loses unit modulus and the
  // accumulated eigenvectors drift from unitarity.
  const R r = hypot(c.x, c.y);
  if (r > eps_of<R>() * R(1e-4) * (fabs(a) + fabs(b)) && r > tiny_normal<R>() * R(1e8)) {
    const R tau = (b - a) / (R(2) * r);
    const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
    o.cs = R(1) / sqrt(R(1) + t * t);
    o.sn = t * o.cs;
    o.emph = cmake<cx_t<R>>(c.x / r, -c.y / r);
  }
  return o;
}

template <class V> __device__ __forceinline__ V cmul(V a, V b) { return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <class V> __device__ __forceinline__ V cmulc(V a, V b) { return cmake<V>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a) b

__device__ __forceinline__ int insert_zero(int x, int p) { return ((x >> p) << (p + 1)) | (x & ((1 << p) - 1)); }

// Coset number c of the pass's subspace: G = 2, {x, x ^ a}; G = 4, {x, x ^ a, x ^ b, x ^ a ^ b}, where the
// representative x has the pivot bits (plo, and phi for G = 4) clear and local index i = (bit 0: a, bit 1: b).
template <int G>
__device__ __forceinline__ void coset_of(int c, int a, int b, int plo, int phi, int (&e)[G]) {
  const int x = G == 2 ? insert_zero(c, plo) : insert_zero(insert_zero(c, plo), phi);
#pragma unroll
  for (int i = 0; i < G; ++i) e[i] = x ^ ((i & 1) ? a : 0) ^ ((i & 2) ? b : 0);
}

template <class R> __device__ __forceinline__ R lane_shfl(R v, int src, int width) {
  return __shfl_sync(0xffffffffu, v, src, width);
}
template <class R> __device__ __forceinline__ R lane_xor(R v, int m, int width) {
  return __shfl_xor_sync(0xffffffffu, v, m, width);
}
template <class R> __device__ __forceinline__ Rot2<R> rot_from_lane(const Rot2<R>& r, int src, int width) {
  Rot2<R> o;
  o.cs = lane_shfl(r.cs, src, width);
  o.sn = lane_shfl(r.sn, src, width);
  o.emph = cmake<cx_t<R>>(lane_shfl(r.emph.x, src, width), lane_shfl(r.emph.y, src, width));
  return o;
}

// X <- X R on columns (p, q) of one row x of B or U (R = [[cs, sn], [-e^{-i phi} sn, e^{-i phi} cs]]).
template <class R, int G>
__device__ __forceinline__ void rotate_cols(cx_t<R> (&x)[G], int p, int q, const Rot2<R>& r) {
  using V = cx_t<R>;
  const V rqp = cmake<V>(-r.emph.x * r.sn, -r.emph.y * r.sn), rqq = cmake<V>(r.emph.x * r.cs, r.emph.y * r.cs);
  const V xp = x[p], xq = x[q];
  x[p] = cadd(cmake<V>(xp.x * r.cs, xp.y * r.cs), cmul(xq, rqp));
  x[q] = cadd(cmake<V>(xp.x * r.sn, xp.y * r.sn), cmul(xq, rqq));
}

// The pass's rotations on one coset, in the order of its rounds (round s pairs local i with i ^ s,
// s = 1 .. G - 1), each computed from the 2 x 2 principal blocks of the coset's G x G principal block B of A
// after the rounds before it: U = R_1 ... R_{G-1}, so that U^dag A[e, e] U is that block after the pass.
// The G lanes of an aligned group take one coset; lane i holds row i of B and of U and returns row i of U.
// A pair's rotation is computed on its lower lane and broadcast; rows are exchanged by shuffles.
template <class R, int G>
__device__ __forceinline__ void coset_unitary_row(const cx_t<R>* __restrict__ A, int d, const int (&e)[G], int i,
                                                  cx_t<R> (&u)[G]) {
  using V = cx_t<R>;
  V b[G];
  int ei = e[0];
#pragma unroll
  for (int jj = 1; jj < G; ++jj)
    if (jj == i) ei = e[jj];
#pragma unroll
  for (int j = 0; j < G; ++j) {
    b[j] = A[(long long)ei * d + e[j]];
    u[j] = cmake<V>(i == j ? R(1) : R(0), R(0));
  }
#pragma unroll
  for (int s = 1; s < G; ++s) {
    R di = R(0);
    V cij = cmake<V>(R(0), R(0));
#pragma unroll
    for (int jj = 0; jj < G; ++jj) {
      if (jj == i) di = b[jj].x;
      if (jj == (i ^ s)) cij = b[jj];
    }
    const R dj = lane_xor(di, s, G);
    const Rot2<R> mine = rotation_for<R>(di, dj, cij);  // the pair's rotation where this lane is the lower one
    const int p1 = s == 1 ? 2 : 1;                      // lower index of the round's second pair (G = 4)
    const Rot2<R> r0 = rot_from_lane(mine, 0, G);
    const Rot2<R> r1 = G == 4 ? rot_from_lane(mine, p1, G) : r0;
    rotate_cols<R, G>(b, 0, s, r0);
    rotate_cols<R, G>(u, 0, s, r0);
    if (G == 4) {
      rotate_cols<R, G>(b, p1 % G, (p1 ^ s) % G, r1);
      rotate_cols<R, G>(u, p1 % G, (p1 ^ s) % G, r1);
    }
    // rows p, q of B <- R^dag rows (p, q): this lane's row with its partner's
    V o[G];
#pragma unroll
    for (int j = 0; j < G; ++j) o[j] = cmake<V>(lane_xor(b[j].x, s, G), lane_xor(b[j].y, s, G));
    const Rot2<R> r = (i == 0 || i == s) ? r0 : r1;
    const V rqp = cmake<V>(-r.emph.x * r.sn, -r.emph.y * r.sn), rqq = cmake<V>(r.emph.x * r.cs, r.emph.y * r.cs);
    const bool lower = i < (i ^ s);
#pragma unroll
    for (int j = 0; j < G; ++j) {
      // lower: conj(R_pp) b_p + conj(R_qp) b_q; upper: conj(R_pq) b_p + conj(R_qq) b_q (b_p the partner's)
      b[j] = lower ? cadd(cmake<V>(r.cs * b[j].x, r.cs * b[j].y), cmulc(rqp, o[j]))
                   : cadd(cmake<V>(r.sn * o[j].x, r.sn * o[j].y), cmulc(rqq, b[j]));
    }
  }
}

// The unitaries of a CTA's cosets in shared memory, entry (r, c) of coset slot s at [r][c][s] (consecutive
// cosets in consecutive words: the 16 column cosets a warp reads are in distinct banks).  FP32 keeps the
// forms the packed products take: u and (u.y, u.x) for products X U, conj(u) and (u.y, u.x) for U^dag X.
template <class R, int G> struct PassSmem {
  cx_t<R> uk[G][G][16], ul[G][G][16];
  cx_t<R> uk2[G][G][16], ul2[G][G][16];  // FP32: conj(u_k), (u_l.y, u_l.x); FP64: unused
  int ek[16][G];
};

// s += m u (complex) as two packed FP32 FMAs: (m.x, m.x) (u.x, u.y) + (-m.y, m.y) (u.y, u.x).
__device__ __forceinline__ float2 cmac2(float2 s, float2 mxx, float2 myn, float2 u, float2 usw) {
  return __ffma2_rn(myn, usw, __ffma2_rn(mxx, u, s));
}

// One pass: the rounds of the subspace {a, b, a ^ b} (G = 4) or the single round a (G = 2).  Every thread owns
// the G x G block (rows of coset k) x (columns of coset l) of A and of V, so each entry is read and written once
// per pass (double-buffered): A' = U_k^dag A U_l, V' = V U_l on rows e_k.  A thread loads its block of A
// first; meanwhile G warps form the unitaries of the CTA's 16 row and 16 column cosets from A.  Vi == NULL:
// no eigenvectors are accumulated; phi != NULL: the vector phi <- U^dag phi in place (the first block
// column, one thread per coset), so that after the sweeps phi = Q^dag phi_0.
template <class R, int G>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_jacobi_pass(const cx_t<R>* __restrict__ A, cx_t<R>* __restrict__ Ao,
                                                      const cx_t<R>* __restrict__ Vi, cx_t<R>* __restrict__ Vo,
                                                      cx_t<R>* __restrict__ phi, int d, int a, int b, int plo,
                                                      int phi_bit) {
  using V = cx_t<R>;
  constexpr int TP = 16;
  constexpr bool kF32 = sizeof(R) == 4;
  __shared__ PassSmem<R, G> sm;
  const int nc = d / G;
  const int k0 = blockIdx.y * TP, l0 = blockIdx.x * TP;
  const int t = threadIdx.x;
  const int kk = t / TP, ll = t % TP;
  const bool active = k0 + kk < nc && l0 + ll < nc;
  long long row[G];
  int col[G];
  {
    int er[G], ec[G];
    coset_of<G>(min(k0 + kk, nc - 1), a, b, plo, phi_bit, er);
    coset_of<G>(min(l0 + ll, nc - 1), a, b, plo, phi_bit, ec);
#pragma unroll
    for (int i = 0; i < G; ++i) {
      row[i] = (long long)er[i] * d;
      col[i] = ec[i];
    }
  }
  V M[G][G];
  if (active) {
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < G; ++j) M[i][j] = A[row[i] + col[j]];
  }
  if (t < 32 * G) {  // G warps: each aligned group of G lanes one coset, 16 of rows then 16 of columns
    const int grp = t / G, i = t % G;
    const bool isrow = grp < TP;
    const int slot = isrow ? grp : grp - TP;
    const int c0 = (isrow ? k0 : l0) + slot;
    const int c = c0 < nc ? c0 : nc - 1;  // every lane of these warps takes part in the shuffles
    int e[G];
    coset_of<G>(c, a, b, plo, phi_bit, e);
    V u[G];
    coset_unitary_row<R, G>(A, d, e, i, u);
    if (c0 < nc) {
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (isrow) {
          sm.uk[i][j][slot] = u[j];
          if (kF32) sm.uk2[i][j][slot] = cmake<V>(u[j].x, -u[j].y);
          if (i == 0) sm.ek[slot][j] = e[j];
        } else {
          sm.ul[i][j][slot] = u[j];
          if (kF32) sm.ul2[i][j][slot] = cmake<V>(u[j].y, u[j].x);
        }
      }
    }
  }
  __syncthreads();
  if (phi != nullptr && blockIdx.x == 0 && t < TP && k0 + t < nc) {
    V x[G];
#pragma unroll
    for (int i = 0; i < G; ++i) x[i] = phi[sm.ek[t][i]];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      V y = cmake<V>(R(0), R(0));
#pragma unroll
      for (int r = 0; r < G; ++r) y = cadd(y, cmulc(sm.uk[r][i][t], x[r]));
      phi[sm.ek[t][i]] = y;
    }
  }
  if (!active) return;
  if constexpr (kF32) {
    // T = M U_l (column c of M at a time), O = U_k^dag T (row r of T at a time), V' = V U_l
    float2 T[G][G];
#pragma unroll
    for (int r = 0; r < G; ++r)
#pragma unroll
      for (int j = 0; j < G; ++j) T[r][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < G; ++c) {
      float2 mxx[G], myn[G];
#pragma unroll
      for (int r = 0; r < G; ++r) {
        mxx[r] = make_float2(M[r][c].x, M[r][c].x);
        myn[r] = make_float2(-M[r][c].y, M[r][c].y);
      }
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const float2 u = sm.ul[c][j][ll], usw = sm.ul2[c][j][ll];
#pragma unroll
        for (int r = 0; r < G; ++r) T[r][j] = cmac2(T[r][j], mxx[r], myn[r], u, usw);
      }
    }
    // conj(u) t = (t.x, t.x) conj(u) + (t.y, t.y) (u.y, u.x)
    float2 O[G][G];
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < G; ++j) O[i][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < G; ++r) {
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const float2 cu = sm.uk2[r][i][kk];
        const float2 u = sm.uk[r][i][kk];
        const float2 usw = make_float2(u.y, u.x);
#pragma unroll
        for (int j = 0; j < G; ++j)
          O[i][j] = __ffma2_rn(make_float2(T[r][j].y, T[r][j].y), usw,
                               __ffma2_rn(make_float2(T[r][j].x, T[r][j].x), cu, O[i][j]));
      }
    }
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < G; ++j) Ao[row[i] + col[j]] = O[i][j];
    if (Vi == nullptr) return;
    asm volatile("" ::: "memory");  // V's loads after A's stores: A's and V's blocks are not live together
    float2 Vb[G][G], W[G][G];
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < G; ++j) {
        Vb[i][j] = Vi[row[i] + col[j]];
        W[i][j] = make_float2(0.f, 0.f);
      }
#pragma unroll
    for (int c = 0; c < G; ++c) {
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const float2 u = sm.ul[c][j][ll], usw = sm.ul2[c][j][ll];
#pragma unroll
        for (int i = 0; i < G; ++i)
          W[i][j] = cmac2(W[i][j], make_float2(Vb[i][c].x, Vb[i][c].x), make_float2(-Vb[i][c].y, Vb[i][c].y), u,
                          usw);
      }
    }
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < G; ++j) Vo[row[i] + col[j]] = W[i][j];
  } else {
    V T[G][G];  // M U_l
#pragma unroll
    for (int r = 0; r < G; ++r)
#pragma unroll
      for (int j = 0; j < G; ++j) {
        V s = cmake<V>(R(0), R(0));
#pragma unroll
        for (int c = 0; c < G; ++c) s = cadd(s, cmul(M[r][c], sm.ul[c][j][ll]));
        T[r][j] = s;
      }
#pragma unroll
    for (int i = 0; i < G; ++i)
#pragma unroll
      for (int j = 0; j < G; ++j) {
        V s = cmake<V>(R(0), R(0));
#pragma unroll
        for (int r = 0; r < G; ++r) s = cadd(s, cmulc(sm.uk[r][i][kk], T[r][j]));
        Ao[row[i] + col[j]] = s;
      }
    if (Vi == nullptr) return;
#pragma unroll
    for (int i = 0; i < G; ++i) {
      V v[G];
#pragma unroll
      for (int c = 0; c < G; ++c) v[c] = Vi[row[i] + col[c]];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        V s = cmake<V>(R(0), R(0));
#pragma unroll
        for (int c = 0; c < G; ++c) s = cadd(s, cmul(v[c], sm.ul[c][j][ll]));
        Vo[row[i] + col[j]] = s;
      }
    }
  }
}

template <class R>
__global__ void k_identity(cx_t<R>* V, int d) {
  using Vt = cx_t<R>;
  const long long n = (long long)d * d;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    V[e] = cmake<Vt>((e / d) == (e % d) ? R(1) : R(0), R(0));
}

// Spectrum: lam_i = Re A_ii, s_i = |lambda_i|^P (|lambda| floored at eps max|lambda| for P <= 1),
// s'_i = d s_i / d lambda_i (0 on the floor).  One block.
template <class R>
__global__ void __launch_bounds__(1024) k_absp_spectrum(const cx_t<R>* __restrict__ A, R* lam, R* s, R* sp, int d,
                                                         double P, double eps) {
  __shared__ R red[32];
  R m = R(0);
  for (int i = threadIdx.x; i < d; i += blockDim.x) m = fmax(m, fabs(A[(long long)i * d + i].x));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    R v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : R(0);
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double floor_v = P <= 1.0 ? eps * (double)red[0] : 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double li = (double)A[(long long)i * d + i].x;
    const double ai = fabs(li);
    const double ui = ai > floor_v ? ai : floor_v;
    lam[i] = (R)li;
    s[i] = (R)pow(ui, P);
    sp[i] = ai > floor_v && ui > 0.0 ? (R)(P * pow(ui, P - 1.0) * (li >= 0.0 ? 1.0 : -1.0)) : R(0);
  }
}

// W = V diag(s)
template <class R>
__global__ void __launch_bounds__(256) k_scale_cols(const cx_t<R>* __restrict__ V, const R* __restrict__ s,
                                                     cx_t<R>* __restrict__ W, int d) {
  const long long n = (long long)d * d;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const R sj = s[e % d];
    W[e] = cmake<cx_t<R>>(V[e].x * sj, V[e].y * sj);
  }
}

// C'_ij = D_ij C_ij / 2 (Daleckii-Krein divided differences of s; the 1/2 makes Y = V C' V^dag satisfy Y + Y^dag = Gamma).
template <class R>
__global__ void __launch_bounds__(256) k_dk_scale(cx_t<R>* C, const R* lam, const R* s, const R* sp, int d, R rel) {
  const long long n = (long long)d * d;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    const R li = lam[i], lj = lam[j];
    const R dl = li - lj;
    const R scale = fabs(li) > fabs(lj) ? fabs(li) : fabs(lj);
    R D;
    if (fabs(dl) <= rel * scale) D = R(0.5) * (sp[i] + sp[j]);
    else D = (s[i] - s[j]) / dl;
    const cx_t<R> c = C[e];
    C[e] = cmake<cx_t<R>>(R(0.5) * D * c.x, R(0.5) * D * c.y);
  }
}

template <class R>
__global__ void __launch_bounds__(256) k_conj_transpose(const cx_t<R>* __restrict__ A, cx_t<R>* __restrict__ B, int d) {
  __shared__ cx_t<R> tile[32][33];
  const int TS = d < 32 ? d : 32;
  const int bi = blockIdx.y, bj = blockIdx.x;
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    tile[r][c] = A[(long long)(bi * TS + r) * d + bj * TS + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    B[(long long)(bj * TS + r) * d + bi * TS + c] = cconj(tile[c][r]);
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

// Partition of the nonzero vectors of GF(2)^n into lines {u, v, u ^ v} and, for odd n, one plane span{p1, p2, p3},
// built from V(n) = V(n - 2) + V(2) (the new coordinates are bits n - 2 and n - 1): the line of the new
// coordinates; each line {u1, u2, u1 ^ u2} of V(n - 2) lifted to the four lines {u1 + x, u2 + w x,
// u1 ^ u2 + (1 + w) x} for x in V(2) = GF(4) (w x and (1 + w) x = w^2 x run over GF(4) with x, so the 12 points
// over the line are each covered once); the plane of V(n - 2) kept, with its 21 points over V(2) \ 0 as the
// seven lines {p(y) + 01, p(a y) + 10, p((1 + a) y) + 11}, y in GF(8)* = GF(2)[a] / (a^3 + a + 1) \ 0 and p
// the coordinates in the plane's basis.  Base cases: V(1) = {1} (a single point), V(2) one line, V(3) one plane.
struct VecPartition {
  std::vector<std::pair<int, int>> lines;
  int plane[3] = {0, 0, 0};
};

VecPartition vec_partition(int n) {
  VecPartition out;
  if (n == 2) out.lines.push_back({1, 2});
  if (n == 3) out.plane[0] = 1, out.plane[1] = 2, out.plane[2] = 4;
  if (n <= 3) return out;
  static const int kTimesW[4] = {0, 2, 3, 1};                 // x -> w x in GF(4), bit 0 = 1, bit 1 = w
  static const int kTimesA[8] = {0, 2, 4, 6, 3, 1, 7, 5};     // y -> a y in GF(8), bits 1, a, a^2
  const VecPartition low = vec_partition(n - 2);
  const int s = n - 2;
  out.lines.push_back({1 << s, 2 << s});
  for (const auto& l : low.lines)
    for (int x = 0; x < 4; ++x) out.lines.push_back({l.first | (x << s), l.second | (kTimesW[x] << s)});
  if (low.plane[0] != 0) {
    const int* P = low.plane;
    auto p = [P](int y) { return ((y & 1) ? P[0] : 0) ^ ((y & 2) ? P[1] : 0) ^ ((y & 4) ? P[2] : 0); };
    for (int y = 1; y < 8; ++y) out.lines.push_back({p(y) | (1 << s), p(kTimesA[y]) | (2 << s)});
    out.plane[0] = P[0], out.plane[1] = P[1], out.plane[2] = P[2];
  }
  return out;
}

int top_bit(int x) { return 31 - __builtin_clz((unsigned)x); }

JacobiPass make_pass(int a, int b) {
  JacobiPass p;
  if (b == 0) {
    p.a = a, p.b = 0, p.plo = top_bit(a), p.phi = 0;
    return p;
  }
  if (top_bit(b) > top_bit(a)) std::swap(a, b);
  if (top_bit(b) == top_bit(a)) b ^= a;
  if ((a >> top_bit(b)) & 1) a ^= b;
  p.a = a, p.b = b, p.plo = top_bit(b), p.phi = top_bit(a);
  return p;
}

std::vector<JacobiPass> build_schedule(int N) {
  std::vector<JacobiPass> out;
  if (N == 1) {
    out.push_back(make_pass(1, 0));
    return out;
  }
  const VecPartition part = vec_partition(N);
  for (const auto& l : part.lines) out.push_back(make_pass(l.first, l.second));
  if (part.plane[0] != 0) {  // the plane as one line and its four other points
    const int p1 = part.plane[0], p2 = part.plane[1], p3 = part.plane[2];
    out.push_back(make_pass(p1, p2));
    for (int m : {p3, p1 ^ p3, p2 ^ p3, p1 ^ p2 ^ p3}) out.push_back(make_pass(m, 0));
  }
  return out;
}

constexpr int kMaxScheduleN = 14;

// One sweep: every pass of the schedule, ping-ponging (Ain, Aout) and (Vin, Vout).
template <class R>
cudaError_t jacobi_sweep(int d, cx_t<R>*& Ain, cx_t<R>*& Aout, cx_t<R>*& Vin, cx_t<R>*& Vout, cx_t<R>* phi,
                         cudaStream_t s) {
  const std::vector<JacobiPass>& sched = jacobi_schedule(top_bit(d));
  const int n4 = d / 4, n2 = d / 2;
  const dim3 g4((n4 + 15) / 16, (n4 + 15) / 16), g2((n2 + 15) / 16, (n2 + 15) / 16);
  for (const JacobiPass& p : sched) {
    if (p.b != 0) k_jacobi_pass<R, 4><<<g4, 256, 0, s>>>(Ain, Aout, Vin, Vout, phi, d, p.a, p.b, p.plo, p.phi);
    else k_jacobi_pass<R, 2><<<g2, 256, 0, s>>>(Ain, Aout, Vin, Vout, phi, d, p.a, 0, p.plo, 0);
    std::swap(Ain, Aout);
    if (Vin != nullptr) std::swap(Vin, Vout);
  }
  return cudaGetLastError();
}

}  // namespace

const std::vector<JacobiPass>& jacobi_schedule(int N) {
  static const std::vector<std::vector<JacobiPass>> all = [] {
    std::vector<std::vector<JacobiPass>> v(kMaxScheduleN + 1);
    for (int n = 1; n <= kMaxScheduleN; ++n) v[n] = build_schedule(n);
    return v;
  }();
  return all[N < 1 ? 1 : (N > kMaxScheduleN ? kMaxScheduleN : N)];
}

long long jacobi_passes_per_sweep(int d) { return (long long)jacobi_schedule(top_bit(d)).size(); }

template <class R>
cudaError_t abs_p_forward(int d, const cx_t<R>* T, AbsPWork<R>& w, int sweeps, bool warm, double P, cx_t<R>* X,
                          cudaStream_t s) {
  using V = cx_t<R>;
  const long long nn = (long long)d * d;
  cudaError_t e;
  if (warm) {
    // previous eigenvectors Q (in V0) and Q^dag (in Qh): start from Q^dag T Q, nearly diagonal
    if ((e = cgemm_simt<R>(d, w.Qh, T, w.W, false, s)) != cudaSuccess) return e;
    if ((e = cgemm_simt<R>(d, w.W, w.V0, w.A0, false, s)) != cudaSuccess) return e;
  } else {
    if ((e = cudaMemcpyAsync(w.A0, T, nn * sizeof(V), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    k_identity<R><<<blocks_for(nn), 256, 0, s>>>(w.V0, d);
  }
  // an even number of sweeps of an odd number of passes brings both ping-pong pairs back to A0 / V0
  V *Ain = w.A0, *Aout = w.A1, *Vin = w.V0, *Vout = w.V1;
  for (int sw = 0; sw < sweeps; ++sw)
    if ((e = jacobi_sweep<R>(d, Ain, Aout, Vin, Vout, nullptr, s)) != cudaSuccess) return e;
  if (Vin != w.V0) {  // an odd number of sweeps: the eigenvectors are kept in V0
    if ((e = cudaMemcpyAsync(w.V0, Vin, nn * sizeof(V), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    Vin = w.V0;
  }
  w.A = Ain;  // diagonalised
  w.Q = Vin;  // eigenvectors in columns (V0)
  k_absp_spectrum<R><<<1, 1024, 0, s>>>(w.A, w.lam, w.s, w.sp, d, P, sizeof(R) == 4 ? 1e-7 : 1e-15);
  k_scale_cols<R><<<blocks_for(nn), 256, 0, s>>>(w.Q, w.s, w.W, d);
  const int TS = d < 32 ? d : 32;
  k_conj_transpose<R><<<dim3(d / TS, d / TS), 256, 0, s>>>(w.Q, w.Qh, d);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // X = (Q diag(s)) Q^dag, lower tiles
  return cgemm_simt<R>(d, w.W, w.Qh, X, true, s);
}

template <class R>
cudaError_t jacobi_values_project(int d, const cx_t<R>* T, AbsPWork<R>& w, int sweeps, double P, const cx_t<R>* psi,
                                  cx_t<R>* phi, cudaStream_t s) {
  using V = cx_t<R>;
  const long long nn = (long long)d * d;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(w.A0, T, nn * sizeof(V), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(phi, psi, (size_t)d * sizeof(V), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  V *Ain = w.A0, *Aout = w.A1, *Vin = nullptr, *Vout = nullptr;
  for (int sw = 0; sw < sweeps; ++sw)
    if ((e = jacobi_sweep<R>(d, Ain, Aout, Vin, Vout, phi, s)) != cudaSuccess) return e;
  w.A = Ain;
  k_absp_spectrum<R><<<1, 1024, 0, s>>>(w.A, w.lam, w.s, w.sp, d, P, sizeof(R) == 4 ? 1e-7 : 1e-15);
  return cudaGetLastError();
}

template <class R> cudaError_t abs_p_restore_q(int d, AbsPWork<R>& w, cudaStream_t s) {
  const int TS = d < 32 ? d : 32;
  k_conj_transpose<R><<<dim3(d / TS, d / TS), 256, 0, s>>>(w.V0, w.Qh, d);
  w.Q = w.V0;
  return cudaGetLastError();
}

template <class R>
cudaError_t abs_p_backward(int d, const cx_t<R>* G, AbsPWork<R>& w, cx_t<R>* Y, cudaStream_t s) {
  const long long nn = (long long)d * d;
  cudaError_t e;
  // C = Q^dag G Q (the Jacobi buffers are free once the spectrum is stored)
  cx_t<R>* C = w.A0 == w.Q ? w.A1 : w.A0;
  if ((e = cgemm_simt<R>(d, w.Qh, G, w.W, false, s)) != cudaSuccess) return e;
  if ((e = cgemm_simt<R>(d, w.W, w.Q, C, false, s)) != cudaSuccess) return e;
  k_dk_scale<R><<<blocks_for(nn), 256, 0, s>>>(C, w.lam, w.s, w.sp, d, sizeof(R) == 4 ? (R)1e-5 : (R)1e-12);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Y = Q C' Q^dag
  if ((e = cgemm_simt<R>(d, w.Q, C, w.W, false, s)) != cudaSuccess) return e;
  return cgemm_simt<R>(d, w.W, w.Qh, Y, false, s);
}

// ------------------------------------------------------------------ tensor-core refinement
// Warm-started steps of the mixed-precision path replace the Jacobi sweeps by one refinement of the
// previous eigenvectors (Ogita and Aishima's iteration for symmetric / Hermitian matrices): four products
// and a first-order correction, all of whose products run on k_tc_cgemm (gemm_tc.cu).  Pairs closer than
// kOaTau max|lambda|, or whose first-order correction would exceed 1/2, are treated as a cluster
// (E_ij = R_ij / 2: kept orthonormal, not separated); within a cluster |lambda|^P differs by little.
namespace {

constexpr float kOaTau = 1e-6f;

// entry (i, j) of a Hermitian matrix of which only the 128 x 128 tiles I >= J were computed
__device__ __forceinline__ float2 herm_entry(const float2* M, int d, int i, int j) {
  if ((i >> 7) >= (j >> 7)) return M[(long long)i * d + j];
  const float2 v = M[(long long)j * d + i];
  return make_float2(v.x, -v.y);
}

// lambda_i = S_ii / (Q^dag Q)_ii, s_i = |lambda_i|^P, s'_i (as k_absp_spectrum), sc[6] = max |lambda|.  One block.
__global__ void __launch_bounds__(1024) k_oa_spectrum(const float2* __restrict__ S, const float2* __restrict__ C1,
                                                       int d, double P, double eps, float* lam, float* s, float* sp,
                                                       double* sc) {
  __shared__ float red[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const float li = S[(long long)i * d + i].x / C1[(long long)i * d + i].x;
    lam[i] = li;
    m = fmaxf(m, fabsf(li));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double lmax = (double)red[0];
  if (threadIdx.x == 0) sc[6] = lmax;
  const double floor_v = P <= 1.0 ? eps * lmax : 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double li = (double)lam[i];
    const double ai = fabs(li);
    const double ui = ai > floor_v ? ai : floor_v;
    s[i] = (float)pow(ui, P);
    sp[i] = ai > floor_v && ui > 0.0 ? (float)(P * pow(ui, P - 1.0) * (li >= 0.0 ? 1.0 : -1.0)) : 0.f;
  }
}

// The correction E (full d x d) from S = Q^dag T Q and C1 = Q^dag Q (lower tiles), R = I - C1; max |E| -> amax[0],
// and max |S_ij| / max |lambda| over the separated pairs whose first-order correction was too large (left as
// a cluster) -> amax[1]: the size of what this refinement could not resolve.
__global__ void __launch_bounds__(256) k_oa_correction(const float2* __restrict__ S, const float2* __restrict__ C1,
                                                        const float* __restrict__ lam, const double* sc, int d,
                                                        float2* __restrict__ E, unsigned int* amax) {
  const long long nn = (long long)d * d;
  const float lmax = (float)sc[6];
  const float tau = kOaTau * lmax;
  float m = 0.f, u = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), j = (int)(e % d);
    const float2 c = herm_entry(C1, d, i, j);
    float2 r = make_float2(-c.x, -c.y);
    float2 out;
    if (i == j) {
      out = make_float2(0.5f * (1.f - c.x), 0.f);
    } else {
      const float2 sij = herm_entry(S, d, i, j);
      const float lj = lam[j], gap = lj - lam[i];
      out = make_float2(0.5f * r.x, 0.5f * r.y);
      if (fabsf(gap) > tau) {
        const float2 q = make_float2((sij.x + lj * r.x) / gap, (sij.y + lj * r.y) / gap);
        if (fmaxf(fabsf(q.x), fabsf(q.y)) <= 0.5f) out = q;
        else u = fmaxf(u, fmaxf(fabsf(sij.x), fabsf(sij.y)) / lmax);
      }
    }
    E[e] = out;
    m = fmaxf(m, fmaxf(fabsf(out.x), fabsf(out.y)));
  }
  block_absmax_to(m, amax);
  __syncthreads();
  block_absmax_to(u, amax + 1);
}

__global__ void __launch_bounds__(256) k_add_to(float2* __restrict__ Q, const float2* __restrict__ D, long long nn) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const float2 a = Q[e], b = D[e];
    Q[e] = make_float2(a.x + b.x, a.y + b.y);
  }
}

// planes of op(M) with the scale of M's own max (absmax_to into *amax first)
cudaError_t planes_of(int d, const float2* M, int op, int np, void* P, int fmt, unsigned int* amax, double* sslot,
                      bool fresh_amax, cudaStream_t s) {
  cudaError_t e;
  if (fresh_amax && (e = absmax_to((long long)d * d, M, amax, s)) != cudaSuccess) return e;
  return tc_planes_op(d, M, op, np, P, fmt, amax, sslot, s);
}

// ---- sorted-eigenvalue block passes (the couplings a first-order correction cannot resolve)
// In the order of increasing lambda, the eigenvectors that T's change mixes by more than their gap are
// neighbours: kBJ x kBJ diagonal blocks of S = Q^dag T Q are diagonalised exactly by Jacobi sweeps in
// shared memory (one CTA per block), Q's columns of each block are rotated by the block's unitary, and a
// second pass on blocks shifted by kBJ / 2 covers the couplings across block borders.
constexpr int kBJ = 64;
constexpr int kBJS = kBJ + 1;
constexpr int kBJSweeps = 8;

__global__ void __launch_bounds__(256) k_block_jacobi(const float2* __restrict__ S, const int* __restrict__ perm,
                                                       int d, int offset, float2* __restrict__ U) {
  extern __shared__ __align__(16) unsigned char sraw[];
  float2* Sb = reinterpret_cast<float2*>(sraw);
  float2* Ub = Sb + kBJ * kBJS;
  constexpr int NP = kBJ / 2;
  __shared__ float2 r_pp[NP], r_qp[NP], r_qq[NP], r_pq[NP];
  __shared__ int pi[NP], qi[NP];
  const int base = offset + kBJ * (int)blockIdx.x;
  for (int e = threadIdx.x; e < kBJ * kBJ; e += blockDim.x) {
    const int a = e / kBJ, b = e % kBJ;
    const int ga = perm ? perm[base + a] : base + a, gb = perm ? perm[base + b] : base + b;
    Sb[a * kBJS + b] = herm_entry(S, d, ga, gb);
    Ub[a * kBJS + b] = make_float2(a == b ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int sw = 0; sw < kBJSweeps; ++sw) {
    for (int r = 0; r < kBJ - 1; ++r) {
      if (threadIdx.x < NP) {  // round m = r + 1 pairs p with p ^ m; its rotations, from the block before it
        const int k = threadIdx.x, m = r + 1;
        const int p = insert_zero(k, 31 - __clz(m)), q = p ^ m;
        const Rot2<float> ro = rotation_for<float>(Sb[p * kBJS + p].x, Sb[q * kBJS + q].x, Sb[p * kBJS + q]);
        r_pp[k] = make_float2(ro.cs, 0.f);
        r_pq[k] = make_float2(ro.sn, 0.f);
        r_qp[k] = make_float2(-ro.emph.x * ro.sn, -ro.emph.y * ro.sn);
        r_qq[k] = make_float2(ro.emph.x * ro.cs, ro.emph.y * ro.cs);
        pi[k] = p;
        qi[k] = q;
      }
      __syncthreads();
      // S <- R^dag S R on the 2 x 2 blocks (pair k rows, pair l columns), each entry in one block
      for (int w = threadIdx.x; w < NP * NP; w += blockDim.x) {
        const int k = w / NP, l = w % NP;
        const int pk = pi[k], qk = qi[k], pl = pi[l], ql = qi[l];
        const float2 m_pp = Sb[pk * kBJS + pl], m_pq = Sb[pk * kBJS + ql];
        const float2 m_qp = Sb[qk * kBJS + pl], m_qq = Sb[qk * kBJS + ql];
        const float2 u_pp = cadd(cmul(m_pp, r_pp[l]), cmul(m_pq, r_qp[l]));
        const float2 u_pq = cadd(cmul(m_pp, r_pq[l]), cmul(m_pq, r_qq[l]));
        const float2 u_qp = cadd(cmul(m_qp, r_pp[l]), cmul(m_qq, r_qp[l]));
        const float2 u_qq = cadd(cmul(m_qp, r_pq[l]), cmul(m_qq, r_qq[l]));
        Sb[pk * kBJS + pl] = cadd(cmulc(r_pp[k], u_pp), cmulc(r_qp[k], u_qp));
        Sb[pk * kBJS + ql] = cadd(cmulc(r_pp[k], u_pq), cmulc(r_qp[k], u_qq));
        Sb[qk * kBJS + pl] = cadd(cmulc(r_pq[k], u_pp), cmulc(r_qq[k], u_qp));
        Sb[qk * kBJS + ql] = cadd(cmulc(r_pq[k], u_pq), cmulc(r_qq[k], u_qq));
      }
      // U <- U R (columns p_l, q_l of every row)
      for (int w = threadIdx.x; w < kBJ * NP; w += blockDim.x) {
        const int row = w / NP, l = w % NP;
        const int pl = pi[l], ql = qi[l];
        const float2 vp = Ub[row * kBJS + pl], vq = Ub[row * kBJS + ql];
        Ub[row * kBJS + pl] = cadd(cmul(vp, r_pp[l]), cmul(vq, r_qp[l]));
        Ub[row * kBJS + ql] = cadd(cmul(vp, r_pq[l]), cmul(vq, r_qq[l]));
      }
      __syncthreads();
    }
  }
  float2* out = U + (size_t)blockIdx.x * kBJ * kBJ;
  for (int e = threadIdx.x; e < kBJ * kBJ; e += blockDim.x) out[e] = Ub[(e / kBJ) * kBJS + e % kBJ];
}

// Q[:, block m] <- Q[:, block m] U_m for the blocks of a pass (columns offset + kBJ m ..), in place: CTA
// (row chunk, m) reads its 64 x kBJ piece of Q and U_m into shared memory before writing the product.
__global__ void __launch_bounds__(256) k_block_apply(float2* __restrict__ Q, int d, int offset,
                                                      const float2* __restrict__ U) {
  extern __shared__ __align__(16) unsigned char sraw[];
  float2* Qt = reinterpret_cast<float2*>(sraw);
  float2* Ut = Qt + 64 * kBJS;
  const int r0 = 64 * (int)blockIdx.x, c0 = offset + kBJ * (int)blockIdx.y;
  const float2* Um = U + (size_t)blockIdx.y * kBJ * kBJ;
  for (int e = threadIdx.x; e < 64 * kBJ; e += blockDim.x) {
    const int r = e / kBJ, c = e % kBJ;
    Qt[r * kBJS + c] = Q[(long long)(r0 + r) * d + c0 + c];
    Ut[r * kBJS + c] = Um[e];
  }
  __syncthreads();
  const int r = threadIdx.x >> 2, j0 = (threadIdx.x & 3) * 16;
  float2 acc[16];
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) acc[jj] = make_float2(0.f, 0.f);
  for (int a = 0; a < kBJ; ++a) {
    const float2 q = Qt[r * kBJS + a];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) acc[jj] = cadd(acc[jj], cmul(q, Ut[a * kBJS + j0 + jj]));
  }
  float2* dst = Q + (long long)(r0 + r) * d + c0 + j0;
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) dst[jj] = acc[jj];
}

__global__ void __launch_bounds__(256) k_permute_cols(const float2* __restrict__ Qi, float2* __restrict__ Qo,
                                                       const int* __restrict__ perm, int d) {
  const long long nn = (long long)d * d;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x)
    Qo[e] = Qi[(e / d) * d + perm[e % d]];
}

}  // namespace

size_t abs_p_tc_plane_bytes(int d) { return (size_t)4 * d * d * 2; }

// S = Q^dag T Q into w.A0 (lower tiles); the planes of Q^dag stay in qa_h (4) and qb_h (6)
cudaError_t abs_p_tc_rotated(int d, const void* Tb, const double* sT, AbsPWork<float>& w, int fmt, unsigned int* err,
                             cudaStream_t s) {
  float2* Q = w.V0;
  double* sc = w.sc;
  cudaError_t e;
  if ((e = planes_of(d, Q, 1, 4, w.qa_h, fmt, w.amax, sc + 1, true, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, Q, 1, 6, w.qb_h, fmt, w.amax, sc + 3, false, s)) != cudaSuccess) return e;
  if ((e = tc_product(d, w.qa_h, Tb, fmt, sc + 1, sT, w.W, false, err, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, w.W, 0, 4, w.wa, fmt, w.amax + 1, sc + 4, true, s)) != cudaSuccess) return e;
  return tc_product(d, w.wa, w.qb_h, fmt, sc + 4, sc + 3, w.A0, true, err, s);
}

cudaError_t abs_p_tc_correction(int d, const void* Tb, const double* sT, AbsPWork<float>& w, double P, int fmt,
                                unsigned int* err, cudaStream_t s) {
  const long long nn = (long long)d * d;
  unsigned int* amE = w.amax + 2;
  double* sc = w.sc;
  cudaError_t e;
  // S = (Q^dag T) Q and C1 = Q^dag Q = I - R, both Hermitian (lower tiles)
  if ((e = abs_p_tc_rotated(d, Tb, sT, w, fmt, err, s)) != cudaSuccess) return e;
  if ((e = tc_product(d, w.qa_h, w.qb_h, fmt, sc + 1, sc + 3, w.A1, true, err, s)) != cudaSuccess) return e;
  k_oa_spectrum<<<1, 1024, 0, s>>>(w.A0, w.A1, d, P, 1e-7, w.lam, w.s, w.sp, sc);
  if ((e = cudaMemsetAsync(amE, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess) return e;
  k_oa_correction<<<blocks_for(nn), 256, 0, s>>>(w.A0, w.A1, w.lam, sc, d, w.W, amE);
  return cudaGetLastError();
}

cudaError_t abs_p_tc_block_phase(int d, const void* Tb, const double* sT, AbsPWork<float>& w, int fmt,
                                 unsigned int* err, cudaStream_t s) {
  if (d % kBJ || d < 2 * kBJ) return cudaErrorInvalidValue;
  const long long nn = (long long)d * d;
  cudaError_t e;
  // the order of increasing lambda (lambda of the latest correction, S of the current Q in A0)
  std::vector<float> lam(d);
  std::vector<int> perm(d);
  if ((e = cudaMemcpyAsync(lam.data(), w.lam, d * sizeof(float), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  for (int i = 0; i < d; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return lam[a] < lam[b]; });
  if ((e = cudaMemcpyAsync(w.perm, perm.data(), d * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  k_permute_cols<<<blocks_for(nn), 256, 0, s>>>(w.V0, w.V1, w.perm, d);
  if ((e = cudaMemcpyAsync(w.V0, w.V1, nn * sizeof(float2), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
  const size_t smem = 2 * (size_t)64 * kBJS * sizeof(float2);
  if ((e = ensure_dynamic_smem((const void*)k_block_jacobi, smem)) != cudaSuccess) return e;
  if ((e = ensure_dynamic_smem((const void*)k_block_apply, smem)) != cudaSuccess) return e;
  float2* U = static_cast<float2*>(w.ublk);
  // pass 1: blocks [kBJ m, kBJ (m + 1)) of S in the sorted order (read through perm)
  const int nb1 = d / kBJ, nb2 = d / kBJ - 1;
  k_block_jacobi<<<nb1, 256, smem, s>>>(w.A0, w.perm, d, 0, U);
  k_block_apply<<<dim3(d / 64, nb1), 256, smem, s>>>(w.V0, d, 0, U);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // pass 2 on the rotated S, blocks shifted by kBJ / 2
  if ((e = abs_p_tc_rotated(d, Tb, sT, w, fmt, err, s)) != cudaSuccess) return e;
  k_block_jacobi<<<nb2, 256, smem, s>>>(w.A0, nullptr, d, kBJ / 2, U);
  k_block_apply<<<dim3(d / 64, nb2), 256, smem, s>>>(w.V0, d, kBJ / 2, U);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);  // the host vectors of the copies go out of scope here
}

cudaError_t abs_p_tc_update(int d, AbsPWork<float>& w, int fmt, unsigned int* err, cudaStream_t s) {
  const long long nn = (long long)d * d;
  float2* Q = w.V0;
  cudaError_t e;
  // Q <- Q + Q E (E in W, its max in amax[2])
  if ((e = planes_of(d, w.W, 1, 6, w.eb, fmt, w.amax + 2, w.sc + 5, false, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, Q, 0, 4, w.qa_n, fmt, w.amax, w.sc + 0, false, s)) != cudaSuccess) return e;
  if ((e = tc_product(d, w.qa_n, w.eb, fmt, w.sc + 0, w.sc + 5, w.V1, false, err, s)) != cudaSuccess) return e;
  k_add_to<<<blocks_for(nn), 256, 0, s>>>(Q, w.V1, nn);
  return cudaGetLastError();
}

cudaError_t abs_p_tc_finish(int d, AbsPWork<float>& w, int fmt, float2* X, unsigned int* err, cudaStream_t s) {
  const long long nn = (long long)d * d;
  float2* Q = w.V0;
  double* sc = w.sc;
  cudaError_t e;
  // X = (Q diag(s)) Q^dag, lower tiles
  k_scale_cols<float><<<blocks_for(nn), 256, 0, s>>>(Q, w.s, w.W, d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = planes_of(d, w.W, 0, 4, w.wa, fmt, w.amax + 1, sc + 4, true, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, Q, 0, 6, w.qb_n, fmt, w.amax, sc + 2, true, s)) != cudaSuccess) return e;
  if ((e = tc_product(d, w.wa, w.qb_n, fmt, sc + 4, sc + 2, X, true, err, s)) != cudaSuccess) return e;
  w.A = w.A0;
  w.Q = Q;
  const int TS = d < 32 ? d : 32;
  k_conj_transpose<float><<<dim3(d / TS, d / TS), 256, 0, s>>>(Q, w.Qh, d);
  return cudaGetLastError();
}

cudaError_t abs_p_backward_tc(int d, const float2* G, AbsPWork<float>& w, int fmt, float2* Y, unsigned int* err,
                              cudaStream_t s) {
  const long long nn = (long long)d * d;
  const float2* Q = w.Q;
  float2* C = w.A0 == w.Q ? w.A1 : w.A0;
  unsigned int *amQ = w.amax, *amW = w.amax + 1, *amE = w.amax + 2;
  double* sc = w.sc;
  cudaError_t e;
  if ((e = planes_of(d, Q, 1, 4, w.qa_h, fmt, amQ, sc + 1, true, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, Q, 1, 6, w.qb_h, fmt, amQ, sc + 3, false, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, Q, 0, 4, w.qa_n, fmt, amQ, sc + 0, false, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, Q, 0, 6, w.qb_n, fmt, amQ, sc + 2, false, s)) != cudaSuccess) return e;
  // C = (Q^dag G) Q
  if ((e = planes_of(d, G, 1, 6, w.eb, fmt, amE, sc + 5, true, s)) != cudaSuccess) return e;
  if ((e = tc_product(d, w.qa_h, w.eb, fmt, sc + 1, sc + 5, w.W, false, err, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, w.W, 0, 4, w.wa, fmt, amW, sc + 4, true, s)) != cudaSuccess) return e;
  if ((e = tc_product(d, w.wa, w.qb_h, fmt, sc + 4, sc + 3, C, false, err, s)) != cudaSuccess) return e;
  k_dk_scale<float><<<blocks_for(nn), 256, 0, s>>>(C, w.lam, w.s, w.sp, d, 1e-5f);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // Y = (Q C') Q^dag
  if ((e = planes_of(d, C, 1, 6, w.eb, fmt, amE, sc + 5, true, s)) != cudaSuccess) return e;
  if ((e = tc_product(d, w.qa_n, w.eb, fmt, sc + 0, sc + 5, w.W, false, err, s)) != cudaSuccess) return e;
  if ((e = planes_of(d, w.W, 0, 4, w.wa, fmt, amW, sc + 4, true, s)) != cudaSuccess) return e;
  return tc_product(d, w.wa, w.qb_n, fmt, sc + 4, sc + 2, Y, false, err, s);
}

template cudaError_t abs_p_forward<float>(int, const float2*, AbsPWork<float>&, int, bool, double, float2*,
                                          cudaStream_t);
template cudaError_t abs_p_forward<double>(int, const double2*, AbsPWork<double>&, int, bool, double, double2*,
                                           cudaStream_t);
template cudaError_t jacobi_values_project<float>(int, const float2*, AbsPWork<float>&, int, double, const float2*,
                                                  float2*, cudaStream_t);
template cudaError_t jacobi_values_project<double>(int, const double2*, AbsPWork<double>&, int, double,
                                                   const double2*, double2*, cudaStream_t);
template cudaError_t abs_p_restore_q<float>(int, AbsPWork<float>&, cudaStream_t);
template cudaError_t abs_p_restore_q<double>(int, AbsPWork<double>&, cudaStream_t);
template cudaError_t abs_p_backward<float>(int, const float2*, AbsPWork<float>&, float2*, cudaStream_t);
template cudaError_t abs_p_backward<double>(int, const double2*, AbsPWork<double>&, double2*, cudaStream_t);

}  // namespace qst
