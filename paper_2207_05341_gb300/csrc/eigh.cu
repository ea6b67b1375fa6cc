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
// sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / 2|c|).  The 2^k - 1 rounds of a k-dimensional
// subspace S of GF(2)^N all act within S's cosets, so the rounds of a sweep are grouped by a partition of the
// nonzero vectors of GF(2)^N into subspaces, and one pass applies all rounds of a subspace, exactly as they
// would run one after another, with one read and one write of A and V: A' = U^dag A U and V' = V U with U
// block-diagonal over the cosets.  N <= 5: lines and single rounds, one kernel per pass (each thread a 4 x 4
// or 2 x 2 block, the CTA's coset unitaries formed by groups of lanes).  N >= 6: subspaces of dimension 3
// and 4, two kernels per pass (the coset unitaries, a warp per coset; then 64 x 64 tiles of A and V in
// shared memory).  At N = 11 and 12 a sweep is 273 passes (2047 / 4095 rounds).
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
    const int hb = s >= 8 ? 3 : (s >= 4 ? 2 : (s >= 2 ? 1 : 0));
    Rot2<R> rs[G / 2];  // every pair's rotation, from its lower lane
#pragma unroll
    for (int l = 0; l < G / 2; ++l) rs[l] = rot_from_lane(mine, insert_zero(l, hb), G);
#pragma unroll
    for (int l = 0; l < G / 2; ++l) {
      const int pl = insert_zero(l, hb), ql = pl ^ s;
      rotate_cols<R, G>(b, pl, ql, rs[l]);
      rotate_cols<R, G>(u, pl, ql, rs[l]);
    }
    // rows p, q of B <- R^dag rows (p, q): this lane's row with its partner's
    V o[G];
#pragma unroll
    for (int j = 0; j < G; ++j) o[j] = cmake<V>(lane_xor(b[j].x, s, G), lane_xor(b[j].y, s, G));
    const int pi = (i >> hb) & 1 ? i ^ s : i;                        // the lower index of this lane's pair
    const int li = ((pi >> (hb + 1)) << hb) | (pi & ((1 << hb) - 1));  // and the pair's number
    Rot2<R> r = rs[0];
#pragma unroll
    for (int l = 1; l < G / 2; ++l)
      if (l == li) r = rs[l];
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

// ---- passes over cosets of 8 or 16 indices (N >= 6): the unitaries first, then the blocks
__device__ __forceinline__ int coset_rep(int c, const JacobiPass& p) {
  int x = c;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < p.k) x = insert_zero(x, p.piv[i]);
  return x;
}
__device__ __forceinline__ int coset_element(int rep, int j, const JacobiPass& p) {
  int x = rep;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < p.k && ((j >> i) & 1)) x ^= p.basis[i];
  return x;
}

// Loads of data the preceding kernel wrote, issued after grid_dep_wait(): volatile, so that the compiler does
// not move them above the wait (a const __restrict__ load may be hoisted across it).
__device__ __forceinline__ float2 ld_after_wait(const float2* p) {
  float2 v;
  asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double2 ld_after_wait(const double2* p) {
  double2 v;
  asm volatile("ld.global.cg.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p) : "memory");
  return v;
}

// One warp per coset: the G x G principal block B of A on the coset and U = R_1 ... R_{G-1} in shared memory,
// round s (s = 1 .. G - 1, the subspace element of local index s) rotating the local pairs {x, x ^ s}, each
// rotation computed from B after the rounds before it (B <- R^dag B R, U <- U R).  Writes U to Ug[coset].
// Lets the pass's block kernel start (its loads of A do not depend on U).
template <class R, int G>
__global__ void __launch_bounds__(32) k_coset_unitaries(const cx_t<R>* __restrict__ A, int d, JacobiPass p,
                                                        cx_t<R>* __restrict__ Ug) {
  using V = cx_t<R>;
  asm volatile("griddepcontrol.launch_dependents;");
  __shared__ V B[G][G + 1], U[G][G + 1];
  __shared__ Rot2<R> rot[G / 2];
  __shared__ int e[G];
  const int c = blockIdx.x, lane = threadIdx.x;
  if (lane < G) e[lane] = coset_element(coset_rep(c, p), lane, p);
  __syncwarp();
  for (int x = lane; x < G * G; x += 32) {
    const int i = x / G, j = x % G;
    B[i][j] = A[(long long)e[i] * d + e[j]];
    U[i][j] = cmake<V>(i == j ? R(1) : R(0), R(0));
  }
  __syncwarp();
  for (int s = 1; s < G; ++s) {
    const int hb = 31 - __clz(s);
    if (lane < G / 2) {
      const int pp = insert_zero(lane, hb), q = pp ^ s;
      rot[lane] = rotation_for<R>(B[pp][pp].x, B[q][q].x, B[pp][q]);
    }
    __syncwarp();
    for (int x = lane; x < G * (G / 2); x += 32) {  // columns p, q of row i of B and of U: X <- X R
      const int i = x / (G / 2), l = x % (G / 2);
      const int pp = insert_zero(l, hb), q = pp ^ s;
      const Rot2<R> r = rot[l];
      const V rqp = cmake<V>(-r.emph.x * r.sn, -r.emph.y * r.sn), rqq = cmake<V>(r.emph.x * r.cs, r.emph.y * r.cs);
      const V bp = B[i][pp], bq = B[i][q];
      B[i][pp] = cadd(cmake<V>(bp.x * r.cs, bp.y * r.cs), cmul(bq, rqp));
      B[i][q] = cadd(cmake<V>(bp.x * r.sn, bp.y * r.sn), cmul(bq, rqq));
      const V up = U[i][pp], uq = U[i][q];
      U[i][pp] = cadd(cmake<V>(up.x * r.cs, up.y * r.cs), cmul(uq, rqp));
      U[i][q] = cadd(cmake<V>(up.x * r.sn, up.y * r.sn), cmul(uq, rqq));
    }
    __syncwarp();
    for (int x = lane; x < (G / 2) * G; x += 32) {  // rows p, q of B: B <- R^dag B
      const int l = x / G, j = x % G;
      const int pp = insert_zero(l, hb), q = pp ^ s;
      const Rot2<R> r = rot[l];
      const V rqp = cmake<V>(-r.emph.x * r.sn, -r.emph.y * r.sn), rqq = cmake<V>(r.emph.x * r.cs, r.emph.y * r.cs);
      const V bp = B[pp][j], bq = B[q][j];
      B[pp][j] = cadd(cmake<V>(r.cs * bp.x, r.cs * bp.y), cmulc(rqp, bq));
      B[q][j] = cadd(cmake<V>(r.sn * bp.x, r.sn * bp.y), cmulc(rqq, bq));
    }
    __syncwarp();
  }
  V* out = Ug + (size_t)c * G * G;
  for (int x = lane; x < G * G; x += 32) out[x] = U[x / G][x % G];
}

// Asynchronous copy of one complex entry from global to shared memory (no register on the way), and the wait
// for all of this thread's copies.
template <class V> __device__ __forceinline__ void cp_async_entry(V* dst, const V* src) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(V) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// RB consecutive unitary entries from shared memory: FP32 two per 16-byte load, as the broadcast pairs
// (u.x, u.x) in ux and (u.y, u.y) in uy that the packed products take; FP64 as they are (uy unused).
template <class R, int RB>
__device__ __forceinline__ void load_u_row(const cx_t<R>* src, cx_t<R> (&ux)[RB], cx_t<R> (&uy)[RB]) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int h = 0; h < RB / 2; ++h) {
      const float4 w = reinterpret_cast<const float4*>(src)[h];
      ux[2 * h] = make_float2(w.x, w.x);
      uy[2 * h] = make_float2(w.y, w.y);
      ux[2 * h + 1] = make_float2(w.z, w.z);
      uy[2 * h + 1] = make_float2(w.w, w.w);
    }
  } else {
#pragma unroll
    for (int h = 0; h < RB; ++h) ux[h] = src[h];
  }
}

// The block kernel's shared memory: the TS x TS tiles of A and V (rows: TS / G row cosets, columns: TS / G
// column cosets, coset-major), the cosets' unitaries, the tile's row and column indices and the first block
// column's piece of phi.
template <class R, int G, int TS> struct TileSmem {
  // column c of a tile at c + c / G (one word after each coset) and one more per row: the reads of a column
  // across the row's cosets, and of a row across the column blocks, fall in distinct banks
  static constexpr int LD = TS + TS / G + 1;
  cx_t<R> a[TS][LD], v[TS][LD];
  cx_t<R> ul[TS / G][G][G], uk[TS / G][G][G];
  int ridx[TS], cidx[TS];
  cx_t<R> ph[TS];
};

// One pass over cosets of G indices: CTA (x, y) stages the tiles of A and V on row cosets y TS / G .. and
// column cosets x TS / G .. in shared memory (loaded before waiting for the pass's unitaries), computes
// T = A U_l and V' = V U_l (U block-diagonal over the cosets), then A' = U_k^dag T, each thread an RB x RB
// block of outputs, and writes both tiles back.  Every entry is read and written once per pass.
template <class R, int G, int TS>
__global__ void __launch_bounds__(256) k_jacobi_tile(const cx_t<R>* __restrict__ A, cx_t<R>* __restrict__ Ao,
                                                      const cx_t<R>* __restrict__ Vi, cx_t<R>* __restrict__ Vo,
                                                      cx_t<R>* __restrict__ phi, int d, JacobiPass p,
                                                      const cx_t<R>* Ug) {
  using V = cx_t<R>;
  constexpr int TPC = TS / G, RB = TS / 16;
  constexpr bool kF32 = sizeof(R) == 4;
  extern __shared__ __align__(16) unsigned char sraw[];
  TileSmem<R, G, TS>& S = *reinterpret_cast<TileSmem<R, G, TS>*>(sraw);
  const int k0 = blockIdx.y * TPC, l0 = blockIdx.x * TPC;
  const int t = threadIdx.x;
  if (t < TS) S.ridx[t] = coset_element(coset_rep(k0 + t / G, p), t % G, p);
  else if (t < 2 * TS) S.cidx[t - TS] = coset_element(coset_rep(l0 + (t - TS) / G, p), (t - TS) % G, p);
  __syncthreads();
  for (int e = t; e < TS * TS; e += 256) {  // every copy of the tiles in flight at once
    const int r = e / TS, c = e % TS;
    const long long off = (long long)S.ridx[r] * d + S.cidx[c];
    cp_async_entry(&S.a[r][c + c / G], A + off);
    if (Vi != nullptr) cp_async_entry(&S.v[r][c + c / G], Vi + off);
  }
  const bool with_phi = phi != nullptr && blockIdx.x == 0;
  if (with_phi && t < TS) S.ph[t] = phi[S.ridx[t]];
  grid_dep_wait();  // the unitaries of this pass
  after_wait(Ug);
  for (int e = t; e < TPC * G * G; e += 256) {
    const int cc = e / (G * G), rc = (e / G) % G, jc = e % G;
    const V ul = ld_after_wait(Ug + (size_t)(l0 + cc) * G * G + rc * G + jc);
    const V uk = ld_after_wait(Ug + (size_t)(k0 + cc) * G * G + rc * G + jc);
    S.ul[cc][rc][jc] = ul;
    S.uk[cc][rc][jc] = uk;
  }
  cp_async_wait_all();
  __syncthreads();
  if (with_phi && t < TS) {  // phi <- U_k^dag phi on the row cosets
    const int rc = t / G, i = t % G;
    V y = cmake<V>(R(0), R(0));
    for (int r = 0; r < G; ++r) {
      y = cadd(y, cmulc(S.uk[rc][r][i], S.ph[rc * G + r]));
    }
    phi[S.ridx[t]] = y;
  }
  // T = A U_l, V' = V U_l: lane l of warp w takes rows rr + 16 i (rr = l % 16) and the RB columns of column
  // block cb = 2 w + l / 16 (inside column coset cc): a warp reads one column of 16 rows (distinct banks) and
  // at most two unitary entries per step
  const int lane = t & 31, warp = t >> 5;
  V acc[RB][RB], accv[RB][RB];
  {
    const int rr = lane % 16, cb = 2 * warp + lane / 16;
    const int c0 = cb * RB, cc = c0 / G, j0 = c0 % G;
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) acc[i][j] = accv[i][j] = cmake<V>(R(0), R(0));
#pragma unroll 4
    for (int q = 0; q < G; ++q) {
      V ux[RB], uy[RB];  // FP32: (u.x, u.x) and (u.y, u.y) of entries j0 .. j0 + RB of row q of U_l
      load_u_row<R, RB>(&S.ul[cc][q][j0], ux, uy);
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const V m = S.a[rr + 16 * i][cc * (G + 1) + q];
        const V w = Vi != nullptr ? S.v[rr + 16 * i][cc * (G + 1) + q] : cmake<V>(R(0), R(0));
        if constexpr (kF32) {
          const float2 msw = make_float2(-m.y, m.x), wsw = make_float2(-w.y, w.x);  // i m, i w
#pragma unroll
          for (int j = 0; j < RB; ++j) {  // m u = u.x m + u.y (i m)
            acc[i][j] = __ffma2_rn(uy[j], msw, __ffma2_rn(ux[j], m, acc[i][j]));
            accv[i][j] = __ffma2_rn(uy[j], wsw, __ffma2_rn(ux[j], w, accv[i][j]));
          }
        } else {
#pragma unroll
          for (int j = 0; j < RB; ++j) {
            acc[i][j] = cadd(acc[i][j], cmul(m, ux[j]));
            accv[i][j] = cadd(accv[i][j], cmul(w, ux[j]));
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        S.a[rr + 16 * i][c0 + j + cc] = acc[i][j];
        S.v[rr + 16 * i][c0 + j + cc] = accv[i][j];
      }
  }
  __syncthreads();
  {  // A' = U_k^dag T: lane l of warp w takes the RB rows of row block rb = 2 w + l / 16 (inside row coset rc)
     // and columns cs + 16 j (cs = l % 16)
    const int cs = lane % 16, rb = 2 * warp + lane / 16;
    const int r0 = rb * RB, rc = r0 / G, i0 = r0 % G;
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) acc[i][j] = cmake<V>(R(0), R(0));
#pragma unroll 4
    for (int q = 0; q < G; ++q) {
      V ux[RB], uy[RB];
      load_u_row<R, RB>(&S.uk[rc][q][i0], ux, uy);
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const int c = cs + 16 * j;
        const V tv = S.a[rc * G + q][c + c / G];
        if constexpr (kF32) {
          const float2 tsw = make_float2(tv.y, -tv.x);  // -i t
#pragma unroll
          for (int i = 0; i < RB; ++i)  // conj(u) t = u.x t + u.y (-i t)
            acc[i][j] = __ffma2_rn(uy[i], tsw, __ffma2_rn(ux[i], tv, acc[i][j]));
        } else {
#pragma unroll
          for (int i = 0; i < RB; ++i) acc[i][j] = cadd(acc[i][j], cmulc(ux[i], tv));
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const int c = cs + 16 * j;
        S.a[r0 + i][c + c / G] = acc[i][j];
      }
  }
  __syncthreads();
#pragma unroll 4
  for (int e = t; e < TS * TS; e += 256) {
    const int r = e / TS, c = e % TS;
    const long long off = (long long)S.ridx[r] * d + S.cidx[c];
    Ao[off] = S.a[r][c + c / G];
    if (Vi != nullptr) Vo[off] = S.v[r][c + c / G];
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

// Partitions of the nonzero vectors of GF(2)^n into subspaces (each a basis), built from V(n) = V(n - k) + V(k),
// the new coordinates at bits n - k .. n - 1: the subspace V(k) of the new coordinates, and each subspace S of
// the partition of V(n - k) (dimension m <= k, basis u_0 .. u_{m-1}) lifted to the 2^k subspaces with bases
// u_i + c x^i (c in GF(2^k), x^i the field's basis element i, the product in GF(2^k)): for u != 0 in S the map
// c -> c iota(u) (iota(u_i) = x^i) is a bijection onto GF(2^k), so every point (u, y) with u in S \ 0 lies in
// exactly one lifted subspace.  For small N the lines (k = 2) and single rounds of the 4-index passes; for
// N >= 6 subspaces of dimension 3 and 4 (8- and 16-index cosets), the lift sizes chosen for the fewest passes.
using Basis = std::vector<int>;

int gf_mul(int k, int a, int b) {  // GF(2^k), moduli x^2 + x + 1, x^3 + x + 1, x^4 + x + 1
  static const int kMod[5] = {0, 0, 0x7, 0xB, 0x13};
  int r = 0;
  for (int i = 0; i < k; ++i)
    if ((b >> i) & 1) r ^= a << i;
  for (int i = 2 * k - 2; i >= k; --i)
    if ((r >> i) & 1) r ^= kMod[k] << (i - k);
  return k == 1 ? (a & b & 1) : r;
}

std::vector<Basis> lift(const std::vector<Basis>& low, int s, int k) {
  std::vector<Basis> out;
  Basis top;
  for (int i = 0; i < k; ++i) top.push_back(1 << (s + i));
  out.push_back(top);
  for (const Basis& S : low)
    for (int c = 0; c < (1 << k); ++c) {
      Basis b;
      for (size_t i = 0; i < S.size(); ++i) b.push_back(S[i] | (gf_mul(k, c, 1 << i) << s));
      out.push_back(b);
    }
  return out;
}

// fewest subspaces of dimension <= m partitioning V(n) \ 0 by repeated lifting (and the first lift size)
long long min_parts(int n, int m, int* best_k) {
  if (n <= m) {
    if (best_k) *best_k = 0;
    return 1;
  }
  long long best = -1;
  for (int k = 1; k <= m && k < n; ++k) {
    const long long v = 1 + ((long long)1 << k) * min_parts(n - k, k, nullptr);
    if (best < 0 || v < best) {
      best = v;
      if (best_k) *best_k = k;
    }
  }
  return best;
}

std::vector<Basis> subspace_partition(int n, int m) {
  int k = 0;
  min_parts(n, m, &k);
  if (k == 0) {
    Basis all;
    for (int i = 0; i < n; ++i) all.push_back(1 << i);
    return {all};
  }
  return lift(subspace_partition(n - k, k), n - k, k);
}

int top_bit(int x) { return 31 - __builtin_clz((unsigned)x); }

JacobiPass make_pass(Basis v) {  // reduced echelon form, pivots ascending
  JacobiPass p = {};
  p.k = (int)v.size();
  for (size_t r = 0; r < v.size(); ++r) {
    size_t best = r;
    for (size_t q = r + 1; q < v.size(); ++q)
      if (top_bit(v[q]) > top_bit(v[best])) best = q;
    std::swap(v[r], v[best]);
    const int pb = top_bit(v[r]);
    for (size_t q = 0; q < v.size(); ++q)
      if (q != r && ((v[q] >> pb) & 1)) v[q] ^= v[r];
  }
  std::sort(v.begin(), v.end());
  for (int i = 0; i < p.k; ++i) {
    p.basis[i] = v[i];
    p.piv[i] = top_bit(v[i]);
  }
  return p;
}

std::vector<JacobiPass> build_schedule(int N) {
  std::vector<JacobiPass> out;
  if (N == 1) {
    out.push_back(make_pass({1}));
    return out;
  }
  if (N >= 6) {
    for (const Basis& b : subspace_partition(N, 4)) out.push_back(make_pass(b));
    return out;
  }
  // lines (lifted through GF(4)), and for odd N one plane taken as a line and its four other points
  for (const Basis& b : subspace_partition(N, 3)) {
    if (b.size() <= 2) {
      out.push_back(make_pass(b));
    } else {
      out.push_back(make_pass({b[0], b[1]}));
      for (int m : {b[2], b[0] ^ b[2], b[1] ^ b[2], b[0] ^ b[1] ^ b[2]}) out.push_back(make_pass({m}));
    }
  }
  return out;
}

constexpr int kMaxScheduleN = 14;

template <class R, int G>
cudaError_t tile_pass(int d, const JacobiPass& p, const cx_t<R>* A, cx_t<R>* Ao, const cx_t<R>* Vi, cx_t<R>* Vo,
                      cx_t<R>* phi, cx_t<R>* ucos, cudaStream_t s) {
  constexpr int TS = sizeof(R) == 4 ? 64 : 32;
  const size_t smem = sizeof(TileSmem<R, G, TS>);
  cudaError_t e = ensure_dynamic_smem((const void*)k_jacobi_tile<R, G, TS>, smem);
  if (e != cudaSuccess) return e;
  k_coset_unitaries<R, G><<<d / G, 32, 0, s>>>(A, d, p, ucos);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_dep(k_jacobi_tile<R, G, TS>, dim3(d / TS, d / TS), dim3(256), smem, s, A, Ao, Vi, Vo, phi, d, p,
                    (const cx_t<R>*)ucos);
}

// One sweep: every pass of the schedule, ping-ponging (Ain, Aout) and (Vin, Vout).  Passes over cosets of 8
// or 16 indices (N >= 6) are a unitary kernel and a block kernel; those over 2 or 4 indices one kernel.
template <class R>
cudaError_t jacobi_sweep(int d, cx_t<R>*& Ain, cx_t<R>*& Aout, cx_t<R>*& Vin, cx_t<R>*& Vout, cx_t<R>* phi,
                         cx_t<R>* ucos, cudaStream_t s) {
  const std::vector<JacobiPass>& sched = jacobi_schedule(top_bit(d));
  const int n4 = d / 4, n2 = d / 2;
  const dim3 g4((n4 + 15) / 16, (n4 + 15) / 16), g2((n2 + 15) / 16, (n2 + 15) / 16);
  for (const JacobiPass& p : sched) {
    cudaError_t e = cudaSuccess;
    if (p.k == 4) e = tile_pass<R, 16>(d, p, Ain, Aout, Vin, Vout, phi, ucos, s);
    else if (p.k == 3) e = tile_pass<R, 8>(d, p, Ain, Aout, Vin, Vout, phi, ucos, s);
    else if (p.k == 2)
      k_jacobi_pass<R, 4><<<g4, 256, 0, s>>>(Ain, Aout, Vin, Vout, phi, d, p.basis[1], p.basis[0], p.piv[0], p.piv[1]);
    else
      k_jacobi_pass<R, 2><<<g2, 256, 0, s>>>(Ain, Aout, Vin, Vout, phi, d, p.basis[0], 0, p.piv[0], 0);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(Ain, Aout);
    if (Vin != nullptr) std::swap(Vin, Vout);
  }
  return cudaSuccess;
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

long long jacobi_kernels_per_sweep(int d) {
  long long k = 0;
  for (const JacobiPass& p : jacobi_schedule(top_bit(d))) k += p.k >= 3 ? 2 : 1;
  return k;
}

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
    if ((e = jacobi_sweep<R>(d, Ain, Aout, Vin, Vout, nullptr, w.ucos, s)) != cudaSuccess) return e;
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
    if ((e = jacobi_sweep<R>(d, Ain, Aout, Vin, Vout, phi, w.ucos, s)) != cudaSuccess) return e;
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

namespace {

// M[i][j] = conj(M[j][i]) wherever the 128 x 128 tile of (i, j) lies above the diagonal: a Hermitian matrix
// of which only the tiles I >= J were computed, made whole.  CTA (x, y): the 32 x 32 block (y, x), read
// transposed from block (x, y) through shared memory.
__global__ void __launch_bounds__(256) k_mirror_upper_tiles(float2* M, int d) {
  __shared__ float2 tile[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if ((bi >> 2) >= (bj >> 2)) return;  // not above the diagonal at 128-tile granularity
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e / 32, c = e % 32;
    tile[r][c] = M[(long long)(bj * 32 + r) * d + bi * 32 + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e / 32, c = e % 32;
    const float2 v = tile[c][r];
    M[(long long)(bi * 32 + r) * d + bj * 32 + c] = make_float2(v.x, -v.y);
  }
}

}  // namespace

cudaError_t abs_p_forward_tc_warm(int d, const void* Tb, const double* sT, AbsPWork<float>& w, int sweeps, double P,
                                  int fmt, float2* X, unsigned int* err, cudaStream_t s) {
  const long long nn = (long long)d * d;
  cudaError_t e;
  // A0 = Q^dag T Q (Q = V0) on tensor cores, lower tiles, then the upper ones
  if ((e = abs_p_tc_rotated(d, Tb, sT, w, fmt, err, s)) != cudaSuccess) return e;
  k_mirror_upper_tiles<<<dim3(d / 32, d / 32), 256, 0, s>>>(w.A0, d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  float2 *Ain = w.A0, *Aout = w.A1, *Vin = w.V0, *Vout = w.V1;
  for (int sw = 0; sw < sweeps; ++sw)
    if ((e = jacobi_sweep<float>(d, Ain, Aout, Vin, Vout, nullptr, w.ucos, s)) != cudaSuccess) return e;
  if (Vin != w.V0 && (e = cudaMemcpyAsync(w.V0, Vin, nn * sizeof(float2), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  if (Ain != w.A0 && (e = cudaMemcpyAsync(w.A0, Ain, nn * sizeof(float2), cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  k_absp_spectrum<float><<<1, 1024, 0, s>>>(w.A0, w.lam, w.s, w.sp, d, P, 1e-7);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // X = Q |Lambda|^P Q^dag on tensor cores (lower tiles), and Q^dag
  return abs_p_tc_finish(d, w, fmt, X, err, s);
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
