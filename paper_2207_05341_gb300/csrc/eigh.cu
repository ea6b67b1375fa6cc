// P-order absolute projection of Sec. 3.2 (eq. abs_P):
//   T = Q Lambda Q^dag,   X = Q |Lambda|^P Q^dag,   rho = X / Tr X,
// and its backward (Daleckii-Krein): with s_i = |lambda_i|^P,
//   dL/dT = Q (D o (Q^dag G Q)) Q^dag,  D_ij = (s_i - s_j) / (lambda_i - lambda_j),  D_ii = s'(lambda_i),
// where G = dL/dX comes from the adjoint POVM map.
//
// The eigendecomposition is a cyclic two-sided Jacobi method for complex
// Hermitian matrices with the parallel round-robin ordering: a sweep is d - 1
// rounds, each rotating d / 2 disjoint index pairs at once.  For a pair (p, q)
// with c = A_pq = |c| e^{i phi}, the 2 x 2 block is first made real by
// diag(1, e^{-i phi}) and then zeroed by the real rotation of Golub and Van
// Loan (tan theta = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / 2|c|).
// One kernel per round: each thread owns the 2 x 2 block (rows of one pair) x
// (columns of another pair) of A and of V, so every entry is read and written
// once per round (double-buffered), and V accumulates the rotations, V <- V R.
#include <float.h>

#include "impl.h"

namespace qst {

namespace {

template <class R> __device__ __forceinline__ R tiny_normal();
template <> __device__ __forceinline__ float tiny_normal<float>() { return FLT_MIN; }
template <> __device__ __forceinline__ double tiny_normal<double>() { return DBL_MIN; }
template <class R> __device__ __forceinline__ R eps_of();
template <> __device__ __forceinline__ float eps_of<float>() { return FLT_EPSILON; }
template <> __device__ __forceinline__ double eps_of<double>() { return DBL_EPSILON; }

__device__ __forceinline__ int player_at(int m, int r, int d) { return m == 0 ? 0 : 1 + ((m - 1 + r) % (d - 1)); }
__device__ __forceinline__ int position_of(int x, int r, int d) {
  if (x == 0) return 0;
  int m = (x - 1 - r) % (d - 1);
  if (m < 0) m += d - 1;
  return m + 1;
}
__device__ __forceinline__ int partner_of(int x, int r, int d) { return player_at(d - 1 - position_of(x, r, d), r, d); }

// Coefficients of column x of the round's rotation R: R[x][x] = alpha, R[partner][x] = beta.
template <class R>
__device__ __forceinline__ void rot_coeffs(const cx_t<R>* A, int d, int x, int px, cx_t<R>& alpha, cx_t<R>& beta) {
  using V = cx_t<R>;
  const int p = x < px ? x : px, q = x < px ? px : x;
  const R a = A[(long long)p * d + p].x, b = A[(long long)q * d + q].x;
  const V c = A[(long long)p * d + q];
  // |c| by hypot (no underflow of c.x^2 once the entry is tiny), and no rotation for entries that are
  // negligible against the diagonal: otherwise e^{i phi} = c / |c| loses unit modulus and the
  // accumulated eigenvectors drift from unitarity.
  const R r = hypot(c.x, c.y);
  R cs = R(1), sn = R(0);
  V eph = cmake<V>(R(1), R(0));  // e^{i phi}
  if (r > eps_of<R>() * R(1e-4) * (fabs(a) + fabs(b)) && r > tiny_normal<R>() * R(1e8)) {
    const R tau = (b - a) / (R(2) * r);
    const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
    cs = R(1) / sqrt(R(1) + t * t);
    sn = t * cs;
    eph = cmake<V>(c.x / r, c.y / r);
  }
  const V emph = cconj(eph);  // e^{-i phi}
  if (x == p) {
    alpha = cmake<V>(cs, R(0));
    beta = cmake<V>(-emph.x * sn, -emph.y * sn);
  } else {
    alpha = cmake<V>(emph.x * cs, emph.y * cs);
    beta = cmake<V>(sn, R(0));
  }
}

template <class V> __device__ __forceinline__ V cmul(V a, V b) { return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <class V> __device__ __forceinline__ V cmulc(V a, V b) { return cmake<V>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a) b

// Rotation of pair k of round r: indices p < q and the 2 x 2 block R = [[cs, sn], [-e^{-i phi} sn, e^{-i phi} cs]]
// (rows / columns in the order p, q), from the current A.
template <class R> struct PairRot {
  int p, q;
  cx_t<R> r_pp, r_pq, r_qp, r_qq;
};

template <class R>
__device__ __forceinline__ PairRot<R> pair_rotation(const cx_t<R>* A, int d, int k, int r) {
  using V = cx_t<R>;
  const int x = player_at(k, r, d), y = player_at(d - 1 - k, r, d);
  PairRot<R> pr;
  pr.p = x < y ? x : y;
  pr.q = x < y ? y : x;
  V alpha, beta;
  rot_coeffs<R>(A, d, pr.p, pr.q, alpha, beta);  // column p: R[p][p] = alpha, R[q][p] = beta
  pr.r_pp = alpha;
  pr.r_qp = beta;
  rot_coeffs<R>(A, d, pr.q, pr.p, alpha, beta);  // column q: R[q][q] = alpha, R[p][q] = beta
  pr.r_qq = alpha;
  pr.r_pq = beta;
  return pr;
}

// One round: every thread owns the 2 x 2 block (rows of pair k) x (columns of pair l) of A and of V,
// so each entry is read and written once: A' = R^dag A R on the block, V' = V R on rows {p_k, q_k}.
// Vi == NULL: no eigenvectors are accumulated; phi != NULL: the vector phi <- R^dag phi in place (the
// first block column, one thread per pair), so that after the sweeps phi = Q^dag phi_0.
template <class R>
__global__ void __launch_bounds__(256) k_jacobi_round(const cx_t<R>* __restrict__ A, cx_t<R>* __restrict__ Ao,
                                                       const cx_t<R>* __restrict__ Vi, cx_t<R>* __restrict__ Vo,
                                                       cx_t<R>* __restrict__ phi, int d, int r) {
  using V = cx_t<R>;
  constexpr int TP = 16;
  __shared__ PairRot<R> rk[TP], rl[TP];
  const int half = d >> 1;
  const int k0 = blockIdx.y * TP, l0 = blockIdx.x * TP;
  const int t = threadIdx.x;
  if (t < TP && k0 + t < half) rk[t] = pair_rotation<R>(A, d, k0 + t, r);
  else if (t >= 32 && t < 32 + TP && l0 + t - 32 < half) rl[t - 32] = pair_rotation<R>(A, d, l0 + t - 32, r);
  __syncthreads();
  if (phi != nullptr && blockIdx.x == 0 && t < TP && k0 + t < half) {
    const PairRot<R> a = rk[t];
    const V xp = phi[a.p], xq = phi[a.q];
    phi[a.p] = cadd(cmulc(a.r_pp, xp), cmulc(a.r_qp, xq));
    phi[a.q] = cadd(cmulc(a.r_pq, xp), cmulc(a.r_qq, xq));
  }
  const int k = k0 + t / TP, l = l0 + t % TP;
  if (k >= half || l >= half) return;
  const PairRot<R> a = rk[t / TP], b = rl[t % TP];
  const long long rp = (long long)a.p * d, rq = (long long)a.q * d;
  const V m_pp = A[rp + b.p], m_pq = A[rp + b.q], m_qp = A[rq + b.p], m_qq = A[rq + b.q];
  // M R_l (columns p_l, q_l)
  const V u_pp = cadd(cmul(m_pp, b.r_pp), cmul(m_pq, b.r_qp));
  const V u_pq = cadd(cmul(m_pp, b.r_pq), cmul(m_pq, b.r_qq));
  const V u_qp = cadd(cmul(m_qp, b.r_pp), cmul(m_qq, b.r_qp));
  const V u_qq = cadd(cmul(m_qp, b.r_pq), cmul(m_qq, b.r_qq));
  // R_k^dag (M R_l): row p' = conj(R[p][p]) row p + conj(R[q][p]) row q; row q' = conj(R[p][q]) row p + conj(R[q][q]) row q
  Ao[rp + b.p] = cadd(cmulc(a.r_pp, u_pp), cmulc(a.r_qp, u_qp));
  Ao[rp + b.q] = cadd(cmulc(a.r_pp, u_pq), cmulc(a.r_qp, u_qq));
  Ao[rq + b.p] = cadd(cmulc(a.r_pq, u_pp), cmulc(a.r_qq, u_qp));
  Ao[rq + b.q] = cadd(cmulc(a.r_pq, u_pq), cmulc(a.r_qq, u_qq));
  if (Vi == nullptr) return;
  // V' = V R on rows p_k, q_k, columns p_l, q_l
  const V v_pp = Vi[rp + b.p], v_pq = Vi[rp + b.q], v_qp = Vi[rq + b.p], v_qq = Vi[rq + b.q];
  Vo[rp + b.p] = cadd(cmul(v_pp, b.r_pp), cmul(v_pq, b.r_qp));
  Vo[rp + b.q] = cadd(cmul(v_pp, b.r_pq), cmul(v_pq, b.r_qq));
  Vo[rq + b.p] = cadd(cmul(v_qp, b.r_pp), cmul(v_qq, b.r_qp));
  Vo[rq + b.q] = cadd(cmul(v_qp, b.r_pq), cmul(v_qq, b.r_qq));
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

}  // namespace

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
  // an even number of sweeps of d - 1 (odd) rounds brings both ping-pong pairs back to A0 / V0
  V *Ain = w.A0, *Aout = w.A1, *Vin = w.V0, *Vout = w.V1;
  const dim3 grid((d / 2 + 15) / 16, (d / 2 + 15) / 16);
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int r = 0; r < d - 1; ++r) {
      k_jacobi_round<R><<<grid, 256, 0, s>>>(Ain, Aout, Vin, Vout, nullptr, d, r);
      V* t = Ain; Ain = Aout; Aout = t;
      t = Vin; Vin = Vout; Vout = t;
    }
  }
  w.A = Ain;  // diagonalised (A0)
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
  V *Ain = w.A0, *Aout = w.A1;
  const dim3 grid((d / 2 + 15) / 16, (d / 2 + 15) / 16);
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int r = 0; r < d - 1; ++r) {
      k_jacobi_round<R><<<grid, 256, 0, s>>>(Ain, Aout, nullptr, nullptr, phi, d, r);
      V* t = Ain; Ain = Aout; Aout = t;
    }
  }
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
