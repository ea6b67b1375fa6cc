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

#include <algorithm>
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
      if (threadIdx.x < NP) {  // the round's rotations, from the block before the round
        const int k = threadIdx.x;
        const int x = player_at(k, r, kBJ), y = player_at(kBJ - 1 - k, r, kBJ);
        const int p = x < y ? x : y, q = x < y ? y : x;
        float2 al, be;
        rot_coeffs<float>(Sb, kBJS, p, q, al, be);
        r_pp[k] = al;
        r_qp[k] = be;
        rot_coeffs<float>(Sb, kBJS, q, p, al, be);
        r_qq[k] = al;
        r_pq[k] = be;
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
