// Quantum state fidelity of Sec. 2.3 (eq. F_QF) on the GPU, through the decomposition route of
// eq. fq_decom, against the targets of the Sec. 4 sweeps:
//   rho = w |psi><psi| / <psi|psi> + (1 - w) I / d   (pure: w = 1; white noise: w = p; depolarising:
//                                                      w = 1 - lambda).
// The state's own decomposition comes from that of T (Sec. 3.2): T = Q Lambda Q^dag gives
// rho^ = Q diag(g) Q^dag / S with g = lambda^2 (Chol_H) or |lambda|^P (A_P) and S = sum g.  eq. fq_decom
// needs the eigenvalues s' of sqrt(rho^) rho sqrt(rho^); in the basis Q that matrix is
//   (1 / S) [ c diag(g) + e u u^dag ],   c = (1 - w) / d,  e = w / <psi|psi>,  u_i = sqrt(g_i) phi_i,
// with phi = Q^dag psi: a diagonal plus a rank-one term.  Its eigenvalues nu_k are the roots of the
// secular equation 1 + e sum_i g_i |phi_i|^2 / (c g_i - nu) = 0, one between each pair of consecutive
// sorted poles c g_(k) <= nu_k <= c g_(k+1) and the largest in [c g_max, c g_max + e sum_i g_i |phi_i|^2]
// (Golub, "Some modified matrix eigenvalue problems", SIAM Review 15, 1973).  Each root is bracketed
// and bisected in FP64, so the small ones (near c g_i) keep their relative accuracy, which a dense
// eigensolver of the d x d matrix does not give (its error on them is of order eps times the largest,
// and their square roots enter the sum); F = (sum_k sqrt(nu_k))^2 / S.
#include "impl.h"

namespace qst {

namespace {

constexpr int kBisect = 100;  // bisection steps at most (the bracket shrinks to one ulp well before)

// phi2_i = |(Q^dag psi)_i|^2, one warp per row of Q^dag, FP64 sums (lanes strided, fixed shuffle tree).
template <class R>
__global__ void __launch_bounds__(256) k_fq_phi(const cx_t<R>* __restrict__ Qh, const cx_t<R>* __restrict__ psi,
                                                 int d, double* __restrict__ phi2) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= d) return;
  double re = 0.0, im = 0.0;
  for (int j = lane; j < d; j += 32) {
    const cx_t<R> q = Qh[(long long)i * d + j], p = psi[j];
    re += (double)q.x * (double)p.x - (double)q.y * (double)p.y;
    im += (double)q.x * (double)p.y + (double)q.y * (double)p.x;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) phi2[i] = re * re + im * im;
}

// phi2_i = |phi_i|^2 of a projection already formed.
template <class R>
__global__ void __launch_bounds__(256) k_fq_abs2(const cx_t<R>* __restrict__ phi, int d, double* __restrict__ phi2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d) phi2[i] = (double)phi[i].x * (double)phi[i].x + (double)phi[i].y * (double)phi[i].y;
}

// One CTA: S = sum g, <psi|psi>, the poles c g_i and weights e g_i phi2_i sorted by pole (bitonic sort
// in shared memory, d a power of two), the upper end of the last bracket; out[0] = S, out[1] = bound.
template <class R>
__global__ void __launch_bounds__(1024) k_fq_sort(const R* __restrict__ g, const double* __restrict__ phi2,
                                                   const cx_t<R>* __restrict__ psi, int d, double w,
                                                   double* __restrict__ pole, double* __restrict__ wt,
                                                   double* __restrict__ out) {
  extern __shared__ double sm[];
  double* key = sm;
  double* val = sm + d;
  __shared__ double red[3][32];
  double sg = 0.0, sp = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    sg += (double)g[i];
    sp += (double)psi[i].x * (double)psi[i].x + (double)psi[i].y * (double)psi[i].y;
  }
  sg = warp_sum(sg);
  sp = warp_sum(sp);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[0][warp] = sg;
    red[1][warp] = sp;
  }
  __syncthreads();
  double S = 0.0, n2 = 0.0;
  for (int q = 0; q < nw; ++q) {
    S += red[0][q];
    n2 += red[1][q];
  }
  const double c = (1.0 - w) / d, e = w / n2;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double gi = (double)g[i];
    key[i] = c * gi;
    val[i] = e * gi * phi2[i];
  }
  __syncthreads();
  for (int k = 2; k <= d; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < d; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const bool up = (i & k) == 0;
          if ((key[i] > key[p]) == up) {
            const double tk = key[i], tv = val[i];
            key[i] = key[p];
            val[i] = val[p];
            key[p] = tk;
            val[p] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  double sv = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    pole[i] = key[i];
    wt[i] = val[i];
    sv += val[i];
  }
  sv = warp_sum(sv);
  if (lane == 0) red[2][warp] = sv;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tv = 0.0;
    for (int q = 0; q < nw; ++q) tv += red[2][q];
    out[0] = S;
    out[1] = key[d - 1] + tv;
  }
}

// One warp per root k: bisection of f(nu) = 1 + sum_i wt_i / (pole_i - nu) on [pole_k, pole_{k+1}]
// (the last on [pole_max, bound]); f increases between poles, so f(mid) < 0 moves the lower end.  An
// empty bracket (equal poles) is its own root.  The last block sums sqrt(nu_k) in order:
// out[2] = (sum_k sqrt(nu_k))^2 / S.
__global__ void __launch_bounds__(256) k_fq_roots(const double* __restrict__ pole, const double* __restrict__ wt,
                                                   int d, double* __restrict__ rs, double* out,
                                                   unsigned int* counter) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k < d) {
    double lo = pole[k];
    double hi = k + 1 < d ? pole[k + 1] : out[1];
    if (hi > lo) {
      for (int it = 0; it < kBisect; ++it) {
        const double mid = lo + 0.5 * (hi - lo);
        if (!(mid > lo && mid < hi)) break;
        double s = 0.0;
        for (int i = lane; i < d; i += 32) s += wt[i] / (pole[i] - mid);
        s = __shfl_sync(0xffffffffu, warp_sum(s), 0);  // every lane takes lane 0's decision
        if (1.0 + s < 0.0) lo = mid;
        else hi = mid;
      }
    }
    const double nu = lo + 0.5 * (hi - lo);
    if (lane == 0) rs[k] = nu > 0.0 ? sqrt(nu) : 0.0;
  }
  if (last_block_arrived(counter)) {
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int i = threadIdx.x; i < d; i += 32) t += __ldcg(rs + i);
      t = warp_sum(t);
      if (threadIdx.x == 0) {
        out[2] = t * t / out[0];
        *counter = 0u;
      }
    }
  }
}

}  // namespace

size_t state_fidelity_scratch_doubles(int d) { return 4 * (size_t)d; }

template <class R>
cudaError_t state_fidelity_from_decomposition(int d, const cx_t<R>* Qh, const cx_t<R>* phi, const R* g,
                                              const cx_t<R>* psi, double w, double* scratch, double* out,
                                              unsigned int* counter, cudaStream_t s) {
  double* phi2 = scratch;
  double* pole = scratch + d;
  double* wt = scratch + 2 * (size_t)d;
  double* rs = scratch + 3 * (size_t)d;
  if (Qh) k_fq_phi<R><<<(d + 7) / 8, 256, 0, s>>>(Qh, psi, d, phi2);
  else k_fq_abs2<R><<<(d + 255) / 256, 256, 0, s>>>(phi, d, phi2);
  const size_t smem = 2 * (size_t)d * sizeof(double);
  cudaError_t e = ensure_dynamic_smem((const void*)k_fq_sort<R>, smem);
  if (e != cudaSuccess) return e;
  k_fq_sort<R><<<1, 1024, smem, s>>>(g, phi2, psi, d, w, pole, wt, out);
  k_fq_roots<<<(d + 7) / 8, 256, 0, s>>>(pole, wt, d, rs, out, counter);
  return cudaGetLastError();
}

template cudaError_t state_fidelity_from_decomposition<float>(int, const float2*, const float2*, const float*,
                                                              const float2*, double, double*, double*, unsigned int*,
                                                              cudaStream_t);
template cudaError_t state_fidelity_from_decomposition<double>(int, const double2*, const double2*, const double*,
                                                               const double2*, double, double*, double*,
                                                               unsigned int*, cudaStream_t);

}  // namespace qst
