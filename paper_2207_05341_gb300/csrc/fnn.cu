// The Sec. 3.1 network (4^N -> 2N LeakyReLU -> 4^N linear), the Hermitian T of
// Sec. 3.2, their backward passes, and Rprop (Sec. 4.1) fused into the weight passes.
//
// Every kernel here streams the parameters once with vector loads; the hidden
// width H = 2N is a template parameter so that the H running sums live in
// registers.  Sums over the 4^N axis are reduced per block and then by the last
// block to arrive, in a fixed order (deterministic, no floating-point atomics).
#include "impl.h"

namespace qst {

template <class R> struct Vec;
template <> struct Vec<float> {
  static constexpr int W = 4;
  __device__ static void ld(const float* p, float* v) { float4 t = *reinterpret_cast<const float4*>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
  __device__ static void st(float* p, const float* v) { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }
};
template <> struct Vec<double> {
  static constexpr int W = 2;
  __device__ static void ld(const double* p, double* v) { double2 t = *reinterpret_cast<const double2*>(p); v[0] = t.x; v[1] = t.y; }
  __device__ static void st(double* p, const double* v) { *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]); }
};

template <class R> __device__ __forceinline__ R leaky(R x, R slope) { return x > R(0) ? x : slope * x; }

// Parameter rows of a weight pass whose loads are issued together before their
// Rprop updates and stores (keeps enough bytes in flight to stream at HBM rate).
constexpr int kRowBatch = 4;

// Reduce M per-thread values over the block; thread 0 writes them (as double) to out[0..M).
template <int M, class R>
__device__ __forceinline__ void block_reduce_to(const R (&v)[M], double* out) {
  __shared__ double red[8][M];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double x = warp_sum((double)v[j]);
    if (lane == 0) red[w][j] = x;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[q][j];
    out[j] = s;
  }
}

// In the last block: warp j sums partials[b * kPartialStride + j] over all blocks b
// (fixed order) for j < M, and calls fin(j, sum) from lane 0.
template <class F>
__device__ __forceinline__ void final_reduce(const double* partials, int M, F fin) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = w; j < M; j += nw) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += partials[(size_t)b * kPartialStride + j];
    s = warp_sum(s);
    if (lane == 0) fin(j, s);
  }
}

// Grid of a grid-stride streaming kernel: one wave of resident 256-thread CTAs (a CTA that had to wait
// for a free slot would run its whole share after the others), at most one thread per vector.
template <class K> static int stream_grid(K kernel, long long nvec) {
  int dev = 0, sms = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0);
  if (per < 1) per = 1;
  long long want = (nvec + 255) / 256;
  long long cap = (long long)per * sms;
  if (cap > kPartialBlocks) cap = kPartialBlocks;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

// ------------------------------------------------------------------ layer 1 forward
// pre = W1 f + b1, hid = LeakyReLU(pre), scal[1] = sum f
template <class R, int H>
__global__ void __launch_bounds__(256) k_l1_forward(const R* __restrict__ theta, const R* __restrict__ f,
                                                     long long n, R* pre, R* hid, double* scal,
                                                     double* partials, unsigned int* counter, R slope) {
  using VV = Vec<R>;
  constexpr int VW = VV::W;
  const R* W1 = theta;
  const R* b1 = theta + 2LL * H * n + n;
  R acc[H + 1];
#pragma unroll
  for (int j = 0; j <= H; ++j) acc[j] = R(0);
  const long long nv = n / VW;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    R fv[VW];
    VV::ld(f + i * VW, fv);
#pragma unroll
    for (int u = 0; u < VW; ++u) acc[H] += fv[u];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      R w[VW];
      VV::ld(W1 + (long long)j * n + i * VW, w);
#pragma unroll
      for (int u = 0; u < VW; ++u) acc[j] += w[u] * fv[u];
    }
  }
  block_reduce_to<H + 1>(acc, partials + (size_t)blockIdx.x * kPartialStride);
  if (last_block_arrived(counter)) {
    final_reduce(partials, H + 1, [&](int j, double s) {
      if (j < H) {
        const R p = (R)(s + (double)b1[j]);
        pre[j] = p;
        hid[j] = leaky(p, slope);
      } else {
        scal[1] = s;
      }
    });
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// ------------------------------------------------------------------ layer 2 + Hermitian T
// t = W2 h + b2 (k_layer2: a streaming pass over W2^T, 4^N-contiguous, every row read once;
// optionally folds max |t_i| into a max slot for the FP16 split of T);
// R = t as d x d row-major; T_ii = R_ii, T_ij = R_ij + i R_ji (i > j), T_ji = conj T_ij
// (k_hermitian_T: one CTA per tile pair (I, J), I >= J, of TS x TS tiles, t read from L2; the
// mixed-precision path writes T's 16-bit planes from t instead, tc_planes_T in gemm_tc.cu).
template <class R, int H>
__global__ void __launch_bounds__(256) k_layer2(const R* __restrict__ theta, const R* __restrict__ hid, long long n,
                                                 R* __restrict__ t, unsigned int* amax, const void* const* tab) {
  __shared__ R hs[H];
  rebind(tab, theta, hid, t, amax);
  grid_dep_wait();
  after_wait(theta, hid, t, amax);
  if (threadIdx.x < H) hs[threadIdx.x] = hid[threadIdx.x];
  __syncthreads();
  using VV = Vec<R>;
  constexpr int VW = VV::W;
  const R* W2T = theta + (long long)H * n;
  const R* b2 = theta + 2LL * H * n;
  const long long nv = n / VW;
  float m = 0.f;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nv; v += (long long)gridDim.x * blockDim.x) {
    const long long i = v * VW;
    R w[H][VW];
#pragma unroll
    for (int j = 0; j < H; ++j) VV::ld(W2T + (long long)j * n + i, w[j]);
    R ta[VW];
    VV::ld(b2 + i, ta);
#pragma unroll
    for (int j = 0; j < H; ++j) {
#pragma unroll
      for (int u = 0; u < VW; ++u) ta[u] += w[j][u] * hs[j];
    }
    VV::st(t + i, ta);
#pragma unroll
    for (int u = 0; u < VW; ++u) m = fmaxf(m, fabsf((float)ta[u]));
  }
  if (amax) block_absmax_to(m, amax);
}

// With Tt != NULL (Chol_Delta, Sec. 2.2.1 eq. T_matrix) the same entries are split: the lower triangle
// with the diagonal goes to T (upper triangle 0), the upper triangle with the diagonal, which is T^dag,
// to Tt (lower triangle 0).
template <class R>
__global__ void __launch_bounds__(256) k_hermitian_T(const R* __restrict__ t, int N, cx_t<R>* __restrict__ T,
                                                      cx_t<R>* __restrict__ Tt, const void* const* tab) {
  using V = cx_t<R>;
  rebind(tab, t, T, Tt);
  __shared__ R Ra[32][33];
  __shared__ R Rb[32][33];
  const int d = 1 << N;
  const int TS = d < 32 ? d : 32;
  int I, J;
  tri_decode(blockIdx.x, I, J);
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    Ra[r][c] = t[(long long)(I * TS + r) * d + J * TS + c];
    if (I != J) Rb[r][c] = t[(long long)(J * TS + r) * d + I * TS + c];
  }
  __syncthreads();
  const V zero = cmake<V>(R(0), R(0));
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    R re, im;
    if (I != J) { re = Ra[r][c]; im = Rb[c][r]; }
    else if (r > c) { re = Ra[r][c]; im = Ra[c][r]; }
    else if (r < c) { re = Ra[c][r]; im = -Ra[r][c]; }
    else { re = Ra[r][r]; im = R(0); }
    const long long o = (long long)(I * TS + r) * d + J * TS + c;
    if (!Tt) {
      T[o] = cmake<V>(re, im);
    } else {  // tile (I, J) holds the lower triangle of T; Tt = T^dag keeps only the upper one
      const bool lower = I != J || r >= c, upper = I == J && r <= c;
      T[o] = lower ? cmake<V>(re, im) : zero;
      Tt[o] = upper ? cmake<V>(re, im) : zero;
    }
  }
  if (I != J) {
    for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
      const int a = e / TS, b = e % TS;
      const long long o = (long long)(J * TS + a) * d + I * TS + b;
      if (!Tt) {
        T[o] = cmake<V>(Ra[b][a], -Rb[a][b]);
      } else {
        T[o] = zero;
        Tt[o] = cmake<V>(Ra[b][a], -Rb[a][b]);
      }
    }
  }
}

// ------------------------------------------------------------------ W2 pass (backward + Rprop)
// db2 = dt, dW2^T[j][i] = h_j dt_i, dh_j = sum_i W2^T[j][i] dt_i (old weights);
// then dpre = dh * LeakyReLU'(pre), db1 = dpre.  update: Rprop on W2^T, b2, b1; else write dtheta.
template <class R, int H, bool UPD>
__global__ void __launch_bounds__(256, 2) k_w2_pass(R* __restrict__ theta, R* __restrict__ step,
                                                  const R* __restrict__ dt, const R* __restrict__ hid,
                                                  const R* __restrict__ pre, R* dpre, R* __restrict__ dtheta,
                                                  long long n, double* partials, unsigned int* counter,
                                                  RpropCfg<R> rc, R slope) {
  using VV = Vec<R>;
  constexpr int VW = VV::W;
  constexpr int JB = kRowBatch;  // rows whose loads are issued together, ahead of their updates
  const long long o2 = (long long)H * n, ob2 = 2LL * H * n, ob1 = 2LL * H * n + n;
  __shared__ R hs[H];
  if (threadIdx.x < H) hs[threadIdx.x] = hid[threadIdx.x];
  __syncthreads();
  R acc[H];
#pragma unroll
  for (int j = 0; j < H; ++j) acc[j] = R(0);
  const long long nv = n / VW;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    const long long x = i * VW;
    R dv[VW];
    VV::ld(dt + x, dv);
    if (UPD) {
      R w[VW], st[VW];
      VV::ld(theta + ob2 + x, w); VV::ld(step + ob2 + x, st);
#pragma unroll
      for (int u = 0; u < VW; ++u) w[u] = rprop1(w[u], dv[u], st[u], rc);
      VV::st(theta + ob2 + x, w); VV::st(step + ob2 + x, st);
    } else {
      VV::st(dtheta + ob2 + x, dv);
    }
#pragma unroll
    for (int j0 = 0; j0 < H; j0 += JB) {
      R w[JB][VW], st[JB][VW];
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) {
        if (j0 + jj < H) {
          const long long oj = o2 + (long long)(j0 + jj) * n + x;
          VV::ld(theta + oj, w[jj]);
          if (UPD) VV::ld(step + oj, st[jj]);
        }
      }
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) {
        if (j0 + jj < H) {
          const int j = j0 + jj;
          const long long oj = o2 + (long long)j * n + x;
          R g[VW];
#pragma unroll
          for (int u = 0; u < VW; ++u) { acc[j] += w[jj][u] * dv[u]; g[u] = hs[j] * dv[u]; }
          if (UPD) {
#pragma unroll
            for (int u = 0; u < VW; ++u) w[jj][u] = rprop1(w[jj][u], g[u], st[jj][u], rc);
            VV::st(theta + oj, w[jj]); VV::st(step + oj, st[jj]);
          } else {
            VV::st(dtheta + oj, g);
          }
        }
      }
    }
  }
  block_reduce_to<H>(acc, partials + (size_t)blockIdx.x * kPartialStride);
  if (last_block_arrived(counter)) {
    final_reduce(partials, H, [&](int j, double s) {
      const R p = pre[j];
      const R dp = (R)s * (p > R(0) ? R(1) : slope);
      dpre[j] = dp;
      if (UPD) {
        R st = step[ob1 + j];
        theta[ob1 + j] = rprop1(theta[ob1 + j], dp, st, rc);
        step[ob1 + j] = st;
      } else {
        dtheta[ob1 + j] = dp;
      }
    });
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// ------------------------------------------------------------------ W1 pass (backward + Rprop + next forward)
// dW1[j][i] = dpre_j f_i.  update: Rprop on W1, then pre = W1' f + b1', hid = LeakyReLU(pre),
// scal[1] = sum f (the hidden layer of the next iteration); else write dtheta.
template <class R, int H, bool UPD>
__global__ void __launch_bounds__(256, 2) k_w1_pass(R* __restrict__ theta, R* __restrict__ step,
                                                  const R* __restrict__ f, const R* __restrict__ dpre, R* pre,
                                                  R* hid, R* __restrict__ dtheta, long long n, double* scal,
                                                  double* partials, unsigned int* counter, RpropCfg<R> rc, R slope) {
  using VV = Vec<R>;
  constexpr int VW = VV::W;
  const long long ob1 = 2LL * H * n + n;
  __shared__ R dps[H];
  if (threadIdx.x < H) dps[threadIdx.x] = dpre[threadIdx.x];
  __syncthreads();
  R acc[H + 1];
#pragma unroll
  for (int j = 0; j <= H; ++j) acc[j] = R(0);
  constexpr int JB = kRowBatch;
  const long long nv = n / VW;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    const long long x = i * VW;
    R fv[VW];
    VV::ld(f + x, fv);
#pragma unroll
    for (int u = 0; u < VW; ++u) acc[H] += fv[u];
#pragma unroll
    for (int j0 = 0; j0 < H; j0 += JB) {
      R w[JB][VW], st[JB][VW];
      if (UPD) {
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          if (j0 + jj < H) {
            const long long oj = (long long)(j0 + jj) * n + x;
            VV::ld(theta + oj, w[jj]); VV::ld(step + oj, st[jj]);
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) {
        if (j0 + jj < H) {
          const int j = j0 + jj;
          const long long oj = (long long)j * n + x;
          R g[VW];
#pragma unroll
          for (int u = 0; u < VW; ++u) g[u] = dps[j] * fv[u];
          if (UPD) {
#pragma unroll
            for (int u = 0; u < VW; ++u) {
              w[jj][u] = rprop1(w[jj][u], g[u], st[jj][u], rc);
              acc[j] += w[jj][u] * fv[u];
            }
            VV::st(theta + oj, w[jj]); VV::st(step + oj, st[jj]);
          } else {
            VV::st(dtheta + oj, g);
          }
        }
      }
    }
  }
  if (!UPD) return;
  block_reduce_to<H + 1>(acc, partials + (size_t)blockIdx.x * kPartialStride);
  if (last_block_arrived(counter)) {
    final_reduce(partials, H + 1, [&](int j, double s) {
      if (j < H) {
        const R p = (R)(s + (double)theta[ob1 + j]);
        pre[j] = p;
        hid[j] = leaky(p, slope);
      } else {
        scal[1] = s;
      }
    });
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// ------------------------------------------------------------------ dL/dt from Y = G T
// Gamma = Y + Y^dag;  dR_ij = 2 Re Gamma_ij, dR_ji = 2 Im Gamma_ij (i > j), dR_ii = Re Gamma_ii.
template <class R>
__global__ void __launch_bounds__(256) k_symmetrize(const cx_t<R>* __restrict__ Y, R* __restrict__ dt, int d,
                                                     const void* const* tab) {
  __shared__ R Ar[32][33], Ai[32][33], Br[32][33], Bi[32][33];
  rebind(tab, Y, dt);
  grid_dep_wait();
  after_wait(Y, dt);
  const int TS = d < 32 ? d : 32;
  int I, J;
  tri_decode(blockIdx.x, I, J);
  if constexpr (sizeof(R) == 4) {
    if (TS == 32 && blockDim.x == 256) {
      // FP32: 16-byte accesses (two complex per load, four outputs per store), so that a tile pair
      // takes a quarter of the global stores and half the loads of the element-wise form below
      const int t = threadIdx.x;
      float4 a[2], b[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int q = t + 256 * k, row = q >> 4, col = (q & 15) * 2;
        a[k] = *reinterpret_cast<const float4*>(Y + (long long)(I * 32 + row) * d + J * 32 + col);
        b[k] = I != J ? *reinterpret_cast<const float4*>(Y + (long long)(J * 32 + row) * d + I * 32 + col)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int q = t + 256 * k, row = q >> 4, col = (q & 15) * 2;
        Ar[row][col] = a[k].x; Ai[row][col] = a[k].y; Ar[row][col + 1] = a[k].z; Ai[row][col + 1] = a[k].w;
        Br[row][col] = b[k].x; Bi[row][col] = b[k].y; Br[row][col + 1] = b[k].z; Bi[row][col + 1] = b[k].w;
      }
      __syncthreads();
      const int r = t >> 3, c = (t & 7) * 4;
      float v[4];
      if (I != J) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = R(2) * (Ar[r][c + u] + Br[c + u][r]);
        *reinterpret_cast<float4*>(dt + (long long)(I * 32 + r) * d + J * 32 + c) = make_float4(v[0], v[1], v[2], v[3]);
        // upper tile (J, I): element (J 32 + r, I 32 + c + u) = 2 Im Gamma_{(I 32 + c + u), (J 32 + r)}
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = R(2) * (Ai[c + u][r] - Bi[r][c + u]);
        *reinterpret_cast<float4*>(dt + (long long)(J * 32 + r) * d + I * 32 + c) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int cc = c + u;
          if (r > cc) v[u] = R(2) * (Ar[r][cc] + Ar[cc][r]);
          else if (r < cc) v[u] = R(2) * (Ai[cc][r] - Ai[r][cc]);
          else v[u] = R(2) * Ar[r][r];
        }
        *reinterpret_cast<float4*>(dt + (long long)(I * 32 + r) * d + J * 32 + c) = make_float4(v[0], v[1], v[2], v[3]);
      }
      return;
    }
  }
  if (TS == 32 && blockDim.x == 256) {  // all 8 loads of a thread in flight at once
    cx_t<R> a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = threadIdx.x + 256 * k, r = e >> 5, c = e & 31;
      a[k] = Y[(long long)(I * 32 + r) * d + J * 32 + c];
      b[k] = Y[(long long)(J * 32 + r) * d + I * 32 + c];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = threadIdx.x + 256 * k, r = e >> 5, c = e & 31;
      Ar[r][c] = a[k].x; Ai[r][c] = a[k].y; Br[r][c] = b[k].x; Bi[r][c] = b[k].y;
    }
  } else {
    for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
      const int r = e / TS, c = e % TS;
      const long long ia = (long long)(I * TS + r) * d + J * TS + c;
      const long long ib = (long long)(J * TS + r) * d + I * TS + c;
      const cx_t<R> a = Y[ia], b = Y[ib];
      Ar[r][c] = a.x; Ai[r][c] = a.y; Br[r][c] = b.x; Bi[r][c] = b.y;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    if (I != J) {
      // lower tile (I, J): rows > cols
      dt[(long long)(I * TS + r) * d + J * TS + c] = R(2) * (Ar[r][c] + Br[c][r]);
      // upper tile (J, I): element (J TS + r, I TS + c) = 2 Im Gamma_{(I TS + c),(J TS + r)}
      dt[(long long)(J * TS + r) * d + I * TS + c] = R(2) * (Ai[c][r] - Bi[r][c]);
    } else {
      R v;
      if (r > c) v = R(2) * (Ar[r][c] + Ar[c][r]);
      else if (r < c) v = R(2) * (Ai[c][r] - Ai[r][c]);
      else v = R(2) * Ar[r][r];
      dt[(long long)(I * TS + r) * d + J * TS + c] = v;
    }
  }
}

// Chol_Delta backward (Sec. 2.2.1 eq. T_matrix): with X = T^dag T and Z = T G (lower tiles computed),
// dL = 2 Re Tr[G T^dag dT] gives dR_ii = 2 Re Z_ii and, for i > j, dR_ij = 2 Re Z_ij, dR_ji = 2 Im Z_ij.
template <class R>
__global__ void __launch_bounds__(256) k_tri_grad(const cx_t<R>* __restrict__ Z, R* __restrict__ dt, int d) {
  __shared__ R Zr[32][33], Zi[32][33];
  const int TS = d < 32 ? d : 32;
  int I, J;
  tri_decode(blockIdx.x, I, J);
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    const cx_t<R> z = Z[(long long)(I * TS + r) * d + J * TS + c];
    Zr[r][c] = z.x;
    Zi[r][c] = z.y;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
    const int r = e / TS, c = e % TS;
    if (I != J) {
      dt[(long long)(I * TS + r) * d + J * TS + c] = R(2) * Zr[r][c];
      dt[(long long)(J * TS + r) * d + I * TS + c] = R(2) * Zi[c][r];  // (J TS + r, I TS + c): Im Z at (I TS + c, J TS + r)
    } else {
      const R v = r > c ? R(2) * Zr[r][c] : (r < c ? R(2) * Zi[c][r] : R(2) * Zr[r][r]);
      dt[(long long)(I * TS + r) * d + J * TS + c] = v;
    }
  }
}

// ------------------------------------------------------------------ launchers
#define QST_SWITCH_H(H, ...)                      \
  switch (H) {                                    \
    case 2: { constexpr int HH = 2; __VA_ARGS__; } break;   \
    case 4: { constexpr int HH = 4; __VA_ARGS__; } break;   \
    case 6: { constexpr int HH = 6; __VA_ARGS__; } break;   \
    case 8: { constexpr int HH = 8; __VA_ARGS__; } break;   \
    case 10: { constexpr int HH = 10; __VA_ARGS__; } break; \
    case 12: { constexpr int HH = 12; __VA_ARGS__; } break; \
    case 14: { constexpr int HH = 14; __VA_ARGS__; } break; \
    case 16: { constexpr int HH = 16; __VA_ARGS__; } break; \
    case 18: { constexpr int HH = 18; __VA_ARGS__; } break; \
    case 20: { constexpr int HH = 20; __VA_ARGS__; } break; \
    case 22: { constexpr int HH = 22; __VA_ARGS__; } break; \
    case 24: { constexpr int HH = 24; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;        \
  }

template <class R> static RpropCfg<R> rcfg(const NetCfg& c) {
  RpropCfg<R> r;
  r.eta_minus = (R)c.eta_minus; r.eta_plus = (R)c.eta_plus; r.step_min = (R)c.step_min; r.step_max = (R)c.step_max;
  return r;
}

template <class R>
cudaError_t net_l1_forward(const Dims& D, const R* theta, const R* f, R* pre, R* hid, double* scal,
                           double* partials, unsigned int* counter, const NetCfg& c, cudaStream_t s) {
  // the grid of the W1 pass, whose sums this forward must reproduce bit for bit
  QST_SWITCH_H(D.H, {
    const int grid = stream_grid(k_w1_pass<R, HH, true>, D.n / Vec<R>::W);
    k_l1_forward<R, HH><<<grid, 256, 0, s>>>(theta, f, D.n, pre, hid, scal, partials, counter, (R)c.slope);
  });
  return cudaGetLastError();
}

template <class R>
cudaError_t net_build_T(const Dims& D, const R* theta, const R* hid, R* t, cx_t<R>* T, unsigned int* amax,
                        cudaStream_t s, cx_t<R>* Tt) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long nv = D.n / Vec<R>::W;
  const long long want = (nv + 255) / 256;
  QST_SWITCH_H(D.H, {
    static const int per_sm = [] {  // resident CTAs per SM: one wave of grid-stride CTAs
      int b = 1;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_layer2<R, HH>, 256, 0);
      return b < 1 ? 1 : b;
    }();
    const long long grid = want < (long long)per_sm * sms ? want : (long long)per_sm * sms;
    BatchArgs ba;
    if (!batch_take(ba, {theta, hid, t, amax})) {
      cudaError_t e = launch_dep(k_layer2<R, HH>, dim3((unsigned)grid, 1, ba.nz), dim3(256), 0, s, theta, hid, D.n, t,
                                 amax, ba.tab);
      if (e != cudaSuccess) return e;
    }
  });
  if (!T) return cudaGetLastError();
  return net_hermitian_T<R>(D, t, T, Tt, s);
}

template <class R> cudaError_t net_hermitian_T(const Dims& D, const R* t, cx_t<R>* T, cx_t<R>* Tt, cudaStream_t s) {
  const int TS = D.d < 32 ? D.d : 32;
  const int nt = D.d / TS;
  const unsigned pairs = (unsigned)(nt * (nt + 1) / 2);
  BatchArgs ba;
  if (batch_take(ba, {t, T, Tt})) return cudaSuccess;
  k_hermitian_T<R><<<dim3(pairs, 1, ba.nz), 256, 0, s>>>(t, D.N, T, Tt, ba.tab);
  return cudaGetLastError();
}

template <class R>
cudaError_t net_w2_pass(const Dims& D, R* theta, R* step, const R* dt, const R* hid, const R* pre,
                        R* dpre, R* dtheta, double* partials, unsigned int* counter, const NetCfg& c, bool update,
                        cudaStream_t s) {
  const long long nv = D.n / Vec<R>::W;
  if (update) {
    QST_SWITCH_H(D.H, k_w2_pass<R, HH, true><<<stream_grid(k_w2_pass<R, HH, true>, nv), 256, 0, s>>>(
                          theta, step, dt, hid, pre, dpre, dtheta, D.n, partials, counter, rcfg<R>(c),
                          (R)c.slope));
  } else {
    QST_SWITCH_H(D.H, k_w2_pass<R, HH, false><<<stream_grid(k_w2_pass<R, HH, false>, nv), 256, 0, s>>>(
                          theta, step, dt, hid, pre, dpre, dtheta, D.n, partials, counter, rcfg<R>(c),
                          (R)c.slope));
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t net_w1_pass(const Dims& D, R* theta, R* step, const R* f, const R* dpre, R* pre, R* hid,
                        R* dtheta, double* scal, double* partials, unsigned int* counter, const NetCfg& c,
                        bool update, cudaStream_t s) {
  const long long nv = D.n / Vec<R>::W;
  // both variants use the grid of the updating pass (the partition k_l1_forward reproduces)
  if (update) {
    QST_SWITCH_H(D.H, k_w1_pass<R, HH, true><<<stream_grid(k_w1_pass<R, HH, true>, nv), 256, 0, s>>>(
                          theta, step, f, dpre, pre, hid, dtheta, D.n, scal, partials, counter, rcfg<R>(c),
                          (R)c.slope));
  } else {
    QST_SWITCH_H(D.H, k_w1_pass<R, HH, false><<<stream_grid(k_w1_pass<R, HH, true>, nv), 256, 0, s>>>(
                          theta, step, f, dpre, pre, hid, dtheta, D.n, scal, partials, counter, rcfg<R>(c),
                          (R)c.slope));
  }
  return cudaGetLastError();
}

template <class R> cudaError_t net_symmetrize(const Dims& D, const cx_t<R>* Y, R* dt, cudaStream_t s) {
  const int TS = D.d < 32 ? D.d : 32;
  const int nt = D.d / TS;
  BatchArgs ba;
  if (batch_take(ba, {Y, dt})) return cudaSuccess;
  return launch_dep(k_symmetrize<R>, dim3((unsigned)(nt * (nt + 1) / 2), 1, ba.nz), dim3(256), 0, s, Y, dt, D.d,
                    ba.tab);
}

template <class R> cudaError_t net_tri_grad(const Dims& D, const cx_t<R>* Z, R* dt, cudaStream_t s) {
  const int TS = D.d < 32 ? D.d : 32;
  const int nt = D.d / TS;
  k_tri_grad<R><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(Z, dt, D.d);
  return cudaGetLastError();
}

#define QST_INST(R)                                                                                              \
  template cudaError_t net_l1_forward<R>(const Dims&, const R*, const R*, R*, R*, double*, double*, unsigned int*, \
                                         const NetCfg&, cudaStream_t);                                           \
  template cudaError_t net_build_T<R>(const Dims&, const R*, const R*, R*, cx_t<R>*, unsigned int*, cudaStream_t,  \
                                      cx_t<R>*);                                                                 \
  template cudaError_t net_tri_grad<R>(const Dims&, const cx_t<R>*, R*, cudaStream_t);                         \
  template cudaError_t net_hermitian_T<R>(const Dims&, const R*, cx_t<R>*, cx_t<R>*, cudaStream_t);            \
  template cudaError_t net_w2_pass<R>(const Dims&, R*, R*, const R*, const R*, const R*, R*, R*, double*, \
                                      unsigned int*, const NetCfg&, bool, cudaStream_t);                         \
  template cudaError_t net_w1_pass<R>(const Dims&, R*, R*, const R*, const R*, R*, R*, R*, double*,     \
                                      double*, unsigned int*, const NetCfg&, bool, cudaStream_t);                \
  template cudaError_t net_symmetrize<R>(const Dims&, const cx_t<R>*, R*, cudaStream_t);
QST_INST(float)
QST_INST(double)
#undef QST_INST

}  // namespace qst
