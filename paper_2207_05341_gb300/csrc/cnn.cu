// The CNN mapping network of App. A, forward and backward with Rprop (the alternative to the 3-layer
// FNN of Sec. 3.1; the state map, likelihood and POVM passes downstream are shared).
//
//   f (4^N) as a d x d matrix (row-major) -> 3 x 3 convolution, stride 1, zero padding 1, 10 maps with
//   bias -> ReLU -> max-pool over 2^(N-3)-square windows (stride the same) -> 640 features
//   -> dense 640 -> 4N (LeakyReLU) -> dense 4N -> 4^N (linear) = t.
//
// theta (CNN layout): [W2^T (H x n) | b2 (n) | W1 (H x 640) | b1 (H) | conv W (10 x 3 x 3) | conv b (10)],
// H = 4N; the Rprop state has the same layout.  The output layer streams like the FNN's (one pass for t,
// one backward pass with Rprop fused); the convolution, pooling and first dense layer are small.
//
// The pooling argmax is a decision taken in floating point: each convolution value is accumulated in
// the context's precision in a fixed order (bias, then the 9 taps row-major), every product and sum
// rounded separately (no fused multiply-add), and ties go to the first row-major position of the
// window, so that a reference evaluating the same expression in the same precision takes the same
// decisions.  All reductions have a fixed order.
#include "impl.h"

namespace qst {

namespace {

constexpr int kMaps = 10;
constexpr int kGrid = 8;
constexpr int kFeat = kMaps * kGrid * kGrid;  // 640
constexpr int kStride = 64;                   // doubles per block in partials (>= H = 4N <= 48)
constexpr int kMaxBlocks = kPartialBlocks * kPartialStride / kStride;  // within the context's partials

template <class R> __device__ __forceinline__ R mul_rn(R a, R b);
template <class R> __device__ __forceinline__ R add_rn(R a, R b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }

template <class R> __device__ __forceinline__ R leaky_c(R x, R s) { return x > R(0) ? x : s * x; }

// One CTA per pooled feature (map c, window (I, J)): the convolution over the window, its argmax
// (first row-major position on ties) and ReLU of the maximum.  The CTAs of map 0 also sum f over their
// windows, which tile the image: the last CTA to finish writes sum f to scal[1] (fixed order).
template <class R>
__global__ void __launch_bounds__(256) k_cnn_features(const R* __restrict__ f, int N, const R* __restrict__ cW,
                                                       const R* __restrict__ cB, R* __restrict__ feats,
                                                       int* __restrict__ pos, R* __restrict__ vals,
                                                       double* partials, unsigned int* counter, double* scal) {
  __shared__ R sv[256];
  __shared__ int si[256];
  __shared__ double sred[8];
  const int d = 1 << N, p = d / kGrid;
  const int i = blockIdx.x, c = i / (kGrid * kGrid), I = (i / kGrid) % kGrid, J = i % kGrid;
  R w[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = cW[c * 9 + k];
  const R b = cB[c];
  R best = R(0);
  int bi = -1;
  double fsum = 0.0;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int y = I * p + e / p, x = J * p + e % p;
    if (c == 0) fsum += (double)f[(long long)y * d + x];
    R acc = b;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int yy = y + ky - 1, xx = x + kx - 1;
        const R v = (yy >= 0 && yy < d && xx >= 0 && xx < d) ? f[(long long)yy * d + xx] : R(0);
        acc = add_rn(acc, mul_rn(w[ky * 3 + kx], v));
      }
    if (bi < 0 || acc > best) { best = acc; bi = e; }  // e grows within a thread: first index kept on ties
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const R v2 = sv[threadIdx.x + s];
      const int i2 = si[threadIdx.x + s];
      const int i1 = si[threadIdx.x];
      if (i2 >= 0 && (i1 < 0 || v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < i1))) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int e = si[0];
    pos[i] = (I * p + e / p) * d + J * p + e % p;
    vals[i] = sv[0];
    feats[i] = sv[0] > R(0) ? sv[0] : R(0);
  }
  fsum = warp_sum(fsum);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = fsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) t += sred[w8];
    partials[blockIdx.x] = t;  // 0 for the CTAs of maps 1..9
  }
  if (last_block_arrived(counter)) {
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int b2 = threadIdx.x; b2 < kGrid * kGrid; b2 += 32) t += partials[b2];  // map 0's windows
      t = warp_sum(t);
      if (threadIdx.x == 0) {
        scal[1] = t;
        *counter = 0u;
      }
    }
  }
}

// Dense 640 -> H with LeakyReLU: one thread per hidden unit, terms in index order.
template <class R>
__global__ void __launch_bounds__(64) k_cnn_dense1(const R* __restrict__ feats, const R* __restrict__ W1,
                                                    const R* __restrict__ b1, int H, R* pre, R* hid, R slope) {
  __shared__ R sf[kFeat];
  for (int m = threadIdx.x; m < kFeat; m += blockDim.x) sf[m] = feats[m];
  __syncthreads();
  const int j = threadIdx.x;
  if (j < H) {
    R acc = b1[j];
    for (int m = 0; m < kFeat; ++m) acc += W1[(long long)j * kFeat + m] * sf[m];
    pre[j] = acc;
    hid[j] = leaky_c(acc, slope);
  }
}

// Output layer: t = W2 h + b2, 4 columns per thread, rows in batches of 8 (loads before the FMAs).
template <class R, int H>
__global__ void __launch_bounds__(256) k_cnn_output(const R* __restrict__ W2T, const R* __restrict__ b2,
                                                     const R* __restrict__ hid, long long n, R* __restrict__ t,
                                                     unsigned int* amax) {
  __shared__ R hs[H];
  if (threadIdx.x < H) hs[threadIdx.x] = hid[threadIdx.x];
  __syncthreads();
  float m = 0.f;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n / 4; v += (long long)gridDim.x * blockDim.x) {
    const long long i = v * 4;
    R acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = b2[i + u];
#pragma unroll
    for (int j0 = 0; j0 < H; j0 += 8) {
      R w[8][4];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (j0 + jj < H)
#pragma unroll
          for (int u = 0; u < 4; ++u) w[jj][u] = W2T[(long long)(j0 + jj) * n + i + u];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (j0 + jj < H)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] += w[jj][u] * hs[j0 + jj];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      t[i + u] = acc[u];
      m = fmaxf(m, fabsf((float)acc[u]));
    }
  }
  if (amax) block_absmax_to(m, amax);
}

// Output-layer backward (Sec. 3.1 layer 2 of the CNN head): db2 = dt, dW2^T[j][i] = h_j dt_i,
// dh_j = sum_i W2^T[j][i] dt_i (old weights) -> dpre_j = dh_j LeakyReLU'(pre_j) by the last block.
// UPD: Rprop in place; else the gradient goes to dW2T / db2.
template <class R, int H, bool UPD>
__global__ void __launch_bounds__(256) k_cnn_output_back(R* __restrict__ W2T, R* __restrict__ S2T,
                                                          R* __restrict__ b2, R* __restrict__ Sb2,
                                                          const R* __restrict__ dt, const R* __restrict__ hid,
                                                          const R* __restrict__ pre, R* dpre, R* __restrict__ dW2T,
                                                          R* __restrict__ db2, long long n, double* partials,
                                                          unsigned int* counter, RpropCfg<R> rc, R slope) {
  __shared__ R hs[H];
  __shared__ double red[8][H];
  if (threadIdx.x < H) hs[threadIdx.x] = hid[threadIdx.x];
  __syncthreads();
  R acc[H];
#pragma unroll
  for (int j = 0; j < H; ++j) acc[j] = R(0);
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n / 4; v += (long long)gridDim.x * blockDim.x) {
    const long long i = v * 4;
    R g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) g[u] = dt[i + u];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (UPD) {
        R s = Sb2[i + u];
        b2[i + u] = rprop1(b2[i + u], g[u], s, rc);
        Sb2[i + u] = s;
      } else {
        db2[i + u] = g[u];
      }
    }
#pragma unroll
    for (int j0 = 0; j0 < H; j0 += 4) {
      R w[4][4], s[4][4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long o = (long long)(j0 + jj) * n + i + u;
          w[jj][u] = W2T[o];
          if (UPD) s[jj][u] = S2T[o];
        }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = j0 + jj;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long o = (long long)j * n + i + u;
          acc[j] += w[jj][u] * g[u];
          const R gw = hs[j] * g[u];
          if (UPD) {
            W2T[o] = rprop1(w[jj][u], gw, s[jj][u], rc);
            S2T[o] = s[jj][u];
          } else {
            dW2T[o] = gw;
          }
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const double x = warp_sum((double)acc[j]);
    if (lane == 0) red[wp][j] = x;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    double sum = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += red[q][j];
    partials[(size_t)blockIdx.x * kStride + j] = sum;
  }
  if (last_block_arrived(counter)) {
    for (int j = wp; j < H; j += (int)(blockDim.x >> 5)) {
      double sum = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) sum += partials[(size_t)b * kStride + j];
      sum = warp_sum(sum);
      if (lane == 0) {
        const R pj = pre[j];
        dpre[j] = (R)sum * (pj > R(0) ? R(1) : slope);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// Backward of the dense layer 640 -> H and of the convolution through the pooling argmax, with Rprop:
//   dfeat_m = sum_j W1[j][m] dpre_j (old W1), dW1[j][m] = dpre_j feat_m, db1 = dpre,
//   for each feature i of map c with positive convolution value at its position (y, x):
//   dW_c[ky][kx] += dfeat_i f[y + ky - 1][x + kx - 1], db_c += dfeat_i (features in index order).
// One CTA of 1024 threads.  UPD: Rprop in place; else the gradients go to the d* pointers.
template <class R, bool UPD>
__global__ void __launch_bounds__(1024) k_cnn_head_back(const R* __restrict__ f, int N, const R* __restrict__ feats,
                                                         const int* __restrict__ pos, const R* __restrict__ vals,
                                                         const R* __restrict__ dpre, int H, R* W1, R* S1, R* b1, R* Sb1,
                                                         R* cW, R* ScW, R* cB, R* ScB, R* dW1, R* db1, R* dcW,
                                                         R* dcB, RpropCfg<R> rc) {
  __shared__ R dfeat[kFeat];
  __shared__ R dp[64];
  const int d = 1 << N;
  if (threadIdx.x < H) dp[threadIdx.x] = dpre[threadIdx.x];
  __syncthreads();
  for (int m = threadIdx.x; m < kFeat; m += blockDim.x) {
    R acc = R(0);
    for (int j = 0; j < H; ++j) acc += W1[(long long)j * kFeat + m] * dp[j];
    dfeat[m] = vals[m] > R(0) ? acc : R(0);  // ReLU'(conv) at the pooled position
  }
  __syncthreads();
  for (int e = threadIdx.x; e < H * kFeat; e += blockDim.x) {
    const int j = e / kFeat, m = e % kFeat;
    const R g = dp[j] * feats[m];
    if (UPD) {
      R s = S1[e];
      W1[e] = rprop1(W1[e], g, s, rc);
      S1[e] = s;
    } else {
      dW1[e] = g;
    }
  }
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    if (UPD) {
      R s = Sb1[j];
      b1[j] = rprop1(b1[j], dp[j], s, rc);
      Sb1[j] = s;
    } else {
      db1[j] = dp[j];
    }
  }
  // convolution: one thread per weight (10 x 9) and per bias (10)
  const int t = threadIdx.x;
  if (t < kMaps * 10) {
    const int c = t / 10, k = t % 10;  // k < 9: tap (k / 3, k % 3); k == 9: bias
    R acc = R(0);
    for (int q = 0; q < kGrid * kGrid; ++q) {
      const int i = c * kGrid * kGrid + q;
      const R g = dfeat[i];
      if (k == 9) {
        acc += g;
      } else {
        const int y = pos[i] / d + k / 3 - 1, x = pos[i] % d + k % 3 - 1;
        const R v = (y >= 0 && y < d && x >= 0 && x < d) ? f[(long long)y * d + x] : R(0);
        acc += g * v;
      }
    }
    R* P = k == 9 ? cB + c : cW + c * 9 + k;
    R* S = k == 9 ? ScB + c : ScW + c * 9 + k;
    if (UPD) {
      R s = *S;
      *P = rprop1(*P, acc, s, rc);
      *S = s;
    } else {
      if (k == 9) dcB[c] = acc;
      else dcW[c * 9 + k] = acc;
    }
  }
}

#define QST_SWITCH_H4(H, ...)                                    \
  switch (H) {                                                   \
    case 12: { constexpr int HH = 12; __VA_ARGS__; } break;      \
    case 16: { constexpr int HH = 16; __VA_ARGS__; } break;      \
    case 20: { constexpr int HH = 20; __VA_ARGS__; } break;      \
    case 24: { constexpr int HH = 24; __VA_ARGS__; } break;      \
    case 28: { constexpr int HH = 28; __VA_ARGS__; } break;      \
    case 32: { constexpr int HH = 32; __VA_ARGS__; } break;      \
    case 36: { constexpr int HH = 36; __VA_ARGS__; } break;      \
    case 40: { constexpr int HH = 40; __VA_ARGS__; } break;      \
    case 44: { constexpr int HH = 44; __VA_ARGS__; } break;      \
    case 48: { constexpr int HH = 48; __VA_ARGS__; } break;      \
    default: return cudaErrorInvalidValue;                       \
  }

template <class K> int resident_grid(K kernel, long long work) {
  int dev = 0, sms = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0);
  if (per < 1) per = 1;
  long long g = (work + 255) / 256;
  long long cap = (long long)per * sms;
  if (cap > kMaxBlocks) cap = kMaxBlocks;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

template <class R> struct CnnParams {
  R *W2T, *b2, *W1, *b1, *cW, *cB;
};
template <class R> CnnParams<R> cnn_params(R* theta, int H, long long n) {
  CnnParams<R> p;
  p.W2T = theta;
  p.b2 = p.W2T + (long long)H * n;
  p.W1 = p.b2 + n;
  p.b1 = p.W1 + (long long)H * kFeat;
  p.cW = p.b1 + H;
  p.cB = p.cW + kMaps * 9;
  return p;
}

}  // namespace

size_t cnn_theta_size(int N) {
  const size_t n = (size_t)1 << (2 * N), H = 4 * (size_t)N;
  return H * n + n + H * kFeat + H + kMaps * 9 + kMaps;
}

template <class R>
cudaError_t cnn_hidden(const Dims& D, const R* theta, const R* f, R* feats, int* pos, R* vals, R* pre, R* hid,
                       double slope, double* partials, unsigned int* counter, double* scal, cudaStream_t s) {
  CnnParams<R> p = cnn_params(const_cast<R*>(theta), D.H, D.n);
  k_cnn_features<R><<<kFeat, 256, 0, s>>>(f, D.N, p.cW, p.cB, feats, pos, vals, partials, counter, scal);
  k_cnn_dense1<R><<<1, 64, 0, s>>>(feats, p.W1, p.b1, D.H, pre, hid, (R)slope);
  return cudaGetLastError();
}

template <class R>
cudaError_t cnn_output(const Dims& D, const R* theta, const R* hid, R* t, unsigned int* amax, cudaStream_t s) {
  CnnParams<R> p = cnn_params(const_cast<R*>(theta), D.H, D.n);
  QST_SWITCH_H4(D.H, {
    const int grid = resident_grid(k_cnn_output<R, HH>, D.n / 4);
    k_cnn_output<R, HH><<<grid, 256, 0, s>>>(p.W2T, p.b2, hid, D.n, t, amax);
  });
  return cudaGetLastError();
}

template <class R>
cudaError_t cnn_backward(const Dims& D, R* theta, R* state, R* dtheta, const R* f, const R* dt, const R* feats,
                         const int* pos, const R* vals, const R* pre, const R* hid, R* dpre, double* partials,
                         unsigned int* counter, const NetCfg& c, cudaStream_t s) {
  const bool upd = dtheta == nullptr;
  CnnParams<R> p = cnn_params(theta, D.H, D.n);
  CnnParams<R> q = upd ? cnn_params(state, D.H, D.n) : CnnParams<R>{};
  CnnParams<R> g = upd ? CnnParams<R>{} : cnn_params(dtheta, D.H, D.n);
  RpropCfg<R> rc{(R)c.eta_minus, (R)c.eta_plus, (R)c.step_min, (R)c.step_max};
  QST_SWITCH_H4(D.H, {
    if (upd) {
      const int grid = resident_grid(k_cnn_output_back<R, HH, true>, D.n / 4);
      k_cnn_output_back<R, HH, true><<<grid, 256, 0, s>>>(p.W2T, q.W2T, p.b2, q.b2, dt, hid, pre, dpre, nullptr,
                                                          nullptr, D.n, partials, counter, rc, (R)c.slope);
    } else {
      const int grid = resident_grid(k_cnn_output_back<R, HH, true>, D.n / 4);
      k_cnn_output_back<R, HH, false><<<grid, 256, 0, s>>>(p.W2T, nullptr, p.b2, nullptr, dt, hid, pre, dpre, g.W2T,
                                                           g.b2, D.n, partials, counter, rc, (R)c.slope);
    }
  });
  if (upd)
    k_cnn_head_back<R, true><<<1, 1024, 0, s>>>(f, D.N, feats, pos, vals, dpre, D.H, p.W1, q.W1, p.b1, q.b1, p.cW,
                                                q.cW, p.cB, q.cB, nullptr, nullptr, nullptr, nullptr, rc);
  else
    k_cnn_head_back<R, false><<<1, 1024, 0, s>>>(f, D.N, feats, pos, vals, dpre, D.H, p.W1, nullptr, p.b1, nullptr,
                                                 p.cW, nullptr, p.cB, nullptr, g.W1, g.b1, g.cW, g.cB, rc);
  return cudaGetLastError();
}

#define QST_CNN_INST(R)                                                                                          \
  template cudaError_t cnn_hidden<R>(const Dims&, const R*, const R*, R*, int*, R*, R*, R*, double, double*,       \
                                     unsigned int*, double*, cudaStream_t);                                     \
  template cudaError_t cnn_output<R>(const Dims&, const R*, const R*, R*, unsigned int*, cudaStream_t);          \
  template cudaError_t cnn_backward<R>(const Dims&, R*, R*, R*, const R*, const R*, const R*, const int*,         \
                                       const R*, const R*, const R*, R*, double*, unsigned int*, const NetCfg&,  \
                                       cudaStream_t);
QST_CNN_INST(float)
QST_CNN_INST(double)
#undef QST_CNN_INST

}  // namespace qst
