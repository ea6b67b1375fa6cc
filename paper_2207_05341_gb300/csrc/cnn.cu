// The CNN mapping network of App. A, forward and backward with Rprop (the alternative to the 3-layer
// FNN of Sec. 3.1; the state map, likelihood and POVM passes downstream are shared).
//
//   f (4^N) as a d x d matrix (row-major) -> 3 x 3 convolution, stride 1, zero padding 1, 10 maps with
//   bias -> ReLU -> max-pool over 2^(N-3)-square windows (stride the same) -> 640 features
//   -> dense 640 -> 4N (LeakyReLU) -> dense 4N -> 4^N (linear) = t.
//
// theta (CNN layout): [W2^T (H x n) | b2 (n) | W1 (H x 640) | b1 (H) | conv W (10 x 3 x 3) | conv b (10)],
// H = 4N; the Rprop state has the same layout.  The output layer streams like the FNN's (one pass for t,
// one backward pass with Rprop fused: in FP32 the bulk-copy W2 pass of the FNN, run on the two halves
// of the 4N rows); the convolution, pooling and first dense layer are small.
//
// Pooling windows of at least 64 x 64 pixels (N >= 9) are cut into 32 x 64 tiles: a CTA stages its
// tile with a one-pixel halo in shared memory, evaluates all 10 maps there and leaves per map the
// tile's best (value, position); a second kernel reduces the tiles of each window.  The best of a set
// is the largest value, on equal values the smallest row-major position, a total order, so the result
// does not depend on how the set is split.  Smaller windows take one CTA per feature.
//
// The pooling argmax is a decision taken in floating point: each convolution value is accumulated in
// the context's precision in a fixed order (bias, then the 9 taps row-major), every product and sum
// rounded separately (no fused multiply-add), and ties go to the first row-major position of the
// window, so that a reference evaluating the same expression in the same precision takes the same
// decisions.  All reductions have a fixed order.
#include <type_traits>

#include "impl.h"

namespace qst {

namespace {

constexpr int kMaps = 10;
constexpr int kGrid = 8;
constexpr int kFeat = kMaps * kGrid * kGrid;  // 640
constexpr int kStride = 64;                   // doubles per block in partials (>= H = 4N <= 48)
constexpr int kMaxBlocks = kPartialBlocks * kPartialStride / kStride;  // within the context's partials
constexpr int kColsPer = 2;                   // tile columns per thread
constexpr int kRowsPer = 8;                   // tile rows per thread
constexpr int kTW = 32 * kColsPer;            // tile columns: a warp across
constexpr int kTH = kRowsPer * 8;             // tile rows: the 8 warps of 256 threads down
constexpr int kTileMinP = 64;                 // tiled path for windows of at least 64 x 64

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

// The dense layer 640 -> H with LeakyReLU, features in shared memory sf: warp w of the block takes
// units w, w + nw, ...; lane l the terms m = l, l + 32, ... (in order, the 20 loads issued together),
// then a fixed shuffle tree and b1.
template <class R>
__device__ __forceinline__ void dense1_block(int H, const R* sf, const R* __restrict__ W1, const R* __restrict__ b1,
                                             R* pre, R* hid, R slope) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = threadIdx.x >> 5; j < H; j += nw) {
    R w[kFeat / 32];
#pragma unroll
    for (int r = 0; r < kFeat / 32; ++r) w[r] = W1[(long long)j * kFeat + r * 32 + lane];
    R acc = R(0);
#pragma unroll
    for (int r = 0; r < kFeat / 32; ++r) acc += w[r] * sf[r * 32 + lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      acc += b1[j];
      pre[j] = acc;
      hid[j] = leaky_c(acc, slope);
    }
  }
}

// Dense 640 -> H with LeakyReLU (one block of 1024 threads: a warp per unit).
template <class R>
__global__ void __launch_bounds__(1024) k_cnn_dense1(const R* __restrict__ feats, const R* __restrict__ W1,
                                                     const R* __restrict__ b1, int H, R* pre, R* hid, R slope) {
  __shared__ R sf[kFeat];
  for (int m = threadIdx.x; m < kFeat; m += blockDim.x) sf[m] = feats[m];
  __syncthreads();
  dense1_block(H, sf, W1, b1, pre, hid, slope);
}

// (v2, i2) beats (v, i): larger value, or equal value at a smaller position.
template <class R> __device__ __forceinline__ bool beats(R v2, int i2, R v, int i) {
  return v2 > v || (v2 == v && i2 < i);
}

// Tiled convolution (windows of p >= 64): CTA b takes tile b % per_win of window b / per_win (tiles
// row-major within the window), lane l of warp w the 16 pixels of columns 2l, 2l + 1 in rows
// 8w .. 8w + 7 of the 64 x 64 tile (scanned row-major, so a thread keeps its first position on ties).
// Per map: the tile's best (value, image position) to tv / ti; sum of f over the tile (FP64, fixed
// order) to tf.
template <class R>
__global__ void __launch_bounds__(256) k_cnn_conv_tiles(const R* __restrict__ f, int N, const R* __restrict__ cW,
                                                         const R* __restrict__ cB, R* __restrict__ tv,
                                                         int* __restrict__ ti, double* __restrict__ tf) {
  __shared__ R tile[kTH + 2][kTW + 2];
  __shared__ R sw[kMaps][10];  // 9 taps row-major, then the bias
  __shared__ R rv[8][kMaps];
  __shared__ int ri[8][kMaps];
  __shared__ double rf[8];
  const int d = 1 << N, p = d / kGrid;
  const int tx = p / kTW, per_win = tx * (p / kTH);
  const int win = blockIdx.x / per_win, r = blockIdx.x % per_win;
  const int y0 = (win / kGrid) * p + (r / tx) * kTH, x0 = (win % kGrid) * p + (r % tx) * kTW;
  for (int e = threadIdx.x; e < (kTH + 2) * (kTW + 2); e += blockDim.x) {
    const int ry = e / (kTW + 2), rx = e % (kTW + 2);
    const int y = y0 + ry - 1, x = x0 + rx - 1;
    tile[ry][rx] = (y >= 0 && y < d && x >= 0 && x < d) ? f[(long long)y * d + x] : R(0);
  }
  if (threadIdx.x < kMaps * 10) {
    const int c = threadIdx.x / 10, k = threadIdx.x % 10;
    sw[c][k] = k < 9 ? cW[c * 9 + k] : cB[c];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cx = lane * kColsPer, rg = warp;
  R v[kRowsPer + 2][kColsPer + 2];
#pragma unroll
  for (int a = 0; a < kRowsPer + 2; ++a)
#pragma unroll
    for (int b = 0; b < kColsPer + 2; ++b) v[a][b] = tile[rg * kRowsPer + a][cx + b];
  double fs = 0.0;
#pragma unroll
  for (int rr = 0; rr < kRowsPer; ++rr)
#pragma unroll
    for (int cc = 0; cc < kColsPer; ++cc) fs += (double)v[rr + 1][cc + 1];
#pragma unroll 1
  for (int c = 0; c < kMaps; ++c) {
    R w[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = sw[c][k];
    const R b = sw[c][9];
    R best = R(0);
    int bi = 0;  // rr * kColsPer + cc of the best
#pragma unroll
    for (int rr = 0; rr < kRowsPer; ++rr)
#pragma unroll
      for (int cc = 0; cc < kColsPer; ++cc) {
        R acc = b;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) acc = add_rn(acc, mul_rn(w[ky * 3 + kx], v[rr + ky][cc + kx]));
        if ((rr == 0 && cc == 0) || acc > best) {  // row-major scan: the first position is kept on ties
          best = acc;
          bi = rr * kColsPer + cc;
        }
      }
    int idx = (y0 + rg * kRowsPer + bi / kColsPer) * d + x0 + cx + bi % kColsPer;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (beats(v2, i2, best, idx)) {
        best = v2;
        idx = i2;
      }
    }
    if (lane == 0) {
      rv[warp][c] = best;
      ri[warp][c] = idx;
    }
  }
  fs = warp_sum(fs);
  if (lane == 0) rf[warp] = fs;
  __syncthreads();
  if (threadIdx.x < kMaps) {
    const int c = threadIdx.x;
    R best = rv[0][c];
    int idx = ri[0][c];
    for (int q = 1; q < 8; ++q)
      if (beats(rv[q][c], ri[q][c], best, idx)) {
        best = rv[q][c];
        idx = ri[q][c];
      }
    tv[(size_t)blockIdx.x * kMaps + c] = best;
    ti[(size_t)blockIdx.x * kMaps + c] = idx;
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += rf[q];
    tf[blockIdx.x] = t;
  }
}

// Pooling over the tiles of each window: warp i < 640 reduces feature i (map i / 64, window i % 64)
// over its window's per_win tiles; warp 640 sums tf (fixed order) into scal[1].  The last block to
// finish evaluates the dense layer 640 -> H (blocks of 1024 threads: a warp per hidden unit).
template <class R>
__global__ void __launch_bounds__(1024) k_cnn_pool(const R* __restrict__ tv, const int* __restrict__ ti,
                                                   const double* __restrict__ tf, int per_win, R* feats, int* pos,
                                                   R* vals, const R* __restrict__ W1, const R* __restrict__ b1, int H,
                                                   R* pre, R* hid, R slope, double* scal, unsigned int* counter) {
  __shared__ R sf[kFeat];
  const int lane = threadIdx.x & 31, gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw < kFeat) {
    const int c = gw / (kGrid * kGrid), win = gw % (kGrid * kGrid);
    R best = R(0);
    int idx = -1;
    for (int t = lane; t < per_win; t += 32) {
      const size_t o = (size_t)(win * per_win + t) * kMaps + c;
      const R v2 = tv[o];
      const int i2 = ti[o];
      if (idx < 0 || beats(v2, i2, best, idx)) {
        best = v2;
        idx = i2;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (i2 >= 0 && (idx < 0 || beats(v2, i2, best, idx))) {
        best = v2;
        idx = i2;
      }
    }
    if (lane == 0) {
      pos[gw] = idx;
      vals[gw] = best;
      feats[gw] = best > R(0) ? best : R(0);
    }
  } else if (gw == kFeat) {
    double t = 0.0;
    for (int b = lane; b < kGrid * kGrid * per_win; b += 32) t += tf[b];
    t = warp_sum(t);
    if (lane == 0) scal[1] = t;
  }
  if (last_block_arrived(counter)) {
    for (int m = threadIdx.x; m < kFeat; m += blockDim.x) sf[m] = __ldcg(feats + m);
    __syncthreads();
    dense1_block(H, sf, W1, b1, pre, hid, slope);
    if (threadIdx.x == 0) *counter = 0u;
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
//   dW_c[ky][kx] += dfeat_i f[y + ky - 1][x + kx - 1], db_c += dfeat_i.
// k_cnn_head_grad (one CTA of 1024 threads) takes dfeat, b1 and the convolution; k_cnn_w1_update,
// launched after it (every read of the old W1 is done), W1.  The 100 convolution gradients are 10
// strided partial sums each (features q = r, r + 10, ... of the map), added in order.
// UPD: Rprop in place; else the gradients go to the d* pointers.
template <class R, int H, bool UPD>
__global__ void __launch_bounds__(1024) k_cnn_head_grad(const R* __restrict__ f, int N, const int* __restrict__ pos,
                                                         const R* __restrict__ vals, const R* __restrict__ dpre,
                                                         const R* __restrict__ W1, R* b1, R* Sb1, R* cW, R* ScW,
                                                         R* cB, R* ScB, R* db1, R* dcW, R* dcB, RpropCfg<R> rc) {
  __shared__ R dfeat[kFeat];
  __shared__ R dp[H];
  __shared__ R part[kMaps * 10][10];
  const int d = 1 << N, t = threadIdx.x;
  if (t < H) dp[t] = dpre[t];
  __syncthreads();
  if (t < kFeat) {
    R w[H];
#pragma unroll
    for (int j = 0; j < H; ++j) w[j] = W1[(long long)j * kFeat + t];
    R acc = R(0);
#pragma unroll
    for (int j = 0; j < H; ++j) acc += w[j] * dp[j];
    dfeat[t] = vals[t] > R(0) ? acc : R(0);  // ReLU'(conv) at the pooled position
  }
  if (t < H) {
    if (UPD) {
      R sj = Sb1[t];
      b1[t] = rprop1(b1[t], dp[t], sj, rc);
      Sb1[t] = sj;
    } else {
      db1[t] = dp[t];
    }
  }
  __syncthreads();
  // convolution: output o = (map c, k) with k < 9 the tap (k / 3, k % 3) and k == 9 the bias;
  // thread (o, r) sums the features q = r, r + 10, ... of map c
  constexpr int kPer = (kGrid * kGrid + 9) / 10;
  if (t < kMaps * 10 * 10) {
    const int o = t / 10, r = t % 10, c = o / 10, k = o % 10;
    R v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = r + 10 * u;
      v[u] = R(1);
      if (q < kGrid * kGrid && k < 9) {
        const int i = c * kGrid * kGrid + q;
        const int y = pos[i] / d + k / 3 - 1, x = pos[i] % d + k % 3 - 1;
        v[u] = (y >= 0 && y < d && x >= 0 && x < d) ? f[(long long)y * d + x] : R(0);
      }
    }
    R acc = R(0);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = r + 10 * u;
      if (q < kGrid * kGrid) acc += dfeat[c * kGrid * kGrid + q] * v[u];  // v = 1 for the bias
    }
    part[o][r] = acc;
  }
  __syncthreads();
  if (t < kMaps * 10) {
    const int c = t / 10, k = t % 10;
    R acc = R(0);
#pragma unroll
    for (int r = 0; r < 10; ++r) acc += part[t][r];
    R* P = k == 9 ? cB + c : cW + c * 9 + k;
    R* S = k == 9 ? ScB + c : ScW + c * 9 + k;
    if (UPD) {
      R sv = *S;
      *P = rprop1(*P, acc, sv, rc);
      *S = sv;
    } else {
      if (k == 9) dcB[c] = acc;
      else dcW[c * 9 + k] = acc;
    }
  }
}

// dW1[j][m] = dpre_j feat_m for the H x 640 weights, one per thread; Rprop in place (UPD) or to dW1.
template <class R, bool UPD>
__global__ void __launch_bounds__(256) k_cnn_w1_update(const R* __restrict__ feats, const R* __restrict__ dpre, int H,
                                                        R* __restrict__ W1, R* __restrict__ S1, R* __restrict__ dW1,
                                                        RpropCfg<R> rc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= H * kFeat) return;
  const R g = dpre[e / kFeat] * feats[e % kFeat];
  if (UPD) {
    R st = S1[e];
    W1[e] = rprop1(W1[e], g, st, rc);
    S1[e] = st;
  } else {
    dW1[e] = g;
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

static long long conv_tiles(int N) {
  const long long p = (1LL << N) / kGrid;
  return p >= kTileMinP ? (long long)kGrid * kGrid * (p / kTW) * (p / kTH) : 0;
}

size_t cnn_part_doubles(int N, size_t real_bytes) {
  const size_t t = (size_t)conv_tiles(N);
  const size_t bytes = t * 8 + t * kMaps * real_bytes + t * kMaps * 4;
  return bytes / 8 + 2;
}

template <class R>
cudaError_t cnn_hidden(const Dims& D, const R* theta, const R* f, R* feats, int* pos, R* vals, R* pre, R* hid,
                       double slope, double* part, double* partials, unsigned int* counter, double* scal,
                       cudaStream_t s) {
  CnnParams<R> p = cnn_params(const_cast<R*>(theta), D.H, D.n);
  const long long tiles = conv_tiles(D.N);
  if (tiles > 0) {
    // part: tf [tiles] doubles | tv [tiles x 10] reals | ti [tiles x 10] ints
    double* tf = part;
    R* tv = reinterpret_cast<R*>(tf + tiles);
    int* ti = reinterpret_cast<int*>(tv + tiles * kMaps);
    k_cnn_conv_tiles<R><<<(unsigned)tiles, 256, 0, s>>>(f, D.N, p.cW, p.cB, tv, ti, tf);
    const int per_win = (int)(tiles / (kGrid * kGrid));
    k_cnn_pool<R><<<(kFeat + 1 + 31) / 32, 1024, 0, s>>>(tv, ti, tf, per_win, feats, pos, vals, p.W1, p.b1, D.H, pre,
                                                      hid, (R)slope, scal, counter);
  } else {
    k_cnn_features<R><<<kFeat, 256, 0, s>>>(f, D.N, p.cW, p.cB, feats, pos, vals, partials, counter, scal);
    k_cnn_dense1<R><<<1, 1024, 0, s>>>(feats, p.W1, p.b1, D.H, pre, hid, (R)slope);
  }
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

bool cnn_bulk_ok(const Dims& D) { return D.H % 2 == 0 && wpass_bulk_ok(D.H / 2, D.n); }

template <class R>
cudaError_t cnn_output_backward(const Dims& D, R* theta, R* state, R* dtheta, const R* dt, const R* hid,
                                const R* pre, R* dpre, double* partials, unsigned int* counter, unsigned int* flags,
                                const NetCfg& c, bool bulk, cudaStream_t s) {
  const bool upd = dtheta == nullptr;
  if constexpr (std::is_same<R, float>::value) {
    if (upd && bulk) {  // the FNN's bulk W2 pass on rows [0, H/2) (with b2), then on rows [H/2, H)
      const int h2 = D.H / 2;
      const long long n = D.n, ob2 = (long long)D.H * n;
      cudaError_t e = w2_rows_pass_bulk(n, h2, theta, state, 0, ob2, dt, hid, pre, dpre, partials, counter, flags,
                                        c, s);
      if (e != cudaSuccess) return e;
      return w2_rows_pass_bulk(n, h2, theta, state, (long long)h2 * n, -1, dt, hid + h2, pre + h2, dpre + h2,
                               partials, counter, flags, c, s);
    }
  }
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
  return cudaGetLastError();
}

template <class R>
cudaError_t cnn_head_backward(const Dims& D, R* theta, R* state, R* dtheta, const R* f, const R* feats,
                              const int* pos, const R* vals, const R* dpre, const NetCfg& c, cudaStream_t s) {
  const bool upd = dtheta == nullptr;
  CnnParams<R> p = cnn_params(theta, D.H, D.n);
  CnnParams<R> q = upd ? cnn_params(state, D.H, D.n) : CnnParams<R>{};
  CnnParams<R> g = upd ? CnnParams<R>{} : cnn_params(dtheta, D.H, D.n);
  RpropCfg<R> rc{(R)c.eta_minus, (R)c.eta_plus, (R)c.step_min, (R)c.step_max};
  QST_SWITCH_H4(D.H, {
    if (upd)
      k_cnn_head_grad<R, HH, true><<<1, 1024, 0, s>>>(f, D.N, pos, vals, dpre, p.W1, p.b1, q.b1, p.cW, q.cW, p.cB,
                                                      q.cB, nullptr, nullptr, nullptr, rc);
    else
      k_cnn_head_grad<R, HH, false><<<1, 1024, 0, s>>>(f, D.N, pos, vals, dpre, p.W1, p.b1, nullptr, p.cW, nullptr,
                                                       p.cB, nullptr, g.b1, g.cW, g.cB, rc);
  });
  const int blocks = (D.H * kFeat + 255) / 256;
  if (upd)
    k_cnn_w1_update<R, true><<<blocks, 256, 0, s>>>(feats, dpre, D.H, p.W1, q.W1, nullptr, rc);
  else
    k_cnn_w1_update<R, false><<<blocks, 256, 0, s>>>(feats, dpre, D.H, p.W1, nullptr, g.W1, rc);
  return cudaGetLastError();
}

#define QST_CNN_INST(R)                                                                                          \
  template cudaError_t cnn_hidden<R>(const Dims&, const R*, const R*, R*, int*, R*, R*, R*, double, double*,       \
                                     double*, unsigned int*, double*, cudaStream_t);                            \
  template cudaError_t cnn_output<R>(const Dims&, const R*, const R*, R*, unsigned int*, cudaStream_t);          \
  template cudaError_t cnn_output_backward<R>(const Dims&, R*, R*, R*, const R*, const R*, const R*, R*, double*, \
                                              unsigned int*, unsigned int*, const NetCfg&, bool, cudaStream_t);  \
  template cudaError_t cnn_head_backward<R>(const Dims&, R*, R*, R*, const R*, const R*, const int*, const R*,   \
                                            const R*, const NetCfg&, cudaStream_t);
QST_CNN_INST(float)
QST_CNN_INST(double)
#undef QST_CNN_INST

}  // namespace qst
