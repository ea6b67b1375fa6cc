// Rprop weight passes of the Sec. 3.1 network (FP32, in-place update) with bulk-copy staging.
//
// Each CTA walks chunks of kCols consecutive columns of the 4^N axis.  For a chunk,
// one thread issues 1-D bulk copies (cp.async.bulk, completion counted on an
// mbarrier) of every parameter row segment (weights, Rprop steps, previous signs)
// and of the chunk of dt (W2 pass) or f (W1 pass) into one of two shared-memory
// stages; all threads then update the chunk in shared memory (one column per
// thread, all H rows), and the same thread writes the rows back with bulk stores.
// The next chunk's loads are in flight while a chunk is updated, so the pass
// streams at HBM rate without depending on registers for bytes in flight.
//
// The arithmetic is that of k_w2_pass / k_w1_pass in fnn.cu (same Rprop; the sums
// over the 4^N axis are per-thread partials reduced in a fixed order, so the pass is
// deterministic, though the partition of those sums differs from fnn.cu's kernel).
// Every mbarrier wait is bounded; a timeout raises flags[1] and the kernel drains
// what it issued (bounded) before returning.
#include "impl.h"

namespace qst {

namespace {

constexpr int kCols = 256;                  // columns per chunk = threads per CTA
constexpr unsigned long long kWait = 4000000000ULL;

__device__ __forceinline__ uint32_t s_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  if (bar_try(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  while (!bar_try(bar, parity))
    if (clock64() - t0 > kWait) return false;
  return true;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   s_u32(dst)),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(s_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Stage layout (bytes): w[H][kCols] f32 | st[H][kCols] f32 | sg[H][kCols] i8 | vec[kCols] f32 (dt or f)
//                       | W2 pass only: b2 w, st [kCols] f32, sg [kCols] i8
template <int H, bool W2> struct Stage {
  static constexpr int kW = 0;
  static constexpr int kSt = kW + H * kCols * 4;
  static constexpr int kSg = kSt + H * kCols * 4;
  static constexpr int kVec = kSg + H * kCols;
  static constexpr int kBw = kVec + kCols * 4;
  static constexpr int kBst = kBw + kCols * 4;
  static constexpr int kBsg = kBst + kCols * 4;
  static constexpr int kBytes = W2 ? kBsg + kCols : kBw;  // multiple of 16
  static constexpr uint32_t kTx = (uint32_t)kBytes;
};

template <class R> __device__ __forceinline__ R leaky_b(R x, R slope) { return x > R(0) ? x : slope * x; }

template <int M>
__device__ __forceinline__ void block_sum_to(const float (&v)[M], double* out) {
  __shared__ double red[8][M];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double x = warp_sum((double)v[j]);
    if (lane == 0) red[w][j] = x;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q][j];
    out[j] = s;
  }
}

template <class F>
__device__ __forceinline__ void final_sum(const double* partials, int M, F fin) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = w; j < M; j += nw) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += partials[(size_t)b * kPartialStride + j];
    s = warp_sum(s);
    if (lane == 0) fin(j, s);
  }
}

// W2 pass (W2 true) or W1 pass (W2 false); see k_w2_pass / k_w1_pass in fnn.cu for the arithmetic.
template <int H, bool W2>
__global__ void __launch_bounds__(kCols, 2) k_wpass_bulk(float* __restrict__ theta, float* __restrict__ step,
                                                        int8_t* __restrict__ sign, const float* __restrict__ vec,
                                                        const float* __restrict__ hidv, const float* __restrict__ pre,
                                                        float* dpre_io, float* pre_out, float* hid_out, double* scal,
                                                        long long n, double* partials, unsigned int* counter,
                                                        unsigned int* flags, RpropCfg<float> rc, float slope) {
  using S = Stage<H, W2>;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ float hs[H];
  __shared__ int s_fail;
  const long long rowoff = W2 ? (long long)H * n : 0;  // W2^T or W1 rows
  const long long ob2 = 2LL * H * n, ob1 = 2LL * H * n + n;
  const long long nchunks = n / kCols;
  const int tid = threadIdx.x;
  if (tid < H) hs[tid] = W2 ? hidv[tid] : dpre_io[tid];  // W2: h; W1: dpre
  if (tid == 0) {
    s_fail = 0;
    bar_init(s_u32(&bars[0]), 1);
    bar_init(s_u32(&bars[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto issue_loads = [&](long long chunk, int s) {
    uint8_t* st = smem + s * S::kBytes;
    const long long c0 = chunk * kCols;
    const uint32_t bar = s_u32(&bars[s]);
    bar_expect(bar, S::kTx);
    for (int j = 0; j < H; ++j) {
      const long long o = rowoff + (long long)j * n + c0;
      bulk_load(st + S::kW + j * kCols * 4, theta + o, kCols * 4, bar);
      bulk_load(st + S::kSt + j * kCols * 4, step + o, kCols * 4, bar);
      bulk_load(st + S::kSg + j * kCols, sign + o, kCols, bar);
    }
    bulk_load(st + S::kVec, vec + c0, kCols * 4, bar);
    if (W2) {
      bulk_load(st + S::kBw, theta + ob2 + c0, kCols * 4, bar);
      bulk_load(st + S::kBst, step + ob2 + c0, kCols * 4, bar);
      bulk_load(st + S::kBsg, sign + ob2 + c0, kCols, bar);
    }
  };
  auto issue_stores = [&](long long chunk, int s) {
    uint8_t* st = smem + s * S::kBytes;
    const long long c0 = chunk * kCols;
    for (int j = 0; j < H; ++j) {
      const long long o = rowoff + (long long)j * n + c0;
      bulk_store(theta + o, st + S::kW + j * kCols * 4, kCols * 4);
      bulk_store(step + o, st + S::kSt + j * kCols * 4, kCols * 4);
      bulk_store(sign + o, st + S::kSg + j * kCols, kCols);
    }
    if (W2) {
      bulk_store(theta + ob2 + c0, st + S::kBw, kCols * 4);
      bulk_store(step + ob2 + c0, st + S::kBst, kCols * 4);
      bulk_store(sign + ob2 + c0, st + S::kBsg, kCols);
    }
    bulk_commit();
  };

  float acc[W2 ? H : H + 1];
#pragma unroll
  for (int j = 0; j < (W2 ? H : H + 1); ++j) acc[j] = 0.f;

  long long chunk = blockIdx.x;
  if (tid == 0 && chunk < nchunks) issue_loads(chunk, 0);
  int k = 0;
  for (; chunk < nchunks; chunk += gridDim.x, ++k) {
    const int s = k & 1;
    const long long next = chunk + gridDim.x;
    if (tid == 0 && next < nchunks) {
      bulk_wait_read_all();  // stage s^1 held chunk k - 1, whose stores must have left shared memory
      issue_loads(next, s ^ 1);
    }
    if (!bar_wait(s_u32(&bars[s]), (uint32_t)((k >> 1) & 1))) {
      if (tid == 0) atomicOr(flags, 4u);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    uint8_t* st = smem + s * S::kBytes;
    float* w = reinterpret_cast<float*>(st + S::kW);
    float* sp = reinterpret_cast<float*>(st + S::kSt);
    int8_t* sg = reinterpret_cast<int8_t*>(st + S::kSg);
    const float v = reinterpret_cast<const float*>(st + S::kVec)[tid];  // dt_i or f_i
    if (W2) {
      float* bw = reinterpret_cast<float*>(st + S::kBw);
      float* bst = reinterpret_cast<float*>(st + S::kBst);
      int8_t* bsg = reinterpret_cast<int8_t*>(st + S::kBsg);
      float bs = bst[tid];
      int8_t bg = bsg[tid];
      bw[tid] = rprop1(bw[tid], v, bs, bg, rc);
      bst[tid] = bs;
      bsg[tid] = bg;
    } else {
      acc[H] += v;
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int e = j * kCols + tid;
      float wj = w[e];
      float sj = sp[e];
      int8_t gj = sg[e];
      if (W2) {
        acc[j] += wj * v;  // dh_j with the old weights
        wj = rprop1(wj, hs[j] * v, sj, gj, rc);
      } else {
        wj = rprop1(wj, hs[j] * v, sj, gj, rc);
        acc[j] += wj * v;  // next pre-activation with the new weights
      }
      w[e] = wj;
      sp[e] = sj;
      sg[e] = gj;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) issue_stores(chunk, s);
  }
  if (tid == 0) bulk_wait_all();
  if (s_fail) {
    // drain: the other stage may still have loads in flight
    if (tid == 0) bar_wait(s_u32(&bars[(k + 1) & 1]), (uint32_t)(((k + 1) >> 1) & 1));
    return;
  }

  if (W2) {
    float a2[H];
#pragma unroll
    for (int j = 0; j < H; ++j) a2[j] = acc[j];
    block_sum_to<H>(a2, partials + (size_t)blockIdx.x * kPartialStride);
  } else {
    float a1[H + 1];
#pragma unroll
    for (int j = 0; j <= H; ++j) a1[j] = acc[j];
    block_sum_to<H + 1>(a1, partials + (size_t)blockIdx.x * kPartialStride);
  }
  if (last_block_arrived(counter)) {
    if (W2) {
      final_sum(partials, H, [&](int j, double sum) {
        const float p = pre[j];
        const float dp = (float)sum * (p > 0.f ? 1.f : slope);
        dpre_io[j] = dp;
        float stp = step[ob1 + j];
        int8_t sgn = sign[ob1 + j];
        theta[ob1 + j] = rprop1(theta[ob1 + j], dp, stp, sgn, rc);
        step[ob1 + j] = stp;
        sign[ob1 + j] = sgn;
      });
    } else {
      final_sum(partials, H + 1, [&](int j, double sum) {
        if (j < H) {
          const float p = (float)(sum + (double)theta[ob1 + j]);
          pre_out[j] = p;
          hid_out[j] = leaky_b(p, slope);
        } else {
          scal[1] = sum;
        }
      });
    }
    __syncthreads();
    if (tid == 0) *counter = 0u;
  }
}

// Layer-1 forward with exactly the partition of the bulk W1 pass (chunk c of the 4^N axis to block
// c mod grid, column t of a chunk to thread t), so that the hidden layer it gives is bit-identical to
// the one the W1 pass leaves for the next iteration (checkpoint resume depends on this).
template <int H>
__global__ void __launch_bounds__(kCols, 2) k_l1_forward_cols(const float* __restrict__ theta,
                                                              const float* __restrict__ f, long long n, float* pre,
                                                              float* hid, double* scal, double* partials,
                                                              unsigned int* counter, float slope) {
  const long long ob1 = 2LL * H * n + n;
  const long long nchunks = n / kCols;
  float acc[H + 1];
#pragma unroll
  for (int j = 0; j <= H; ++j) acc[j] = 0.f;
  for (long long chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const long long c = chunk * kCols + threadIdx.x;
    const float v = f[c];
    acc[H] += v;
#pragma unroll
    for (int j = 0; j < H; ++j) acc[j] += theta[(long long)j * n + c] * v;
  }
  block_sum_to<H + 1>(acc, partials + (size_t)blockIdx.x * kPartialStride);
  if (last_block_arrived(counter)) {
    final_sum(partials, H + 1, [&](int j, double sum) {
      if (j < H) {
        const float p = (float)(sum + (double)theta[ob1 + j]);
        pre[j] = p;
        hid[j] = leaky_b(p, slope);
      } else {
        scal[1] = sum;
      }
    });
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
  }
}

long long bulk_grid(long long n) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = 2LL * sms;
  const long long nchunks = n / kCols;
  if (grid > nchunks) grid = nchunks;
  if (grid > kPartialBlocks) grid = kPartialBlocks;
  return grid;
}

template <int H, bool W2> cudaError_t launch_bulk(float* theta, float* step, int8_t* sign, const float* vec,
                                                   const float* hid, const float* pre, float* dpre, float* pre_out,
                                                   float* hid_out, double* scal, long long n, double* partials,
                                                   unsigned int* counter, unsigned int* flags,
                                                   const RpropCfg<float>& rc, float slope, cudaStream_t s) {
  using S = Stage<H, W2>;
  const int smem = 2 * S::kBytes;
  static bool set = false;
  if (!set) {
    cudaError_t e = cudaFuncSetAttribute(k_wpass_bulk<H, W2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    set = true;
  }
  const long long grid = bulk_grid(n);
  k_wpass_bulk<H, W2><<<(unsigned)grid, kCols, smem, s>>>(theta, step, sign, vec, hid, pre, dpre, pre_out, hid_out,
                                                          scal, n, partials, counter, flags, rc, slope);
  return cudaGetLastError();
}

}  // namespace

bool wpass_bulk_ok(int H, long long n) { return H >= 8 && H <= 24 && n % kCols == 0 && n >= kCols; }

#define QST_BULK_SWITCH(H, ...)                                 \
  switch (H) {                                                  \
    case 8: { constexpr int HH = 8; __VA_ARGS__; } break;       \
    case 10: { constexpr int HH = 10; __VA_ARGS__; } break;     \
    case 12: { constexpr int HH = 12; __VA_ARGS__; } break;     \
    case 14: { constexpr int HH = 14; __VA_ARGS__; } break;     \
    case 16: { constexpr int HH = 16; __VA_ARGS__; } break;     \
    case 18: { constexpr int HH = 18; __VA_ARGS__; } break;     \
    case 20: { constexpr int HH = 20; __VA_ARGS__; } break;     \
    case 22: { constexpr int HH = 22; __VA_ARGS__; } break;     \
    case 24: { constexpr int HH = 24; __VA_ARGS__; } break;     \
    default: return cudaErrorInvalidValue;                      \
  }

cudaError_t w2_pass_bulk(const Dims& D, float* theta, float* step, int8_t* sign, const float* dt, const float* hid,
                         const float* pre, float* dpre, double* partials, unsigned int* counter, unsigned int* flags,
                         const NetCfg& c, cudaStream_t s) {
  RpropCfg<float> rc{(float)c.eta_minus, (float)c.eta_plus, (float)c.step_min, (float)c.step_max};
  QST_BULK_SWITCH(D.H, return (launch_bulk<HH, true>(theta, step, sign, dt, hid, pre, dpre, nullptr, nullptr, nullptr,
                                                     D.n, partials, counter, flags, rc, (float)c.slope, s)));
  return cudaSuccess;
}

cudaError_t l1_forward_bulk(const Dims& D, const float* theta, const float* f, float* pre, float* hid, double* scal,
                            double* partials, unsigned int* counter, const NetCfg& c, cudaStream_t s) {
  const long long grid = bulk_grid(D.n);
  QST_BULK_SWITCH(D.H, k_l1_forward_cols<HH><<<(unsigned)grid, kCols, 0, s>>>(theta, f, D.n, pre, hid, scal, partials,
                                                                              counter, (float)c.slope));
  return cudaGetLastError();
}

cudaError_t w1_pass_bulk(const Dims& D, float* theta, float* step, int8_t* sign, const float* f, float* dpre,
                         float* pre, float* hid, double* scal, double* partials, unsigned int* counter,
                         unsigned int* flags, const NetCfg& c, cudaStream_t s) {
  RpropCfg<float> rc{(float)c.eta_minus, (float)c.eta_plus, (float)c.step_min, (float)c.step_max};
  QST_BULK_SWITCH(D.H, return (launch_bulk<HH, false>(theta, step, sign, f, nullptr, nullptr, dpre, pre, hid, scal,
                                                      D.n, partials, counter, flags, rc, (float)c.slope, s)));
  return cudaSuccess;
}

}  // namespace qst
