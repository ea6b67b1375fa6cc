// Rprop weight passes of the Sec. 3.1 network (FP32, in-place update) with bulk-copy staging.
//
// Each CTA walks chunks of kCols consecutive columns of the 4^N axis (chunk c to CTA
// c mod grid, one CTA per SM).  The CTA is warp-specialised: one producer thread issues,
// per chunk, one 2-D tensor copy (cp.async.bulk.tensor, box kCols x H) of each parameter
// array (weights, Rprop state words: H rows n apart) and 1-D bulk copies of the
// chunk of dt (W2 pass) or f (W1 pass) and of b2's state, all counted on the stage's
// "full" mbarrier, into a ring of kStages shared-memory stages.  The consumer threads
// (kGroups per column, each with about H / kGroups of the rows, enough warps to hide the
// latency of the update) update the chunk in shared memory and arrive on the stage's
// "empty" mbarrier; the producer then writes the boxes back with tensor stores and
// refills the stage once the stores have read it.  A handful of copies per chunk keeps
// the copy engine's per-instruction cost off the critical path, and nobody waits for a
// store to drain.  The shape (256 columns, 2 row groups, 3 stages, one CTA per SM) is
// the fastest of a sweep over chunk width, row groups, ring depth and CTAs per SM.
//
// The arithmetic is that of k_w2_pass / k_w1_pass in fnn.cu (same Rprop; the sums
// over the 4^N axis are per-thread partials reduced in a fixed order, so the pass is
// deterministic, though the partition of those sums differs from fnn.cu's kernel).
// Every mbarrier wait is bounded; a timeout raises flags bit 4 and the kernel drains
// the loads it issued (bounded) before returning.
#include <cuda.h>

#include "impl.h"

namespace qst {

namespace {

constexpr int kCols = 256;                  // columns per chunk
constexpr int kConsumerWarps = kCols / 32;  // warps over the columns of one row group
constexpr int kGroups = 2;                  // row groups: consumer threads per column
constexpr int kConsumers = kCols * kGroups;
constexpr int kThreads = kConsumers + 32;   // + one producer warp
constexpr int kMaxStages = 3;
constexpr int kCtasPerSm = 1;
constexpr int kRingBytes = 220 * 1024;      // shared memory of one CTA's ring (228 KB per SM)
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
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int x, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          s_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(0), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store_box(const CUtensorMap* map, int x, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(0), "r"(s_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all_but_1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor maps of the H x n parameter rows of one pass (W1, or W2^T) in theta and in the Rprop state.
struct WMaps {
  CUtensorMap w, st;
};

// Stage layout (bytes, every part 128-byte aligned): w[H][kCols] f32 | st[H][kCols] f32 (Rprop state)
//                       | vec[kCols] f32 (dt or f) | W2 pass only: b2 w, st [kCols] f32
template <int H, bool W2> struct Stage {
  static constexpr int kW = 0;
  static constexpr int kSt = kW + H * kCols * 4;
  static constexpr int kVec = kSt + H * kCols * 4;
  static constexpr int kBw = kVec + kCols * 4;
  static constexpr int kBst = kBw + kCols * 4;
  static constexpr int kUsed = W2 ? kBst + kCols * 4 : kBw;  // bytes the copies of one chunk bring in
  static constexpr int kBytes = (kUsed + 127) / 128 * 128;  // stage pitch: every stage 128-byte aligned
  static constexpr uint32_t kTx = (uint32_t)kUsed;
  static_assert(kSt % 128 == 0 && kVec % 128 == 0 && kBw % 16 == 0 && kBst % 16 == 0 && kCols % 16 == 0 &&
                    kCols <= 256,
                "tensor-copy destinations must be 128-byte aligned, bulk-copy ones 16-byte aligned");
  // ring depth: as many stages as fit in kRingBytes, at most kMaxStages (a deeper ring measured slower)
  static constexpr int kStages = kRingBytes / kBytes < kMaxStages ? kRingBytes / kBytes : kMaxStages;
  static_assert(kStages >= 3, "the ring needs three stages");
};

template <class R> __device__ __forceinline__ R leaky_b(R x, R slope) { return x > R(0) ? x : slope * x; }

// Sum v over the kConsumerWarps warps of consumer threads (fixed order) into out[0..M); every
// thread of the block calls it (the producer warp contributes nothing).
template <int M>
__device__ __forceinline__ void block_sum_to(const float (&v)[M], double* out) {
  __shared__ double red[kConsumerWarps][M];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < kConsumerWarps) {
#pragma unroll
    for (int j = 0; j < M; ++j) {
      double x = warp_sum((double)v[j]);
      if (lane == 0) red[w][j] = x;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kConsumerWarps; ++q) s += red[q][j];
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
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_wpass_bulk(const __grid_constant__ WMaps maps,
                                                          float* __restrict__ theta, float* __restrict__ step,
                                                          const float* __restrict__ vec,
                                                          const float* __restrict__ hidv, const float* __restrict__ pre,
                                                          float* dpre_io, float* pre_out, float* hid_out, double* scal,
                                                          long long n, long long ob2, long long ob1,
                                                          double* partials, unsigned int* counter,
                                                          unsigned int* flags, RpropCfg<float> rc, float slope,
                                                          int no_loads, const void* const* tab) {
  using S = Stage<H, W2>;
  const WMaps* mp = &maps;
  rebind(tab, mp, theta, step, vec, hidv, pre, dpre_io, pre_out, hid_out, scal, partials, counter, flags);
  grid_dep_wait();
  after_wait(mp, theta, step, vec, hidv, pre, dpre_io, pre_out, hid_out, scal, partials, counter, flags);
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((128u - (s_u32(smem_raw) & 127u)) & 127u);  // 128-byte aligned ring
  constexpr int kStages = S::kStages;
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ float hs[H];
  __shared__ int s_fail;
  // ob2: offset of b2 in theta and step, < 0 when this launch leaves b2 alone (W2 pass);
  // ob1: offset of b1, < 0 when the W2 pass only writes dpre (the caller updates b1)
  const bool with_b2 = W2 && ob2 >= 0;
  const uint32_t tx = with_b2 ? S::kTx : (uint32_t)S::kBw;  // bytes one chunk's copies bring in
  const long long nchunks = n / kCols;
  const long long nk = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;  // chunks of this CTA
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < H) hs[tid] = W2 ? hidv[tid] : dpre_io[tid];  // W2: h; W1: dpre
  if (tid == 0) {
    s_fail = 0;
    for (int q = 0; q < kStages; ++q) {
      bar_init(s_u32(&full[q]), 1);
      bar_init(s_u32(&empty[q]), kConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  constexpr int RPT = (H + kGroups - 1) / kGroups;  // rows per consumer thread
  const int col = tid % kCols, rg = tid / kCols;      // column of a chunk, row group
  float acc[RPT], accf = 0.f, hr[RPT];
#pragma unroll
  for (int l = 0; l < RPT; ++l) {
    acc[l] = 0.f;
    hr[l] = rg * RPT + l < H ? hs[rg * RPT + l] : 0.f;  // W2: h_j; W1: dpre_j
  }
  if (warp == kConsumers / 32) {
    // ---------------- producer
    if (lane == 0) {
      if (tab) {  // the maps are this tomography's copies in global memory
        tensormap_acquire(&mp->w);
        tensormap_acquire(&mp->st);
      }
      auto issue_loads = [&](long long k) {
        const int q = (int)(k % kStages);
        uint8_t* st = smem + q * S::kBytes;
        const long long c0 = (blockIdx.x + k * gridDim.x) * kCols;
        const uint32_t bar = s_u32(&full[q]);
        bar_expect(bar, tx);
        tma_load_box(st + S::kW, &mp->w, (int)c0, bar);
        tma_load_box(st + S::kSt, &mp->st, (int)c0, bar);
        bulk_load(st + S::kVec, vec + c0, kCols * 4, bar);
        if (with_b2) {
          bulk_load(st + S::kBw, theta + ob2 + c0, kCols * 4, bar);
          bulk_load(st + S::kBst, step + ob2 + c0, kCols * 4, bar);
        }
      };
      auto issue_stores = [&](long long k) {
        const int q = (int)(k % kStages);
        uint8_t* st = smem + q * S::kBytes;
        const long long c0 = (blockIdx.x + k * gridDim.x) * kCols;
        tma_store_box(&mp->w, (int)c0, st + S::kW);
        tma_store_box(&mp->st, (int)c0, st + S::kSt);
        if (with_b2) {
          bulk_store(theta + ob2 + c0, st + S::kBw, kCols * 4);
          bulk_store(step + ob2 + c0, st + S::kBst, kCols * 4);
        }
        bulk_commit();
      };
      long long loaded = 0;  // chunks [0, loaded) have been issued
      // no_loads (qst_inject_wait_timeout): issue nothing, so that every bounded wait of the pass runs out
      const long long nload = no_loads ? 0 : nk;
      for (; loaded < nload && loaded < kStages; ++loaded) issue_loads(loaded);
      for (long long k = 0; k < nk; ++k) {
        if (!bar_wait(s_u32(&empty[k % kStages]), (uint32_t)((k / kStages) & 1))) {
          atomicOr(flags, 4u);
          s_fail = 1;
          break;
        }
        issue_stores(k);
        // refill the stage of chunk k - 1, whose stores were committed one chunk ago
        if (k >= 1 && loaded < nload) {
          bulk_wait_read_all_but_1();
          issue_loads(loaded++);
        }
      }
      bulk_wait_all();
      if (s_fail) {  // drain: wait (bounded) for the last load issued into every stage
        for (int q = 0; q < kStages; ++q) {
          long long last = -1;
          for (long long k = loaded - 1; k >= 0 && k >= loaded - kStages; --k)
            if (k % kStages == q) last = k;
          if (last >= 0) bar_wait(s_u32(&full[q]), (uint32_t)((last / kStages) & 1));
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------- consumers: column col, rows rg * RPT + l, of every chunk
    for (long long k = 0; k < nk; ++k) {
      const int q = (int)(k % kStages);
      if (!bar_wait(s_u32(&full[q]), (uint32_t)((k / kStages) & 1))) {
        if (tid == 0) atomicOr(flags, 4u);
        s_fail = 1;
        break;
      }
      uint8_t* st = smem + q * S::kBytes;
      float* w = reinterpret_cast<float*>(st + S::kW);
      float* sp = reinterpret_cast<float*>(st + S::kSt);
      const float v = reinterpret_cast<const float*>(st + S::kVec)[col];  // dt_i or f_i
      if (rg == 0) {
        if (with_b2) {
          float* bw = reinterpret_cast<float*>(st + S::kBw);
          float* bst = reinterpret_cast<float*>(st + S::kBst);
          float bs = bst[col];
          bw[col] = rprop1(bw[col], v, bs, rc);
          bst[col] = bs;
        } else if (!W2) {
          accf += v;
        }
      }
#pragma unroll
      for (int l = 0; l < RPT; ++l) {
        const int j = rg * RPT + l;
        if (RPT * kGroups != H && j >= H) continue;
        const int e = j * kCols + col;
        float wj = w[e];
        float sj = sp[e];
        if (W2) {
          acc[l] += wj * v;  // dh_j with the old weights
          wj = rprop1(wj, hr[l] * v, sj, rc);
        } else {
          wj = rprop1(wj, hr[l] * v, sj, rc);
          acc[l] += wj * v;  // next pre-activation with the new weights
        }
        w[e] = wj;
        sp[e] = sj;
      }
      fence_async_smem();  // the producer's tensor stores read what this thread wrote
      bar_arrive(s_u32(&empty[q]));
    }
  }
  __syncthreads();
  if (s_fail) return;

  // per row j: the thread partials of its group's kCols columns, summed per warp (FP64) and over the
  // group's kConsumerWarps warps in order (the partition of k_l1_forward_cols)
  {
    __shared__ double red[kGroups * kConsumerWarps][RPT + 1];
    if (warp < kConsumers / 32) {
#pragma unroll
      for (int l = 0; l < RPT; ++l) {
        const double x = warp_sum((double)acc[l]);
        if (lane == 0) red[warp][l] = x;
      }
      if (!W2 && rg == 0) {
        const double x = warp_sum((double)accf);
        if (lane == 0) red[warp][RPT] = x;
      }
    }
    __syncthreads();
    double* out = partials + (size_t)blockIdx.x * kPartialStride;
    for (int j = tid; j < (W2 ? H : H + 1); j += blockDim.x) {
      const int g = j < H ? j / RPT : 0, l = j < H ? j % RPT : RPT;
      double sum = 0.0;
      for (int q = 0; q < kConsumerWarps; ++q) sum += red[g * kConsumerWarps + q][l];
      out[j] = sum;
    }
  }
  if (last_block_arrived(counter)) {
    if (W2) {
      final_sum(partials, H, [&](int j, double sum) {
        const float p = pre[j];
        const float dp = (float)sum * (p > 0.f ? 1.f : slope);
        dpre_io[j] = dp;
        if (ob1 >= 0) {
          float stp = step[ob1 + j];
          theta[ob1 + j] = rprop1(theta[ob1 + j], dp, stp, rc);
          step[ob1 + j] = stp;
        }
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
  long long grid = (long long)kCtasPerSm * sms;
  const long long nchunks = n / kCols;
  // at least bulk_chunks_per_cta chunks per CTA: a CTA's ring fill and store drain are then a small
  // share of its time, and a batch of small tomographies keeps few CTAs per tomography
  const long long per = tuning().bulk_chunks_per_cta;
  const long long want = nchunks / per < 1 ? 1 : nchunks / per;
  if (grid > want) grid = want;
  if (grid > kPartialBlocks) grid = kPartialBlocks;
  return grid;
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// H x n FP32 rows starting at base (row stride n elements), box kCols x H, no swizzle.
bool make_rows_map(CUtensorMap* m, void* base, long long n, int H) {
  EncodeFn enc = reinterpret_cast<EncodeFn>(tma_encoder());
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)H};
  cuuint64_t strides[1] = {(cuuint64_t)n * 4};
  cuuint32_t box[2] = {(cuuint32_t)kCols, (cuuint32_t)H};
  cuuint32_t estr[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// rowoff: first element of the H x n rows this launch streams (in theta and step); ob2, ob1 as in
// k_wpass_bulk.
template <int H, bool W2> cudaError_t launch_bulk(float* theta, float* step, const float* vec,
                                                   const float* hid, const float* pre, float* dpre, float* pre_out,
                                                   float* hid_out, double* scal, long long n, long long rowoff,
                                                   long long ob2, long long ob1, double* partials,
                                                   unsigned int* counter, unsigned int* flags,
                                                   const RpropCfg<float>& rc, float slope, cudaStream_t s) {
  using S = Stage<H, W2>;
  const int smem = S::kStages * S::kBytes + 128;
  static bool set = false;
  if (!set) {
    cudaError_t e = cudaFuncSetAttribute(k_wpass_bulk<H, W2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    set = true;
  }
  WMaps maps;
  if (!make_rows_map(&maps.w, theta + rowoff, n, H) || !make_rows_map(&maps.st, step + rowoff, n, H))
    return cudaErrorInvalidValue;
  const long long grid = bulk_grid(n);
  BatchArgs ba;
  if (batch_take(ba, {theta, step, vec, hid, pre, dpre, pre_out, hid_out, scal, partials, counter, flags}, &maps,
                 sizeof(WMaps)))
    return cudaSuccess;
  const int no_loads = inject_take(INJ_WPASS_LOADS) ? 1 : 0;
  return launch_dep(k_wpass_bulk<H, W2>, dim3((unsigned)grid, 1, ba.nz), dim3(kThreads), (size_t)smem, s, maps, theta,
                    step, vec, hid, pre, dpre, pre_out, hid_out, scal, n, ob2, ob1, partials, counter, flags, rc,
                    slope, no_loads, ba.tab);
}

}  // namespace

bool wpass_bulk_ok(int H, long long n) {
  return H >= 8 && H <= 24 && n % kCols == 0 && n >= kCols && tma_encoder() != nullptr;
}

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

cudaError_t w2_pass_bulk(const Dims& D, float* theta, float* step, const float* dt, const float* hid,
                         const float* pre, float* dpre, double* partials, unsigned int* counter, unsigned int* flags,
                         const NetCfg& c, cudaStream_t s) {
  RpropCfg<float> rc{(float)c.eta_minus, (float)c.eta_plus, (float)c.step_min, (float)c.step_max};
  const long long n = D.n, H = D.H;  // theta = [W1 | W2^T | b2 | b1]
  QST_BULK_SWITCH(D.H, return (launch_bulk<HH, true>(theta, step, dt, hid, pre, dpre, nullptr, nullptr, nullptr,
                                                     n, H * n, 2 * H * n, 2 * H * n + n, partials, counter, flags, rc,
                                                     (float)c.slope, s)));
  return cudaSuccess;
}

cudaError_t w2_rows_pass_bulk(long long n, int rows, float* theta, float* step, long long rowoff, long long ob2,
                              const float* dt, const float* hid, const float* pre, float* dpre, double* partials,
                              unsigned int* counter, unsigned int* flags, const NetCfg& c, cudaStream_t s) {
  RpropCfg<float> rc{(float)c.eta_minus, (float)c.eta_plus, (float)c.step_min, (float)c.step_max};
  QST_BULK_SWITCH(rows, return (launch_bulk<HH, true>(theta, step, dt, hid, pre, dpre, nullptr, nullptr, nullptr, n,
                                                      rowoff, ob2, -1, partials, counter, flags, rc, (float)c.slope,
                                                      s)));
  return cudaSuccess;
}

cudaError_t l1_forward_bulk(const Dims& D, const float* theta, const float* f, float* pre, float* hid, double* scal,
                            double* partials, unsigned int* counter, const NetCfg& c, cudaStream_t s) {
  const long long grid = bulk_grid(D.n);
  QST_BULK_SWITCH(D.H, k_l1_forward_cols<HH><<<(unsigned)grid, kCols, 0, s>>>(theta, f, D.n, pre, hid, scal, partials,
                                                                              counter, (float)c.slope));
  return cudaGetLastError();
}

cudaError_t w1_pass_bulk(const Dims& D, float* theta, float* step, const float* f, float* dpre,
                         float* pre, float* hid, double* scal, double* partials, unsigned int* counter,
                         unsigned int* flags, const NetCfg& c, cudaStream_t s) {
  RpropCfg<float> rc{(float)c.eta_minus, (float)c.eta_plus, (float)c.step_min, (float)c.step_max};
  const long long n = D.n, H = D.H;
  QST_BULK_SWITCH(D.H, return (launch_bulk<HH, false>(theta, step, f, nullptr, nullptr, dpre, pre, hid, scal, n, 0,
                                                      -1, 2 * H * n + n, partials, counter, flags, rc,
                                                      (float)c.slope, s)));
  return cudaSuccess;
}

}  // namespace qst
