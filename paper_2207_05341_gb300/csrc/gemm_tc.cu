// Tensor-core (tcgen05) complex products of the mixed-precision path:
//   X = T T   (Sec. 3.2 eq. unified_DP; lower 128 x 128 tiles only, X is Hermitian)
//   Y = G T   (backward of X = T T)
//
// A complex product is run as one real GEMM with the K axis doubled and the N
// axis doubled.  With T Hermitian (T_re symmetric, T_im antisymmetric) and the
// row-major planes P_re = T_re, P_im = T_im, P_nim = -T_im:
//   Re(A T)[m, n] = sum_k A_re[m,k] P_re[n,k] + A_im[m,k] P_im[n,k]
//   Im(A T)[m, n] = sum_k A_re[m,k] P_nim[n,k] + A_im[m,k] P_re[n,k]
// so both outputs are A' B'^T with A' = [A_re | A_im] (K = 2d) and, stacked along
// N, B1 = [P_re | P_im] and B2 = [P_nim | P_re]; every operand is K-major.  A = T
// for the forward, A = G for the backward.
//
// Precision: each FP32 operand x is split into a 16-bit hi + lo pair (lo = x - hi
// rounded again) and the product keeps hi*hi + hi*lo + lo*hi with FP32
// accumulation in TMEM.  Two operand formats:
//   FP16 (default): the operand is first scaled by a power of two s so that
//     max |s x| lies in [1, 2); hi + lo then carry ~22 bits and the result is
//     unscaled exactly in the epilogue (relative error ~2^-21).
//   BF16: no scaling; hi + lo carry ~16 bits (relative error ~2^-16).
//
// Kernel: one CTA (4 warps) per 128 x 128 complex output tile; two accumulators
// of 128 lanes x 256 FP32 columns (Re | Im) in TMEM, one for hi*hi and one for
// the small cross terms, so that the cross terms are not added into the large
// running sum (the tensor core's FP32 accumulation truncates; keeping the chains
// apart keeps that error on the large sum to the hi*hi steps alone).  Warp 0 lane 0 streams
// operands with TMA (64-byte swizzled rows of 32 K elements) into a 4-stage ring (48 KB per stage:
// A_hi, A_lo, B_hi = [B1_hi; B2_hi], B_lo; three stages stay in flight, which covers the L2 latency
// that a 2-stage ring of 96 KB stages left exposed), warp 1 lane 0 issues tcgen05.mma
// (M = 128, N = 256, K = 16) and commits each stage back to the producer; all
// four warps then read TMEM (tcgen05.ld 32x32b) and store the tile.  Every
// mbarrier wait is bounded: on timeout the kernel raises an error flag, drains
// what it issued (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "impl.h"

namespace qst {

namespace {

constexpr int kBM = 128;              // output rows per tile
constexpr int kBN = 128;              // complex output columns per tile (N = 256 reals)
constexpr int kBK = 32;               // K elements per stage (64 bytes of 16-bit operand per row)
constexpr int kStages = 4;            // 3 stages in flight while the MMA warp consumes the fourth
constexpr int kRowBytes = kBK * 2;    // one row of a box: the swizzle span (64 B)
static_assert(kRowBytes == 64 || kRowBytes == 128, "64- or 128-byte swizzled rows");
constexpr int kTileBytes = 128 * kBK * 2;        // one 128-row x 32-col 16-bit box: 8 KB
constexpr int kStageBytes = 6 * kTileBytes;      // 96 KB
constexpr int kTmemCols = 512;   // two 128 x 256 FP32 accumulators: hi*hi, and hi*lo + lo*hi
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr unsigned long long kWaitCycles = 4000000000ULL;  // ~2 s at 2 GHz

struct TcMaps {
  CUtensorMap a[4];  // A planes: re_hi, im_hi, re_lo, im_lo
  CUtensorMap b[6];  // T planes: re_hi, im_hi, nim_hi, re_lo, im_lo, nim_lo
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false after ~kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, swizzled rows of kRowBytes, 8-row atoms of 8 kRowBytes bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * kRowBytes) >> 4) << 32;      // stride byte offset: one 8-row atom
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)(kRowBytes == 128 ? 2 : 4) << 61;  // 128- or 64-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B FP16 (fmt 0) or BF16 (fmt 1), both
// K-major, M = 128, N = 256.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(2 * kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// tab: a batched launch (grid z = tomography); row z holds the tensor maps' device copy, C, sA, sB, err, clear
__global__ void __launch_bounds__(128, 1) k_tc_cgemm(const __grid_constant__ TcMaps maps, float2* __restrict__ C,
                                                      int d, int lower, uint32_t idesc, const double* sA,
                                                      const double* sB, unsigned int* err, unsigned int* clear,
                                                      int no_loads, const void* const* tab) {
  const TcMaps* mp = &maps;
  rebind(tab, mp, C, sA, sB, err, clear);
  grid_dep_wait();
  after_wait(mp, C, sA, sB, err, clear);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  const uint32_t full0 = smem_u32(bars);                  // full[s]  = bars[s]
  const uint32_t empty0 = smem_u32(bars + kStages);       // empty[s] = bars[kStages + s]
  const uint32_t done = smem_u32(bars + 2 * kStages);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
  __shared__ int s_fail;

  int I, J;
  if (lower) tri_decode(blockIdx.x, I, J);
  else { I = blockIdx.y; J = blockIdx.x; }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // the max slot behind this product's operand scale was read by the kernel that made the planes
  if (clear && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *clear = 0u;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int nkb = 2 * d / kBK;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    if (tab) {  // the maps are this tomography's copies in global memory
      for (int p = 0; p < 4; ++p) tensormap_acquire(&mp->a[p]);
      for (int p = 0; p < 6; ++p) tensormap_acquire(&mp->b[p]);
    }
    int issued = 0;
    // no_loads (qst_inject_wait_timeout): issue nothing, so that the MMA warp's bounded wait runs out
    for (int kb = 0; kb < (no_loads ? 0 : nkb); ++kb) {
      const int s = kb % kStages, it = kb / kStages;
      if (kb >= kStages && !mbar_wait(empty0 + 8 * s, (uint32_t)((it - 1) & 1))) {
        s_fail = 1;
        atomicOr(err, 1u);
        break;
      }
      const uint32_t fb = full0 + 8 * s;
      mbar_expect_tx(fb, kStageBytes);
      const int part = (kb * kBK) < d ? 0 : 1;
      const int col = kb * kBK - part * d;
      const CUtensorMap* a_hi = &mp->a[part == 0 ? 0 : 1];
      const CUtensorMap* a_lo = &mp->a[part == 0 ? 2 : 3];
      const CUtensorMap* b1_hi = &mp->b[part == 0 ? 0 : 1];
      const CUtensorMap* b1_lo = &mp->b[part == 0 ? 3 : 4];
      const CUtensorMap* b2_hi = &mp->b[part == 0 ? 2 : 0];
      const CUtensorMap* b2_lo = &mp->b[part == 0 ? 5 : 3];
      const uint32_t base = smem_u32(smem + s * kStageBytes);
      tma_load_2d(base + 0 * kTileBytes, a_hi, col, I * kBM, fb);
      tma_load_2d(base + 1 * kTileBytes, a_lo, col, I * kBM, fb);
      tma_load_2d(base + 2 * kTileBytes, b1_hi, col, J * kBN, fb);
      tma_load_2d(base + 3 * kTileBytes, b2_hi, col, J * kBN, fb);
      tma_load_2d(base + 4 * kTileBytes, b1_lo, col, J * kBN, fb);
      tma_load_2d(base + 5 * kTileBytes, b2_lo, col, J * kBN, fb);
      ++issued;
    }
    // drain: every stage issued must have landed before the CTA may exit
    for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb) {
      const int s = kb % kStages, it = kb / kStages;
      if (!mbar_wait(full0 + 8 * s, (uint32_t)(it & 1))) {
        s_fail = 1;
        atomicOr(err, 1u);
        break;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % kStages, it = kb / kStages;
      if (!mbar_wait(full0 + 8 * s, (uint32_t)(it & 1))) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint64_t ah = smem_desc(base + 0 * kTileBytes + kk * 32);
        const uint64_t al = smem_desc(base + 1 * kTileBytes + kk * 32);
        const uint64_t bh = smem_desc(base + 2 * kTileBytes + kk * 32);
        const uint64_t bl = smem_desc(base + 4 * kTileBytes + kk * 32);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        mma_f16(tmem, ah, bh, idesc, acc);
        mma_f16(tmem + 256, ah, bl, idesc, acc);
        mma_f16(tmem + 256, al, bh, idesc, 1u);
      }
      mma_commit(empty0 + 8 * s);
    }
    if (!ok) {
      s_fail = 1;
      atomicOr(err, 2u);
    }
    mma_commit(done);  // arrives once all MMAs issued so far have completed
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> registers -> global
  const bool ready = mbar_wait(done, 0u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready && !s_fail) {
    const float unscale = (float)(1.0 / (*sA * *sB));  // exact: both scales are powers of two
    const int row = I * kBM + warp * 32 + lane;
    float2* out = C + (long long)row * d + (long long)J * kBN;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < kBN; c += 16) {
      uint32_t re[16], im[16], re2[16], im2[16];
      tmem_ld16(lane_base + (uint32_t)c, re);
      tmem_ld16(lane_base + (uint32_t)(kBN + c), im);
      tmem_ld16(lane_base + 256u + (uint32_t)c, re2);
      tmem_ld16(lane_base + 256u + (uint32_t)(kBN + c), im2);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        const float r0 = __uint_as_float(re[u]) + __uint_as_float(re2[u]);
        const float i0 = __uint_as_float(im[u]) + __uint_as_float(im2[u]);
        const float r1 = __uint_as_float(re[u + 1]) + __uint_as_float(re2[u + 1]);
        const float i1 = __uint_as_float(im[u + 1]) + __uint_as_float(im2[u + 1]);
        float4 v = make_float4(unscale * r0, unscale * i0, unscale * r1, unscale * i1);
        *reinterpret_cast<float4*>(out + c + u) = v;
      }
    }
  }
  if (!ready || s_fail) {
    if (threadIdx.x == 0) atomicOr(err, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <class H> struct Pair16;
template <> struct Pair16<__half> { using T = __half2; };
template <> struct Pair16<__nv_bfloat16> { using T = __nv_bfloat162; };

template <class H> __device__ __forceinline__ H to16(float v);
template <> __device__ __forceinline__ __half to16<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from16(__half v) { return __half2float(v); }
__device__ __forceinline__ float from16(__nv_bfloat16 v) { return __bfloat162float(v); }

// Scale of the FP16 split: 2^-e for the largest |re|, |im| in [2^e, 2^(e+1)) (*amax, float bits, folded
// in by the kernel that wrote the matrix), i.e. the power of two that brings it into [1, 2); 1 without amax.
__device__ __forceinline__ double split_scale(const unsigned int* amax) {
  if (!amax) return 1.0;
  const double m = (double)__uint_as_float(*reinterpret_cast<const volatile unsigned int*>(amax));
  return (m > 0.0 && isfinite(m)) ? ldexp(1.0, -ilogb(m)) : 1.0;
}

// hi = 16-bit rounding of v, lo = 16-bit rounding of the remainder
template <class H> __device__ __forceinline__ void hi_lo(float v, H& hi, H& lo) {
  hi = to16<H>(v);
  lo = to16<H>(v - from16(hi));
}

// Complex FP32 matrix -> 16-bit hi / lo planes of s * x (G: re, im (hi), re, im (lo)); s = split_scale(amax),
// written to *s_slot.  Each thread converts 8 consecutive entries (four 16-byte loads, one 16-byte store
// per plane); nn is a multiple of 8.
template <class H>
__global__ void __launch_bounds__(256) k_split(const float2* __restrict__ A, H* __restrict__ P, long long nn,
                                                const unsigned int* amax, double* s_slot, const void* const* tab) {
  rebind(tab, A, P, amax, s_slot);
  grid_dep_wait();
  after_wait(A, P, amax, s_slot);
  const double sd = split_scale(amax);
  const float sc = (float)sd;
  if (blockIdx.x == 0 && threadIdx.x == 0) *s_slot = sd;
  union Pack {
    uint4 v;
    H h[8];
  };
  const long long n8 = nn / 8;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n8; q += (long long)gridDim.x * blockDim.x) {
    const float4* src = reinterpret_cast<const float4*>(A + 8 * q);
    Pack rh, ih, rl, il;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 a = src[u];
      hi_lo(sc * a.x, rh.h[2 * u], rl.h[2 * u]);
      hi_lo(sc * a.y, ih.h[2 * u], il.h[2 * u]);
      hi_lo(sc * a.z, rh.h[2 * u + 1], rl.h[2 * u + 1]);
      hi_lo(sc * a.w, ih.h[2 * u + 1], il.h[2 * u + 1]);
    }
    *reinterpret_cast<uint4*>(P + 8 * q) = rh.v;
    *reinterpret_cast<uint4*>(P + nn + 8 * q) = ih.v;
    *reinterpret_cast<uint4*>(P + 2 * nn + 8 * q) = rl.v;
    *reinterpret_cast<uint4*>(P + 3 * nn + 8 * q) = il.v;
  }
}

// The Hermitian T of t (R = t as d x d row-major; T_ii = R_ii, T_ij = R_ij + i R_ji for i > j,
// T_ji = conj T_ij), written straight into the 6 planes of s * T: re, im, -im (hi), then (lo);
// s = split_scale(amax) (max |t| folded in by the kernel that wrote t), written to *s_slot.  One CTA
// per 32 x 32 tile pair (I, J), I >= J (d >= 32): each thread loads one float4 of each tile, and
// writes 8 adjacent columns of one row of every plane with one 16-byte store (threads 0-127 the
// tile (I, J), 128-255 the tile (J, I)).
template <class H>
__global__ void __launch_bounds__(256) k_hermitian_planes(const float* __restrict__ t, int d, H* __restrict__ P,
                                                           const unsigned int* amax, double* s_slot,
                                                           const void* const* tab) {
  rebind(tab, t, P, amax, s_slot);
  __shared__ float Ra[32][33];
  __shared__ float Rb[32][33];
  const double sd = split_scale(amax);
  const float sc = (float)sd;
  if (blockIdx.x == 0 && threadIdx.x == 0) *s_slot = sd;
  const long long nn = (long long)d * d;
  int I, J;
  tri_decode(blockIdx.x, I, J);
  const int tid = threadIdx.x;
  {
    const int row = tid >> 3, col = (tid & 7) * 4;
    const float4 a = *reinterpret_cast<const float4*>(t + (long long)(I * 32 + row) * d + J * 32 + col);
    const float4 b = I != J ? *reinterpret_cast<const float4*>(t + (long long)(J * 32 + row) * d + I * 32 + col)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    Ra[row][col] = a.x; Ra[row][col + 1] = a.y; Ra[row][col + 2] = a.z; Ra[row][col + 3] = a.w;
    Rb[row][col] = b.x; Rb[row][col + 1] = b.y; Rb[row][col + 2] = b.z; Rb[row][col + 3] = b.w;
  }
  __syncthreads();
  const bool upper = tid >= 128;
  if (upper && I == J) return;
  const int r = (tid & 127) >> 2, c = (tid & 3) * 8;
  float re[8], im[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int cc = c + u;
    if (upper) { re[u] = Ra[cc][r]; im[u] = -Rb[r][cc]; }  // T[J 32 + r][I 32 + cc] = conj T[I 32 + cc][J 32 + r]
    else if (I != J) { re[u] = Ra[r][cc]; im[u] = Rb[cc][r]; }
    else if (r > cc) { re[u] = Ra[r][cc]; im[u] = Ra[cc][r]; }
    else if (r < cc) { re[u] = Ra[cc][r]; im[u] = -Ra[r][cc]; }
    else { re[u] = Ra[r][r]; im[u] = 0.f; }
  }
  union Pack {
    uint4 v;
    H h[8];
  };
  Pack pk[6];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    hi_lo(sc * re[u], pk[0].h[u], pk[3].h[u]);
    hi_lo(sc * im[u], pk[1].h[u], pk[4].h[u]);
    hi_lo(-(sc * im[u]), pk[2].h[u], pk[5].h[u]);
  }
  const long long idx = upper ? (long long)(J * 32 + r) * d + I * 32 + c : (long long)(I * 32 + r) * d + J * 32 + c;
#pragma unroll
  for (int p = 0; p < 6; ++p) *reinterpret_cast<uint4*>(P + p * nn + idx) = pk[p].v;
}

// The same planes from 64 x 64 tile pairs (d a multiple of 64): every plane row segment a thread group
// writes is 128 bytes, a whole L2 line (the 32 x 32 form writes half lines).  Threads 0-127 write tile
// (I, J), 128-255 tile (J, I); each thread 8 adjacent columns of 4 rows.
template <class H>
__global__ void __launch_bounds__(256) k_hermitian_planes64(const float* __restrict__ t, int d, H* __restrict__ P,
                                                             const unsigned int* amax, double* s_slot,
                                                             const void* const* tab) {
  rebind(tab, t, P, amax, s_slot);
  grid_dep_wait();
  after_wait(t, P, amax, s_slot);
  __shared__ float Ra[64][65];
  __shared__ float Rb[64][65];
  const double sd = split_scale(amax);
  const float sc = (float)sd;
  if (blockIdx.x == 0 && threadIdx.x == 0) *s_slot = sd;
  const long long nn = (long long)d * d;
  int I, J;
  tri_decode(blockIdx.x, I, J);
  const int tid = threadIdx.x;
  {
    float4 a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // 1024 float4 per tile: row q >> 4, columns 4 (q & 15) ..
      const int q = tid + 256 * k, row = q >> 4, col = (q & 15) * 4;
      a[k] = *reinterpret_cast<const float4*>(t + (long long)(I * 64 + row) * d + J * 64 + col);
      b[k] = I != J ? *reinterpret_cast<const float4*>(t + (long long)(J * 64 + row) * d + I * 64 + col)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = tid + 256 * k, row = q >> 4, col = (q & 15) * 4;
      Ra[row][col] = a[k].x; Ra[row][col + 1] = a[k].y; Ra[row][col + 2] = a[k].z; Ra[row][col + 3] = a[k].w;
      Rb[row][col] = b[k].x; Rb[row][col + 1] = b[k].y; Rb[row][col + 2] = b[k].z; Rb[row][col + 3] = b[k].w;
    }
  }
  __syncthreads();
  const bool upper = tid >= 128;
  if (upper && I == J) return;
  union Pack {
    uint4 v;
    H h[8];
  };
  const int c = (tid & 7) * 8;
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const int r = ((tid & 127) >> 3) + 16 * k;
    float re[8], im[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int cc = c + u;
      if (upper) { re[u] = Ra[cc][r]; im[u] = -Rb[r][cc]; }  // T[J 64 + r][I 64 + cc] = conj T[I 64 + cc][J 64 + r]
      else if (I != J) { re[u] = Ra[r][cc]; im[u] = Rb[cc][r]; }
      else if (r > cc) { re[u] = Ra[r][cc]; im[u] = Ra[cc][r]; }
      else if (r < cc) { re[u] = Ra[cc][r]; im[u] = -Ra[r][cc]; }
      else { re[u] = Ra[r][r]; im[u] = 0.f; }
    }
    Pack pk[6];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      hi_lo(sc * re[u], pk[0].h[u], pk[3].h[u]);
      hi_lo(sc * im[u], pk[1].h[u], pk[4].h[u]);
      hi_lo(-(sc * im[u]), pk[2].h[u], pk[5].h[u]);
    }
    const long long idx = upper ? (long long)(J * 64 + r) * d + I * 64 + c : (long long)(I * 64 + r) * d + J * 64 + c;
#pragma unroll
    for (int p = 0; p < 6; ++p) *reinterpret_cast<uint4*>(P + p * nn + idx) = pk[p].v;
  }
}

// Largest |re|, |im| of n complex entries folded into *amax (float bits; the slot is cleared before).
__global__ void __launch_bounds__(256) k_amax(const float2* __restrict__ M, long long n, unsigned int* amax) {
  float m = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = M[i];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  block_absmax_to(m, amax);
}

// 16-bit hi / lo planes of s * Z for a general product operand, Z = M (op 0) or M^dag (op 1), d x d
// row-major: 4 planes (re, im; hi then lo: the left operand A of C = A B) or 6 planes (re, im, -im; hi
// then lo: the right operand given as B^dag, which k_tc_cgemm reads row by row).  s = split_scale(amax),
// written to *s_slot.  One CTA per 32 x 32 tile of Z; the transpose goes through shared memory.
template <class H>
__global__ void __launch_bounds__(256) k_planes_op(const float2* __restrict__ M, int d, int op, int six,
                                                    H* __restrict__ P, const unsigned int* amax, double* s_slot) {
  __shared__ float2 tile[32][33];
  const double sd = split_scale(amax);
  const float sc = (float)sd;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *s_slot = sd;
  const long long nn = (long long)d * d;
  const int bi = blockIdx.y, bj = blockIdx.x;  // tile (bi, bj) of Z
  // Z tile (bi, bj) = M tile (bi, bj) (op 0) or the conjugate transpose of M tile (bj, bi) (op 1)
  const int si = op ? bj : bi, sj = op ? bi : bj;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    tile[r][c] = M[(long long)(si * 32 + r) * d + sj * 32 + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int r = e >> 5, c = e & 31;
    float2 z = op ? tile[c][r] : tile[r][c];
    if (op) z.y = -z.y;
    const long long o = (long long)(bi * 32 + r) * d + bj * 32 + c;
    H rh, rl, ih, il;
    hi_lo(sc * z.x, rh, rl);
    hi_lo(sc * z.y, ih, il);
    if (six) {
      H nh, nl;
      hi_lo(-(sc * z.y), nh, nl);
      P[o] = rh; P[nn + o] = ih; P[2 * nn + o] = nh; P[3 * nn + o] = rl; P[4 * nn + o] = il; P[5 * nn + o] = nl;
    } else {
      P[o] = rh; P[nn + o] = ih; P[2 * nn + o] = rl; P[3 * nn + o] = il;
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map over one d x d 16-bit plane, box kBK columns x 128 rows, rows swizzled over kRowBytes.
bool make_plane_map(CUtensorMap* m, const void* plane, int d, int fmt) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)d};
  cuuint64_t strides[1] = {(cuuint64_t)d * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, 128u};
  cuuint32_t estr[2] = {1u, 1u};
  return enc(m, fmt == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
             const_cast<void*>(plane), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, kRowBytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t build_maps(TcMaps* M, int d, const void* Ab, int a_planes_are_T, const void* Tb, int fmt) {
  const size_t nn = (size_t)d * d;
  const uint16_t* t = static_cast<const uint16_t*>(Tb);
  for (int p = 0; p < 6; ++p)
    if (!make_plane_map(&M->b[p], t + p * nn, d, fmt)) return cudaErrorInvalidValue;
  const uint16_t* a = static_cast<const uint16_t*>(Ab);
  // A planes in the order re_hi, im_hi, re_lo, im_lo
  const int tidx[4] = {0, 1, 3, 4};
  for (int p = 0; p < 4; ++p) {
    const uint16_t* src = a_planes_are_T ? t + tidx[p] * nn : a + p * nn;
    if (!make_plane_map(&M->a[p], src, d, fmt)) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_tc(const TcMaps& M, float2* C, int d, bool lower, int fmt, const double* sA, const double* sB,
                      unsigned int* err, unsigned int* clear, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int nt = d / kBM;
  BatchArgs ba;
  if (batch_take(ba, {C, sA, sB, err, clear}, &M, sizeof(TcMaps))) return cudaSuccess;
  const int no_loads = inject_take(INJ_TC_LOADS) ? 1 : 0;
  if (lower) {
    return launch_dep(k_tc_cgemm, dim3((unsigned)(nt * (nt + 1) / 2), 1, ba.nz), dim3(128), (size_t)kSmemBytes, s, M,
                      C, d, 1, make_idesc(fmt), sA, sB, err, clear, no_loads, ba.tab);
  }
  return launch_dep(k_tc_cgemm, dim3(nt, nt, ba.nz), dim3(128), (size_t)kSmemBytes, s, M, C, d, 0, make_idesc(fmt), sA,
                    sB, err, clear, no_loads, ba.tab);
}

}  // namespace

void* tma_encoder() { return reinterpret_cast<void*>(encode_fn()); }

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return false;
  return encode_fn() != nullptr;
}

cudaError_t tc_planes_T(int d, const float* t, void* Tb, int fmt, double* scal, const unsigned int* amax,
                        cudaStream_t s) {
  if (d < 32 || d % 32) return cudaErrorInvalidValue;
  const unsigned int* am = fmt == TC_BF16 ? nullptr : amax;
  BatchArgs ba;
  if (batch_take(ba, {t, Tb, am, scal + kScaleT})) return cudaSuccess;
  if (d % 64 == 0) {
    const int n64 = d / 64;
    const unsigned p64 = (unsigned)(n64 * (n64 + 1) / 2);
    if (fmt == TC_BF16)
      return launch_dep(k_hermitian_planes64<__nv_bfloat16>, dim3(p64, 1, ba.nz), dim3(256), 0, s, t, d,
                        (__nv_bfloat16*)Tb, am, scal + kScaleT, ba.tab);
    return launch_dep(k_hermitian_planes64<__half>, dim3(p64, 1, ba.nz), dim3(256), 0, s, t, d, (__half*)Tb, am,
                      scal + kScaleT, ba.tab);
  }
  const int nt = d / 32;
  const unsigned pairs = (unsigned)(nt * (nt + 1) / 2);
  if (fmt == TC_BF16)
    k_hermitian_planes<__nv_bfloat16><<<dim3(pairs, 1, ba.nz), 256, 0, s>>>(t, d, (__nv_bfloat16*)Tb, am,
                                                                            scal + kScaleT, ba.tab);
  else
    k_hermitian_planes<__half><<<dim3(pairs, 1, ba.nz), 256, 0, s>>>(t, d, (__half*)Tb, am, scal + kScaleT, ba.tab);
  return cudaGetLastError();
}

cudaError_t tc_split_G(int d, const float2* G, void* Gb, int fmt, double* scal, const unsigned int* amax,
                       cudaStream_t s) {
  const long long nn = (long long)d * d;
  if (nn % 8) return cudaErrorInvalidValue;
  long long blocks = (nn / 8 + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  const unsigned int* am = fmt == TC_BF16 ? nullptr : amax;
  BatchArgs ba;
  if (batch_take(ba, {G, Gb, am, scal + kScaleG})) return cudaSuccess;
  if (fmt == TC_BF16)
    return launch_dep(k_split<__nv_bfloat16>, dim3((unsigned)blocks, 1, ba.nz), dim3(256), 0, s, G,
                      (__nv_bfloat16*)Gb, nn, am, scal + kScaleG, ba.tab);
  return launch_dep(k_split<__half>, dim3((unsigned)blocks, 1, ba.nz), dim3(256), 0, s, G, (__half*)Gb, nn, am,
                    scal + kScaleG, ba.tab);
  return cudaGetLastError();
}

cudaError_t tc_herm_square(int d, const void* Tb, int fmt, const double* scal, float2* X, unsigned int* err,
                           unsigned int* clear, cudaStream_t s) {
  if (d < 128 || d % 128) return cudaErrorInvalidValue;
  TcMaps M;
  cudaError_t e = build_maps(&M, d, Tb, 1, Tb, fmt);
  if (e != cudaSuccess) return e;
  return launch_tc(M, X, d, true, fmt, scal + kScaleT, scal + kScaleT, err, clear, s);
}

cudaError_t absmax_to(long long n, const float2* M, unsigned int* amax, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  long long blocks = (n + 255) / 256;
  if (blocks > 1184) blocks = 1184;
  k_amax<<<(unsigned)blocks, 256, 0, s>>>(M, n, amax);
  return cudaGetLastError();
}

cudaError_t tc_planes_op(int d, const float2* M, int op, int nplanes, void* P, int fmt, const unsigned int* amax,
                         double* s_slot, cudaStream_t s) {
  if (d < 32 || d % 32 || (nplanes != 4 && nplanes != 6)) return cudaErrorInvalidValue;
  const dim3 grid(d / 32, d / 32);
  const int six = nplanes == 6 ? 1 : 0;
  if (fmt == TC_BF16)
    k_planes_op<__nv_bfloat16><<<grid, 256, 0, s>>>(M, d, op, six, (__nv_bfloat16*)P, nullptr, s_slot);
  else
    k_planes_op<__half><<<grid, 256, 0, s>>>(M, d, op, six, (__half*)P, amax, s_slot);
  return cudaGetLastError();
}

cudaError_t tc_product(int d, const void* Ab, const void* Bb, int fmt, const double* sA, const double* sB, float2* C,
                       bool lower, unsigned int* err, cudaStream_t s) {
  if (d < 128 || d % 128) return cudaErrorInvalidValue;
  TcMaps M;
  cudaError_t e = build_maps(&M, d, Ab, 0, Bb, fmt);
  if (e != cudaSuccess) return e;
  return launch_tc(M, C, d, lower, fmt, sA, sB, err, nullptr, s);
}

cudaError_t tc_gt_product(int d, const void* Gb, const void* Tb, int fmt, const double* scal, float2* Y,
                          unsigned int* err, unsigned int* clear, cudaStream_t s) {
  if (d < 128 || d % 128) return cudaErrorInvalidValue;
  TcMaps M;
  cudaError_t e = build_maps(&M, d, Gb, 0, Tb, fmt);
  if (e != cudaSuccess) return e;
  return launch_tc(M, Y, d, false, fmt, scal + kScaleG, scal + kScaleT, err, clear, s);
}

}  // namespace qst
