// qst_probs_static: the POVM map of qst_probs without any device allocation.
//
// Some callers cannot call cudaMalloc: a host framework that hands the whole
// device memory to its own pool allocator (an extra allocation can fail or
// fragment that pool), or a latency-bounded loop that must not take the implicit
// device synchronisation cudaMalloc and cudaFree can cause, or code that wants a
// single one-off evaluation without creating a qst_ctx (qst_init allocates).
// For them this entry point runs the same two kernels as qst_probs, with the
// packed intermediate in a fixed, file-scope device array instead of context
// memory.  It allocates nothing and calls no allocating library routine.
#include <mutex>

#include "../../include/qst.h"
#include "impl.h"

namespace {

// Largest supported problem: N = 10 qubits, whose packed intermediate holds
// 4^10 floats (4 MiB).  Every GPU that loads the library keeps this array
// until the process exits.
constexpr int kStaticMaxQubits = 10;
constexpr long long kStaticScratchFloats = 1LL << (2 * kStaticMaxQubits);

static __device__ __align__(256) float g_probs_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_probs_scratch on the current device, looked up once per
// device (host code only sees a stand-in symbol, never the device address).
cudaError_t scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_probs_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" qst_status qst_probs_static(int N, const double* povm, int K, const void* rho, void* p, void* stream) {
  if (N < 1 || N > kStaticMaxQubits) return QST_E_INVAL;
  if (rho == nullptr || p == nullptr) return QST_E_INVAL;
  // the kernels read rho and write p directly: host memory is refused before anything is launched
  if (!qst::is_device_ptr(rho) || !qst::is_device_ptr(p)) return QST_E_INVAL;
  qst::PovmB<double> Bd;
  const qst_status st = (qst_status)qst::check_povm(povm, K, &Bd);
  if (st != QST_OK) return st;
  const qst::PovmPlan plan = qst::make_povm_plan(Bd);  // FP32 coefficients rounded as qst_init rounds them
  float* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return QST_E_CUDA;
  const qst::Dims D = qst::make_dims(N, false);
  if (D.n > kStaticScratchFloats) return QST_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // Pass 1 writes every packed entry that pass 2 reads, so the array needs no clearing.
  if (qst::povm_fast_ok(D)) {
    if (qst::povm_fwd_fast(D, (const float2*)rho, scratch, (float*)p, plan, s) != cudaSuccess) return QST_E_CUDA;
    return QST_OK;
  }
  if (qst::povm_lo_fwd<float>(D, (const float2*)rho, scratch, plan.B, s) != cudaSuccess) return QST_E_CUDA;
  if (qst::povm_hi_fwd<float>(D, scratch, (float*)p, plan.B, s) != cudaSuccess) return QST_E_CUDA;
  return QST_OK;
}
