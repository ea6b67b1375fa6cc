// C ABI of libqst (include/qst.h): context management and the per-iteration
// sequence of the NN-QST hot path (Fig. 1 loop of arXiv:2207.05341).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <algorithm>
#include <atomic>
#include <vector>

#include "../../include/qst.h"
#include "impl.h"
#include "tuned.h"

using namespace qst;

namespace qst {

int ptr_kind(const void* p) {
  if (p == nullptr) return 0;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 2;
  return a.type == cudaMemoryTypeHost ? 1 : 0;
}
bool is_device_ptr(const void* p) { return ptr_kind(p) == 2; }

int check_povm(const double* povm, int K, PovmB<double>* Bd) {
  if (povm == nullptr || K != 4) return QST_E_INVAL;
  double sum[8] = {0};
  for (int a = 0; a < 4; ++a) {
    const double* m = povm + 8 * a;  // m00 (re, im), m01, m10, m11
    for (int q = 0; q < 8; ++q) {
      if (!isfinite(m[q])) return QST_E_INVAL;
      sum[q] += m[q];
    }
    // Hermitian: real diagonal, m01 = conj(m10)
    if (fabs(m[1]) > 1e-12 || fabs(m[7]) > 1e-12) return QST_E_INVAL;
    if (fabs(m[2] - m[4]) > 1e-12 || fabs(m[3] + m[5]) > 1e-12) return QST_E_INVAL;
    // Pauli coefficients: M = b0 I + b1 X + b2 Y + b3 Z, m10 = b1 + i b2
    Bd->b[a][0] = 0.5 * (m[0] + m[6]);
    Bd->b[a][1] = m[4];
    Bd->b[a][2] = m[5];
    Bd->b[a][3] = 0.5 * (m[0] - m[6]);
  }
  const double eye[8] = {1, 0, 0, 0, 0, 0, 1, 0};
  for (int q = 0; q < 8; ++q)
    if (fabs(sum[q] - eye[q]) > 1e-12) return QST_E_INVAL;
  return QST_OK;
}

static std::atomic<int> g_bulk_chunks{kTunedBulkChunksPerCta};
static std::atomic<int> g_fused_ctas{kTunedFusedCtasPerSm};
static std::atomic<int> g_fused_max{kTunedFusedMaxQubits};
static std::atomic<int> g_concurrent{kTunedBatchConcurrentRuns};

Tuning tuning() {
  return Tuning{g_bulk_chunks.load(), g_fused_ctas.load(), g_fused_max.load(), g_concurrent.load()};
}

static std::atomic<int> g_inject[INJ_SITES];

bool inject_take(int site) {
  int v = g_inject[site].load();
  while (v > 0)
    if (g_inject[site].compare_exchange_weak(v, v - 1)) return true;
  return false;
}

BatchRec*& batch_rec() {
  static thread_local BatchRec* rec = nullptr;
  return rec;
}

bool batch_take(BatchArgs& ba, std::initializer_list<const void*> ptrs, const void* blob, size_t blob_bytes) {
  BatchRec* r = batch_rec();
  ba = BatchArgs{};
  if (r == nullptr) return false;
  const int k = r->call++;
  const int nptr = (int)ptrs.size() + (blob ? 1 : 0);
  if (r->mode == BatchRec::LAUNCH) {
    if (k >= (int)r->calls.size() || r->calls[k].nptr != nptr || r->calls[k].blob_bytes != blob_bytes) {
      r->bad = true;  // not the sequence that was recorded: launch nothing
      return true;
    }
    ba.tab = r->calls[k].dtab;
    ba.nz = (unsigned)r->count;
    return false;
  }
  if (r->member == 0 && k == (int)r->calls.size()) {
    r->calls.emplace_back();
    r->calls[k].nptr = nptr;
    r->calls[k].blob_bytes = blob_bytes;
  }
  if (k >= (int)r->calls.size() || r->calls[k].nptr != nptr || r->calls[k].blob_bytes != blob_bytes) {
    r->bad = true;
    return true;
  }
  BatchRec::Call& c = r->calls[k];
  c.ptrs.insert(c.ptrs.end(), ptrs.begin(), ptrs.end());
  if (blob) {
    const unsigned char* b = static_cast<const unsigned char*>(blob);
    c.blobs.insert(c.blobs.end(), b, b + blob_bytes);
  }
  return true;
}

}  // namespace qst

namespace {

// tensor-core eigenvector refinement of QST_MIXED A_P steps: acceptance threshold on max |E|
constexpr float kOaAccept = 5e-3f;
constexpr int kOaMaxIters = 6;
constexpr float kOaLeft = 1e-5f;  // largest unresolved coupling, relative to max |lambda|
constexpr int kOaBackoff = 15;    // after a step handed to the sweeps, the next attempt comes 16 steps later

constexpr unsigned long long kStateMagic = 0x5153545354415432ULL;  // "QSTSTAT2": theta, Rprop state words

}  // namespace

struct qst_ctx {
  int N = 0;
  int prec = QST_FP32;
  qst_options opt;
  Dims D;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<void*> allocs;
  size_t dev_bytes = 0;  // device memory held in allocs
  void* work = nullptr;  // Work<float> or Work<double>
  PovmB<float> Bf;
  PovmB<double> Bd;
  PovmPlan plan;  // FP32 fast POVM kernels (povm_fast.cu): structure of the POVM
  const void* fperm_of = nullptr;  // the f whose permuted copy is in Work::fperm (values fixed while the pointer is)
  bool fperm_stale = false;        // set by calls whose f may hold new values under the same pointer
  NetCfg net;
  bool params_set = false;
  bool hidden_valid = false;
  const void* f_last = nullptr;
  long long iters = 0;
  long long launches = 0;
  double* h_scal = nullptr;     // pinned host mirror of scal (16 doubles)
  unsigned int* h_flags = nullptr;
  size_t partial_doubles = 0;
  // per-phase timing (qst_timing_enable)
  std::vector<cudaEvent_t> tev;   // max_steps * (QST_NPHASE + 1) events
  std::vector<unsigned int> tmask;
  int tmax = 0, tcount = 0, tslot = -1;
  void* apw = nullptr;  // AbsPWork<R> (QST_MAP_ABS_P)
  double* cdf = nullptr;  // scratch of the sampled classical fidelity, allocated on first use
  double* fq = nullptr;   // scratch of the state fidelity, allocated on first use
  size_t P = 0;           // parameters: qst_theta_size_net(N, network)
  bool cnn = false;       // the App. A CNN head instead of the 3-layer FNN
  unsigned long long* samp = nullptr;  // scratch of qst_sample_counts, allocated on first use
  long long oa_refinements = 0;  // tensor-core refinements taken (QST_MIXED A_P), Jacobi fallbacks
  long long oa_fallbacks = 0;
  double oa_last[2] = {0.0, 0.0};  // max |E| and the unresolved coupling of the latest refinement
  int oa_skip = 0;                 // warm steps left that go to the sweeps without a refinement attempt
  int sweeps = 12;       // cold-start Jacobi sweeps
  int warm_sweeps = 2;   // warm-start sweeps (0: never warm-start)
  bool warm_valid = false;
  bool bulk_passes = true;  // FP32 weight passes with bulk-copy staging (fnn_bulk.cu)
  // CUDA graph of one steady-state qst_step (qst_graph_enable)
  bool graph_on = false;
  bool graph_timed = false;  // the captured graph records the phase events into slot 0
  cudaGraphExec_t gexec = nullptr;
  const void* gf = nullptr;
  long long gnodes = 0;  // kernel launches in one replay of gexec
  bool capturing = false;
  // a captured step with a page-locked host f copies f on a side stream, beside its first kernels
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_f = nullptr;
  bool f_wait = false;  // the stream must join ev_f before its first read of f
};

namespace {

qst_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return QST_OK;
  if (e == cudaErrorMemoryAllocation) return QST_E_NOMEM;
  return QST_E_CUDA;
}

#define QST_CU(expr)                               \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

// Before the first read of f: join the copy of a host f issued on the side stream (a captured step's
// copy runs beside the kernels that come before this point).
cudaError_t join_f(qst_ctx* c) {
  if (!c->f_wait) return cudaSuccess;
  c->f_wait = false;
  return cudaStreamWaitEvent(c->stream, c->ev_f, 0);
}

// Under stream capture an event record becomes a graph node only with cudaEventRecordExternal.
void record_mark(qst_ctx* c, cudaEvent_t e) {
  if (c->capturing)
    cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(e, c->stream);
}
// Timing marks: slot `tslot` holds a start event and one event per phase.
void tmark_begin(qst_ctx* c) {
  c->tslot = -1;
  if (c->tmax <= 0 || c->tcount >= c->tmax) return;
  c->tslot = c->tcount++;
  c->tmask[c->tslot] = 0u;
  record_mark(c, c->tev[(size_t)c->tslot * (QST_NPHASE + 1)]);
}
void tmark(qst_ctx* c, int phase) {
  if (c->tslot < 0) return;
  record_mark(c, c->tev[(size_t)c->tslot * (QST_NPHASE + 1) + 1 + phase]);
  c->tmask[c->tslot] |= 1u << phase;
}

template <class T> cudaError_t dalloc(qst_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = count * sizeof(T) < 256 ? 256 : count * sizeof(T);
  // the context's device-memory budget (qst_options.device_memory_limit): refused before cudaMalloc
  if (c->opt.device_memory_limit && c->dev_bytes + bytes > c->opt.device_memory_limit)
    return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return e;
  c->dev_bytes += bytes;
  c->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return cudaSuccess;
}

template <class R> Work<R>* W(qst_ctx* c) { return reinterpret_cast<Work<R>*>(c->work); }
template <class R> const PovmB<R>& povmB(qst_ctx* c);
template <> const PovmB<float>& povmB<float>(qst_ctx* c) { return c->Bf; }
template <> const PovmB<double>& povmB<double>(qst_ctx* c) { return c->Bd; }

size_t theta_size(int N) {
  const size_t n = (size_t)1 << (2 * N), H = 2 * (size_t)N;
  return 2 * H * n + n + H;
}

size_t rsize(const qst_ctx* c) { return c->prec == QST_FP64 ? sizeof(double) : sizeof(float); }
bool is_mixed(const qst_ctx* c) { return c->prec == QST_MIXED || c->prec == QST_MIXED_BF16; }
int tc_fmt(const qst_ctx* c) { return c->prec == QST_MIXED_BF16 ? TC_BF16 : TC_FP16_SCALED; }

template <class R> qst_status alloc_work(qst_ctx* c) {
  Work<R>* w = new (std::nothrow) Work<R>();
  if (!w) return QST_E_NOMEM;
  memset(w, 0, sizeof(*w));
  c->work = w;
  const Dims& D = c->D;
  const size_t P = c->P;
  const size_t nn = (size_t)D.d * D.d;
  QST_CU(dalloc(c, &w->theta, P));
  QST_CU(dalloc(c, &w->step, P));
  QST_CU(dalloc(c, &w->pre, 64));
  QST_CU(dalloc(c, &w->hid, 64));
  QST_CU(dalloc(c, &w->dpre, 64));
  if (c->cnn) {
    QST_CU(dalloc(c, &w->feats, 640));
    QST_CU(dalloc(c, &w->vals, 640));
    QST_CU(dalloc(c, &w->pos, 640));
    QST_CU(dalloc(c, &w->cnn_part, cnn_part_doubles(D.N, sizeof(R))));
  }
  QST_CU(dalloc(c, &w->T, nn));
  QST_CU(dalloc(c, &w->X, nn));
  QST_CU(dalloc(c, &w->G, nn));
  QST_CU(dalloc(c, &w->Y, nn));
  QST_CU(dalloc(c, &w->Wlo, (size_t)D.n));
  QST_CU(dalloc(c, &w->Whi, (size_t)D.n));
  QST_CU(dalloc(c, &w->dt, (size_t)D.n));
  QST_CU(dalloc(c, &w->fstage, (size_t)D.n));
  if (std::is_same<R, float>::value && povm_fast_ok(D) && povm_needs_fperm(c->plan))
    QST_CU(dalloc(c, &w->fperm, (size_t)D.n));
  QST_CU(dalloc(c, &w->scal, 16));
  // per-block partial sums: the largest reducing grid is the tile-pair grid of build_T
  const int TS = D.d < 32 ? D.d : 32;
  const size_t pairs = (size_t)(D.d / TS) * (D.d / TS + 1) / 2;
  size_t blocks = (size_t)kPartialBlocks;
  if (pairs > blocks) blocks = pairs;
  const size_t p2 = ((size_t)1 << (2 * D.g)) / D.C;
  if (p2 > blocks) blocks = p2;
  c->partial_doubles = blocks * kPartialStride;
  QST_CU(dalloc(c, &w->partials, c->partial_doubles));
  QST_CU(dalloc(c, &w->counters, (size_t)CNT_COUNT));
  QST_CU(dalloc(c, &w->flags, 8));
  QST_CU(cudaMemsetAsync(w->counters, 0, CNT_COUNT * sizeof(unsigned int), c->stream));
  QST_CU(cudaMemsetAsync(w->flags, 0, 8 * sizeof(unsigned int), c->stream));
  QST_CU(cudaMemsetAsync(w->scal, 0, 16 * sizeof(double), c->stream));
  if (c->opt.mapping == QST_MAP_ABS_P) {
    AbsPWork<R>* ap = new (std::nothrow) AbsPWork<R>();
    if (!ap) return QST_E_NOMEM;
    memset(ap, 0, sizeof(*ap));
    c->apw = ap;
    QST_CU(dalloc(c, &ap->A0, nn));
    QST_CU(dalloc(c, &ap->A1, nn));
    QST_CU(dalloc(c, &ap->V0, nn));
    QST_CU(dalloc(c, &ap->V1, nn));
    QST_CU(dalloc(c, &ap->W, nn));
    QST_CU(dalloc(c, &ap->Qh, nn));
    QST_CU(dalloc(c, &ap->lam, (size_t)D.d));
    QST_CU(dalloc(c, &ap->s, (size_t)D.d));
    QST_CU(dalloc(c, &ap->sp, (size_t)D.d));
    QST_CU(dalloc(c, &ap->ucos, 16 * (size_t)D.d));
    if (is_mixed(c)) {  // operand planes of the tensor-core refinement
      const size_t pb = abs_p_tc_plane_bytes(D.d);
      unsigned char* buf = nullptr;
      QST_CU(dalloc(c, &buf, 3 * pb + 3 * (pb + pb / 2)));
      ap->qa_n = buf;
      ap->qa_h = buf + pb;
      ap->wa = buf + 2 * pb;
      ap->qb_n = buf + 3 * pb;
      ap->qb_h = buf + 3 * pb + (pb + pb / 2);
      ap->eb = buf + 3 * pb + 2 * (pb + pb / 2);
      QST_CU(dalloc(c, &ap->amax, 8));
      QST_CU(dalloc(c, &ap->sc, 8));
      QST_CU(dalloc(c, &ap->perm, (size_t)D.d));
      float2* ublk = nullptr;
      QST_CU(dalloc(c, &ublk, (size_t)D.d * 64));
      ap->ublk = ublk;
    }
    c->sweeps = c->opt.eig_sweeps > 0 ? c->opt.eig_sweeps : 12;
    c->sweeps += c->sweeps & 1;
    c->warm_sweeps = c->opt.eig_warm_sweeps < 0 ? 0 : (c->opt.eig_warm_sweeps > 0 ? c->opt.eig_warm_sweeps : 2);
    c->warm_sweeps += c->warm_sweeps & 1;
  }
  if (is_mixed(c)) {
    unsigned short* tb = nullptr;
    QST_CU(dalloc(c, &tb, 6 * nn));
    w->Tb = tb;
    unsigned short* gb = nullptr;
    QST_CU(dalloc(c, &gb, 4 * nn));
    w->Gb = gb;
  }
  return QST_OK;
}

template <class R> void free_work(qst_ctx* c) {
  delete W<R>(c);
  delete reinterpret_cast<AbsPWork<R>*>(c->apw);
}

// ---- stream helpers
const void* stage_input(qst_ctx* c, const void* f, size_t bytes, void* stage, qst_status* st) {
  *st = QST_OK;
  if (is_device_ptr(f)) return f;
  cudaError_t e = cudaMemcpyAsync(stage, f, bytes, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) { *st = cuda_status(e); return nullptr; }
  return stage;
}

// Validate f (finite, >= 0, sum 1 within 1e-4) on the host: copies n reals back.
template <class R> qst_status validate_f(qst_ctx* c, const void* fdev) {
  const size_t n = (size_t)c->D.n;
  std::vector<R> h(n);
  QST_CU(cudaMemcpyAsync(h.data(), fdev, n * sizeof(R), cudaMemcpyDeviceToHost, c->stream));
  QST_CU(cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) {
    const double v = (double)h[i];
    if (!(v >= 0.0) || !isfinite(v)) return QST_E_INPUT;
    s += v;
  }
  if (fabs(s - 1.0) > 1e-4) return QST_E_INPUT;
  return QST_OK;
}

// The producer-side max slot of the scaled FP16 split (NULL on the other paths).
unsigned int* amax_slot(qst_ctx* c, int slot) {
  if (!is_mixed(c) || tc_fmt(c) != TC_FP16_SCALED) return nullptr;
  return (c->prec == QST_FP64 ? W<double>(c)->counters : W<float>(c)->counters) + slot;
}

// ---- the hot path ------------------------------------------------------------
template <class R> struct Engine {
  using V = cx_t<R>;

  // X = T T (lower tiles) from the hidden activation already in w->hid; Tr X -> scal[0]
  static qst_status forward_state(qst_ctx* c, const R* theta, bool own_params = true) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    const bool mixed = is_mixed(c);
    // t = W2 h + b2 in the dt buffer (free until the backward writes dL/dt), then T (or its 16-bit planes)
    // Chol_Delta: T lower triangular and T^dag (in Y, free until the backward) for X = T^dag T
    const bool delta = c->opt.mapping == QST_MAP_CHOL_DELTA;
    if (c->cnn) {
      QST_CU(cnn_output<R>(D, theta, w->hid, w->dt, amax_slot(c, CNT_AMAXT), c->stream));
      if (!mixed) QST_CU(net_hermitian_T<R>(D, w->dt, w->T, delta ? w->Y : nullptr, c->stream));
    } else {
      const bool absp = c->opt.mapping == QST_MAP_ABS_P;  // the cold start's Jacobi sweeps read T itself
      QST_CU(net_build_T<R>(D, theta, w->hid, w->dt, mixed && !absp ? nullptr : w->T, amax_slot(c, CNT_AMAXT),
                            c->stream, delta ? w->Y : nullptr));
    }
    if (mixed) {
      QST_CU(tc_planes_T(D.d, reinterpret_cast<const float*>(w->dt), w->Tb, tc_fmt(c), w->scal,
                         amax_slot(c, CNT_AMAXT), c->stream));
    }
    c->launches += 2;
    tmark(c, QST_PH_BUILD_T);
    if (c->opt.mapping == QST_MAP_ABS_P) {
      // the context's own parameters change slowly: start from the last eigenvectors
      const bool warm = own_params && c->warm_valid && c->warm_sweeps > 0;
      const int sw = warm ? c->warm_sweeps : c->sweeps;
      bool done = false;
      if constexpr (std::is_same<R, float>::value) {
        if (mixed && warm && c->oa_skip > 0) {
          --c->oa_skip;  // T moved too far at the latest attempt: the sweeps, without trying first
        } else if (mixed && warm && c->opt.eig_refine) {
          // Refinements of the previous eigenvectors on tensor cores, each judged by its largest correction
          // max |E| and the largest coupling it left unresolved (near-degenerate pairs): a refinement with
          // unresolved couplings is followed by the block passes over neighbours in the order of lambda,
          // any other is applied, and the eigenvectors are taken once max |E| is at most kOaAccept (the
          // error left is of its square) with nothing unresolved.  kOaMaxIters refinements without that
          // (or a correction above 1) hand the step to Jacobi sweeps from the eigenvectors it started with.
          // Inside a graph capture there is no host check: two refinements, taken.
          AbsPWork<float>& ap = *reinterpret_cast<AbsPWork<float>*>(c->apw);
          const size_t qbytes = (size_t)D.d * D.d * sizeof(float2);
          QST_CU(cudaMemcpyAsync(ap.Qh, ap.V0, qbytes, cudaMemcpyDeviceToDevice, c->stream));  // the start
          for (int it = 0; it < kOaMaxIters && !done; ++it) {
            QST_CU(abs_p_tc_correction(D.d, w->Tb, w->scal + kScaleT, ap, c->opt.P, tc_fmt(c), w->flags + 1,
                                       c->stream));
            c->launches += 12;
            float emax = 0.f, left = 0.f;
            if (!c->capturing) {
              QST_CU(cudaMemcpyAsync(c->h_flags + 4, ap.amax + 2, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                     c->stream));
              QST_CU(cudaStreamSynchronize(c->stream));
              memcpy(&emax, c->h_flags + 4, sizeof(float));
              memcpy(&left, c->h_flags + 5, sizeof(float));
              c->oa_last[0] = emax;
              c->oa_last[1] = left;
            }
            if (emax != emax || left != left || emax > 1.f) break;
            if (!(left <= kOaLeft)) {
              // couplings of near-degenerate pairs: exact Jacobi diagonalisations of blocks of neighbours in
              // the order of lambda, then another correction
              if (c->capturing || it + 1 >= kOaMaxIters) break;
              QST_CU(abs_p_tc_block_phase(D.d, w->Tb, w->scal + kScaleT, ap, tc_fmt(c), w->flags + 1, c->stream));
              c->launches += 14;
              continue;
            }
            QST_CU(abs_p_tc_update(D.d, ap, tc_fmt(c), w->flags + 1, c->stream));
            c->launches += 4;
            if (emax <= kOaAccept || (c->capturing && it == 1)) {
              QST_CU(abs_p_tc_finish(D.d, ap, tc_fmt(c), reinterpret_cast<float2*>(w->X), w->flags + 1,
                                     c->stream));
              c->launches += 7;
              c->oa_refinements += it + 1;
              done = true;
            }
          }
          if (!done) {  // back to the start, with its Q^dag for the sweeps' warm start
            QST_CU(cudaMemcpyAsync(ap.V0, ap.Qh, qbytes, cudaMemcpyDeviceToDevice, c->stream));
            QST_CU(abs_p_restore_q<float>(D.d, ap, c->stream));
            c->oa_fallbacks += 1;
            c->oa_skip = kOaBackoff;
          }
        }
      }
      if (!done) {
        bool on_tc = false;
        if constexpr (std::is_same<R, float>::value) {
          if (mixed && warm) {  // the products around the sweeps (Q^dag T Q, X) on tensor cores
            QST_CU(abs_p_forward_tc_warm(D.d, w->Tb, w->scal + kScaleT, *reinterpret_cast<AbsPWork<float>*>(c->apw),
                                         sw, c->opt.P, tc_fmt(c), reinterpret_cast<float2*>(w->X), w->flags + 1,
                                         c->stream));
            c->launches += 17 + (long long)sw * jacobi_kernels_per_sweep(D.d);
            on_tc = true;
          }
        }
        if (!on_tc) {
          QST_CU(abs_p_forward<R>(D.d, w->T, *reinterpret_cast<AbsPWork<R>*>(c->apw), sw, warm, c->opt.P, w->X,
                                  c->stream));
          c->launches += 4 + (long long)sw * jacobi_kernels_per_sweep(D.d);
        }
      }
      if (mixed && amax_slot(c, CNT_AMAXT))  // the planes of T are made: restart the max of the next t
        QST_CU(cudaMemsetAsync(amax_slot(c, CNT_AMAXT), 0, sizeof(unsigned int), c->stream));
      c->warm_valid = own_params;
    } else if (mixed) {
      QST_CU(tc_herm_square(D.d, w->Tb, tc_fmt(c), w->scal, reinterpret_cast<float2*>(w->X), w->flags + 1,
                            amax_slot(c, CNT_AMAXT), c->stream));
    } else {
      QST_CU(cgemm_simt<R>(D.d, delta ? w->Y : w->T, w->T, w->X, true, c->stream));
    }
    QST_CU(trace_X<R>(D, w->X, w->scal, c->stream));
    c->launches += 2;
    tmark(c, QST_PH_XFWD);
    return QST_OK;
  }

  // FP32 contexts with N in [7, 11] run the register-blocked POVM kernels of povm_fast.cu
  static bool fast_povm(const qst_ctx* c) { return std::is_same<R, float>::value && povm_fast_ok(c->D); }

  // loss -> scal[2]; with backward, G = sum_k g_k M_k -> w->G
  static qst_status povm_likelihood(qst_ctx* c, const R* f, bool backward) {
    QST_CU(join_f(c));  // the first read of f in a step (the CNN's comes earlier, in its hidden layer)
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    if constexpr (std::is_same<R, float>::value) {
      if (fast_povm(c)) {
        const float* fl = f;
        if (povm_needs_fperm(c->plan)) {  // f in the likelihood pass's order, made again only for a new f
          if (f != c->fperm_of || f == w->fstage || c->fperm_stale) {
            QST_CU(povm_permute_f(D, f, w->fperm, c->plan, c->stream));
            c->launches += 1;
            c->fperm_of = f;
            c->fperm_stale = false;
          }
          fl = w->fperm;
        }
        QST_CU(povm_lo_fwd_fast(D, w->X, w->Wlo, c->plan, c->stream));
        tmark(c, QST_PH_POVM_LO);
        QST_CU(povm_hi_nll_fast(D, w->Wlo, fl, w->scal, w->Whi, w->partials, w->counters + CNT_NLL, w->flags,
                                c->plan, backward, c->stream));
        tmark(c, QST_PH_POVM_HI);
        c->launches += 2;
        if (backward) {
          QST_CU(povm_lo_adj_fast(D, w->Whi, w->G, c->plan, amax_slot(c, CNT_AMAXG), c->stream));
          c->launches += 1;
          tmark(c, QST_PH_POVM_ADJ);
        }
        return QST_OK;
      }
    }
    const PovmB<R>& B = povmB<R>(c);
    QST_CU(povm_lo_fwd<R>(D, w->X, w->Wlo, B, c->stream));
    tmark(c, QST_PH_POVM_LO);
    QST_CU(povm_hi_nll<R>(D, w->Wlo, f, w->scal, w->Whi, w->partials, w->counters + CNT_NLL, w->flags, B,
                          backward, c->stream));
    tmark(c, QST_PH_POVM_HI);
    c->launches += 2;
    if (backward) {
      QST_CU(povm_lo_adj<R>(D, w->Whi, w->G, B, amax_slot(c, CNT_AMAXG), c->stream));
      c->launches += 1;
      tmark(c, QST_PH_POVM_ADJ);
    }
    return QST_OK;
  }

  // dL/dt from G and T -> w->dt
  static qst_status backward_state(qst_ctx* c) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    if (is_mixed(c) && c->opt.mapping == QST_MAP_ABS_P) {
      if constexpr (std::is_same<R, float>::value) {
        QST_CU(abs_p_backward_tc(D.d, reinterpret_cast<const float2*>(w->G),
                                 *reinterpret_cast<AbsPWork<float>*>(c->apw), tc_fmt(c),
                                 reinterpret_cast<float2*>(w->Y), w->flags + 1, c->stream));
      }
      c->launches += 13;
      tmark(c, QST_PH_GT);
      QST_CU(net_symmetrize<R>(D, w->Y, w->dt, c->stream));
      tmark(c, QST_PH_SYM);
      c->launches += 1;
    } else if (is_mixed(c)) {
      QST_CU(tc_split_G(D.d, reinterpret_cast<const float2*>(w->G), w->Gb, tc_fmt(c), w->scal,
                        amax_slot(c, CNT_AMAXG), c->stream));
      QST_CU(tc_gt_product(D.d, w->Gb, w->Tb, tc_fmt(c), w->scal, reinterpret_cast<float2*>(w->Y), w->flags + 1,
                           amax_slot(c, CNT_AMAXG), c->stream));
      tmark(c, QST_PH_GT);
      QST_CU(net_symmetrize<R>(D, w->Y, w->dt, c->stream));
      tmark(c, QST_PH_SYM);
      c->launches += 3;
    } else if (c->opt.mapping == QST_MAP_ABS_P) {
      QST_CU(abs_p_backward<R>(D.d, w->G, *reinterpret_cast<AbsPWork<R>*>(c->apw), w->Y, c->stream));
      c->launches += 4;
      tmark(c, QST_PH_GT);
      QST_CU(net_symmetrize<R>(D, w->Y, w->dt, c->stream));
      tmark(c, QST_PH_SYM);
      c->launches += 2;
    } else if (c->opt.mapping == QST_MAP_CHOL_DELTA) {
      // dL = 2 Re Tr[G T^dag dT] for lower-triangular dT: only the lower tiles of Z = T G are needed
      QST_CU(cgemm_simt<R>(D.d, w->T, w->G, w->Y, true, c->stream));
      tmark(c, QST_PH_GT);
      QST_CU(net_tri_grad<R>(D, w->Y, w->dt, c->stream));
      tmark(c, QST_PH_SYM);
      c->launches += 2;
    } else {
      QST_CU(cgemm_simt<R>(D.d, w->G, w->T, w->Y, false, c->stream));
      tmark(c, QST_PH_GT);
      QST_CU(net_symmetrize<R>(D, w->Y, w->dt, c->stream));
      tmark(c, QST_PH_SYM);
      c->launches += 2;
    }
    return QST_OK;
  }

  // The bulk weight passes apply to FP32 contexts with H >= 8 and a 16-byte aligned f.
  static bool use_bulk(qst_ctx* c, const R* f) {
    if constexpr (std::is_same<R, float>::value)
      return !c->cnn && c->bulk_passes && wpass_bulk_ok(c->D.H, c->D.n) && ((uintptr_t)f & 15u) == 0;
    return false;
  }

  static qst_status hidden(qst_ctx* c, const R* theta, const R* f) {
    Work<R>* w = W<R>(c);
    if (c->cnn) {  // convolution, pooling and the first dense layer of the CNN head (App. A)
      QST_CU(cnn_hidden<R>(c->D, theta, f, w->feats, w->pos, w->vals, w->pre, w->hid, c->net.slope, w->cnn_part,
                           w->partials, w->counters + CNT_L1, w->scal, c->stream));
      c->launches += 2;
      tmark(c, QST_PH_HIDDEN);
      return QST_OK;
    }
    bool done = false;
    if constexpr (std::is_same<R, float>::value) {
      if (use_bulk(c, f)) {
        QST_CU(l1_forward_bulk(c->D, theta, f, w->pre, w->hid, w->scal, w->partials, w->counters + CNT_L1, c->net,
                               c->stream));
        done = true;
      }
    }
    if (!done)
      QST_CU(net_l1_forward<R>(c->D, theta, f, w->pre, w->hid, w->scal, w->partials, w->counters + CNT_L1, c->net,
                               c->stream));
    c->launches += 1;
    tmark(c, QST_PH_HIDDEN);
    return QST_OK;
  }

  static qst_status read_loss(qst_ctx* c, double* loss) {
    Work<R>* w = W<R>(c);
    QST_CU(cudaMemcpyAsync(c->h_scal, w->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    QST_CU(cudaMemcpyAsync(c->h_flags, w->flags, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream));
    QST_CU(cudaStreamSynchronize(c->stream));
    *loss = c->h_scal[2];
    if (c->h_flags[1] != 0u) {
      // a kernel that gave up returned before its last-block reduction: restart every counter
      QST_CU(cudaMemsetAsync(w->flags, 0, 2 * sizeof(unsigned int), c->stream));
      QST_CU(cudaMemsetAsync(w->counters, 0, CNT_COUNT * sizeof(unsigned int), c->stream));
      QST_CU(cudaStreamSynchronize(c->stream));
      return QST_E_TIMEOUT;
    }
    if (c->h_flags[0] != 0u) {
      QST_CU(cudaMemsetAsync(w->flags, 0, sizeof(unsigned int), c->stream));
      return QST_W_CLAMP;
    }
    return QST_OK;
  }

  // Small FP32 tomographies of the 3-layer network with Chol_H run a whole iteration in one CTA
  static bool fused(const qst_ctx* c) {
    return std::is_same<R, float>::value && !c->cnn && c->opt.mapping == QST_MAP_CHOL_H && !is_mixed(c) &&
           tomo_fused_ok(c->N, c->opt.fused_max_qubits);
  }
  static TomoDesc tomo_desc(qst_ctx* c, const R* f) {
    TomoDesc td{};
    if constexpr (std::is_same<R, float>::value) {
      Work<R>* w = W<R>(c);
      td.theta = w->theta;
      td.step = w->step;
      td.f = f;
      td.pre = w->pre;
      td.hid = w->hid;
      td.t = w->dt;
      td.T = w->T;
      td.X = w->X;
      td.G = w->G;
      td.Y = w->Y;
      td.scal = w->scal;
      td.flags = w->flags;
      td.N = c->N;
    }
    return td;
  }

  // Iterations whose every launcher takes part in grouped launches (batch_take): the mixed or FP32 Chol_H
  // path of the 3-layer network with the structured fast POVM kernels and the bulk weight passes.
  static bool groupable(qst_ctx* c, const R* f) {
    return std::is_same<R, float>::value && !c->cnn && c->opt.mapping == QST_MAP_CHOL_H && !fused(c) &&
           fast_povm(c) && povm_needs_fperm(c->plan) && use_bulk(c, f) && c->tmax == 0;
  }

  // The steady-state iteration after the hidden layer is known: forward, likelihood,
  // backward, Rprop on W2 / b2 / b1, Rprop on W1 with the next hidden layer.  Stream
  // work only (no host synchronisation), so that it can be captured into a graph.
  static qst_status step_body(qst_ctx* c, const R* f) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    qst_status st;
    if (fused(c)) {
      if constexpr (std::is_same<R, float>::value) {
        QST_CU(join_f(c));
        QST_CU(tomo_fused_one(tomo_desc(c, f), c->Bf, c->net, c->stream));
        c->launches += 1;
        tmark(c, QST_PH_FUSED);
        return QST_OK;
      }
    }
    if (c->cnn) {  // the head changes every step, and its convolution reads f first
      QST_CU(join_f(c));
      if ((st = hidden(c, w->theta, f)) != QST_OK) return st;
    }
    if ((st = forward_state(c, w->theta)) != QST_OK) return st;
    if ((st = povm_likelihood(c, f, true)) != QST_OK) return st;
    if ((st = backward_state(c)) != QST_OK) return st;
    if (c->cnn) {
      const bool bulk = std::is_same<R, float>::value && c->bulk_passes && cnn_bulk_ok(D);
      QST_CU(cnn_output_backward<R>(D, w->theta, w->step, nullptr, w->dt, w->hid, w->pre, w->dpre, w->partials,
                                    w->counters + CNT_W2, w->flags + 1, c->net, bulk, c->stream));
      tmark(c, QST_PH_W2);
      QST_CU(cnn_head_backward<R>(D, w->theta, w->step, nullptr, f, w->feats, w->pos, w->vals, w->dpre, c->net,
                                  c->stream));
      tmark(c, QST_PH_W1);
      c->launches += bulk ? 2 : 1;  // the output layer in two halves; the head in two kernels
    } else if (use_bulk(c, f)) {
      if constexpr (std::is_same<R, float>::value) {
        QST_CU(w2_pass_bulk(D, w->theta, w->step, w->dt, w->hid, w->pre, w->dpre, w->partials,
                            w->counters + CNT_W2, w->flags + 1, c->net, c->stream));
        tmark(c, QST_PH_W2);
        QST_CU(w1_pass_bulk(D, w->theta, w->step, f, w->dpre, w->pre, w->hid, w->scal, w->partials,
                            w->counters + CNT_W1, w->flags + 1, c->net, c->stream));
        tmark(c, QST_PH_W1);
      }
    } else {
      QST_CU(net_w2_pass<R>(D, w->theta, w->step, w->dt, w->hid, w->pre, w->dpre, nullptr, w->partials,
                            w->counters + CNT_W2, c->net, true, c->stream));
      tmark(c, QST_PH_W2);
      QST_CU(net_w1_pass<R>(D, w->theta, w->step, f, w->dpre, w->pre, w->hid, nullptr, w->scal,
                            w->partials, w->counters + CNT_W1, c->net, true, c->stream));
      tmark(c, QST_PH_W1);
    }
    c->launches += 2;
    return QST_OK;
  }

  // Capture step_body for input f into c->gexec (replaces an earlier graph).  A
  // page-locked host f is copied into the staging buffer by a node of the graph.
  static qst_status capture(qst_ctx* c, const void* f_user, bool host_f) {
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    Work<R>* w = W<R>(c);
    const long long l0 = c->launches;
    const bool timed = c->tmax > 0;
    if (host_f && !c->copy_stream) {
      QST_CU(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
      QST_CU(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
      QST_CU(cudaEventCreateWithFlags(&c->ev_f, cudaEventDisableTiming));
    }
    QST_CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    const R* f = (const R*)f_user;
    cudaError_t ec = cudaSuccess;
    if (host_f) {  // fork: the copy node runs beside the kernels up to the first read of f
      ec = cudaEventRecord(c->ev_fork, c->stream);
      if (ec == cudaSuccess) ec = cudaStreamWaitEvent(c->copy_stream, c->ev_fork, 0);
      if (ec == cudaSuccess)
        ec = cudaMemcpyAsync(w->fstage, f_user, (size_t)c->D.n * sizeof(R), cudaMemcpyHostToDevice,
                             c->copy_stream);
      if (ec == cudaSuccess) ec = cudaEventRecord(c->ev_f, c->copy_stream);
      c->f_wait = ec == cudaSuccess;
      f = (const R*)w->fstage;
    }
    if (timed) {  // the phase events become nodes of the graph; every replay re-records them (slot 0)
      c->tcount = 0;
      tmark_begin(c);
    }
    qst_status st = ec == cudaSuccess ? step_body(c, f) : cuda_status(ec);
    const cudaError_t ej = join_f(c);  // the side stream must have joined before the capture ends
    if (st == QST_OK && ej != cudaSuccess) st = cuda_status(ej);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->capturing = false;
    c->tslot = -1;
    c->graph_timed = timed;
    const long long kernels = c->launches - l0;
    c->launches = l0;
    if (st != QST_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_status(e);
    const cudaError_t e2 = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) { c->gexec = nullptr; return cuda_status(e2); }
    c->gnodes = kernels;
    c->gf = f_user;
    return QST_OK;
  }

  static qst_status step(qst_ctx* c, const void* f_user, double* loss) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    qst_status st;
    const int kind = ptr_kind(f_user);
    const bool new_f = !c->hidden_valid || f_user != c->f_last;
    if (c->graph_on && kind != 0 && !new_f) {
      if (!c->gexec || c->gf != f_user) {
        if ((st = capture(c, f_user, kind == 1)) != QST_OK) return st;
      }
      QST_CU(cudaGraphLaunch(c->gexec, c->stream));
      c->launches += c->gnodes;
    } else {
      const R* f = kind == 2 ? (const R*)f_user
                             : (const R*)stage_input(c, f_user, (size_t)D.n * sizeof(R), w->fstage, &st);
      if (kind != 2 && st != QST_OK) return st;
      if (new_f && (st = validate_f<R>(c, f)) != QST_OK) return st;
      tmark_begin(c);
      if (new_f && !c->cnn) {
        if ((st = hidden(c, w->theta, f)) != QST_OK) return st;
      }
      if ((st = step_body(c, f)) != QST_OK) return st;
      c->tslot = -1;
    }
    c->hidden_valid = true;
    c->f_last = f_user;
    c->iters += 1;
    if (loss) return read_loss(c, loss);
    return QST_OK;
  }

  static qst_status loss_grad(qst_ctx* c, const void* theta_v, const void* f_user, double* loss, void* dtheta_v) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    R* theta = (R*)theta_v;
    R* dtheta = (R*)dtheta_v;
    qst_status st;
    const R* f = (const R*)stage_input(c, f_user, (size_t)D.n * sizeof(R), w->fstage, &st);
    if (st != QST_OK) return st;
    if ((st = validate_f<R>(c, f)) != QST_OK) return st;
    c->hidden_valid = false;  // the hidden buffers now hold the external parameters' activation
    c->fperm_stale = true;    // f is taken as new on every call
    if ((st = hidden(c, theta, f)) != QST_OK) return st;
    if ((st = forward_state(c, theta, false)) != QST_OK) return st;
    if ((st = povm_likelihood(c, f, true)) != QST_OK) return st;
    if ((st = backward_state(c)) != QST_OK) return st;
    if (c->cnn) {
      QST_CU(cnn_output_backward<R>(D, theta, nullptr, dtheta, w->dt, w->hid, w->pre, w->dpre, w->partials,
                                    w->counters + CNT_W2, w->flags + 1, c->net, false, c->stream));
      QST_CU(cnn_head_backward<R>(D, theta, nullptr, dtheta, f, w->feats, w->pos, w->vals, w->dpre, c->net,
                                  c->stream));
      c->launches += 1;  // the head in two kernels
    } else {
      QST_CU(net_w2_pass<R>(D, theta, nullptr, w->dt, w->hid, w->pre, w->dpre, dtheta, w->partials,
                            w->counters + CNT_W2, c->net, false, c->stream));
      QST_CU(net_w1_pass<R>(D, theta, nullptr, f, w->dpre, w->pre, w->hid, dtheta, w->scal, w->partials,
                            w->counters + CNT_W1, c->net, false, c->stream));
    }
    c->launches += 2;
    return read_loss(c, loss);
  }

  static qst_status probs(qst_ctx* c, const void* rho, void* p) {
    Work<R>* w = W<R>(c);
    if constexpr (std::is_same<R, float>::value) {
      if (fast_povm(c)) {
        QST_CU(povm_fwd_fast(c->D, (const float2*)rho, w->Wlo, (float*)p, c->plan, c->stream));
        c->launches += 2;
        return QST_OK;
      }
    }
    const PovmB<R>& B = povmB<R>(c);
    QST_CU(povm_lo_fwd<R>(c->D, (const V*)rho, w->Wlo, B, c->stream));
    QST_CU(povm_hi_fwd<R>(c->D, w->Wlo, (R*)p, B, c->stream));
    c->launches += 2;
    return QST_OK;
  }

  // Sec. 2.3 eq. F_CF (samples == 0) or eq. fc_sample between rho^ of the current parameters (input f)
  // and the target distribution P.
  static qst_status classical_fidelity(qst_ctx* c, const void* f_user, const void* P_user, long long samples,
                                       unsigned long long seed, double* Fc) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    qst_status st;
    const R* f = (const R*)stage_input(c, f_user, (size_t)D.n * sizeof(R), w->fstage, &st);
    if (st != QST_OK) return st;
    if (c->cnn || !c->hidden_valid || f_user != c->f_last) {
      if ((st = validate_f<R>(c, f)) != QST_OK) return st;
      if ((st = hidden(c, w->theta, f)) != QST_OK) return st;
      c->hidden_valid = true;
      c->f_last = f_user;
    }
    if ((st = forward_state(c, w->theta)) != QST_OK) return st;
    bool done = false;
    if constexpr (std::is_same<R, float>::value) {
      if (fast_povm(c)) {
        QST_CU(povm_fwd_fast(D, w->X, w->Wlo, w->Whi, c->plan, c->stream));  // q, unnormalised, in Whi
        done = true;
      }
    }
    if (!done) {
      const PovmB<R>& B = povmB<R>(c);
      QST_CU(povm_lo_fwd<R>(D, w->X, w->Wlo, B, c->stream));
      QST_CU(povm_hi_fwd<R>(D, w->Wlo, w->Whi, B, c->stream));  // q, unnormalised, in Whi
    }
    const R* P = (const R*)stage_input(c, P_user, (size_t)D.n * sizeof(R), w->fstage, &st);  // f is consumed
    if (st != QST_OK) return st;
    double* out = w->scal + 5;
    if (samples == 0) {
      QST_CU(classical_fidelity_exact<R>(D.n, w->Whi, P, w->scal, w->partials, w->counters + CNT_FID, out,
                                         c->stream));
      c->launches += 3;
    } else {
      if (!c->cdf) QST_CU(dalloc(c, &c->cdf, (size_t)fidelity_cdf_len(D.n)));
      QST_CU(classical_fidelity_sampled<R>(D.n, w->Whi, P, samples, seed, w->scal, c->cdf, w->partials,
                                           w->counters + CNT_FID, out, c->stream));
      c->launches += 6;
    }
    QST_CU(cudaMemcpyAsync(c->h_scal, w->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    QST_CU(cudaStreamSynchronize(c->stream));
    *Fc = c->h_scal[5];
    return QST_OK;
  }

  // Sec. 2.3 eq. F_QF through eq. fq_decom between rho^ of the current parameters (input f) and
  // w |psi><psi| / <psi|psi> + (1 - w) I / d, from the eigendecomposition of T (Chol_H: a cold Jacobi
  // run of `sweeps` sweeps that rotates psi instead of forming Q, on a workspace made on first use;
  // A_P: the decomposition of the forward, with Q).
  static qst_status state_fidelity(qst_ctx* c, const void* f_user, const void* psi_user, double wgt, int sweeps,
                                   double* Fq) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    qst_status st;
    const R* f = (const R*)stage_input(c, f_user, (size_t)D.n * sizeof(R), w->fstage, &st);
    if (st != QST_OK) return st;
    if (c->cnn || !c->hidden_valid || f_user != c->f_last) {
      if ((st = validate_f<R>(c, f)) != QST_OK) return st;
      if ((st = hidden(c, w->theta, f)) != QST_OK) return st;
      c->hidden_valid = true;
      c->f_last = f_user;
    }
    if (c->opt.mapping == QST_MAP_ABS_P) {
      if ((st = forward_state(c, w->theta)) != QST_OK) return st;
    } else {
      // T itself (complex, also in the mixed-precision path), then its decomposition
      if (c->cnn) {
        QST_CU(cnn_output<R>(D, w->theta, w->hid, w->dt, nullptr, c->stream));
        QST_CU(net_hermitian_T<R>(D, w->dt, w->T, nullptr, c->stream));
      } else {
        QST_CU(net_build_T<R>(D, w->theta, w->hid, w->dt, w->T, nullptr, c->stream));
      }
      c->launches += 2;
      if (!c->apw) {  // the eigenvalue workspace only: two d x d buffers, three d-vectors, coset unitaries
        AbsPWork<R>* ap = new (std::nothrow) AbsPWork<R>();
        if (!ap) return QST_E_NOMEM;
        memset(ap, 0, sizeof(*ap));
        c->apw = ap;
        const size_t nn = (size_t)D.d * D.d;
        QST_CU(dalloc(c, &ap->A0, nn));
        QST_CU(dalloc(c, &ap->A1, nn));
        QST_CU(dalloc(c, &ap->lam, (size_t)D.d));
        QST_CU(dalloc(c, &ap->s, (size_t)D.d));
        QST_CU(dalloc(c, &ap->sp, (size_t)D.d));
        QST_CU(dalloc(c, &ap->ucos, 16 * (size_t)D.d));
      }
    }
    const V* psi = (const V*)stage_input(c, psi_user, (size_t)D.d * sizeof(V), w->Wlo, &st);
    if (st != QST_OK) return st;
    // scratch: the fidelity's 4 d doubles, then phi = Q^dag psi (d complex)
    if (!c->fq) QST_CU(dalloc(c, &c->fq, state_fidelity_scratch_doubles(D.d) + 2 * (size_t)D.d));
    V* phi = reinterpret_cast<V*>(c->fq + state_fidelity_scratch_doubles(D.d));
    AbsPWork<R>& ap = *reinterpret_cast<AbsPWork<R>*>(c->apw);
    const bool absp = c->opt.mapping == QST_MAP_ABS_P;
    if (!absp) {
      const int sw = (sweeps > 0 ? sweeps : c->sweeps) + ((sweeps > 0 ? sweeps : c->sweeps) & 1);
      QST_CU(jacobi_values_project<R>(D.d, w->T, ap, sw, 2.0, psi, phi, c->stream));
      c->launches += 1 + (long long)sw * jacobi_kernels_per_sweep(D.d);
    }
    double* out = w->scal + 8;
    QST_CU(state_fidelity_from_decomposition<R>(D.d, absp ? ap.Qh : nullptr, phi, ap.s, psi, wgt, c->fq, out,
                                                w->counters + CNT_FID, c->stream));
    c->launches += 3;
    QST_CU(cudaMemcpyAsync(c->h_scal, w->scal, 11 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    QST_CU(cudaStreamSynchronize(c->stream));
    *Fq = c->h_scal[10];
    return QST_OK;
  }

  static qst_status get_rho(qst_ctx* c, const void* f_user, void* rho_out, double* loss) {
    Work<R>* w = W<R>(c);
    const Dims& D = c->D;
    qst_status st;
    const R* f = (const R*)stage_input(c, f_user, (size_t)D.n * sizeof(R), w->fstage, &st);
    if (st != QST_OK) return st;
    if (c->cnn || !c->hidden_valid || f_user != c->f_last) {
      if ((st = validate_f<R>(c, f)) != QST_OK) return st;
      if ((st = hidden(c, w->theta, f)) != QST_OK) return st;
      c->hidden_valid = true;
      c->f_last = f_user;
    }
    if ((st = forward_state(c, w->theta)) != QST_OK) return st;
    const bool dev = is_device_ptr(rho_out);
    V* dst = dev ? (V*)rho_out : w->G;
    if (rho_out) {
      QST_CU(hermitian_complete<R>(D, w->X, dst, w->scal, c->stream));
      c->launches += 1;
      if (!dev) {
        QST_CU(cudaMemcpyAsync(rho_out, dst, (size_t)D.d * D.d * sizeof(V), cudaMemcpyDeviceToHost, c->stream));
        QST_CU(cudaStreamSynchronize(c->stream));
      }
    }
    if (loss) {
      if ((st = povm_likelihood(c, f, false)) != QST_OK) return st;
      return read_loss(c, loss);
    }
    return QST_OK;
  }
};

#define QST_DISPATCH(c, call) ((c)->prec == QST_FP64 ? Engine<double>::call : Engine<float>::call)

template <class R> qst_status reset_rprop(qst_ctx* c) {
  Work<R>* w = W<R>(c);
  const size_t P = c->P;
  std::vector<R> h(P, rprop_encode((R)c->opt.lr, 0));  // step lr, previous sign 0
  QST_CU(cudaMemcpyAsync(w->step, h.data(), P * sizeof(R), cudaMemcpyHostToDevice, c->stream));
  QST_CU(cudaStreamSynchronize(c->stream));
  return QST_OK;
}

double* ctx_scal(qst_ctx* c) {
  return c->prec == QST_FP64 ? W<double>(c)->scal : W<float>(c)->scal;
}

__global__ void k_gather_losses(double* const* scal, double* out, int B) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) out[b] = scal[b][2];
}

}  // namespace

struct qst_batch {
  int B = 0;
  std::vector<qst_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  cudaStream_t root = nullptr;
  bool own_root = false;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> gf;
  long long gnodes = 0;
  long long launches = 0;
  double** d_scal = nullptr;
  double* d_losses = nullptr;
  double* h_losses = nullptr;
  // the tomographies that run as one-CTA iterations: one persistent launch over this work list
  TomoDesc* d_list = nullptr;
  int list_cap = 0;
  unsigned int* d_next = nullptr;
  cudaStream_t fused_stream = nullptr;
  cudaEvent_t fused_done = nullptr;
  // groups of tomographies of one size that run each kernel of their iteration as one launch
  std::vector<BatchRec> groups;
  unsigned char* d_tab = nullptr;  // their pointer tables and tensor-map copies
  size_t tab_cap = 0;
};

namespace {

// Record one iteration of every member of a group with the launches skipped (inside a capture that is
// thrown away, so that a launcher that does not take part shows up as a node and nothing runs); false
// when the group cannot run as grouped launches.
bool record_group(qst_batch* bt, const std::vector<int>& mem, const void* const* f, BatchRec& rec) {
  rec = BatchRec();
  rec.mode = BatchRec::RECORD;
  rec.count = (int)mem.size();
  for (int i = 0; i < rec.count; ++i) {
    qst_ctx* c = bt->ctx[mem[i]];
    if (!Engine<float>::groupable(c, (const float*)f[mem[i]])) return false;
    rec.member = i;
    rec.call = 0;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const long long l0 = c->launches;
    batch_rec() = &rec;
    const qst_status st = Engine<float>::step_body(c, (const float*)f[mem[i]]);
    batch_rec() = nullptr;
    c->launches = l0;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    size_t nodes = 1;
    if (g) {
      if (cudaGraphGetNodes(g, nullptr, &nodes) != cudaSuccess) nodes = 1;
      cudaGraphDestroy(g);
    }
    if (st != QST_OK || e != cudaSuccess || nodes != 0 || rec.bad || rec.call != (int)rec.calls.size()) {
      cudaGetLastError();
      return false;
    }
  }
  return !rec.calls.empty();
}

// Copy the groups' pointer tables (row z: tomography z's pointers, a blob's device address first) and
// blobs into one device buffer, and point every call at its table.
cudaError_t upload_groups(qst_batch* bt) {
  auto up = [](size_t x, size_t a) { return (x + a - 1) / a * a; };
  size_t total = 0;
  for (const BatchRec& r : bt->groups)
    for (const BatchRec::Call& c : r.calls) {
      if (c.blob_bytes) total = up(total, 128) + c.blob_bytes * r.count;
      total = up(total, 16) + sizeof(void*) * c.nptr * r.count;
    }
  if (total == 0) return cudaSuccess;
  if (total > bt->tab_cap) {
    if (bt->d_tab) cudaFree(bt->d_tab);
    bt->d_tab = nullptr;
    bt->tab_cap = 0;
    cudaError_t e = cudaMalloc(&bt->d_tab, total);
    if (e != cudaSuccess) return e;
    bt->tab_cap = total;
  }
  std::vector<unsigned char> img(total);
  size_t off = 0;
  for (BatchRec& r : bt->groups)
    for (BatchRec::Call& c : r.calls) {
      size_t boff = 0;
      if (c.blob_bytes) {
        off = up(off, 128);
        boff = off;
        memcpy(&img[off], c.blobs.data(), c.blob_bytes * r.count);
        off += c.blob_bytes * r.count;
      }
      off = up(off, 16);
      const void** row = reinterpret_cast<const void**>(&img[off]);
      const int np = c.nptr - (c.blob_bytes ? 1 : 0);
      for (int z = 0; z < r.count; ++z) {
        int k = 0;
        if (c.blob_bytes) row[(size_t)z * c.nptr + k++] = bt->d_tab + boff + (size_t)z * c.blob_bytes;
        for (int q = 0; q < np; ++q) row[(size_t)z * c.nptr + k++] = c.ptrs[(size_t)z * np + q];
      }
      c.dtab = reinterpret_cast<const void* const*>(bt->d_tab + off);
      off += sizeof(void*) * c.nptr * r.count;
    }
  return cudaMemcpy(bt->d_tab, img.data(), total, cudaMemcpyHostToDevice);
}

// One iteration of every tomography of the batch, captured once into a single graph:
// the root stream forks to one stream per tomography and joins them again.
qst_status batch_capture(qst_batch* bt, const void* const* f) {
  if (bt->gexec) { cudaGraphExecDestroy(bt->gexec); bt->gexec = nullptr; }
  std::vector<int> order(bt->B);
  for (int b = 0; b < bt->B; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bt->ctx[a]->N > bt->ctx[b]->N; });
  // The work list of the fused tomographies, largest first (the last CTAs to start get the shortest work).
  std::vector<TomoDesc> list;
  const qst_ctx* fc = nullptr;
  for (int b : order) {
    qst_ctx* c = bt->ctx[b];
    if (c->prec == QST_FP64 || !Engine<float>::fused(c)) continue;
    list.push_back(Engine<float>::tomo_desc(c, (const float*)f[b]));
    fc = c;
  }
  // The others, in runs of one qubit count (largest first).  A run of two or more FP32-based tomographies
  // runs each kernel of its iteration once for the whole run (grid z = the tomography) when every
  // launcher of its iteration takes part; otherwise every tomography runs its own chain of kernels.
  order.erase(std::remove_if(order.begin(), order.end(),
                             [&](int b) { return bt->ctx[b]->prec != QST_FP64 && Engine<float>::fused(bt->ctx[b]); }),
              order.end());
  const int nrest = (int)order.size();
  std::vector<std::pair<int, int>> runs;
  for (int i = 0; i < nrest;) {
    int j = i;
    while (j < nrest && bt->ctx[order[j]]->N == bt->ctx[order[i]]->N) ++j;
    runs.emplace_back(i, j);
    i = j;
  }
  std::vector<int> run_group(runs.size(), -1);
  bt->groups.clear();
  for (size_t r = 0; r < runs.size(); ++r) {
    const int i = runs[r].first, j = runs[r].second;
    if (j - i < 2 || bt->ctx[order[i]]->prec == QST_FP64) continue;
    const std::vector<int> mem(order.begin() + i, order.begin() + j);
    BatchRec rec;
    if (record_group(bt, mem, f, rec)) {
      run_group[r] = (int)bt->groups.size();
      bt->groups.push_back(std::move(rec));
    }
  }
  if (!list.empty() || !bt->groups.empty())
    QST_CU(cudaStreamSynchronize(bt->root));  // an earlier graph may still read the old list and tables
  if (!list.empty()) {
    if ((int)list.size() > bt->list_cap) {
      if (bt->d_list) cudaFree(bt->d_list);
      bt->d_list = nullptr;
      bt->list_cap = 0;
      QST_CU(cudaMalloc(&bt->d_list, list.size() * sizeof(TomoDesc)));
      bt->list_cap = (int)list.size();
    }
    if (!bt->d_next) QST_CU(cudaMalloc(&bt->d_next, sizeof(unsigned int)));
    if (!bt->fused_stream) {
      QST_CU(cudaStreamCreateWithFlags(&bt->fused_stream, cudaStreamNonBlocking));
      QST_CU(cudaEventCreateWithFlags(&bt->fused_done, cudaEventDisableTiming));
    }
    QST_CU(cudaMemcpy(bt->d_list, list.data(), list.size() * sizeof(TomoDesc), cudaMemcpyHostToDevice));
  }
  QST_CU(upload_groups(bt));
  QST_CU(cudaStreamBeginCapture(bt->root, cudaStreamCaptureModeThreadLocal));
  qst_status st = QST_OK;
  long long kernels = 0;
  cudaError_t e = cudaSuccess;
  if (!list.empty()) {  // forked at the start: beside the launches of the other tomographies
    e = cudaEventRecord(bt->fork, bt->root);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->fused_stream, bt->fork, 0);
    if (e == cudaSuccess)
      e = tomo_fused_list(bt->d_list, (int)list.size(), fc->Bf, fc->net, bt->d_next, bt->fused_stream);
    if (e == cudaSuccess) e = cudaEventRecord(bt->fused_done, bt->fused_stream);
    kernels += 1;
  }
  // The runs go one after another, largest first.  Within a run of chains the tomographies run
  // concurrently: mixing sizes in one fork lets the full-GPU kernels of the large ones hold SMs while
  // the short chains of the small ones wait (measured 34 ms per iteration of the 512-tomography batch
  // mixed, against about 14 ms as the sum of its same-N groups).
  for (size_t r = 0; r < runs.size() && st == QST_OK && e == cudaSuccess; ++r) {
    const int i = runs[r].first, j = runs[r].second;
    // the run starts when the previous one has joined, or (batch_concurrent_runs) with all the others
    if (r == 0 || !tuning().batch_concurrent_runs) e = cudaEventRecord(bt->fork, bt->root);
    if (e != cudaSuccess) break;
    if (run_group[r] >= 0) {  // one launch per kernel, on the first member's stream
      BatchRec& rec = bt->groups[run_group[r]];
      const int b0 = order[i];
      qst_ctx* c = bt->ctx[b0];
      e = cudaStreamWaitEvent(c->stream, bt->fork, 0);
      if (e != cudaSuccess) break;
      rec.mode = BatchRec::LAUNCH;
      rec.call = 0;
      rec.bad = false;
      const long long l0 = c->launches;
      batch_rec() = &rec;
      st = Engine<float>::step_body(c, (const float*)f[b0]);
      batch_rec() = nullptr;
      c->launches = l0;
      if (st == QST_OK && (rec.bad || rec.call != (int)rec.calls.size())) st = QST_E_CUDA;
      kernels += (long long)rec.calls.size();
      if (st != QST_OK) break;
      e = cudaEventRecord(bt->done[b0], c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->root, bt->done[b0], 0);
      continue;
    }
    for (int k = i; k < j && st == QST_OK && e == cudaSuccess; ++k) {
      const int b = order[k];
      qst_ctx* c = bt->ctx[b];
      e = cudaStreamWaitEvent(c->stream, bt->fork, 0);
      if (e != cudaSuccess) break;
      const long long l0 = c->launches;
      st = c->prec == QST_FP64 ? Engine<double>::step_body(c, (const double*)f[b])
                               : Engine<float>::step_body(c, (const float*)f[b]);
      kernels += c->launches - l0;
      c->launches = l0;
      if (st != QST_OK) break;
      e = cudaEventRecord(bt->done[b], c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->root, bt->done[b], 0);
    }
  }
  if (!list.empty() && e == cudaSuccess) e = cudaStreamWaitEvent(bt->root, bt->fused_done, 0);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(bt->root, &g);
  if (st != QST_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_status(e); }
  if (e2 != cudaSuccess) return cuda_status(e2);
  const cudaError_t e3 = cudaGraphInstantiate(&bt->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) { bt->gexec = nullptr; return cuda_status(e3); }
  bt->gnodes = kernels;
  bt->gf.assign(f, f + bt->B);
  return QST_OK;
}

}  // namespace

// =============================================================================== C ABI
extern "C" {

void qst_default_options(qst_options* o) {
  if (!o) return;
  o->mapping = QST_MAP_CHOL_H;
  o->precision = QST_FP32;
  o->P = 2.0;
  o->lr = 1e-3;
  o->eta_minus = 0.5;
  o->eta_plus = 1.2;
  o->step_min = 1e-6;
  o->step_max = 50.0;
  o->leaky_slope = 0.01;
  o->eig_sweeps = 0;
  o->eig_warm_sweeps = 0;
  o->network = QST_NET_FNN;
  o->device_memory_limit = 0;
  o->fused_max_qubits = 0;
  o->eig_refine = 1;
}

size_t qst_theta_size(int N) {
  if (N < 1 || N > 12) return 0;
  return theta_size(N);
}

size_t qst_theta_size_net(int N, int network) {
  if (network == QST_NET_CNN) return N < 3 || N > 12 ? 0 : cnn_theta_size(N);
  return network == QST_NET_FNN ? qst_theta_size(N) : 0;
}

qst_status qst_init(qst_ctx** out, int N, const double* povm, int K, const qst_options* opt, void* stream) {
  if (out == nullptr) return QST_E_INVAL;
  *out = nullptr;
  qst_options o;
  qst_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != QST_FP64 && o.precision != QST_FP32 && o.precision != QST_MIXED &&
      o.precision != QST_MIXED_BF16)
    return QST_E_INVAL;
  if (N < 1 || N > (o.precision == QST_FP64 ? 10 : 12)) return QST_E_INVAL;
  if (o.mapping != QST_MAP_CHOL_H && o.mapping != QST_MAP_ABS_P && o.mapping != QST_MAP_CHOL_DELTA)
    return QST_E_INVAL;
  if (o.mapping == QST_MAP_CHOL_DELTA && (o.precision == QST_MIXED || o.precision == QST_MIXED_BF16))
    return QST_E_UNSUPPORTED;
  if (o.network != QST_NET_FNN && o.network != QST_NET_CNN) return QST_E_INVAL;
  if (o.network == QST_NET_CNN && N < 3) return QST_E_INVAL;  // 2^(N-3)-square pooling windows
  if (o.fused_max_qubits < -1 || o.fused_max_qubits > kFusedMaxQubits) return QST_E_INVAL;
  if (o.eig_refine != 0 && o.eig_refine != 1) return QST_E_INVAL;
  if (o.mapping == QST_MAP_ABS_P) {
    if (!(o.P > 0.0) || !isfinite(o.P) || o.eig_sweeps < 0) return QST_E_INVAL;
  }
  // steps within [2^-33, 2^30]: the Rprop state word then holds the previous sign exactly (rprop_encode)
  const double lo = ldexp(1.0, -33), hi = ldexp(1.0, 30);
  if (!(o.lr >= lo && o.lr <= hi) || !(o.eta_minus > 0 && o.eta_minus < 1) || !(o.eta_plus > 1) ||
      !(o.step_min >= lo) || !(o.step_max >= o.step_min && o.step_max <= hi) || !(o.leaky_slope >= 0))
    return QST_E_INVAL;
  PovmB<double> Bd;
  qst_status st = (qst_status)check_povm(povm, K, &Bd);
  if (st != QST_OK) return st;
  if (o.precision == QST_MIXED || o.precision == QST_MIXED_BF16) {
    if (N < 7) return QST_E_UNSUPPORTED;
    if (!tc_available()) return QST_E_UNSUPPORTED;
  }
  qst_ctx* c = new (std::nothrow) qst_ctx();
  if (!c) return QST_E_NOMEM;
  c->N = N;
  c->opt = o;
  c->prec = o.precision;
  c->D = make_dims(N, o.precision == QST_FP64);
  c->cnn = o.network == QST_NET_CNN;
  if (c->cnn) {
    c->D.cnn = 1;
    c->D.H = 4 * N;
  }
  c->P = c->cnn ? cnn_theta_size(N) : theta_size(N);
  c->stream = (cudaStream_t)stream;
  c->Bd = Bd;
  for (int a = 0; a < 4; ++a)
    for (int m = 0; m < 4; ++m) c->Bf.b[a][m] = (float)Bd.b[a][m];
  c->plan = make_povm_plan(Bd);
  c->net.slope = o.leaky_slope;
  c->net.eta_minus = o.eta_minus;
  c->net.eta_plus = o.eta_plus;
  c->net.step_min = o.step_min;
  c->net.step_max = o.step_max;
  cudaGetDevice(&c->device);
  cudaError_t e = cudaMallocHost((void**)&c->h_scal, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_flags, 8 * sizeof(unsigned int));
  if (e != cudaSuccess) {
    qst_destroy(c);
    return cuda_status(e);
  }
  st = c->prec == QST_FP64 ? alloc_work<double>(c) : alloc_work<float>(c);
  if (st != QST_OK) {
    qst_destroy(c);
    return st;
  }
  *out = c;
  return QST_OK;
}

qst_status qst_set_params(qst_ctx* c, const void* theta) {
  if (!c || !theta) return QST_E_INVAL;
  const size_t bytes = c->P * rsize(c);
  void* dst = c->prec == QST_FP64 ? (void*)W<double>(c)->theta : (void*)W<float>(c)->theta;
  QST_CU(cudaMemcpyAsync(dst, theta, bytes, cudaMemcpyDefault, c->stream));
  qst_status st = c->prec == QST_FP64 ? reset_rprop<double>(c) : reset_rprop<float>(c);
  if (st != QST_OK) return st;
  c->params_set = true;
  c->hidden_valid = false;
  c->warm_valid = false;
  c->iters = 0;
  return QST_OK;
}

qst_status qst_get_params(qst_ctx* c, void* theta) {
  if (!c || !theta) return QST_E_INVAL;
  if (!c->params_set) return QST_E_STATE;
  const size_t bytes = c->P * rsize(c);
  const void* src = c->prec == QST_FP64 ? (void*)W<double>(c)->theta : (void*)W<float>(c)->theta;
  QST_CU(cudaMemcpyAsync(theta, src, bytes, cudaMemcpyDefault, c->stream));
  if (!is_device_ptr(theta)) QST_CU(cudaStreamSynchronize(c->stream));
  return QST_OK;
}

qst_status qst_probs(qst_ctx* c, const void* rho, void* p) {
  if (!c || !rho || !p) return QST_E_INVAL;
  if (!is_device_ptr(rho) || !is_device_ptr(p)) return QST_E_INVAL;
  return QST_DISPATCH(c, probs(c, rho, p));
}

qst_status qst_loss_grad(qst_ctx* c, const void* theta, const void* f, double* loss, void* dtheta) {
  if (!c || !theta || !f || !loss || !dtheta) return QST_E_INVAL;
  if (!is_device_ptr(theta) || !is_device_ptr(dtheta)) return QST_E_INVAL;
  return QST_DISPATCH(c, loss_grad(c, theta, f, loss, dtheta));
}

qst_status qst_step(qst_ctx* c, const void* f, double* loss) {
  if (!c || !f) return QST_E_INVAL;
  if (!c->params_set) return QST_E_STATE;
  return QST_DISPATCH(c, step(c, f, loss));
}

qst_status qst_get_rho(qst_ctx* c, const void* f, void* rho_out, double* loss) {
  if (!c || !f) return QST_E_INVAL;
  if (!c->params_set) return QST_E_STATE;
  return QST_DISPATCH(c, get_rho(c, f, rho_out, loss));
}

qst_status qst_classical_fidelity(qst_ctx* c, const void* f, const void* P, long long samples,
                                  unsigned long long seed, double* Fc) {
  if (!c || !f || !P || !Fc || samples < 0) return QST_E_INVAL;
  if (!c->params_set) return QST_E_STATE;
  return QST_DISPATCH(c, classical_fidelity(c, f, P, samples, seed, Fc));
}

qst_status qst_state_fidelity(qst_ctx* c, const void* f, const void* psi, double w, int sweeps, double* Fq) {
  if (!c || !f || !psi || !Fq || !(w >= 0.0 && w <= 1.0) || sweeps < 0) return QST_E_INVAL;
  if (c->opt.mapping == QST_MAP_CHOL_DELTA) return QST_E_UNSUPPORTED;
  if (!c->params_set) return QST_E_STATE;
  return QST_DISPATCH(c, state_fidelity(c, f, psi, w, sweeps, Fq));
}

qst_status qst_test_state(qst_ctx* c, int kind, double w, void* rho) {
  if (!c || !rho || !(w >= 0.0 && w <= 1.0)) return QST_E_INVAL;
  if (kind != QST_STATE_PRODUCT && kind != QST_STATE_GHZI && kind != QST_STATE_W) return QST_E_INVAL;
  if (!is_device_ptr(rho)) return QST_E_INVAL;
  cudaError_t e = c->prec == QST_FP64 ? make_test_state<double>(c->N, kind, w, (cx_t<double>*)rho, c->stream)
                                      : make_test_state<float>(c->N, kind, w, (cx_t<float>*)rho, c->stream);
  QST_CU(e);
  c->launches += 1;
  return QST_OK;
}

qst_status qst_sample_counts(qst_ctx* c, const double* P, long long shots, unsigned long long seed,
                             long long* counts, void* f) {
  if (!c || !P || !counts || shots < 0) return QST_E_INVAL;
  if (!is_device_ptr(P) || !is_device_ptr(counts) || (f && !is_device_ptr(f))) return QST_E_INVAL;
  const long long n = c->D.n;
  if (!c->samp) QST_CU(dalloc(c, &c->samp, (size_t)sampler_scratch_words(n)));
  unsigned int* flags = c->prec == QST_FP64 ? W<double>(c)->flags : W<float>(c)->flags;
  QST_CU(cudaMemsetAsync(flags + 2, 0, sizeof(unsigned int), c->stream));
  QST_CU(multinomial_prepare(n, P, c->samp, counts, flags + 2, c->stream));
  // the total weight and the input check decide whether draws can be made
  unsigned long long W = 0;
  QST_CU(cudaMemcpyAsync(c->h_flags + 2, flags + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream));
  QST_CU(cudaMemcpyAsync(&W, c->samp + n - 1, sizeof(W), cudaMemcpyDeviceToHost, c->stream));
  QST_CU(cudaStreamSynchronize(c->stream));
  c->launches += 3;
  if (c->h_flags[2] != 0u || W == 0ull) return QST_E_INPUT;
  QST_CU(multinomial_draw(n, shots, seed, c->samp, counts, c->stream));
  c->launches += shots > 0 ? 1 : 0;
  if (f && shots > 0) {
    cudaError_t e = c->prec == QST_FP64 ? counts_to_frequencies<double>(n, counts, shots, (double*)f, c->stream)
                                        : counts_to_frequencies<float>(n, counts, shots, (float*)f, c->stream);
    QST_CU(e);
    c->launches += 1;
  }
  return QST_OK;
}

qst_status qst_reconstruct(qst_ctx* c, const void* f, int iters, void* rho_out, double* final_loss) {
  if (!c || !f || iters < 0) return QST_E_INVAL;
  if (!c->params_set) return QST_E_STATE;
  for (int i = 0; i < iters; ++i) {
    qst_status st = qst_step(c, f, nullptr);
    if (st < 0) return st;
  }
  if (rho_out || final_loss) return qst_get_rho(c, f, rho_out, final_loss);
  return QST_OK;
}

// Warm-start eigenvectors in a checkpoint (QST_MAP_ABS_P): a flag word, then d x d complex.
size_t warm_bytes(const qst_ctx* c) {
  if (c->opt.mapping != QST_MAP_ABS_P) return 0;
  return sizeof(unsigned long long) + (size_t)c->D.d * c->D.d * 2 * rsize(c);
}

void* warm_q(qst_ctx* c) {
  return c->prec == QST_FP64 ? (void*)reinterpret_cast<AbsPWork<double>*>(c->apw)->V0
                             : (void*)reinterpret_cast<AbsPWork<float>*>(c->apw)->V0;
}

size_t qst_state_bytes(const qst_ctx* c) {
  if (!c) return 0;
  const size_t P = c->P;
  return 4 * sizeof(unsigned long long) + 2 * P * rsize(c) + warm_bytes(c);
}

qst_status qst_get_state(qst_ctx* c, void* host_buf, size_t bytes) {
  if (!c || !host_buf) return QST_E_INVAL;
  if (!c->params_set) return QST_E_STATE;
  if (bytes < qst_state_bytes(c)) return QST_E_INVAL;
  const size_t P = c->P, rs = rsize(c);
  unsigned long long* hdr = (unsigned long long*)host_buf;
  hdr[0] = kStateMagic;
  hdr[1] = (unsigned long long)c->N | ((unsigned long long)c->prec << 8);
  hdr[2] = (unsigned long long)c->iters;
  hdr[3] = (unsigned long long)P;
  char* p = (char*)host_buf + 4 * sizeof(unsigned long long);
  const void *th, *stp;
  if (c->prec == QST_FP64) { th = W<double>(c)->theta; stp = W<double>(c)->step; }
  else { th = W<float>(c)->theta; stp = W<float>(c)->step; }
  QST_CU(cudaMemcpyAsync(p, th, P * rs, cudaMemcpyDeviceToHost, c->stream));
  QST_CU(cudaMemcpyAsync(p + P * rs, stp, P * rs, cudaMemcpyDeviceToHost, c->stream));
  if (warm_bytes(c)) {
    char* q = p + 2 * P * rs;
    *(unsigned long long*)q = c->warm_valid ? 1ULL : 0ULL;
    if (c->warm_valid)
      QST_CU(cudaMemcpyAsync(q + sizeof(unsigned long long), warm_q(c), warm_bytes(c) - sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
  }
  QST_CU(cudaStreamSynchronize(c->stream));
  return QST_OK;
}

qst_status qst_set_state(qst_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf) return QST_E_INVAL;
  if (bytes < qst_state_bytes(c)) return QST_E_INVAL;
  const size_t P = c->P, rs = rsize(c);
  const unsigned long long* hdr = (const unsigned long long*)host_buf;
  if (hdr[0] != kStateMagic || hdr[1] != ((unsigned long long)c->N | ((unsigned long long)c->prec << 8)) ||
      hdr[3] != (unsigned long long)P)
    return QST_E_INVAL;
  const char* p = (const char*)host_buf + 4 * sizeof(unsigned long long);
  void *th, *stp;
  if (c->prec == QST_FP64) { th = W<double>(c)->theta; stp = W<double>(c)->step; }
  else { th = W<float>(c)->theta; stp = W<float>(c)->step; }
  QST_CU(cudaMemcpyAsync(th, p, P * rs, cudaMemcpyHostToDevice, c->stream));
  QST_CU(cudaMemcpyAsync(stp, p + P * rs, P * rs, cudaMemcpyHostToDevice, c->stream));
  c->warm_valid = false;
  if (warm_bytes(c)) {
    const char* q = p + 2 * P * rs;
    if (*(const unsigned long long*)q) {
      QST_CU(cudaMemcpyAsync(warm_q(c), q + sizeof(unsigned long long), warm_bytes(c) - sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, c->stream));
      if (c->prec == QST_FP64)
        QST_CU(abs_p_restore_q<double>(c->D.d, *reinterpret_cast<AbsPWork<double>*>(c->apw), c->stream));
      else
        QST_CU(abs_p_restore_q<float>(c->D.d, *reinterpret_cast<AbsPWork<float>*>(c->apw), c->stream));
      c->warm_valid = true;
    }
  }
  QST_CU(cudaStreamSynchronize(c->stream));
  c->params_set = true;
  c->hidden_valid = false;
  c->iters = (long long)hdr[2];
  return QST_OK;
}

qst_status qst_eig_counts(const qst_ctx* c, long long* refinements, long long* fallbacks, double* last) {
  if (!c) return QST_E_INVAL;
  if (refinements) *refinements = c->oa_refinements;
  if (fallbacks) *fallbacks = c->oa_fallbacks;
  if (last) {
    last[0] = c->oa_last[0];
    last[1] = c->oa_last[1];
  }
  return QST_OK;
}

qst_status qst_jacobi_schedule(int N, int* count, int* dims, int* basis, int cap) {
  if (N < 1 || N > 12 || !count || cap < 0 || (cap > 0 && (!dims || !basis))) return QST_E_INVAL;
  const std::vector<qst::JacobiPass>& s = qst::jacobi_schedule(N);
  *count = (int)s.size();
  for (int k = 0; k < cap && k < (int)s.size(); ++k) {
    dims[k] = s[k].k;
    for (int i = 0; i < 4; ++i) basis[4 * k + i] = i < s[k].k ? s[k].basis[i] : 0;
  }
  return QST_OK;
}

long long qst_iterations(const qst_ctx* c) { return c ? c->iters : -1; }
long long qst_kernel_launches(const qst_ctx* c) { return c ? c->launches : -1; }

qst_status qst_timing_enable(qst_ctx* c, int max_steps) {
  if (!c || max_steps < 0) return QST_E_INVAL;
  QST_CU(cudaStreamSynchronize(c->stream));
  if (c->gexec) {  // recaptured on the next step, with or without the phase events
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gf = nullptr;
  }
  c->graph_timed = false;
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  c->tev.clear();
  c->tmask.clear();
  c->tmax = 0;
  c->tcount = 0;
  c->tslot = -1;
  if (max_steps == 0) return QST_OK;
  const size_t ne = (size_t)max_steps * (QST_NPHASE + 1);
  c->tev.resize(ne);
  for (size_t i = 0; i < ne; ++i) QST_CU(cudaEventCreate(&c->tev[i]));
  c->tmask.assign((size_t)max_steps, 0u);
  c->tmax = max_steps;
  return QST_OK;
}

qst_status qst_timing_read(qst_ctx* c, double* phase_ms, long long* phase_count, int nphase) {
  if (!c || !phase_ms || !phase_count || nphase < 1) return QST_E_INVAL;
  QST_CU(cudaStreamSynchronize(c->stream));
  for (int p = 0; p < nphase; ++p) { phase_ms[p] = 0.0; phase_count[p] = 0; }
  // With a timed graph, slot 0 holds the events of the latest replay (if any replay ran).
  const int slots = c->graph_timed ? (c->gexec && c->iters > 0 ? 1 : 0) : c->tcount;
  for (int s = 0; s < slots; ++s) {
    cudaEvent_t prev = c->tev[(size_t)s * (QST_NPHASE + 1)];
    for (int p = 0; p < QST_NPHASE; ++p) {
      if (!(c->tmask[s] & (1u << p))) continue;
      cudaEvent_t e = c->tev[(size_t)s * (QST_NPHASE + 1) + 1 + p];
      float ms = 0.f;
      QST_CU(cudaEventElapsedTime(&ms, prev, e));
      if (p < nphase) { phase_ms[p] += ms; phase_count[p] += 1; }
      prev = e;
    }
  }
  if (!c->graph_timed) c->tcount = 0;
  return QST_OK;
}

qst_status qst_inject_wait_timeout(int what, int count) {
  if (count < 0) return QST_E_INVAL;
  if (what == QST_INJECT_TC_LOADS) g_inject[INJ_TC_LOADS].store(count);
  else if (what == QST_INJECT_WPASS_LOADS) g_inject[INJ_WPASS_LOADS].store(count);
  else return QST_E_INVAL;
  return QST_OK;
}

void qst_get_tuning(qst_tuning* t) {
  if (!t) return;
  const Tuning u = tuning();
  t->bulk_chunks_per_cta = u.bulk_chunks_per_cta;
  t->fused_ctas_per_sm = u.fused_ctas_per_sm;
  t->fused_max_qubits = u.fused_max_qubits;
  t->batch_concurrent_runs = u.batch_concurrent_runs;
}

qst_status qst_set_tuning(const qst_tuning* t) {
  if (!t || t->bulk_chunks_per_cta < 1 || t->bulk_chunks_per_cta > (1 << 20) || t->fused_ctas_per_sm < 1 ||
      t->fused_ctas_per_sm > kFusedCtasPerSmMax || t->fused_max_qubits < 0 || t->fused_max_qubits > kFusedMaxQubits ||
      (t->batch_concurrent_runs != 0 && t->batch_concurrent_runs != 1))
    return QST_E_INVAL;
  g_bulk_chunks.store(t->bulk_chunks_per_cta);
  g_fused_ctas.store(t->fused_ctas_per_sm);
  g_fused_max.store(t->fused_max_qubits);
  g_concurrent.store(t->batch_concurrent_runs);
  return QST_OK;
}

qst_status qst_graph_enable(qst_ctx* c, int enable) {
  if (!c) return QST_E_INVAL;
  if (enable && c->stream == nullptr) return QST_E_UNSUPPORTED;  // the legacy stream cannot be captured
  c->graph_on = enable != 0;
  if (!c->graph_on && c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gf = nullptr;
  }
  return QST_OK;
}

qst_status qst_sync(qst_ctx* c) {
  if (!c) return QST_E_INVAL;
  QST_CU(cudaStreamSynchronize(c->stream));
  return QST_OK;
}

const char* qst_strerror(qst_status s) {
  switch (s) {
    case QST_OK: return "ok";
    case QST_E_INVAL: return "invalid argument";
    case QST_E_INPUT: return "invalid input data (f must be finite, >= 0 and sum to 1)";
    case QST_E_NOMEM: return "device allocation failed";
    case QST_E_CUDA: return "CUDA runtime error";
    case QST_E_TIMEOUT: return "device-side wait timed out";
    case QST_E_STATE: return "call not valid in the context's state";
    case QST_E_UNSUPPORTED: return "unsupported configuration";
    case QST_W_CLAMP: return "warning: non-positive probability clamped before its logarithm";
  }
  return "unknown status";
}

void qst_destroy(qst_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (void* p : c->allocs) cudaFree(p);
  if (c->work) {
    if (c->prec == QST_FP64) free_work<double>(c);
    else free_work<float>(c);
  }
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_f) cudaEventDestroy(c->ev_f);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  delete c;
}

}  // extern "C"

// =============================================================================== batches of tomographies
extern "C" {

qst_status qst_batch_init(qst_batch** out, int B, const int* Ns, const double* povm, int K, const qst_options* opt,
                          void* stream) {
  if (!out || B < 1 || !Ns) return QST_E_INVAL;
  *out = nullptr;
  qst_batch* bt = new (std::nothrow) qst_batch();
  if (!bt) return QST_E_NOMEM;
  bt->B = B;
  auto fail = [&](qst_status st) { qst_batch_destroy(bt); return st; };
  if (stream) {
    bt->root = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&bt->root, cudaStreamNonBlocking) != cudaSuccess) return fail(QST_E_CUDA);
    bt->own_root = true;
  }
  if (cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming) != cudaSuccess) return fail(QST_E_CUDA);
  qst_options o;
  qst_default_options(&o);
  if (opt) o = *opt;
  bt->ctx.assign(B, nullptr);
  bt->streams.assign(B, nullptr);
  bt->done.assign(B, nullptr);
  std::vector<double*> scal(B);
  for (int b = 0; b < B; ++b) {
    if (cudaStreamCreateWithFlags(&bt->streams[b], cudaStreamNonBlocking) != cudaSuccess) return fail(QST_E_CUDA);
    if (cudaEventCreateWithFlags(&bt->done[b], cudaEventDisableTiming) != cudaSuccess) return fail(QST_E_CUDA);
    qst_options ob = o;
    if ((ob.precision == QST_MIXED || ob.precision == QST_MIXED_BF16) && Ns[b] < 7) ob.precision = QST_FP32;
    const qst_status st = qst_init(&bt->ctx[b], Ns[b], povm, K, &ob, bt->streams[b]);
    if (st != QST_OK) return fail(st);
    scal[b] = ctx_scal(bt->ctx[b]);
  }
  if (cudaMalloc(&bt->d_scal, B * sizeof(double*)) != cudaSuccess) return fail(QST_E_NOMEM);
  if (cudaMalloc(&bt->d_losses, B * sizeof(double)) != cudaSuccess) return fail(QST_E_NOMEM);
  if (cudaMallocHost(&bt->h_losses, B * sizeof(double)) != cudaSuccess) return fail(QST_E_NOMEM);
  if (cudaMemcpy(bt->d_scal, scal.data(), B * sizeof(double*), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(QST_E_CUDA);
  *out = bt;
  return QST_OK;
}

qst_ctx* qst_batch_context(qst_batch* bt, int b) {
  if (!bt || b < 0 || b >= bt->B) return nullptr;
  return bt->ctx[b];
}

qst_status qst_batch_set_params(qst_batch* bt, int b, const void* theta) {
  if (!bt || b < 0 || b >= bt->B) return QST_E_INVAL;
  return qst_set_params(bt->ctx[b], theta);
}

qst_status qst_batch_step(qst_batch* bt, const void* const* f, double* losses) {
  if (!bt || !f) return QST_E_INVAL;
  bool steady = true;
  for (int b = 0; b < bt->B; ++b) {
    qst_ctx* c = bt->ctx[b];
    if (!f[b] || !is_device_ptr(f[b])) return QST_E_INVAL;
    if (!c->params_set) return QST_E_STATE;
    if (!c->hidden_valid || c->f_last != f[b]) steady = false;
  }
  if (!steady) {
    // first iteration for these inputs: validate all of them before any tomography steps (a refused call
    // changes nothing), then build each hidden layer (not captured)
    for (int b = 0; b < bt->B; ++b) {
      qst_ctx* c = bt->ctx[b];
      if (c->hidden_valid && c->f_last == f[b]) continue;
      const qst_status st = c->prec == QST_FP64 ? validate_f<double>(c, f[b]) : validate_f<float>(c, f[b]);
      if (st != QST_OK) return st;
    }
    QST_CU(cudaEventRecord(bt->fork, bt->root));
    for (int b = 0; b < bt->B; ++b) {
      qst_ctx* c = bt->ctx[b];
      QST_CU(cudaStreamWaitEvent(c->stream, bt->fork, 0));
      const long long l0 = c->launches;
      const qst_status st = qst_step(c, f[b], nullptr);
      if (st < 0) return st;
      bt->launches += c->launches - l0;
      QST_CU(cudaEventRecord(bt->done[b], c->stream));
      QST_CU(cudaStreamWaitEvent(bt->root, bt->done[b], 0));
    }
  } else {
    bool same = bt->gexec != nullptr && (int)bt->gf.size() == bt->B;
    for (int b = 0; same && b < bt->B; ++b) same = bt->gf[b] == f[b];
    if (!same) {
      const qst_status st = batch_capture(bt, f);
      if (st != QST_OK) return st;
    }
    QST_CU(cudaGraphLaunch(bt->gexec, bt->root));
    bt->launches += bt->gnodes;
    for (int b = 0; b < bt->B; ++b) bt->ctx[b]->iters += 1;
  }
  if (losses) {
    k_gather_losses<<<(bt->B + 255) / 256, 256, 0, bt->root>>>(bt->d_scal, bt->d_losses, bt->B);
    QST_CU(cudaGetLastError());
    QST_CU(cudaMemcpyAsync(bt->h_losses, bt->d_losses, bt->B * sizeof(double), cudaMemcpyDeviceToHost, bt->root));
    QST_CU(cudaStreamSynchronize(bt->root));
    memcpy(losses, bt->h_losses, bt->B * sizeof(double));
  }
  return QST_OK;
}

qst_status qst_batch_reconstruct(qst_batch* bt, const void* const* f, int iters, void* const* rho_out,
                                 double* final_losses) {
  if (!bt || !f || iters < 0) return QST_E_INVAL;
  for (int i = 0; i < iters; ++i) {
    const qst_status st = qst_batch_step(bt, f, nullptr);
    if (st < 0) return st;
  }
  QST_CU(cudaStreamSynchronize(bt->root));
  for (int b = 0; b < bt->B; ++b) {
    if (!rho_out && !final_losses) break;
    const qst_status st = qst_get_rho(bt->ctx[b], f[b], rho_out ? rho_out[b] : nullptr,
                                      final_losses ? final_losses + b : nullptr);
    if (st < 0) return st;
  }
  return QST_OK;
}

long long qst_batch_kernel_launches(const qst_batch* bt) { return bt ? bt->launches : -1; }

qst_status qst_batch_sync(qst_batch* bt) {
  if (!bt) return QST_E_INVAL;
  QST_CU(cudaStreamSynchronize(bt->root));
  return QST_OK;
}

void qst_batch_destroy(qst_batch* bt) {
  if (!bt) return;
  if (bt->root) cudaStreamSynchronize(bt->root);
  if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
  for (qst_ctx* c : bt->ctx)
    if (c) qst_destroy(c);
  for (cudaStream_t s : bt->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : bt->done)
    if (e) cudaEventDestroy(e);
  if (bt->fork) cudaEventDestroy(bt->fork);
  if (bt->d_scal) cudaFree(bt->d_scal);
  if (bt->d_losses) cudaFree(bt->d_losses);
  if (bt->h_losses) cudaFreeHost(bt->h_losses);
  if (bt->d_list) cudaFree(bt->d_list);
  if (bt->d_next) cudaFree(bt->d_next);
  if (bt->fused_done) cudaEventDestroy(bt->fused_done);
  if (bt->fused_stream) cudaStreamDestroy(bt->fused_stream);
  if (bt->d_tab) cudaFree(bt->d_tab);
  if (bt->own_root && bt->root) cudaStreamDestroy(bt->root);
  delete bt;
}

}  // extern "C"
