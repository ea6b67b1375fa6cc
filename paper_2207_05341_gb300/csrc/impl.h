// Internal interface between the C ABI (api.cu) and the kernel files of libqst.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>
#include <vector>

#include "common.cuh"

namespace qst {

// ---- one launch per kernel for a group of tomographies of one size ----
// The launchers of the iteration are called as for a single tomography.  While a recorder is active on
// the calling thread, a batch-aware launcher, just before each kernel launch, either (RECORD) stores the
// kernel's pointer arguments for the tomography being recorded and skips the launch, or (LAUNCH)
// launches the kernel once with grid z = the group and the device table of that launch, whose row z
// holds tomography z's pointers (rebind in common.cuh).  A per-tomography structure (tensor maps) is
// stored as a blob; the table's entry is then the device address of the tomography's copy.
struct BatchRec {
  enum Mode { RECORD = 0, LAUNCH = 1 };
  struct Call {
    int nptr = 0;                       // entries per row (the blob's address first, when there is one)
    size_t blob_bytes = 0;
    std::vector<const void*> ptrs;      // RECORD: count rows of nptr - (blob ? 1 : 0) pointers
    std::vector<unsigned char> blobs;   // RECORD: count blobs
    const void* const* dtab = nullptr;  // LAUNCH: the device table
  };
  int mode = RECORD;
  int count = 0;   // tomographies in the group
  int member = 0;  // RECORD: the tomography being recorded
  int call = 0;    // index of the next kernel launch of the iteration
  bool bad = false;  // the members' launch sequences differ
  std::vector<Call> calls;
};
BatchRec*& batch_rec();  // the calling thread's recorder (NULL: plain launches)
struct BatchArgs {
  const void* const* tab = nullptr;
  unsigned nz = 1;
};
// Before each batch-aware kernel launch: true when the launch is to be skipped (RECORD).
bool batch_take(BatchArgs& ba, std::initializer_list<const void*> ptrs, const void* blob = nullptr,
                size_t blob_bytes = 0);

// Launch with programmatic stream serialisation: the kernel's CTAs may start while the previous kernel
// on the stream drains (its launch and prologue then overlap that tail); the kernel calls
// grid_dep_wait() before its first access to global memory.
template <class... KArgs, class... Args>
cudaError_t launch_dep(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, static_cast<KArgs>(args)...);
}

// Process-wide launch parameters (qst_set_tuning; defaults in tuned.h).
struct Tuning {
  int bulk_chunks_per_cta;  // least 256-column chunks per CTA of a bulk weight pass (fixes its partition)
  int fused_ctas_per_sm;    // resident CTAs per SM of the persistent fused batch launch (1 or 2)
  int fused_max_qubits;     // largest N run as one fused iteration when the context asks for the default
  int batch_concurrent_runs;  // 1: a batch's runs of one size start together, 0: one after another
};
Tuning tuning();
// qst_inject_wait_timeout: true when this launch of `site` is to issue no operand copies (counts it off)
enum InjectSite { INJ_TC_LOADS = 0, INJ_WPASS_LOADS = 1, INJ_SITES = 2 };
bool inject_take(int site);

// Sizes of one N-qubit problem and of the two-pass POVM split.
//   d = 2^N, n = 4^N, H = 2N.
//   The POVM map runs in two passes: the low g qubits inside S x S tiles of the
//   d x d matrix (S = 2^g), then the high h = N - g qubits over an nb x nb grid
//   (nb = 2^h) for chunks of C low outcomes at a time.
struct Dims {
  int N, d, H, g, h, S, nb, C;
  long long n;
  int cnn = 0;  // the App. A CNN head (H = 4N) instead of the 3-layer FNN (H = 2N)
};

Dims make_dims(int N, bool fp64);

// Raise a kernel's dynamic shared-memory limit to `bytes` (cached: one attribute call per size).
cudaError_t ensure_dynamic_smem(const void* fn, size_t bytes);

// Device buffers of a context (all owned by the context).
template <class R> struct Work {
  using V = cx_t<R>;
  R* theta;            // parameters, qst_theta_size(N)
  R* step;             // Rprop state, same layout: step with the previous gradient sign (rprop_encode)
  R* pre;              // hidden pre-activation [H]
  R* hid;              // hidden activation [H]
  R* dpre;             // dL/dpre [H]
  V* T;                // T, d x d complex (SIMT products)
  V* X;                // X = T T (lower tiles written), or rho
  V* G;                // dL/dX, d x d complex
  V* Y;                // G T, d x d complex
  R* Wlo;              // packed low-pass intermediate, n reals
  R* Whi;              // packed adjoint intermediate, n reals
  R* dt;               // dL/dt, n reals
  R* feats;            // CNN: the 640 pooled features, their convolution values and positions
  R* vals;
  int* pos;
  double* cnn_part;    // CNN: per-tile pooling scratch (cnn_part_doubles)
  R* fstage;           // staging copy of a host f, n reals
  R* fperm;            // f in the order of the structured likelihood pass (FP32 fast path), n reals
  double* scal;        // [0] Tr X, [1] sum f, [2] loss, [3] scale of T, [4] scale of G, [5] F_c,
                       // [8..10] state fidelity (sum g, bracket bound, F_q)
  double* partials;    // per-block partial sums
  unsigned int* counters;  // last-block counters, one per reduction site
  unsigned int* flags;     // [0] clamp count, [1] device-side wait timeouts
  // mixed precision operands (BF16 hi / lo planes), NULL when unused
  void* Tb;            // 6 planes of d x d bf16: re_hi, im_hi, nim_hi, re_lo, im_lo, nim_lo
  void* Gb;            // 4 planes of d x d bf16: re_hi, im_hi, re_lo, im_lo
};

// Host helpers of the C ABI entry points (api.cu).
// 0: pageable or unknown host memory, 1: page-locked host memory, 2: device or managed memory.
int ptr_kind(const void* p);
bool is_device_ptr(const void* p);
// Validate a K = 4 POVM of Hermitian 2 x 2 matrices (interleaved complex doubles, element a at
// povm[8a .. 8a+7]) summing to I within 1e-12, and write its Pauli coefficients; returns a
// qst_status (QST_OK or QST_E_INVAL).
int check_povm(const double* povm, int K, PovmB<double>* Bd);

enum Counter {
  CNT_L1 = 0, CNT_T = 1, CNT_NLL = 2, CNT_W2 = 3, CNT_W1 = 4,
  CNT_AMAXT = 8,  // max |re|, |im| of T as float bits: folded in by the producer of t, read by the plane
                  // writer, cleared by the product that reads the planes
  CNT_AMAXG = 9,  // the same for G
  CNT_FID = 10,   // classical fidelity reductions
  CNT_COUNT = 16
};
constexpr int kScaleT = 3;  // scal slot of the power-of-two scale of T (mixed path)
constexpr int kScaleG = 4;  // scal slot of the scale of G
constexpr int kPartialBlocks = 1024;   // max blocks of a reducing kernel
constexpr int kPartialStride = 32;     // doubles per block in `partials` (>= H + 1)

struct NetCfg {
  double slope;
  double eta_minus, eta_plus, step_min, step_max;
};

// ---- POVM map (povm.cu) ----
template <class R> cudaError_t povm_lo_fwd(const Dims& D, const cx_t<R>* X, R* W, const PovmB<R>& B, cudaStream_t s);
template <class R> cudaError_t povm_hi_fwd(const Dims& D, const R* W, R* p, const PovmB<R>& B, cudaStream_t s);
// high-qubit forward, loss and (optionally) high-qubit adjoint; loss -> scal[2]
template <class R> cudaError_t povm_hi_nll(const Dims& D, const R* W, const R* f, double* scal, R* Wadj,
                                           double* partials, unsigned int* counter, unsigned int* flags,
                                           const PovmB<R>& B, bool adjoint, cudaStream_t s);
// amax (may be NULL): the largest |re|, |im| of G is folded into *amax (float bits).
template <class R>
cudaError_t povm_lo_adj(const Dims& D, const R* Wadj, cx_t<R>* G, const PovmB<R>& B, unsigned int* amax,
                        cudaStream_t s);
// Pauli-basis implementations of the high pass (povm_pauli.cu), used when povm_hi_pauli_ok(D)
bool povm_hi_pauli_ok(const Dims& D);
template <class R> cudaError_t povm_hi_fwd_pauli(const Dims& D, const R* W, R* p, const PovmB<R>& B, cudaStream_t s);
template <class R> cudaError_t povm_hi_nll_pauli(const Dims& D, const R* W, const R* f, double* scal, R* Wadj,
                                                 double* partials, unsigned int* counter, unsigned int* flags,
                                                 const PovmB<R>& B, bool adjoint, cudaStream_t s);
// scal[0] = Tr X = sum_i Re X_ii of the computed X (fixed-order FP64 sum)
template <class R> cudaError_t trace_X(const Dims& D, const cx_t<R>* X, double* scal, cudaStream_t s);
// full Hermitian matrix from its lower tiles, scaled by 1 / scal[0] (rho = X / Tr X)
template <class R> cudaError_t hermitian_complete(const Dims& D, const cx_t<R>* Xlow, cx_t<R>* rho,
                                                  const double* scal, cudaStream_t s);

// ---- POVM map for FP32 contexts with g = 6 low qubits and N >= 7 (povm_fast.cu) ----
// A POVM is "structured" when its Pauli coefficients factor as
//   b[a][mu] = beta_mu (-1)^(alpha(a) x_mu + zeta(a) z_mu)   (mu = I, X, Y, Z with (x, z) = (0,0), (1,0),
//                                                              (1,1), (0,1); (alpha, zeta) a bijection)
// i.e. every single-qubit map is a scaling of the Pauli components followed by a Walsh-Hadamard
// transform over (x, z): the tetrahedral POVM of Sec. 4.1 is of this form.
struct PovmPlan {
  PovmB<float> B;      // the generic coefficients b[a][mu]
  int structured;      // 1: beta and out below describe the POVM
  float beta[4];       // beta_mu
  int out[4];          // the outcome a of the canonical slot s = 2 alpha + zeta (identity when generic)
};
PovmPlan make_povm_plan(const PovmB<double>& Bd);
// fast kernels apply: FP32, N in [7, 11] (g = 6, h = N - 6 high qubits)
bool povm_fast_ok(const Dims& D);
// Pass 1 (low qubits) forward: X lower tiles -> packed W (slot layout: XOR diagonals when structured,
// row-major tile pairs otherwise).  Pass 2 (high qubits): the structured path's own kernels, else the
// Pauli-basis kernels of povm_pauli.cu on the row-major layout.
cudaError_t povm_fwd_fast(const Dims& D, const float2* X, float* W, float* p, const PovmPlan& P, cudaStream_t s);
cudaError_t povm_lo_fwd_fast(const Dims& D, const float2* X, float* W, const PovmPlan& P, cudaStream_t s);
// The structured likelihood pass reads f permuted into its own consumption order (povm_permute_f,
// n reals): f is constant while its pointer is, so the copy is made once per new f.
bool povm_needs_fperm(const PovmPlan& P);
cudaError_t povm_permute_f(const Dims& D, const float* f, float* fperm, const PovmPlan& P, cudaStream_t s);
// f: the permuted copy when povm_needs_fperm(P), else f itself
cudaError_t povm_hi_nll_fast(const Dims& D, const float* W, const float* f, double* scal, float* Wadj,
                             double* partials, unsigned int* counter, unsigned int* flags, const PovmPlan& P,
                             bool adjoint, cudaStream_t s);
cudaError_t povm_lo_adj_fast(const Dims& D, const float* Wadj, float2* G, const PovmPlan& P, unsigned int* amax,
                             cudaStream_t s);

// ---- one iteration of a small tomography in one CTA (tomo_fused.cu) ----
// FP32, 3-layer network, Chol_H: t, T, X = T T, the POVM map, likelihood, G, Y = G T, dL/dt, and the
// Rprop updates of both layers with the next hidden layer, for N <= kFusedMaxQubits (H <= 14).
constexpr int kFusedMaxQubits = 7;
struct TomoDesc {
  float* theta;         // parameters and Rprop state (qst_theta_size(N) reals each)
  float* step;
  const float* f;       // frequencies, n reals
  float* pre;           // hidden pre-activation and activation [H], read and replaced by the next ones
  float* hid;
  float* t;             // n reals: t, then dL/dt
  float2 *T, *X, *G, *Y;  // d x d complex scratch
  double* scal;         // [0] Tr X, [1] sum f (read, then rewritten), [2] loss
  unsigned int* flags;  // [0] clamp count
  int N;
};
// max_qubits: the context's option (0: the tuned default, < 0: never)
bool tomo_fused_ok(int N, int max_qubits);
cudaError_t tomo_fused_one(const TomoDesc& td, const PovmB<float>& B, const NetCfg& cfg, cudaStream_t s);
// every tomography of the device array `list` (count entries, largest first is best) in one persistent
// launch; next: a device counter (reset by this call on s)
cudaError_t tomo_fused_list(const TomoDesc* list, int count, const PovmB<float>& B, const NetCfg& cfg,
                            unsigned int* next, cudaStream_t s);

// ---- network (fnn.cu) ----
template <class R> cudaError_t net_l1_forward(const Dims& D, const R* theta, const R* f, R* pre, R* hid,
                                              double* scal, double* partials, unsigned int* counter,
                                              const NetCfg& c, cudaStream_t s);
// t = W2 h + b2 into the scratch t (n reals); then, when T != NULL, the Hermitian T of t (a second
// launch).  amax (may be NULL): max |t_i| (= the largest |re|, |im| of T) is folded into *amax (float bits).
// With Tt != NULL (Chol_Delta) T is the lower-triangular matrix of eq. T_matrix and Tt = T^dag.
template <class R>
cudaError_t net_build_T(const Dims& D, const R* theta, const R* hid, R* t, cx_t<R>* T, unsigned int* amax,
                        cudaStream_t s, cx_t<R>* Tt = nullptr);
// The Hermitian (or, with Tt, lower-triangular) T of an already computed t (second half of net_build_T).
template <class R> cudaError_t net_hermitian_T(const Dims& D, const R* t, cx_t<R>* T, cx_t<R>* Tt, cudaStream_t s);

// ---- the CNN head of App. A (cnn.cu); theta [W2^T (H x n) | b2 | W1 (H x 640) | b1 | conv W (90) | conv b (10)]
size_t cnn_theta_size(int N);
// doubles of the per-tile pooling scratch `part` of cnn_hidden (reals of real_bytes bytes)
size_t cnn_part_doubles(int N, size_t real_bytes);
// features (conv, ReLU, max-pool) and the first dense layer: pre, hid (H = 4N); sum f -> scal[1]; two launches
template <class R>
cudaError_t cnn_hidden(const Dims& D, const R* theta, const R* f, R* feats, int* pos, R* vals, R* pre, R* hid,
                       double slope, double* part, double* partials, unsigned int* counter, double* scal,
                       cudaStream_t s);
// t = W2 h + b2 (amax as for net_build_T)
template <class R>
cudaError_t cnn_output(const Dims& D, const R* theta, const R* hid, R* t, unsigned int* amax, cudaStream_t s);
// backward from dt, with dtheta == NULL Rprop in place on theta / state, else the gradient into dtheta:
// the output layer (dpre out; bulk: FP32 update through two bulk-copy W2 passes, usable when cnn_bulk_ok,
// two launches, else one; a timed-out wait ORs 4 into *flags), then the dense head and the convolution
// (two launches).
bool cnn_bulk_ok(const Dims& D);
template <class R>
cudaError_t cnn_output_backward(const Dims& D, R* theta, R* state, R* dtheta, const R* dt, const R* hid,
                                const R* pre, R* dpre, double* partials, unsigned int* counter, unsigned int* flags,
                                const NetCfg& c, bool bulk, cudaStream_t s);
template <class R>
cudaError_t cnn_head_backward(const Dims& D, R* theta, R* state, R* dtheta, const R* f, const R* feats,
                              const int* pos, const R* vals, const R* dpre, const NetCfg& c, cudaStream_t s);

// Chol_Delta: dL/dt from Z = T G (lower tiles): dR_ii = 2 Re Z_ii, dR_ij = 2 Re Z_ij, dR_ji = 2 Im Z_ij (i > j)
template <class R> cudaError_t net_tri_grad(const Dims& D, const cx_t<R>* Z, R* dt, cudaStream_t s);
template <class R> cudaError_t net_w2_pass(const Dims& D, R* theta, R* step, const R* dt,
                                           const R* hid, const R* pre, R* dpre, R* dtheta,
                                           double* partials, unsigned int* counter, const NetCfg& c,
                                           bool update, cudaStream_t s);
template <class R> cudaError_t net_w1_pass(const Dims& D, R* theta, R* step, const R* f,
                                           const R* dpre, R* pre, R* hid, R* dtheta, double* scal,
                                           double* partials, unsigned int* counter, const NetCfg& c,
                                           bool update, cudaStream_t s);
// FP32 in-place weight passes with bulk-copy staging (fnn_bulk.cu); usable when wpass_bulk_ok(H, n)
// and every streamed array is 16-byte aligned.  flags: a timed-out wait ORs 4 into *flags.
bool wpass_bulk_ok(int H, long long n);
// the W2 pass over `rows` rows of W2^T starting at element rowoff of theta / step, with b2 at ob2 (< 0: b2
// left alone); hid, pre, dpre point at the rows' first hidden unit; only dpre is written (no b1 update)
cudaError_t w2_rows_pass_bulk(long long n, int rows, float* theta, float* step, long long rowoff, long long ob2,
                              const float* dt, const float* hid, const float* pre, float* dpre, double* partials,
                              unsigned int* counter, unsigned int* flags, const NetCfg& c, cudaStream_t s);
cudaError_t w2_pass_bulk(const Dims& D, float* theta, float* step, const float* dt, const float* hid,
                         const float* pre, float* dpre, double* partials, unsigned int* counter, unsigned int* flags,
                         const NetCfg& c, cudaStream_t s);
// layer-1 forward with the same summation partition as w1_pass_bulk
cudaError_t l1_forward_bulk(const Dims& D, const float* theta, const float* f, float* pre, float* hid, double* scal,
                            double* partials, unsigned int* counter, const NetCfg& c, cudaStream_t s);
cudaError_t w1_pass_bulk(const Dims& D, float* theta, float* step, const float* f, float* dpre,
                         float* pre, float* hid, double* scal, double* partials, unsigned int* counter,
                         unsigned int* flags, const NetCfg& c, cudaStream_t s);
// dL/dt from Y = G T:  dR_ij = 2(Re Y_ij + Re Y_ji), dR_ji = 2(Im Y_ij - Im Y_ji) (i > j), dR_ii = 2 Re Y_ii
template <class R> cudaError_t net_symmetrize(const Dims& D, const cx_t<R>* Y, R* dt, cudaStream_t s);

// ---- P-order absolute projection (eigh.cu) ----
template <class R> struct AbsPWork {
  cx_t<R> *A0, *A1, *V0, *V1;  // Jacobi double buffers (matrix, eigenvectors)
  cx_t<R> *W, *Qh;             // scratch, Q^dag
  R *lam, *s, *sp;             // eigenvalues, |lambda|^P, derivative
  cx_t<R> *A, *Q;              // set by abs_p_forward: diagonalised matrix, eigenvectors
  // tensor-core refinement (eigh_tc.cu; QST_MIXED / QST_MIXED_BF16): 16-bit operand planes of Q (4 planes
  // of Q and of Q^dag, 6 planes of Q and of Q^dag), of an intermediate W (4) and of a right operand (6),
  // max slots and scales
  void *qa_n, *qa_h, *qb_n, *qb_h, *wa, *eb;
  unsigned int* amax;          // [0] Q, [1] W, [2] right operand, [3] unresolved size of a refinement
  int* perm;                   // the order of increasing lambda (d) and the unitaries of a block pass
  void* ublk;                  // (d / 64 blocks of 64 x 64 complex)
  double* sc;                  // scales of qa_n, qa_h, qb_n, qb_h, wa, eb; [6] max |lambda|, [7] refinement size
  cx_t<R>* ucos;               // the coset unitaries of a Jacobi pass (16 d complex)
};
// Warm-started refinement of the eigenvectors in w.V0 for the Hermitian T (6 planes Tb with scale *sT) on
// tensor cores, Ogita and Aishima's iteration:
//   R = I - Q^dag Q,  S = Q^dag T Q,  lambda_i = S_ii / (1 - R_ii),
//   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)  (well separated i != j),  E_ij = R_ij / 2 otherwise,
//   Q <- Q + Q E.
// abs_p_tc_correction: lambda, |lambda|^P and its derivative, and E (in w.W, max |E| in w.amax[2], and in
// amax[3] max |S_ij| / max |lambda| over the separated pairs too far apart for a first-order correction);
// abs_p_tc_update: Q <- Q + Q E; abs_p_tc_finish: X = Q |Lambda|^P Q^dag (lower tiles) and Q^dag.
// A timed-out wait of a product ORs into *err.
cudaError_t abs_p_tc_correction(int d, const void* Tb, const double* sT, AbsPWork<float>& w, double P, int fmt,
                                unsigned int* err, cudaStream_t s);
cudaError_t abs_p_tc_update(int d, AbsPWork<float>& w, int fmt, unsigned int* err, cudaStream_t s);
// The couplings a first-order correction cannot resolve (near-degenerate pairs): Q's columns sorted by
// the latest lambda, then two passes of exact Jacobi diagonalisations of 64 x 64 diagonal blocks of
// S = Q^dag T Q (the second shifted by 32), each block's unitary applied to Q's columns.  Synchronises.
cudaError_t abs_p_tc_block_phase(int d, const void* Tb, const double* sT, AbsPWork<float>& w, int fmt,
                                 unsigned int* err, cudaStream_t s);
cudaError_t abs_p_tc_finish(int d, AbsPWork<float>& w, int fmt, float2* X, unsigned int* err, cudaStream_t s);
// The backward of abs_p_forward (either form) with the products on tensor cores: Y with Y + Y^dag = dL/dT.
cudaError_t abs_p_backward_tc(int d, const float2* G, AbsPWork<float>& w, int fmt, float2* Y, unsigned int* err,
                              cudaStream_t s);
size_t abs_p_tc_plane_bytes(int d);  // bytes of one 4-plane buffer (a 6-plane one is 1.5 times that)
// One sweep of the Jacobi eigensolver for d = 2^N in the XOR ordering (round m rotates the pairs {x, x ^ m},
// m = 1 .. d - 1), as passes: each pass applies the 2^k - 1 rounds of one k-dimensional subspace of GF(2)^N
// (they act within its cosets of 2^k indices), k = 1 .. 4.  basis[0 .. k) is the subspace's basis in reduced
// form: piv[i] = top bit of basis[i], ascending, and bit piv[i] clear in every other basis vector; local
// index j of a coset stands for rep ^ (XOR of basis[i] over the bits i of j), rep having the pivot bits clear.
struct JacobiPass {
  int k;
  int basis[4];
  int piv[4];
};
const std::vector<JacobiPass>& jacobi_schedule(int N);  // 1 <= N <= 14
long long jacobi_passes_per_sweep(int d);
long long jacobi_kernels_per_sweep(int d);  // a pass over cosets of 8 or 16 indices is two kernels
// A warm-started step of the mixed path on the Jacobi sweeps: A0 = Q^dag T Q (Q in V0, T as its 6 planes Tb
// with scale *sT) and X = Q |Lambda|^P Q^dag (lower tiles) on tensor cores, `sweeps` (even) sweeps between;
// leaves Q in V0 and Q^dag in Qh, as abs_p_forward does.
cudaError_t abs_p_forward_tc_warm(int d, const void* Tb, const double* sT, AbsPWork<float>& w, int sweeps, double P,
                                  int fmt, float2* X, unsigned int* err, cudaStream_t s);
// X = Q |Lambda|^P Q^dag (lower tiles) from T via `sweeps` (even) Jacobi sweeps; warm == true starts
// from the previous eigenvectors (V0, with Q^dag in Qh).  Leaves Q in V0 and Q^dag in Qh.
template <class R> cudaError_t abs_p_forward(int d, const cx_t<R>* T, AbsPWork<R>& w, int sweeps, bool warm,
                                             double P, cx_t<R>* X, cudaStream_t s);
// Eigenvalues of Hermitian T (lam, s = |lam|^P, into w) and phi = Q^dag psi (d complex) from `sweeps` cold
// Jacobi sweeps that rotate the vector instead of accumulating Q: only w.A0, w.A1, w.lam, w.s, w.sp are used.
template <class R> cudaError_t jacobi_values_project(int d, const cx_t<R>* T, AbsPWork<R>& w, int sweeps, double P,
                                                     const cx_t<R>* psi, cx_t<R>* phi, cudaStream_t s);
// After restoring Q into V0 (checkpoint), recompute Q^dag.
template <class R> cudaError_t abs_p_restore_q(int d, AbsPWork<R>& w, cudaStream_t s);
// Y with Y + Y^dag = dL/dT = Q (D o (Q^dag G Q)) Q^dag, from G = dL/dX
template <class R> cudaError_t abs_p_backward(int d, const cx_t<R>* G, AbsPWork<R>& w, cx_t<R>* Y, cudaStream_t s);

// ---- quantum state fidelity (fidelity_q.cu) ----
// F_q (Sec. 2.3 eq. F_QF via eq. fq_decom) between rho^ = Q diag(g) Q^dag / sum g (Qh = Q^dag, d x d;
// g >= 0, d) and w |psi><psi| / <psi|psi> + (1 - w) I / d; scratch: state_fidelity_scratch_doubles(d);
// out[0] = sum g, out[1] = bracket bound, out[2] = F_q.  d a power of two up to 4096.
// The same from phi = Q^dag psi already formed (Qh == NULL, phi given) instead of Qh.
size_t state_fidelity_scratch_doubles(int d);
template <class R>
cudaError_t state_fidelity_from_decomposition(int d, const cx_t<R>* Qh, const cx_t<R>* phi, const R* g,
                                              const cx_t<R>* psi, double w, double* scratch, double* out,
                                              unsigned int* counter, cudaStream_t s);

// ---- complex products (gemm_simt.cu) ----
// C = A B for d x d complex row-major matrices; lower == true computes only tiles I >= J.
template <class R> cudaError_t cgemm_simt(int d, const cx_t<R>* A, const cx_t<R>* B, cx_t<R>* C, bool lower,
                                          cudaStream_t s);

// ---- tensor-core products (gemm_tc.cu) ----
enum TcFormat { TC_FP16_SCALED = 0, TC_BF16 = 1 };
// 16-bit hi / lo operand planes of T (6 planes: re, im, -im; hi then lo), made straight from t (T is the
// Hermitian matrix of t, as in net_build_T), and of G (4 planes: re, im; hi then lo).  TC_FP16_SCALED first
// scales by the power of two (written to scal[kScaleT] / scal[kScaleG]) that brings *amax, the largest
// magnitude folded in by the producer of t or G, into [1, 2).
cudaError_t tc_planes_T(int d, const float* t, void* Tb, int fmt, double* scal, const unsigned int* amax,
                        cudaStream_t s);
cudaError_t tc_split_G(int d, const float2* G, void* Gb, int fmt, double* scal, const unsigned int* amax,
                       cudaStream_t s);
// X = T T (lower 128 x 128 tiles) and Y = G T (full) on tcgen05, complex FP32 out (unscaled);
// a device-side wait that runs out sets *err != 0.  clear (may be NULL) is zeroed by the kernel: the max
// slot of the operand planes it reads, ready for the next producer.
cudaError_t tc_herm_square(int d, const void* Tb, int fmt, const double* scal, float2* X, unsigned int* err,
                           unsigned int* clear, cudaStream_t s);
cudaError_t tc_gt_product(int d, const void* Gb, const void* Tb, int fmt, const double* scal, float2* Y,
                          unsigned int* err, unsigned int* clear, cudaStream_t s);
bool tc_available();
// General products on the same kernel: C = A B (lower: 128 x 128 tiles I >= J only) from the 4 planes of A
// (re, im; hi then lo) and the 6 planes of B^dag (re, im, -im; hi then lo), with their scales sA, sB.
cudaError_t tc_product(int d, const void* Ab, const void* Bb, int fmt, const double* sA, const double* sB, float2* C,
                       bool lower, unsigned int* err, cudaStream_t s);
// Planes of op(M) (op 0: M, 1: M^dag), nplanes 4 or 6 as above, scaled by the power of two that brings *amax
// into [1, 2) (TC_FP16_SCALED; 1 for TC_BF16), the scale written to *s_slot.  d a multiple of 32.
cudaError_t tc_planes_op(int d, const float2* M, int op, int nplanes, void* P, int fmt, const unsigned int* amax,
                         double* s_slot, cudaStream_t s);
// *amax = the largest |re|, |im| of n complex entries (float bits; the slot is cleared first)
cudaError_t absmax_to(long long n, const float2* M, unsigned int* amax, cudaStream_t s);

// ---- synthetic data on the GPU (sampler.cu) ----
// rho = w |psi><psi| + (1 - w) I / d for the test state `kind` (QST_STATE_*), d x d complex.
template <class R> cudaError_t make_test_state(int N, int kind, double w, cx_t<R>* rho, cudaStream_t s);
// Multinomial counts: prepare (integer weights of P and their exact running sum into scratch of
// sampler_scratch_words(n) words, counts zeroed, *bad |= 1 for a probability that is not in [0, 1]);
// the total weight is scratch[n - 1]; then draw `shots` outcomes into counts.
long long sampler_scratch_words(long long n);
cudaError_t multinomial_prepare(long long n, const double* P, unsigned long long* scratch, long long* counts,
                                unsigned int* bad, cudaStream_t s);
cudaError_t multinomial_draw(long long n, long long shots, unsigned long long seed, const unsigned long long* scratch,
                             long long* counts, cudaStream_t s);
template <class R> cudaError_t counts_to_frequencies(long long n, const long long* counts, long long shots, R* f,
                                                     cudaStream_t s);

// ---- classical fidelity (fidelity.cu) ----
// eq. F_CF from q (unnormalised Born probabilities of X, Tr X in scal[0]) and a target P: (sum sqrt(q P / Tr X))^2
// -> *out (device).  Sampled (eq. fc_sample): needs cdf with fidelity_cdf_len(n) doubles of scratch.
long long fidelity_cdf_len(long long n);
template <class R>
cudaError_t classical_fidelity_exact(long long n, const R* q, const R* P, const double* scal, double* partials,
                                     unsigned int* counter, double* out, cudaStream_t s);
template <class R>
cudaError_t classical_fidelity_sampled(long long n, const R* q, const R* P, long long samples,
                                       unsigned long long seed, const double* scal, double* cdf, double* partials,
                                       unsigned int* counter, double* out, cudaStream_t s);
// cuTensorMapEncodeTiled from the driver (NULL when unavailable).
void* tma_encoder();

}  // namespace qst
