/*
 * qst.h -- C ABI of the GB300 NN-QST maximum-likelihood library (libqst.so).
 *
 * Method: Wang, Cheng, Li, Chen, "Ultrafast quantum state tomography with
 * feed-forward neural networks" (arXiv:2207.05341).  The library runs the
 * per-iteration hot path of that method on one GPU:
 *
 *   Sec. 3.1   network  f (4^N) -> LeakyReLU hidden (2N) -> linear output t (4^N)
 *   Sec. 3.2   t -> Hermitian T -> X = T^dag T = T T ("Chol_H", eq. unified_DP),
 *              rho = X / Tr X
 *   Sec. 3.3   q_k = Tr[(M_k1 (x) ... (x) M_kN) X]  (product POVM, eq. PS), p = q / Tr X
 *   Sec. 3.1   L = -sum_k f_k log p_k   (eq. MLE objective)
 *   backward through all of the above, then Rprop (Sec. 4.1).
 *
 * Conventions shared by every call
 *   N         number of qubits, 1 <= N <= 12 (FP32 / MIXED), 1 <= N <= 10 (FP64).
 *   d = 2^N, n = 4^N, H = 2N.
 *   Outcome index k = sum_q a_q 4^(N-q): qubit 1 is the most significant base-4
 *   digit and the most significant Kronecker factor (row/column bit N-1).
 *   real      double for QST_FP64 contexts, float for QST_FP32 / QST_MIXED.
 *   complex   two interleaved reals (re, im); matrices are d x d row-major.
 *   theta     flat array of qst_theta_size(N) reals:
 *               [ W1 (H x n, row-major) | W2^T (H x n, row-major) | b2 (n) | b1 (H) ]
 *             layer 1: pre = W1 f + b1, h = LeakyReLU(pre);
 *             layer 2: t_i = sum_j W2^T[j][i] h_j + b2_i.
 *   T from t  R = t as a d x d row-major matrix; T_ii = R_ii,
 *             T_ij = R_ij + i R_ji for i > j, T_ji = conj(T_ij).
 *
 * Memory and ownership
 *   The caller owns every pointer it passes.  A pointer documented "device or
 *   host" may be either; host buffers are staged through context memory.  A
 *   qst_ctx owns its network parameters, Rprop state and scratch buffers and
 *   frees them in qst_destroy.  All work is ordered on the stream given to
 *   qst_init (NULL = the legacy default stream).  A call returns once its work
 *   is enqueued, except that writing a host scalar (loss) or a host buffer
 *   synchronises the stream first.
 *
 * Errors
 *   Every call returns a qst_status; nothing is thrown across the ABI.  A
 *   negative status means the call did nothing observable (or, for QST_E_CUDA,
 *   that a CUDA call failed and the context should be destroyed).
 *   QST_W_CLAMP (positive) is a warning: some q_k below q_min (the smallest
 *   normal number of the precision; for the positive semidefinite X of the
 *   state maps only rounding brings q_k to 0 or below) had f_k > 0.  Such a
 *   term is clamped: it adds the constant -f_k log q_min to the loss and
 *   nothing to its gradient; the results are otherwise complete.
 */
#ifndef QST_H
#define QST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qst_ctx qst_ctx;

typedef enum {
    QST_OK = 0,
    QST_E_INVAL = -1,       /* bad argument: N out of range, NULL pointer, K != 4, POVM not summing to I */
    QST_E_INPUT = -2,       /* bad data: f not finite, negative, or not summing to 1 within 1e-4 */
    QST_E_NOMEM = -3,       /* device allocation failed */
    QST_E_CUDA = -4,        /* a CUDA runtime call failed */
    QST_E_TIMEOUT = -5,     /* a bounded device-side wait ran out */
    QST_E_STATE = -6,       /* call not valid in the context's state (e.g. no parameters set) */
    QST_E_UNSUPPORTED = -7, /* valid request this build does not run (e.g. precision not compiled) */
    QST_W_CLAMP = 1
} qst_status;

/* State maps of Sec. 3.2.  QST_MAP_ABS_P (eq. abs_P, any P > 0) diagonalises T every
 * iteration with a cyclic Jacobi method on the GPU.  QST_MAP_CHOL_DELTA is the Cholesky
 * decomposition of Sec. 2.2.1 (eq. T_matrix): T is complex lower triangular (T_ii = R_ii,
 * T_ij = R_ij + i R_ji for i > j, 0 above the diagonal, from the same R = reshape(t)) and
 * rho = T^dag T / Tr(T^dag T).  The mixed modes support QST_MAP_CHOL_H only
 * (QST_E_UNSUPPORTED otherwise). */
enum { QST_MAP_CHOL_H = 0, QST_MAP_ABS_P = 1, QST_MAP_CHOL_DELTA = 2 };
/* Precisions.  QST_MIXED runs the two complex d x d products on tensor cores
 * (tcgen05) with each FP32 operand split into FP16 hi + lo after a power-of-two
 * scaling (about 2^-21 relative error); QST_MIXED_BF16 uses a BF16 hi + lo split
 * without scaling (about 2^-16).  Everything else stays FP32 in both.  Mixed
 * modes need N >= 7 (d a multiple of 128). */
enum { QST_FP64 = 0, QST_FP32 = 1, QST_MIXED = 2, QST_MIXED_BF16 = 3 };

typedef struct qst_options {
    int mapping;        /* QST_MAP_CHOL_H (paper default, Sec. 4.3), QST_MAP_ABS_P (eq. abs_P) or
                           QST_MAP_CHOL_DELTA (eq. T_matrix) */
    int precision;      /* QST_FP64, QST_FP32, QST_MIXED or QST_MIXED_BF16 (see above) */
    double P;           /* order of the absolute projection A_P; used when mapping == QST_MAP_ABS_P */
    double lr;          /* Rprop initial step (Sec. 4.1: 0.001); lr, step_min and step_max must lie in
                           [2^-33, 2^30] (QST_E_INVAL otherwise): the library keeps each parameter's
                           step and previous gradient sign in one word, exactly, within that range */
    double eta_minus;   /* Rprop shrink factor (0.5) */
    double eta_plus;    /* Rprop growth factor (1.2) */
    double step_min;    /* Rprop step lower bound (1e-6) */
    double step_max;    /* Rprop step upper bound (50) */
    double leaky_slope; /* LeakyReLU negative slope (0.01) */
    int eig_sweeps;     /* QST_MAP_ABS_P: Jacobi sweeps from a cold start (0 = default 12; rounded up
                           to even) */
    int eig_warm_sweeps;/* QST_MAP_ABS_P: sweeps when qst_step starts from the previous iteration's
                           eigenvectors (0 = default 2; -1 = always cold; rounded up to even) */
    int network;        /* QST_NET_FNN (Sec. 3.1, default) or QST_NET_CNN (App. A, N >= 3) */
    size_t device_memory_limit; /* bytes of device memory the context may hold (parameters, Rprop state,
                           scratch, and the scratch some calls allocate on first use); 0 = no limit.  An
                           allocation that would exceed it fails with QST_E_NOMEM before cudaMalloc is
                           called, and qst_init then frees what it had allocated. */
    int fused_max_qubits; /* FP32 contexts of the 3-layer network with QST_MAP_CHOL_H and N at most this
                           run each qst_step iteration (and their share of a batch iteration) as one
                           kernel on one CTA (QST_PH_FUSED); 0 = qst_tuning.fused_max_qubits, -1 =
                           never; at most 7.  The result is the same method, summed in another order. */
    int eig_refine;     /* QST_MAP_ABS_P with QST_MIXED / QST_MIXED_BF16: 1 (default) = a warm-started step
                           first refines the previous eigenvectors on tensor cores (qst_eig_counts); 0 = warm
                           steps go to the Jacobi sweeps directly (their products on tensor cores) */
} qst_options;

/* Mapping networks.  QST_NET_FNN: the 3-layer network of Sec. 3.1, theta as described above.
 * QST_NET_CNN: the convolutional network of App. A: f as a 2^N x 2^N matrix (row-major), a 3 x 3
 * convolution (stride 1, zero padding 1, 10 maps with bias), ReLU, max-pooling over 2^(N-3)-square
 * windows (640 features), a dense layer to 4N units (LeakyReLU), a dense linear layer to 4^N outputs.
 * Its theta (qst_theta_size_net(N, QST_NET_CNN) reals) is
 *   [W2^T (4N x 4^N) | b2 (4^N) | W1 (4N x 640) | b1 (4N) | conv W (10 x 3 x 3) | conv b (10)],
 * features ordered (map, window row, window column); on pooling ties the first row-major position of
 * the window is taken. */
enum { QST_NET_FNN = 0, QST_NET_CNN = 1 };

/* Fill *opt with the paper's settings (Sec. 4.1) and the defaults stated above. */
void qst_default_options(qst_options* opt);

/* Number of reals in theta for N qubits: 2*H*n + n + H. */
size_t qst_theta_size(int N);

/* Number of reals in theta for N qubits and mapping network `network` (0 when unsupported). */
size_t qst_theta_size_net(int N, int network);

/* Create a context for N qubits.
 *   povm   host, K*2*2 complex doubles (interleaved re, im), element a at
 *          povm[8a .. 8a+7] as the row-major 2x2 matrix M_a.  K must be 4; the
 *          M_a must be Hermitian and sum to the identity within 1e-12
 *          (Sec. 2.1 eq. qst; Sec. 3.3 uses the same M_a on every qubit).
 *   opt    host, may be NULL for qst_default_options.
 *   stream cudaStream_t (as void*), may be NULL.
 * Allocates all device memory the context needs (QST_E_NOMEM on failure). */
qst_status qst_init(qst_ctx** out, int N, const double* povm, int K,
                    const qst_options* opt, void* stream);

/* Load network parameters (theta layout above, qst_theta_size(N) reals, device
 * or host) and reset the Rprop state (steps = lr, previous signs = 0). */
qst_status qst_set_params(qst_ctx* ctx, const void* theta);

/* Copy the current parameters out (device or host buffer of qst_theta_size(N) reals). */
qst_status qst_get_params(qst_ctx* ctx, void* theta);

/* Sec. 3.3 eq. PS: p_k = Tr[(M_k1 (x) ... (x) M_kN) rho] for all k.
 *   rho  device, d x d complex, row-major.  Only the lower triangle (i >= j) is
 *        read; the upper triangle is taken to be its conjugate transpose.
 *   p    device, n reals (written).  No normalisation is applied. */
qst_status qst_probs(qst_ctx* ctx, const void* rho, void* p);

/* Allocation-free variant of qst_probs, for callers that cannot call cudaMalloc
 * (a framework whose own pool allocator owns the device memory, a latency-bound
 * loop that must avoid the synchronisation allocation can cause, or a one-off
 * evaluation without a context, which qst_init would allocate).  The paper has
 * no counterpart; this is an interface convenience.
 *   N       1 <= N <= 10 (larger N returns QST_E_INVAL): the packed intermediate
 *           lives in a fixed 4 MiB device array (4^10 floats) inside libqst,
 *           which every GPU that loads the library holds until the process exits.
 *   povm    as for qst_init (host, K = 4, Hermitian, summing to I).
 *   rho, p  device, FP32: d x d complex rho (lower triangle read, as qst_probs)
 *           and n reals written.  Host memory is refused (QST_E_INVAL) before
 *           anything is launched.
 *   stream  cudaStream_t (as void*), may be NULL.
 * The first call on a device looks up the array's device address (set-up, once
 * per device, with that device current); make that first call before any
 * stream capture.  All calls share the one array: calls whose work overlaps on
 * the GPU (different streams, or different host threads on one device) race
 * and must be serialised by the caller.  The array keeps the previous call's
 * contents; every entry a call reads is first written by the same call, so
 * nothing needs clearing.  Calls no cudaMalloc, cudaFree or allocating
 * library routine. */
qst_status qst_probs_static(int N, const double* povm, int K, const void* rho, void* p, void* stream);

/* Loss and gradient of Sec. 3.1 for externally held parameters, no update.
 *   theta  device, qst_theta_size(N) reals (read only).
 *   f      device or host, n reals: measured frequencies (Sec. 2.1), f >= 0, sum 1.
 *   loss   host, written: L = -sum_k f_k log p_k (terms with f_k = 0 omitted).
 *   dtheta device, qst_theta_size(N) reals (written): dL/dtheta in theta's layout. */
qst_status qst_loss_grad(qst_ctx* ctx, const void* theta, const void* f, double* loss, void* dtheta);

/* One iteration of the Fig. 1 loop on the context's parameters: forward, loss,
 * backward, Rprop update.
 *   f     device or host, n reals.  The hidden layer of the next iteration is
 *         computed inside this call from this f; passing a different pointer
 *         to the next call recomputes it, passing the same pointer assumes the
 *         values did not change.
 *   loss  host or NULL: loss of the parameters before the update (synchronises). */
qst_status qst_step(qst_ctx* ctx, const void* f, double* loss);

/* Run `iters` iterations of qst_step, then write the reconstructed state.
 *   rho_out     device or host or NULL, d x d complex: rho of the final parameters.
 *   final_loss  host or NULL: loss of that rho. */
qst_status qst_reconstruct(qst_ctx* ctx, const void* f, int iters, void* rho_out, double* final_loss);

/* rho of the current parameters for input f (device or host), written to rho_out
 * (device or host, d x d complex), and its loss if loss != NULL. */
qst_status qst_get_rho(qst_ctx* ctx, const void* f, void* rho_out, double* loss);

/* Classical fidelity of Sec. 2.3 between rho^ of the current parameters (network input f, device or
 * host, n reals) and a target distribution P (device or host, n reals, P_k = Tr[M_k rho] of the
 * target state), computed on the GPU:
 *   samples == 0: eq. F_CF, F_c = (sum_k sqrt(P^_k P_k))^2 (an upper bound on the state fidelity);
 *   samples  > 0: eq. fc_sample, (mean_s sqrt(P_{k_s} / P^_{k_s}))^2 over `samples` draws k_s ~ P^:
 *                 u_s = (splitmix64(seed, s) >> 11) 2^-53 (SplitMix64, Steele, Lea and Flood 2014:
 *                 x = seed + (s + 1) 0x9E3779B97F4A7C15, then its published mix) and k_s is the
 *                 smallest k whose running sum of max(P^, 0) exceeds u_s times the total.
 * P^_k are the Born probabilities of X / Tr X (Sec. 3.3).  Fc: host, written.  The first sampled
 * call allocates (n + n / 2048) doubles of scratch for the running sum. */
qst_status qst_classical_fidelity(qst_ctx* ctx, const void* f, const void* P, long long samples,
                                  unsigned long long seed, double* Fc);

/* Quantum (state) fidelity of Sec. 2.3 eq. F_QF between rho^ of the current parameters (network input
 * f, device or host, n reals) and the target rho = w |psi><psi| / <psi|psi> + (1 - w) I / d of the Sec. 4
 * sweeps (pure: w = 1; white noise of strength p: w = p; depolarising channel lambda: w = 1 - lambda),
 * computed on the GPU by the decomposition route of eq. fq_decom.  The decomposition of rho^ comes from
 * that of T (Sec. 3.2: T = Q Lambda Q^dag, rho^ = Q g(Lambda) Q^dag / Tr g(Lambda), g = lambda^2 for
 * Chol_H, |lambda|^P for A_P): for Chol_H a cold Jacobi run of `sweeps` sweeps (0: 12; rounded up to
 * even), for A_P the decomposition of the forward pass.  The eigenvalues of sqrt(rho^) rho sqrt(rho^)
 * (diagonal plus rank one in the basis Q) are the roots of its secular equation, found by bisection in
 * FP64; F_q = (sum sqrt(eigenvalue))^2.
 *   psi  device or host, d complex of the context precision (interleaved re, im), not all zero;
 *   w    in [0, 1];  Fq  host, written.
 * For Chol_H the sweeps rotate psi along (phi = Q^dag psi) instead of forming Q.
 * QST_E_UNSUPPORTED for Chol_Delta contexts.  The first call of a Chol_H context allocates the
 * eigensolver's workspace (2 d x d complex); no call allocates anything after the first. */
qst_status qst_state_fidelity(qst_ctx* ctx, const void* f, const void* psi, double w, int sweeps, double* Fq);

/* ---- synthetic data on the GPU (Sec. 4: the test states of the sweeps, multinomial sampling) ---- */
enum { QST_STATE_PRODUCT = 0,  /* ((|0> + |1>) / sqrt 2)^N */
       QST_STATE_GHZI = 1,     /* (|0...0> + i |1...1>) / sqrt 2 */
       QST_STATE_W = 2 };      /* equal superposition of the N one-excitation basis states */

/* rho = w |psi><psi| + (1 - w) I / d for the state `kind`, with w in [0, 1]: white noise of strength p
 * is w = p, the depolarising channel with lambda is w = 1 - lambda.  rho: device, d x d complex of the
 * context's precision (complex64, or complex128 for QST_FP64), row-major, written. */
qst_status qst_test_state(qst_ctx* ctx, int kind, double w, void* rho);

/* Seeded multinomial counts of `shots` draws from P (device, n = 4^N doubles, each in [0, 1]; need not
 * sum to 1 exactly).  Each P_k becomes the integer weight floor(P_k 2^52); shot s draws
 * t_s = floor((splitmix64(seed, s) >> 11) W / 2^53) (W = total weight; SplitMix64 as in
 * qst_classical_fidelity) and counts outcome k_s = the smallest k whose running weight exceeds t_s.
 * All integer arithmetic: the counts are exact and reproducible.  counts: device, n int64, written;
 * f: device or NULL, n reals of the context precision, written with counts / shots.  QST_E_INPUT for a
 * P that is not finite, above 1, or all zero.  The first call allocates (n + n / 2048) words of scratch. */
qst_status qst_sample_counts(qst_ctx* ctx, const double* P, long long shots, unsigned long long seed,
                             long long* counts, void* f);

/* Checkpoint of parameters, Rprop state and iteration count (and, for
 * QST_MAP_ABS_P, the eigenvectors that warm-start the next eigendecomposition),
 * as an opaque host byte buffer of qst_state_bytes(ctx) bytes.  Restoring it
 * into a context with the same N, precision and options resumes bit-identically. */
size_t qst_state_bytes(const qst_ctx* ctx);
qst_status qst_get_state(qst_ctx* ctx, void* host_buf, size_t bytes);
qst_status qst_set_state(qst_ctx* ctx, const void* host_buf, size_t bytes);

/* Number of Rprop steps taken since the last qst_set_params / qst_set_state. */
long long qst_iterations(const qst_ctx* ctx);

/* QST_MAP_ABS_P with QST_MIXED / QST_MIXED_BF16 (instrumentation): a warm-started step refines the
 * previous eigenvectors on tensor cores (Ogita and Aishima's iteration; couplings of near-degenerate
 * pairs that a first-order correction leaves unresolved go to exact Jacobi diagonalisations of 64 x 64
 * blocks of neighbours in the order of the eigenvalues), up to 6 refinements until the largest
 * correction is at most 5e-3 with no coupling above 1e-5 max |lambda| unresolved, and hands the step to
 * Jacobi sweeps from the previous eigenvectors otherwise; after such a step the next 15 warm steps go to
 * the sweeps directly.  Counts since qst_init: refinements taken, and steps handed to the sweeps; last
 * (2 doubles, may be NULL): the latest refinement's largest correction and its largest unresolved
 * coupling relative to max |lambda|. */
qst_status qst_eig_counts(const qst_ctx* ctx, long long* refinements, long long* fallbacks, double* last);

/* The ordering of the Jacobi eigensolver behind QST_MAP_ABS_P and qst_state_fidelity (Sec. 3.2,
 * eq. abs_P; inspection only, no GPU needed): for d = 2^N, round m of a sweep rotates the index pairs
 * {x, x ^ m}, m = 1 .. d - 1, and each pass applies the 2^k - 1 rounds of one k-dimensional subspace of
 * GF(2)^N (its nonzero elements; they act within the subspace's cosets of 2^k indices), k = 1 .. 4: a
 * partition of GF(2)^N \ {0} into such subspaces is one sweep.  count = passes per sweep; for the first
 * min(count, cap) passes, dims[p] = k and basis[4 p .. 4 p + k) the subspace's basis in reduced form (top
 * bits distinct and ascending, each top bit clear in the other vectors; unused entries 0).  Host arrays;
 * may be NULL when cap == 0.  QST_E_INVAL for N outside 1..12 or NULL arrays with cap > 0. */
qst_status qst_jacobi_schedule(int N, int* count, int* dims, int* basis, int cap);

/* Number of kernel launches the library has enqueued on this context (graph
 * replays count every kernel node). */
long long qst_kernel_launches(const qst_ctx* ctx);

/* Per-phase timing of qst_step (instrumentation; the paper has no counterpart).
 * With timing enabled, every qst_step records a CUDA event on the context's
 * stream after each phase below; qst_timing_read synchronises, adds the
 * elapsed times per phase over all steps recorded since the last read, writes
 * the totals (milliseconds) and step counts, and starts a new window.
 * max_steps bounds the window (extra steps are not recorded); 0 disables.
 * With qst_graph_enable on, the events are nodes of the captured graph and
 * qst_timing_read returns the phases of the latest replay only (one step). */
enum {
    QST_PH_HIDDEN = 0,   /* layer-1 forward (only when the input changed) */
    QST_PH_BUILD_T = 1,  /* layer 2 + Hermitian T (+ Tr T^2) */
    QST_PH_XFWD = 2,     /* X = T T */
    QST_PH_POVM_LO = 3,  /* POVM map, low qubits */
    QST_PH_POVM_HI = 4,  /* POVM map high qubits + likelihood + adjoint high qubits */
    QST_PH_POVM_ADJ = 5, /* adjoint low qubits -> G */
    QST_PH_GT = 6,       /* Y = G T (incl. operand conversion) */
    QST_PH_SYM = 7,      /* dL/dt from Y */
    QST_PH_W2 = 8,       /* layer-2 backward + Rprop */
    QST_PH_W1 = 9,       /* layer-1 backward + Rprop + next hidden layer */
    QST_PH_FUSED = 10,   /* the whole iteration as one kernel (qst_options.fused_max_qubits): the
                            phases 1-9 are then not recorded */
    QST_NPHASE = 11
};
qst_status qst_timing_enable(qst_ctx* ctx, int max_steps);
qst_status qst_timing_read(qst_ctx* ctx, double* phase_ms, long long* phase_count, int nphase);

/* Capture the steady-state iteration of qst_step into a CUDA graph and replay it
 * (enable != 0), or go back to launching kernel by kernel (0).  Needs a context
 * created with a non-NULL stream (QST_E_UNSUPPORTED otherwise).  The graph is
 * captured on the first qst_step whose input f was also given to the previous
 * step (the hidden layer is then known) and is re-captured when f's pointer
 * changes.  f may be device memory or page-locked host memory (then a copy node
 * of the graph stages it on every replay, on a side stream beside the kernels that
 * come before the first read of f; the context owns that stream); pageable host
 * inputs use the launch-by-launch path.  A replay has no host work between kernels.
 * Instrumentation of the library, not part of the method. */
qst_status qst_graph_enable(qst_ctx* ctx, int enable);

/* Launch parameters of the library, process-wide (instrumentation of the library, not part of the
 * method; the shipped defaults were chosen by the package's autotuner on the target GPU).
 *   bulk_chunks_per_cta  least number of 256-column chunks that one CTA of an FP32 weight pass (and of
 *                        the layer-1 forward that shares its partition) streams, >= 1; the grid is at
 *                        most one CTA per SM.  It fixes how the passes' sums over 4^N terms are split,
 *                        so results change in the last bits with it.
 *   fused_ctas_per_sm    resident CTAs per SM of the persistent launch of a batch's fused tomographies
 *                        (1 or 2); results do not depend on it.
 *   fused_max_qubits     the limit qst_options.fused_max_qubits = 0 stands for (0..7; 0 = never).
 *   batch_concurrent_runs 1: the runs of one qubit count of a batch iteration start together (their
 *                        kernels share the GPU), 0: one after another, largest first; results do not
 *                        depend on it.
 * Set them between iterations, with no call of the library running on another thread; a batch captured
 * earlier keeps the values it was captured with until its inputs change.  QST_E_INVAL for values out of
 * range (nothing changed). */
/* Testing hook for the device-side wait limits; it involves no GPU fault.  With what =
 * QST_INJECT_TC_LOADS the next `count` launches of the tensor-core products (QST_MIXED, QST_MIXED_BF16),
 * with QST_INJECT_WPASS_LOADS the next `count` launches of the FP32 bulk weight passes, issue none of
 * their operand copies: the waits for those copies run out after their limit (about 2 s), the kernels
 * leave their results unwritten and return, and the call that reads the loss (qst_step, qst_loss_grad,
 * qst_reconstruct) returns QST_E_TIMEOUT; the context stays usable (reload its parameters with
 * qst_set_params: the failed step may have updated some of them).  count = 0 clears.  Process-wide;
 * steps replayed from a captured graph are not affected.  QST_E_INVAL for an unknown `what` or
 * count < 0. */
enum { QST_INJECT_TC_LOADS = 1, QST_INJECT_WPASS_LOADS = 2 };
qst_status qst_inject_wait_timeout(int what, int count);

typedef struct qst_tuning {
    int bulk_chunks_per_cta;
    int fused_ctas_per_sm;
    int fused_max_qubits;
    int batch_concurrent_runs;
} qst_tuning;
void qst_get_tuning(qst_tuning* t);
qst_status qst_set_tuning(const qst_tuning* t);

/* Wait for all work enqueued on the context's stream. */
qst_status qst_sync(qst_ctx* ctx);

/* ---- batches of independent tomographies (one graph launch per iteration) ----
 * B tomographies of possibly different qubit counts Ns[b], each with its own
 * context (parameters, Rprop state, scratch) and stream.  From the second
 * qst_batch_step with the same inputs on, one iteration of all B is a single
 * cudaGraphLaunch on `stream` whose graph forks to one kernel chain per
 * tomography and joins them.  QST_MIXED / QST_MIXED_BF16 apply to the
 * tomographies with N >= 7; smaller ones run FP32.  The tomographies share
 * nothing, so this is the method applied B times (Sec. 4 runs many states).
 * qst_batch_step validates every new input (as qst_step does) before any
 * tomography steps: a call that returns QST_E_INPUT or QST_E_INVAL has
 * advanced none of them. */
typedef struct qst_batch qst_batch;
qst_status qst_batch_init(qst_batch** out, int B, const int* Ns, const double* povm, int K,
                          const qst_options* opt, void* stream);
/* Context of tomography b (for qst_get_params, qst_get_rho, ...); owned by the batch. */
qst_ctx* qst_batch_context(qst_batch* batch, int b);
qst_status qst_batch_set_params(qst_batch* batch, int b, const void* theta);
/* One iteration of every tomography.  f: host array of B device pointers (n_b reals
 * each).  losses: host array of B doubles or NULL (synchronises). */
qst_status qst_batch_step(qst_batch* batch, const void* const* f, double* losses);
/* iters iterations, then each rho_out[b] (device or host, or rho_out NULL) and final loss. */
qst_status qst_batch_reconstruct(qst_batch* batch, const void* const* f, int iters, void* const* rho_out,
                                 double* final_losses);
long long qst_batch_kernel_launches(const qst_batch* batch);
qst_status qst_batch_sync(qst_batch* batch);
void qst_batch_destroy(qst_batch* batch);

const char* qst_strerror(qst_status s);

void qst_destroy(qst_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* QST_H */
