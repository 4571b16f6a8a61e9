/*
 * linview.h -- C ABI of the GB300 LINVIEW library (incremental maintenance of
 * iterative linear-algebra programs under factored low-rank updates,
 * arXiv 1403.6968).
 *
 * The paper states a program as a list of statements <A_i, E_i> over a set of
 * input matrices (Section 3.4, Algorithm 1); each input gets a trigger that
 * receives an update in factored form dX = U V^T (Section 3.2, Example 3.8),
 * derives the factored deltas of every materialised view, and refreshes the
 * views in place ("A += ...; B += ...; C += ..." in Example 3.8).
 * Re-evaluation means: apply the update to the inputs, then recompute every
 * view from scratch (Section 4.2.2, "Re-evaluation").  This header exposes the
 * four program kinds the paper analyses (Section 4): matrix powers, sums of
 * matrix powers, the general form T_{i+1} = A T_i + B, and OLS.
 *
 * Conventions for every call:
 *  - Matrices are row-major with an explicit leading dimension ``ld`` (in
 *    elements, ld >= number of columns).  Element type is double for
 *    LINVIEW_F64 programs and float for LINVIEW_F32 programs.
 *  - ``stream`` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Work is enqueued on it; calls return once the work is
 *    enqueued (host-side argument checks are synchronous).
 *  - ``*_on_device`` flags say whether a pointer is device memory (1) or host
 *    memory (0).  Host inputs are copied to the device before the call
 *    returns; host outputs are written before the call returns.
 *  - Device inputs passed to a call are read in stream order; the caller keeps
 *    them alive until the call's work has completed (e.g. an event or sync).
 *  - The library owns every view and internal buffer of a program and frees
 *    them in linview_destroy; it never frees caller memory.
 *  - Errors are reported by status code only (no exceptions cross the ABI).
 *    linview_last_error() returns a thread-local message for the last failure.
 *  - Every pointer an entry point takes as device memory (on_device = 1, a
 *    device destination, the stand-alone passes' and GEMM's operands) must be
 *    device or managed memory of the current (or the program's) device; other
 *    memory is EINVAL before any work is queued.  Sizes cannot be checked
 *    from a pointer: the caller keeps every buffer at least as large as the
 *    shapes and leading dimensions it passes.
 *    Problems detected on the device (a non-finite factor core, a singular
 *    Woodbury core, an expired bounded wait) are latched in a device status
 *    word and returned by the next linview_sync() on that program.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns LINVIEW_EDEVICE.
 */
#ifndef LINVIEW_H_
#define LINVIEW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct linview_program linview_program; /* opaque, library-owned */

typedef enum {
  LINVIEW_OK = 0,
  LINVIEW_EINVAL = 1,       /* null pointer, bad id, negative size, bad flag */
  LINVIEW_ESHAPE = 2,       /* size or leading dimension inconsistent with the program */
  LINVIEW_ENOMEM = 3,       /* device allocation failed */
  LINVIEW_ERANK = 4,        /* update rank * growth exceeds the factor arena (r_max) */
  LINVIEW_ESINGULAR = 5,    /* Woodbury core (C^-1 + U^T W U) numerically singular */
  LINVIEW_ENONFINITE = 6,   /* NaN or Inf met in a factor core */
  LINVIEW_ETIMEOUT = 7,     /* a bounded device-side wait expired */
  LINVIEW_EDEVICE = 8,      /* CUDA runtime, driver or cuBLAS error; no device */
  LINVIEW_EUNSUPPORTED = 9  /* valid request this build does not implement */
} linview_status;

typedef enum {
  LINVIEW_POWER = 0,      /* views A^h, h = 1, 2, 4, ..., k  (Table 1, exponential model) */
  LINVIEW_POWER_SUM = 1,  /* as POWER plus S'_h = A + A^2 + ... + A^h  (Section 4.2.3) */
  LINVIEW_ITERATION = 2,  /* views T_1..T_k of T_i = A T_{i-1} + B  (Section 4.3) */
  LINVIEW_OLS = 3         /* W = (X^T X)^-1, beta = W X^T Y  (Section 4.1) */
} linview_kind;

typedef enum { LINVIEW_F64 = 0, LINVIEW_F32 = 1 } linview_precision;

/* GEMM arithmetic used by linview_reeval (the re-evaluation strategy) and by
 * residual correction.  The default is the library's own GEMM; the cuBLAS
 * arithmetics (FP32, TF32, BF16X9) are comparison denominators, selected
 * explicitly, for power and iteration programs. */
typedef enum {
  LINVIEW_REEVAL_DEFAULT = 0, /* FP64 programs: LINVIEW_REEVAL_FP64; FP32: LINVIEW_REEVAL_TC3 */
  LINVIEW_REEVAL_FP32 = 1,    /* comparison: IEEE FP32 GEMM on the CUDA cores (cuBLAS, pedantic) */
  LINVIEW_REEVAL_TF32 = 2,    /* comparison: one TF32 tensor-core pass (cuBLAS; ~1e-3 relative) */
  LINVIEW_REEVAL_BF16X9 = 3,  /* comparison: FP32 emulated by nine BF16 products (cuBLAS) */
  LINVIEW_REEVAL_FP64 = 4,    /* FP64 programs: the library's FP64 GEMM on the CUDA cores */
  LINVIEW_REEVAL_TC3 = 5      /* FP32 programs: the library's tcgen05 GEMM in split TF32
                                 (three TF32 products per operand pair, FP32 accuracy) */
} linview_reeval_mode;

typedef struct {
  int32_t kind;              /* linview_kind */
  int32_t precision;         /* linview_precision */
  int64_t n;                 /* A is n x n (POWER, POWER_SUM, ITERATION); X has n columns (OLS) */
  int64_t m;                 /* OLS: rows of X and Y; otherwise 0 */
  int64_t p;                 /* ITERATION: columns of B and T_i; OLS: columns of Y; otherwise 0 */
  int32_t k;                 /* POWER/POWER_SUM: highest power (a power of two >= 1 in
                                the exponential model, >= 2 in the linear model);
                                ITERATION: number of steps >= 1 (a power of two >= 2 in the
                                exponential model, a multiple of s >= 2s in the skip
                                model); OLS: largest row block */
  int32_t r_max;             /* largest rank accepted by linview_apply_delta (>= 1) */
  int32_t correction_period; /* >0: correct every this many updates (residual
                                correction of accumulated rounding, see
                                desc.correction); 0 = never */
  int32_t reeval_mode;       /* linview_reeval_mode used by linview_reeval and by correction */
  int32_t model;             /* POWER/POWER_SUM: linview_model; ITERATION:
                                LINVIEW_MODEL_LINEAR (views T_1..T_k), LINVIEW_MODEL_EXP
                                (views T_1, T_2, T_4, .., T_k) or LINVIEW_MODEL_SKIP
                                (T_1, T_2, .., T_s, T_2s, .., T_k; Appendix B); OLS: 0 */
  int32_t skip;              /* LINVIEW_MODEL_SKIP: the step s; otherwise 0 */
  int32_t strategy;          /* ITERATION: linview_strategy; other kinds: 0 */
  /*
   * Device memory of the program (its materialised views, Example 3.8's
   * "A += ...; B += ..." targets, the factor arenas and the passes' scratch).
   * Both NULL: the library calls cudaMalloc / cudaFree.  Otherwise every device
   * allocation the program makes -- at creation and the few made lazily by
   * later calls (host-factor staging, adjoint and re-evaluation work space) --
   * is alloc(bytes, stream, alloc_ctx), with ``stream`` the cudaStream_t of the
   * call that needs it (the memory is first used there, in stream order);
   * alloc returns a device pointer, 256-byte aligned, or NULL (the call then
   * fails with LINVIEW_ENOMEM).  Sizes are multiples of 512 bytes.  Each block
   * is returned exactly once, by free(ptr, bytes, NULL, alloc_ctx) inside
   * linview_destroy after the device has finished all of the program's work;
   * temporary blocks of a single call are returned by that call as
   * free(ptr, bytes, stream, alloc_ctx) in its stream order.  This is how a
   * caching allocator (PyTorch's) owns the program's memory; the library never
   * frees memory it did not obtain this way.  The callbacks are called from the
   * thread making the library call.  linview_program_device_bytes counts the
   * blocks the program holds.
   */
  void* (*alloc)(size_t bytes, void* stream, void* alloc_ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* alloc_ctx);
  void* alloc_ctx;
  int32_t correction;        /* linview_correction: what a residual correction does (every
                                correction_period updates, or on linview_correct) */
} linview_program_desc;

/* Residual correction (desc.correction).  LINVIEW_CORRECT_REEVAL: re-evaluate
 * every view (linview_reeval), any program.  LINVIEW_CORRECT_NEWTON: OLS
 * programs in FP32 only.  The program also keeps Z = X^T X as double-float
 * pairs (two n x n FP32 arrays, initialised from the FP64 X^T X of every
 * re-evaluation and refreshed by the rank-2k update Z += X'_R^T X'_R -
 * X_R^T X_R of every row block, on the side stream next to the Woodbury
 * passes); a correction is then one Newton-Schulz step for the inverse of Z,
 * W <- W + W (I - Z W), with the residual I - Z W in double-float and W (I - Z W)
 * on the split-TF32 GEMM, followed by beta = W X^T Y.  The step squares the
 * error of W in the residual sense (W - Z^-1 -> -(W - Z^-1) Z (W - Z^-1)), so
 * a W that has drifted by rounding returns to FP32 rounding of Z^-1 without
 * the re-evaluation's FP64 X^T X over all m rows.  Other kinds or FP64 OLS
 * programs with LINVIEW_CORRECT_NEWTON fail creation with LINVIEW_EUNSUPPORTED. */
typedef enum { LINVIEW_CORRECT_REEVAL = 0, LINVIEW_CORRECT_NEWTON = 1 } linview_correction;

/* Evaluation strategy of an iteration program's updates (Section 4.3). */
typedef enum {
  LINVIEW_STRATEGY_FACTORED = 0, /* incremental: dT_i = U_i V_i^T in factored form (App. B,
                                    linear model with Krylov reuse) */
  LINVIEW_STRATEGY_HYBRID = 1    /* hybrid: dT_i kept as one dense n x p matrix D_i,
                                    D_i = A D_{i-1} + (rank-r term), one n x n x p product
                                    with A per step (Sec. 4.3; App. B, hybrid linear) */
} linview_strategy;

/* Iterative model of a power program (Section 3.3; Appendix A), or of an
 * iteration program (LINEAR or EXP; Appendix B). */
typedef enum {
  LINVIEW_MODEL_EXP = 0,     /* P_{2h} = P_h P_h: views A, A^2, A^4, ..., A^k */
  LINVIEW_MODEL_LINEAR = 1,  /* P_i = A P_{i-1}: views A, A^2, A^3, ..., A^k; r_max * k <= 64 */
  LINVIEW_MODEL_SKIP = 2     /* exponential up to A^s, then P_i = A^s P_{i-s}: views A, A^2,
                                A^4, ..., A^s, A^2s, ..., A^k (POWER_SUM adds S'_h for the same
                                h > 1); s a power of two, k a multiple of s, k >= 2s,
                                r_max * k <= 64 */
} linview_model;

/*
 * Create a program and materialise its views by re-evaluation on the device
 * (the paper precomputes and preloads the initial view values, Section 6).
 *  inputs[i] / lds[i]: the program's input matrices, row-major:
 *    POWER, POWER_SUM: {A (n x n)}
 *    ITERATION:        {A (n x n), B (n x p), T_0 (n x p)}
 *    OLS:              {X (m x n), Y (m x p)}
 *  inputs_on_device: 1 if the input pointers are device memory, 0 for host.
 *  On success *out receives the program; the caller destroys it with
 *  linview_destroy.  Errors: EINVAL, ESHAPE, ENOMEM, EDEVICE, EUNSUPPORTED.
 */
linview_status linview_create_program(const linview_program_desc* desc, const void* const* inputs,
                                      const int64_t* lds, int inputs_on_device, void* stream,
                                      linview_program** out);

/*
 * Fire the trigger of input ``input_id`` for the factored update
 * dX = U V^T (Section 3.2; Example 3.8 for powers, Appendix A; Appendix B for
 * the iteration).  Input 0 (A): U is n x rank (row-major, ldu >= rank), V is
 * n x rank (ldv >= rank); POWER, POWER_SUM and ITERATION.  Input 1 (B) of an
 * ITERATION program: U is n x rank, V is p x rank; with A unchanged,
 * dT_i = A dT_{i-1} + dB, so dT_i = [U, A U, .., A^(i-1) U][V, .., V]^T (the
 * paper omits changes in B, Section 4.3.2; this is the rule the recurrence
 * gives).  Every view is refreshed in place: view += (its factored delta).
 * Errors: EINVAL, ESHAPE, ERANK (rank > r_max), EDEVICE.  On error the views
 * are unchanged.
 */
linview_status linview_apply_delta(linview_program* prog, int input_id, int64_t rank, const void* U,
                                   int64_t ldu, const void* V, int64_t ldv, int on_device,
                                   void* stream);

/*
 * Row update dA = e_row v^T (the paper's workload: "each update affects one
 * row", Section 6): U = e_row is formed on the device.  v has n entries.
 */
linview_status linview_apply_row_delta(linview_program* prog, int input_id, int64_t row,
                                       const void* v, int on_device, void* stream);

/*
 * OLS only: replace ``kr`` distinct rows of X (indices ``rows``, host array)
 * by ``new_rows`` (kr x n, row-major, ld).  Y is unchanged.  W is maintained
 * by block Woodbury with a 2kr x 2kr core (the rank-2kr generalisation of the
 * two Sherman-Morrison steps of Example 3.3), inverted in FP64 for FP64
 * programs and as double-float pairs (Newton-Schulz, Gauss-Jordan fallback)
 * for FP32 programs; beta = W X^T Y is
 * refreshed from the same factors (the delta of a product, Section 3.2), with
 * no further pass over W.
 * Errors: EINVAL, ESHAPE (kr > desc.k), ESINGULAR (latched, see linview_sync):
 * W is then left as it was while X and X^T Y hold the new rows, so the views
 * no longer agree with X until linview_reeval succeeds.
 */
linview_status linview_apply_row_block(linview_program* prog, int64_t kr, const int64_t* rows,
                                       const void* new_rows, int64_t ld, int on_device,
                                       void* stream);

/*
 * Number of views and the shape of view ``view_id``.
 * View ids:
 *   POWER:     0 = A = P_1, j = P_{2^j} (j = 1..log2 k)
 *   POWER_SUM: as POWER, then log2(k) + j = S'_{2^j} (j = 1..log2 k); S'_1 = A
 *   linear model (LINVIEW_MODEL_LINEAR): i - 1 = P_i (i = 1..k); POWER_SUM adds
 *              k = S'_k
 *   skip-s model (LINVIEW_MODEL_SKIP): j = P_{2^j} (j = 0..log2 s), then
 *              log2(s) + i - 1 = P_{is} (i = 2..k/s); with N such power views,
 *              POWER_SUM adds N + j - 1 = S'_h for the power view j >= 1
 *   ITERATION, linear model: 0 = A, i = T_i (i = 1..k), k + 1 = B, k + 2 = T_0
 *   ITERATION, skip-s model (exponential model: s = k/2): with the T views
 *              T_1, T_2, T_4, .., T_s, T_2s, T_3s, .., T_k (NT = log2(s) + k/s of
 *              them): 0 = A, 1 + j = the j-th T view (j = 0..NT-1), NT + 1 = B,
 *              NT + 2 = T_0, then the auxiliary views NT + 2 + l = P_{2^l} and
 *              NT + 2 + log2(s) + l = S'_{2^l} (l = 1..log2 s), with
 *              T_2h = P_h T_h + S_h B (h < s), T_i = P_s T_{i-s} + S_s B (i > s),
 *              S_h = I + S'_h - P_h; updates to B: dT_i = P dT_j + S dB; the
 *              adjoints recompute T_0 .. T_k from (A, B, T_0) first
 *   OLS:       0 = W (n x n), 1 = beta (n x p), 2 = X^T Y (n x p), 3 = X (m x n)
 */
int linview_num_views(const linview_program* prog);
linview_status linview_view_shape(const linview_program* prog, int view_id, int64_t* rows,
                                  int64_t* cols);

/* Destinations of linview_read_view / linview_read_view_rows (dst_on_device). */
enum {
  LINVIEW_DST_HOST = 0,       /* host memory; the call synchronises the stream */
  LINVIEW_DST_DEVICE = 1,     /* device memory; asynchronous on the stream */
  LINVIEW_DST_HOST_ASYNC = 2  /* host memory, asynchronous on the stream: the caller
                                 synchronises the stream (or an event recorded after
                                 the call) before reading dst and keeps dst alive until
                                 then; page-locked dst makes the copy overlap later work */
};

/*
 * Copy view ``view_id`` into dst (row-major, ld >= cols).  dst_on_device
 * selects the destination (LINVIEW_DST_*).  For LINVIEW_DST_HOST the call
 * synchronises the stream before returning.  Errors: EINVAL (null, bad id or
 * destination), ESHAPE (ld < cols).
 */
linview_status linview_read_view(const linview_program* prog, int view_id, void* dst, int64_t ld,
                                 int dst_on_device, void* stream);

/*
 * Copy rows [row0, row0 + nrows) of view ``view_id`` into dst (nrows x cols,
 * row-major, ld >= cols).  Same destinations and synchronisation as
 * linview_read_view.
 */
linview_status linview_read_view_rows(const linview_program* prog, int view_id, int64_t row0,
                                      int64_t nrows, void* dst, int64_t ld, int dst_on_device,
                                      void* stream);

/*
 * Device pointer and leading dimension of a view (library-owned; valid until
 * linview_destroy; the caller must not write through it).
 */
linview_status linview_view_device_ptr(const linview_program* prog, int view_id, void** ptr,
                                       int64_t* ld);

/* Re-evaluate every view from the current inputs (Section 4.2.2,
 * "Re-evaluation"), with the program's reeval_mode arithmetic. */
linview_status linview_reeval(linview_program* prog, void* stream);

/* Run the program's residual correction now (desc.correction): linview_reeval,
 * or for an OLS program with LINVIEW_CORRECT_NEWTON one Newton-Schulz step on
 * W and beta = W X^T Y.  Enqueued on ``stream``; LINVIEW_ENOMEM if its
 * temporaries (two n x n FP32 arrays and the GEMM's split operands) cannot be
 * allocated. */
linview_status linview_correct(linview_program* prog, void* stream);
linview_status linview_set_reeval_mode(linview_program* prog, int reeval_mode);

/* Synchronise ``stream`` and return (and clear) the latched device status. */
/*
 * Diagnostic of the bounded device waits (failure detection without a fault).
 * Runs one kernel whose single wait is on an mbarrier that nothing ever
 * completes, with a limit of limit_ns (1e6 .. 1e10).  The wait gives up after
 * the limit and latches the timeout bit exactly as a view pass does when a
 * copy never lands (every pass waits with limit 2 s); the device context stays
 * usable.  Returns LINVIEW_ETIMEOUT, the expected outcome, with *waited_ns the
 * time the wait took (>= limit_ns); LINVIEW_OK would mean the barrier
 * completed (never expected); EINVAL for a bad limit or null pointer,
 * EDEVICE on a CUDA error.  Synchronises ``stream``.
 */
linview_status linview_check_bounded_wait(int64_t limit_ns, void* stream, int64_t* waited_ns);

linview_status linview_sync(linview_program* prog, void* stream);

/*
 * Capture the per-update propagation graphs of ranks 1..max_rank now, ahead
 * of the first update of each rank (which would otherwise capture it): a
 * warm-up for latency-sensitive callers.  Queues no work.  Power, power-sum
 * and iteration programs (updates to A); a no-op for OLS.  Errors: EINVAL,
 * ERANK (max_rank outside 1..r_max), EDEVICE.
 */
linview_status linview_prepare_updates(linview_program* prog, int32_t max_rank, void* stream);

void linview_destroy(linview_program* prog);
const char* linview_last_error(void);

/*
 * Adjoints (reverse mode) on the device.  Outputs are device pointers,
 * row-major.
 *  linview_adjoint_iteration: L = ||T_k||_F^2 over the current views;
 *    dA (n x n) = sum_{i=1..k} G_i T_{i-1}^T, dB (n x p) = sum_i G_i with
 *    G_k = 2 T_k, G_i = A^T G_{i+1}.  dA or dB may be NULL.
 *  linview_adjoint_power: G = dL/dP_k (device, n x n); dA = dL/dA
 *    = sum_j (A^T)^j G (A^T)^{k-1-j}, evaluated back through the squaring
 *    chain Gbar_h = Gbar_{2h} P_h^T + P_h^T Gbar_{2h} on the maintained views.
 */
linview_status linview_adjoint_iteration(linview_program* prog, void* dA, int64_t ld_dA, void* dB,
                                         int64_t ld_dB, void* stream);
/*
 * linview_adjoint_iteration_seed: the same reverse pass from an arbitrary
 * upstream gradient Gk = dL/dT_k (device, n x p, row-major, ldg >= p) instead
 * of 2 T_k: G_k = Gk, G_i = A^T G_{i+1}; dA = sum_i G_i T_{i-1}^T,
 * dB = sum_i G_i, dT0 (n x p, may be NULL) = A^T G_1.  This is the vector-
 * Jacobian product of the map (A, B, T_0) -> T_k, for reverse-mode autodiff.
 */
linview_status linview_adjoint_iteration_seed(linview_program* prog, const void* Gk, int64_t ldg,
                                              void* dA, int64_t ld_dA, void* dB, int64_t ld_dB,
                                              void* dT0, int64_t ld_dT0, void* stream);
linview_status linview_adjoint_power(linview_program* prog, const void* G, int64_t ldg, void* dA,
                                     int64_t ld_dA, void* stream);

/*
 * One level pass of the exponential model as a stand-alone operation
 * (Appendix A: the products P_h U_h and P_h^T V_h that build U_{2h} and V_{2h},
 * and the in-place refresh P_h += U_h V_h^T), on caller-owned device memory.
 *  P: n x n, row-major, ldp (ldp % 4 == 0 for float, % 2 == 0 for double;
 *     16-byte aligned base).
 *  U, V: n x r, column-major (column stride ldf >= n).  1 <= r <= 64.
 *  X (may be NULL): n x r column-major, ldf, receives P U (P before the update).
 *  Y (may be NULL): n x r column-major, ldf, receives P^T V (P before the update).
 *  do_update: 1 to apply P += U V^T, 0 to leave P unchanged.
 *  precision: LINVIEW_F32 or LINVIEW_F64.
 * Scratch for the cross-block partial sums is allocated stream-ordered on
 * ``stream`` and released before the call returns.
 */
linview_status linview_level_pass(int precision, int64_t n, void* P, int64_t ldp, const void* U,
                                  const void* V, int64_t ldf, int64_t r, void* X, void* Y,
                                  int do_update, void* stream);

/*
 * The library's own dense product on caller device memory: the contraction of
 * the re-evaluation strategy's squarings and sums (Section 4.2.2,
 * "Re-evaluation"; Table 1) and of the reverse pass, as a stand-alone
 * operation.
 *   C (M x N) = alpha op(A) op(B) + beta C,  all row-major; op(X) = X^T when
 *   the flag (ta / tb) is set.  A is M x K (ld >= K), or K x M when ta
 *   (ld >= M); B is K x N (ld >= N), or N x K when tb (ld >= K).  beta = 0
 *   ignores C's old contents.  M = 0 or N = 0 is an empty product (OK, no
 *   pointer is read); K >= 1.
 *  precision LINVIEW_F32: the tcgen05 split-TF32 GEMM (near-FP32 accuracy,
 *   three TF32 products per operand pair, FP32 accumulation) when M >= 128,
 *   N >= 8 and K >= 128, else the CUDA-core GEMM in FP32; LINVIEW_F64: the
 *   FP64 CUDA-core GEMM.
 * Temporary device memory (split operands, partial sums) is allocated
 * stream-ordered on ``stream`` and released before the call returns; the call
 * synchronises ``stream``.  Errors: EINVAL, ESHAPE, ENOMEM, ETIMEOUT (a
 * bounded device wait expired), EDEVICE.
 */
linview_status linview_gemm(int precision, int ta, int tb, int64_t M, int64_t N, int64_t K,
                            double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                            double beta, void* C, int64_t ldc, void* stream);

/*
 * linview_level_pass without any device allocation.  The paper has no
 * counterpart: this entry exists for callers that may not allocate device
 * memory on their call path (a process or engine plugin that reserved the GPU's
 * memory up front, or a latency-critical loop that must avoid the implicit
 * synchronisation of cudaMalloc/cudaFree).  Arguments and layouts are those of
 * linview_level_pass; the cross-block partial sums live in one array built
 * into the library (16 MiB of device memory, reserved on a device once the
 * library's kernels are first used there -- CUDA's lazy module loading -- and
 * held until the process exits) instead of stream-ordered allocations.  It
 * launches the allocating entry's CUDA-core products passes and reductions;
 * FP32 blocks wider than 16 columns run on the CUDA-core passes here (products
 * in blocks of 16, updates in blocks of 32), where the allocating entry uses
 * the tensor-core passes (which need factor scratch buffers), so for those the
 * two entries agree within FP32 rounding rather than bit for bit.  Sizes whose
 * partial sums do not fit (roughly n * r beyond 8192 * 8 for FP32 on a 152-SM
 * GPU) return LINVIEW_ESHAPE with the needed byte count, before the array is
 * touched.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture begins.  All calls share the array and it keeps the last
 * call's contents: calls whose work overlaps on the GPU race on it and must be
 * serialised.  The call synchronises ``stream`` before returning (to read the
 * status word).
 */
linview_status linview_level_pass_noalloc(int precision, int64_t n, void* P, int64_t ldp,
                                          const void* U, const void* V, int64_t ldf, int64_t r,
                                          void* X, void* Y, int do_update, void* stream);

/*
 * Kernel timing for measurement: when enabled, the library records CUDA
 * events around each launch of its view-pass kernels on the launching
 * stream.  linview_pass_stats returns, for ``kernel`` = 0 (all view passes),
 * 1 (fused products + update pass) or 2 (update-only pass), the number of
 * launches since the last reset, their summed device time (ms; the call
 * waits for the recorded events), and the algorithmic bytes those launches
 * move (each view element read once and, when refreshed, written once).
 * *all_launches counts every kernel and library call the program issued.
 * Power programs replay their per-update propagation as CUDA graphs; with
 * profiling enabled each rank's propagation is captured as 16 instrumented
 * copies (event-record nodes around every view pass) replayed round-robin,
 * and the statistics cover the last replay of every copy replayed since the
 * last reset (so at most the last 16 updates).
 */
linview_status linview_set_profiling(linview_program* prog, int enable);
linview_status linview_pass_stats(linview_program* prog, int kernel, int64_t* launches, double* ms,
                                  double* bytes, int64_t* all_launches);
linview_status linview_reset_stats(linview_program* prog);

/*
 * Device memory of a program.  linview_program_device_bytes: the bytes the
 * program holds (the sum of its device allocations: views, factor arenas,
 * partial sums, staging).  linview_estimate_device_bytes: the same figure for
 * a LINVIEW_POWER or LINVIEW_POWER_SUM program that linview_create_program
 * would build from ``desc`` on the current device, without allocating
 * (other kinds return LINVIEW_EUNSUPPORTED).
 */
linview_status linview_program_device_bytes(const linview_program* prog, int64_t* bytes);
linview_status linview_estimate_device_bytes(const linview_program_desc* desc, int64_t* bytes);

/*
 * Serving: many maintained matrix-power programs (Section 4.2, A^k by
 * repeated squaring, FP32) kept resident in device memory under a stream of
 * factored updates dA = U V^T (Section 3.2: updates and deltas in factored
 * form) that arrive over time, with continuous batching:
 *  - a scheduler thread owned by the server takes queued requests as soon as
 *    a slot is free (at most ``max_inflight`` views refreshing at once, each
 *    on its own CUDA stream, so their work overlaps on the GPU);
 *  - the requests queued for one view while it is busy are coalesced into a
 *    single delta of higher rank, [U_1 .. U_m][V_1 .. V_m]^T = sum_j U_j V_j^T
 *    (the concatenation rule of factored deltas, Section 3.2; the paper's
 *    batch updates, Section 6, Table 4): in arrival order, every queued
 *    request that keeps the total rank within ``r_cap`` joins (deltas add,
 *    so the order of application does not change the result); the oldest
 *    request always joins, the others wait for the next refresh;
 *  - a view is admitted (its program created) only when its device bytes
 *    (linview_estimate_device_bytes) fit both the server budget and the free
 *    device memory; otherwise it waits, with its requests queued, and is
 *    admitted when a removed view frees memory.
 * Times are seconds on the server clock (a monotonic clock started by
 * linview_server_create; linview_server_clock reads it).  Latency of a
 * request = done_s - arrival_s, where done_s is when the scheduler saw the
 * refresh's completion event.
 *
 * linview_server_create: hbm_budget_bytes <= 0 means the free device memory
 *   at creation minus 1 GiB; max_inflight >= 1; 1 <= r_cap and r_cap * k <= 128
 *   for every view.  Uses the current device.
 * linview_server_add_view: A is n x n FP32 row-major (lda), host or device;
 *   the server copies it before returning.  *view receives the view id; the
 *   view is admitted at once if memory allows (state 1), else it waits
 *   (state 0).  k is a power of two.  The view's program ids are those of a
 *   LINVIEW_POWER program: 0 = A, j = A^(2^j).
 * linview_server_submit: one request dA = U V^T for ``view``; U, V are n x
 *   rank FP32 row-major host arrays (ldu, ldv >= rank), copied before the
 *   call returns; 1 <= rank <= n, else LINVIEW_ERANK.  Requests of rank <=
 *   r_cap coalesce as described above.  A request of rank > r_cap is served
 *   by re-evaluation (Section 4.2.2, "Re-evaluation"): when it is the oldest
 *   request of its view, it and every request queued behind it are added to
 *   A (update-only level passes on the device) and every view of the program
 *   is recomputed from the new A (linview_reeval; its temporary operands are
 *   device memory the admission budget does not reserve, so ENOMEM is
 *   possible on a full GPU).  arrival_s < 0 stamps the current server time.
 *   *ticket receives the request id (tickets count from 1 in submission
 *   order).
 * linview_server_submit_row: a row update dA = e_row v^T (v: n floats, host,
 *   copied).  Row updates queued for one view coalesce by row: requests to a
 *   row already in the delta add their v to that row's column and no rank,
 *   so a delta's rank is its number of distinct rows (plus the ranks of the
 *   factored requests in it); the paper's batch updates with skewed row
 *   frequencies (Section 6, Table 4).
 * linview_server_replay: open-loop load for measurement.  The calling thread
 *   submits request i at server time t0 + t_s[i] (t0 = the time of the call,
 *   t_s non-decreasing) with arrival_s = t0 + t_s[i], and returns after the
 *   last one.  Its factors are NOT copied: U_i is the n_view x rank[i]
 *   row-major array at factors + offset[i] (floats), V_i follows it
 *   directly; when ``rows`` is not NULL and rows[i] >= 0, request i is the
 *   row update e_rows[i] v^T with v the n_view floats at factors + offset[i]
 *   (rank[i] ignored).  The caller keeps ``factors`` alive until
 *   linview_server_drain returns.
 * linview_server_poll: moves up to ``max`` completion records (oldest first)
 *   to ``out``; *count receives how many.  Never blocks.
 * linview_server_drain: waits until every request submitted so far has
 *   completed (LINVIEW_ETIMEOUT after timeout_s seconds; timeout_s <= 0
 *   waits without limit).
 * linview_server_view_state: 0 waiting for admission, 1 resident, 2 removed.
 * linview_server_view_program: the program of a resident view, for
 *   linview_read_view & co.  Only valid while the view is resident; read it
 *   only after linview_server_drain (the scheduler thread issues its work).
 * linview_server_remove_view: the scheduler lets the view's refresh in flight
 *   finish, completes its still-queued requests with status LINVIEW_EINVAL,
 *   destroys the program and admits waiting views that now fit.  Returns
 *   at once; the view's state turns 2 when it is gone.
 * linview_server_stats: counters since creation (see the struct).
 * linview_server_destroy: stops the scheduler after the refreshes in flight
 *   have finished (queued requests are dropped) and frees every view.
 * A refresh that fails on the device reports its status in the completion
 * records of its requests; the view stays resident.
 */
typedef struct linview_server linview_server; /* opaque, library-owned */

typedef struct {
  uint64_t ticket;     /* request id from submit / replay order */
  int32_t view;        /* view id */
  int32_t rank;        /* rank of this request */
  int32_t batch_rank;  /* rank of the coalesced delta the request was applied in */
  int32_t batch_size;  /* requests coalesced into that delta */
  int32_t status;      /* linview_status of the refresh */
  int32_t reserved;
  double arrival_s;    /* server time the request arrived */
  double start_s;      /* server time its refresh was issued */
  double done_s;       /* server time its refresh was seen complete */
} linview_completion;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t refreshes;          /* coalesced deltas applied */
  int64_t coalesced_rank_sum; /* sum of their ranks */
  int32_t views_resident, views_waiting;
  int32_t max_inflight_seen;  /* most views refreshing at the same time */
  int32_t reevals;            /* refreshes served by re-evaluation (a rank past r_cap) */
  int64_t bytes_used, bytes_budget;
} linview_server_stats;

linview_status linview_server_create(int64_t hbm_budget_bytes, int32_t max_inflight, int32_t r_cap,
                                     linview_server** out);
linview_status linview_server_add_view(linview_server* srv, int64_t n, int32_t k, const void* A,
                                       int64_t lda, int on_device, int32_t* view);
linview_status linview_server_submit(linview_server* srv, int32_t view, int32_t rank, const void* U,
                                     int64_t ldu, const void* V, int64_t ldv, double arrival_s,
                                     uint64_t* ticket);
linview_status linview_server_submit_row(linview_server* srv, int32_t view, int64_t row,
                                         const void* v, double arrival_s, uint64_t* ticket);
linview_status linview_server_replay(linview_server* srv, int64_t count, const double* t_s,
                                     const int32_t* view, const int32_t* rank, const void* factors,
                                     const int64_t* offset, const int64_t* rows);
linview_status linview_server_poll(linview_server* srv, linview_completion* out, int32_t max,
                                   int32_t* count);
linview_status linview_server_drain(linview_server* srv, double timeout_s);
linview_status linview_server_view_state(linview_server* srv, int32_t view, int32_t* state);
linview_status linview_server_view_program(linview_server* srv, int32_t view,
                                           linview_program** prog);
linview_status linview_server_remove_view(linview_server* srv, int32_t view);
linview_status linview_server_stats_get(linview_server* srv, linview_server_stats* out);
double linview_server_clock(const linview_server* srv);
void linview_server_destroy(linview_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* LINVIEW_H_ */
