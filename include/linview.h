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

/* GEMM arithmetic used by linview_reeval (the re-evaluation strategy). */
typedef enum {
  LINVIEW_REEVAL_DEFAULT = 0, /* FP64 programs: DGEMM; FP32 programs: LINVIEW_REEVAL_FP32 */
  LINVIEW_REEVAL_FP32 = 1,    /* IEEE FP32 GEMM on the CUDA cores (cuBLAS, pedantic) */
  LINVIEW_REEVAL_TF32 = 2,    /* one TF32 tensor-core pass (fast, ~1e-3 relative) */
  LINVIEW_REEVAL_BF16X9 = 3,  /* FP32 emulated by nine BF16 tensor-core products */
  LINVIEW_REEVAL_FP64 = 4     /* DGEMM (FP64 programs) */
} linview_reeval_mode;

typedef struct {
  int32_t kind;              /* linview_kind */
  int32_t precision;         /* linview_precision */
  int64_t n;                 /* A is n x n (POWER, POWER_SUM, ITERATION); X has n columns (OLS) */
  int64_t m;                 /* OLS: rows of X and Y; otherwise 0 */
  int64_t p;                 /* ITERATION: columns of B and T_i; OLS: columns of Y; otherwise 0 */
  int32_t k;                 /* POWER/POWER_SUM: highest power, a power of two >= 1;
                                ITERATION: number of steps >= 1; OLS: largest row block */
  int32_t r_max;             /* largest rank accepted by linview_apply_delta (>= 1) */
  int32_t correction_period; /* >0: re-evaluate every this many updates (residual
                                correction of accumulated rounding); 0 = never */
  int32_t reeval_mode;       /* linview_reeval_mode used by linview_reeval and by correction */
} linview_program_desc;

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
 * the iteration).  Only input 0 (A) is supported for POWER, POWER_SUM and
 * ITERATION.  U is n x rank (row-major, ldu >= rank); V is n x rank (ldv >=
 * rank).  Every view is refreshed in place: view += (its factored delta).
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
 * by block Woodbury with an FP64 2kr x 2kr core (the rank-2kr generalisation
 * of the two Sherman-Morrison steps of Example 3.3), beta = W X^T Y.
 * Errors: EINVAL, ESHAPE (kr > desc.k), ESINGULAR (latched, see linview_sync).
 */
linview_status linview_apply_row_block(linview_program* prog, int64_t kr, const int64_t* rows,
                                       const void* new_rows, int64_t ld, int on_device,
                                       void* stream);

/*
 * Number of views and the shape of view ``view_id``.
 * View ids:
 *   POWER:     0 = A = P_1, j = P_{2^j} (j = 1..log2 k)
 *   POWER_SUM: as POWER, then log2(k) + j = S'_{2^j} (j = 1..log2 k); S'_1 = A
 *   ITERATION: 0 = A, i = T_i (i = 1..k), k + 1 = B, k + 2 = T_0
 *   OLS:       0 = W (n x n), 1 = beta (n x p), 2 = X^T Y (n x p), 3 = X (m x n)
 */
int linview_num_views(const linview_program* prog);
linview_status linview_view_shape(const linview_program* prog, int view_id, int64_t* rows,
                                  int64_t* cols);

/*
 * Copy view ``view_id`` into dst (row-major, ld >= cols).  dst_on_device
 * selects device or host destination.  For a host destination the call
 * synchronises the stream before returning.
 */
linview_status linview_read_view(const linview_program* prog, int view_id, void* dst, int64_t ld,
                                 int dst_on_device, void* stream);

/*
 * Copy rows [row0, row0 + nrows) of view ``view_id`` into dst (nrows x cols,
 * row-major, ld >= cols).  Same device/host rules as linview_read_view.
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
linview_status linview_set_reeval_mode(linview_program* prog, int reeval_mode);

/* Synchronise ``stream`` and return (and clear) the latched device status. */
linview_status linview_sync(linview_program* prog, void* stream);

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
 * linview_level_pass without any device allocation.  The paper has no
 * counterpart: this entry exists for callers that may not allocate device
 * memory on their call path (a process or engine plugin that reserved the GPU's
 * memory up front, or a latency-critical loop that must avoid the implicit
 * synchronisation of cudaMalloc/cudaFree).  Arguments, layouts and results are
 * those of linview_level_pass; the cross-block partial sums live in one array
 * built into the library (16 MiB of device memory, held on every GPU that
 * loads the library until the process exits) instead of stream-ordered
 * allocations.  Sizes whose partial sums do not fit (roughly n * r beyond
 * 8192 * 8 for FP32 on a 152-SM GPU) return LINVIEW_ESHAPE with the needed
 * byte count.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture.  All calls share the array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU race on it and must be serialised.
 * The call synchronises ``stream`` before returning (to read the status word).
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
 */
linview_status linview_set_profiling(linview_program* prog, int enable);
linview_status linview_pass_stats(linview_program* prog, int kernel, int64_t* launches, double* ms,
                                  double* bytes, int64_t* all_launches);
linview_status linview_reset_stats(linview_program* prog);

#ifdef __cplusplus
}
#endif

#endif /* LINVIEW_H_ */
