/*
 * luqr.h - C interface of the GB300 hybrid LU-QR dense solver.
 *
 * Method: Faverge, Herrmann, Langou, Lowery, Robert, Dongarra, "Designing LU-QR
 * hybrid solvers for performance and stability" (arXiv 1401.5522).  A square
 * matrix of order N is split into n = ceil(N/nb) tile rows/columns of nb x nb
 * tiles.  At every step k (Alg. 1) the diagonal tile is LU-factored with partial
 * pivoting inside the tile, a robustness criterion (Sec. III: Eq. 2 Max, Eq. 3 Sum,
 * Eq. 4 MUMPS) decides between an LU step (Alg. 2, variant A1: GETRF, TRSM,
 * SWPTRSM, GEMM) and a QR step (Alg. 3 with the TS/TT kernels of Alg. 4), and the
 * transformations are applied to [A | b] before one N x N triangular solve
 * (Sec. II-D).
 *
 * Conventions shared by every entry point:
 *  - Matrices are column-major FP64 device arrays with a leading dimension.
 *  - Device pointers are caller-owned; the library never frees them.  A handle
 *    owns all of its own device workspace and releases it in luqr_destroy.
 *  - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Entry points that return device results to
 *    the host (luqr_decisions, luqr_info, luqr_sync, luqr_refine) synchronise
 *    that stream.
 *  - Every call returns an luqr_status code; nothing is thrown across the ABI.
 *    Errors found on the device (singular pivot, non-finite panel) are recorded
 *    in the handle and reported by the next synchronising call.
 *  - N not a multiple of nb is handled by padding the last tile with an identity
 *    block (Sec. II-D, "No restriction on N"); results equal those of native
 *    ragged tiles.
 *  - nb must be a multiple of 32 with 32 <= nb <= 512.
 *  - Distinct handles may be used from distinct host threads.
 */
#ifndef LUQR_H
#define LUQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LUQR_OK = 0,
  LUQR_ERR_INVALID = -1,       /* bad argument (N, nb, lda, alpha, criterion, pointer) */
  LUQR_ERR_NOMEM = -2,         /* device allocation failed */
  LUQR_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  LUQR_ERR_SINGULAR = -4,      /* exact zero pivot where an LU step/back solve needs one */
  LUQR_ERR_NONFINITE = -5,     /* NaN or Inf met in a panel */
  LUQR_ERR_TIMEOUT = -6,       /* a bounded device wait expired */
  LUQR_ERR_NOT_CONVERGED = -7  /* iterative refinement did not reach the tolerance */
} luqr_status;

/* Per-step decision codes returned by luqr_decisions. */
enum { LUQR_DEC_QR = 0, LUQR_DEC_LU = 1, LUQR_DEC_ABORTED = 2 };

/* Robustness criteria (Sec. III).  FORCE_LU is the alpha = infinity limit and
 * FORCE_QR the alpha = 0 limit of Sec. V-B. */
enum { LUQR_MAX = 0, LUQR_SUM = 1, LUQR_MUMPS = 2, LUQR_FORCE_LU = 3, LUQR_FORCE_QR = 4,
       LUQR_RANDOM = 5 };
/* LUQR_RANDOM: the random choice of Sec. V-B (Fig. 2, fourth row): step k is LU with
 * probability alpha/100 (alpha in percent; alpha >= 100 always LU), drawn as
 * u_k = (SplitMix64 output k of the stream seeded with opt->seed >> 11) * 2^-53 and
 * LU iff u_k < alpha/100; a zero pivot in the diagonal GETRF still selects QR.  The
 * margin is log2((alpha/100) / u_k). */

/* QR elimination trees (Alg. 3: the eliminator of each tile is free). */
enum {
  LUQR_TREE_FLAT_TS = 0,   /* eliminator(i,k) = k, TS kernels (Alg. 4a) */
  LUQR_TREE_BINARY_TT = 1, /* binary reduction with TT kernels (Alg. 4b) */
  LUQR_TREE_GROUPED = 2    /* flat TS inside groups of `group` tiles, binary TT across heads */
};

/* Arithmetic of the factorization.  The criterion's norms and comparison are
 * always evaluated in FP64. */
enum {
  LUQR_PREC_FP64 = 0,      /* FP64 tiles and kernels */
  LUQR_PREC_FP32 = 1       /* FP32 tiles and kernels (use luqr_refine for FP64 accuracy) */
};

/* Options; a zero-initialised struct selects the defaults. */
typedef struct luqr_options {
  int tree;                /* LUQR_TREE_*, default flat TS */
  int group;               /* group size for LUQR_TREE_GROUPED (default 4) */
  int precision;           /* LUQR_PREC_* */
  int mumps_mode;          /* 0: est(j) = away(j)*pivot(j)/local(j); 1: cumulative product */
  const uint8_t* forced;   /* optional HOST array of n decisions replacing the criterion */
  const int* inject;       /* optional HOST list of steps whose tile row of [A^(k)|b^(k)] is
                              scaled by 2^-27 before the criterion (run-time injection) */
  int n_inject;
  int fp32_kernels;        /* FP32 only: 0 = default = 2; 1 = CUDA-core trailing updates
                              (fused shared-memory QR kernels, register-tiled GEMM);
                              2 = tcgen05 tensor-core trailing updates (3xTF32) */
  int speculate;           /* predicted-branch speculation (not in the paper; decisions and
                              results are those of the plain method in every mode):
                              0 off; 1 decision-MLP predictor (mlp_params required);
                              2 repeat-the-previous-decision predictor.  A step predicted QR
                              factors its panel on a copy while the diagonal GETRF and the
                              criterion run; the copy is committed when the criterion
                              selects QR and discarded otherwise. */
  int log_features;        /* != 0: store the LUQR_MLP_FEATURES features of every step
                              (read with luqr_features); implied by speculate != 0 */
  const float* mlp_params; /* DEVICE, LUQR_MLP_PARAMS floats (layout at luqr_mlp_forward);
                              read during the factorization, caller-owned */
  int norm_mode;           /* ||A_kk^-1||_1 for Max and Sum: 0 exact (default, X = U^-1 L^-1 P);
                              1 the Hager-Higham estimate (Sec. III-D's iterative O(nb^2)
                              estimate; a lower bound of the exact norm, so LU is admitted at
                              least as often).  luqr_factor only (the batched solver
                              returns LUQR_ERR_INVALID for 1). */
  uint64_t seed;           /* LUQR_RANDOM: SplitMix64 seed of the per-step draws */
  int lu_variant;          /* LU step of Sec. II-B: 0 = A1 (GETRF of the diagonal tile with
                              partial pivoting, default); 1 = A2 (GEQRT of the diagonal tile:
                              ||A_kk^-1||_1 = ||R^-1 Q^T||_1, pivots |R_jj| for MUMPS, a zero
                              on R's diagonal selects QR; an LU step applies Q^T to A_kj and b_k
                              and R^-1 to A_ik).  A2 needs norm_mode = 0 and speculate = 0;
                              luqr_factor only (the batched solver returns LUQR_ERR_INVALID). */
  int timeout_ms;          /* budget of the bounded waits of the persistent second-pass kernel
                              (a task waiting for the tasks it depends on), in milliseconds at
                              the 2.07 GHz maximum SM clock; 0 = default (about 500 ms).  A wait
                              that runs out records LUQR_ERR_TIMEOUT in the handle's status,
                              stops the kernel and leaves the device usable.  The tensor-core
                              update kernel bounds its own waits at about 500 ms. */
  int domain;              /* diagonal-domain pivoting (Sec. II-B, the variant of the paper's
                              experiments): 0 or 1 = partial pivoting inside the diagonal tile
                              (default); d > 1 = the Factor step pivots over tiles k .. k+d-1 of
                              the panel (a tall GETRF), the criterion reads the pivoted panel,
                              and an LU step applies the exchanges to columns k.. of those rows
                              and to b before the tile LU step.  Needs speculate = 0 and
                              lu_variant = 0; luqr_factor only. */
  int tree_small;          /* per-step tree (Alg. 3 leaves the eliminator of each tile free):
                              the tree (LUQR_TREE_*) of the steps below tree_switch */
  int tree_switch;         /* steps with fewer than tree_switch sub-diagonal tiles use
                              tree_small, the others `tree`; 0 (default) uses `tree` at every
                              step.  The Python package's tree autotuner picks (tree,
                              tree_small, tree_switch) by timing. */
  int reserved[3];
} luqr_options;

typedef struct luqr_handle* luqr_handle_t;

/*
 * luqr_factor - hybrid LU-QR factorization (Alg. 1-4, Eq. 1-4).
 *   dA        device, column-major N x N FP64, leading dimension lda >= N; read only.
 *   db        device FP64 vector of length N or NULL.  When given, b is carried as an
 *             augmented column through every step (Sec. II-D) and, after the N x N
 *             triangular solve, overwritten in place with the solution x.
 *   criterion LUQR_MAX / SUM / MUMPS / FORCE_LU / FORCE_QR / RANDOM; alpha >= 0 (may be +inf).
 *             alpha = 0 selects QR at every step.
 *   opt       may be NULL.
 *   stream    CUDA stream; all work is enqueued, nothing is synchronised.
 *   out       receives the new handle (also on device-side errors, which surface later).
 * Returns LUQR_ERR_INVALID for N < 1, nb not in {32,64,...,512}, lda < N, dA NULL,
 * alpha < 0 or NaN, unknown criterion/tree/precision; LUQR_ERR_NOMEM or
 * LUQR_ERR_CUDA when the workspace cannot be set up (then *out is NULL).
 */
int luqr_factor(const double* dA, int64_t lda, double* db, int64_t N, int nb,
                int criterion, double alpha, const luqr_options* opt, void* stream,
                luqr_handle_t* out);

/*
 * luqr_solve - second-pass solve (Sec. II-D): replays every stored LU/QR step on
 * nrhs right-hand sides and back-substitutes.  db: device, column-major N x nrhs
 * FP64 (ldb >= N), overwritten with X.  Work is enqueued on `stream`.
 */
int luqr_solve(luqr_handle_t h, double* db, int nrhs, int64_t ldb, void* stream);

/*
 * luqr_refine - iterative refinement on the original matrix: x <- x + solve(b - A x)
 * with the residual, the update and the backward error in FP64.
 *   dA, lda   the matrix that was factored (device, FP64, read only).
 *   db        device right-hand side (length N, read only).
 *   dx        device output solution (length N).
 *   tol       target normwise backward error ||b-Ax||_inf/(||A||_inf||x||_inf+||b||_inf).
 *   max_iter  maximum number of corrections.
 *   iters     (host, nullable) corrections applied; eta (host, nullable) final error.
 * Synchronises the stream once per iteration.  Returns LUQR_ERR_NOT_CONVERGED when
 * tol was not reached; dx then holds the iterate with the smallest backward error and
 * *eta that error.
 */
int luqr_refine(luqr_handle_t h, const double* dA, int64_t lda, const double* db,
                double* dx, double tol, int max_iter, int* iters, double* eta,
                void* stream);

/*
 * luqr_refine_gmres - GMRES-based iterative refinement (GMRES-IR, Carson and Higham):
 * each correction solves A d = r by restarted GMRES in FP64, left-preconditioned by the
 * handle's factorization applied in its own precision (second pass + back substitution);
 * then x <- x + d and r = b - A x in FP64.  It converges where classic refinement
 * (luqr_refine) stagnates, i.e. when kappa(A) times the factorization's unit roundoff
 * is near or above 1 (for instance FP32 factors of kappa = 1e8 systems).
 *   restart   Krylov basis size per GMRES cycle, 1..200.
 *   max_iter  maximum number of outer corrections.
 *   iters     (host, nullable) total preconditioned GMRES iterations; eta (nullable) final
 *             normwise backward error.
 * Other arguments and errors as luqr_refine.  Synchronises once per GMRES iteration.
 */
int luqr_refine_gmres(luqr_handle_t h, const double* dA, int64_t lda, const double* db,
                      double* dx, double tol, int max_iter, int restart, int* iters, double* eta,
                      void* stream);

/*
 * luqr_debug_replay_skip - test hook for the failure path of the bounded device waits.  The
 * single-vector second pass (luqr_solve with nrhs = 1, and every correction of
 * luqr_refine) runs as one persistent launch of tasks that wait on each other's completion
 * signals; this makes task number `task` (in the launch's program order) skip its signal, so
 * that the next task on the same tile row waits until the handle's timeout_ms budget runs out
 * and the call reports LUQR_ERR_TIMEOUT.  -1 restores normal operation.  LUQR_ERR_INVALID for
 * a NULL handle, a task out of range, or a handle whose second pass takes the per-step
 * launches (FP64 with nb = 512).  Not for production use.
 */
int luqr_debug_replay_skip(luqr_handle_t h, int task);

/*
 * luqr_debug_tc_skip - test hook for the failure path of the bounded waits of the
 * persistent tensor-core update kernel (the FP32 factorization's trailing updates).  While
 * chunk >= 0, CTA 0 of every launch of that kernel leaves the arrival of its raw B chunk
 * number `chunk` unsignalled, so the waits on it run out after the timeout_ms budget of the
 * factorization's options: the kernel records LUQR_ERR_TIMEOUT in the handle's status word,
 * waits (bounded) for its own copies and tensor-core operations, frees its tensor memory
 * and returns, and the later kernels of the factorization exit at once.  Process-wide,
 * applies to launches enqueued after the call; -1 restores normal operation.
 * LUQR_ERR_INVALID for chunk < -1.  Not for production use.
 */
int luqr_debug_tc_skip(int chunk);

/*
 * luqr_accuracy - accuracy of the solution that the last luqr_refine / luqr_refine_gmres
 * call returned (Sec. V-A), from the FP64 infinity norms that refinement computed on the
 * GPU: eta = ||b - A x|| / (||A|| ||x|| + ||b||) (normwise backward error) and
 * HPL3 = ||A x - b|| / (||A|| ||x|| eps N) with eps = 2^-53.  norms (HOST, nullable)
 * receives {||A||, ||b - A x||, ||x||, ||b||}.  Any output may be NULL.  Host-only (no
 * synchronisation).  LUQR_ERR_INVALID before the handle's first refinement.
 */
int luqr_accuracy(luqr_handle_t h, double* eta, double* hpl3, double* norms);

/*
 * luqr_decisions - copies the per-step decisions (LUQR_DEC_*) and margins
 * log2(lhs/rhs) of the criterion (minimum over columns for MUMPS; +-inf for forced
 * steps) to HOST arrays of length n = ceil(N/nb).  margin may be NULL.  *n_out = n.
 * Synchronises the factorization stream; returns the device status.
 */
int luqr_decisions(luqr_handle_t h, uint8_t* dec, double* margin, int* n_out);

/*
 * luqr_step_stats - copies per-step criterion quantities to HOST arrays of length n:
 * lhs = alpha/||A_kk^-1||_1 and rhs = max or sum of ||A_ik||_1 (Max/Sum; NaN otherwise).
 * Either pointer may be NULL.  Synchronises.
 */
int luqr_step_stats(luqr_handle_t h, double* lhs, double* rhs);

/* luqr_factor_data - copies the transformed padded workspace (column-major, n*nb rows,
 * n*nb columns, converted to FP64) to a HOST array with leading dimension ld >= n*nb.
 * Synchronises.  Intended for tests and inspection. */
int luqr_factor_data(luqr_handle_t h, double* host, int64_t ld);

/* luqr_sync - waits for the handle's work and returns its device status. */
int luqr_sync(luqr_handle_t h);

/* luqr_info - device status of the handle and where it was raised (0-based step and
 * row; -1 when not applicable).  Synchronises. */
int luqr_info(luqr_handle_t h, int* status, int* step, int* row);

/* luqr_dims - n (tiles), padded order and the handle's precision. */
int luqr_dims(luqr_handle_t h, int* n, int64_t* npad, int* precision);

/* luqr_destroy - frees the handle's workspace (synchronises its stream first).
 * NULL is accepted. */
void luqr_destroy(luqr_handle_t h);

/*
 * luqr_profile - launch profiler for benchmarks.  With enable != 0 every kernel launch
 * of the library is bracketed by CUDA events recorded on the launch's own stream and
 * attributed to the kernel's name; enable == 0 stops recording.  reset != 0 clears
 * the table.  Process-wide; not meant for concurrent use from several host threads.
 */
int luqr_profile(int enable, int reset);

/*
 * luqr_profile_select - restricts the profiler's CUDA events to the launches whose kernel
 * name is one of names[0..count) (host strings, copied); the other launches are still
 * counted by luqr_profile_read, with 0 ms.  count == 0 times every launch again (default).
 * Keeps the event overhead off a timed run that needs only some kernels' durations.
 * Returns LUQR_ERR_INVALID for count < 0 or names == NULL with count > 0.
 */
int luqr_profile_select(const char* const* names, int count);

/*
 * luqr_profile_trace - the launch timeline recorded while luqr_profile(2, .) (trace mode)
 * was on: for up to cap launches, in the order they were enqueued, the kernel's name
 * (static string owned by the library), start and end in milliseconds since trace mode
 * was switched on (device clock, CUDA events), and the stream the launch ran on (an
 * opaque id).  Waits for the recorded events.  Any array may be NULL.  Returns the number
 * of recorded launches (which may exceed cap; at most 4M are kept).  Enabling with
 * enable == 2 records a base event on the legacy default stream.  Returns LUQR_ERR_INVALID
 * from luqr_profile for enable outside 0..2.
 */
int luqr_profile_trace(const char** names, float* t0_ms, float* t1_ms, uint64_t* stream,
                       int64_t cap);

/*
 * luqr_profile_read - waits for the recorded events, then writes up to cap entries
 * (host arrays): kernel names (static strings owned by the library), launch counts
 * and total device milliseconds.  Any array may be NULL.  Returns the entry count.
 */
int luqr_profile_read(const char** names, int64_t* launches, double* total_ms, int cap);

/*
 * luqr_gemm_sub_f32 - the library's tensor-core update kernel on its own:
 * C <- C - A B for FP32 column-major device matrices (C: M x N, ldc >= M; A: M x K,
 * lda >= M; B: K x N, ldb >= K).  The product runs on the tcgen05 tensor cores with
 * 3xTF32 splitting and FP32 accumulation (about FP32 accuracy).  This is the contraction
 * the factorization uses for its FP32 GEMM trailing updates (Alg. 2, Update).  dstatus
 * (device int[8], nullable) receives LUQR_ERR_TIMEOUT if a bounded internal wait
 * expires.  Enqueued on `stream`; returns LUQR_ERR_INVALID or LUQR_ERR_CUDA on bad
 * arguments or a failed launch.
 */
int luqr_gemm_sub_f32(float* C, int64_t ldc, const float* A, int64_t lda, const float* B,
                      int64_t ldb, int64_t M, int64_t N, int64_t K, int* dstatus, void* stream);

/*
 * Batched solves: many independent systems of uneven order in ONE persistent kernel
 * launch.  Each CTA claims systems largest-first from a device queue and runs the whole
 * hybrid method for one system at a time (Alg. 1-4 with the flat TS tree, in-kernel
 * decisions), back-substitutes the augmented right-hand side and, with precision
 * LUQR_PREC_FP32, refines x with FP64 residuals until eta <= tol (at most max_iter
 * corrections).
 *
 * luqr_batched_create - uploads the description of the batch and allocates scratch.
 *   dA, db   HOST arrays of `count` DEVICE pointers: A_i column-major N_i x N_i (lda = N_i,
 *            read only), b_i of length N_i (overwritten with x_i by luqr_batched_run).
 *   N, nb    HOST arrays: orders (1..8192) and tile sizes (32 or 64) per system (pick nb
 *            with the autotuner of the Python package or pass a fixed value).
 *   criterion, alpha, opt (precision, mumps_mode), tol, max_iter as for luqr_factor/refine.
 * luqr_batched_run - enqueues one persistent launch on `stream`; it allocates nothing and
 *   synchronises nothing.  The batch keeps its own copy of every b_i (taken at create), so
 *   repeated runs solve the same systems and write x_i into the caller's b_i each time.
 * luqr_batched_run_graph - the same work as a CUDA graph: the first call captures the
 *   queue reset and the persistent launch into a graph owned by the batch (on a private
 *   stream), every call launches that graph on `stream`.  LUQR_ERR_CUDA if capture or
 *   instantiation fails.
 * luqr_batched_results - synchronises the device and copies to HOST arrays (any may be
 *   NULL): per-system decisions (count x nmax, LUQR_DEC_*, 255 past the system's last
 *   step), status, refinement iterations and final eta; *nmax_out = nmax.
 * luqr_batched_destroy - frees the batch (synchronises the device first).
 */
/*
 * Decision predictor (not in the paper).  Per step k the factorization can compute
 * LUQR_MLP_FEATURES FP32 features from the panel statistics that precede the criterion
 * (all log2-scaled where they are magnitudes):
 *   0 ||A_kk||_1   1 max_{i>k} ||A_ik||_1   2 sum_{i>k} ||A_ik||_1
 *   3 min_j max_i |A_kk(i,j)|   4 max_j |A_kk(j,j)| / max|A_kk|   5 min_j |A_kk(j,j)| / max|A_kk|
 *   6 max_j log2(away(j)/local(j))   7 mean_j log2(away(j)/local(j))  (away: column max
 *     over the sub-diagonal tiles, local: over A_kk; 64 when local(j) = 0)
 *   8 previous decision (1 LU, 0 QR, 0.5 at k = 0)   9, 10 margins of steps k-1, k-2
 *     (log2(lhs/rhs) of the criterion, clamped to [-64, 64])
 *   11 k/n   12 log2 alpha (64 for infinity)   13 log2 (n - k)   14 criterion / 4
 *   15 fraction of QR steps before k.
 * The network maps 16 -> 64 -> 64 -> 1 with ReLU hidden layers; logit > 0 predicts LU.
 * Parameter vector (FP32, LUQR_MLP_PARAMS): W1[64][16] row-major, b1[64], W2[64][64],
 * b2[64], W3[64], b3.  All pointers are DEVICE pointers; work is enqueued on `stream`.
 *
 * luqr_mlp_forward - dlogits[s] = network(dX[s*16 .. s*16+15]) for s < B (B = 0: no-op,
 *                    pointers may then be NULL).
 * luqr_mlp_grad    - ADDS to dgrad the gradient of the mean binary cross-entropy with
 *                    logits over the batch (labels 1 = LU, 0 = QR) and, if dloss is not
 *                    NULL, adds the mean loss to *dloss.  Zero dgrad/dloss first.
 * luqr_mlp_adam    - one Adam step (Kingma and Ba) at iteration t >= 1 on all parameters
 *                    with first/second moment buffers dm, dv (zero before t = 1).
 * Errors: LUQR_ERR_INVALID for NULL pointers, B < 0 (B < 1 for grad) or t < 1;
 * LUQR_ERR_CUDA if the launch fails.
 *
 * luqr_features - copies the logged features (n x 16, row k = step k) and the
 *   predictions made during the factorization (n bytes, LUQR_DEC_*; NULL to skip)
 *   to HOST arrays.  LUQR_ERR_INVALID when the handle logged no features.
 */
#define LUQR_MLP_FEATURES 16
#define LUQR_MLP_PARAMS 5313
int luqr_mlp_forward(const float* dparams, const float* dX, float* dlogits, int B, void* stream);
int luqr_mlp_grad(const float* dparams, const float* dX, const float* dlabels, int B,
                  float* dgrad, float* dloss, void* stream);
int luqr_mlp_adam(float* dparams, const float* dgrad, float* dm, float* dv, int t, float lr,
                  float beta1, float beta2, float eps, void* stream);
int luqr_features(luqr_handle_t h, float* feat, uint8_t* predicted, int* n_out);

/*
 * Batched solver: many independent systems A_i x_i = b_i of uneven order N_i, each solved
 * by the hybrid method (Alg. 1 with Eq. 2-4, the LU step of Alg. 2, the QR step of Alg. 3
 * with the flat TS tree of Alg. 4(a), back substitution of the augmented right-hand side,
 * Sec. II-D) inside ONE persistent launch: each CTA claims the next system from a queue
 * ordered largest first, copies it into its own padded scratch slot and decides every
 * step in-kernel.  Not in the paper (its experiments solve one system at a time).
 *
 * luqr_batched_create - sets up a batch; nothing runs yet.
 *   dA        HOST array of `count` DEVICE pointers; dA[i] is column-major FP64 N[i] x N[i]
 *             with leading dimension N[i]; read only, caller-owned, valid until destroy.
 *   db        HOST array of `count` DEVICE pointers to FP64 vectors of length N[i]; every
 *             run overwrites db[i] with x_i.  The batch keeps its own copy of the right-hand
 *             sides taken at create time, so runs are repeatable.
 *   N, nb     HOST arrays: order 1 <= N[i] <= 8192 and tile size nb[i] in {32, 64}.
 *   criterion LUQR_MAX / SUM / MUMPS / FORCE_LU / FORCE_QR (not RANDOM); alpha >= 0.
 *   opt       may be NULL; uses precision (FP64, or FP32 tiles with FP64 refinement inside
 *             the kernel) and mumps_mode; norm_mode must be 0; the other fields are ignored.
 *   tol, max_iter  FP32 mode: refine until eta <= tol, at most max_iter corrections.
 *   out       receives the batch (device workspace: one slot per resident CTA plus the
 *             per-system results), owned by the batch until luqr_batched_destroy.
 * Synchronous (copies the metadata to the device).  Returns LUQR_ERR_INVALID for NULL
 * arrays, count < 1, a size or tile size outside the limits, a bad criterion, alpha < 0 or
 * NaN, tol < 0 or max_iter < 0, bad options; LUQR_ERR_NOMEM / LUQR_ERR_CUDA when the
 * workspace cannot be set up (then *out is NULL).
 *
 * luqr_batched_run       - enqueues one solve of every system on `stream` (one launch).
 * luqr_batched_run_graph - the same through a CUDA graph, captured on a private stream at
 *                          the first call and replayed on `stream` afterwards.
 *   Both return LUQR_ERR_INVALID for a NULL batch and LUQR_ERR_CUDA if the launch fails.
 * luqr_batched_results - synchronises the device, then copies to HOST arrays (any may be
 *   NULL): dec (count x nmax bytes, row i = system i's decisions LUQR_DEC_*, 255 for steps
 *   past its last tile), status (count ints, LUQR_OK or LUQR_ERR_*), iters (refinement
 *   corrections used), eta (normwise backward error per system), *nmax_out (the largest
 *   tile count).  Returns LUQR_ERR_CUDA if the device reports an error.
 * luqr_batched_destroy - synchronises the device and frees the batch (NULL: no-op).
 */
typedef struct luqr_batched* luqr_batched_t;
int luqr_batched_create(const double* const* dA, double* const* db, const int* N, const int* nb,
                        int count, int criterion, double alpha, const luqr_options* opt,
                        double tol, int max_iter, luqr_batched_t* out);
int luqr_batched_run(luqr_batched_t b, void* stream);
int luqr_batched_run_graph(luqr_batched_t b, void* stream);
int luqr_batched_results(luqr_batched_t b, uint8_t* dec, int* status, int* iters, double* eta,
                         int* nmax_out);
void luqr_batched_destroy(luqr_batched_t b);

/* Maximum sizes accepted by luqr_panel_test_noalloc (its scratch is a fixed array). */
#define LUQR_NOALLOC_MAX_NB 256
#define LUQR_NOALLOC_MAX_TILES 1024

/*
 * luqr_panel_test_noalloc - the per-step robustness test of one panel (panel statistics,
 * LU with partial pivoting of a scratch copy of the diagonal tile, exact ||A_kk^-1||_1 and
 * the Max / Sum / MUMPS comparison) without allocating any device memory.  The paper has
 * no counterpart: this entry exists for callers that cannot call cudaMalloc, e.g. code
 * confined to a pre-reserved memory budget or to a pool that the host application owns,
 * or latency-critical paths that must not wait on the allocator (which can synchronise
 * the device).
 *   dpanel    device, column-major FP64 panel of `rows` x nb: the diagonal tile on top,
 *             then the (rows/nb - 1) sub-diagonal tiles; leading dimension ld >= rows.
 *   rows      a multiple of nb, at most LUQR_NOALLOC_MAX_TILES * nb (pad with zero tiles).
 *   nb        multiple of 32 with 32 <= nb <= LUQR_NOALLOC_MAX_NB.
 *   criterion LUQR_MAX, LUQR_SUM, LUQR_MUMPS, LUQR_FORCE_LU or LUQR_FORCE_QR; LUQR_RANDOM
 *             is not accepted (its draw needs the step index of a whole factorization) and
 *             returns LUQR_ERR_INVALID.  alpha >= 0 and mumps_mode (0 or 1) as luqr_factor.
 *   ddec      device uint8: receives LUQR_DEC_LU, LUQR_DEC_QR, or LUQR_DEC_ABORTED when the
 *             panel holds a NaN/Inf or FORCE_LU meets an exact zero pivot.
 *   dmargin   device double: log2(lhs/rhs) of the test (as luqr_decisions).
 * Work is enqueued on `stream`; nothing is synchronised and no device memory is allocated
 * or freed.  Scratch: one file-scope device array of about 0.53 MB per GPU, shared by every
 * call and kept until the process exits.  Calls that overlap on the GPU (different streams
 * or devices sharing the array's contents on one GPU) race on it and must be serialised by
 * the caller.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture begins.  Returns LUQR_ERR_INVALID for sizes beyond the limits above or bad
 * arguments, LUQR_ERR_CUDA if the set-up or a launch fails, or if an earlier launch left
 * a CUDA error pending (the call then runs nothing and leaves that error in place).
 */
int luqr_panel_test_noalloc(const double* dpanel, int64_t ld, int64_t rows, int nb, int criterion,
                            double alpha, int mumps_mode, uint8_t* ddec, double* dmargin,
                            void* stream);

/* luqr_status_string - static text for a status code. */
const char* luqr_status_string(int status);

/* luqr_version - library version string. */
const char* luqr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LUQR_H */
