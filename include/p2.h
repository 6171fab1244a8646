/*
 * p2 — PARAFAC2-ALS (SPARTan formulation) on one NVIDIA GB300 GPU.
 *
 * C ABI of libp2.so.  All compute runs in the library's own CUDA kernels
 * (sm_103a); there is no CPU fallback.  Paper references are to Perros et
 * al., "SPARTan: Scalable PARAFAC2 for Large & Sparse Data", KDD 2017
 * (arXiv:1703.04219).
 *
 * Problem (Section 3.1-3.2): a collection of sparse slices X_k (I_k x J),
 * k = 0..K-1, is modelled as X_k ~ Q_k H S_k V^T with Q_k^T Q_k = I,
 * H (R x R), V (J x R) and S_k = diag(W(k,:)), W (K x R).  One iteration is
 * Algorithm 2's loop body: the Procrustes Q-step for every k, then a single
 * CP-ALS sweep (Algorithm 1) on the implicit tensor Y with slices
 * Y_k = Q_k^T X_k, whose MTTKRPs are Algorithm 3's.
 *
 * Conventions shared by every call:
 *  - Return value: P2_OK (0) or one of the P2_E* codes; a human readable
 *    message for the last failure on the calling thread is p2_last_error().
 *  - Matrices are row-major, indices 0-based, FP32 unless stated.
 *  - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *    Outputs go to caller-allocated buffers.
 *  - Device work is enqueued on the context's stream.  Calls that return
 *    host data (p2_load_slices, p2_iterate with fit_out, p2_fit,
 *    p2_get_*) synchronise that stream before returning.
 *  - A context is not thread safe: one host thread at a time.
 */
#ifndef P2_H
#define P2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    P2_OK = 0,
    P2_EINVAL = 1,     /* invalid argument or malformed slices */
    P2_ENOMEM = 2,     /* device or host allocation failed */
    P2_ECUDA = 3,      /* a CUDA runtime call failed */
    P2_ENUMERIC = 4,   /* non-finite loss detected */
    P2_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
    P2_ESTATE = 6,     /* call out of order (e.g. p2_iterate before p2_init) */
    P2_EEXCHANGE = 7   /* the exchange hook of a sharded context reported a failure */
};

/* Storage precision of V and of the in-flight mode-2 rows P_k = Q_k H S_k (a
 * mixed-precision form of the iteration; the paper itself runs in FP64 on
 * the CPU).  P2_FP32 stores them as float; P2_BF16 stores them as bfloat16
 * (round to nearest even).  H (R x R) and the per-subject Procrustes state
 * T_k stay float in both modes (Q_k = Z_k T_k^T is formed from T_k with a
 * cancellation that amplifies its rounding by the condition number of A_k).
 * All sparse products accumulate in FP32; the Gram, the Procrustes step, the
 * solves and the fit are FP64-accurate. */
enum { P2_FP32 = 0, P2_BF16 = 1 };

typedef struct p2_ctx p2_ctx;

typedef struct {
    int32_t R;            /* target rank, 1 <= R <= 64 */
    int32_t precision;    /* P2_FP32 or P2_BF16 (storage of V and P_k; see above) */
    int32_t device;       /* CUDA device ordinal */
    int32_t use_graph;    /* non-zero: one iteration is captured in a CUDA graph and replayed */
    double rank_rtol;     /* Procrustes rank cut: singular values <= rank_rtol * sigma_1 of
                             X_k V S_k H^T are dropped; <= 0 selects the default 1e-5 */
    void *stream;         /* cudaStream_t to enqueue on; NULL: the context creates its own */
    int32_t timing;       /* non-zero: CUDA events around each phase of an iteration (p2_stats) */
    uint64_t seed;        /* seed of the initial factors p2_init draws when given NULLs */
    int32_t nonneg;       /* non-zero: S_k and V constrained non-negative (Section 5.1), the
                             W and V updates solved row by row as non-negative least squares
                             (one lane per row for R <= 16, one warp per row above) */
    int32_t fp64_procrustes; /* non-zero: the Procrustes step's eigen-decomposition and the
                             formation of T_k run in FP64 on the FP64 pipe (same algorithm,
                             Householder + implicit QR); zero (default): in double-word
                             (float-float) arithmetic on the FP32 pipe, ~2^-46 normwise */
    int32_t autotune;     /* non-zero: the first p2_iterate times the launch choices of
                             p2_tuning on this context's data (split or fused Procrustes
                             step for R >= 2, subject bins on or off for the sparse passes)
                             and keeps the fastest; zero (default): the built-in rules */
    const char *tune_cache; /* nullable: a file of tuned choices, one JSON object per line
                             keyed by rank, precision, variant and the collection's K, J and
                             non-zero count; a matching line is used instead of timing, and a
                             newly timed choice is appended */
    int32_t tensor_core_m; /* R in 13..48, double-word Procrustes step: the matrix
                             M = H S_k G_k S_k H^T whose eigen-decomposition gives the polar
                             factor is formed on the tensor cores (bf16 MMAs made exact by
                             splitting every entry into seven 8-bit digits, FP32 accumulation
                             in tensor memory, the digit products recombined in double-word
                             arithmetic: ~2^-48 normwise, the accuracy of the double-word
                             product it replaces, not its rounding) instead of on the FP32
                             pipe.  Measured slower end to end on GB300 (250M nnz, R = 40:
                             the digit split and recombination cost more FP32-pipe work than
                             the product saves), so it is opt-in: 1 = on for 13 <= R <= 48;
                             0 or -1 (default) = off.  Ignored with fp64_procrustes. */
} p2_options;

/* Launch choices that change the speed, never the results (every choice
 * computes the same values bit for bit). */
typedef struct {
    int32_t procrustes_split;  /* R >= 2, double-word Procrustes step: 1 (default) = split into
                                  a Householder kernel, a one-lane-per-subject QR kernel that
                                  records its Givens rotations, and a kernel that applies them;
                                  0 = one fused kernel */
    int32_t subject_bins;      /* sparse passes take the subjects in bins of their non-zero
                                  count (1), in their own order (0), or by the rule R > 16 (-1,
                                  default) */
    int32_t split_record_cap;  /* split Procrustes step: Givens rotations recorded per subject
                                  (0 = all the scratch holds, 2 R^2 + 2 R); a subject that needs
                                  more is finished by the fused kernel */
    int32_t m2_block_kib;      /* mode-2 pass: row blocks whose P rows take at most this many
                                  KiB, so that they are read back from L2 (0 = one block, the
                                  whole collection: the default, measured fastest at 63M-555M
                                  non-zeros); takes effect at the next p2_load_slices */
} p2_tuning;

int p2_get_tuning(p2_ctx *ctx, p2_tuning *out);
/* How the autotuner chose ("" before it ran; "cache", or the timings it took).
 * The string belongs to the context. */
const char *p2_tuning_note(p2_ctx *ctx);
/* P2_EINVAL for a value out of range; a captured iteration is re-captured. */
int p2_set_tuning(p2_ctx *ctx, const p2_tuning *t);

/* Counters and timings of a context (p2_stats). */
typedef struct {
    int64_t kernel_launches;    /* kernels this context has enqueued (graph replays included) */
    int64_t iterations;         /* ALS iterations completed */
    double polar_fp64_flops;    /* FP64 flops executed by the Procrustes kernel so far
                                   (fused multiply-add = 2), counted from the operations the
                                   kernel performed, including its data-dependent QR steps */
    int32_t n_phases;           /* 7 when timing is on, else 0 */
    float phase_ms[8];          /* last iteration: H solve, pass beta (mode 2), V solve,
                                   pass alpha (mode 3 + W + Gram), Procrustes,
                                   subject statistics (mode 1, W^TW), fit */
} p2_stats_t;

/* Fill *opt with defaults for rank R (precision FP32, device 0, graph on,
 * rank_rtol 1e-5, own stream, timing off, seed 20170314, unconstrained,
 * double-word Procrustes, no autotuning, no tuning cache). */
void p2_default_options(p2_options *opt, int32_t R);

/* Create a context on opt->device.  *out receives the handle (NULL on error).
 * The context owns every device allocation it makes. */
int p2_create(p2_ctx **out, const p2_options *opt);

/* Free the context and all its device memory.  NULL is accepted. */
int p2_destroy(p2_ctx *ctx);

/*
 * Load the collection {X_k} (Algorithm 2, REQUIRE: X_k in R^{I_k x J}).
 *   K         number of subjects, K >= 1
 *   J         number of variables (columns), 1 <= J <= 65535
 *   subj_ptr  int64[K+1]: rows of X_k are subj_ptr[k] .. subj_ptr[k+1]-1 of
 *             the stacked row list; subj_ptr[0] = 0, non-decreasing
 *   row_ptr   int64[N+1], N = subj_ptr[K]: CSR row pointers into col/val;
 *             row_ptr[0] = 0, non-decreasing, at most 65535 entries per row
 *   col       int32[nnz]: column ids in [0, J), strictly increasing in a row
 *   val       float[nnz]: finite values
 *   location  0: all four pointers are host memory; 1: device memory
 * Empty rows and subjects with no rows are allowed (they add nothing to the
 * model; Section 3.3 notes zero rows can be dropped without effect).  Limits:
 * N < 2^31, nnz < 2^31.  Malformed input returns P2_EINVAL; after any
 * failure the context holds no slices (load again).  The columns are relabelled internally by
 * decreasing frequency; every factor the API returns is in the caller's
 * column order.  Synchronises.
 */
int p2_load_slices(p2_ctx *ctx, int64_t K, int32_t J, const int64_t *subj_ptr,
                   const int64_t *row_ptr, const int32_t *col, const float *val,
                   int32_t location);

/*
 * Set the initial factors (Algorithm 2, "Initialize H, V, {S_k}") and run the
 * first Q-step so that p2_iterate can start.  H0: R x R, V0: J x R (caller's
 * column order), W0: K x R; host memory, FP32.  All three NULL: the library
 * draws them uniform in [0, 1) from opt.seed (the paper leaves the
 * initialisation open): element i (row-major) of array a (H: a = 1, V: 2,
 * W: 3) is (x >> 40) 2^-24 for the first SplitMix64 output x (Steele, Lea &
 * Flood, OOPSLA 2014; mixer constants 0xBF58476D1CE4E5B9, 0x94D049BB133111EB)
 * of the state mix(seed + g (t + 1)) ^ mix(i g + t), with t = 5 + 16 a,
 * g = 0x9E3779B97F4A7C15 and mix the SplitMix64 finaliser.  Some but not all
 * NULL: P2_EINVAL.  Any other error leaves the context uninitialised
 * (p2_iterate returns P2_ESTATE until an initialisation succeeds).
 */
int p2_init(p2_ctx *ctx, const float *H0, const float *V0, const float *W0);

/*
 * Deterministic alternative to p2_init, the rational start of Kiers, ten
 * Berge and Bro (J. Chemometrics 13, 1999): H = I, S_k = I (W = 1) and V =
 * the R leading eigenvectors of sum_k X_k^T X_k, in decreasing order of
 * eigenvalue, each column's entry of largest magnitude positive; then the
 * first Q-step, as p2_init.  The eigenvectors come from subspace iteration
 * with a Rayleigh-Ritz step per product on a block of b = min(J, 64,
 * max(2R, R + 8)) columns, so they converge at the rate lambda_{b+1} /
 * lambda_R; the products X^T (X V) run in FP64 without the J x J matrix.
 * The block starts uniform in [0, 1) from opt.seed.  The loop stops when the
 * sum of the squared sines of the principal angles between two successive
 * leading R-dimensional subspaces is at most tol^2, or after max_iter
 * products; a final Rayleigh-Ritz step gives V.  Columns for the null space
 * of sum_k X_k^T X_k, when its rank is below R, are an orthonormal
 * completion.  V is then stored in the context's precision.  Transient
 * device scratch: 4 J b doubles and (N + S) w doubles (N stacked rows, S
 * column segments of the mode-2 layout), the product's column width w <= b
 * chosen so that N w doubles take at most a quarter of the free device
 * memory and 16 GiB.  n_done (nullable, host) receives the iterations run.
 * Synchronises after every product.  P2_EINVAL for J < R, max_iter < 1 or
 * tol < 0 (the context is left as it was); P2_ENUMERIC if an eigen step
 * failed to converge.  Any error other than P2_EINVAL leaves the context
 * uninitialised.
 */
int p2_init_eig(p2_ctx *ctx, int32_t max_iter, double tol, int32_t *n_done);

/*
 * Run n_iter >= 0 iterations of PARAFAC2-ALS (Algorithm 2 loop body: Q-step,
 * one CP-ALS sweep on Y with Algorithm 3's MTTKRPs, S_k = diag(W(k,:))).
 * fit_out (nullable, host): fit after the last iteration, as p2_fit.  With
 * fit_out == NULL the call only enqueues and returns; with fit_out it
 * synchronises and returns P2_ENUMERIC if a non-finite loss was detected
 * (p2_fit reports the same later otherwise).
 */
int p2_iterate(p2_ctx *ctx, int32_t n_iter, double *fit_out);

/*
 * Outer loop of Algorithm 2 with a stopping rule (the paper leaves the
 * convergence criterion open): iterate until the fit changes by at most tol
 * between two iterations, or max_iter iterations.  n_done and fit_out
 * (nullable, host) receive the iterations run and the last fit.  Reads the
 * fit back after every iteration (one synchronisation each).
 */
int p2_iterate_until(p2_ctx *ctx, int32_t max_iter, double tol, int32_t *n_done,
                     double *fit_out);

/*
 * Loss and fit of the last completed iteration (the objective of Section 3.2):
 *   loss = sum_k ||X_k||^2 - 2 <Y_k, H S_k V^T> + ||H S_k V^T||_F^2
 *        = ||X||^2 - 2 <W, M3> + 1^T (W^TW * H^TH * V^TV) 1,
 *   fit  = 1 - sqrt(max(loss, 0)) / ||X||_F.
 * Either pointer may be NULL.  P2_ESTATE before the first iteration.
 */
int p2_fit(p2_ctx *ctx, double *fit, double *loss);

/* Current factors into host buffers (any may be NULL): H R x R, V J x R in
 * the caller's column order, W K x R (W carries the scale; S_k = diag(W(k,:))). */
int p2_get_factors(p2_ctx *ctx, float *H, float *V, float *W);

/*
 * Replace the current factors (host FP32; same layouts as p2_get_factors) and
 * redo the Q-step for them, exactly as p2_init.  Used to resume from a
 * checkpoint.
 */
int p2_set_factors(p2_ctx *ctx, const float *H, const float *V, const float *W);

/*
 * MTTKRPs of the last completed iteration (Algorithm 3), into host FP64
 * buffers: mode 1 -> R x R (M1, with the Y and W of that iteration's H step),
 * mode 2 -> J x R (M2, caller's column order), mode 3 -> K x R (M3).
 */
int p2_get_mttkrp(p2_ctx *ctx, int32_t mode, double *out);

/*
 * Per-subject Procrustes transform of the current Q-step, into a host FP32
 * buffer of (k1 - k0) x R x R: T_k = C_k H S_k, where Q_k = X_k V T_k^T and
 * C_k is the pseudo-inverse square root of (X_k V S_k H^T)^T (X_k V S_k H^T)
 * (polar factor of Section 3.2's Procrustes problem).  0 <= k0 <= k1 <= K.
 */
int p2_get_procrustes(p2_ctx *ctx, int64_t k0, int64_t k1, float *T);

/*
 * The subjects' factor matrices U_k = Q_k H (Algorithm 2's ENSURE output,
 * Section 3.2: X_k ~ U_k S_k V^T), for subjects k0 .. k1-1, into a host FP32
 * buffer of (subj_ptr[k1] - subj_ptr[k0]) x R holding their rows in the
 * stacked row order.  Q_k is the Procrustes factor of the current Q-step,
 * i.e. the one computed for the factors that p2_get_factors returns (the
 * Q-step that opens the next iteration).  Rows of V are gathered per
 * non-zero (Q_k = X_k V T_k^T), so the call costs one pass over the
 * subjects' non-zeros; it allocates a device buffer of the output's size
 * and synchronises.  0 <= k0 <= k1 <= K; U may be NULL only when the range
 * holds no rows.
 */
int p2_get_U(p2_ctx *ctx, int64_t k0, int64_t k1, float *U);

/*
 * Projection of new subjects onto the current model (serving).  For each new
 * subject X (I x J), with the model's H and V fixed, alternate Algorithm 2's
 * Q-step (Procrustes, Section 3.2) and Algorithm 1's W update restricted to
 * that subject (mode-3 MTTKRP, Eq. mttkrp3_row_wise, times (V^TV * H^TH)^+),
 * starting from s = 1, n_iter times.  Subjects are independent: a subject's
 * result does not depend on the batch it is sent in.
 *
 * A projector owns device scratch for batches of at most max_subjects
 * subjects, max_rows rows and max_nnz non-zeros, and its own stream (or the
 * given one); several projectors run their batches concurrently.  The model
 * context must stay loaded and its factors must not change while projectors
 * use it (they read H, V and (V^TV * H^TH)^+ from it at each p2_project).
 */
typedef struct p2_projector p2_projector;
int p2_projector_create(p2_ctx *model, int64_t max_subjects, int64_t max_rows, int64_t max_nnz,
                        void *stream, p2_projector **out);
int p2_projector_destroy(p2_projector *pj);

/* Device bytes a projector of these capacities allocates on the model's
 * device (its scratch: the batch's CSR arrays in both formats and the
 * per-subject Gram, S, T and state), into *bytes.  A server that admits
 * requests by memory sizes its projectors with it. */
int p2_projector_bytes(p2_ctx *model, int64_t max_subjects, int64_t max_rows, int64_t max_nnz,
                       int64_t *bytes);

/*
 * Enqueue the projection of n_req subjects given like p2_load_slices (column
 * ids in the model's original column order; location 0: host, validated on
 * the host before anything is enqueued; 1: device, validated on the device,
 * which costs one synchronisation).  Outputs (out_location 0: host, 1:
 * device): S_out n_req x R FP32, the subjects' S_k diagonals; T_out
 * (nullable) n_req x R x R FP32, the Procrustes transforms for the final s
 * (Q = X V T^T, as p2_get_procrustes).  Returns after enqueueing: host
 * outputs and host inputs must stay valid until p2_projector_sync; use
 * pinned host memory for asynchronous copies.
 */
int p2_project(p2_projector *pj, int64_t n_req, const int64_t *subj_ptr, const int64_t *row_ptr,
               const int32_t *col, const float *val, int32_t location, int32_t n_iter,
               float *S_out, float *T_out, int32_t out_location);

/* Wait until the projector's enqueued work has finished. */
int p2_projector_sync(p2_projector *pj);

/*
 * Subject-sharded form.  The subjects are independent except for a few sums
 * over all of them (Algorithm 3's mode-1 and mode-2 MTTKRPs, W^TW and the
 * loss terms), so a collection may be split into contiguous subject ranges,
 * one context per range (on one GPU or several), each loading only its own
 * slices.  An exchange hook then sums the contexts' partial results, and H
 * and V are solved redundantly (identically) on every shard; W's rows stay
 * with their shard.
 *
 * The hook is called with a device buffer of `count` doubles (on the
 * context's device) and the context's stream, after the work that produced
 * the buffer has been enqueued on that stream.  It must replace the buffer
 * by its elementwise sum over all shards so that work enqueued on `stream`
 * afterwards sees the sum (for example by enqueueing an allreduce on that
 * stream, or by synchronising the stream, combining through the host and
 * copying back), and return 0, or non-zero on failure (the library call
 * then returns P2_EEXCHANGE).  Every shard makes the same sequence of hook
 * calls with the same counts: at p2_load_slices (J + 1 values: column
 * counts, so that every shard relabels the columns alike, and ||X||^2),
 * after every Q-step's statistics (2 R^2 + 1 values: mode 1, W^TW,
 * <W, M3>) and after every mode-2 pass (J R values: M2).  Each sum must be
 * bitwise the same on every shard (an allreduce gives that), so that the
 * replicated H and V stay identical.
 *
 * p2_set_exchange must be called before p2_load_slices (P2_ESTATE
 * otherwise).  A sharded context does not capture its iteration in a CUDA
 * graph (use_graph is ignored), and p2_init_eig returns P2_EINVAL.  fn ==
 * NULL leaves the context unsharded.
 */
typedef int (*p2_exchange_fn)(double *buf, int64_t count, void *stream, void *user);
int p2_set_exchange(p2_ctx *ctx, p2_exchange_fn fn, void *user);

/* Counters and the last iteration's phase timings.  Synchronises. */
int p2_stats(p2_ctx *ctx, p2_stats_t *out);

/* Bytes of device memory the context holds now. */
int p2_device_bytes(p2_ctx *ctx, int64_t *bytes);

/*
 * Mode-1 MTTKRP and W^TW from caller-owned device buffers, allocating no
 * device memory.  The paper has no counterpart: this is a service for callers
 * that cannot call cudaMalloc where they need the reduction (code running
 * while a CUDA graph is captured, real-time loops that must not take the
 * allocator's device-wide synchronisation, hosts that hand out all GPU memory
 * from their own arena).
 *   T    device, K x R x R FP32: per-subject Procrustes transforms, the layout
 *        p2_get_procrustes returns
 *   G    device, K x R(R+1)/2 FP64: per-subject Gram Z_k^T Z_k of Z_k = X_k V,
 *        lower triangle row by row (element (i, j), j <= i, at i(i+1)/2 + j);
 *        each entry is rounded to FP32 before the products, as in the
 *        library's own mode-1 pass
 *   W    device, K x R FP32
 *   M1   device, R x R FP64 out: sum_k (T_k G_k) * 1 W(k,:)  (as p2_get_mttkrp
 *        mode 1 returns for the iteration that starts from this state)
 *   WtW  device, R x R FP64 out, or NULL
 *   stream  cudaStream_t to enqueue on (NULL: the legacy default stream)
 * Limits and behaviour: 1 <= R <= 16 (P2_EINVAL otherwise); every buffer
 * must be device (or managed) memory of the current device, and where the
 * driver reports the extent of the allocation that holds it, large enough
 * for the sizes above (P2_EINVAL otherwise, before anything is enqueued).
 * The scratch is one fixed 541,696-byte array per device, held until the
 * process exits, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Every call looks up
 * the scratch's device address (cudaGetSymbolAddress, which allocates
 * nothing); the first call on a device also loads the library's kernels
 * there, so make that first call before any stream capture.  Returns after
 * enqueueing.
 */
int p2_mode1_stats_noalloc(int64_t K, int32_t R, const float *T, const double *G,
                           const float *W, double *M1, double *WtW, void *stream);

/* Message describing the last error on the calling thread ("" if none). */
const char *p2_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* P2_H */
