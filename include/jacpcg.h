/*
 * jacpcg.h -- C ABI of the GB300 (sm_103a) Jac-PCG regularized zero-forcing
 * precoder library.
 *
 * The operation (arXiv 2305.13925, Xu, Zhang, Li, Xiao, Ai):
 *   for each channel H (M base-station antennas x K single-antenna users,
 *   complex), form the regularised Gram matrix A = H^H H + xi I (Sec. II,
 *   definition of P_i after Eq. 7), solve A X = I_K by Jacobi-preconditioned
 *   conjugate gradients (Sec. III-B Steps 1-4, Eqs. 19-21, Algorithm 1),
 *   and form the unnormalised precoder W = H X (Eq. 7; Eq. 15 per symbol)
 *   with its power factor beta = sqrt(P / ||W||_F^2) (Sec. II after Eq. 7).
 *
 * Layout.  Complex values are complex64: two float32 (re, im) interleaved.
 * Matrices are column-major: element (m, k) of H sits at H[m + k * ldh].
 * W is M x K with leading dimension ldw; X and A are K x K with leading
 * dimension K.  All H / W / X / A pointers are DEVICE pointers owned by the
 * caller, 16-byte aligned, and must stay valid until the work enqueued on
 * the stream has completed.  The library never frees or retains them.
 *
 * Errors.  Every call returns a jacpcg_status.  Call-level errors (invalid
 * arguments, out of memory) leave all outputs untouched.  Per-instance
 * outcomes (not converged, not Hermitian positive definite, non-finite
 * values) are written to the caller's per-instance status array on the
 * device.  No call aborts, traps or throws across this boundary.  A CUDA
 * error reported by the runtime maps to JACPCG_ECUDA and leaves the context
 * unusable (destroy it).
 *
 * Threading.  A context (and each plan made from it) may be used from one
 * host thread at a time.  Work is enqueued asynchronously on the stream the
 * caller passes (a cudaStream_t, passed as void*; NULL is the legacy
 * default stream); the caller synchronises.
 */
#ifndef JACPCG_H
#define JACPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JACPCG_OK = 0,
    JACPCG_EINVAL = 1,      /* invalid argument (null pointer, size limit, alignment) */
    JACPCG_ENOMEM = 2,      /* device or pinned host memory exhausted, or arena budget */
    JACPCG_ECUDA = 3,       /* CUDA runtime error; the context is unusable afterwards */
    JACPCG_ENOTCONV = 4,    /* per instance: tolerance not met within max_iter */
    JACPCG_ENOTHPD = 5,     /* per instance: d^H A d <= 0 met, A is not positive definite */
    JACPCG_ENONFINITE = 6,  /* per instance: NaN or Inf in W */
    JACPCG_ETIMEOUT = 7,    /* a bounded wait ran out (serving) */
    JACPCG_EBUSY = 8        /* serving queue full or ticket still in flight */
} jacpcg_status;

/* Iteration form (Sec. III-B).  STANDARD: Steps 1-4 with C = D (Eq. 21),
 * written in residual form with the standard PCG step and direction ratios
 * (the printed ratio of Eq. 20 is garbled).  ALG1: Algorithm 1 as printed
 * (conjugate gradients with Euclidean inner products on the left-scaled
 * system D^{-1} A X = D^{-1} B; its step alpha is complex).  CG: plain
 * conjugate gradients (C = I).  JOR: the stationary Jacobi over-relaxation
 * of Sec. III-A, w^{t+1} = (I - omega D^{-1} A) w^t + omega D^{-1} b, run in
 * residual form (x += omega D^{-1} r, r -= A omega D^{-1} r) with the
 * instance's omega; it converges for 0 < omega < 2 / lambda_max(D^{-1} A)
 * (the paper gives no omega).  Algorithm 1 and JOR run on the SIMT kernels.
 * DIRECT: the direct RZF the paper compares against (Appendix): P = L L^H
 * by Cholesky, then X = P^{-1} B by forward and back substitution, in FP32;
 * max_iter, tol and X0 are ignored, iters and resid report 0, a pivot <= 0
 * gives NOTHPD (X = 0); refinement is not offered with it (EINVAL). */
enum { JACPCG_STANDARD = 0, JACPCG_ALG1 = 1, JACPCG_CG = 2, JACPCG_JOR = 3, JACPCG_DIRECT = 4 };

/* Arithmetic of the Gram and W = H X contractions.
 * FP32:   FP32 FMA on the SIMT pipes.
 * TF32X3: tensor cores (tcgen05, kind::tf32) with each FP32 operand split
 *         into a TF32 head and a TF32 tail, three products accumulated in
 *         FP32 (about FP32 accuracy).
 * The iteration's vectors and scalars are FP32 in both cases; with TF32X3
 * its product A P runs on the tensor cores (standard and CG forms): in
 * 3xTF32 for the 64 class, and for the 128 and 256 classes as FP16 heads and
 * tails of A and P scaled by exact powers of two (22 bits per entry, every
 * product exact).  Every per-column dot product whose terms can cancel (p^H A
 * p; Algorithm 1's complex denominator) is compensated (Dot2); the squared
 * norms r^H D^{-1} r and ||r||^2 are sums of nonnegative terms (no
 * cancellation), compensated on the SIMT kernel and summed pairwise (a few
 * ulps) on the tensor-core kernels.  Refinement correction solves of the 128
 * and 256 classes run with refine_solve_tol >= 5e-3 on the FP16 heads alone
 * (11 bits) with plain pairwise p^H A p: the next accurate residual corrects
 * what such a loose solve leaves. */
enum { JACPCG_FP32 = 0, JACPCG_TF32X3 = 1 };

/* Storage type of H (jacpcg_instance.h_dtype).  BF16: each complex entry is
 * two bfloat16 (re, im), 4 bytes, column-major with leading dimension ldh
 * (entries); the values are used exactly (bfloat16 converts to FP32 and
 * TF32 without rounding).  W, X and A are complex64 in both cases. */
enum { JACPCG_H_C64 = 0, JACPCG_H_BF16 = 1 };

/* Evaluation of the refinement residual R = I - A X (jacpcg_config.refine_residual).
 * DOT2: FP32 error-free transformations (TwoProduct by FMA + TwoSum, the
 * compensated dot product of Ogita, Rump and Oishi, 2005), as accurate as
 * twice the working precision, on the FP32 pipes.  FP64: products and sums
 * in FP64 (exact products of the FP32 operands); slower on this GPU.
 * SLICED: for the K = 128 and 256 classes, products on the FP16 tensor cores
 * (the Ozaki scheme on tensor cores: Mukunoki, Ozaki, Ogita and Imamura, ISC
 * 2020).  A and X are balanced by exact powers of two near sqrt(diag A), and
 * each row of the balanced A and each column of the balanced X is cut into five
 * 8-bit integer slices on fixed-point grids of their own; slice products are
 * exact, the sums of the fifteen kept slice pairs are exact (the top class to
 * one unit of 2^-46 of its grid), and the classes are combined with B by TwoSum
 * pairs and rounded once.  On the bench channels R comes out within 1e-4 of its
 * own size (Dot2: within FP32 rounding), far more than the FP32 correction
 * solves can use.  The other classes, and channels with M <= 2 K, use DOT2.
 * Requires the entries of A and X within 2^-60 .. 2^60 of magnitude. */
enum { JACPCG_RESID_DOT2 = 0, JACPCG_RESID_FP64 = 1, JACPCG_RESID_SLICED = 2 };

/* config flags */
enum {
    JACPCG_FLAG_PROFILE = 1,         /* record per-phase CUDA events on each execute */
    JACPCG_FLAG_SIMT_ITERATION = 2,  /* TF32X3: keep the iteration of every class on the FP32 SIMT
                                        kernel (by default the A P product of the 64, 128 and 256
                                        classes runs on the tensor cores for the standard and CG
                                        forms) */
    JACPCG_FLAG_REFINE_SELECTIVE = 4 /* with refine_sweeps > 0: refine only the channels with
                                        M <= 2 K (few antennas per user: Jacobi-scaled condition
                                        numbers up to thousands); the others keep the iteration's
                                        result, whose W lies within a few 1e-6 of the RZF at a 1e-5
                                        tolerance on the channels of Sec. II.  Their residual is not
                                        evaluated and resid_hist is not written for them */
};
/* Other flag bits are rejected (EINVAL). */

typedef struct {
    int device;              /* CUDA device ordinal */
    int max_instances;       /* most instances in one plan or precode call (>= 1) */
    int max_M;               /* largest M accepted (>= 1) */
    int max_K;               /* largest K accepted, 1 <= max_K <= 256 */
    size_t arena_bytes;      /* device workspace arena; 0 = sized for one call at the limits */
    int precision;           /* JACPCG_FP32 or JACPCG_TF32X3 */
    int variant;             /* JACPCG_STANDARD, JACPCG_ALG1, JACPCG_CG, JACPCG_JOR or
                                JACPCG_DIRECT */
    int flags;               /* JACPCG_FLAG_* */
    int refine_sweeps;       /* 0..3 iterative-refinement sweeps after the solve: R = I - A X
                                evaluated as refine_residual says, A dX = R solved by the same
                                FP32 iteration (the instance's max_iter and tol, relative to
                                ||R||), X += dX.  After the last sweep R is evaluated once more
                                only when some instance of the call asks for resid_hist (it
                                could change nothing else) */
    int refine_residual;     /* JACPCG_RESID_DOT2 (default), JACPCG_RESID_FP64 or
                                JACPCG_RESID_SLICED.  With
                                refinement, channels with M <= 2 K form A with compensated
                                (Dot2) sums on the SIMT pipes instead of the FP32 / 3xTF32
                                Gram: refinement converges to the solution for the A it is
                                given, and these channels' Jacobi-scaled condition numbers
                                (up to thousands) would turn an FP32 Gram's rounding into an
                                error floor near 1e-5 in W */
    float refine_tol;        /* 0 (default): every sweep runs for every instance.  > 0: an
                                instance stops refining (its remaining correction solves and
                                residual evaluations are skipped) once its largest per-column
                                relative true residual ||B_j - A X_j|| / ||B_j|| is at most
                                refine_tol, or has not fallen below half its value before the
                                last sweep (the FP32 iteration's floor); finite, >= 0 */
    float refine_solve_tol;  /* 0 (default): each correction solve A dX = R stops a column at the
                                instance's tol relative to ||R_j||.  > 0: at this tolerance
                                instead (a sweep needs only to cut the error by a fixed factor;
                                the residual is recomputed accurately before the next one).  The
                                solve still stops at the instance's max_iter; finite, >= 0 */
} jacpcg_config;

typedef struct {
    int M, K;                /* 1 <= K <= max_K, K <= M <= max_M (K > M needs xi > 0) */
    int ldh;                 /* leading dimension of H, >= M, even */
    const void *H;           /* device, complex64 M x K column-major, 16-byte aligned */
    double xi;               /* regulariser, >= 0 (> 0 when K > M) */
    double power;            /* total transmit power P for beta; <= 0 means 1 */
    void *W;                 /* device out, complex64 M x n column-major (n = K, or n_rhs when B
                                is given): W = H X, the precoder of Eq. 7 (B = I) or the
                                transmit block of Eq. 15 (before the power factor) */
    int ldw;                 /* leading dimension of W, >= M, even */
    void *X;                 /* optional device out, complex64 K x n (ld K): the iterate */
    void *A;                 /* optional device out, complex64 K x K (ld K): H^H H + xi I */
    int max_iter;            /* T, 0 <= T <= 4096 */
    float tol;               /* > 0: stop a column once ||r|| <= tol ||b||; <= 0: exactly T steps */
    int h_dtype;             /* JACPCG_H_C64 (0) or JACPCG_H_BF16 */
    float *resid_hist;       /* optional device out, refine_sweeps + 1 floats: ||B - A X||_F / sqrt(n)
                                before each sweep and after the last, evaluated as the
                                refinement residual (Dot2 by default, FP64 on request) */
    /* Right-hand sides, Eq. 16 per symbol vector: P w = s for the n_rhs columns
     * s of B (Sec. III, "Stationary Iterative Methods", Eqs. 15-16).  NULL: B = I_K,
     * the RZF precoder of Eq. 7.  With B, beta normalises the block's mean
     * transmit power: beta = sqrt(P n_rhs / ||W||_F^2), which is Eq. 7's beta in
     * expectation over unit-power symbols. */
    const void *B;           /* optional device in, complex64 K x n_rhs column-major, 16-byte aligned */
    int ldb;                 /* leading dimension of B, >= K */
    int n_rhs;               /* columns of B: 1 .. the K class (8, 16, .. 256: the next power of
                                two >= max(K, 8)); ignored when B is NULL */
    const void *X0;          /* optional device in, complex64 K x n (ld K), 16-byte aligned: the
                                initial point of the iteration (Sec. III-B Step 1; e.g. the
                                previous slot's X); NULL: 0.  The tolerance stays relative to
                                ||b||; iters counts the updates after X0 */
    float omega;             /* JOR relaxation factor (variant JACPCG_JOR only), 0 <= omega < 2;
                                0 means 1 (the Jacobi iteration); e.g. 2 / (lambda_min +
                                lambda_max) of D^{-1} A, which always converges */
    float *sinr;             /* optional device out, K floats: the per-user SINR of Eq. 9
                                (centralised form, single-antenna users, G = beta W):
                                gamma_k = beta^2 |h_k^H w_k|^2 / (beta^2 sum_{j!=k}
                                |h_k^H w_j|^2 + noise), computed on the GPU from this call's W
                                and beta after the precoder; the sum SE of Eq. 10 is
                                sum_k log2(1 + gamma_k).  Only with B = NULL (EINVAL otherwise);
                                4-byte aligned */
    float noise;             /* noise power sigma^2 of sinr; 0 means 1; finite, >= 0 */
} jacpcg_instance;

typedef struct jacpcg_ctx jacpcg_ctx;
typedef struct jacpcg_plan jacpcg_plan;

/* Create a context on cfg->device: validates the limits, reserves the
 * device workspace arena and pinned staging memory, and encodes the arena's
 * tensor map (rows of 256 bytes, for the iteration's tiled copies).  *out
 * receives the context.  Errors: EINVAL (bad limits), ENOMEM (arena), ECUDA
 * (events, streams, or the driver's tensor-map encoder unavailable). */
jacpcg_status jacpcg_create(const jacpcg_config *cfg, jacpcg_ctx **out);

/* Precode n_inst independent channels in one batched launch sequence on
 * `stream` (Eq. 7 for each instance with B = I_K, or Eqs. 15-16 for a block
 * of symbol vectors B, from X0 when given).  inst[i] describes instance
 * i (host array, read during the call).  Per-instance outputs are device
 * arrays of n_inst entries (any may be NULL): status (jacpcg_status per
 * instance), iters (largest per-column iteration count), resid (largest
 * per-column recurrence residual ||r|| / ||b||), beta (power factor; 0 when
 * W = 0, e.g. max_iter = 0 or an all-zero channel, where it is undefined).
 * n_inst = 0 is an empty batch: nothing is enqueued and JACPCG_OK returned
 * (inst may then be NULL).
 * The call waits, on the host, until the previous precode call of this
 * context has finished reading its staging memory; it does not wait for
 * the GPU work it enqueues.  Calls on one context must use one stream (or
 * be ordered by the caller).  Errors: EINVAL, ENOMEM, ECUDA. */
jacpcg_status jacpcg_precode(jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst,
                             int32_t *status_dev, int32_t *iters_dev, float *resid_dev,
                             float *beta_dev, void *stream);

/* Plans: the same work as jacpcg_precode, prepared once (instance table,
 * tile lists and workspace resident on the device, carved from the context
 * arena) and executed any number of times.  With use_graph != 0 the first
 * execute captures the whole launch sequence into one CUDA graph and every
 * execute replays it (graph replays are not profiled).  Plans of one context may
 * execute concurrently on different streams (each owns its workspace).
 * Errors: EINVAL, ENOMEM (arena budget), ECUDA. */
jacpcg_status jacpcg_plan_create(jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst,
                                 int32_t *status_dev, int32_t *iters_dev, float *resid_dev,
                                 float *beta_dev, int use_graph, jacpcg_plan **out);
jacpcg_status jacpcg_plan_execute(jacpcg_plan *plan, void *stream);
jacpcg_status jacpcg_plan_destroy(jacpcg_plan *plan);

/* Bytes of arena workspace a plan for these instances needs, and bytes
 * still free in the context arena (for admission control). */
jacpcg_status jacpcg_plan_bytes(const jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst,
                                size_t *bytes);
jacpcg_status jacpcg_arena_free_bytes(const jacpcg_ctx *ctx, size_t *bytes);

/* Per-phase device time of the executes (plan executes and precode calls,
 * not graph replays) made since the previous read, when the context was
 * created with JACPCG_FLAG_PROFILE.  Events are recorded on the caller's
 * stream around each phase; this call waits for the last of them.
 * ms[0..3] = total milliseconds in Gram, iteration, W = H X, finalise
 * (summed over K classes and executes); *n_executes = executes covered (at
 * most 4096 are recorded between reads); *launches_per_execute = kernels
 * the last execute launched.  Resets the record. */
jacpcg_status jacpcg_profile_read(jacpcg_ctx *ctx, float ms[4], int *n_executes,
                                  int *launches_per_execute);

/* ---- autotuning --------------------------------------------------------
 * Per K class the iteration runs either on the tensor cores (shape -1: the
 * 64 class's kernel with A in tensor memory, or the 128 / 256 classes'
 * kernel with A streamed; allowed with TF32X3, STANDARD or CG and without
 * JACPCG_FLAG_SIMT_ITERATION) or on the SIMT kernel in one of several launch
 * shapes (0 .. n_shapes - 1: columns per warp x warps per CTA; all SIMT
 * shapes give bit-identical results; the tensor path agrees with them within
 * the FP32 tolerance).  The default is -1 (SIMT shape 0 where the tensor path
 * is not allowed).  jacpcg_autotune times every candidate -- the tensor path
 * where allowed, then each SIMT shape -- on the instances of each K class
 * present in inst[0..n) (a plan of that class alone, 2 warm-up and 5 timed
 * executes, CUDA events on `stream`, which it synchronises) and keeps the
 * fastest in the context for later plans and calls: small batches of a
 * class can run faster on the SIMT kernel, which spreads one instance over
 * more CTAs.  If table is not NULL it receives a NUL-terminated JSON object
 * (truncated to table_cap bytes):
 *   {"<K class>": {"shape": i, "path": "tensor"|"simt", "cols_per_warp": c,
 *                  "warps_per_cta": w, "instances": n, "candidates": [...],
 *                  "ms_per_candidate": [...]}, ...}
 * which a caller can persist and replay with jacpcg_set_shape.
 * Errors: EINVAL, ENOMEM, ECUDA. */
jacpcg_status jacpcg_autotune(jacpcg_ctx *ctx, const jacpcg_instance *inst, int n_inst,
                              void *stream, char *table, size_t table_cap);
/* Choose candidate `shape` for K class k_class (8, 16, ..., 256): -1 the
 * tensor-core path where allowed (the default), 0 .. n_shapes - 1 a SIMT
 * launch shape.  EINVAL outside -1 .. n_shapes - 1. */
jacpcg_status jacpcg_set_shape(jacpcg_ctx *ctx, int k_class, int shape);
/* Current choice of a K class (-1 when the tensor path is in use), the
 * number of SIMT shapes, and the SIMT geometry (of shape 0 for the tensor
 * path). */
jacpcg_status jacpcg_get_shape(const jacpcg_ctx *ctx, int k_class, int *shape, int *n_shapes,
                               int *cols_per_warp, int *warps_per_cta);

/* Description of the CUDA error that made the context unusable (after an
 * ECUDA), or "no error".  Static string. */
const char *jacpcg_last_cuda_error(const jacpcg_ctx *ctx);

/* Kernels launched by this context since creation (all entry points). */
int64_t jacpcg_launch_count(const jacpcg_ctx *ctx);

/* ---- serving: continuous batching of precoding requests -----------------
 * A server owns a context (do not use that context elsewhere while the
 * server lives) and a scheduler thread.  Each request is one instance whose
 * H and W are device buffers that stay valid until the request completes.
 * While fewer than max_inflight batches are on the GPU, the scheduler takes
 * the waiting requests (at most max_batch; by default only those of the
 * oldest waiting request's cost class, see batch_policy), admits them if the
 * context arena has room for their plan (else it waits for a running batch
 * to retire, or launches fewer), and runs them as one ragged batch on its
 * own stream: requests that arrive while others run join the next batch and
 * their work overlaps on the device.  Results are bitwise the same as the
 * request's result alone.  Latency = host time from submit to the end of
 * its batch on the GPU (a host callback on the batch's stream). */
typedef struct jacpcg_server jacpcg_server;
typedef struct {
    int max_batch;          /* most requests per launched batch (>= 1) */
    int max_inflight;       /* batches on the GPU at once, 1..64 (one stream each) */
    int max_queue;          /* waiting requests before submit returns EBUSY; <= 0: unbounded */
    int plain;              /* 1: run each batch with the plain per-instance comparator
                               (jacpcg_precode_plain) instead of the batched path */
    int plain_variant;      /* iteration form for plain = 1 */
    int batch_policy;       /* JACPCG_BATCH_COST_CLASS (0, default) or JACPCG_BATCH_FIFO */
} jacpcg_server_config;

/* Batch formation (jacpcg_server_config.batch_policy).  A batch ends when its
 * slowest request does, so one expensive request delays every request
 * launched with it.  COST_CLASS: a batch takes, in arrival order, only the
 * waiting requests of the oldest waiting request's cost class -- the K class
 * (8 .. 64, 128, 256), with K = 256 split further into channels with
 * M >= 4 K and the rest (near-square channels, often ill-conditioned and
 * slow to converge) -- so cheap requests never wait inside an expensive
 * batch, and the classes overlap on the device in separate batches; the two
 * 256-user classes hold at most max_inflight - 1 of the in-flight batches at
 * once (with max_inflight >= 2), so a slot always stays for the cheaper
 * classes.  FIFO: every waiting request in arrival order. */
enum { JACPCG_BATCH_COST_CLASS = 0, JACPCG_BATCH_FIFO = 1 };

jacpcg_status jacpcg_server_create(jacpcg_ctx *ctx, const jacpcg_server_config *cfg,
                                   jacpcg_server **out);
/* Queue one request; *ticket identifies it.  Thread-safe.  Errors: EINVAL
 * (invalid instance), EBUSY (queue full or shutting down), ECUDA. */
jacpcg_status jacpcg_submit(jacpcg_server *srv, const jacpcg_instance *inst, uint64_t *ticket);
/* Result of a request: returns EBUSY while it runs (blocking == 0), or waits
 * (at most 60 s, then ETIMEOUT).  On JACPCG_OK, *result is the request's
 * status (as jacpcg_precode's per-instance status) and *latency_us (may be
 * NULL) its latency; the ticket is then forgotten.  Thread-safe. */
jacpcg_status jacpcg_poll(jacpcg_server *srv, uint64_t ticket, jacpcg_status *result,
                          double *latency_us, int blocking);
/* Load driver: submit request i (instance pool[which[i]]) at arrival_us[i]
 * microseconds after the call starts (open loop, busy-waiting on a steady
 * clock), then collect every result.  latency_us / status (may be NULL)
 * receive n_req values (latency -1 when a request was refused). */
jacpcg_status jacpcg_server_replay(jacpcg_server *srv, const jacpcg_instance *pool, int n_pool,
                                   const int *which, const double *arrival_us, int n_req,
                                   double *latency_us, int32_t *status);
/* Requests completed, batches launched and the mean batch size so far. */
jacpcg_status jacpcg_server_stats(jacpcg_server *srv, uint64_t *n_done, uint64_t *n_batches,
                                  double *mean_batch);
/* Drain the queue, wait for running batches, free the server (not the context). */
jacpcg_status jacpcg_server_destroy(jacpcg_server *srv);

/* The plain FP32 per-instance comparator: the same precoder (same variant
 * semantics, Eq. 7 with B = I) computed one instance at a time with simple
 * one-thread-per-entry SIMT kernels, one launch per step and per iteration,
 * plain FP32 sums, no batching, no CUDA graphs, no tensor cores.  It is the
 * baseline the batched path is measured against.  No context: the caller
 * passes a device workspace of at least 5 K^2 * 8 + 16 K + 256 bytes for the
 * largest K of the batch (ENOMEM otherwise).  Per-instance outputs as in
 * jacpcg_precode.  B, X0 and sinr must be NULL.  Errors: EINVAL, ENOMEM, ECUDA. */
jacpcg_status jacpcg_precode_plain(const jacpcg_instance *inst, int n_inst, int variant,
                                   void *workspace, size_t workspace_bytes, int32_t *status_dev,
                                   int32_t *iters_dev, float *resid_dev, float *beta_dev,
                                   void *stream);

/* Precode without allocating anything (no counterpart in the paper: this
 * is an integration aid).  For callers that cannot call cudaMalloc or any
 * allocating routine -- real-time slot loops that forbid allocator latency,
 * integrations whose memory was fixed at start-up.  The same work and SIMT
 * kernels as jacpcg_precode with a context of the given variant (STANDARD,
 * ALG1 or CG) and FP32 precision, each K class on its default launch shape (a context's
 * autotuner may pick another, so W agrees with jacpcg_precode within the
 * 1e-5 relative W tolerance, not bit for bit), but no context: the tables,
 * accumulators and Gram / iterate workspace live in one static device
 * array of JACPCG_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits; the tables reach it as kernel parameters.
 * Runs on the current device.  The first call on a device looks up the
 * array's device address (make that first call before any stream capture);
 * the lookup is repeated if the device's context is replaced
 * (cudaDeviceReset).  All calls share the array: calls whose GPU work
 * overlaps race, so serialise them (one stream, one thread).  Returns ENOMEM, and enqueues nothing,
 * when the batch needs more scratch than the array holds (about 120
 * instances of M = 1024, K = 64, or 7 of K = 256); EINVAL for invalid
 * arguments as jacpcg_precode (K <= 256, no max_M limit; B, X0 and sinr
 * must be NULL, complex64 H only). */
#define JACPCG_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
jacpcg_status jacpcg_precode_noalloc(const jacpcg_instance *inst, int n_inst, int variant,
                                     int32_t *status_dev, int32_t *iters_dev, float *resid_dev,
                                     float *beta_dev, void *stream);

/* Per-subarray (block) RZF, Eq. 7 and the block structure of Eq. 6: the
 * array's antennas are split into row ranges, each serving its own set of
 * users, and each block G_i = beta_i H_i (H_i^H H_i + xi I)^{-1} is an
 * independent RZF precoder with its own power factor (beta_i over the
 * block's own F_i).  A block is a row range [row0, row0 + rows) of antennas
 * and a column range [col0, col0 + cols) of users of the full channel. */
typedef struct {
    int row0, rows;          /* antennas of the block */
    int col0, cols;          /* users of the block */
} jacpcg_block;

/* Host-only helper: describe the n_blocks blocks of `full` as independent
 * instances (out[i], host array of n_blocks), to be precoded together by
 * jacpcg_precode (a ragged batch) or any entry point that takes instances.
 * out[i] copies full's scalars (xi, power, max_iter, tol, h_dtype, omega) and
 * points H_i and W_i into full->H and full->W: W_i is the (row0, col0)
 * block of W, so one call fills the blocks of the block precoder G and
 * leaves the rest of W untouched (the caller zeroes it once).  X, A,
 * resid_hist, B and X0 of the blocks are NULL.  Errors, checked before
 * anything is written: EINVAL for a block outside full's M x K, an empty
 * block, more users than antennas in a block when xi = 0, or a block whose
 * H or W would not start on a 16-byte boundary (row0 must be even for
 * complex64 H, a multiple of 4 for bfloat16 H; W is complex64). */
jacpcg_status jacpcg_blocks(const jacpcg_instance *full, const jacpcg_block *blocks, int n_blocks,
                            jacpcg_instance *out);

/* Measurement aid (no counterpart in the paper): enqueue on `stream` one
 * launch of `blocks` CTAs of 256 threads, each thread running 8 independent
 * FP32 FMA chains of 16 * iters steps, so that the caller can time the FP32
 * FMA roof of the device with CUDA events (the roof the SIMT kernels are
 * reported against).  *flops (may be NULL) receives the flops of the launch,
 * blocks * 256 * iters * 16 * 8 * 2.  scratch_dev: device array of `blocks`
 * floats (never written in practice).  Errors: EINVAL, ECUDA. */
jacpcg_status jacpcg_probe_fp32_fma(int blocks, int iters, float *scratch_dev, void *stream,
                                    double *flops);

/* Destroy a context (and any plans still alive).  Waits for the device. */
jacpcg_status jacpcg_destroy(jacpcg_ctx *ctx);

/* Static string for a status code. */
const char *jacpcg_strerror(jacpcg_status s);

/* Library version, "MAJOR.MINOR.PATCH". */
const char *jacpcg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JACPCG_H */
