/*
 * ntf.h -- C ABI of libntf: GB300 (sm_103a) kernels for the unfolding-free
 * beta-divergence majorization-minimization updates of nonnegative CP and Tucker
 * decompositions (Leplat, arXiv 2602.14683).
 *
 * Conventions shared by every call
 *   - Pointers are DEVICE pointers unless the name ends in _host or the comment says
 *     "host".  Arrays of pointers (factors, COO coordinates) are host arrays whose
 *     elements are device pointers.
 *   - Tensors are row-major (C order, last mode fastest).  A factor A^(n) is I_n x R
 *     (CP) or I_n x J_n (Tucker), row-major FP32.  The Tucker core is J_1 x ... x J_N
 *     row-major FP32.
 *   - The caller owns X, the factors, the core and every output buffer.  The context
 *     owns all workspaces (padded factor copies, partial sums, Tucker partial tensors,
 *     COO permutations); it grows them on demand with cudaMalloc, so the first call at
 *     a new size allocates.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  Factors are updated in place when the call's work on
 *     the stream completes.  Objective outputs are FP64 device scalars written on the
 *     same stream.
 *   - Once a call's workspaces exist (after one call of the same kind, shapes and
 *     options on the context, and before any larger one), a repeated call makes no
 *     allocation, no host synchronisation and no host-to-device copy: it may be captured
 *     on a capturing `stream` into a CUDA graph and replayed, and the replays give
 *     bit-identical results to eager calls (the first sparse call per tensor, which builds
 *     the mode orders, must be made outside capture).
 *   - Return value: NTF_OK (0) or a negative ntf_status.  On error nothing has been
 *     launched that modifies caller buffers, except NTF_ERR_CUDA (a launch failed; the
 *     caller's buffers are in an unspecified state).  ntf_last_error(ctx) returns a
 *     message for the last error on that context; it stays valid until the next call.
 *   - beta must lie in [0, 2) (the range of Remark "Exponent gamma(beta)"), else
 *     NTF_ERR_BETA.  Ranks and core dimensions must lie in 1..64, else
 *     NTF_ERR_UNSUPPORTED.  Dense kernels accept orders 3 <= N <= 8 (the extrapolated entries
 *     and the server order 3 only; other orders return NTF_ERR_UNSUPPORTED); COO accepts
 *     2 <= N <= 8.  Order N >= 4 runs on the 3-way passes with the modes cut into three runs
 *     of consecutive modes (ntf_opts.merge), the same memory read as a 3-way tensor.
 *   - Data must be nonnegative and finite; factors and core must be >= eps on entry
 *     (Assumption "Positivity safeguard").  These are preconditions, not checked on the
 *     device.  At beta = 0 the data are floored at eps_x (Remark "The case beta = 0").
 *   - A context is used by one host thread at a time.
 */
#ifndef NTF_H
#define NTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ntf_ctx ntf_ctx;

typedef enum {
    NTF_OK = 0,
    NTF_ERR_ARG = -1,         /* null pointer, bad enum, inconsistent sizes */
    NTF_ERR_BETA = -2,        /* beta outside [0, 2) or not finite */
    NTF_ERR_SHAPE = -3,       /* dims <= 0, nnz out of range, core dims > tensor dims */
    NTF_ERR_OOM = -4,         /* workspace allocation failed */
    NTF_ERR_NONFINITE = -5,   /* reserved for host-side input checks */
    NTF_ERR_TIMEOUT = -6,     /* a bounded device-side wait ran out (serving loop) */
    NTF_ERR_CUDA = -7,        /* a CUDA runtime call or launch failed */
    NTF_ERR_UNSUPPORTED = -8  /* valid request outside what the kernels implement */
} ntf_status;

enum { NTF_DENSE = 0, NTF_COO = 1 };
enum { NTF_CP = 0, NTF_TUCKER = 1 };
/* Arithmetic of the contraction tiles.  FP32: CUDA-core FP32 FMA.  TF32: tcgen05 tensor
 * cores (dense CP, rank padded to 32): the reconstruction Xhat on TF32 operands rounded to
 * nearest (one MMA pass), the Num / Den contractions on BF16 operands, FP32 accumulation.
 * 3XTF32: the same, with the reconstruction split into high and low TF32 parts (three MMA
 * passes, about FP32 accuracy for Xhat and the objective).  Dense Tucker on the tensor cores
 * (third core dimension <= 32): the passes over X as for CP, and the small contractions of
 * Appendix C (the partial tensor B^(3), the core and factor products) as tcgen05 GEMMs on TF32
 * operands (split high / low with 3XTF32), FP32 accumulation.  The beta-powers are always
 * FP32 and the objective is accumulated in FP64. */
enum { NTF_PREC_FP32 = 0, NTF_PREC_TF32 = 1, NTF_PREC_3XTF32 = 2 };

typedef struct {
    int order;                 /* N */
    const int64_t *dims;       /* host array [N], each >= 1 */
    int kind;                  /* NTF_DENSE or NTF_COO */
    const float *values;       /* dense: prod(dims) values; COO: nnz values */
    const int32_t *const *idx; /* COO only: host array of N device arrays of nnz coords */
    int64_t nnz;               /* COO only: number of stored entries (unique coords) */
} ntf_tensor;

typedef struct {
    double eps;    /* floor on every parameter and on Xhat inside the powers (1e-12) */
    double eps_x;  /* data floor used only at beta = 0 (1e-12) */
    int inner_L;   /* J-CoMM inner sweeps per outer iteration, >= 1 (1) */
    int precision; /* NTF_PREC_FP32 (default), NTF_PREC_TF32 or NTF_PREC_3XTF32 */
    int autotune;  /* 1 = pick launch plans by timing (0).  Dense CP: the pass's slab split; on the
                      first call for a given shape, rank padding, precision, beta class and pass
                      variant in this process, the call times the pass it is about to run under a
                      few grid plans (about one to four waves of CTAs, plus the cost model's choice).
                      Tucker on the tensor cores: every contraction's tile width and reduction split
                      (each width with its rule's split, and the rule's width with half and twice
                      its split), on the first call for that product's shape and strides.  The
                      timing runs on the call's own stream, synchronizing it, and the fastest plan
                      goes to a process-wide table that every later call and context reuses.  A plan
                      sets the order of partial sums, so results may differ from a run with another
                      table in the last bits.  Ignored (rule's plan, nothing cached) while the
                      stream is being captured. */
    int merge;     /* dense CP and Tucker of order N >= 4, which run on the 3-way passes with the
                      modes cut into three runs of consecutive modes [0, a), [a, b), [b, N) (a run
                      of several modes is one 3-way mode whose factor is the Khatri-Rao product
                      (CP) or Kronecker product (Tucker) of the run's blocks): 0 = the library
                      picks the cut (0); else 16 * a + b, 1 <= a < b <= N - 1 (NTF_ERR_ARG
                      otherwise; Tucker: NTF_ERR_UNSUPPORTED when the last run's core extent
                      exceeds 64).  Ignored at N = 3.  Results depend on the cut only through
                      the order of floating-point sums. */
    int cache;     /* J-CoMM at beta != 1, dense 3-way CP on the tensor-core passes: whether the
                      reference-powered tensors P~ = X (.) X~^(beta-2), Q~ = X~^(beta-1) of an outer
                      iteration (Section 5.3; Algorithm 2) are kept.  NTF_CACHE_AUTO (0): kept
                      (with autotune = 1: the choice is timed once per shape and beta class);
                      NTF_CACHE_NONE: every inner block pass recomputes X~ from the reference;
                      NTF_CACHE_BF16: the first pass writes the BF16 P~ / Q~ tiles its
                      contractions consume (2 + 2 bytes per entry of context workspace) and every
                      later pass of the outer iteration contracts them without reading X.  The
                      two modes give the same results bit for bit.  Ignored elsewhere. */
} ntf_opts;

#define NTF_CACHE_AUTO 0
#define NTF_CACHE_NONE 1
#define NTF_CACHE_BF16 2

/* Fills *o with the defaults shown above. */
void ntf_opts_default(ntf_opts *o);

/* Creates a context bound to CUDA device `device`.  Returns NTF_ERR_CUDA if the device
 * cannot be used. */
int ntf_ctx_create(ntf_ctx **ctx, int device);
/* Frees the context's workspaces.  Waits for its in-flight work (device sync). */
void ntf_ctx_destroy(ntf_ctx *ctx);
/* Last error message of this context (static storage inside ctx, never NULL). */
const char *ntf_last_error(const ntf_ctx *ctx);
/* Number of kernels this context has launched since creation (for accounting). */
int64_t ntf_launch_count(const ntf_ctx *ctx);
/* Profiling of the fused passes (the kernels that read X).  While enabled, every such
 * launch is bracketed by a pair of CUDA events recorded on the launch's own stream.
 * ntf_pass_timing waits for the recorded events, returns their summed elapsed time in
 * milliseconds and the number of bracketed launches, and clears the record.  Not for use
 * during stream capture. */
int ntf_set_pass_timing(ntf_ctx *ctx, int enable);
int ntf_pass_timing(ntf_ctx *ctx, double *total_ms, int64_t *launches);
/* Device-side status of the context's kernels.  Kernels whose waits are bounded (the
 * tensor-core passes wait on TMA and MMA completion barriers) set a status word in device
 * memory instead of hanging when a wait runs out.  This call synchronizes `stream`, reads
 * and clears that word, and returns NTF_OK or NTF_ERR_TIMEOUT (the results of the calls
 * since the last check are then invalid). */
int ntf_device_status(ntf_ctx *ctx, void *stream);
/* Testing aid for the bounded waits above (the paper has no counterpart).  polls > 0 sets
 * the number of polls after which a wait of the context's tensor-core passes gives up
 * (polls <= 0 restores the built-in limit, seconds at worst); with probe != 0, each such
 * pass first waits on a barrier that nothing arrives on, so that this wait runs out before
 * the pass has issued any copy or MMA, and the pass then aborts as a real timeout would
 * (status word set, TMEM freed, no further work issued).  Results of passes run with the
 * probe on are invalid; ntf_device_status reports NTF_ERR_TIMEOUT for them.
 * NTF_ERR_ARG for a NULL context. */
int ntf_debug_wait_limit(ntf_ctx *ctx, int polls, int probe);

/* One B-CoMM sweep for CP (Algorithm 1; Theorem "CP block multiplicative update";
 * CPContr of Section 6.1): for n = 1..N in order, rebuild Xhat from the current
 * factors, P = X*Xhat^(beta-2), Q = Xhat^(beta-1), Num^(n) = CPContr^(n)(P; A),
 * Den^(n) = CPContr^(n)(Q; A) (at beta = 1 the closed form prod_{m!=n} colsum A^(m),
 * Section 6.3), A^(n) <- max(A^(n) * (Num/Den)^gamma(beta), eps).
 *   factors:       host array of N device pointers, A^(n) is I_n x rank, updated in place
 *   objective_dev: device double or NULL; receives D_beta(X, Xhat) of the INCOMING
 *                  iterate (before this sweep).
 * Dense (N = 3..8) and COO tensors.  COO (Section 6.3): Num^(n) runs over the stored entries
 * (P vanishes where X does); at beta = 1 Den^(n) is the closed form, at other beta it contracts
 * Xhat^(beta-1) over the whole index space in a pass that reads no X (FP32, N >= 3; the modes cut
 * into three runs as for dense tensors).  COO at beta = 0 (d_0 needs X > 0 everywhere) and COO of
 * order 2 at beta != 1 return NTF_ERR_UNSUPPORTED. */
int ntf_cp_mu_sweep(ntf_ctx *ctx, const ntf_tensor *X, float beta, int rank,
                    float *const *factors, const ntf_opts *opts, double *objective_dev,
                    void *stream);

/* One extrapolated B-CoMM sweep for dense 3-way CP (Section "Going beyond: Majorization-
 * Minimization with Extrapolation", item (i)).  For n = 1..3: with D = [A^(n) - Aprev^(n)]_+
 * (componentwise positive part) and alpha_n = min(alpha, cap / (||D||_F + delta)), the block
 * is first moved to Ahat = max(A^(n) + alpha_n D, eps); Xhat is rebuilt from Ahat and the
 * current other blocks, P and Q formed as in ntf_cp_mu_sweep, and
 * A^(n) <- max(Ahat * (Num / Den)^gamma(beta), eps) with Num / Den the contractions against the
 * current other blocks.
 *   factors:       host array of 3 device pointers, A^(n) is I_n x rank: the current iterate
 *                  A^t on entry, A^(t+1) on exit
 *   factors_prev:  host array of 3 device pointers, same shapes: the previous iterate A^(t-1) on
 *                  entry, overwritten with the incoming A^t (ready for the next call); pass a copy
 *                  of factors on the first call (no displacement: a plain B-CoMM sweep)
 *   alpha:         extrapolation weight of this outer iteration (>= 0; e.g. a Nesterov-type
 *                  sequence chosen by the caller), the same for every block
 *   cap, delta:    displacement cap (>= 0; INFINITY disables it) and its regulariser (> 0)
 *   objective_dev: device double or NULL; receives D_beta of the incoming iterate A^t (one more
 *                  pass over X when requested).
 * Dense order-3 tensors only, else NTF_ERR_UNSUPPORTED; other arguments and errors as
 * ntf_cp_mu_sweep. */
int ntf_cp_mu_sweep_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, int rank, float *const *factors,
                           float *const *factors_prev, float alpha, float cap, float delta,
                           const ntf_opts *opts, double *objective_dev, void *stream);

/* One J-CoMM outer iteration for dense 3-way CP from an extrapolated outer reference
 * (Section "Going beyond: Majorization-Minimization with Extrapolation", item (iii)): every
 * block is first moved to max(A^(n) + alpha_n [A^(n) - Aprev^(n)]_+, eps) with alpha_n as in
 * ntf_cp_mu_sweep_extrap, and the outer iteration of ntf_jcomm_outer (Algorithm 2, opts->inner_L
 * inner sweeps) runs with that point as its reference and as the inner iterations' start.
 * The paper gives this variant as a heuristic without a convergence result.
 *   factors / factors_prev / alpha / cap / delta: as ntf_cp_mu_sweep_extrap
 *   objective_dev: device double or NULL; receives D_beta of the incoming iterate A^t (one more
 *                  pass over X when requested).
 * Dense order-3 tensors only, else NTF_ERR_UNSUPPORTED. */
int ntf_cp_jcomm_outer_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, int rank, float *const *factors,
                              float *const *factors_prev, float alpha, float cap, float delta,
                              const ntf_opts *opts, double *objective_dev, void *stream);

/* One block-MM sweep for Tucker (Theorem "Tucker block multiplicative updates";
 * Appendix C.2, eqs. (block_core_num_den), (block_Bn), (block_factor_num/den)): the
 * core first, then factors 1..N, each block rebuilt from the current blocks, followed
 * by the eps clip.
 *   core_dims: host array [N] of J_n; core: device J_1 x ... x J_N, updated in place
 *   factors:   host array of N device pointers, A^(n) is I_n x J_n, updated in place
 *   objective_dev: device double or NULL; D_beta of the incoming iterate.
 * Dense N = 3..8 (N >= 4: the last run of the cut needs a core extent <= 64), and COO of order 3
 * at beta != 0 (Section 6.3: numerators over the stored entries; denominators in closed form at
 * beta = 1, else from X-free passes over the whole index space; FP32 passes whatever the
 * precision); other COO Tucker requests return NTF_ERR_UNSUPPORTED. */
int ntf_tucker_mu_sweep(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims,
                        float *core, float *const *factors, const ntf_opts *opts,
                        double *objective_dev, void *stream);

/* One extrapolated block-MM sweep for dense 3-way Tucker (Section "Going beyond:
 * Majorization-Minimization with Extrapolation", item (ii)): the core, then factors 1..3;
 * before its update each block Z is moved to max(Z + alpha_Z [Z - Zprev]_+, eps) with
 * alpha_Z = min(alpha, cap / (||[Z - Zprev]_+||_F + delta)), the reconstruction uses that
 * block and the current others, and it is the multiplicative pre-factor (Theorem "Tucker block
 * multiplicative updates").
 *   core / factors: the current iterate in, the new iterate out (as ntf_tucker_mu_sweep)
 *   core_prev / factors_prev: the previous iterate in (same shapes), overwritten with the
 *                  incoming iterate; pass copies of core / factors on the first call
 *   alpha / cap / delta: as ntf_cp_mu_sweep_extrap
 *   objective_dev: device double or NULL; receives D_beta of the incoming iterate (one more
 *                  pass over X when requested).
 * Dense N = 3 only. */
int ntf_tucker_mu_sweep_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
                               float *const *factors, float *core_prev, float *const *factors_prev, float alpha,
                               float cap, float delta, const ntf_opts *opts, double *objective_dev, void *stream);

/* One J-CoMM outer iteration (Algorithm 2; Section 5.3; Appendix C.3): the reference is
 * the incoming iterate, Ptilde = X*Xtilde^(beta-2) and Qtilde = Xtilde^(beta-1) are
 * fixed for opts->inner_L inner sweeps; every inner block update uses chi1 of the
 * other current blocks for the numerator and chi2 for the denominator, the reference
 * block as pre-factor, then the eps clip.  Reference tensors are recomputed from the
 * reference factors inside each pass (never stored).
 *   model: NTF_CP (rank_or_0 = R, core arguments NULL) or NTF_TUCKER (rank_or_0 = 0)
 *   objective_ref_dev: device double or NULL; receives D_beta at the reference.
 * CP dense N = 3..8 (any beta), CP COO (as ntf_cp_mu_sweep), Tucker dense N = 3..8 (any beta),
 * Tucker COO (order 3, beta != 0). */
int ntf_jcomm_outer(ntf_ctx *ctx, int model, const ntf_tensor *X, float beta, int rank_or_0,
                    const int64_t *core_dims_or_null, float *core_or_null, float *const *factors,
                    const ntf_opts *opts, double *objective_ref_dev, void *stream);

/* One Tucker J-CoMM outer iteration (dense 3-way) from an extrapolated outer reference
 * (Section "Going beyond: Majorization-Minimization with Extrapolation", item (iii)): the core
 * and every factor are first moved to max(Z + alpha_Z [Z - Zprev]_+, eps) (alpha_Z as in
 * ntf_tucker_mu_sweep_extrap), and the outer iteration of ntf_jcomm_outer (NTF_TUCKER) runs with
 * that point as its reference.  A heuristic without a convergence result in the paper.
 *   core / factors / core_prev / factors_prev / alpha / cap / delta: as ntf_tucker_mu_sweep_extrap
 *   objective_dev: device double or NULL; receives D_beta of the incoming iterate. */
int ntf_tucker_jcomm_outer_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims,
                                  float *core, float *const *factors, float *core_prev, float *const *factors_prev,
                                  float alpha, float cap, float delta, const ntf_opts *opts, double *objective_dev,
                                  void *stream);

/* D_beta(X, Xhat) = sum_i d_beta(X_i | max(Xhat_i, eps)) (Section 3.2, Definition
 * "beta-divergence") in FP64, written to *out_dev.  Per-entry terms use stable forms
 * in FP32 (log1p/expm1) and are summed in FP64.  For COO the unstored entries (x = 0) add
 * d_beta(0 | Xhat) = Xhat^beta / beta: at beta = 1 the closed form sum of Xhat (CP:
 * sum_r prod_n colsum(A^(n))_r; Tucker, order 3: the same from B^(3) and A^(3)), at other beta
 * a pass over the whole index space that reads no X; COO requests as ntf_cp_mu_sweep /
 * ntf_tucker_mu_sweep. */
int ntf_beta_div(ntf_ctx *ctx, int model, const ntf_tensor *X, float beta, int rank_or_0,
                 const int64_t *core_dims_or_null, const float *core_or_null,
                 const float *const *factors, const ntf_opts *opts, double *out_dev,
                 void *stream);

/* The cut of a dense order-N (4 <= N <= 8) CP or Tucker problem into the three runs of consecutive
 * modes [0, a), [a, b), [b, N) that ntf_cp_mu_sweep / ntf_tucker_mu_sweep / ntf_jcomm_outer /
 * ntf_beta_div use for it (Section 6.1: the contractions over a merged index), as chosen from the
 * shapes and opts (opts->merge when nonzero, else the library's choice) for a 16-byte-aligned X.
 * Host-only planning: no context and no device work.
 *   model: NTF_CP (rank_or_0 = R, core_dims_or_null = NULL) or NTF_TUCKER (rank_or_0 = 0,
 *          core_dims_or_null = host array [N] of J_n)
 *   dims:  host array [N]; beta: the divergence (Tucker tensor-core passes depend on it)
 *   a_out, b_out: the run boundaries.
 * The cut depends on opts->precision.  ntf_beta_div evaluates the objective on the FP32 passes
 * whatever opts->precision says, so the cut it uses is the one returned for
 * opts->precision = NTF_PREC_FP32 (for example CP 80 x 70 x 60 x 50 at R = 10: (1, 2) at
 * NTF_PREC_TF32 for the sweeps, (1, 3) for ntf_beta_div).
 * NTF_ERR_ARG (NULL pointers, bad model or merge, eps or eps_x <= 0, inner_L < 1, unknown
 * precision), NTF_ERR_BETA (beta outside [0, 2)), NTF_ERR_UNSUPPORTED (order outside 4..8, rank
 * or core extents outside 1..64, no cut with a last-run core extent <= 64), NTF_ERR_SHAPE
 * (dims outside 1..2^31 - 1, or a run's extent beyond 32 bits). */
int ntf_plan_cut(int model, int order, const int64_t *dims, int rank_or_0, const int64_t *core_dims_or_null,
                 const ntf_opts *opts, float beta, int *a_out, int *b_out);

/* Stable permutation of 0..nnz-1 by key (a COO coordinate array), bit-identical to a
 * stable sort: equal keys keep their input order.  keys: device int32 [nnz] with values
 * in [0, key_range); perm_out: device int32 [nnz].  Used internally to order COO
 * entries per mode; exposed for testing. */
int ntf_coo_stable_perm(ntf_ctx *ctx, const int32_t *keys, int64_t nnz, int64_t key_range,
                        int32_t *perm_out, void *stream);

/* ---------------------------------------------------------------------------------
 * Continuous-batching server for many small dense 3-way jobs (CP or Tucker).
 * A scheduler thread admits submitted jobs into two lanes, each in FIFO order.  Dense CP
 * jobs with precision NTF_PREC_FP32 join a batch (ntf_batch_* below) whose arena is half of
 * the memory budget: they are admitted when their workspace fits the arena and share every
 * launch of an iteration with the other resident jobs of their class, a few iterations per
 * graph launch.  All other jobs (and a CP job larger than the whole arena) use the slot lane:
 * the server owns `slots` execution slots (a context and a stream each); the lane's head is
 * admitted into a free slot when its estimated workspace fits the other half of the budget
 * (a job larger than the budget runs alone).  An admitted job runs one iteration eagerly (sizing its slot's workspaces), then
 * the rest of the job as one CUDA graph launch: a conditional WHILE node over one captured
 * iteration of its method followed by a one-thread kernel that applies the stopping test on
 * the device to the FP64 objective of the iteration's incoming iterate (Section 3.2): stop
 * when |F_{t-1} - F_t| / F_{t-1} <= rtol or after max_iters iterations.  No host round trip
 * happens between iterations.  Jobs in different slots run concurrently.  A job's result
 * does not depend on what else runs.
 * The caller owns X, factors and core (device memory) and must keep them alive and
 * untouched until the job's result has been polled; factors and core are updated in
 * place.  Server functions are thread-safe; each job uses the device of the server.
 * While jobs run, a slot stream may be capturing its job's graph: other threads of the process
 * must not call cudaDeviceSynchronize (or anything else that synchronizes the whole device)
 * until ntf_server_poll(..., wait_all = 1) has returned; synchronizing their own streams or
 * events is fine (the slot streams are non-blocking).
 * --------------------------------------------------------------------------------- */
typedef struct ntf_server ntf_server;

typedef struct {
    int model;             /* NTF_CP or NTF_TUCKER */
    int method;            /* 0: J-CoMM (Algorithm 2) with inner_L = 1; 1: block MM */
    int precision;         /* NTF_PREC_FP32, NTF_PREC_TF32 or NTF_PREC_3XTF32 (CP only) */
    int64_t dims[3];       /* I_1, I_2, I_3 */
    int rank;              /* CP rank (1..64) */
    int64_t core_dims[3];  /* Tucker core dimensions (1..64 each) */
    float beta;            /* in [0, 2) */
    double eps;            /* parameter floor; <= 0 selects 1e-12 */
    double rtol;           /* relative objective change that stops the job */
    int max_iters;         /* iteration cap, >= 1 */
    const float *X;        /* device, dense row-major */
    float *factors[3];     /* device, I_n x rank (CP) or I_n x J_n (Tucker), in place */
    float *core;           /* device, Tucker core (NULL for CP), in place */
} ntf_job;

typedef struct {
    int64_t id;            /* id returned by ntf_server_submit */
    int status;            /* NTF_OK or the failing call's status */
    int iterations;        /* iterations run */
    double objective;      /* D_beta of the incoming iterate of the last iteration */
    double t_submit, t_admit, t_done; /* host steady-clock seconds */
} ntf_result;

/* mem_budget_bytes = 0 selects half of the device memory free at creation. */
int ntf_server_create(ntf_server **server, int device, int slots, size_t mem_budget_bytes);
/* Queues a copy of *job; returns at once.  id_out (may be NULL) receives the job id. */
int ntf_server_submit(ntf_server *server, const ntf_job *job, int64_t *id_out);
/* Moves up to max_results completed results into out and returns how many; with
 * wait_all != 0 it first waits until every submitted job has completed. */
int ntf_server_poll(ntf_server *server, ntf_result *out, int max_results, int wait_all);
/* Stops the scheduler (queued jobs are dropped), waits for running work, frees slots. */
void ntf_server_destroy(ntf_server *server);

/* ---------------------------------------------------------------------------------
 * Launches shared by many small dense 3-way CP jobs (FP32 passes).
 * A batch keeps resident jobs -- the ntf_job requests above with model NTF_CP and precision
 * NTF_PREC_FP32, J-CoMM (Algorithm 2, inner_L = 1) or block MM (Algorithm 1) -- in classes
 * by rank padding (8, 16, 32, 64) and iteration shape (J-CoMM at beta = 1: one pass with
 * all numerators; beta = 1 block MM: three passes with closed-form denominators; beta != 1:
 * three passes with numerators and denominators).  One iteration of a class is one launch
 * per step for ALL its jobs: a persistent grid walks a device-resident work table in which
 * each job owns the work items of its own single-job launch, so every job computes exactly
 * what ntf_jcomm_outer / ntf_cp_mu_sweep compute for it on the FP32 path (the same bits),
 * whatever else is resident.  ntf_batch_tick runs up to `iters` iterations of every class as
 * one graph launch per class (a conditional WHILE node over the captured iteration and a
 * device stopping test: |F_{t-1} - F_t| / F_{t-1} <= rtol on the FP64 objective of the
 * incoming iterate, or the iteration cap); classes run concurrently on their own streams.
 * Between launches the batch retires stopped jobs and admits new ones (continuous batching
 * at iteration granularity).  Workspaces come from one device arena of mem_budget_bytes
 * allocated at creation (0: a quarter of the free device memory): ntf_batch_add returns
 * NTF_ERR_OOM when the job does not fit now (retry after a tick has retired jobs) or when
 * `capacity` jobs are resident; NTF_ERR_UNSUPPORTED for Tucker or tensor-core requests.
 * The caller owns X and the factors (device memory), keeps them alive and untouched until
 * the job's result has been returned, and finds the factors updated in place.  A batch is
 * driven by one host thread; its calls are not thread-safe.
 * --------------------------------------------------------------------------------- */
typedef struct ntf_batch ntf_batch;
int ntf_batch_create(ntf_batch **batch, int device, int capacity, size_t mem_budget_bytes);
/* Makes the job resident (it joins the next launch of its class); id_out (may be NULL)
 * receives its id.  job->X and job->factors must stay valid while it is resident. */
int ntf_batch_add(ntf_batch *batch, const ntf_job *job, int64_t *id_out);
/* For every class whose previous launch has finished (with wait != 0: after waiting for
 * it): moves the stopped jobs' results to the result list and frees their workspaces; then,
 * if the class still holds jobs, launches up to `iters` (>= 1) more iterations of all of
 * them.  Asynchronous apart from the wait.  Returns the number of resident jobs (>= 0; with
 * wait != 0, 0 means every job has finished) or a negative ntf_status.  A failed launch
 * ends all jobs of its class with NTF_ERR_CUDA. */
int ntf_batch_tick(ntf_batch *batch, int iters, int wait);
/* Moves up to max_results finished results (oldest first) into out; returns how many. */
int ntf_batch_results(ntf_batch *batch, ntf_result *out, int max_results);
int ntf_batch_resident(const ntf_batch *batch);
/* Waits for running launches, then frees the batch (resident jobs are dropped). */
void ntf_batch_destroy(ntf_batch *batch);

/* Allocation-free objective for dense CP tensors.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory when they call -- a process whose
 * device memory is reserved up front by another framework's allocator, or one held to a
 * fixed device-memory budget, where a cudaMalloc inside the library would fail or take
 * memory the caller has already given out.  The other entry points grow workspaces with
 * cudaMalloc; this one allocates nothing.  It computes the same value as
 * ntf_beta_div(ctx, NTF_CP, X, beta, rank, NULL, NULL, factors, opts, out_dev, stream)
 * with opts = {eps, eps_x}, on the current device, asynchronously on `stream`.
 *   - Scratch: a file-scope device array of NTF_NOALLOC_SCRATCH_BYTES that every GPU
 *     loading the library holds until the process exits.  It must fit the padded factor
 *     copies and one FP64 partial per CTA: about (I_1 + I_2 + I_3) * 32 * 4 bytes at
 *     rank <= 32; larger problems return NTF_ERR_UNSUPPORTED before any work is queued.
 *   - The first call on a device looks up the array's device address (one
 *     cudaGetSymbolAddress with that device current); make that first call before any
 *     stream capture.
 *   - Every call on a device shares the same array and each call overwrites what it uses.
 *     Calls whose GPU work overlaps (different streams, or concurrent host threads) race;
 *     order them on one stream or synchronize between them.
 *   - Dense order-3 tensors only; other arguments and errors as ntf_beta_div.  No
 *     context, so no message: the return code is the only error report. */
#define NTF_NOALLOC_SCRATCH_BYTES (4u << 20)
int ntf_cp_beta_div_noalloc(const ntf_tensor *X, float beta, int rank, const float *const *factors,
                            double eps, double eps_x, double *out_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NTF_H */
