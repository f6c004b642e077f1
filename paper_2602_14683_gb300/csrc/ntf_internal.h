// Internal declarations shared by the libntf translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ntf {

// ---------------------------------------------------------------------------------
// beta specialisations of the powers P = X*Y^(beta-2), Q = Y^(beta-1) (Section 4.1):
// the four values used by the workloads get a single-MUFU form, any other beta goes
// through powf.
// ---------------------------------------------------------------------------------
enum BetaKind : int { BK_IS = 0, BK_HALF = 1, BK_KL = 2, BK_THREEHALF = 3, BK_GEN = 4 };

inline int beta_kind(float b) {
    if (b == 0.0f) return BK_IS;
    if (b == 0.5f) return BK_HALF;
    if (b == 1.0f) return BK_KL;
    if (b == 1.5f) return BK_THREEHALF;
    return BK_GEN;
}

// gamma(beta) of Remark "Exponent gamma(beta)".
inline float mu_gamma(float b) { return b < 1.0f ? 1.0f / (2.0f - b) : 1.0f; }

#ifdef __CUDACC__
// y: clipped reconstruction max(Xhat, eps) > 0; x: data (already floored at beta = 0).
__device__ __forceinline__ void pq_powers(int bk, float beta, float x, float y, float &P, float &Q) {
    switch (bk) {
        case BK_IS: {
            float r = __frcp_rn(y);
            Q = r;
            P = x * r * r;
            break;
        }
        case BK_HALF: {
            float s = rsqrtf(y);
            Q = s;
            P = x * s * s * s;
            break;
        }
        case BK_KL: {
            P = __fdiv_rn(x, y);
            Q = 1.0f;
            break;
        }
        case BK_THREEHALF: {
            float s = rsqrtf(y);
            Q = y * s;
            P = x * s;
            break;
        }
        default: {
            Q = powf(y, beta - 1.0f);
            P = x * powf(y, beta - 2.0f);
            break;
        }
    }
}

// d_beta(x|y) (Section 3.2) in FP32.  Near x = y the terms of the definition cancel,
// so there the divergence is written through exact factorisations (beta = 1/2, 3/2, see
// below) or through log1p/expm1 of the ratio:
//   KL : x (t - log1p t),  t = y/x - 1
//   IS : s - log1p s,      s = x/y - 1
//   else: x^b ((b-1) expm1(b L) - b expm1((b-1) L)) / (b (b-1)),  L = log1p(y/x - 1)
// Far from x = y (ratio outside [1e-4, 1e4]) the ratio minus one loses the small
// operand to rounding, and the definition itself has no cancellation; it is used there.
__device__ __forceinline__ float dbeta_stable(int bk, float beta, float x, float y) {
    if (bk == BK_IS) {
        const float u = __fdiv_rn(x, y);
        if (u > 1e-4f && u < 1e4f) {
            const float s = u - 1.0f;
            return s - log1pf(s);
        }
        return u - (logf(x) - logf(y)) - 1.0f;
    }
    if (!(x > 0.0f)) return bk == BK_KL ? y : powf(y, beta) / beta;
    if (bk == BK_THREEHALF || bk == BK_HALF) {
        // exact factorisations in t = sqrt(y / x), free of cancellation:
        //   beta = 3/2: d = (2/3) x^(3/2) (t - 1)^2 (t + 2);   beta = 1/2: d = 2 x^(1/2) (t - 1)^2 / t
        const float t = sqrtf(__fdiv_rn(y, x)), sx = sqrtf(x), e = t - 1.0f;
        if (bk == BK_THREEHALF) return (2.0f / 3.0f) * x * sx * e * e * (t + 2.0f);
        return 2.0f * sx * e * __fdiv_rn(e, t);
    }
    const float r = __fdiv_rn(y, x);
    const bool near = r > 1e-4f && r < 1e4f;
    if (bk == BK_KL) {
        if (near) {
            const float t = r - 1.0f;
            return x * (t - log1pf(t));
        }
        return x * (logf(x) - logf(y)) - x + y;
    }
    if (near) {
        const float L = log1pf(r - 1.0f);
        const float e1 = expm1f(beta * L), e2 = expm1f((beta - 1.0f) * L);
        return powf(x, beta) * ((beta - 1.0f) * e1 - beta * e2) / (beta * (beta - 1.0f));
    }
    return (powf(x, beta) + (beta - 1.0f) * powf(y, beta) - beta * x * powf(y, beta - 1.0f)) /
           (beta * (beta - 1.0f));
}

// Transforms chi1, chi2 of Section 5.3 on one entry (z: current, zt: reference).
__device__ __forceinline__ float chi1_f(float beta, float z, float zt) {
    if (beta == 1.0f) return zt;
    return powf(zt, 2.0f - beta) * powf(z, beta - 1.0f);
}
__device__ __forceinline__ float chi2_f(float beta, float z, float zt) {
    if (beta < 1.0f) return z;
    if (beta == 1.0f) return z;
    return powf(z, beta) * powf(zt, 1.0f - beta);
}
#endif

// ---------------------------------------------------------------------------------
// Dense 3-way CP pass (the fused reconstruct -> powers -> contract kernel)
// ---------------------------------------------------------------------------------
// PM_NOX (FP32 pass; tensor-core pass at beta != 1): the entries of X are taken as 0 and X is not read -- the dense part
// of a sparse tensor's update (Section 6.3): only the denominator side (Q = Xhat^(beta-1)
// against the den factors) is contracted, and the objective term is d_beta(0 | Xhat).
enum PassMode : int { PM_M1 = 1, PM_M2 = 2, PM_M3 = 4, PM_OBJ = 8, PM_NOX = 16 };

struct Cp3Args {
    const float *X;
    int I, J, K;
    const float *rec[3];  // factors that rebuild Xhat, padded [I_n][RP]
    const float *num[3];  // factors of the numerator contraction
    const float *den[3];  // factors of the denominator contraction
    // Optional explicit row factors [I*J][RP] (Tucker partial tensors): when rrow is set,
    // GEMM1 uses rrow[i*J + j] instead of rec[0][i] * rec[1][j]; nrow / drow replace
    // num[0][i] * num[1][j] and den[0][i] * den[1][j] in the mode-3 contraction.
    const float *rrow, *nrow, *drow;
    int bkind;
    float beta, eps, eps_x;
    int n_jt, n_kb, n_is;  // grid decomposition: row tiles x column blocks x slab splits
    int vec16;             // 1: K % 4 == 0 and X 16-byte aligned (16-byte async copies)
    float *p1n, *p1d;      // mode-1 partials [parts1][I][RP] (parts1 = n_jt*n_kb, x4 on tensor cores)
    float *p2n, *p2d;      // mode-2 partials [n_kb*n_is][J][RP]
    float *p3n, *p3d;      // mode-3 partials [n_jt*n_is][K][RP]
    double *obj;           // per-CTA objective partials [grid]
    int *err;              // device status word: set non-zero when a bounded wait gives up
    int wait_limit;        // polls before a bounded wait gives up (<= 0: the built-in limit)
    int timeout_probe;     // 1: one wait on a barrier nothing arrives on, before any copy or MMA
    // J-CoMM reference-powered tensors P~, Q~ as BF16 [I*J][kp] (kp = K rounded up to 8): the
    // tensor-core pass writes them when pc is set; the contraction-only pass reads them
    void *pc, *qc;
    int kp;
};

// ---------------------------------------------------------------------------------
// Jobs that run many iterations on the device (serving slots and batched launches)
// ---------------------------------------------------------------------------------
// Stopping state of one job, updated on the device after every iteration.
struct JobState {
    double F_prev, F_last;  // objectives of the last two iterations' incoming iterates
    double rtol;
    int iters, max_iters, done, pad;
};

#ifdef __CUDACC__
// One more iteration done: its incoming iterate's objective is *F.  Stop when t > 1 and
// |F_{t-1} - F_t| / F_{t-1} <= rtol (Section 3.2's objective, relative change), or at
// t = max_iters.
__device__ __forceinline__ void job_step(JobState *s, const double *F) {
    s->iters += 1;
    s->F_prev = s->F_last;
    s->F_last = *F;
    const double a = s->F_prev, b = s->F_last;
    const bool conv = s->iters > 1 && a > 0.0 && (a - b) / a <= s->rtol && (b - a) / a <= s->rtol;
    s->done = (conv || s->iters >= s->max_iters) ? 1 : 0;
}
#endif

// Work table of one step of a batched iteration: resident job j owns the step's work items
// [pfx[j], pfx[j+1]) (its own launch grid for that step) and the arguments args[j]; a
// persistent grid walks all items in one launch and skips the jobs whose state says done.
// Every pointer is device memory; n and the tables change between launches, never during one.
template <class A>
struct BatchTable {
    const int *n;           // number of resident jobs
    const int *pfx;         // [n + 1] item prefix (pfx[0] = 0)
    const A *args;          // [n]
    const JobState *state;  // [n]
};

#ifdef __CUDACC__
// The job that owns work item `item` (pfx non-decreasing, pfx[0] = 0 <= item < pfx[n]).
__device__ __forceinline__ int batch_job_of(const int *pfx, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pfx[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
#endif

struct Cp3Plan {
    int tc;  // 1: tensor-core (tcgen05) pass, else FP32 CUDA-core pass
    int s3;  // tensor-core pass: reconstruction on split (hi / lo) TF32 operands
    int RP, TJ, KB;
    int n_jt, n_kb, n_is;
    int grid;
    int parts1, parts2, parts3;
};

// kb: columns per CTA block (64 for the FP32 pass; 128 for the tensor-core pass, 256 for its
// KL single-TF32 variants); n_is > 0 forces the slab split instead of the cost model's choice
Cp3Plan cp3_plan(int I, int J, int K, int RP, int num_sms, int kb = 64, int n_is = 0);
// Launches one pass.  mode_set: OR of PassMode; den: 1 when the denominator partials are
// needed (beta != 1).  Returns a cudaError_t.
cudaError_t cp3_launch(const Cp3Plan &plan, const Cp3Args &a, int mode_set, int den,
                       cudaStream_t s);

// Tensor-core (tcgen05) variant of the same pass (plan with kb = 128): TF32 reconstruction
// GEMM, BF16 contraction GEMMs, FP32 accumulation; same partial-sum layouts.
// Eligible when RP == 32, K % 4 == 0 and X is 16-byte aligned.
bool cp3_tc_eligible(int RP, int K, const float *X);
// rx: explicit rows (Tucker): modes M1 | M2 (W rows out, optionally with the objective) or
// M3, and only with the denominator side (beta != 1).
bool cp3_tc_supported(int mode_set, int den, bool rx = false);
cudaError_t cp3_tc_launch(const Cp3Plan &plan, const Cp3Args &a, int mode_set, int den,
                          cudaStream_t s);
// Contraction-only pass over the cached BF16 P~ / Q~ (a.pc, a.qc, row stride a.kp) of a J-CoMM
// outer iteration at beta != 1: mode_set one of PM_M1, PM_M2, PM_M3; same plan, partial-sum
// layouts and results as the recomputing tensor-core pass.
cudaError_t cp3_tc_contract_launch(const Cp3Plan &plan, const Cp3Args &a, int mode_set, cudaStream_t s);

// Batched FP32 pass over the work table (every job of the table padded to rank RP): mode_set
// PM_M1 | PM_OBJ, PM_M2 or PM_M3 (den 0 or 1), or PM_M1 | PM_M2 | PM_M3 | PM_OBJ (den 0).
// grid <= 0: a persistent grid of every CTA that fits on the current device at once.
cudaError_t cp3_batched_launch(int RP, const BatchTable<Cp3Args> &t, int mode_set, int den, int grid,
                               cudaStream_t s);

// ---------------------------------------------------------------------------------
// Small kernels (epilogue.cu)
// ---------------------------------------------------------------------------------
cudaError_t pad_factor(const float *src, int rows, int R, float *dst, int RP, cudaStream_t s);
cudaError_t unpad_factor(const float *src, int rows, int R, int RP, float *dst, cudaStream_t s);
// out[r] = prod over the given factors of colsum(f)[r] (FP64 sums), r < RP.
cudaError_t colsum_prod(int nf, const float *const *f, const int *rows, int RP, float *out,
                        cudaStream_t s);
// Reduce partial sums (fixed order) and apply the multiplicative update:
//   out = max(pre * (sum pn / D)^gamma, eps), D = sum pd or den_closed[r];
// optionally chi1_out = chi1(out, ref), chi2_out = chi2(out, ref).  Columns r >= R -> 0.
struct MuEpiArgs {
    const float *pn, *pd;
    int n_parts, rows, RP, R;
    const float *den_closed;
    const float *pre;
    float *out;
    const float *ref;
    float *chi1_out, *chi2_out;
    float beta, gamma, eps;
};
cudaError_t mu_epilogue(const MuEpiArgs &e, cudaStream_t s);

// Row blocking shared by prep_factors and mode_update: blocks of rows_per_block(rows, RP)
// rows (a multiple of 256 / RP, at most 512 blocks), column-sum partials [block][RP] in FP64.
__host__ __device__ inline int rows_per_block(int rows, int RP) {
    const int G = 256 / RP;
    const int per = (rows + 512 * G - 1) / (512 * G);
    return G * (per > 0 ? per : 1);
}
__host__ __device__ inline int row_blocks(int rows, int RP) { return (rows + rows_per_block(rows, RP) - 1) / rows_per_block(rows, RP); }

// One launch over the three factors: F[m] = padded copy of src[m] (rows x R -> rows x RP,
// zero columns r >= R), optional extra copies into Ft / C1 / C2, and optional FP64
// column-sum partials cs[m][block][RP] of the padded rows.
struct PrepArgs {
    const float *src[3];
    int rows[3];
    int R, RP;
    float *F[3], *Ft[3], *C1[3], *C2[3];
    double *cs[3];
};
cudaError_t prep_factors(const PrepArgs &p, cudaStream_t s);

// Multiplicative update of one padded factor in row blocks (same arithmetic as mu_epilogue):
//   out = max(pre * (sum_p pn / D)^gamma, eps), D = sum_p pd, den_closed[r], or, with cs_in,
//   prod_k sum_b cs_in[k][b][r] (the closed-form KL denominator from column-sum partials);
// optional chi1 / chi2 outputs, an unpadded copy user_out (rows x R), FP64 column-sum
// partials of the result cs_out[block][RP], and (block 0) the fixed-order FP64 sum of
// obj_n objective partials into *obj_out.
// Extrapolated block MM: per factor m < 3, A / Aprev are the user's I_m x R iterate and
// previous iterate (Aprev is overwritten with A), F the padded iterate, D / E padded
// workspaces (displacement, extrapolated block), nrm FP64 norm partials [row block][RP].
// Optional: E2 / E3 receive copies of E, cs the FP64 column-sum partials of E ([row block][RP],
// the row blocking of prep_factors).
struct ExtrapArgs {
    const float *A[3];
    float *Aprev[3];
    const float *F[3];
    float *D[3], *E[3];
    float *E2[3], *E3[3];
    double *nrm[3];
    double *cs[3];
    int rows[3];
    int R, RP;
    float alpha, cap, delta, eps;
};
cudaError_t extrapolate(const ExtrapArgs &x, cudaStream_t s);

// Order N >= 4 on the 3-way kernels (runs of consecutive modes merged): Khatri-Rao factor of a
// run's padded factors L (rows = prod of the run's dims, row-major) with FP64 column-sum partials,
// and the update of a mode inside a run from the run's contraction.
struct KrArgs {
    const float *L[8];
    int dims[8];
    int M, rows, RP;
    float *out;   // KR [rows][RP] or null
    double *cs;   // column-sum partials [row block][RP] or null
};
cudaError_t kr_merge(const KrArgs &k, cudaStream_t s);
// Update of mode n inside a merged run, one launch: Num (and Den unless closed) folded from the
// run's partials (parts summed in part order in FP32, the fold over the run's other indices in
// FP64: CPContr^(n) over the merged index); at beta = 1 Den[r] =
// prod over cf of the column sums (FP64); then out = max(pre * (Num / Den)^gamma, eps) with
// optional chi1 / chi2 against ref and an unpadded copy into user.
struct RunUpdArgs {
    const float *pn, *pd;  // [n_parts][rows][RP]; pd null: closed form from cf
    const float *num_rows; // when set: Num^(n) itself, [dims[n]][RP] (pn and Ln unused)
    int n_parts, rows;
    const float *Ln[8], *Ld[8];
    int dims[8];
    int M, n;
    const float *cf[8];
    int cf_rows[8];
    int ncf;
    const float *pre, *ref;
    float *out, *chi1, *chi2, *user;
    int R, RP;
    float beta, gamma, eps;
};
cudaError_t run_update(const RunUpdArgs &u, cudaStream_t s);

struct UpdArgs {
    MuEpiArgs e;
    const double *cs_in[2];
    int cs_nb[2];
    int n_cs;
    double *cs_out;
    float *user_out;
    const double *obj_parts;
    int obj_n;
    double *obj_out;
};
cudaError_t mode_update(const UpdArgs &u, cudaStream_t s);
// The same two kernels over a batched work table (items: row blocks of each job's factors for
// prep; row blocks of mode u.e's factor, plus the objective block when obj_out is set, for the
// update), on a persistent grid of `grid` CTAs.
int prep_items(const PrepArgs &p);
int mode_update_items(const UpdArgs &u);
cudaError_t prep_batched(const BatchTable<PrepArgs> &t, int grid, cudaStream_t s);
cudaError_t mode_update_batched(const BatchTable<UpdArgs> &t, int grid, cudaStream_t s);
cudaError_t reduce_objective(const double *parts, int n, double add_const_unused, double *out,
                             cudaStream_t s);
// *out = (fixed-order sum of a[0..na)) + (fixed-order sum of b[0..nb)).
cudaError_t reduce_objective2(const double *a, int na, const double *b, int nb, double *out, cudaStream_t s);
cudaError_t copy_f32(const float *src, float *dst, int64_t n, cudaStream_t s);

}  // namespace ntf
