// C ABI of libntf: argument validation, workspaces and the orchestration of the fused
// passes for B-CoMM (Algorithm 1), J-CoMM (Algorithm 2) and the objective.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <string>

#include "../../include/ntf.h"
#include "ntf_internal.h"
#include "ntf_tucker.h"
#include "ntf_coo.h"

struct ntf_ctx {
    int device = 0;
    int num_sms = 0;
    char err[512] = {0};
    int64_t launches = 0;
    std::map<std::string, std::pair<void *, size_t>> ws;
    // pass timing (profiling only)
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // pairs: ev[2k] start, ev[2k+1] stop
    size_t ev_used = 0;           // pairs in use
    int *status = nullptr;        // device status word (bounded waits that gave up)
};

namespace {

int fail(ntf_ctx *c, int code, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define NTF_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(ctx, NTF_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
        ++ctx->launches;                                                                     \
    } while (0)

void *ws_get(ntf_ctx *c, const std::string &name, size_t bytes) {
    if (bytes == 0) bytes = 16;
    auto &e = c->ws[name];
    if (e.first && e.second >= bytes) return e.first;
    if (e.first) cudaFree(e.first);
    e = {nullptr, 0};
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    e = {p, bytes};
    return p;
}

int rank_pad(int R) { return R <= 8 ? 8 : R <= 16 ? 16 : R <= 32 ? 32 : 64; }

ntf_opts resolve_opts(const ntf_opts *o) {
    ntf_opts d;
    ntf_opts_default(&d);
    return o ? *o : d;
}

int check_common(ntf_ctx *ctx, const ntf_tensor *X, float beta, const ntf_opts &o) {
    if (!ctx) return NTF_ERR_ARG;
    if (!X || !X->dims) return fail(ctx, NTF_ERR_ARG, "tensor descriptor or dims is NULL");
    if (!(beta >= 0.0f && beta < 2.0f))
        return fail(ctx, NTF_ERR_BETA, "beta = %g outside [0, 2)", (double)beta);
    if (!(o.eps > 0.0) || !(o.eps_x > 0.0)) return fail(ctx, NTF_ERR_ARG, "eps and eps_x must be > 0");
    if (o.inner_L < 1) return fail(ctx, NTF_ERR_ARG, "inner_L must be >= 1");
    if (o.precision != NTF_PREC_FP32 && o.precision != NTF_PREC_TF32 && o.precision != NTF_PREC_3XTF32)
        return fail(ctx, NTF_ERR_ARG, "unknown precision %d", o.precision);
    if (X->kind != NTF_DENSE && X->kind != NTF_COO) return fail(ctx, NTF_ERR_ARG, "unknown tensor kind");
    if (X->order < 2 || X->order > 8) return fail(ctx, NTF_ERR_UNSUPPORTED, "order %d not in 2..8", X->order);
    for (int n = 0; n < X->order; ++n)
        if (X->dims[n] < 1 || X->dims[n] > (int64_t)0x7fffffff)
            return fail(ctx, NTF_ERR_SHAPE, "dims[%d] = %lld out of range", n, (long long)X->dims[n]);
    if (!X->values) return fail(ctx, NTF_ERR_ARG, "tensor values pointer is NULL");
    if (X->kind == NTF_DENSE && X->order < 3)
        return fail(ctx, NTF_ERR_UNSUPPORTED, "dense kernels implement orders 3..8, got %d", X->order);
    if (X->kind == NTF_COO) {
        if (!X->idx) return fail(ctx, NTF_ERR_ARG, "COO coordinate array is NULL");
        for (int n = 0; n < X->order; ++n)
            if (!X->idx[n]) return fail(ctx, NTF_ERR_ARG, "COO coordinates of mode %d are NULL", n);
        if (X->nnz < 0 || X->nnz > (int64_t)0x7fffffff)
            return fail(ctx, NTF_ERR_SHAPE, "nnz = %lld out of range", (long long)X->nnz);
    }
    return NTF_OK;
}

int check_factors(ntf_ctx *ctx, const ntf_tensor *X, int rank, const float *const *factors) {
    if (rank < 1 || rank > 64) return fail(ctx, NTF_ERR_UNSUPPORTED, "rank %d not in 1..64", rank);
    if (!factors) return fail(ctx, NTF_ERR_ARG, "factor array is NULL");
    for (int n = 0; n < X->order; ++n)
        if (!factors[n]) return fail(ctx, NTF_ERR_ARG, "factor %d is NULL", n);
    return NTF_OK;
}

// ------------------------------------------------------------------ dense CP state
struct CpDense {
    int I, J, K, R, RP;
    ntf::Cp3Plan plan;
    bool tc;
    std::vector<int> tune;  // slab splits to time (empty: plan fixed)
    float *F[3];   // current (padded)
    float *Ft[3];  // reference (padded)
    float *C1[3], *C2[3];
    float *pn[3], *pd[3];
    double *obj;
    float *denc;
    double *cs[3];  // FP64 column-sum partials of F[n] ([row block][RP]), closed-form KL Den
};

// ------------------------------------------------------------------ autotuner
// Process-wide table of timed slab splits for the dense CP pass, keyed by device, shape,
// rank padding, tensor-core use, split TF32, beta class and the pass variant timed.
struct TuneKey {
    int dev, I, J, K, RP, tc, s3, bk, ms;
    bool operator<(const TuneKey &o) const {
        return std::tie(dev, I, J, K, RP, tc, s3, bk, ms) < std::tie(o.dev, o.I, o.J, o.K, o.RP, o.tc, o.s3, o.bk, o.ms);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

// candidate slab splits: the cost model's, and the splits whose grids come closest to 1..4
// waves of one CTA per SM from below and above
std::vector<int> tune_candidates(const ntf::Cp3Plan &model, int I, int sms) {
    const int base = model.n_jt * model.n_kb;
    std::vector<int> c = {model.n_is};
    for (int w = 1; w <= 4; ++w) {
        const int lo = std::max(1, (w * sms) / base), hi = std::max(1, (w * sms + base - 1) / base);
        if (lo <= I) c.push_back(lo);
        if (hi <= I) c.push_back(hi);
    }
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    return c;
}

int cp_dense_setup(ntf_ctx *ctx, const ntf_tensor *X, int R, bool jcomm, bool need_den, int precision,
                   CpDense &s, const ntf_opts *tune_opts = nullptr, int tune_bk = 0, int tune_ms = 0) {
    s.I = (int)X->dims[0];
    s.J = (int)X->dims[1];
    s.K = (int)X->dims[2];
    s.R = R;
    s.RP = rank_pad(R);
    // tensor-core passes where the request asks for them and the shapes allow (rank padded
    // to 32, rows of X 16-byte aligned for TMA); FP32 CUDA-core passes otherwise
    const bool tc = precision != NTF_PREC_FP32 && ntf::cp3_tc_eligible(s.RP, s.K, X->values);
    s.tc = tc;
    // 256-column blocks where the tensor memory allows them (KL: no denominator accumulators;
    // single TF32: no low-part C tile)
    const int kb = tc ? ((!need_den && precision == NTF_PREC_TF32) ? 256 : 128) : 64;
    s.plan = ntf::cp3_plan(s.I, s.J, s.K, s.RP, ctx->num_sms, kb);
    s.plan.s3 = tc && precision == NTF_PREC_3XTF32;
    s.tune.clear();
    ntf::Cp3Plan sizing = s.plan;  // the plan with the most partial sums among those that may run
    if (tune_opts && tune_opts->autotune) {
        const TuneKey key{ctx->device, s.I, s.J, s.K, s.RP, tc, s.plan.s3, tune_bk, tune_ms};
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            const int s3 = s.plan.s3;
            s.plan = ntf::cp3_plan(s.I, s.J, s.K, s.RP, ctx->num_sms, kb, it->second);
            s.plan.s3 = s3;
            sizing = s.plan;
        } else {
            s.tune = tune_candidates(s.plan, s.I, ctx->num_sms);
            sizing = ntf::cp3_plan(s.I, s.J, s.K, s.RP, ctx->num_sms, kb, s.tune.back());
        }
    }
    const int dims[3] = {s.I, s.J, s.K};
    const int parts[3] = {sizing.parts1, std::max(sizing.parts2, s.plan.parts2), std::max(sizing.parts3, s.plan.parts3)};
    for (int n = 0; n < 3; ++n) {
        size_t fb = sizeof(float) * (size_t)dims[n] * s.RP;
        s.F[n] = (float *)ws_get(ctx, "cpF" + std::to_string(n), fb);
        s.Ft[n] = jcomm ? (float *)ws_get(ctx, "cpFt" + std::to_string(n), fb) : nullptr;
        s.C1[n] = jcomm ? (float *)ws_get(ctx, "cpC1" + std::to_string(n), fb) : nullptr;
        s.C2[n] = jcomm ? (float *)ws_get(ctx, "cpC2" + std::to_string(n), fb) : nullptr;
        size_t pb = sizeof(float) * (size_t)parts[n] * dims[n] * s.RP;
        s.pn[n] = (float *)ws_get(ctx, "cpPn" + std::to_string(n), pb);
        s.pd[n] = need_den ? (float *)ws_get(ctx, "cpPd" + std::to_string(n), pb) : nullptr;
        if (!s.F[n] || !s.pn[n] || (jcomm && (!s.Ft[n] || !s.C1[n] || !s.C2[n])) || (need_den && !s.pd[n]))
            return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    }
    s.obj = (double *)ws_get(ctx, "cpObj", sizeof(double) * (size_t)std::max(s.plan.grid, sizing.grid));
    s.denc = (float *)ws_get(ctx, "cpDenc", sizeof(float) * 64);
    if (!s.obj || !s.denc) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    for (int n = 0; n < 3; ++n) {
        s.cs[n] = (double *)ws_get(ctx, "cpCs" + std::to_string(n),
                                   sizeof(double) * (size_t)ntf::row_blocks(dims[n], s.RP) * s.RP);
        if (!s.cs[n]) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    }
    return NTF_OK;
}

ntf::Cp3Args cp_args(const ntf_tensor *X, const CpDense &s, const ntf_opts &o, float beta) {
    ntf::Cp3Args a{};
    a.X = X->values;
    a.I = s.I;
    a.J = s.J;
    a.K = s.K;
    a.bkind = ntf::beta_kind(beta);
    a.beta = beta;
    a.eps = (float)o.eps;
    a.eps_x = (float)o.eps_x;
    a.n_jt = s.plan.n_jt;
    a.n_kb = s.plan.n_kb;
    a.n_is = s.plan.n_is;
    a.vec16 = (s.K % 4 == 0) && ((reinterpret_cast<uintptr_t>(X->values) & 15) == 0);
    a.p1n = s.pn[0];
    a.p1d = s.pd[0];
    a.p2n = s.pn[1];
    a.p2d = s.pd[1];
    a.p3n = s.pn[2];
    a.p3d = s.pd[2];
    a.obj = s.obj;
    a.err = nullptr;
    return a;
}

// Brackets a fused-pass launch with timing events when profiling is enabled.
struct PassTimer {
    ntf_ctx *c;
    cudaStream_t st;
    cudaEvent_t stop = nullptr;
    PassTimer(ntf_ctx *c_, cudaStream_t s) : c(c_), st(s) {
        if (!c->timing) return;
        if (c->ev_used * 2 + 2 > c->ev.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
            c->ev.push_back(a);
            c->ev.push_back(b);
        }
        cudaEventRecord(c->ev[c->ev_used * 2], st);
        stop = c->ev[c->ev_used * 2 + 1];
        ++c->ev_used;
    }
    ~PassTimer() {
        if (stop) cudaEventRecord(stop, st);
    }
};

int launch_pass(ntf_ctx *ctx, const CpDense &s, const ntf::Cp3Args &a_in, int ms, int den, cudaStream_t st) {
    PassTimer t(ctx, st);
    if (s.plan.tc) {
        if (!ntf::cp3_tc_supported(ms, den))
            return fail(ctx, NTF_ERR_UNSUPPORTED, "pass variant %d/%d has no tensor-core kernel", ms, den);
        ntf::Cp3Args a = a_in;
        a.err = ctx->status;
        NTF_CUDA(ntf::cp3_tc_launch(s.plan, a, ms, den, st));
    } else {
        NTF_CUDA(ntf::cp3_launch(s.plan, a_in, ms, den, st));
    }
    return NTF_OK;
}

// Padded working copies of the user's factors (and reference / chi copies) in one launch.
ntf::PrepArgs prep_args(const CpDense &s, float *const *factors, bool ref, bool chi, bool colsums) {
    ntf::PrepArgs p{};
    const int dims[3] = {s.I, s.J, s.K};
    for (int n = 0; n < 3; ++n) {
        p.src[n] = factors[n];
        p.rows[n] = dims[n];
        p.F[n] = s.F[n];
        p.Ft[n] = ref ? s.Ft[n] : nullptr;
        p.C1[n] = chi ? s.C1[n] : nullptr;
        p.C2[n] = chi ? s.C2[n] : nullptr;
        p.cs[n] = colsums ? s.cs[n] : nullptr;
    }
    p.R = s.R;
    p.RP = s.RP;
    return p;
}

// Update of mode n from its partial sums; closed-form KL denominators from the other two
// factors' column-sum partials when `closed`; the result also goes unpadded to `user`.
ntf::UpdArgs upd_args(const CpDense &s, int n, float beta, const ntf_opts &o, bool closed, const float *pre,
                      float *user) {
    const int dims[3] = {s.I, s.J, s.K};
    const int parts[3] = {s.plan.parts1, s.plan.parts2, s.plan.parts3};
    ntf::UpdArgs u{};
    ntf::MuEpiArgs &e = u.e;
    e.pn = s.pn[n];
    e.pd = closed ? nullptr : s.pd[n];
    e.n_parts = parts[n];
    e.rows = dims[n];
    e.RP = s.RP;
    e.R = s.R;
    e.pre = pre;
    e.out = s.F[n];
    e.beta = beta;
    e.gamma = ntf::mu_gamma(beta);
    e.eps = (float)o.eps;
    if (closed) {
        for (int m = 0; m < 3; ++m)
            if (m != n) {
                u.cs_in[u.n_cs] = s.cs[m];
                u.cs_nb[u.n_cs] = ntf::row_blocks(dims[m], s.RP);
                ++u.n_cs;
            }
        u.cs_out = s.cs[n];
    }
    u.user_out = user;
    return u;
}

// Times the pass variant `ms` (factors as in `a`) under each candidate slab split, keeps the
// fastest for this key and switches s.plan to it.  The timing launches write only the
// partial-sum workspaces, which the real passes overwrite.
int tune_plan(ntf_ctx *ctx, const ntf_tensor *X, CpDense &s, const ntf_opts &o, float beta, ntf::Cp3Args a, int ms,
              int den, cudaStream_t st) {
    if (s.tune.empty()) return NTF_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NTF_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        s.tune.clear();  // cost-model plan; nothing is timed or cached during capture
        return NTF_OK;
    }
    cudaEvent_t e0, e1;
    NTF_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, NTF_ERR_CUDA, "event creation failed");
    }
    const ntf::Cp3Plan model = s.plan;
    int best = model.n_is, rc = NTF_OK;
    float best_ms = 0.0f;
    for (int n_is : s.tune) {
        s.plan = ntf::cp3_plan(s.I, s.J, s.K, s.RP, ctx->num_sms, model.KB, n_is);
        s.plan.s3 = model.s3;
        a.n_jt = s.plan.n_jt;
        a.n_kb = s.plan.n_kb;
        a.n_is = s.plan.n_is;
        float t = 0.0f;
        if ((rc = launch_pass(ctx, s, a, ms, den, st))) break;  // untimed: caches, clocks
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = NTF_ERR_CUDA; break; }
        for (int r = 0; r < 2 && !rc; ++r) rc = launch_pass(ctx, s, a, ms, den, st);
        if (rc) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = NTF_ERR_CUDA;
            break;
        }
        if (best_ms == 0.0f || t < best_ms) {
            best_ms = t;
            best = n_is;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc == NTF_ERR_CUDA ? fail(ctx, rc, "autotuning launch failed") : rc;
    s.plan = ntf::cp3_plan(s.I, s.J, s.K, s.RP, ctx->num_sms, model.KB, best);
    s.plan.s3 = model.s3;
    s.tune.clear();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[TuneKey{ctx->device, s.I, s.J, s.K, s.RP, s.tc, s.plan.s3, ntf::beta_kind(beta), ms}] = best;
    return NTF_OK;
}

int cp_dense_mu_sweep(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors,
                      const ntf_opts &o, double *objective_dev, cudaStream_t st) {
    const int bk = ntf::beta_kind(beta);
    const int den = bk != ntf::BK_KL;
    CpDense s{};
    const int tune_ms = ntf::PM_M1 | (objective_dev ? ntf::PM_OBJ : 0);
    int rc = cp_dense_setup(ctx, X, R, false, den, o.precision, s, &o, bk, tune_ms);
    if (rc) return rc;
    NTF_CUDA(ntf::prep_factors(prep_args(s, factors, false, false, !den), st));
    ntf::Cp3Args a = cp_args(X, s, o, beta);
    if (!s.tune.empty()) {
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
        if ((rc = tune_plan(ctx, X, s, o, beta, a, tune_ms, den, st))) return rc;
        a = cp_args(X, s, o, beta);
    }
    for (int n = 0; n < 3; ++n) {
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
        int ms = (n == 0 ? ntf::PM_M1 : n == 1 ? ntf::PM_M2 : ntf::PM_M3);
        if (n == 0 && objective_dev) ms |= ntf::PM_OBJ;
        rc = launch_pass(ctx, s, a, ms, den, st);
        if (rc) return rc;
        ntf::UpdArgs u = upd_args(s, n, beta, o, !den, s.F[n], factors[n]);
        if (n == 0 && objective_dev) {
            u.obj_parts = s.obj;
            u.obj_n = s.plan.grid;
            u.obj_out = objective_dev;
        }
        NTF_CUDA(ntf::mode_update(u, st));
    }
    return NTF_OK;
}

// Outer-reference extrapolation of J-CoMM (Section "Going beyond: Majorization-Minimization
// with Extrapolation", item (iii)): previous iterate and weights of the caller.
struct JExtrap {
    float *const *prev;
    float alpha, cap, delta;
};

int cp_dense_jcomm(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors,
                   const ntf_opts &o, double *objective_dev, cudaStream_t st, const JExtrap *xe = nullptr) {
    const int bk = ntf::beta_kind(beta);
    const bool kl = bk == ntf::BK_KL;
    CpDense s{};
    const int tune_ms = kl ? (ntf::PM_M1 | ntf::PM_M2 | ntf::PM_M3 | ntf::PM_OBJ) : (ntf::PM_M1 | ntf::PM_OBJ);
    int rc = cp_dense_setup(ctx, X, R, true, !kl, o.precision, s, &o, bk, tune_ms);
    if (rc) return rc;
    NTF_CUDA(ntf::prep_factors(prep_args(s, factors, true, !kl, kl), st));
    ntf::Cp3Args a = cp_args(X, s, o, beta);
    if (!s.tune.empty()) {
        for (int m = 0; m < 3; ++m) {
            a.rec[m] = s.Ft[m];
            a.num[m] = kl ? s.Ft[m] : s.C1[m];
            a.den[m] = kl ? s.Ft[m] : s.C2[m];
        }
        if ((rc = tune_plan(ctx, X, s, o, beta, a, tune_ms, kl ? 0 : 1, st))) return rc;
        a = cp_args(X, s, o, beta);
    }
    double *obj_parts = s.obj;
    if (xe) {
        // objective of the incoming iterate, from a mode-1 pass over the unextrapolated blocks
        // with outputs of its own; then the reference (and the starting point of the inner
        // iterations) moves to max(A + alpha_n [A - Aprev]_+, eps), written over Ft (and the chi
        // copies C1, C2), with the column sums of the new reference for the KL denominators
        const int dims[3] = {s.I, s.J, s.K};
        if (objective_dev) {
            const size_t pb = sizeof(float) * (size_t)s.plan.parts1 * s.I * s.RP;
            float *scr = (float *)ws_get(ctx, "cpXscr", pb);
            float *scr2 = kl ? nullptr : (float *)ws_get(ctx, "cpXscr2", pb);
            obj_parts = (double *)ws_get(ctx, "cpXobj", sizeof(double) * (size_t)s.plan.grid);
            if (!scr || (!kl && !scr2) || !obj_parts) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
            ntf::Cp3Args ao = a;
            for (int m = 0; m < 3; ++m) ao.rec[m] = ao.num[m] = ao.den[m] = s.F[m];
            ao.p1n = scr;
            ao.p1d = scr2;
            ao.obj = obj_parts;
            rc = launch_pass(ctx, s, ao, ntf::PM_M1 | ntf::PM_OBJ, kl ? 0 : 1, st);
            if (rc) return rc;
        }
        ntf::ExtrapArgs x{};
        for (int n = 0; n < 3; ++n) {
            const size_t fb = sizeof(float) * (size_t)dims[n] * s.RP;
            x.A[n] = factors[n];
            x.Aprev[n] = xe->prev[n];
            x.F[n] = s.F[n];
            x.D[n] = (float *)ws_get(ctx, "cpXD" + std::to_string(n), fb);
            x.E[n] = s.Ft[n];
            x.E2[n] = kl ? nullptr : s.C1[n];
            x.E3[n] = kl ? nullptr : s.C2[n];
            x.nrm[n] = (double *)ws_get(ctx, "cpXN" + std::to_string(n),
                                        sizeof(double) * (size_t)ntf::row_blocks(dims[n], s.RP) * s.RP);
            x.cs[n] = kl ? s.cs[n] : nullptr;
            x.rows[n] = dims[n];
            if (!x.D[n] || !x.nrm[n]) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
        }
        x.R = R;
        x.RP = s.RP;
        x.alpha = xe->alpha;
        x.cap = xe->cap;
        x.delta = xe->delta;
        x.eps = (float)o.eps;
        NTF_CUDA(ntf::extrapolate(x, st));
    }
    auto update = [&](int l, int n) {
        ntf::UpdArgs u = upd_args(s, n, beta, o, kl, s.Ft[n], l == o.inner_L - 1 ? factors[n] : nullptr);
        if (!kl) {
            u.e.ref = s.Ft[n];
            u.e.chi1_out = s.C1[n];
            u.e.chi2_out = s.C2[n];
        }
        if (l == 0 && n == 0 && objective_dev) {  // D_beta at the reference (incoming iterate)
            u.obj_parts = obj_parts;
            u.obj_n = s.plan.grid;
            u.obj_out = objective_dev;
        }
        return ntf::mode_update(u, st);
    };
    if (kl) {
        // beta = 1: chi1(Z, Zt) = Zt, so every Num_J^(n) depends on the reference only and
        // one pass over X yields all three numerators (and D_beta at the reference);
        // Qtilde == 1 makes each Den_J^(n) the product of column sums of the other
        // current blocks (chi2(Z, Zt) = Z at beta = 1).
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.Ft[m];
        rc = launch_pass(ctx, s, a, ntf::PM_M1 | ntf::PM_M2 | ntf::PM_M3 | ntf::PM_OBJ, 0, st);
        if (rc) return rc;
        for (int l = 0; l < o.inner_L; ++l)
            for (int n = 0; n < 3; ++n) NTF_CUDA(update(l, n));
    } else {
        for (int l = 0; l < o.inner_L; ++l) {
            for (int n = 0; n < 3; ++n) {
                for (int m = 0; m < 3; ++m) {
                    a.rec[m] = s.Ft[m];
                    a.num[m] = s.C1[m];
                    a.den[m] = s.C2[m];
                }
                int ms = (n == 0 ? ntf::PM_M1 : n == 1 ? ntf::PM_M2 : ntf::PM_M3);
                if (l == 0 && n == 0) ms |= ntf::PM_OBJ;
                rc = launch_pass(ctx, s, a, ms, 1, st);
                if (rc) return rc;
                NTF_CUDA(update(l, n));
            }
        }
    }
    return NTF_OK;
}

// Extrapolated B-CoMM sweep (Section "Going beyond: Majorization-Minimization with
// Extrapolation", item (i)): the block of mode n is first moved to
// Ahat = max(A + alpha_n [A - Aprev]_+, eps), Xhat is rebuilt from Ahat and the current
// other blocks, and Ahat is the multiplicative pre-factor.  All Ahat depend only on the
// incoming iterate, so they are formed once, before the first pass.
int cp_dense_mu_sweep_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors,
                             float *const *factors_prev, float alpha, float cap, float delta, const ntf_opts &o,
                             double *objective_dev, cudaStream_t st) {
    const int bk = ntf::beta_kind(beta);
    const int den = bk != ntf::BK_KL;
    CpDense s{};
    // the plan (and its autotuned table entry) of the plain sweep's first pass
    const int tune_ms = ntf::PM_M1 | (objective_dev ? ntf::PM_OBJ : 0);
    int rc = cp_dense_setup(ctx, X, R, false, den, o.precision, s, &o, bk, tune_ms);
    if (rc) return rc;
    const int dims[3] = {s.I, s.J, s.K};
    ntf::ExtrapArgs x{};
    for (int n = 0; n < 3; ++n) {
        const size_t fb = sizeof(float) * (size_t)dims[n] * s.RP;
        x.A[n] = factors[n];
        x.Aprev[n] = factors_prev[n];
        x.F[n] = s.F[n];
        x.D[n] = (float *)ws_get(ctx, "cpXD" + std::to_string(n), fb);
        x.E[n] = (float *)ws_get(ctx, "cpXE" + std::to_string(n), fb);
        x.nrm[n] = (double *)ws_get(ctx, "cpXN" + std::to_string(n),
                                    sizeof(double) * (size_t)ntf::row_blocks(dims[n], s.RP) * s.RP);
        x.rows[n] = dims[n];
        if (!x.D[n] || !x.E[n] || !x.nrm[n]) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    }
    x.R = R;
    x.RP = s.RP;
    x.alpha = alpha;
    x.cap = cap;
    x.delta = delta;
    x.eps = (float)o.eps;
    NTF_CUDA(ntf::prep_factors(prep_args(s, factors, false, false, !den), st));
    ntf::Cp3Args a = cp_args(X, s, o, beta);
    if (!s.tune.empty()) {  // timed on the unextrapolated blocks, before factors_prev changes
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
        if ((rc = tune_plan(ctx, X, s, o, beta, a, tune_ms, den, st))) return rc;
        a = cp_args(X, s, o, beta);
    }
    NTF_CUDA(ntf::extrapolate(x, st));
    if (objective_dev) {
        // D_beta of the incoming iterate: a mode-1 pass from the unextrapolated blocks (its
        // partial sums are overwritten by the first extrapolated pass)
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
        rc = launch_pass(ctx, s, a, ntf::PM_M1 | ntf::PM_OBJ, den, st);
        if (rc) return rc;
    }
    for (int n = 0; n < 3; ++n) {
        for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
        a.rec[n] = x.E[n];
        const int ms = n == 0 ? ntf::PM_M1 : n == 1 ? ntf::PM_M2 : ntf::PM_M3;
        rc = launch_pass(ctx, s, a, ms, den, st);
        if (rc) return rc;
        ntf::UpdArgs u = upd_args(s, n, beta, o, !den, x.E[n], factors[n]);
        if (n == 0 && objective_dev) {
            u.obj_parts = s.obj;
            u.obj_n = s.plan.grid;
            u.obj_out = objective_dev;
        }
        NTF_CUDA(ntf::mode_update(u, st));
    }
    return NTF_OK;
}

// ------------------------------------------------------------ dense CP of order N >= 4
// The leading modes 0..M-1 (M = N - 2) are merged: X (row-major) is then the 3-way tensor
// (prod_{m<M} I_m) x I_{N-2} x I_{N-1}, whose first factor is the Khatri-Rao product of the
// leading factors.  Modes N-2 and N-1 are 3-way modes 2 and 3 of that view; a leading mode n
// takes the view's mode-1 contraction and folds it against the other leading factors
// (CPContr^(n) over the merged index), Section 6.1.
struct NWay {
    int N, M;
    int64_t dims[8];
    int64_t merged;
    ntf_tensor X3;
    int64_t dims3[3];
    float *L[8], *Lt[8];  // padded current / reference leading factors
    float *num, *den;     // folded Num / Den of a leading mode, [max I_n][RP]
};

int nway_setup(ntf_ctx *ctx, const ntf_tensor *X, int R, bool jcomm, bool need_den, int precision, CpDense &s,
               NWay &w, const ntf_opts *tune_opts, int tune_bk, int tune_ms) {
    w.N = X->order;
    w.M = w.N - 2;
    w.merged = 1;
    for (int n = 0; n < w.N; ++n) w.dims[n] = X->dims[n];
    for (int m = 0; m < w.M; ++m) w.merged *= X->dims[m];
    if (w.merged > (int64_t)0x7fffffff) return fail(ctx, NTF_ERR_SHAPE, "product of the leading dimensions too large");
    w.dims3[0] = w.merged;
    w.dims3[1] = X->dims[w.N - 2];
    w.dims3[2] = X->dims[w.N - 1];
    w.X3 = *X;
    w.X3.order = 3;
    w.X3.dims = w.dims3;
    int rc = cp_dense_setup(ctx, &w.X3, R, jcomm, need_den, precision, s, tune_opts, tune_bk, tune_ms);
    if (rc) return rc;
    int64_t maxI = 1;
    for (int m = 0; m < w.M; ++m) {
        const size_t fb = sizeof(float) * (size_t)w.dims[m] * s.RP;
        w.L[m] = (float *)ws_get(ctx, "nwL" + std::to_string(m), fb);
        w.Lt[m] = jcomm ? (float *)ws_get(ctx, "nwLt" + std::to_string(m), fb) : w.L[m];
        if (!w.L[m] || !w.Lt[m]) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
        maxI = std::max(maxI, w.dims[m]);
    }
    w.num = (float *)ws_get(ctx, "nwNum", sizeof(float) * (size_t)maxI * s.RP);
    w.den = (float *)ws_get(ctx, "nwDen", sizeof(float) * (size_t)maxI * s.RP);
    if (!w.num || !w.den) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    return NTF_OK;
}

ntf::KrArgs kr_args(const NWay &w, const CpDense &s, float *const *L, float *out, double *cs) {
    ntf::KrArgs k{};
    for (int m = 0; m < w.M; ++m) {
        k.L[m] = L[m];
        k.dims[m] = (int)w.dims[m];
    }
    k.M = w.M;
    k.rows = (int)w.merged;
    k.RP = s.RP;
    k.out = out;
    k.cs = cs;
    return k;
}

// pads the trailing two factors into the view's F[1], F[2] (and, for J-CoMM, the reference
// copies Ft[1], Ft[2]) with FP64 column-sum partials; the view's mode 1 is left to kr_merge
int nway_prep_trailing(ntf_ctx *ctx, NWay &w, CpDense &s, float *const *factors, bool ref, cudaStream_t st) {
    ntf::PrepArgs p{};
    p.rows[0] = 0;  // no row blocks for the merged slot
    for (int m = 1; m < 3; ++m) {
        p.src[m] = factors[w.M + m - 1];
        p.rows[m] = (int)w.dims[w.M + m - 1];
        p.F[m] = s.F[m];
        p.Ft[m] = ref ? s.Ft[m] : nullptr;
        p.cs[m] = s.cs[m];
    }
    p.R = s.R;
    p.RP = s.RP;
    NTF_CUDA(ntf::prep_factors(p, st));
    return NTF_OK;
}

// update of leading mode n from the view's mode-1 partial sums: fold, closed-form KL
// denominator (product of the column sums of every other current factor) or folded Den, MU
int nway_leading_update(ntf_ctx *ctx, NWay &w, CpDense &s, int n, float beta, const ntf_opts &o, bool kl,
                        float *const *Lfold, const float *pre, float *out, float *user, cudaStream_t st) {
    ntf::FoldArgs f{};
    f.parts = s.pn[0];
    f.n_parts = s.plan.parts1;
    for (int m = 0; m < w.M; ++m) {
        f.L[m] = Lfold[m];
        f.dims[m] = (int)w.dims[m];
    }
    f.M = w.M;
    f.n = n;
    f.rows = (int)w.merged;
    f.R = s.R;
    f.RP = s.RP;
    f.out = w.num;
    NTF_CUDA(ntf::kr_fold(f, st));
    ntf::MuEpiArgs e{};
    e.pn = w.num;
    e.n_parts = 1;
    e.rows = (int)w.dims[n];
    e.RP = s.RP;
    e.R = s.R;
    if (kl) {
        const float *cf[8];
        int rows[8], q = 0;
        for (int m = 0; m < w.M; ++m)
            if (m != n) { cf[q] = w.L[m]; rows[q] = (int)w.dims[m]; ++q; }
        cf[q] = s.F[1]; rows[q] = (int)w.dims[w.N - 2]; ++q;
        cf[q] = s.F[2]; rows[q] = (int)w.dims[w.N - 1]; ++q;
        NTF_CUDA(ntf::colsum_prod(q, cf, rows, s.RP, s.denc, st));
        e.den_closed = s.denc;
    } else {
        f.parts = s.pd[0];
        f.out = w.den;
        NTF_CUDA(ntf::kr_fold(f, st));
        e.pd = w.den;
    }
    e.pre = pre;
    e.out = out;
    e.beta = beta;
    e.gamma = ntf::mu_gamma(beta);
    e.eps = (float)o.eps;
    NTF_CUDA(ntf::mu_epilogue(e, st));
    if (user) NTF_CUDA(ntf::unpad_factor(out, (int)w.dims[n], s.R, s.RP, user, st));
    return NTF_OK;
}

int cp_nway_mu_sweep(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors, const ntf_opts &o,
                     double *objective_dev, cudaStream_t st) {
    const int bk = ntf::beta_kind(beta);
    const bool kl = bk == ntf::BK_KL;
    CpDense s{};
    NWay w{};
    int rc = nway_setup(ctx, X, R, false, !kl, o.precision, s, w, nullptr, 0, 0);
    if (rc) return rc;
    for (int m = 0; m < w.M; ++m) NTF_CUDA(ntf::pad_factor(factors[m], (int)w.dims[m], R, w.L[m], s.RP, st));
    if ((rc = nway_prep_trailing(ctx, w, s, factors, false, st))) return rc;
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
    for (int n = 0; n < w.N; ++n) {
        if (n <= w.M) NTF_CUDA(ntf::kr_merge(kr_args(w, s, w.L, s.F[0], s.cs[0]), st));  // current leading blocks
        if (n < w.M) {
            const int ms = ntf::PM_M1 | ((n == 0 && objective_dev) ? ntf::PM_OBJ : 0);
            if ((rc = launch_pass(ctx, s, a, ms, kl ? 0 : 1, st))) return rc;
            if (n == 0 && objective_dev) NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, objective_dev, st));
            if ((rc = nway_leading_update(ctx, w, s, n, beta, o, kl, w.L, w.L[n], w.L[n], factors[n], st))) return rc;
        } else {
            const int k = n - w.M + 1;  // the view's mode 2 or 3
            if ((rc = launch_pass(ctx, s, a, k == 1 ? ntf::PM_M2 : ntf::PM_M3, kl ? 0 : 1, st))) return rc;
            ntf::UpdArgs u = upd_args(s, k, beta, o, kl, s.F[k], factors[n]);
            NTF_CUDA(ntf::mode_update(u, st));
        }
    }
    return NTF_OK;
}

// J-CoMM at beta = 1 (Section 5.3 with chi1(Z, Zt) = Zt): one pass over X from the reference
// gives every numerator (the leading ones by folding with the reference leading blocks);
// Den^(n) = prod_{m != n} colsum of the current blocks.
int cp_nway_jcomm(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors, const ntf_opts &o,
                  double *objective_dev, cudaStream_t st) {
    if (ntf::beta_kind(beta) != ntf::BK_KL)
        return fail(ctx, NTF_ERR_UNSUPPORTED, "J-CoMM for dense orders N >= 4 is implemented at beta = 1");
    CpDense s{};
    NWay w{};
    int rc = nway_setup(ctx, X, R, true, false, o.precision, s, w, nullptr, 0, 0);
    if (rc) return rc;
    for (int m = 0; m < w.M; ++m) {
        NTF_CUDA(ntf::pad_factor(factors[m], (int)w.dims[m], R, w.Lt[m], s.RP, st));
        NTF_CUDA(ntf::copy_f32(w.Lt[m], w.L[m], w.dims[m] * s.RP, st));
    }
    if ((rc = nway_prep_trailing(ctx, w, s, factors, true, st))) return rc;
    NTF_CUDA(ntf::kr_merge(kr_args(w, s, w.Lt, s.Ft[0], s.cs[0]), st));
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.Ft[m];
    if ((rc = launch_pass(ctx, s, a, ntf::PM_M1 | ntf::PM_M2 | ntf::PM_M3 | ntf::PM_OBJ, 0, st))) return rc;
    if (objective_dev) NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, objective_dev, st));
    for (int l = 0; l < o.inner_L; ++l) {
        for (int n = 0; n < w.N; ++n) {
            float *user = l == o.inner_L - 1 ? factors[n] : nullptr;
            if (n < w.M) {
                // the trailing current blocks sit in the view's F[1], F[2]: until their first
                // update they equal the reference (F = Ft after the prep copies)
                if ((rc = nway_leading_update(ctx, w, s, n, beta, o, true, w.Lt, w.Lt[n], w.L[n], user, st)))
                    return rc;
            } else {
                const int k = n - w.M + 1;
                if (n == w.M) NTF_CUDA(ntf::kr_merge(kr_args(w, s, w.L, nullptr, s.cs[0]), st));  // current leading
                ntf::UpdArgs u = upd_args(s, k, beta, o, true, s.Ft[k], user);
                NTF_CUDA(ntf::mode_update(u, st));
            }
        }
    }
    return NTF_OK;
}

int cp_nway_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, const float *const *factors,
                     const ntf_opts &o, double *out_dev, cudaStream_t st) {
    CpDense s{};
    NWay w{};
    int rc = nway_setup(ctx, X, R, false, false, NTF_PREC_FP32, s, w, nullptr, 0, 0);
    if (rc) return rc;
    for (int m = 0; m < w.M; ++m) NTF_CUDA(ntf::pad_factor(factors[m], (int)w.dims[m], R, w.L[m], s.RP, st));
    NTF_CUDA(ntf::pad_factor(factors[w.N - 2], (int)w.dims[w.N - 2], R, s.F[1], s.RP, st));
    NTF_CUDA(ntf::pad_factor(factors[w.N - 1], (int)w.dims[w.N - 1], R, s.F[2], s.RP, st));
    NTF_CUDA(ntf::kr_merge(kr_args(w, s, w.L, s.F[0], nullptr), st));
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
    {
        PassTimer t(ctx, st);
        NTF_CUDA(ntf::cp3_launch(s.plan, a, ntf::PM_OBJ, 0, st));
    }
    NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, out_dev, st));
    return NTF_OK;
}

int cp_dense_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, const float *const *factors,
                      const ntf_opts &o, double *out_dev, cudaStream_t st) {
    CpDense s{};
    int rc = cp_dense_setup(ctx, X, R, false, false, NTF_PREC_FP32, s);
    if (rc) return rc;
    const int dims[3] = {s.I, s.J, s.K};
    for (int n = 0; n < 3; ++n) NTF_CUDA(ntf::pad_factor(factors[n], dims[n], R, s.F[n], s.RP, st));
    ntf::Cp3Args a = cp_args(X, s, o, beta);
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
    {
        PassTimer t(ctx, st);
        NTF_CUDA(ntf::cp3_launch(s.plan, a, ntf::PM_OBJ, 0, st));
    }
    NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, out_dev, st));
    return NTF_OK;
}

}  // namespace

// =================================================================================== ABI

extern "C" {

void ntf_opts_default(ntf_opts *o) {
    if (!o) return;
    o->eps = 1e-12;
    o->eps_x = 1e-12;
    o->inner_L = 1;
    o->precision = NTF_PREC_FP32;
    o->autotune = 0;
}

int ntf_ctx_create(ntf_ctx **out, int device) {
    if (!out) return NTF_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return NTF_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return NTF_ERR_CUDA;
    ntf_ctx *c = new ntf_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (c->num_sms <= 0) c->num_sms = 1;
    if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess || cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return NTF_ERR_CUDA;
    }
    *out = c;
    return NTF_OK;
}

void ntf_ctx_destroy(ntf_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &kv : c->ws)
        if (kv.second.first) cudaFree(kv.second.first);
    for (auto e : c->ev) cudaEventDestroy(e);
    if (c->status) cudaFree(c->status);
    ntf::tucker_release(c);
    ntf::coo_release(c);
    delete c;
}

const char *ntf_last_error(const ntf_ctx *c) { return c ? c->err : "null context"; }

int64_t ntf_launch_count(const ntf_ctx *c) { return c ? c->launches : 0; }

int ntf_set_pass_timing(ntf_ctx *c, int enable) {
    if (!c) return NTF_ERR_ARG;
    c->timing = enable != 0;
    return NTF_OK;
}

int ntf_device_status(ntf_ctx *c, void *stream) {
    if (!c) return NTF_ERR_ARG;
    cudaSetDevice(c->device);
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(c, NTF_ERR_CUDA, "reading the device status failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (h) {
        cudaMemsetAsync(c->status, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        return fail(c, NTF_ERR_TIMEOUT, "a bounded device-side wait ran out (status %d)", h);
    }
    return NTF_OK;
}

int ntf_pass_timing(ntf_ctx *c, double *total_ms, int64_t *launches) {
    if (!c || !total_ms || !launches) return NTF_ERR_ARG;
    cudaSetDevice(c->device);
    double t = 0.0;
    for (size_t k = 0; k < c->ev_used; ++k) {
        float ms = 0.0f;
        if (cudaEventSynchronize(c->ev[2 * k + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]) != cudaSuccess) {
            cudaGetLastError();
            c->ev_used = 0;
            return fail(c, NTF_ERR_CUDA, "pass timing events failed");
        }
        t += ms;
    }
    *total_ms = t;
    *launches = (int64_t)c->ev_used;
    c->ev_used = 0;
    return NTF_OK;
}

int ntf_cp_mu_sweep(ntf_ctx *ctx, const ntf_tensor *X, float beta, int rank, float *const *factors,
                    const ntf_opts *opts, double *objective_dev, void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    rc = check_factors(ctx, X, rank, factors);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (X->kind == NTF_COO) {
        if (ntf::beta_kind(beta) != ntf::BK_KL)
            return fail(ctx, NTF_ERR_UNSUPPORTED, "COO tensors are implemented for beta = 1 only");
        return ntf::coo_kl_sweep(ctx, X, rank, factors, o, objective_dev, st, /*jcomm=*/false);
    }
    if (X->order > 3) return cp_nway_mu_sweep(ctx, X, beta, rank, factors, o, objective_dev, st);
    return cp_dense_mu_sweep(ctx, X, beta, rank, factors, o, objective_dev, st);
}

int ntf_cp_mu_sweep_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, int rank, float *const *factors,
                           float *const *factors_prev, float alpha, float cap, float delta, const ntf_opts *opts,
                           double *objective_dev, void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    rc = check_factors(ctx, X, rank, factors);
    if (rc) return rc;
    if (X->kind != NTF_DENSE || X->order != 3)
        return fail(ctx, NTF_ERR_UNSUPPORTED, "extrapolated sweeps are implemented for dense order-3 tensors");
    if (!factors_prev) return fail(ctx, NTF_ERR_ARG, "previous-iterate array is NULL");
    for (int n = 0; n < 3; ++n)
        if (!factors_prev[n]) return fail(ctx, NTF_ERR_ARG, "previous iterate %d is NULL", n);
    if (!(alpha >= 0.0f) || !(cap >= 0.0f) || !(delta > 0.0f))
        return fail(ctx, NTF_ERR_ARG, "alpha and cap must be >= 0 and delta > 0");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    return cp_dense_mu_sweep_extrap(ctx, X, beta, rank, factors, factors_prev, alpha, cap, delta, o, objective_dev,
                                    (cudaStream_t)stream);
}

int ntf_cp_jcomm_outer_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, int rank, float *const *factors,
                              float *const *factors_prev, float alpha, float cap, float delta, const ntf_opts *opts,
                              double *objective_dev, void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    rc = check_factors(ctx, X, rank, factors);
    if (rc) return rc;
    if (X->kind != NTF_DENSE || X->order != 3)
        return fail(ctx, NTF_ERR_UNSUPPORTED, "extrapolated outer iterations are implemented for dense order-3 tensors");
    if (!factors_prev) return fail(ctx, NTF_ERR_ARG, "previous-iterate array is NULL");
    for (int n = 0; n < 3; ++n)
        if (!factors_prev[n]) return fail(ctx, NTF_ERR_ARG, "previous iterate %d is NULL", n);
    if (!(alpha >= 0.0f) || !(cap >= 0.0f) || !(delta > 0.0f))
        return fail(ctx, NTF_ERR_ARG, "alpha and cap must be >= 0 and delta > 0");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    const JExtrap xe{factors_prev, alpha, cap, delta};
    return cp_dense_jcomm(ctx, X, beta, rank, factors, o, objective_dev, (cudaStream_t)stream, &xe);
}

int ntf_tucker_mu_sweep(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
                        float *const *factors, const ntf_opts *opts, double *objective_dev, void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    if (X->kind != NTF_DENSE) return fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker is implemented for dense tensors");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    return ntf::tucker_run(ctx, X, beta, core_dims, core, factors, o, objective_dev, (cudaStream_t)stream,
                           /*jcomm=*/false);
}

int ntf_tucker_mu_sweep_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
                               float *const *factors, float *core_prev, float *const *factors_prev, float alpha,
                               float cap, float delta, const ntf_opts *opts, double *objective_dev, void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    if (X->kind != NTF_DENSE) return fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker is implemented for dense tensors");
    if (!(alpha >= 0.0f) || !(cap >= 0.0f) || !(delta > 0.0f))
        return fail(ctx, NTF_ERR_ARG, "alpha and cap must be >= 0 and delta > 0");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    return ntf::tucker_run_extrap(ctx, X, beta, core_dims, core, factors, core_prev, factors_prev, alpha, cap, delta, o,
                                  objective_dev, (cudaStream_t)stream);
}

int ntf_tucker_jcomm_outer_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims,
                                  float *core, float *const *factors, float *core_prev, float *const *factors_prev,
                                  float alpha, float cap, float delta, const ntf_opts *opts, double *objective_dev,
                                  void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    if (X->kind != NTF_DENSE) return fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker is implemented for dense tensors");
    if (!core_prev || !factors_prev) return fail(ctx, NTF_ERR_ARG, "previous iterate is NULL");
    for (int n = 0; n < 3 && n < X->order; ++n)
        if (!factors_prev[n]) return fail(ctx, NTF_ERR_ARG, "previous factor %d is NULL", n);
    if (!(alpha >= 0.0f) || !(cap >= 0.0f) || !(delta > 0.0f))
        return fail(ctx, NTF_ERR_ARG, "alpha and cap must be >= 0 and delta > 0");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    const ntf::TuckerExtrap xe{core_prev, factors_prev, alpha, cap, delta};
    return ntf::tucker_run(ctx, X, beta, core_dims, core, factors, o, objective_dev, (cudaStream_t)stream,
                           /*jcomm=*/true, &xe);
}

int ntf_jcomm_outer(ntf_ctx *ctx, int model, const ntf_tensor *X, float beta, int rank_or_0,
                    const int64_t *core_dims_or_null, float *core_or_null, float *const *factors,
                    const ntf_opts *opts, double *objective_ref_dev, void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (model == NTF_CP) {
        rc = check_factors(ctx, X, rank_or_0, factors);
        if (rc) return rc;
        if (X->kind == NTF_COO) {
            if (ntf::beta_kind(beta) != ntf::BK_KL)
                return fail(ctx, NTF_ERR_UNSUPPORTED, "COO tensors are implemented for beta = 1 only");
            return ntf::coo_kl_sweep(ctx, X, rank_or_0, factors, o, objective_ref_dev, st, /*jcomm=*/true);
        }
        if (X->order > 3) return cp_nway_jcomm(ctx, X, beta, rank_or_0, factors, o, objective_ref_dev, st);
        return cp_dense_jcomm(ctx, X, beta, rank_or_0, factors, o, objective_ref_dev, st);
    }
    if (model == NTF_TUCKER) {
        if (X->kind != NTF_DENSE) return fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker is implemented for dense tensors");
        return ntf::tucker_run(ctx, X, beta, core_dims_or_null, core_or_null, factors, o, objective_ref_dev, st,
                               /*jcomm=*/true);
    }
    return fail(ctx, NTF_ERR_ARG, "unknown model %d", model);
}

int ntf_beta_div(ntf_ctx *ctx, int model, const ntf_tensor *X, float beta, int rank_or_0,
                 const int64_t *core_dims_or_null, const float *core_or_null, const float *const *factors,
                 const ntf_opts *opts, double *out_dev, void *stream) {
    ntf_opts o = resolve_opts(opts);
    int rc = check_common(ctx, X, beta, o);
    if (rc) return rc;
    if (!out_dev) return fail(ctx, NTF_ERR_ARG, "out_dev is NULL");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (model == NTF_CP) {
        rc = check_factors(ctx, X, rank_or_0, factors);
        if (rc) return rc;
        if (X->kind == NTF_COO) {
            if (ntf::beta_kind(beta) != ntf::BK_KL)
                return fail(ctx, NTF_ERR_UNSUPPORTED, "COO tensors are implemented for beta = 1 only");
            return ntf::coo_kl_objective(ctx, X, rank_or_0, factors, o, out_dev, st);
        }
        if (X->order > 3) return cp_nway_beta_div(ctx, X, beta, rank_or_0, factors, o, out_dev, st);
        return cp_dense_beta_div(ctx, X, beta, rank_or_0, factors, o, out_dev, st);
    }
    if (model == NTF_TUCKER) {
        if (X->kind != NTF_DENSE) return fail(ctx, NTF_ERR_UNSUPPORTED, "Tucker is implemented for dense tensors");
        return ntf::tucker_beta_div(ctx, X, beta, core_dims_or_null, core_or_null, factors, o, out_dev, st);
    }
    return fail(ctx, NTF_ERR_ARG, "unknown model %d", model);
}

int ntf_coo_stable_perm(ntf_ctx *ctx, const int32_t *keys, int64_t nnz, int64_t key_range, int32_t *perm_out,
                        void *stream) {
    if (!ctx) return NTF_ERR_ARG;
    if ((!keys || !perm_out) && nnz > 0) return fail(ctx, NTF_ERR_ARG, "keys or perm_out is NULL");
    if (nnz < 0 || nnz > (int64_t)0x7fffffff) return fail(ctx, NTF_ERR_SHAPE, "nnz out of range");
    if (key_range < 1 || key_range > (int64_t)0x7fffffff) return fail(ctx, NTF_ERR_SHAPE, "key_range out of range");
    cudaSetDevice(ctx->device);
    ctx->err[0] = 0;
    return ntf::coo_stable_perm(ctx, keys, nnz, key_range, perm_out, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------ helpers for other units
namespace ntf {
void *ctx_ws(ntf_ctx *c, const char *name, size_t bytes) { return ws_get(c, name, bytes); }
int ctx_fail(ntf_ctx *c, int code, const char *msg) { return fail(c, code, "%s", msg); }
void ctx_count(ntf_ctx *c, int n) { c->launches += n; }
int ctx_num_sms(const ntf_ctx *c) { return c->num_sms; }
int *ctx_status(ntf_ctx *c) { return c->status; }
}  // namespace ntf
