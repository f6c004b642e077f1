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
    int wait_limit = 0;           // polls of a bounded wait (0: the kernels' built-in limit)
    int timeout_probe = 0;        // next tensor-core passes: one wait that runs out, nothing issued
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
    if (o.cache != NTF_CACHE_AUTO && o.cache != NTF_CACHE_NONE && o.cache != NTF_CACHE_BF16)
        return fail(ctx, NTF_ERR_ARG, "unknown cache mode %d", o.cache);
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
// J-CoMM cache choice (beta != 1, tensor-core passes): per shape / precision / beta class, the
// timed extra cost of the cache-writing first pass and one recomputing / contraction-only pass
struct CacheTimes {
    float write_extra_ms, recompute_ms, contract_ms;
};
std::map<TuneKey, CacheTimes> g_cache_tuned;

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
                   CpDense &s, const ntf_opts *tune_opts = nullptr, int tune_bk = 0, int tune_ms = 0, int min_rp = 0,
                   bool nox = false) {
    s.I = (int)X->dims[0];
    s.J = (int)X->dims[1];
    s.K = (int)X->dims[2];
    s.R = R;
    // tensor-core passes where the request asks for them and the shapes allow (rank padded
    // to 32, rows of X 16-byte aligned for TMA); FP32 CUDA-core passes otherwise
    // (an X-free pass reads no X, so neither K's alignment nor X's matters to it)
    const bool tc = precision != NTF_PREC_FP32 && R <= 32 && (nox || ntf::cp3_tc_eligible(32, s.K, X->values));
    s.RP = tc ? 32 : std::max(rank_pad(R), min_rp);
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
        a.wait_limit = ctx->wait_limit;
        a.timeout_probe = ctx->timeout_probe;
        NTF_CUDA(ntf::cp3_tc_launch(s.plan, a, ms, den, st));
    } else {
        NTF_CUDA(ntf::cp3_launch(s.plan, a_in, ms, den, st));
    }
    return NTF_OK;
}

int launch_contract(ntf_ctx *ctx, const CpDense &s, const ntf::Cp3Args &a_in, int ms, cudaStream_t st) {
    PassTimer t(ctx, st);
    ntf::Cp3Args a = a_in;
    a.err = ctx->status;
    a.wait_limit = ctx->wait_limit;
    a.timeout_probe = ctx->timeout_probe;
    NTF_CUDA(ntf::cp3_tc_contract_launch(s.plan, a, ms, st));
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
    if (rc == NTF_ERR_CUDA) {
        char prev[sizeof(ctx->err)];
        snprintf(prev, sizeof(prev), "%s", ctx->err);
        return fail(ctx, rc, "autotuning launch failed: %s", prev);
    }
    if (rc) return rc;
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

// Times, once per key, the extra cost of the cache-writing first pass and one mode-2 pass of
// each kind (the timing launches write only the partial-sum workspaces and the cache, which the
// real passes overwrite).  Skipped during stream capture (the cache is then used).
int tune_cache(ntf_ctx *ctx, const CpDense &s, const ntf::Cp3Args &a, const ntf::Cp3Args &c, float beta,
               CacheTimes &out, cudaStream_t st) {
    const TuneKey key{ctx->device, s.I, s.J, s.K, s.RP, s.tc, s.plan.s3, ntf::beta_kind(beta), -1};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_cache_tuned.find(key);
        if (it != g_cache_tuned.end()) {
            out = it->second;
            return NTF_OK;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NTF_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        out = CacheTimes{0.0f, 1.0f, 0.0f};
        return NTF_OK;
    }
    cudaEvent_t ev[2];
    NTF_CUDA(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(ctx, NTF_ERR_CUDA, "event creation failed");
    }
    int rc = NTF_OK;
    float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // 0: first pass without, 1: with the cache outputs; 2: mode-2 recompute; 3: mode-2 contraction
    for (int v = 0; v < 4 && !rc; ++v) {
        auto go = [&]() {
            if (v == 0) return launch_pass(ctx, s, a, ntf::PM_M1 | ntf::PM_OBJ, 1, st);
            if (v == 1) return launch_pass(ctx, s, c, ntf::PM_M1 | ntf::PM_OBJ, 1, st);
            if (v == 2) return launch_pass(ctx, s, a, ntf::PM_M2, 1, st);
            return launch_contract(ctx, s, c, ntf::PM_M2, st);
        };
        if ((rc = go())) break;  // untimed
        if (cudaEventRecord(ev[0], st) != cudaSuccess) { rc = NTF_ERR_CUDA; break; }
        for (int r = 0; r < 2 && !rc; ++r) rc = go();
        if (rc) break;
        if (cudaEventRecord(ev[1], st) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess ||
            cudaEventElapsedTime(&t[v], ev[0], ev[1]) != cudaSuccess)
            rc = NTF_ERR_CUDA;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc == NTF_ERR_CUDA) {
        char prev[sizeof(ctx->err)];
        snprintf(prev, sizeof(prev), "%s", ctx->err);
        return fail(ctx, rc, "cache autotuning failed: %s", prev);
    }
    if (rc) return rc;
    out = CacheTimes{(t[1] - t[0]) / 2, t[2] / 2, t[3] / 2};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_cache_tuned[key] = out;
    return NTF_OK;
}

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
        for (int m = 0; m < 3; ++m) {
            a.rec[m] = s.Ft[m];
            a.num[m] = s.C1[m];
            a.den[m] = s.C2[m];
        }
        // Reference-powered tensors (Section 5.3): with the cache, the first pass also writes
        // the BF16 P~ / Q~ its contractions consume and the other 3 L - 1 passes contract them
        bool cache = s.plan.tc && o.cache != NTF_CACHE_NONE;
        ntf::Cp3Args c = a;
        if (cache) {
            c.kp = (s.K + 7) & ~7;
            const size_t bytes = sizeof(uint16_t) * (size_t)s.I * s.J * c.kp;
            c.pc = ws_get(ctx, "cpPc", bytes);
            c.qc = ws_get(ctx, "cpQc", bytes);
            if (!c.pc || !c.qc) return fail(ctx, NTF_ERR_OOM, "P~ / Q~ cache allocation failed");
            if (o.cache == NTF_CACHE_AUTO && o.autotune) {
                CacheTimes ct{};
                if ((rc = tune_cache(ctx, s, a, c, beta, ct, st))) return rc;
                const int later = 3 * o.inner_L - 1;
                cache = ct.write_extra_ms + later * ct.contract_ms < later * ct.recompute_ms;
            }
        }
        for (int l = 0; l < o.inner_L; ++l) {
            for (int n = 0; n < 3; ++n) {
                int ms = (n == 0 ? ntf::PM_M1 : n == 1 ? ntf::PM_M2 : ntf::PM_M3);
                if (l == 0 && n == 0) {
                    if (objective_dev) ms |= ntf::PM_OBJ;
                    rc = launch_pass(ctx, s, cache ? c : a, ms, 1, st);
                } else {
                    rc = cache ? launch_contract(ctx, s, c, ms, st) : launch_pass(ctx, s, a, ms, 1, st);
                }
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
// The N modes are cut into three runs of consecutive modes, [0, a), [a, b), [b, N); X
// (row-major) is then the 3-way tensor (prod of each run's dims), and a run of several modes
// has the Khatri-Rao product of its factors (row-major over the run) as its 3-way factor.  A
// mode alone in its run is a 3-way mode; a mode inside a longer run takes that run's 3-way
// contraction and folds it against the run's other factors (CPContr^(n) over the merged index,
// Section 6.1).
struct NWay {
    int N;
    int64_t dims[8];
    int gb[3], ge[3];      // runs of modes
    int view[8];           // run of each mode
    ntf_tensor X3;
    int64_t dims3[3];
    // padded current / reference / chi1 / chi2 blocks of each mode: the view's slot for a
    // mode alone in its run, a buffer of its own otherwise (the slot then holds the run's
    // Khatri-Rao product)
    float *P[8], *Pt[8], *C1P[8], *C2P[8];
};

bool nway_single(const NWay &w, int v) { return w.ge[v] - w.gb[v] == 1; }

// Run boundaries: opts->merge when given, else the split whose padded 3-way tile work is
// least, tensor-core eligibility (rank <= 32, last run's extent a multiple of 4) weighing 8x.
int nway_split(ntf_ctx *ctx, const ntf_tensor *X, int R, const ntf_opts &o, int precision, int &a, int &b,
               bool nox = false) {
    const int N = X->order;
    auto extents = [&](int ca, int cb, double *e) {  // the runs' extents; false past 32 bits
        e[0] = e[1] = e[2] = 1.0;
        for (int m = 0; m < N; ++m) e[m < ca ? 0 : m < cb ? 1 : 2] *= (double)X->dims[m];
        return e[0] <= 2147483647.0 && e[1] <= 2147483647.0 && e[2] <= 2147483647.0;
    };
    double e[3];
    if (o.merge) {
        a = o.merge / 16;
        b = o.merge % 16;
        if (!(1 <= a && a < b && b <= N - 1))
            return fail(ctx, NTF_ERR_ARG, "merge %d does not split %d modes into three runs", o.merge, N);
        if (!extents(a, b, e)) return fail(ctx, NTF_ERR_SHAPE, "a run of the requested cut exceeds 32-bit extents");
        return NTF_OK;
    }
    double best = -1.0;
    for (int ca = 1; ca <= N - 2; ++ca)
        for (int cb = ca + 1; cb <= N - 1; ++cb) {
            if (!extents(ca, cb, e)) continue;
            const bool tc = precision != NTF_PREC_FP32 && R <= 32 &&
                            (nox || ntf::cp3_tc_eligible(32, (int)e[2], X->values));
            const double kb = tc ? 128.0 : 64.0;
            const double cells = e[0] * std::ceil(e[1] / 128.0) * 128.0 * std::ceil(e[2] / kb) * kb;
            const double cost = cells * (tc ? 1.0 : 8.0);
            if (best < 0.0 || cost < best) {
                best = cost;
                a = ca;
                b = cb;
            }
        }
    if (best < 0.0) return fail(ctx, NTF_ERR_SHAPE, "no split of the modes fits 32-bit extents");
    return NTF_OK;
}

int nway_setup(ntf_ctx *ctx, const ntf_tensor *X, int R, bool jcomm, bool need_den, int precision,
               const ntf_opts &o, CpDense &s, NWay &w, int min_rp = 0, bool nox = false) {
    w.N = X->order;
    int a = 0, b = 0;
    int rc = nway_split(ctx, X, R, o, precision, a, b, nox);
    if (rc) return rc;
    w.gb[0] = 0, w.ge[0] = a, w.gb[1] = a, w.ge[1] = b, w.gb[2] = b, w.ge[2] = w.N;
    for (int v = 0; v < 3; ++v) {
        w.dims3[v] = 1;
        for (int m = w.gb[v]; m < w.ge[v]; ++m) {
            w.dims[m] = X->dims[m];
            w.dims3[v] *= X->dims[m];
            w.view[m] = v;
        }
    }
    w.X3 = *X;
    w.X3.order = 3;
    w.X3.dims = w.dims3;
    if ((rc = cp_dense_setup(ctx, &w.X3, R, jcomm, need_den, precision, s, nullptr, 0, 0, min_rp, nox))) return rc;
    const bool chi = jcomm && need_den;
    for (int m = 0; m < w.N; ++m) {
        const int v = w.view[m];
        if (nway_single(w, v)) {
            w.P[m] = s.F[v];
            w.Pt[m] = jcomm ? s.Ft[v] : s.F[v];
            w.C1P[m] = chi ? s.C1[v] : nullptr;
            w.C2P[m] = chi ? s.C2[v] : nullptr;
            continue;
        }
        const size_t fb = sizeof(float) * (size_t)w.dims[m] * s.RP;
        const std::string k = std::to_string(m);
        w.P[m] = (float *)ws_get(ctx, "nwL" + k, fb);
        w.Pt[m] = jcomm ? (float *)ws_get(ctx, "nwLt" + k, fb) : w.P[m];
        w.C1P[m] = chi ? (float *)ws_get(ctx, "nwC1" + k, fb) : nullptr;
        w.C2P[m] = chi ? (float *)ws_get(ctx, "nwC2" + k, fb) : nullptr;
        if (!w.P[m] || !w.Pt[m] || (chi && (!w.C1P[m] || !w.C2P[m])))
            return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    }
    return NTF_OK;
}

// Khatri-Rao product of run v's blocks B[m] (row-major over the run) into out, with FP64
// column-sum partials into cs (either may be null)
cudaError_t nway_merge(const NWay &w, const CpDense &s, int v, float *const *B, float *out, double *cs,
                       cudaStream_t st) {
    ntf::KrArgs k{};
    k.M = w.ge[v] - w.gb[v];
    for (int j = 0; j < k.M; ++j) {
        k.L[j] = B[w.gb[v] + j];
        k.dims[j] = (int)w.dims[w.gb[v] + j];
    }
    k.rows = (int)w.dims3[v];
    k.RP = s.RP;
    k.out = out;
    k.cs = cs;
    return ntf::kr_merge(k, st);
}

// Padded working blocks from the user's factors: the 3-way slots of single-mode runs in one
// prep launch (with reference / chi copies and column sums), the merged runs' own buffers, then
// the merged slots (reference slot for J-CoMM, chi slots equal to it at the start).
int nway_init(ntf_ctx *ctx, NWay &w, CpDense &s, const float *const *factors, bool ref, bool chi,
              cudaStream_t st) {
    ntf::PrepArgs p{};
    for (int v = 0; v < 3; ++v) {
        if (!nway_single(w, v)) continue;  // rows 0: no blocks for this slot
        const int m = w.gb[v];
        p.src[v] = factors[m];
        p.rows[v] = (int)w.dims[m];
        p.F[v] = s.F[v];
        p.Ft[v] = ref ? s.Ft[v] : nullptr;
        p.C1[v] = chi ? s.C1[v] : nullptr;
        p.C2[v] = chi ? s.C2[v] : nullptr;
        p.cs[v] = s.cs[v];
    }
    p.R = s.R;
    p.RP = s.RP;
    NTF_CUDA(ntf::prep_factors(p, st));
    for (int m = 0; m < w.N; ++m) {
        if (nway_single(w, w.view[m])) continue;
        const int64_t nel = w.dims[m] * s.RP;
        NTF_CUDA(ntf::pad_factor(factors[m], (int)w.dims[m], s.R, w.Pt[m], s.RP, st));
        if (ref) NTF_CUDA(ntf::copy_f32(w.Pt[m], w.P[m], nel, st));
        if (chi) {
            NTF_CUDA(ntf::copy_f32(w.Pt[m], w.C1P[m], nel, st));
            NTF_CUDA(ntf::copy_f32(w.Pt[m], w.C2P[m], nel, st));
        }
    }
    for (int v = 0; v < 3; ++v) {
        if (nway_single(w, v)) continue;
        float *slot = ref ? s.Ft[v] : s.F[v];
        NTF_CUDA(nway_merge(w, s, v, w.Pt, slot, s.cs[v], st));
        if (chi) {
            NTF_CUDA(ntf::copy_f32(slot, s.C1[v], w.dims3[v] * s.RP, st));
            NTF_CUDA(ntf::copy_f32(slot, s.C2[v], w.dims3[v] * s.RP, st));
        }
    }
    return NTF_OK;
}

// Update of a mode inside a merged run from the run's 3-way partial sums: Num folded against
// Lnum, Den folded against Lden or, at beta = 1, the closed form (product of the column sums of
// every other current block); MU from pre into out, with chi1 / chi2 of the result against ref
// when those are given, and an unpadded copy into user when given.
struct RunUpd {
    float *const *Lnum, *const *Lden;
    const float *pre;
    float *out, *user;
    const float *ref;
    float *chi1, *chi2;
};

int nway_run_update(ntf_ctx *ctx, NWay &w, CpDense &s, int n, float beta, const ntf_opts &o, bool kl,
                    const RunUpd &q, cudaStream_t st, const float *num_rows = nullptr) {
    const int v = w.view[n];
    const int parts[3] = {s.plan.parts1, s.plan.parts2, s.plan.parts3};
    ntf::RunUpdArgs u{};
    u.pn = s.pn[v];
    u.pd = kl ? nullptr : s.pd[v];
    u.num_rows = num_rows;
    u.n_parts = parts[v];
    u.rows = (int)w.dims3[v];
    u.M = w.ge[v] - w.gb[v];
    for (int j = 0; j < u.M; ++j) {
        u.Ln[j] = q.Lnum[w.gb[v] + j];
        u.Ld[j] = q.Lden[w.gb[v] + j];
        u.dims[j] = (int)w.dims[w.gb[v] + j];
    }
    u.n = n - w.gb[v];
    if (kl)
        for (int m = 0; m < w.N; ++m)
            if (m != n) {
                u.cf[u.ncf] = w.P[m];
                u.cf_rows[u.ncf] = (int)w.dims[m];
                ++u.ncf;
            }
    u.pre = q.pre;
    u.out = q.out;
    u.ref = q.ref;
    u.chi1 = q.chi1;
    u.chi2 = q.chi2;
    u.user = q.user;
    u.R = s.R;
    u.RP = s.RP;
    u.beta = beta;
    u.gamma = ntf::mu_gamma(beta);
    u.eps = (float)o.eps;
    NTF_CUDA(ntf::run_update(u, st));
    return NTF_OK;
}

int mode_flag(int v) { return v == 0 ? ntf::PM_M1 : v == 1 ? ntf::PM_M2 : ntf::PM_M3; }

// B-CoMM sweep (Algorithm 1) over the N modes in order on the 3-way view.
int cp_nway_mu_sweep(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors, const ntf_opts &o,
                     double *objective_dev, cudaStream_t st) {
    const bool kl = ntf::beta_kind(beta) == ntf::BK_KL;
    CpDense s{};
    NWay w{};
    int rc = nway_setup(ctx, X, R, false, !kl, o.precision, o, s, w);
    if (rc) return rc;
    if ((rc = nway_init(ctx, w, s, factors, false, false, st))) return rc;
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
    for (int n = 0; n < w.N; ++n) {
        const int v = w.view[n];
        const bool obj = n == 0 && objective_dev;
        if ((rc = launch_pass(ctx, s, a, mode_flag(v) | (obj ? ntf::PM_OBJ : 0), kl ? 0 : 1, st))) return rc;
        if (nway_single(w, v)) {
            ntf::UpdArgs u = upd_args(s, v, beta, o, kl, s.F[v], factors[n]);
            if (obj) {  // the objective sum rides on the update (its own block)
                u.obj_parts = s.obj;
                u.obj_n = s.plan.grid;
                u.obj_out = objective_dev;
            }
            NTF_CUDA(ntf::mode_update(u, st));
        } else {
            if (obj) NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, objective_dev, st));
            const RunUpd q{w.P, w.P, w.P[n], w.P[n], factors[n], nullptr, nullptr, nullptr};
            if ((rc = nway_run_update(ctx, w, s, n, beta, o, kl, q, st))) return rc;
            NTF_CUDA(nway_merge(w, s, v, w.P, s.F[v], s.cs[v], st));
        }
    }
    return NTF_OK;
}

// J-CoMM (Algorithm 2) on the 3-way view.  The reference blocks stay in Pt / Ft, the current
// ones in P / F.  At beta = 1 (chi1(Z, Zt) = Zt) one pass over X from the reference gives every
// numerator (a merged mode's by folding with the reference blocks of its run) and
// Den^(n) = prod_{m != n} colsum of the current blocks.  Otherwise every block update takes a
// pass with Xhat from the reference and Num / Den contracted against chi1 / chi2 of the current
// blocks (folded inside a merged run, whose slots hold the Khatri-Rao products of its chi blocks).
int cp_nway_jcomm(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors, const ntf_opts &o,
                  double *objective_dev, cudaStream_t st) {
    const bool kl = ntf::beta_kind(beta) == ntf::BK_KL;
    CpDense s{};
    NWay w{};
    int rc = nway_setup(ctx, X, R, true, !kl, o.precision, o, s, w);
    if (rc) return rc;
    if ((rc = nway_init(ctx, w, s, factors, true, !kl, st))) return rc;
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    for (int m = 0; m < 3; ++m) {
        a.rec[m] = s.Ft[m];
        a.num[m] = kl ? s.Ft[m] : s.C1[m];
        a.den[m] = kl ? s.Ft[m] : s.C2[m];
    }
    if (kl) {
        if ((rc = launch_pass(ctx, s, a, ntf::PM_M1 | ntf::PM_M2 | ntf::PM_M3 | ntf::PM_OBJ, 0, st))) return rc;
        if (objective_dev) NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, objective_dev, st));
    }
    for (int l = 0; l < o.inner_L; ++l) {
        for (int n = 0; n < w.N; ++n) {
            const int v = w.view[n];
            float *user = l == o.inner_L - 1 ? factors[n] : nullptr;
            if (!kl) {
                const bool obj = l == 0 && n == 0 && objective_dev;
                if ((rc = launch_pass(ctx, s, a, mode_flag(v) | (obj ? ntf::PM_OBJ : 0), 1, st))) return rc;
                if (obj) NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, objective_dev, st));
            }
            if (nway_single(w, v)) {
                ntf::UpdArgs u = upd_args(s, v, beta, o, kl, s.Ft[v], user);
                if (!kl) {
                    u.e.ref = s.Ft[v];
                    u.e.chi1_out = s.C1[v];
                    u.e.chi2_out = s.C2[v];
                }
                NTF_CUDA(ntf::mode_update(u, st));
                continue;
            }
            const RunUpd q = kl ? RunUpd{w.Pt, w.Pt, w.Pt[n], w.P[n], user, nullptr, nullptr, nullptr}
                                : RunUpd{w.C1P, w.C2P, w.Pt[n], w.P[n], user, w.Pt[n], w.C1P[n], w.C2P[n]};
            if ((rc = nway_run_update(ctx, w, s, n, beta, o, kl, q, st))) return rc;
            if (kl) {
                NTF_CUDA(nway_merge(w, s, v, w.P, nullptr, s.cs[v], st));  // current column sums
            } else {
                NTF_CUDA(nway_merge(w, s, v, w.C1P, s.C1[v], nullptr, st));
                NTF_CUDA(nway_merge(w, s, v, w.C2P, s.C2[v], nullptr, st));
            }
        }
    }
    return NTF_OK;
}

int cp_nway_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, const float *const *factors,
                     const ntf_opts &o, double *out_dev, cudaStream_t st) {
    CpDense s{};
    NWay w{};
    int rc = nway_setup(ctx, X, R, false, false, NTF_PREC_FP32, o, s, w);
    if (rc) return rc;
    if ((rc = nway_init(ctx, w, s, factors, false, false, st))) return rc;
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
    {
        PassTimer t(ctx, st);
        NTF_CUDA(ntf::cp3_launch(s.plan, a, ntf::PM_OBJ, 0, st));
    }
    NTF_CUDA(ntf::reduce_objective(s.obj, s.plan.grid, 0.0, out_dev, st));
    return NTF_OK;
}

// ------------------------------------------------- sparse COO tensors at beta != 1
// Section 6.3: P = X (.) Xhat^(beta-2) vanishes where X does, so Num^(n) is a sum over the
// stored entries (a COO pass, coo.cu); Q = Xhat^(beta-1) does not, so Den^(n) contracts it over
// the whole index space: a dense pass that reads no X (PM_NOX), on the N modes cut into three
// runs as for dense tensors of order N.  The objective splits the same way: the stored entries
// contribute d_beta(x | y) - d_beta(0 | y) and the dense pass sum_i d_beta(0 | y_i).  beta = 0
// is excluded: d_0(x | y) needs x > 0 everywhere, which a tensor with unstored zeros is not.
int coo_beta_check(ntf_ctx *ctx, const ntf_tensor *X, float beta) {
    if (ntf::beta_kind(beta) == ntf::BK_IS)
        return fail(ctx, NTF_ERR_UNSUPPORTED, "beta = 0 needs positive data; a COO tensor has unstored zeros");
    if (X->order < 3) return fail(ctx, NTF_ERR_UNSUPPORTED, "COO tensors at beta != 1 need order >= 3");
    return NTF_OK;
}

// precision: NTF_PREC_FP32 for the FP32 X-free pass, else the tensor-core one (R <= 32; TF32
// reconstruction, BF16 contraction of Q, as for dense tensors)
int cp_coo_beta_setup(ntf_ctx *ctx, const ntf_tensor *X, int R, bool jcomm, const ntf_opts &o, int precision,
                      CpDense &s, NWay &w) {
    ntf_tensor Xv = *X;  // the index space of X, cut into three runs like a dense tensor
    Xv.kind = NTF_DENSE;
    ntf_opts od = o;
    od.precision = precision;
    return nway_setup(ctx, &Xv, R, jcomm, true, precision, od, s, w, R <= 32 ? 32 : 64, /*nox=*/true);
}

// B-CoMM sweep (Algorithm 1; jcomm = false) or J-CoMM outer iteration (Algorithm 2).
int cp_coo_beta(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, float *const *factors, const ntf_opts &o,
                double *objective_dev, cudaStream_t st, bool jcomm) {
    int rc = coo_beta_check(ctx, X, beta);
    if (rc) return rc;
    CpDense s{};
    NWay w{};
    if ((rc = cp_coo_beta_setup(ctx, X, R, jcomm, o, o.precision, s, w))) return rc;
    if ((rc = nway_init(ctx, w, s, factors, jcomm, jcomm, st))) return rc;
    int64_t maxdim = 1;
    for (int m = 0; m < w.N; ++m) maxdim = std::max(maxdim, w.dims[m]);
    float *num = (float *)ws_get(ctx, "coobNum", sizeof(float) * (size_t)maxdim * s.RP);
    if (!num) return fail(ctx, NTF_ERR_OOM, "workspace allocation failed");
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    a.X = nullptr;
    a.vec16 = 0;
    for (int m = 0; m < 3; ++m) {
        a.rec[m] = jcomm ? s.Ft[m] : s.F[m];
        a.num[m] = a.den[m] = jcomm ? s.C2[m] : s.F[m];
    }
    // per-mode blocks for the stored-entry pass: Xhat from rec, Num against chi_1 (J-CoMM)
    float *const *rec = jcomm ? w.Pt : w.P;
    float *const *nf = jcomm ? w.C1P : w.P;
    const int L = jcomm ? o.inner_L : 1;
    for (int l = 0; l < L; ++l) {
        for (int n = 0; n < w.N; ++n) {
            const int v = w.view[n];
            const bool obj = l == 0 && n == 0 && objective_dev;
            if ((rc = launch_pass(ctx, s, a, mode_flag(v) | ntf::PM_NOX | (obj ? ntf::PM_OBJ : 0), 1, st))) return rc;
            double *objp = nullptr;
            int nobj = 0;
            if ((rc = ntf::coo_num_rows(ctx, X, n, s.RP, rec, nf, beta, (float)o.eps, num, obj ? &objp : nullptr,
                                        &nobj, st)))
                return rc;
            if (obj) NTF_CUDA(ntf::reduce_objective2(objp, nobj, s.obj, s.plan.grid, objective_dev, st));
            float *user = l == L - 1 ? factors[n] : nullptr;
            const RunUpd q = jcomm ? RunUpd{w.C1P, w.C2P, w.Pt[n], w.P[n], user, w.Pt[n], w.C1P[n], w.C2P[n]}
                                   : RunUpd{w.P, w.P, w.P[n], w.P[n], user, nullptr, nullptr, nullptr};
            if ((rc = nway_run_update(ctx, w, s, n, beta, o, false, q, st, num))) return rc;
            if (!nway_single(w, v)) {  // the run's 3-way slots follow its updated blocks
                if (jcomm) {
                    NTF_CUDA(nway_merge(w, s, v, w.C1P, s.C1[v], nullptr, st));
                    NTF_CUDA(nway_merge(w, s, v, w.C2P, s.C2[v], nullptr, st));
                } else {
                    NTF_CUDA(nway_merge(w, s, v, w.P, s.F[v], nullptr, st));
                }
            }
        }
    }
    return NTF_OK;
}

int cp_coo_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, int R, const float *const *factors,
                    const ntf_opts &o, double *out_dev, cudaStream_t st) {
    int rc = coo_beta_check(ctx, X, beta);
    if (rc) return rc;
    CpDense s{};
    NWay w{};
    if ((rc = cp_coo_beta_setup(ctx, X, R, false, o, NTF_PREC_FP32, s, w))) return rc;
    if ((rc = nway_init(ctx, w, s, factors, false, false, st))) return rc;
    ntf::Cp3Args a = cp_args(&w.X3, s, o, beta);
    a.X = nullptr;
    a.vec16 = 0;
    for (int m = 0; m < 3; ++m) a.rec[m] = a.num[m] = a.den[m] = s.F[m];
    {
        PassTimer t(ctx, st);
        NTF_CUDA(ntf::cp3_launch(s.plan, a, ntf::PM_OBJ | ntf::PM_NOX, 0, st));
    }
    double *objp = nullptr;
    int nobj = 0;
    if ((rc = ntf::coo_num_rows(ctx, X, 0, s.RP, w.P, w.P, beta, (float)o.eps, nullptr, &objp, &nobj, st))) return rc;
    NTF_CUDA(ntf::reduce_objective2(objp, nobj, s.obj, s.plan.grid, out_dev, st));
    return NTF_OK;
}

// Tucker on a COO tensor, order 3 (Section 6.3): the numerators over the stored entries; at beta = 1
// Q = 1 keeps every denominator a closed form, at other beta the denominators come from X-free dense
// passes.  beta = 0 is excluded (d_0 needs X > 0 everywhere), and so are orders >= 4.
int tucker_kind_check(ntf_ctx *ctx, const ntf_tensor *X, float beta) {
    if (X->kind == NTF_DENSE) return NTF_OK;
    if (X->order != 3) return fail(ctx, NTF_ERR_UNSUPPORTED, "COO Tucker is implemented for order 3");
    if (ntf::beta_kind(beta) == ntf::BK_IS)
        return fail(ctx, NTF_ERR_UNSUPPORTED, "beta = 0 needs positive data; a COO tensor has unstored zeros");
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
    o->merge = 0;
    o->cache = NTF_CACHE_AUTO;
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

int ntf_debug_wait_limit(ntf_ctx *c, int polls, int probe) {
    if (!c) return NTF_ERR_ARG;
    c->wait_limit = polls > 0 ? polls : 0;
    c->timeout_probe = probe != 0;
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
            return cp_coo_beta(ctx, X, beta, rank, factors, o, objective_dev, st, /*jcomm=*/false);
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
    if ((rc = tucker_kind_check(ctx, X, beta))) return rc;
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
                return cp_coo_beta(ctx, X, beta, rank_or_0, factors, o, objective_ref_dev, st, /*jcomm=*/true);
            return ntf::coo_kl_sweep(ctx, X, rank_or_0, factors, o, objective_ref_dev, st, /*jcomm=*/true);
        }
        if (X->order > 3) return cp_nway_jcomm(ctx, X, beta, rank_or_0, factors, o, objective_ref_dev, st);
        return cp_dense_jcomm(ctx, X, beta, rank_or_0, factors, o, objective_ref_dev, st);
    }
    if (model == NTF_TUCKER) {
        if ((rc = tucker_kind_check(ctx, X, beta))) return rc;
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
                return cp_coo_beta_div(ctx, X, beta, rank_or_0, factors, o, out_dev, st);
            return ntf::coo_kl_objective(ctx, X, rank_or_0, factors, o, out_dev, st);
        }
        if (X->order > 3) return cp_nway_beta_div(ctx, X, beta, rank_or_0, factors, o, out_dev, st);
        return cp_dense_beta_div(ctx, X, beta, rank_or_0, factors, o, out_dev, st);
    }
    if (model == NTF_TUCKER) {
        if ((rc = tucker_kind_check(ctx, X, beta))) return rc;
        return ntf::tucker_beta_div(ctx, X, beta, core_dims_or_null, core_or_null, factors, o, out_dev, st);
    }
    return fail(ctx, NTF_ERR_ARG, "unknown model %d", model);
}

int ntf_plan_cut(int model, int order, const int64_t *dims, int rank_or_0, const int64_t *core_dims_or_null,
                 const ntf_opts *opts, float beta, int *a_out, int *b_out) {
    if (!dims || !a_out || !b_out) return NTF_ERR_ARG;
    if (order < 4 || order > 8) return NTF_ERR_UNSUPPORTED;
    for (int n = 0; n < order; ++n)
        if (dims[n] < 1 || dims[n] > (int64_t)0x7fffffff) return NTF_ERR_SHAPE;
    const ntf_opts o = resolve_opts(opts);
    // the option checks of the calls being planned (check_common), without a context
    if (!(beta >= 0.0f && beta < 2.0f)) return NTF_ERR_BETA;
    if (!(o.eps > 0.0) || !(o.eps_x > 0.0) || o.inner_L < 1) return NTF_ERR_ARG;
    if (o.precision != NTF_PREC_FP32 && o.precision != NTF_PREC_TF32 && o.precision != NTF_PREC_3XTF32)
        return NTF_ERR_ARG;
    ntf_tensor X{};
    X.order = order;
    X.dims = dims;
    X.kind = NTF_DENSE;
    X.values = nullptr;  // planning only: a 16-byte-aligned tensor is assumed
    int a = 0, b = 0, rc;
    if (model == NTF_CP) {
        if (rank_or_0 < 1 || rank_or_0 > 64) return NTF_ERR_UNSUPPORTED;
        rc = nway_split(nullptr, &X, rank_or_0, o, o.precision, a, b);
    } else if (model == NTF_TUCKER) {
        if (!core_dims_or_null) return NTF_ERR_ARG;
        rc = ntf::tucker_plan_cut(&X, core_dims_or_null, o, beta, a, b);
    } else {
        return NTF_ERR_ARG;
    }
    if (rc) return rc;
    *a_out = a;
    *b_out = b;
    return NTF_OK;
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
void ctx_wait_opts(ntf_ctx *c, Cp3Args &a) {
    a.err = c->status;
    a.wait_limit = c->wait_limit;
    a.timeout_probe = c->timeout_probe;
}
}  // namespace ntf
