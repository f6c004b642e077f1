// Internal: dense 3-way Tucker block MM and J-CoMM (tucker.cu).
#pragma once
#include "../../include/ntf.h"
#include "ntf_internal.h"

namespace ntf {
void *ctx_ws(ntf_ctx *c, const char *name, size_t bytes);
int ctx_fail(ntf_ctx *c, int code, const char *msg);
void ctx_count(ntf_ctx *c, int n);
int ctx_num_sms(const ntf_ctx *c);
int *ctx_status(ntf_ctx *c);  // device status word of the bounded-wait kernels
void ctx_wait_opts(ntf_ctx *c, Cp3Args &a);  // status word, wait limit and timeout probe of the context

// previous iterate and weights of an outer-reference extrapolation (J-CoMM)
struct TuckerExtrap {
    float *core_prev;
    float *const *factors_prev;
    float alpha, cap, delta;
};
int tucker_run(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
               float *const *factors, const ntf_opts &o, double *objective_dev, cudaStream_t st, bool jcomm,
               const TuckerExtrap *xe = nullptr);
int tucker_beta_div(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, const float *core,
                    const float *const *factors, const ntf_opts &o, double *out_dev, cudaStream_t st);
int tucker_run_extrap(ntf_ctx *ctx, const ntf_tensor *X, float beta, const int64_t *core_dims, float *core,
                      float *const *factors, float *core_prev, float *const *factors_prev, float alpha, float cap,
                      float delta, const ntf_opts &o, double *objective_dev, cudaStream_t st);
void tucker_release(ntf_ctx *ctx);
// the cut of an order N >= 4 Tucker problem into three runs (planning only, no device work)
int tucker_plan_cut(const ntf_tensor *X, const int64_t *core_dims, const ntf_opts &o, float beta, int &a, int &b);
}  // namespace ntf
