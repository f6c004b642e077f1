#include "ntf_coo.h"
#include "ntf_tucker.h"
namespace ntf {
int coo_kl_sweep(ntf_ctx *ctx, const ntf_tensor *, int, float *const *, const ntf_opts &, double *, cudaStream_t,
                 bool) {
    return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "COO not built yet");
}
int coo_kl_objective(ntf_ctx *ctx, const ntf_tensor *, int, const float *const *, const ntf_opts &, double *,
                     cudaStream_t) {
    return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "COO not built yet");
}
int coo_stable_perm(ntf_ctx *ctx, const int32_t *, int64_t, int64_t, int32_t *, cudaStream_t) {
    return ctx_fail(ctx, NTF_ERR_UNSUPPORTED, "COO not built yet");
}
void coo_release(ntf_ctx *) {}
}  // namespace ntf
