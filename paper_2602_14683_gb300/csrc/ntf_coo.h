// Internal: sparse COO tensors under KL (coo.cu).
#pragma once
#include "../../include/ntf.h"
#include "ntf_internal.h"

namespace ntf {
int coo_kl_sweep(ntf_ctx *ctx, const ntf_tensor *X, int R, float *const *factors, const ntf_opts &o,
                 double *objective_dev, cudaStream_t st, bool jcomm);
int coo_kl_objective(ntf_ctx *ctx, const ntf_tensor *X, int R, const float *const *factors, const ntf_opts &o,
                     double *out_dev, cudaStream_t st);
int coo_stable_perm(ntf_ctx *ctx, const int32_t *keys, int64_t nnz, int64_t key_range, int32_t *perm_out,
                    cudaStream_t st);
void coo_release(ntf_ctx *ctx);
}  // namespace ntf
