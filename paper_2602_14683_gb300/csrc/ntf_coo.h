// Internal: sparse COO tensors (coo.cu).
#pragma once
#include "../../include/ntf.h"
#include "ntf_internal.h"

namespace ntf {
int coo_kl_sweep(ntf_ctx *ctx, const ntf_tensor *X, int R, float *const *factors, const ntf_opts &o,
                 double *objective_dev, cudaStream_t st, bool jcomm);
int coo_kl_objective(ntf_ctx *ctx, const ntf_tensor *X, int R, const float *const *factors, const ntf_opts &o,
                     double *out_dev, cudaStream_t st);
// Num^(n) of a COO tensor over its stored entries (Section 6.3): rows [dims[n]][RP] (RP 32 or
// 64) of sum_e p_e prod_{m != n} num[m][i_m(e)], p_e = x_e max(Xhat_e, eps)^(beta - 2) with
// Xhat from the padded factors rec, into out (may be null: objective only).  With obj_parts:
// per-unit FP64 partials of sum_e [d_beta(x_e | y_e) - d_beta(0 | y_e)] (beta != 1; the KL
// form at beta = 1), returned in *obj_parts (context workspace) with their count in *n_obj.
int coo_num_rows(ntf_ctx *ctx, const ntf_tensor *X, int n, int RP, const float *const *rec, const float *const *num,
                 float beta, float eps, float *out, double **obj_parts, int *n_obj, cudaStream_t st);
// The KL objective of a COO tensor from the stored-entry partials of coo_num_rows (parts, n_parts)
// plus the closed-form dense part sum_{r < R} prod_n colsum(F[n])_r (F: padded blocks, RP columns,
// X->dims[n] rows), into *out_dev.  The pointer table it reads lives in the context's workspace.
int coo_kl_objective_total(ntf_ctx *ctx, const ntf_tensor *X, const float *const *F, int R, int RP,
                           const double *parts, int n_parts, double *out_dev, cudaStream_t st);
int coo_stable_perm(ntf_ctx *ctx, const int32_t *keys, int64_t nnz, int64_t key_range, int32_t *perm_out,
                    cudaStream_t st);
void coo_release(ntf_ctx *ctx);
}  // namespace ntf
