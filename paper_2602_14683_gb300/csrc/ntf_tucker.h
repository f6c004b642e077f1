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

// Strided batched GEMM with a two-level reduction index, the small contractions of the Tucker
// updates (Appendix C):
//   C[bt][m][n] = sum_{k1 < K1, k2 < K2} A(bt, m, k1, k2) * B(bt, k1, k2, n),
//   A(bt, m, k1, k2) = A[bt sab + m sam + k1 sak1 + k2 sak2], B(bt, k1, k2, n) = B[bt sbb + k1 sbk1 +
//   k2 sbk2 + n sbn], C at bt scb + m scm + n scn.
// The reduction index k = k1 K2 + k2 may be cut into `splits` contiguous ranges of `kchunks`
// chunks each; every range's sum then goes to `part` and the ranges are added in order (FP64 for
// the CUDA-core form, FP32 for the tensor-core one).
struct Gemm {
    const float *A, *B;
    float *C;
    int M, N, K1, K2, batch;
    int64_t sab, sam, sak1, sak2;
    int64_t sbb, sbk1, sbk2, sbn;
    int64_t scb, scm, scn;
    int splits, kchunks;  // reduction ranges and chunks per range (set by the launcher)
    float *part;          // [splits][batch][M][N] when splits > 1
    int *err;             // tensor-core form: status word set when a bounded wait gives up
    int nin;              // > 0: the batch is folded into n (A shared by all batches, sab = 0): N counts
                          // batch x nin columns, column b nin + n stands for (batch b, column n), and
                          // batch is 1; B and C then step by sbb / scb from one batch block to the next
    int mfold;            // > 0 (tensor-core form only, 32-column tiles, scm = 1, nin = 0): row m of A and C
    int64_t samb, scmb;   // is (m / mfold) samb + (m % mfold) sam and (m / mfold) scmb + (m % mfold) scm (a
                          // second index folded into the rows); the range partials are then [splits][n][m]
};
// Tensor-core form of the same product (tucker_gemm_tc.cu): tcgen05 kind::tf32 MMAs on operands
// rounded to TF32 (s3: split into high and low TF32 parts, three products, about FP32 accuracy),
// FP32 accumulation in tensor memory; tiles of 128 rows m x ntt columns n (ntt in 32, 64, 128,
// 256), chunks of 32 reduction indices (g.kchunks counts those), grid (n tiles, m tiles,
// batch x splits).  Writes C, or g.part when g.splits > 1.  Returns a cudaError_t.
cudaError_t gemm_tc_launch(const Gemm &g, bool s3, int ntt, cudaStream_t s);

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
