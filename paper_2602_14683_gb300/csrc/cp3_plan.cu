// Work decomposition of the fused dense CP pass and the precision dispatch.
#include "ntf_internal.h"

namespace ntf {

cudaError_t cp3_launch_fp32_r8(const Cp3Plan &, const Cp3Args &, int, int, cudaStream_t);
cudaError_t cp3_launch_fp32_r16(const Cp3Plan &, const Cp3Args &, int, int, cudaStream_t);
cudaError_t cp3_launch_fp32_r32(const Cp3Plan &, const Cp3Args &, int, int, cudaStream_t);
cudaError_t cp3_launch_fp32_r64(const Cp3Plan &, const Cp3Args &, int, int, cudaStream_t);
cudaError_t cp3_batched_fp32_r8(const BatchTable<Cp3Args> &, int, int, int, cudaStream_t);
cudaError_t cp3_batched_fp32_r16(const BatchTable<Cp3Args> &, int, int, int, cudaStream_t);
cudaError_t cp3_batched_fp32_r32(const BatchTable<Cp3Args> &, int, int, int, cudaStream_t);
cudaError_t cp3_batched_fp32_r64(const BatchTable<Cp3Args> &, int, int, int, cudaStream_t);

// Row tiles of TJ rows (128 on the tensor cores, 64 on the FP32 pass), column blocks of KB columns, and the slab
// axis split so that the grid quantises well onto the SMs (one resident CTA per SM):
// the split minimises waves * (ceil(I / n_is) + c0), where c0 = 4 slab-equivalents is
// the per-CTA cost of staging factor blocks and writing partial sums; ties go to fewer
// CTAs.
Cp3Plan cp3_plan(int I, int J, int K, int RP, int num_sms, int kb, int force_is) {
    Cp3Plan p{};
    p.tc = kb >= 128;
    p.RP = RP;
    p.TJ = p.tc ? 128 : 64;
    p.KB = kb;
    p.n_jt = (J + p.TJ - 1) / p.TJ;
    p.n_kb = (K + p.KB - 1) / p.KB;
    const int base = p.n_jt * p.n_kb;
    int best = 1;
    int64_t best_cost = -1;
    const int lim = I < 4096 ? I : 4096;
    for (int n = 1; n <= lim; ++n) {
        int64_t grid = (int64_t)base * n;
        int64_t waves = (grid + num_sms - 1) / num_sms;
        int64_t per = (I + n - 1) / n;
        int64_t cost = waves * (per + 4);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = n;
        }
    }
    if (force_is > 0) best = force_is < I ? force_is : I;
    p.n_is = best;
    p.grid = base * best;
    p.parts1 = p.n_jt * p.n_kb * (p.tc ? 4 : 1);  // tensor-core pass: one per 32-row quarter
    p.parts2 = p.n_kb * p.n_is;
    p.parts3 = p.n_jt * p.n_is;
    return p;
}

cudaError_t cp3_launch(const Cp3Plan &p, const Cp3Args &a, int ms, int den, cudaStream_t s) {
    switch (p.RP) {
        case 8: return cp3_launch_fp32_r8(p, a, ms, den, s);
        case 16: return cp3_launch_fp32_r16(p, a, ms, den, s);
        case 32: return cp3_launch_fp32_r32(p, a, ms, den, s);
        case 64: return cp3_launch_fp32_r64(p, a, ms, den, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t cp3_batched_launch(int RP, const BatchTable<Cp3Args> &t, int ms, int den, int grid, cudaStream_t s) {
    switch (RP) {
        case 8: return cp3_batched_fp32_r8(t, ms, den, grid, s);
        case 16: return cp3_batched_fp32_r16(t, ms, den, grid, s);
        case 32: return cp3_batched_fp32_r32(t, ms, den, grid, s);
        case 64: return cp3_batched_fp32_r64(t, ms, den, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntf
