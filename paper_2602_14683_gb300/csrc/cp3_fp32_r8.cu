// Instantiations of the fused FP32 CP pass for rank padding RP = 8 (compiled in its own
// translation unit so the library builds in parallel).
#include "cp3_fp32.cuh"

namespace ntf {
cudaError_t cp3_launch_fp32_r8(const Cp3Plan &p, const Cp3Args &a, int ms, int den, cudaStream_t s) {
    return fp32::launch_rp<8>(p, a, ms, den, s);
}
cudaError_t cp3_batched_fp32_r8(const BatchTable<Cp3Args> &t, int ms, int den, int grid, cudaStream_t s) {
    return fp32::launch_batched_rp<8>(t, ms, den, grid, s);
}
}  // namespace ntf
