// Tensor-core pass instantiations for one beta class (compiled in parallel).
#include "cp3_tc.cuh"

namespace ntf {
cudaError_t cp3_tc_launch_bk4(const Cp3Plan &p, const Cp3Args &a, int ms, cudaStream_t s) {
    return p.s3 ? tc::launch_bk<4, true>(p, a, ms, s) : tc::launch_bk<4, false>(p, a, ms, s);
}
}  // namespace ntf
