#include "ntf_internal.h"
namespace ntf {
bool cp3_tc_supported(int, int, int) { return false; }
cudaError_t cp3_tc_launch(const Cp3Plan &, const Cp3Args &, int, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace ntf
