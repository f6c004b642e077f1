// Host side of the tensor-core pass: the TMA descriptor of X and the dispatch over the
// beta class (kernels in cp3_tc.cuh, instantiated in cp3_tc_bk*.cu).
#include <mutex>

#include "cp3_tc.cuh"

namespace ntf {

cudaError_t cp3_tc_launch_bk0(const Cp3Plan &, const Cp3Args &, int, cudaStream_t);
cudaError_t cp3_tc_launch_bk1(const Cp3Plan &, const Cp3Args &, int, cudaStream_t);
cudaError_t cp3_tc_launch_bk2(const Cp3Plan &, const Cp3Args &, int, cudaStream_t);
cudaError_t cp3_tc_launch_bk3(const Cp3Plan &, const Cp3Args &, int, cudaStream_t);
cudaError_t cp3_tc_launch_bk4(const Cp3Plan &, const Cp3Args &, int, cudaStream_t);

namespace tc {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// X as a 2-D FP32 tensor [I*J rows][K columns]; boxes of 32 columns x 128 rows with the
// 128-byte swizzle that the MMA descriptors and the epilogue addressing assume.  Boxes
// past the last row or column are zero-filled by the copy engine.
cudaError_t launch_x_map(const Cp3Args &a, CUtensorMap *map) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)a.I * (cuuint64_t)a.J};
    const cuuint64_t strides[1] = {(cuuint64_t)a.K * 4};
    const cuuint32_t box[2] = {32, 128}, es[2] = {1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)a.X, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t cache_map(void *base, const Cp3Args &a, CUtensorMap *map) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)a.K, (cuuint64_t)a.J, (cuuint64_t)a.I};
    const cuuint64_t strides[2] = {(cuuint64_t)a.kp * 2, (cuuint64_t)a.kp * 2 * (cuuint64_t)a.J};
    const cuuint32_t box[3] = {64, 128, 1}, es[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

}  // namespace tc

bool cp3_tc_eligible(int RP, int K, const float *X) {
    return RP == 32 && K % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
}

bool cp3_tc_supported(int ms, int den, bool rx) {
    if (ms & PM_NOX) {
        const int m = ms & ~PM_NOX;
        return !rx && den && (m == PM_M1 || m == (PM_M1 | PM_OBJ) || m == PM_M2 || m == PM_M3);
    }
    if (rx) return ms == (PM_M1 | PM_M2) || ms == (PM_M1 | PM_M2 | PM_OBJ) || ms == PM_M3;
    switch (ms) {
        case PM_M1: case PM_M1 | PM_OBJ: case PM_M2: case PM_M3: return true;
        case PM_M1 | PM_M2 | PM_M3 | PM_OBJ: return den == 0;
        default: return false;
    }
}

cudaError_t cp3_tc_launch(const Cp3Plan &p, const Cp3Args &a, int ms, int den, cudaStream_t s) {
    if (!p.tc || p.RP != 32 || (p.KB != tc::KBLK && p.KB != 2 * tc::KBLK)) return cudaErrorInvalidValue;
    if ((a.bkind == BK_KL) != (den == 0)) return cudaErrorInvalidValue;
    switch (a.bkind) {
        case 0: return cp3_tc_launch_bk0(p, a, ms, s);
        case 1: return cp3_tc_launch_bk1(p, a, ms, s);
        case 2: return cp3_tc_launch_bk2(p, a, ms, s);
        case 3: return cp3_tc_launch_bk3(p, a, ms, s);
        case 4: return cp3_tc_launch_bk4(p, a, ms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ntf
