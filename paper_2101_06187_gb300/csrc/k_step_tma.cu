// Launcher and tensor maps of the TMA-pipelined fused step (k_step_tma.cuh).
#include <cudaTypedefs.h>

#include <mutex>

#include "k_step_tma.cuh"
#include "rlbm_internal.h"

namespace rlbk {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 3D map over an FP32 array [planes][ny][pitch]: x (nx elements, unit
// stride), y (ny rows, pitch elements apart), plane (plane elements apart);
// out-of-range cells read as zero.
static cudaError_t encode_planes(CUtensorMap *map, const void *base, const StepParams &p, int planes, int box_x,
                                 int box_y, int box_planes) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)p.pitch * 4, (cuuint64_t)p.plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tma_encode_state(CUtensorMap *map, const void *q, const StepParams &p) {
    return encode_planes(map, q, p, NC, kTmaSW, kTmaSH, NC);
}

cudaError_t tma_encode_force(CUtensorMap *map, const void *F, const StepParams &p) {
    return encode_planes(map, F, p, 2, kTmaTW, kTmaTH, 2);
}

static int sm_count_of_current_device() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return 0;
    return n;
}

template <bool FORCED>
static cudaError_t launch_tma_t(int ctas_per_sm, const CUtensorMap &mq, const CUtensorMap &mf, const float *qin,
                                float *qout, const StepParams &p, cudaStream_t s, int unarmed) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(k_step_tma<FORCED>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmemBytes);
    });
    if (attr != cudaSuccess) return attr;
    const int sms = sm_count_of_current_device();
    if (sms <= 0) return cudaErrorInvalidDevice;
    const int tiles = ((p.nx + kTmaTW - 1) / kTmaTW) * ((p.ny + kTmaTH - 1) / kTmaTH);
    const int grid = std::max(1, std::min(tiles, ctas_per_sm * sms));
    k_step_tma<FORCED><<<grid, dim3(kTmaTW / 2, kTmaTH, 1), kTmaSmemBytes, s>>>(mq, mf, qin, qout, p, unarmed);
    return cudaGetLastError();
}

cudaError_t launch_step_tma(const LaunchCfg &cfg, bool forced, const CUtensorMap &mq, const CUtensorMap &mf,
                            const void *qin, void *qout, const StepParams &p, cudaStream_t s, int unarmed) {
    if (p.nx % 2 != 0 || p.cfl != 1.0 || p.eta_k != 0.0) return cudaErrorInvalidValue;
    const int per_sm = cfg.minb == 1 ? 1 : 2;
    const float *in = static_cast<const float *>(qin);
    float *out = static_cast<float *>(qout);
    return forced ? launch_tma_t<true>(per_sm, mq, mf, in, out, p, s, unarmed)
                  : launch_tma_t<false>(per_sm, mq, mf, in, out, p, s, unarmed);
}

}  // namespace rlbk
