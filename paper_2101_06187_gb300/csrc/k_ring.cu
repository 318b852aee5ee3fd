// Launchers of the 2D ring variant (k_ring.cuh) for every storage form.
#include "k_ring.cuh"
#include "k_ring_fused2.cuh"
#include "rlbm_internal.h"

namespace rlbk {

// Two ring steps per launch: tile TW x TH of cfg.bx x cfg.by, with the
// thread count and resident CTAs per SM fixed per tile (<= 85 registers).
template <typename TS>
static cudaError_t ring_fused2_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                                 const StepParams &p, cudaStream_t s) {
    if (p.nx % 2 != 0 || p.cfl != 1.0) return cudaErrorInvalidValue;
    const TS *in = static_cast<const TS *>(qin);
    TS *out = static_cast<TS *>(qout);
    const float *f = static_cast<const float *>(F);
#define RLBM_RING_TILE(TW, TH, NT, MB)                                                                  \
    if (cfg.bx == TW && cfg.by == TH) {                                                                 \
        const dim3 grid((p.nx + TW - 1) / TW, (p.ny + TH - 1) / TH, 1);                                \
        if (forced) k_ring_fused2<TS, true, TW, TH, NT, MB><<<grid, NT, 0, s>>>(in, out, f, p);         \
        else k_ring_fused2<TS, false, TW, TH, NT, MB><<<grid, NT, 0, s>>>(in, out, f, p);               \
        return cudaGetLastError();                                                                      \
    }
    RLBM_RING_TILE(64, 16, 256, 3)
    RLBM_RING_TILE(64, 8, 128, 6)
    RLBM_RING_TILE(32, 16, 128, 6)
    RLBM_RING_TILE(128, 8, 256, 3)
#undef RLBM_RING_TILE
    return cudaErrorInvalidConfiguration;
}

template <typename TS, typename TC, typename TL>
static cudaError_t ring_step_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                               const StepParams &p, cudaStream_t s) {
    if (cfg.kernel == RLBM_KERNEL_FUSED2) {
        if constexpr (std::is_same<TC, float>::value && std::is_same<TL, float>::value)
            return ring_fused2_t<TS>(cfg, forced, qin, qout, F, p, s);
        else
            return cudaErrorInvalidValue;  // packed lanes: FP32 compute with the FP32 Landau solve
    }
    if (cfg.bx < 1 || cfg.by < 1 || cfg.bx * cfg.by > 256) return cudaErrorInvalidConfiguration;
    const dim3 block(cfg.bx, cfg.by, 1);
    if (cfg.kernel == RLBM_KERNEL_PACKED) {
        if constexpr (std::is_same<TC, float>::value && std::is_same<TL, float>::value) {
            if (p.nx % 2 != 0) return cudaErrorInvalidValue;
            const dim3 g2((p.nx / 2 + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
            const TS *in = static_cast<const TS *>(qin);
            TS *out = static_cast<TS *>(qout);
            const float *f = static_cast<const float *>(F);
            if (forced) k_ring_step_pair<TS, true><<<g2, block, 0, s>>>(in, out, f, p);
            else k_ring_step_pair<TS, false><<<g2, block, 0, s>>>(in, out, f, p);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;  // packed lanes: FP32 compute with the FP32 Landau solve
        }
    }
    const dim3 grid((p.nx + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
    const TS *in = static_cast<const TS *>(qin);
    TS *out = static_cast<TS *>(qout);
    const TC *f = static_cast<const TC *>(F);
    if (forced) k_ring_step<TS, TC, TL, true><<<grid, block, 0, s>>>(in, out, f, p);
    else k_ring_step<TS, TC, TL, false><<<grid, block, 0, s>>>(in, out, f, p);
    return cudaGetLastError();
}

cudaError_t launch_ring_step(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                             const void *F, const StepParams &p, cudaStream_t s) {
    if ((long long)NR * p.plane >= (1ll << 31)) return cudaErrorInvalidValue;
    const bool l32 = landau == RLBM_LANDAU_FP32;
    switch (dtype) {
    case RLBM_F64: return ring_step_t<double, double, double>(cfg, forced, qin, qout, F, p, s);
    case RLBM_F32:
        return l32 ? ring_step_t<float, float, float>(cfg, forced, qin, qout, F, p, s)
                   : ring_step_t<float, float, double>(cfg, forced, qin, qout, F, p, s);
    case RLBM_BF16:
        return l32 ? ring_step_t<__nv_bfloat16, float, float>(cfg, forced, qin, qout, F, p, s)
                   : ring_step_t<__nv_bfloat16, float, double>(cfg, forced, qin, qout, F, p, s);
    default:
        return l32 ? ring_step_t<__half, float, float>(cfg, forced, qin, qout, F, p, s)
                   : ring_step_t<__half, float, double>(cfg, forced, qin, qout, F, p, s);
    }
}

cudaError_t launch_ring_moments(int dtype, const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                                double *partials, int *bad, cudaStream_t s) {
    const dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
    switch (dtype) {
    case RLBM_F64:
        k_ring_moments<double, double><<<g, b, 0, s>>>(static_cast<const double *>(qin), p, eps, vx, vy, partials, bad);
        break;
    case RLBM_F32:
        k_ring_moments<float, float><<<g, b, 0, s>>>(static_cast<const float *>(qin), p, eps, vx, vy, partials, bad);
        break;
    case RLBM_BF16:
        k_ring_moments<__nv_bfloat16, float><<<g, b, 0, s>>>(static_cast<const __nv_bfloat16 *>(qin), p, eps, vx, vy,
                                                             partials, bad);
        break;
    default:
        k_ring_moments<__half, float><<<g, b, 0, s>>>(static_cast<const __half *>(qin), p, eps, vx, vy, partials, bad);
    }
    return cudaGetLastError();
}

cudaError_t launch_ring_init(int dtype, void *q, const StepParams &p, const double *eps, const double *vx,
                             const double *vy, cudaStream_t s) {
    const dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
    switch (dtype) {
    case RLBM_F64: k_ring_init<double, double><<<g, b, 0, s>>>(static_cast<double *>(q), p, eps, vx, vy); break;
    case RLBM_F32: k_ring_init<float, float><<<g, b, 0, s>>>(static_cast<float *>(q), p, eps, vx, vy); break;
    case RLBM_BF16:
        k_ring_init<__nv_bfloat16, float><<<g, b, 0, s>>>(static_cast<__nv_bfloat16 *>(q), p, eps, vx, vy);
        break;
    default: k_ring_init<__half, float><<<g, b, 0, s>>>(static_cast<__half *>(q), p, eps, vx, vy);
    }
    return cudaGetLastError();
}

}  // namespace rlbk
