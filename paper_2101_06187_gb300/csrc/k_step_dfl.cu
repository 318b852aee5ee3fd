// The packed single-step and two-steps-per-launch kernels with the Landau
// frame refined to FP64 accuracy on the FP32 lanes (landau_refine_df): the
// library's RLBM_LANDAU_FP64 solve for the FP32 and 16-bit storage forms on
// these kernels.  CFL 1, nx even; FP32, BF16 and FP16 storage.
#include "k_fused2_launch.cuh"

namespace rlbk {
namespace {

template <typename TS>
cudaError_t pair_dfl_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                       const StepParams &p, cudaStream_t s) {
    if (cfg.bx < 1 || cfg.by < 1 || cfg.bx * cfg.by > 256) return cudaErrorInvalidConfiguration;
    if (cfg.minb != 1 && cfg.minb != 2) return cudaErrorInvalidValue;  // the budgets instantiated here
    const TS *in = static_cast<const TS *>(qin);
    TS *out = static_cast<TS *>(qout);
    const float *f = static_cast<const float *>(F);
    const dim3 block(cfg.bx, cfg.by, 1);
    const dim3 grid((p.nx / 2 + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
    const bool idx32 = (long long)NC * p.plane < (1ll << 31) - 1;
#define RLBM_PAIR_DFL(MB)                                                                                     \
    do {                                                                                                      \
        if (idx32) {                                                                                          \
            if (forced) k_step_pair<TS, true, MB, int, kStreamCfl1, true><<<grid, block, 0, s>>>(in, out, f, p); \
            else k_step_pair<TS, false, MB, int, kStreamCfl1, true><<<grid, block, 0, s>>>(in, out, f, p);      \
        } else {                                                                                              \
            if (forced)                                                                                       \
                k_step_pair<TS, true, MB, long long, kStreamCfl1, true><<<grid, block, 0, s>>>(in, out, f, p);   \
            else                                                                                              \
                k_step_pair<TS, false, MB, long long, kStreamCfl1, true><<<grid, block, 0, s>>>(in, out, f, p);  \
        }                                                                                                     \
    } while (0)
    if (cfg.minb == 2) RLBM_PAIR_DFL(2);
    else RLBM_PAIR_DFL(1);
#undef RLBM_PAIR_DFL
    return cudaGetLastError();
}

// The two-step kernel with the refined frame: 64 x 8 tiles (128 threads,
// four CTAs per SM), the tile shape the FP32 solve's tuning picks.
template <typename TS>
struct Fused2Dfl {
    static constexpr int TW = 64, TH = 8, NT = 128, MINB = 4;
    static constexpr int smem = fused2_smem_bytes<TS, TW, TH>();
    template <bool FORCED, typename I>
    static void *fn() {
        return reinterpret_cast<void *>(&k_step_fused2<TS, FORCED, TW, TH, NT, MINB, I, kStreamCfl1, true>);
    }
    static cudaError_t prepare() {
        for (void *f : {fn<true, int>(), fn<false, int>(), fn<true, long long>(), fn<false, long long>()}) {
            const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    static cudaError_t launch(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                              const StepParams &p, cudaStream_t s) {
        if (cfg.bx != TW || cfg.by != TH) return cudaErrorInvalidConfiguration;
        const TS *in = static_cast<const TS *>(qin);
        TS *out = static_cast<TS *>(qout);
        const float *f = static_cast<const float *>(F);
        const dim3 grid((p.nx + TW - 1) / TW, (p.ny + TH - 1) / TH, 1);
        const bool idx32 = (long long)NC * p.plane < (1ll << 31) - 1;
        if (idx32) {
            if (forced)
                k_step_fused2<TS, true, TW, TH, NT, MINB, int, kStreamCfl1, true><<<grid, NT, smem, s>>>(in, out, f, p);
            else
                k_step_fused2<TS, false, TW, TH, NT, MINB, int, kStreamCfl1, true><<<grid, NT, smem, s>>>(in, out, f,
                                                                                                          p);
        } else {
            if (forced)
                k_step_fused2<TS, true, TW, TH, NT, MINB, long long, kStreamCfl1, true><<<grid, NT, smem, s>>>(in, out,
                                                                                                               f, p);
            else
                k_step_fused2<TS, false, TW, TH, NT, MINB, long long, kStreamCfl1, true><<<grid, NT, smem, s>>>(
                    in, out, f, p);
        }
        return cudaGetLastError();
    }
};

}  // namespace

cudaError_t launch_step_pair_dfl(int dtype, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                                 const void *F, const StepParams &p, cudaStream_t s) {
    if (p.nx % 2 != 0 || p.cfl != 1.0) return cudaErrorInvalidValue;
    switch (dtype) {
    case RLBM_F32: return pair_dfl_t<float>(cfg, forced, qin, qout, F, p, s);
    case RLBM_BF16: return pair_dfl_t<__nv_bfloat16>(cfg, forced, qin, qout, F, p, s);
    case RLBM_F16: return pair_dfl_t<__half>(cfg, forced, qin, qout, F, p, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fused2_dfl_prepare() {
    cudaError_t e = Fused2Dfl<float>::prepare();
    if (e == cudaSuccess) e = Fused2Dfl<__nv_bfloat16>::prepare();
    if (e == cudaSuccess) e = Fused2Dfl<__half>::prepare();
    return e;
}

cudaError_t launch_step_fused2_dfl(int dtype, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                                   const void *F, const StepParams &p, cudaStream_t s) {
    if (p.nx % 2 != 0 || p.cfl != 1.0) return cudaErrorInvalidValue;
    switch (dtype) {
    case RLBM_F32: return Fused2Dfl<float>::launch(cfg, forced, qin, qout, F, p, s);
    case RLBM_BF16: return Fused2Dfl<__nv_bfloat16>::launch(cfg, forced, qin, qout, F, p, s);
    case RLBM_F16: return Fused2Dfl<__half>::launch(cfg, forced, qin, qout, F, p, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rlbk
