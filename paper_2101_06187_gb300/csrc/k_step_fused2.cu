// Two-steps-per-launch (temporally blocked) form of the packed step:
// instantiations and launcher.  FP32 arithmetic with the FP32 Landau
// solve, FP32 / BF16 / FP16 storage, CFL 1, nx even.
#include "k_step_fused2.cuh"
#include "rlbm_internal.h"

namespace rlbk {
namespace {

// Tile shapes: output tile TW x TH, NT threads, MINB resident CTAs per SM
// (shared memory per CTA: 17 (TW + 4)(TH + 2) stored values).
template <typename TS, int TW, int TH, int NT, int MINB>
struct Fused2 {
    static constexpr int smem = fused2_smem_bytes<TS, TW, TH>();

    template <bool FORCED, typename I>
    static void *fn() {
        return reinterpret_cast<void *>(&k_step_fused2<TS, FORCED, TW, TH, NT, MINB, I>);
    }
    static cudaError_t prepare() {
        for (void *f : {fn<true, int>(), fn<false, int>(), fn<true, long long>(), fn<false, long long>(),
                        reinterpret_cast<void *>(&k_step_batch_fused2<TS, TW, TH, NT, MINB, true>),
                        reinterpret_cast<void *>(&k_step_batch_fused2<TS, TW, TH, NT, MINB, false>)}) {
            const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    static cudaError_t launch(bool forced, const void *qin, void *qout, const void *F, const StepParams &p,
                              cudaStream_t s) {
        const TS *in = static_cast<const TS *>(qin);
        TS *out = static_cast<TS *>(qout);
        const float *f = static_cast<const float *>(F);
        const dim3 grid((p.nx + TW - 1) / TW, (p.ny + TH - 1) / TH, 1);
        const bool idx32 = (long long)NC * p.plane < (1ll << 31) - 1;
        if (idx32) {
            if (forced) k_step_fused2<TS, true, TW, TH, NT, MINB, int><<<grid, NT, smem, s>>>(in, out, f, p);
            else k_step_fused2<TS, false, TW, TH, NT, MINB, int><<<grid, NT, smem, s>>>(in, out, f, p);
        } else {
            if (forced) k_step_fused2<TS, true, TW, TH, NT, MINB, long long><<<grid, NT, smem, s>>>(in, out, f, p);
            else k_step_fused2<TS, false, TW, TH, NT, MINB, long long><<<grid, NT, smem, s>>>(in, out, f, p);
        }
        return cudaGetLastError();
    }
    static cudaError_t launch_batch(int grid, const void *runs, int nruns, int ntiles, int two, cudaStream_t s) {
        const BatchRun *r = static_cast<const BatchRun *>(runs);
        if (two) k_step_batch_fused2<TS, TW, TH, NT, MINB, true><<<grid, NT, smem, s>>>(r, nruns, ntiles);
        else k_step_batch_fused2<TS, TW, TH, NT, MINB, false><<<grid, NT, smem, s>>>(r, nruns, ntiles);
        return cudaGetLastError();
    }
};

// The tile shapes on offer, by (bx, by) = (TW, TH) of the launch shape.
#define RLBM_FUSED2_SHAPES(X) \
    X(64, 16, 256, 2)         \
    X(64, 8, 128, 4)          \
    X(32, 16, 128, 4)         \
    X(128, 8, 256, 2)

template <typename TS>
cudaError_t prepare_t() {
#define X(TW, TH, NT, MB)                                              \
    {                                                                  \
        const cudaError_t e = Fused2<TS, TW, TH, NT, MB>::prepare();   \
        if (e != cudaSuccess) return e;                                \
    }
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaSuccess;
}

template <typename TS>
cudaError_t launch_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                     const StepParams &p, cudaStream_t s) {
#define X(TW, TH, NT, MB) \
    if (cfg.bx == TW && cfg.by == TH) return Fused2<TS, TW, TH, NT, MB>::launch(forced, qin, qout, F, p, s);
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

template <typename TS>
cudaError_t launch_batch_t(const LaunchCfg &cfg, int grid, const void *runs, int nruns, int ntiles, int two,
                           cudaStream_t s) {
#define X(TW, TH, NT, MB)                                                                       \
    if (cfg.bx == TW && cfg.by == TH)                                                           \
        return Fused2<TS, TW, TH, NT, MB>::launch_batch(grid, runs, nruns, ntiles, two, s);
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

}  // namespace

cudaError_t fused2_prepare() {
    cudaError_t e = prepare_t<float>();
    if (e == cudaSuccess) e = prepare_t<__nv_bfloat16>();
    if (e == cudaSuccess) e = prepare_t<__half>();
    return e;
}

cudaError_t launch_step_fused2(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                               const void *F, const StepParams &p, cudaStream_t s) {
    if (landau != RLBM_LANDAU_FP32 || p.cfl != 1.0 || p.nx % 2 != 0) return cudaErrorInvalidValue;
    switch (dtype) {
    case RLBM_F32: return launch_t<float>(cfg, forced, qin, qout, F, p, s);
    case RLBM_BF16: return launch_t<__nv_bfloat16>(cfg, forced, qin, qout, F, p, s);
    case RLBM_F16: return launch_t<__half>(cfg, forced, qin, qout, F, p, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_fused2(int dtype, int landau, const LaunchCfg &cfg, int grid, const void *runs, int nruns,
                                int ntiles, int two, cudaStream_t s) {
    if (landau != RLBM_LANDAU_FP32 || grid < 1) return cudaErrorInvalidValue;
    switch (dtype) {
    case RLBM_F32: return launch_batch_t<float>(cfg, grid, runs, nruns, ntiles, two, s);
    case RLBM_BF16: return launch_batch_t<__nv_bfloat16>(cfg, grid, runs, nruns, ntiles, two, s);
    case RLBM_F16: return launch_batch_t<__half>(cfg, grid, runs, nruns, ntiles, two, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rlbk
