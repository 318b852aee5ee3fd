// k_fused2_launch.cuh -- host-side launch templates of the two-steps-per-
// launch kernels (k_step_fused2.cuh), shared by the translation units that
// instantiate them for each streaming mode.
#pragma once

#include "k_step_fused2.cuh"
#include "rlbm_internal.h"

namespace rlbk {

// Tile shape: output tile TW x TH, NT threads, MINB resident CTAs per SM
// (shared memory per CTA: 17 (TW + 4)(TH + 2) stored values); SM is the
// streaming mode of the single-lattice kernels.
template <typename TS, int TW, int TH, int NT, int MINB, int SM>
struct Fused2 {
    static constexpr int smem = fused2_smem_bytes<TS, TW, TH>();

    template <bool FORCED, typename I>
    static void *fn() {
        return reinterpret_cast<void *>(&k_step_fused2<TS, FORCED, TW, TH, NT, MINB, I, SM>);
    }
    static cudaError_t set_smem(void *f) {
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    static cudaError_t prepare() {
        for (void *f : {fn<true, int>(), fn<false, int>(), fn<true, long long>(), fn<false, long long>()}) {
            const cudaError_t e = set_smem(f);
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
            if (forced) k_step_fused2<TS, true, TW, TH, NT, MINB, int, SM><<<grid, NT, smem, s>>>(in, out, f, p);
            else k_step_fused2<TS, false, TW, TH, NT, MINB, int, SM><<<grid, NT, smem, s>>>(in, out, f, p);
        } else {
            if (forced) k_step_fused2<TS, true, TW, TH, NT, MINB, long long, SM><<<grid, NT, smem, s>>>(in, out, f, p);
            else k_step_fused2<TS, false, TW, TH, NT, MINB, long long, SM><<<grid, NT, smem, s>>>(in, out, f, p);
        }
        return cudaGetLastError();
    }
};

// The tile shapes on offer, by (bx, by) = (TW, TH) of the launch shape.
#define RLBM_FUSED2_SHAPES(X) \
    X(64, 16, 256, 2)         \
    X(64, 8, 128, 4)          \
    X(32, 16, 128, 4)         \
    X(128, 8, 256, 2)

template <typename TS, int SM>
cudaError_t fused2_prepare_t() {
#define X(TW, TH, NT, MB)                                                  \
    {                                                                      \
        const cudaError_t e = Fused2<TS, TW, TH, NT, MB, SM>::prepare();   \
        if (e != cudaSuccess) return e;                                    \
    }
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaSuccess;
}

template <typename TS, int SM>
cudaError_t fused2_launch_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                            const StepParams &p, cudaStream_t s) {
#define X(TW, TH, NT, MB) \
    if (cfg.bx == TW && cfg.by == TH) return Fused2<TS, TW, TH, NT, MB, SM>::launch(forced, qin, qout, F, p, s);
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

// Every storage form in streaming mode SM: prepare, and launch by dtype.
template <int SM>
cudaError_t fused2_prepare_mode() {
    cudaError_t e = fused2_prepare_t<float, SM>();
    if (e == cudaSuccess) e = fused2_prepare_t<__nv_bfloat16, SM>();
    if (e == cudaSuccess) e = fused2_prepare_t<__half, SM>();
    return e;
}

template <int SM>
cudaError_t fused2_launch_mode(int dtype, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                               const void *F, const StepParams &p, cudaStream_t s) {
    switch (dtype) {
    case RLBM_F32: return fused2_launch_t<float, SM>(cfg, forced, qin, qout, F, p, s);
    case RLBM_BF16: return fused2_launch_t<__nv_bfloat16, SM>(cfg, forced, qin, qout, F, p, s);
    case RLBM_F16: return fused2_launch_t<__half, SM>(cfg, forced, qin, qout, F, p, s);
    default: return cudaErrorInvalidValue;
    }
}

// The cfl < 1 instantiations (k_step_fused2_sub.cu).
cudaError_t fused2_prepare_sub1();
cudaError_t fused2_launch_sub1(int dtype, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                               const void *F, const StepParams &p, cudaStream_t s);

}  // namespace rlbk
