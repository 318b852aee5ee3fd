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

// The ensemble kernels of tile shape TW x TH (CFL 1).
template <typename TS, int TW, int TH, int NT, int MINB>
struct Fused2Batch {
    static constexpr int smem = fused2_smem_bytes<TS, TW, TH>();
    static cudaError_t prepare() {
        for (void *f : {reinterpret_cast<void *>(&k_step_batch_fused2<TS, TW, TH, NT, MINB, true>),
                        reinterpret_cast<void *>(&k_step_batch_fused2<TS, TW, TH, NT, MINB, false>)}) {
            const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    static cudaError_t launch(int grid, const void *runs, int nruns, int ntiles, int two, cudaStream_t s) {
        const BatchRun *r = static_cast<const BatchRun *>(runs);
        if (two) k_step_batch_fused2<TS, TW, TH, NT, MINB, true><<<grid, NT, smem, s>>>(r, nruns, ntiles);
        else k_step_batch_fused2<TS, TW, TH, NT, MINB, false><<<grid, NT, smem, s>>>(r, nruns, ntiles);
        return cudaGetLastError();
    }
};

template <typename TS>
cudaError_t batch_prepare_t() {
#define X(TW, TH, NT, MB)                                                  \
    {                                                                      \
        const cudaError_t e = Fused2Batch<TS, TW, TH, NT, MB>::prepare();  \
        if (e != cudaSuccess) return e;                                    \
    }
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaSuccess;
}

template <typename TS>
cudaError_t batch_launch_t(const LaunchCfg &cfg, int grid, const void *runs, int nruns, int ntiles, int two,
                           cudaStream_t s) {
#define X(TW, TH, NT, MB)                                                                       \
    if (cfg.bx == TW && cfg.by == TH)                                                           \
        return Fused2Batch<TS, TW, TH, NT, MB>::launch(grid, runs, nruns, ntiles, two, s);
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

// Per storage type and streaming mode, one translation unit each
// (k_fused2_inst.cuh), so the many kernel instantiations compile in
// parallel: the single-lattice kernels at CFL 1 with the ensemble kernels,
// and the single-lattice kernels at 0 < cfl < 1.
#define RLBM_FUSED2_TYPE_ENTRIES(SFX)                                                                          \
    cudaError_t fused2_prepare_cfl1_##SFX();                                                                   \
    cudaError_t fused2_launch_cfl1_##SFX(const LaunchCfg &cfg, bool forced, const void *qin, void *qout,        \
                                         const void *F, const StepParams &p, cudaStream_t s);                  \
    cudaError_t fused2_launch_batch_##SFX(const LaunchCfg &cfg, int grid, const void *runs, int nruns,         \
                                          int ntiles, int two, cudaStream_t s);                                \
    cudaError_t fused2_prepare_sub1_##SFX();                                                                   \
    cudaError_t fused2_launch_sub1_##SFX(const LaunchCfg &cfg, bool forced, const void *qin, void *qout,        \
                                         const void *F, const StepParams &p, cudaStream_t s);
RLBM_FUSED2_TYPE_ENTRIES(f32)
RLBM_FUSED2_TYPE_ENTRIES(bf16)
RLBM_FUSED2_TYPE_ENTRIES(f16)
#undef RLBM_FUSED2_TYPE_ENTRIES

}  // namespace rlbk
