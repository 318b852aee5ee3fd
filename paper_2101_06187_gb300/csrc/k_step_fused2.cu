// Two-steps-per-launch (temporally blocked) form of the packed step:
// CFL-1 and ensemble instantiations, and the launchers.  FP32 arithmetic
// with the FP32 Landau solve, FP32 / BF16 / FP16 storage, cfl <= 1, nx even.
#include "k_fused2_launch.cuh"

namespace rlbk {
namespace {

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
cudaError_t launch_batch_t(const LaunchCfg &cfg, int grid, const void *runs, int nruns, int ntiles, int two,
                           cudaStream_t s) {
#define X(TW, TH, NT, MB)                                                                       \
    if (cfg.bx == TW && cfg.by == TH)                                                           \
        return Fused2Batch<TS, TW, TH, NT, MB>::launch(grid, runs, nruns, ntiles, two, s);
    RLBM_FUSED2_SHAPES(X)
#undef X
    return cudaErrorInvalidConfiguration;
}

}  // namespace

cudaError_t fused2_prepare() {
    cudaError_t e = fused2_prepare_mode<kStreamCfl1>();
    if (e == cudaSuccess) e = fused2_prepare_sub1();
    if (e == cudaSuccess) e = batch_prepare_t<float>();
    if (e == cudaSuccess) e = batch_prepare_t<__nv_bfloat16>();
    if (e == cudaSuccess) e = batch_prepare_t<__half>();
    return e;
}

cudaError_t launch_step_fused2(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                               const void *F, const StepParams &p, cudaStream_t s) {
    if (landau != RLBM_LANDAU_FP32 || p.nx % 2 != 0 || !(p.cfl > 0.0 && p.cfl <= 1.0)) return cudaErrorInvalidValue;
    if (p.cfl == 1.0) return fused2_launch_mode<kStreamCfl1>(dtype, cfg, forced, qin, qout, F, p, s);
    return fused2_launch_sub1(dtype, cfg, forced, qin, qout, F, p, s);
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
