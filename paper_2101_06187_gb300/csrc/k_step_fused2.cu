// Two-steps-per-launch (temporally blocked) form of the packed step: the
// launchers, dispatching by storage type and streaming mode to the
// per-type translation units (k_fused2_*.cu).  FP32 arithmetic with the
// FP32 Landau solve, FP32 / BF16 / FP16 storage, cfl <= 1, nx even.
#include "k_fused2_launch.cuh"

namespace rlbk {

cudaError_t fused2_prepare() {
    cudaError_t (*const prep[])() = {fused2_prepare_cfl1_f32, fused2_prepare_cfl1_bf16, fused2_prepare_cfl1_f16,
                                     fused2_prepare_sub1_f32, fused2_prepare_sub1_bf16, fused2_prepare_sub1_f16};
    for (auto f : prep) {
        const cudaError_t e = f();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_step_fused2(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                               const void *F, const StepParams &p, cudaStream_t s) {
    if (landau != RLBM_LANDAU_FP32 || p.nx % 2 != 0 || !(p.cfl > 0.0 && p.cfl <= 1.0)) return cudaErrorInvalidValue;
    const bool cfl1 = p.cfl == 1.0;
    switch (dtype) {
    case RLBM_F32:
        return cfl1 ? fused2_launch_cfl1_f32(cfg, forced, qin, qout, F, p, s)
                    : fused2_launch_sub1_f32(cfg, forced, qin, qout, F, p, s);
    case RLBM_BF16:
        return cfl1 ? fused2_launch_cfl1_bf16(cfg, forced, qin, qout, F, p, s)
                    : fused2_launch_sub1_bf16(cfg, forced, qin, qout, F, p, s);
    case RLBM_F16:
        return cfl1 ? fused2_launch_cfl1_f16(cfg, forced, qin, qout, F, p, s)
                    : fused2_launch_sub1_f16(cfg, forced, qin, qout, F, p, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_fused2(int dtype, int landau, const LaunchCfg &cfg, int grid, const void *runs, int nruns,
                                int ntiles, int two, cudaStream_t s) {
    if (landau != RLBM_LANDAU_FP32 || grid < 1) return cudaErrorInvalidValue;
    switch (dtype) {
    case RLBM_F32: return fused2_launch_batch_f32(cfg, grid, runs, nruns, ntiles, two, s);
    case RLBM_BF16: return fused2_launch_batch_bf16(cfg, grid, runs, nruns, ntiles, two, s);
    case RLBM_F16: return fused2_launch_batch_f16(cfg, grid, runs, nruns, ntiles, two, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rlbk
