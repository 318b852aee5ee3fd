// BF16 storage of the scaled deviation, FP32 arithmetic; Landau solve in FP32
// or FP64-accurate: the single-step, moments and ensemble kernels.
#include "k_launch.cuh"

namespace rlbk {
cudaError_t launch_step_bf16(const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout, const void *F,
                           const StepParams &p, cudaStream_t s) {
    if (landau == RLBM_LANDAU_FP32) return launch_step_t<__nv_bfloat16, float, float>(cfg, forced, qin, qout, F, p, s);
    return launch_step_t<__nv_bfloat16, float, double>(cfg, forced, qin, qout, F, p, s);
}
cudaError_t launch_moments_bf16(const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                              double *partials, int *bad, cudaStream_t s) {
    // diagnostics always solve the frame to FP64 accuracy (the refined FP32 frame)
    return launch_moments_t<__nv_bfloat16, float, float>(qin, p, eps, vx, vy, partials, bad, s);
}
cudaError_t launch_batch_bf16(const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns, int ntiles,
                            cudaStream_t s) {
    if (landau == RLBM_LANDAU_FP32) return launch_batch_t<__nv_bfloat16, float, float>(cfg, grid, runs, nruns, ntiles, s);
    return launch_batch_t<__nv_bfloat16, float, double>(cfg, grid, runs, nruns, ntiles, s);
}
}  // namespace rlbk
