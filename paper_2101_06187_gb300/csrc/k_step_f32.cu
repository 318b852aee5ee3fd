// FP32 form: FP32 storage and arithmetic; Landau solve in FP64 or FP32.
#include "k_launch.cuh"

namespace rlbk {
cudaError_t launch_step_f32(const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout, const void *F,
                            const StepParams &p, cudaStream_t s) {
    if (landau == RLBM_LANDAU_FP32) return launch_step_t<float, float, float>(cfg, forced, qin, qout, F, p, s);
    return launch_step_t<float, float, double>(cfg, forced, qin, qout, F, p, s);
}
cudaError_t launch_moments_f32(int landau, const void *qin, const StepParams &p, double *eps, double *vx,
                               double *vy, double *partials, int *bad, cudaStream_t s) {
    (void)landau;  // diagnostics always solve the frame to FP64 accuracy (refined FP32 frame)
    return launch_moments_t<float, float, float>(qin, p, eps, vx, vy, partials, bad, s);
}
cudaError_t launch_batch_f32(const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns, int ntiles,
                             cudaStream_t s) {
    if (landau == RLBM_LANDAU_FP32) return launch_batch_t<float, float, float>(cfg, grid, runs, nruns, ntiles, s);
    return launch_batch_t<float, float, double>(cfg, grid, runs, nruns, ntiles, s);
}
}  // namespace rlbk
