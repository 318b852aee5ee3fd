// 16-bit forms: BF16 or FP16 storage of the scaled deviation, FP32
// arithmetic; Landau solve in FP64 or FP32.
#include "k_launch.cuh"

namespace rlbk {
cudaError_t launch_step_h16(int dtype, const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout,
                            const void *F, const StepParams &p, cudaStream_t s) {
    if (dtype == RLBM_BF16) {
        if (landau == RLBM_LANDAU_FP32)
            return launch_step_t<__nv_bfloat16, float, float>(cfg, forced, qin, qout, F, p, s);
        return launch_step_t<__nv_bfloat16, float, double>(cfg, forced, qin, qout, F, p, s);
    }
    if (landau == RLBM_LANDAU_FP32) return launch_step_t<__half, float, float>(cfg, forced, qin, qout, F, p, s);
    return launch_step_t<__half, float, double>(cfg, forced, qin, qout, F, p, s);
}
cudaError_t launch_moments_h16(int dtype, int landau, const void *qin, const StepParams &p, double *eps, double *vx,
                               double *vy, double *partials, int *bad, cudaStream_t s) {
    (void)landau;  // diagnostics always solve the frame to FP64 accuracy (refined FP32 frame)
    if (dtype == RLBM_BF16)
        return launch_moments_t<__nv_bfloat16, float, float>(qin, p, eps, vx, vy, partials, bad, s);
    return launch_moments_t<__half, float, float>(qin, p, eps, vx, vy, partials, bad, s);
}
cudaError_t launch_batch_h16(int dtype, const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns,
                             int ntiles, cudaStream_t s) {
    if (dtype == RLBM_BF16) {
        if (landau == RLBM_LANDAU_FP32)
            return launch_batch_t<__nv_bfloat16, float, float>(cfg, grid, runs, nruns, ntiles, s);
        return launch_batch_t<__nv_bfloat16, float, double>(cfg, grid, runs, nruns, ntiles, s);
    }
    if (landau == RLBM_LANDAU_FP32) return launch_batch_t<__half, float, float>(cfg, grid, runs, nruns, ntiles, s);
    return launch_batch_t<__half, float, double>(cfg, grid, runs, nruns, ntiles, s);
}
}  // namespace rlbk
