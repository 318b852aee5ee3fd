// FP64 form: FP64 storage, FP64 arithmetic, FP64 Landau solve.
#include "k_launch.cuh"

namespace rlbk {
cudaError_t launch_step_f64(const LaunchCfg &cfg, int, bool forced, const void *qin, void *qout, const void *F,
                            const StepParams &p, cudaStream_t s) {
    return launch_step_t<double, double, double>(cfg, forced, qin, qout, F, p, s);
}
cudaError_t launch_moments_f64(int, const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                               double *partials, int *bad, cudaStream_t s) {
    return launch_moments_t<double, double, double>(qin, p, eps, vx, vy, partials, bad, s);
}
cudaError_t launch_batch_f64(const LaunchCfg &cfg, int, int grid, const void *runs, int nruns, int ntiles,
                             cudaStream_t s) {
    return launch_batch_t<double, double, double>(cfg, grid, runs, nruns, ntiles, s);
}
}  // namespace rlbk
