// 16-bit forms: BF16 or FP16 storage of the scaled deviation, FP32
// arithmetic; dispatch to the per-type translation units (k_step_bf16.cu,
// k_step_f16.cu), which compile in parallel.
#include "rlbm_internal.h"

namespace rlbk {
cudaError_t launch_step_bf16(const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout,
                             const void *F, const StepParams &p, cudaStream_t s);
cudaError_t launch_step_f16(const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout, const void *F,
                            const StepParams &p, cudaStream_t s);
cudaError_t launch_moments_bf16(const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                                double *partials, int *bad, cudaStream_t s);
cudaError_t launch_moments_f16(const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                               double *partials, int *bad, cudaStream_t s);
cudaError_t launch_batch_bf16(const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns, int ntiles,
                              cudaStream_t s);
cudaError_t launch_batch_f16(const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns, int ntiles,
                             cudaStream_t s);

cudaError_t launch_step_h16(int dtype, const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout,
                            const void *F, const StepParams &p, cudaStream_t s) {
    if (dtype == RLBM_BF16) return launch_step_bf16(cfg, landau, forced, qin, qout, F, p, s);
    return launch_step_f16(cfg, landau, forced, qin, qout, F, p, s);
}
cudaError_t launch_moments_h16(int dtype, int landau, const void *qin, const StepParams &p, double *eps, double *vx,
                               double *vy, double *partials, int *bad, cudaStream_t s) {
    (void)landau;
    if (dtype == RLBM_BF16) return launch_moments_bf16(qin, p, eps, vx, vy, partials, bad, s);
    return launch_moments_f16(qin, p, eps, vx, vy, partials, bad, s);
}
cudaError_t launch_batch_h16(int dtype, const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns,
                             int ntiles, cudaStream_t s) {
    if (dtype == RLBM_BF16) return launch_batch_bf16(cfg, landau, grid, runs, nruns, ntiles, s);
    return launch_batch_f16(cfg, landau, grid, runs, nruns, ntiles, s);
}
}  // namespace rlbk
