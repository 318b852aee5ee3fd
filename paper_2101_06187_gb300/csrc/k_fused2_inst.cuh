// k_fused2_inst.cuh -- the two-steps-per-launch kernels of one storage type
// in one streaming mode, behind plain entry points (declared in
// k_fused2_launch.cuh).  Included once per translation unit with
//   RLBM_F2_TS     the storage type (float, __nv_bfloat16, __half),
//   RLBM_F2_SFX    the entry points' suffix (f32, bf16, f16),
//   RLBM_F2_SUB1   0: CFL 1, single-lattice and ensemble kernels;
//                  1: 0 < cfl < 1, single-lattice kernels,
// so the instantiations compile in parallel.
#include "k_fused2_launch.cuh"

#define RLBM_F2_CAT2(a, b) a##b
#define RLBM_F2_CAT(a, b) RLBM_F2_CAT2(a, b)

namespace rlbk {

#if RLBM_F2_SUB1
cudaError_t RLBM_F2_CAT(fused2_prepare_sub1_, RLBM_F2_SFX)() { return fused2_prepare_t<RLBM_F2_TS, kStreamSub1>(); }

cudaError_t RLBM_F2_CAT(fused2_launch_sub1_, RLBM_F2_SFX)(const LaunchCfg &cfg, bool forced, const void *qin,
                                                          void *qout, const void *F, const StepParams &p,
                                                          cudaStream_t s) {
    return fused2_launch_t<RLBM_F2_TS, kStreamSub1>(cfg, forced, qin, qout, F, p, s);
}
#else
cudaError_t RLBM_F2_CAT(fused2_prepare_cfl1_, RLBM_F2_SFX)() {
    const cudaError_t e = fused2_prepare_t<RLBM_F2_TS, kStreamCfl1>();
    return e == cudaSuccess ? batch_prepare_t<RLBM_F2_TS>() : e;
}

cudaError_t RLBM_F2_CAT(fused2_launch_cfl1_, RLBM_F2_SFX)(const LaunchCfg &cfg, bool forced, const void *qin,
                                                          void *qout, const void *F, const StepParams &p,
                                                          cudaStream_t s) {
    return fused2_launch_t<RLBM_F2_TS, kStreamCfl1>(cfg, forced, qin, qout, F, p, s);
}

cudaError_t RLBM_F2_CAT(fused2_launch_batch_, RLBM_F2_SFX)(const LaunchCfg &cfg, int grid, const void *runs, int nruns,
                                                           int ntiles, int two, cudaStream_t s) {
    return batch_launch_t<RLBM_F2_TS>(cfg, grid, runs, nruns, ntiles, two, s);
}
#endif

}  // namespace rlbk
