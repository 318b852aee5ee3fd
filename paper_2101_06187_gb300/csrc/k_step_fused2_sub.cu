// Two steps per launch at 0 < cfl < 1 (runtime bilinear weights, halo 1):
// the instantiations of the single-lattice kernels in that streaming mode.
#include "k_fused2_launch.cuh"

namespace rlbk {

cudaError_t fused2_prepare_sub1() { return fused2_prepare_mode<kStreamSub1>(); }

cudaError_t fused2_launch_sub1(int dtype, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                               const void *F, const StepParams &p, cudaStream_t s) {
    return fused2_launch_mode<kStreamSub1>(dtype, cfg, forced, qin, qout, F, p, s);
}

}  // namespace rlbk
