// Two steps per launch, __half storage, CFL 1: single-lattice and ensemble kernels.
#define RLBM_F2_TS __half
#define RLBM_F2_SFX f16
#define RLBM_F2_SUB1 0
#include "k_fused2_inst.cuh"
