// Two steps per launch, float storage, CFL 1: single-lattice and ensemble kernels.
#define RLBM_F2_TS float
#define RLBM_F2_SFX f32
#define RLBM_F2_SUB1 0
#include "k_fused2_inst.cuh"
