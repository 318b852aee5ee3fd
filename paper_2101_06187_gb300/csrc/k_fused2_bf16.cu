// Two steps per launch, __nv_bfloat16 storage, CFL 1: single-lattice and ensemble kernels.
#define RLBM_F2_TS __nv_bfloat16
#define RLBM_F2_SFX bf16
#define RLBM_F2_SUB1 0
#include "k_fused2_inst.cuh"
