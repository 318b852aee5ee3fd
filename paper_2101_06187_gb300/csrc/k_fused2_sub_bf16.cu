// Two steps per launch, __nv_bfloat16 storage, 0 < cfl < 1 (the launch's bilinear weights).
#define RLBM_F2_TS __nv_bfloat16
#define RLBM_F2_SFX bf16
#define RLBM_F2_SUB1 1
#include "k_fused2_inst.cuh"
