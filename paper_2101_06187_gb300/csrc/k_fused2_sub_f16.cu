// Two steps per launch, __half storage, 0 < cfl < 1 (the launch's bilinear weights).
#define RLBM_F2_TS __half
#define RLBM_F2_SFX f16
#define RLBM_F2_SUB1 1
#include "k_fused2_inst.cuh"
