// Two steps per launch, float storage, 0 < cfl < 1 (the launch's bilinear weights).
#define RLBM_F2_TS float
#define RLBM_F2_SFX f32
#define RLBM_F2_SUB1 1
#include "k_fused2_inst.cuh"
