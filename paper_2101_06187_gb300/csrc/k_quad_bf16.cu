// Four nodes per thread, BF16 storage, FP32 Landau frame.
#define RLBM_Q_TS __nv_bfloat16
#define RLBM_Q_SFX bf16
#define RLBM_Q_DFL 0
#include "k_quad_inst.cuh"
