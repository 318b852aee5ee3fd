// Four nodes per thread, BF16 storage, Landau frame refined to FP64 accuracy.
#define RLBM_Q_TS __nv_bfloat16
#define RLBM_Q_SFX bf16
#define RLBM_Q_DFL 1
#include "k_quad_inst.cuh"
