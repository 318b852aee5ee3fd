// Four nodes per thread, FP16 storage, FP32 Landau frame.
#define RLBM_Q_TS __half
#define RLBM_Q_SFX f16
#define RLBM_Q_DFL 0
#include "k_quad_inst.cuh"
