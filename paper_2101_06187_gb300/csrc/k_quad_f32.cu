// Four nodes per thread, FP32 storage, FP32 Landau frame.
#define RLBM_Q_TS float
#define RLBM_Q_SFX f32
#define RLBM_Q_DFL 0
#include "k_quad_inst.cuh"
