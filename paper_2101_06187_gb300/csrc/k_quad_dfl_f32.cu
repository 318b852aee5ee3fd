// Four nodes per thread, FP32 storage, Landau frame refined to FP64 accuracy.
#define RLBM_Q_TS float
#define RLBM_Q_SFX f32
#define RLBM_Q_DFL 1
#include "k_quad_inst.cuh"
