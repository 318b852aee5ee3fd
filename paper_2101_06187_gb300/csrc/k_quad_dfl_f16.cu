// Four nodes per thread, FP16 storage, Landau frame refined to FP64 accuracy.
#define RLBM_Q_TS __half
#define RLBM_Q_SFX f16
#define RLBM_Q_DFL 1
#include "k_quad_inst.cuh"
