// k_quad_inst.cuh -- the four-nodes-per-thread packed step (k_step_quad.cuh)
// of one storage type and one Landau precision behind a plain entry point
// (declared in rlbm_internal.h).  Included once per translation unit with
//   RLBM_Q_TS    the storage type (float, __nv_bfloat16, __half),
//   RLBM_Q_SFX   the entry point's suffix (f32, bf16, f16),
//   RLBM_Q_DFL   0: the FP32 Landau frame (launch_step_quad_<sfx>);
//                1: the frame refined to FP64 accuracy (launch_step_quad_dfl_<sfx>),
// so the instantiations compile in parallel.
#include "k_step_quad.cuh"
#include "rlbm_internal.h"

#define RLBM_Q_CAT2(a, b) a##b
#define RLBM_Q_CAT(a, b) RLBM_Q_CAT2(a, b)

namespace rlbk {
namespace {

// cfg.bx x cfg.by threads (at most 128), each a run of four nodes; cfg.minb
// 3 or 4 blocks per SM (at most 168 or 128 registers).  The rounding of
// 16-bit stores (p.round_sr) picks the instantiation here, once per launch.
template <typename TS, bool DFL>
cudaError_t quad_launch_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                          const StepParams &p, cudaStream_t s) {
    if (cfg.bx < 1 || cfg.by < 1 || cfg.bx * cfg.by > 128) return cudaErrorInvalidConfiguration;
    if (cfg.minb != 3 && cfg.minb != 4) return cudaErrorInvalidValue;
    if (p.nx % 4 != 0 || p.pitch % 4 != 0 || p.cfl != 1.0 || p.nz != 1) return cudaErrorInvalidValue;
    const TS *in = static_cast<const TS *>(qin);
    TS *out = static_cast<TS *>(qout);
    const float *f = static_cast<const float *>(F);
    const dim3 block(cfg.bx, cfg.by, 1);
    const dim3 grid((p.nx / 4 + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
    const bool idx32 = (long long)NC * p.plane < (1ll << 31) - 1;
    constexpr bool h16 = std::is_same<TS, __nv_bfloat16>::value || std::is_same<TS, __half>::value;
    auto go = [&](auto mb, auto sr) {
        constexpr int MB = decltype(mb)::value;
        constexpr bool SR = decltype(sr)::value;
        if (idx32) {
            if (forced) k_step_quad<TS, true, MB, int, DFL, SR><<<grid, block, 0, s>>>(in, out, f, p);
            else k_step_quad<TS, false, MB, int, DFL, SR><<<grid, block, 0, s>>>(in, out, f, p);
        } else {
            if (forced) k_step_quad<TS, true, MB, long long, DFL, SR><<<grid, block, 0, s>>>(in, out, f, p);
            else k_step_quad<TS, false, MB, long long, DFL, SR><<<grid, block, 0, s>>>(in, out, f, p);
        }
    };
    auto budget = [&](auto sr) {
        if (cfg.minb == 3) go(std::integral_constant<int, 3>{}, sr);
        else go(std::integral_constant<int, 4>{}, sr);
    };
    if constexpr (h16) {
        if (p.round_sr) budget(std::true_type{});
        else budget(std::false_type{});
    } else {
        budget(std::false_type{});
    }
    return cudaGetLastError();
}

}  // namespace

#if RLBM_Q_DFL
cudaError_t RLBM_Q_CAT(launch_step_quad_dfl_, RLBM_Q_SFX)(const LaunchCfg &cfg, bool forced, const void *qin,
                                                          void *qout, const void *F, const StepParams &p,
                                                          cudaStream_t s) {
    return quad_launch_t<RLBM_Q_TS, true>(cfg, forced, qin, qout, F, p, s);
}
#else
cudaError_t RLBM_Q_CAT(launch_step_quad_, RLBM_Q_SFX)(const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                                                      const void *F, const StepParams &p, cudaStream_t s) {
    return quad_launch_t<RLBM_Q_TS, false>(cfg, forced, qin, qout, F, p, s);
}
#endif

}  // namespace rlbk
