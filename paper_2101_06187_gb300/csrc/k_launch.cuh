// k_launch.cuh -- launch helpers instantiated once per storage form (one
// translation unit each, so the forms compile in parallel).
#pragma once

#include "k_step_gather.cuh"
#include "k_step_pair.cuh"
#include "k_step_vec.cuh"
#include "rlbm_internal.h"

namespace rlbk {

inline dim3 gather_block() { return dim3(32, 8, 1); }
inline dim3 gather_grid(const StepParams &p) { return dim3((p.nx + 31) / 32, (p.ny + 7) / 8, 1); }

template <typename TS, typename TC, typename TL>
cudaError_t launch_step_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                          const StepParams &p, cudaStream_t s) {
    const TS *in = static_cast<const TS *>(qin);
    TS *out = static_cast<TS *>(qout);
    const TC *f = static_cast<const TC *>(F);
    if (cfg.bx < 1 || cfg.by < 1 || cfg.bx * cfg.by > 256) return cudaErrorInvalidConfiguration;
    const dim3 block(cfg.bx, cfg.by, 1);
    if ((cfg.kernel == RLBM_KERNEL_GATHER_VEC || cfg.kernel == RLBM_KERNEL_GATHER_VEC2 ||
         cfg.kernel == RLBM_KERNEL_TWOPASS) &&
        p.cfl != 1.0)
        return cudaErrorInvalidValue;  // the vector kernels stream at CFL 1 only
    if (cfg.kernel == RLBM_KERNEL_TWOPASS) {
        if constexpr (std::is_same<TC, float>::value && std::is_same<TL, float>::value) {
            if (p.nx % 2 != 0) return cudaErrorInvalidValue;
            const dim3 grid((p.nx / 2 + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
#define RLBM_PAIR2(MB)                                                                  \
    do {                                                                                \
        if (forced) k_step_pair2<TS, true, MB><<<grid, block, 0, s>>>(in, out, f, p);   \
        else k_step_pair2<TS, false, MB><<<grid, block, 0, s>>>(in, out, f, p);         \
    } while (0)
            if (cfg.minb >= 4) RLBM_PAIR2(4);
            else if (cfg.minb == 3) RLBM_PAIR2(3);
            else RLBM_PAIR2(2);
#undef RLBM_PAIR2
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;  // packed lanes are FP32 with the FP32 Landau solve
        }
    }
    if (cfg.kernel == RLBM_KERNEL_PACKED) {
        if constexpr (std::is_same<TC, float>::value && std::is_same<TL, float>::value) {
            if (p.nx % 2 != 0) return cudaErrorInvalidValue;
            const dim3 grid((p.nx / 2 + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
            const bool idx32p = (long long)NC * p.plane < (1ll << 31) - 1;
            if (p.cfl != 1.0) {
                // runtime weights (0 < cfl < 1) or halo 2 (1 < cfl < 2); budgets 1 (unconstrained)
                // and 2 (<= 128 registers)
#define RLBM_PAIR_SUB(MB, SMV)                                                                         \
    do {                                                                                               \
        if (idx32p) {                                                                                  \
            if (forced) k_step_pair<TS, true, MB, int, SMV><<<grid, block, 0, s>>>(in, out, f, p);     \
            else k_step_pair<TS, false, MB, int, SMV><<<grid, block, 0, s>>>(in, out, f, p);           \
        } else {                                                                                       \
            if (forced) k_step_pair<TS, true, MB, long long, SMV><<<grid, block, 0, s>>>(in, out, f, p); \
            else k_step_pair<TS, false, MB, long long, SMV><<<grid, block, 0, s>>>(in, out, f, p);     \
        }                                                                                              \
    } while (0)
                const bool halo2 = stream_mode(p.cfl) == kStreamHalo2;
                if (cfg.minb == 1) {
                    if (halo2) RLBM_PAIR_SUB(1, kStreamHalo2);
                    else RLBM_PAIR_SUB(1, kStreamSub1);
                } else {
                    if (cfg.bx * cfg.by > 256) return cudaErrorInvalidConfiguration;
                    if (halo2) RLBM_PAIR_SUB(2, kStreamHalo2);
                    else RLBM_PAIR_SUB(2, kStreamSub1);
                }
#undef RLBM_PAIR_SUB
                return cudaGetLastError();
            }
#define RLBM_PAIR(MB)                                                                          \
    do {                                                                                       \
        if (idx32p) {                                                                          \
            if (forced) k_step_pair<TS, true, MB, int><<<grid, block, 0, s>>>(in, out, f, p);  \
            else k_step_pair<TS, false, MB, int><<<grid, block, 0, s>>>(in, out, f, p);        \
        } else {                                                                               \
            if (forced) k_step_pair<TS, true, MB><<<grid, block, 0, s>>>(in, out, f, p);       \
            else k_step_pair<TS, false, MB><<<grid, block, 0, s>>>(in, out, f, p);             \
        }                                                                                      \
    } while (0)
            if (cfg.minb == 5) {
                if (cfg.bx * cfg.by > 128) return cudaErrorInvalidConfiguration;
                RLBM_PAIR(5);
            } else if (cfg.minb == 3) {
                RLBM_PAIR(3);
            } else if (cfg.minb == 2) {
                RLBM_PAIR(2);
            } else {
                RLBM_PAIR(1);
            }
#undef RLBM_PAIR
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;  // packed lanes are FP32 with the FP32 Landau solve
        }
    }
    if (cfg.kernel == RLBM_KERNEL_GATHER_VEC || cfg.kernel == RLBM_KERNEL_GATHER_VEC2) {
        constexpr int V4 = VecOf<TS>::V;
        const int V = (cfg.kernel == RLBM_KERNEL_GATHER_VEC2) ? 2 : V4;
        if (p.nx % V != 0 || p.pitch % V != 0) return cudaErrorInvalidValue;
        const int runs = p.nx / V;
        const dim3 grid((runs + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
        if (V == V4) {
            if (forced)
                k_step_vec<TS, TC, TL, true, V4><<<grid, block, 0, s>>>(in, out, f, p);
            else
                k_step_vec<TS, TC, TL, false, V4><<<grid, block, 0, s>>>(in, out, f, p);
        } else if constexpr (V4 != 2) {
            if (forced)
                k_step_vec<TS, TC, TL, true, 2><<<grid, block, 0, s>>>(in, out, f, p);
            else
                k_step_vec<TS, TC, TL, false, 2><<<grid, block, 0, s>>>(in, out, f, p);
        }
        return cudaGetLastError();
    }
    const dim3 grid((p.nx + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, 1);
    const bool idx32 = (long long)NC * p.plane < (1ll << 31) - 1;
    const int sm = stream_mode(p.cfl);
#define RLBM_GATHER(FOR, IDX, SM) k_step_gather<TS, TC, TL, FOR, IDX, SM><<<grid, block, 0, s>>>(in, out, f, p)
#define RLBM_GATHER_SM(SM)                                 \
    do {                                                   \
        if (idx32) {                                       \
            if (forced) RLBM_GATHER(true, int, SM);        \
            else RLBM_GATHER(false, int, SM);              \
        } else {                                           \
            if (forced) RLBM_GATHER(true, long long, SM);  \
            else RLBM_GATHER(false, long long, SM);        \
        }                                                  \
    } while (0)
    if (sm == kStreamCfl1) RLBM_GATHER_SM(kStreamCfl1);
    else if (sm == kStreamSub1) RLBM_GATHER_SM(kStreamSub1);
    else RLBM_GATHER_SM(kStreamHalo2);
#undef RLBM_GATHER_SM
#undef RLBM_GATHER
    return cudaGetLastError();
}

template <typename TS, typename TC, typename TL>
cudaError_t launch_batch_t(const LaunchCfg &cfg, int grid, const void *runs, int nruns, int ntiles, cudaStream_t s) {
    if (cfg.bx < 1 || cfg.by < 1 || cfg.bx * cfg.by > 256 || grid < 1) return cudaErrorInvalidConfiguration;
    const dim3 block(cfg.bx, cfg.by, 1);
    const BatchRun *r = static_cast<const BatchRun *>(runs);
    if (cfg.kernel == RLBM_KERNEL_PACKED) {
        if constexpr (std::is_same<TC, float>::value && std::is_same<TL, float>::value) {
            if (cfg.minb == 3) k_step_batch_pair<TS, 3><<<grid, block, 0, s>>>(r, nruns, ntiles);
            else k_step_batch_pair<TS, 1><<<grid, block, 0, s>>>(r, nruns, ntiles);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    k_step_batch<TS, TC, TL><<<grid, block, 0, s>>>(r, nruns, ntiles);
    return cudaGetLastError();
}

template <typename TS, typename TC, typename TL>
cudaError_t launch_moments_t(const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                             double *partials, int *bad, cudaStream_t s) {
    const TS *q = static_cast<const TS *>(qin);
    const int sm = stream_mode(p.cfl);
    if (sm == kStreamCfl1)
        k_moments<TS, TC, TL, kStreamCfl1><<<gather_grid(p), gather_block(), 0, s>>>(q, p, eps, vx, vy, partials, bad);
    else if (sm == kStreamSub1)
        k_moments<TS, TC, TL, kStreamSub1><<<gather_grid(p), gather_block(), 0, s>>>(q, p, eps, vx, vy, partials, bad);
    else
        k_moments<TS, TC, TL, kStreamHalo2><<<gather_grid(p), gather_block(), 0, s>>>(q, p, eps, vx, vy, partials, bad);
    return cudaGetLastError();
}

}  // namespace rlbk
