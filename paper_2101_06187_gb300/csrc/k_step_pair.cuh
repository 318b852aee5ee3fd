// k_step_pair.cuh -- fused stream + collide + force step for two x-adjacent
// nodes per thread whose whole arithmetic runs in packed FP32 lanes
// (packed.cuh): one instruction advances both nodes.  FP32 compute (FP32,
// BF16, FP16 storage), FP32 Landau solve, CFL 1, nx even.
#pragma once

#include "k_step_vec.cuh"
#include "packed.cuh"

namespace rlbk {

// The fused step of the node pair (x0, x0 + 1) of row y in packed lanes.
template <typename TS, bool FORCED>
__device__ __forceinline__ void step_pair(const TS *__restrict__ qin, TS *__restrict__ qout,
                                          const float *__restrict__ F, const StepParams &p, int x0, int y) {
    const int ym = (y == 0) ? p.ny - 1 : y - 1;
    const int yp = (y == p.ny - 1) ? 0 : y + 1;
    const int xl = (x0 == 0) ? p.nx - 1 : x0 - 1;
    const int xr = (x0 + 2 == p.nx) ? 0 : x0 + 2;
    const long long rowoff[3] = {(long long)ym * p.pitch, (long long)y * p.pitch, (long long)yp * p.pitch};

    pf2 q[NC];
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        constexpr int ox = cls_ox(c), oy = cls_oy(c);
        constexpr double tx = cls_tx(c), ty = cls_ty(c);
        const TS *plane = qin + (long long)c * p.plane;
        float a[4];  // columns x0-1 .. x0+2
        load_class_row<c, TS, float, 2>(plane + rowoff[oy + 1], x0, xl, xr, a);
        pf2 v = pf2((float)((1.0 - tx) * (1.0 - ty))) * pf2(a[ox + 1], a[ox + 2]);
        if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * (1.0 - ty))), pf2(a[ox + 2], a[ox + 3]), v);
        if constexpr (ty != 0.0) {
            float b[4];
            load_class_row<c, TS, float, 2>(plane + rowoff[oy + 2], x0, xl, xr, b);
            v = fmadd(pf2((float)((1.0 - tx) * ty)), pf2(b[ox + 1], b[ox + 2]), v);
            if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * ty)), pf2(b[ox + 2], b[ox + 3]), v);
        }
        q[c] = v;
    });

    const long long n0 = (long long)y * p.pitch + x0;
    pf2 Fx = 0.0f, Fy = 0.0f;
    if constexpr (FORCED) {
        float fx[2], fy[2];
        load_run<float, float, 2>(F + n0, fx);
        load_run<float, float, 2>(F + p.plane + n0, fy);
        Fx = pf2(fx[0], fx[1]);
        Fy = pf2(fy[0], fy[1]);
    }
    collide_node<pf2, pf2, FORCED>(q, Fx, Fy, p);

    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        const float out[2] = {q[c].v.x, q[c].v.y};
        store_run<TS, float, 2>(qout + (long long)c * p.plane + n0, out);
    });
}

// MINB: minimum resident blocks of 256 threads per SM asked of the register
// allocator (1: unconstrained; 2: <= 128 registers; 3: <= 80), so the
// autotuner can trade registers for occupancy.
template <typename TS, bool FORCED, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step_pair(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                         const float *__restrict__ F, StepParams p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
    step_pair<TS, FORCED>(qin, qout, F, p, x0, y);
}

// Ensemble step with the packed body (see k_step_batch).
template <typename TS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step_batch_pair(const BatchRun *__restrict__ runs, int nruns,
                                                               int ntiles) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int lo = 0, hi = nruns - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (runs[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchRun &r = runs[lo];
        const int local = t - r.tile0;
        const int tx = local % r.tiles_x, ty = local / r.tiles_x;
        const int x0 = (tx * blockDim.x + threadIdx.x) * 2;
        const int y = ty * blockDim.y + threadIdx.y;
        if (x0 < r.p.nx && y < r.p.ny) {
            if (r.F)
                step_pair<TS, true>(static_cast<const TS *>(r.qin), static_cast<TS *>(r.qout),
                                    static_cast<const float *>(r.F), r.p, x0, y);
            else
                step_pair<TS, false>(static_cast<const TS *>(r.qin), static_cast<TS *>(r.qout), nullptr, r.p, x0, y);
        }
    }
}

}  // namespace rlbk
