// k_ring_fused2.cuh -- two time steps per launch for the 2D ring variant
// (k_ring.cuh), in packed FP32 lanes: the tile scheme of k_step_fused2.cuh
// with the ring's 8 directions.  Each CTA updates its TW x TH tile plus a
// one-cell halo ((TW + 4) x (TH + 2) nodes; the extra columns keep node
// pairs 8-byte aligned) by one step into shared memory in the storage type,
// then the tile by a second step from there, with the arithmetic of
// k_ring_step_pair, so two steps here equal two packed ring steps bit for
// bit.  CFL 1, nx even, fewer than 2^31 elements in the 8 planes.
#pragma once

#include "k_ring.cuh"
#include "k_step_fused2.cuh"

namespace rlbk {

// Pull of ring direction k for the node pair at window column x0 (rows[j]:
// offsets of the window rows above, at and below the pair), from shared
// memory; the taps, weights and order of ring_gather_pair.
template <int k, typename TS>
__device__ __forceinline__ pf2 ring_pull_pair_shared(const TS *src, int cbase, const int (&rows)[3], int x0) {
    constexpr int ox = ring_ox(k), oy = ring_oy(k);
    constexpr double tx = ring_tx(k), ty = ring_ty(k);
    auto row = [&](const TS *r, float (&a)[4]) {
        lds_run2<TS>(r + x0, &a[1]);
        if constexpr (ox == -1) a[0] = lds1<TS>(r + (x0 - 1));
        if constexpr (ox == 1 || (ox == 0 && tx != 0.0)) a[3] = lds1<TS>(r + (x0 + 2));
    };
    float a[4];
    row(src + (cbase + rows[oy + 1]), a);
    pf2 v = pf2((float)((1.0 - tx) * (1.0 - ty))) * pf2(a[ox + 1], a[ox + 2]);
    if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * (1.0 - ty))), pf2(a[ox + 2], a[ox + 3]), v);
    if constexpr (ty != 0.0) {
        float b[4];
        row(src + (cbase + rows[oy + 2]), b);
        v = fmadd(pf2((float)((1.0 - tx) * ty)), pf2(b[ox + 1], b[ox + 2]), v);
        if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * ty)), pf2(b[ox + 2], b[ox + 3]), v);
    }
    return v;
}

template <typename TS, int TW, int TH>
constexpr int ring_fused2_smem_bytes() {
    return NR * (TW + 4) * (TH + 2) * (int)sizeof(TS);
}

// Two ring steps, one TW x TH tile per CTA (blockIdx.x, blockIdx.y), NT
// threads; the window lives in static shared memory (under 48 KB).
template <typename TS, bool FORCED, int TW, int TH, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_ring_fused2(const TS *__restrict__ qin, TS *__restrict__ qout, const float *__restrict__ F, StepParams p) {
    static_assert(TW % 2 == 0, "tiles hold whole node pairs");
    static_assert(ring_fused2_smem_bytes<TS, TW, TH>() <= 48 * 1024, "static shared memory");
    constexpr int SW = TW + 4, SH = TH + 2, SPLANE = SW * SH;
    constexpr int PW1 = SW / 2, NP1 = PW1 * SH;
    constexpr int PW2 = TW / 2, NP2 = PW2 * TH;
    __shared__ __align__(16) TS S[NR * SPLANE];
    const int tx0 = blockIdx.x * TW, ty0 = blockIdx.y * TH;

    // step t -> t+1 on the window: local (lr, lc) <-> node
    // ((tx0 - 2 + lc) mod nx, (ty0 - 1 + lr) mod ny)
    for (int i = threadIdx.x; i < NP1; i += NT) {
        const int lr = i / PW1, lc = (i - lr * PW1) * 2;
        const int x0 = wrap_window(tx0 - 2 + lc, p.nx), y = wrap_window(ty0 - 1 + lr, p.ny);
        const int ym = (y == 0) ? p.ny - 1 : y - 1;
        const int yp = (y == p.ny - 1) ? 0 : y + 1;
        const int xl = (x0 == 0) ? p.nx - 1 : x0 - 1;
        const int xr = (x0 + 2 == p.nx) ? 0 : x0 + 2;
        const long long rowoff[3] = {(long long)ym * p.pitch, (long long)y * p.pitch, (long long)yp * p.pitch};
        pf2 q[NR];
        static_for<0, NR>([&](auto K) {
            constexpr int k = decltype(K)::value;
            q[k] = ring_gather_pair<k, TS>(qin, (long long)k * p.plane, rowoff, x0, xl, xr);
        });
        const long long n0 = rowoff[1] + x0;
        pf2 Fx = 0.0f, Fy = 0.0f;
        if constexpr (FORCED) {
            float fx[2], fy[2];
            load_run<float, float, 2>(F + n0, fx);
            load_run<float, float, 2>(F + p.plane + n0, fy);
            Fx = pf2(fx[0], fx[1]);
            Fy = pf2(fy[0], fy[1]);
        }
        ring_collide<pf2, pf2, FORCED>(q, Fx, Fy, p);
        static_for<0, NR>([&](auto K) {
            constexpr int k = decltype(K)::value;
            const float out[2] = {q[k].v.x, q[k].v.y};
            store_run<TS, float, 2>(S + (k * SPLANE + lr * SW + lc), out);
        });
    }
    __syncthreads();

    // step t+1 -> t+2 on the tile, pulling from the window
    for (int i = threadIdx.x; i < NP2; i += NT) {
        const int r = i / PW2, c2 = (i - r * PW2) * 2;
        const int x0 = tx0 + c2, y = ty0 + r;
        if (x0 >= p.nx || y >= p.ny) continue;
        const int lr = r + 1, lc = c2 + 2;
        const int rows[3] = {(lr - 1) * SW, lr * SW, (lr + 1) * SW};
        pf2 q[NR];
        static_for<0, NR>([&](auto K) {
            constexpr int k = decltype(K)::value;
            q[k] = ring_pull_pair_shared<k, TS>(S, k * SPLANE, rows, lc);
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
        ring_collide<pf2, pf2, FORCED>(q, Fx, Fy, p);
        static_for<0, NR>([&](auto K) {
            constexpr int k = decltype(K)::value;
            const float out[2] = {q[k].v.x, q[k].v.y};
            store_run<TS, float, 2>(qout + (long long)k * p.plane + n0, out);
        });
    }
}

}  // namespace rlbk
