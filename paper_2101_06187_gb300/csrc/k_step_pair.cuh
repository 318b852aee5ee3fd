// k_step_pair.cuh -- fused stream + collide + force step for two x-adjacent
// nodes per thread whose whole arithmetic runs in packed FP32 lanes
// (packed.cuh): one instruction advances both nodes.  FP32 compute (FP32,
// BF16, FP16 storage), FP32 Landau solve, 0 < cfl < 2, nx even.
#pragma once

#include "k_step_vec.cuh"
#include "packed.cuh"

namespace rlbk {

// Stochastic rounding of the two values (a at x0, b at x0 + 1) of a node
// pair to the 16-bit storage type: the hardware conversion with stochastic
// rounding (cvt.rs) rounds up with probability equal to the value's
// distance from the lower neighbour in units of the gap, using the random
// bits supplied.  Those are hashed, once per node pair, from the pair's
// index and the bits of its two updated rest-class values (xor-combined
// with odd multipliers, then the "lowbias32" finaliser from C. Wellons'
// hash-prospector), and per class from that seed xor the bits of the
// class's value times an odd multiplier of the class.  The rounding is thus a
// deterministic function of the state: runs repeat bit for bit, a halo node
// recomputed by two tiles rounds the same way in both, and checkpoints
// resume bitwise; the rest values change every step wherever the fluid
// moves, so the draws do too.
__device__ __forceinline__ unsigned sr_pair_seed(unsigned node, float a0, float b0) {
    unsigned h = (node * 0x85EBCA77u) ^ __float_as_uint(a0) ^ (__float_as_uint(b0) * 0x9E3779B1u);
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}

// Odd multiplier of class c (distinct per class).
__host__ __device__ constexpr unsigned sr_class_mult(int c) { return 0xC2B2AE3Du + 0x27D4EB2Eu * (unsigned)c; }

template <typename TS>
__device__ __forceinline__ unsigned cvt_pair_sr(float a, float b, unsigned rbits) {
    unsigned d;
    // the first source goes to the upper half (the element at x0 + 1)
    if constexpr (std::is_same<TS, __half>::value)
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(b), "f"(a), "r"(rbits));
    else
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(b), "f"(a), "r"(rbits));
    return d;
}

// Whether a lattice with storage TS rounds its stores stochastically.
template <typename TS>
__device__ __forceinline__ bool rounds_sr(const StepParams &p) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value || std::is_same<TS, __half>::value) return p.round_sr != 0;
    else return false;
}

// Store of a node pair's two values of class c: rounded to nearest, or
// stochastically (pair seed `seed`) for the 16-bit types when the lattice
// asks for it.
template <typename TS, int C>
__device__ __forceinline__ void store_pair(TS *p, float a, float b, const StepParams &prm, unsigned seed) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value || std::is_same<TS, __half>::value) {
        if (prm.round_sr) {
            const unsigned r = (seed ^ __float_as_uint(a)) * sr_class_mult(C);
            *reinterpret_cast<unsigned *>(p) = cvt_pair_sr<TS>(a, b, r);
            return;
        }
    }
    const float out[2] = {a, b};
    store_run<TS, float, 2>(p, out);
}

// The fused step of the node pair (x0, x0 + 1) of row y in packed lanes.
// I is the index type of the element offsets: 32-bit when all 17 planes fit,
// so each load address is one 32-bit sum and one widening add.  SM is the
// streaming mode: kStreamCfl1 (corners and weights fixed at compile time),
// kStreamSub1 (0 < cfl < 1: each moving class interpolates between the
// cell it streams from and its own, with the launch's per-class weights) or
// kStreamHalo2 (1 < cfl < 2: the corner of an axis with cfl |c| > 1 lies two
// cells away; each x-moving class row is read as the two aligned column
// pairs that cover both candidate corners, and a register select picks the
// launch's corner).
// DFL: the Landau frame refined to FP64 accuracy on the FP32 lanes
// (landau_refine_df), the library's FP64 Landau solve for these kernels.
template <typename TS, bool FORCED, typename I = long long, int SM = kStreamCfl1, bool DFL = false>
__device__ __forceinline__ void step_pair(const TS *__restrict__ qin, TS *__restrict__ qout,
                                          const float *__restrict__ F, const StepParams &p, int x0, int y) {
    const int ym = (y == 0) ? p.ny - 1 : y - 1;
    const int yp = (y == p.ny - 1) ? 0 : y + 1;
    const int xl = (x0 == 0) ? p.nx - 1 : x0 - 1;
    const int xr = (x0 + 2 == p.nx) ? 0 : x0 + 2;
    const I rowoff[3] = {(I)ym * (I)p.pitch, (I)y * (I)p.pitch, (I)yp * (I)p.pitch};
    const I plane = (I)p.plane;
    [[maybe_unused]] I rowoff5[5];
    [[maybe_unused]] int xl2 = 0, xr2 = 0;
    if constexpr (SM == kStreamHalo2) {
        const int ym2 = (ym == 0) ? p.ny - 1 : ym - 1;
        const int yp2 = (yp == p.ny - 1) ? 0 : yp + 1;
        rowoff5[0] = (I)ym2 * (I)p.pitch;
        rowoff5[1] = rowoff[0];
        rowoff5[2] = rowoff[1];
        rowoff5[3] = rowoff[2];
        rowoff5[4] = (I)yp2 * (I)p.pitch;
        xl2 = (x0 == 0) ? p.nx - 2 : x0 - 2;  // the aligned pair (x0-2, x0-1), periodic (nx even)
        xr2 = (x0 + 2 == p.nx) ? 0 : x0 + 2;  // the aligned pair (x0+2, x0+3)
    }

    pf2 q[NC];
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        constexpr int ox = cls_ox(c), oy = cls_oy(c);
        constexpr double tx = cls_tx(c), ty = cls_ty(c);
        auto row = [&](I r, float (&a)[4]) {
            const I base = (I)c * plane + r;
            load_run<TS, float, 2>(qin + (base + (I)x0), &a[1]);
            if constexpr (ox == -1) a[0] = load_q<TS, float>(qin + (base + (I)xl));
            if constexpr (ox == 1 || (ox == 0 && tx != 0.0)) a[3] = load_q<TS, float>(qin + (base + (I)xr));
        };
        if constexpr (SM == kStreamCfl1) {
            float a[4];  // columns x0-1 .. x0+2
            row(rowoff[oy + 1], a);
            // a whole-cell shift (weight 1) needs no multiply: 1 * a is a exactly
            pf2 v = (tx == 0.0 && ty == 0.0) ? pf2(a[ox + 1], a[ox + 2])
                                              : pf2((float)((1.0 - tx) * (1.0 - ty))) * pf2(a[ox + 1], a[ox + 2]);
            if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * (1.0 - ty))), pf2(a[ox + 2], a[ox + 3]), v);
            if constexpr (ty != 0.0) {
                float b[4];
                row(rowoff[oy + 2], b);
                v = fmadd(pf2((float)((1.0 - tx) * ty)), pf2(b[ox + 1], b[ox + 2]), v);
                if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * ty)), pf2(b[ox + 2], b[ox + 3]), v);
            }
            q[c] = v;
        } else if constexpr (SM == kStreamHalo2) {
            constexpr double cx = cls_cx(c), cy = cls_cy(c);
            constexpr int nx_ = cx > 0 ? -1 : 0, ny_ = cy > 0 ? -1 : 0;  // near corner
            constexpr int fy = cy > 0 ? -1 : 1;                              // step to the far row
            constexpr bool mx = cx != 0.0, my = cy != 0.0;
            const bool farx = mx && ((p.far_x >> c) & 1u);
            const bool fary = my && ((p.far_y >> c) & 1u);
            // the three columns of the pair's bilinear taps: near or far corner
            auto row3 = [&](I r, float (&t)[3]) {
                const I base = (I)c * plane + r;
                float mid[2], side[2];
                load_run<TS, float, 2>(qin + (base + (I)x0), mid);
                if constexpr (!mx) {
                    t[0] = mid[0];
                    t[1] = mid[1];
                } else if constexpr (nx_ == -1) {  // columns x0-2 .. x0+1
                    load_run<TS, float, 2>(qin + (base + (I)xl2), side);
                    t[0] = farx ? side[0] : side[1];
                    t[1] = farx ? side[1] : mid[0];
                    t[2] = farx ? mid[0] : mid[1];
                } else {  // columns x0 .. x0+3
                    load_run<TS, float, 2>(qin + (base + (I)xr2), side);
                    t[0] = farx ? mid[1] : mid[0];
                    t[1] = farx ? side[0] : mid[1];
                    t[2] = farx ? side[1] : side[0];
                }
            };
            const I ra = fary ? rowoff5[ny_ + fy + 2] : rowoff5[ny_ + 2];
            float t[3];
            row3(ra, t);
            if constexpr (!mx && !my) {
                q[c] = pf2(t[0], t[1]);
            } else {
                pf2 v = pf2(par_wt<float>(p, c, 0)) * pf2(t[0], t[1]);
                if constexpr (mx) v = fmadd(pf2(par_wt<float>(p, c, 1)), pf2(t[1], t[2]), v);
                if constexpr (my) {
                    const I rb = fary ? rowoff5[ny_ + fy + 3] : rowoff5[ny_ + 3];
                    float u[3];
                    row3(rb, u);
                    v = fmadd(pf2(par_wt<float>(p, c, 2)), pf2(u[0], u[1]), v);
                    if constexpr (mx) v = fmadd(pf2(par_wt<float>(p, c, 3)), pf2(u[1], u[2]), v);
                }
                q[c] = v;
            }
        } else {
            // near corner (the class's own cell on an axis where it does not move)
            constexpr double cx = cls_cx(c), cy = cls_cy(c);
            constexpr int nx_ = cx > 0 ? -1 : 0, ny_ = cy > 0 ? -1 : 0;
            constexpr bool mx = cx != 0.0, my = cy != 0.0;
            auto row2 = [&](I r, float (&d)[4]) {
                const I base = (I)c * plane + r;
                load_run<TS, float, 2>(qin + (base + (I)x0), &d[1]);
                if constexpr (mx && nx_ == -1) d[0] = load_q<TS, float>(qin + (base + (I)xl));
                if constexpr (mx && nx_ == 0) d[3] = load_q<TS, float>(qin + (base + (I)xr));
            };
            float a[4];  // columns x0-1 .. x0+2
            row2(rowoff[ny_ + 1], a);
            if constexpr (!mx && !my) {
                q[c] = pf2(a[1], a[2]);
            } else {
                pf2 v = pf2(par_wt<float>(p, c, 0)) * pf2(a[nx_ + 1], a[nx_ + 2]);
                if constexpr (mx) v = fmadd(pf2(par_wt<float>(p, c, 1)), pf2(a[nx_ + 2], a[nx_ + 3]), v);
                if constexpr (my) {
                    float b[4];
                    row2(rowoff[ny_ + 2], b);
                    v = fmadd(pf2(par_wt<float>(p, c, 2)), pf2(b[nx_ + 1], b[nx_ + 2]), v);
                    if constexpr (mx) v = fmadd(pf2(par_wt<float>(p, c, 3)), pf2(b[nx_ + 2], b[nx_ + 3]), v);
                }
                q[c] = v;
            }
        }
    });

    const I n0 = rowoff[1] + (I)x0;
    pf2 Fx = 0.0f, Fy = 0.0f;
    if constexpr (FORCED) {
        float fx[2], fy[2];
        load_run<float, float, 2>(F + n0, fx);
        load_run<float, float, 2>(F + (plane + n0), fy);
        Fx = pf2(fx[0], fx[1]);
        Fy = pf2(fy[0], fy[1]);
    }
    // FP32 storage keeps the deviation unscaled (s = 1)
    collide_node<pf2, pf2, FORCED, DFL, std::is_same<TS, float>::value>(q, Fx, Fy, p);

    const unsigned seed =
        rounds_sr<TS>(p) ? sr_pair_seed((unsigned)y * (unsigned)p.nx + (unsigned)x0, q[0].v.x, q[0].v.y) : 0u;
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        store_pair<TS, c>(qout + ((I)c * plane + n0), q[c].v.x, q[c].v.y, p, seed);
    });
}

// Two-pass form of step_pair: the first pass gathers one opposite pair at a
// time and keeps only the moment sums; the collision coefficients follow
// from them; the second pass gathers each pair again (from L1/L2: the same
// lines were just read) and writes its updated values.  No node keeps its
// 17 populations live across the Landau solve, which halves the registers
// per thread and doubles the warps an SM can hold.  Same arithmetic as
// step_pair, in the same order.
template <typename TS, bool FORCED>
__device__ __forceinline__ void step_pair_twopass(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                  const float *__restrict__ F, const StepParams &p, int x0, int y) {
    const int ym = (y == 0) ? p.ny - 1 : y - 1;
    const int yp = (y == p.ny - 1) ? 0 : y + 1;
    const int xl = (x0 == 0) ? p.nx - 1 : x0 - 1;
    const int xr = (x0 + 2 == p.nx) ? 0 : x0 + 2;
    const long long rowoff[3] = {(long long)ym * p.pitch, (long long)y * p.pitch, (long long)yp * p.pitch};
    auto gather = [&](const TS *src, auto C) -> pf2 {
        constexpr int c = decltype(C)::value;
        constexpr int ox = cls_ox(c), oy = cls_oy(c);
        constexpr double tx = cls_tx(c), ty = cls_ty(c);
        const TS *plane = src + (long long)c * p.plane;
        float a[4];
        load_class_row<c, TS, float, 2>(plane + rowoff[oy + 1], x0, xl, xr, a);
        pf2 v = pf2((float)((1.0 - tx) * (1.0 - ty))) * pf2(a[ox + 1], a[ox + 2]);
        if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * (1.0 - ty))), pf2(a[ox + 2], a[ox + 3]), v);
        if constexpr (ty != 0.0) {
            float b[4];
            load_class_row<c, TS, float, 2>(plane + rowoff[oy + 2], x0, xl, xr, b);
            v = fmadd(pf2((float)((1.0 - tx) * ty)), pf2(b[ox + 1], b[ox + 2]), v);
            if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * ty)), pf2(b[ox + 2], b[ox + 3]), v);
        }
        return v;
    };
    using I0 = std::integral_constant<int, 0>;

    MomentSums<pf2> acc = moments_begin<pf2>(gather(qin, I0{}));
    static_for<0, NPAIR>([&](auto K) {
        constexpr int k = decltype(K)::value;
        moments_add_pair<k, pf2>(acc, gather(qin, std::integral_constant<int, pair_pos(k)>{}),
                                 gather(qin, std::integral_constant<int, pair_neg(k)>{}));
    });
    const NodeMoments<pf2> m = moments_end<pf2>(acc, par_scale<pf2>(p));

    const long long n0 = (long long)y * p.pitch + x0;
    pf2 Fx = 0.0f, Fy = 0.0f;
    if constexpr (FORCED) {
        float fx[2], fy[2];
        load_run<float, float, 2>(F + n0, fx);
        load_run<float, float, 2>(F + p.plane + n0, fy);
        Fx = pf2(fx[0], fx[1]);
        Fy = pf2(fy[0], fy[1]);
    }
    CollideCoef<pf2> cf;
    collide_coef<pf2, pf2, FORCED>(m, Fx, Fy, p, cf);

    const TS *again = qin + p.reload_offset;
    auto store = [&](int c, pf2 v) {
        const float out[2] = {v.v.x, v.v.y};
        store_run<TS, float, 2>(qout + (long long)c * p.plane + n0, out);
    };
    store(0, collide_rest<pf2>(gather(again, I0{}), cf));
    static_for<0, NPAIR>([&](auto K) {
        constexpr int k = decltype(K)::value;
        pf2 qp = gather(again, std::integral_constant<int, pair_pos(k)>{});
        pf2 qn = gather(again, std::integral_constant<int, pair_neg(k)>{});
        collide_pair<k, pf2, FORCED>(qp, qn, cf);
        store(pair_pos(k), qp);
        store(pair_neg(k), qn);
    });
}

template <typename TS, bool FORCED, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step_pair2(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                          const float *__restrict__ F, StepParams p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
    step_pair_twopass<TS, FORCED>(qin, qout, F, p, x0, y);
}

// MINB: minimum resident blocks of 256 threads per SM asked of the register
// allocator (1: unconstrained; 2: <= 128 registers; 3: <= 80), so the
// autotuner can trade registers for occupancy.
// MINB 5: blocks of at most 128 threads, five resident per SM (at most 102
// registers per thread: 20 warps per SM).
template <typename TS, bool FORCED, int MINB, typename I = long long, int SM = kStreamCfl1, bool DFL = false>
__global__ void __launch_bounds__(MINB == 5 ? 128 : 256, MINB)
    k_step_pair(const TS *__restrict__ qin, TS *__restrict__ qout, const float *__restrict__ F, StepParams p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
    step_pair<TS, FORCED, I, SM, DFL>(qin, qout, F, p, x0, y);
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
        if (x0 < r.p.nx && y < r.p.ny) {  // members hold fewer than 2^31 / 17 elements per plane: 32-bit offsets
            if (r.F)
                step_pair<TS, true, int>(static_cast<const TS *>(r.qin), static_cast<TS *>(r.qout),
                                         static_cast<const float *>(r.F), r.p, x0, y);
            else
                step_pair<TS, false, int>(static_cast<const TS *>(r.qin), static_cast<TS *>(r.qout), nullptr, r.p, x0,
                                          y);
        }
    }
}

}  // namespace rlbk
