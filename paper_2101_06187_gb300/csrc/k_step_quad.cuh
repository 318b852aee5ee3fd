// k_step_quad.cuh -- the packed fused step for four x-adjacent nodes per
// thread: the node pairs (x0, x0 + 1) and (x0 + 2, x0 + 3), each in packed
// FP32 lanes.  Each class row around the four nodes is read as one aligned
// run of four stored values plus at most one side value (x0 - 1 or x0 + 4),
// so per node a thread issues half the loads, and half the load-address
// arithmetic, of the two-node kernel, and its two pairs are independent
// chains for the scheduler.  Per lane the taps, weights, operation order and
// store rounding are those of step_pair at CFL 1, so results equal
// k_step_pair's bit for bit.  Needs nx divisible by 4 and the pitch by 4
// (aligned runs).
#pragma once

#include "k_step_pair.cuh"

namespace rlbk {

// Store of class c for the two pairs (a0, a1) at x0 and (b0, b1) at x0 + 2:
// one 4-value store, rounded as two store_pair calls would round.  SR: the
// lattice rounds its 16-bit stores stochastically (fixed per launch, so the
// choice is made once on the host, not per class).
template <typename TS, int C, bool SR>
__device__ __forceinline__ void store_quad(TS *p, float a0, float a1, float b0, float b1, unsigned seed_a,
                                           unsigned seed_b) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value || std::is_same<TS, __half>::value) {
        if constexpr (SR) {
            const unsigned ra = (seed_a ^ __float_as_uint(a0)) * sr_class_mult(C);
            const unsigned rb = (seed_b ^ __float_as_uint(b0)) * sr_class_mult(C);
            *reinterpret_cast<uint2 *>(p) = make_uint2(cvt_pair_sr<TS>(a0, a1, ra), cvt_pair_sr<TS>(b0, b1, rb));
            return;
        }
    }
    const float out[4] = {a0, a1, b0, b1};
    store_run<TS, float, 4>(p, out);
}

// Columns a class row of a run of four reads besides the run itself: x0 - 1
// (a class pulling from the left) or x0 + 4 (from the right), at CFL 1.
__host__ __device__ constexpr bool quad_left(int c) { return cls_ox(c) == -1; }
__host__ __device__ constexpr bool quad_right(int c) {
    return cls_ox(c) == 1 || (cls_ox(c) == 0 && cls_tx(c) != 0.0);
}

// Bilinear pull at CFL 1 (Sec. 3.2) of the pairs (x0, x0 + 1) -> qa and
// (x0 + 2, x0 + 3) -> qb.  row(C, r, a) fills the class row r around the
// run: a[1..4] = columns x0 .. x0 + 3, a[0] = x0 - 1 if quad_left(c), a[5] =
// x0 + 4 if quad_right(c) (pair j reads a[2j .. 2j + 3]); rows[k] is row
// y - 1 + k in whatever offsets row() takes.  Taps, weights and operation
// order per lane are those of step_pair.
template <typename I, typename RowFn>
__device__ __forceinline__ void pull_quad(RowFn &&row, const I (&rows)[3], pf2 (&qa)[NC], pf2 (&qb)[NC]) {
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        constexpr int ox = cls_ox(c), oy = cls_oy(c);
        constexpr double tx = cls_tx(c), ty = cls_ty(c);
        constexpr float w00 = (float)((1.0 - tx) * (1.0 - ty)), w10 = (float)(tx * (1.0 - ty));
        constexpr float w01 = (float)((1.0 - tx) * ty), w11 = (float)(tx * ty);
        float a[6];
        row(C, rows[oy + 1], a);
        // a whole-cell shift (weight 1) needs no multiply: 1 * a is a exactly
        pf2 va, vb;
        if constexpr (tx == 0.0 && ty == 0.0) {
            va = pf2(a[ox + 1], a[ox + 2]);
            vb = pf2(a[ox + 3], a[ox + 4]);
        } else {
            va = pf2(w00) * pf2(a[ox + 1], a[ox + 2]);
            vb = pf2(w00) * pf2(a[ox + 3], a[ox + 4]);
        }
        if constexpr (tx != 0.0) {
            va = fmadd(pf2(w10), pf2(a[ox + 2], a[ox + 3]), va);
            vb = fmadd(pf2(w10), pf2(a[ox + 4], a[ox + 5]), vb);
        }
        if constexpr (ty != 0.0) {
            float b[6];
            row(C, rows[oy + 2], b);
            va = fmadd(pf2(w01), pf2(b[ox + 1], b[ox + 2]), va);
            vb = fmadd(pf2(w01), pf2(b[ox + 3], b[ox + 4]), vb);
            if constexpr (tx != 0.0) {
                va = fmadd(pf2(w11), pf2(b[ox + 2], b[ox + 3]), va);
                vb = fmadd(pf2(w11), pf2(b[ox + 4], b[ox + 5]), vb);
            }
        }
        qa[c] = va;
        qb[c] = vb;
    });
}

// A class row of a run of four from global memory, addressed from three
// per-thread pointers to the run in rows y - 1, y, y + 1 of class 0 plus the
// class's plane offset; the side columns lie at fixed distances dl = xl - x0
// and dr = xr - x0 from the run (-1 and +4 away from the periodic edge).
// (Measured against one 32-bit element offset per load, 10 fewer integer
// instructions per node.)
template <typename TS>
struct QuadRowPtr {
    const TS *rp[3];
    long long plane;
    int dl, dr;
    template <typename C>
    __device__ __forceinline__ void operator()(C, int k, float (&a)[6]) const {
        constexpr int c = C::value;
        const TS *p = rp[k] + (long long)c * plane;
        load_run<TS, float, 4>(p, &a[1]);
        if constexpr (quad_left(c)) a[0] = load_q<TS, float>(p + dl);
        if constexpr (quad_right(c)) a[5] = load_q<TS, float>(p + dr);
    }
};

template <typename TS, bool FORCED, typename I, bool DFL, bool SR>
__device__ __forceinline__ void step_quad(const TS *__restrict__ qin, TS *__restrict__ qout,
                                          const float *__restrict__ F, const StepParams &p, int x0, int y) {
    const int ym = (y == 0) ? p.ny - 1 : y - 1;
    const int yp = (y == p.ny - 1) ? 0 : y + 1;
    const int xl = (x0 == 0) ? p.nx - 1 : x0 - 1;
    const int xr = (x0 + 4 == p.nx) ? 0 : x0 + 4;
    const I rowoff[3] = {(I)ym * (I)p.pitch, (I)y * (I)p.pitch, (I)yp * (I)p.pitch};
    const I plane = (I)p.plane;

    pf2 qa[NC], qb[NC];
    const int rows[3] = {0, 1, 2};
    pull_quad<int>(QuadRowPtr<TS>{{qin + (rowoff[0] + (I)x0), qin + (rowoff[1] + (I)x0), qin + (rowoff[2] + (I)x0)},
                                  (long long)plane, xl - x0, xr - x0},
                   rows, qa, qb);

    const I n0 = rowoff[1] + (I)x0;
    pf2 Fxa = 0.0f, Fya = 0.0f, Fxb = 0.0f, Fyb = 0.0f;
    if constexpr (FORCED) {
        float fx[4], fy[4];
        load_run<float, float, 4>(F + n0, fx);
        load_run<float, float, 4>(F + (plane + n0), fy);
        Fxa = pf2(fx[0], fx[1]);
        Fxb = pf2(fx[2], fx[3]);
        Fya = pf2(fy[0], fy[1]);
        Fyb = pf2(fy[2], fy[3]);
    }
    // FP32 storage keeps the deviation unscaled (s = 1)
    constexpr bool unit = std::is_same<TS, float>::value;
    collide_node<pf2, pf2, FORCED, DFL, unit>(qa, Fxa, Fya, p);
    collide_node<pf2, pf2, FORCED, DFL, unit>(qb, Fxb, Fyb, p);

    unsigned seed_a = 0u, seed_b = 0u;
    if constexpr (SR) {
        const unsigned node = (unsigned)y * (unsigned)p.nx + (unsigned)x0;
        seed_a = sr_pair_seed(node, qa[0].v.x, qa[0].v.y);
        seed_b = sr_pair_seed(node + 2u, qb[0].v.x, qb[0].v.y);
    }
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        store_quad<TS, c, SR>(qout + ((I)c * plane + n0), qa[c].v.x, qa[c].v.y, qb[c].v.x, qb[c].v.y, seed_a,
                              seed_b);
    });
}

// The four-node step over the lattice: blocks of at most 128 threads, each
// thread one run of four nodes; MINB resident blocks per SM asked of the
// register allocator (3: at most 168 registers, 4: at most 128); SR:
// stochastic rounding of the 16-bit stores (the lattice's p.round_sr).
template <typename TS, bool FORCED, int MINB, typename I, bool DFL, bool SR>
__global__ void __launch_bounds__(128, MINB)
    k_step_quad(const TS *__restrict__ qin, TS *__restrict__ qout, const float *__restrict__ F, StepParams p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
    step_quad<TS, FORCED, I, DFL, SR>(qin, qout, F, p, x0, y);
}

}  // namespace rlbk
