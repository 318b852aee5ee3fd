// k_step_gather.cuh -- fused stream + collide + force step, one node per
// thread, gathering the streamed populations straight from global memory
// (the 3x3 neighbourhood rows are re-read through L1/L2; HBM sees each
// stored value about once).  Also the moments kernel, which runs the same
// gather + moments + Landau solve without writing populations back.
#pragma once

#include "rlbm_device.cuh"

namespace rlbk {

// Gather class c at node (x, y) by bilinear pull interpolation (Sec. 3.2).
// rowoff[k] / cols[k], k = 0..4, are the periodic neighbours y-2..y+2
// (x-2..x+2); SM is the streaming mode (kStreamCfl1: corners in {-1, 0, +1}
// and weights fixed at compile time; kStreamSub1: same corners, runtime
// weights; kStreamHalo2: the corner of an axis with cfl |c| > 1 moves one
// cell further, to -2 or +1, picked by a register select).  I is the index
// type: 32-bit when 17 planes fit, so each load costs one add.
template <int c, typename TS, typename TC, typename I, int SM>
__device__ __forceinline__ TC gather_class(const TS *__restrict__ qin, I cbase, const I (&rowoff)[5],
                                           const I (&cols)[5], const StepParams &p) {
    if constexpr (SM == kStreamCfl1) {
        constexpr int ox = cls_ox(c), oy = cls_oy(c);
        constexpr double tx = cls_tx(c), ty = cls_ty(c);
        const I r0 = cbase + rowoff[oy + 2];
        TC v = (TC)((1.0 - tx) * (1.0 - ty)) * load_q<TS, TC>(qin + (r0 + cols[ox + 2]));
        if constexpr (tx != 0.0) v += (TC)(tx * (1.0 - ty)) * load_q<TS, TC>(qin + (r0 + cols[ox + 3]));
        if constexpr (ty != 0.0) {
            const I r1 = cbase + rowoff[oy + 3];
            v += (TC)((1.0 - tx) * ty) * load_q<TS, TC>(qin + (r1 + cols[ox + 2]));
            if constexpr (tx != 0.0) v += (TC)(tx * ty) * load_q<TS, TC>(qin + (r1 + cols[ox + 3]));
        }
        return v;
    } else {
        // cfl != 1: every moving class interpolates between the two cells
        // around x - cfl c, with the launch's per-class weights
        constexpr double cx = cls_cx(c), cy = cls_cy(c);
        constexpr int ox = cx > 0 ? -1 : 0, oy = cy > 0 ? -1 : 0;  // near corner
        constexpr int fx = cx > 0 ? -1 : 1, fy = cy > 0 ? -1 : 1;  // step to the far corner
        constexpr bool mx = cx != 0.0, my = cy != 0.0;
        if constexpr (!mx && !my) return load_q<TS, TC>(qin + (cbase + rowoff[2] + cols[2]));
        I x0 = cols[ox + 2], x1 = cols[ox + 3], ra = rowoff[oy + 2], rb = rowoff[oy + 3];
        if constexpr (SM == kStreamHalo2) {
            if (mx && ((p.far_x >> c) & 1u)) {
                x0 = cols[ox + fx + 2];
                x1 = cols[ox + fx + 3];
            }
            if (my && ((p.far_y >> c) & 1u)) {
                ra = rowoff[oy + fy + 2];
                rb = rowoff[oy + fy + 3];
            }
        }
        const I r0 = cbase + ra;
        TC v = par_wt<TC>(p, c, 0) * load_q<TS, TC>(qin + (r0 + x0));
        if constexpr (mx) v += par_wt<TC>(p, c, 1) * load_q<TS, TC>(qin + (r0 + x1));
        if constexpr (my) {
            const I r1 = cbase + rb;
            v += par_wt<TC>(p, c, 2) * load_q<TS, TC>(qin + (r1 + x0));
            if constexpr (mx) v += par_wt<TC>(p, c, 3) * load_q<TS, TC>(qin + (r1 + x1));
        }
        return v;
    }
}

// Periodic neighbour a + d, |d| <= 2, of a in [0, n), n >= 4.
__device__ __forceinline__ int wrap2(int a, int d, int n) {
    const int b = a + d;
    return b < 0 ? b + n : (b >= n ? b - n : b);
}

template <typename TS, typename TC, typename I = long long, int SM = kStreamCfl1>
__device__ __forceinline__ void gather_node(const TS *__restrict__ qin, const StepParams &p, int x, int y,
                                            TC (&q)[NC]) {
    I rowoff[5], cols[5];
    static_for<0, 5>([&](auto D) {
        constexpr int d = decltype(D)::value - 2;
        if constexpr (SM == kStreamHalo2 || (d >= -1 && d <= 1)) {
            rowoff[d + 2] = (I)wrap2(y, d, p.ny) * (I)p.pitch;
            cols[d + 2] = (I)wrap2(x, d, p.nx);
        } else {
            rowoff[d + 2] = 0;  // not referenced below CFL 1
            cols[d + 2] = 0;
        }
    });
    const I plane = (I)p.plane;
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        q[c] = gather_class<c, TS, TC, I, SM>(qin, (I)c * plane, rowoff, cols, p);
    });
}

template <typename TS, typename TC, typename TL, bool FORCED, typename I, int SM>
__global__ void __launch_bounds__(256) k_step_gather(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                     const TC *__restrict__ F, StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    TC q[NC];
    gather_node<TS, TC, I, SM>(qin, p, x, y, q);
    const I n = (I)y * (I)p.pitch + (I)x;
    const I plane = (I)p.plane;
    TC Fx = 0, Fy = 0;
    if constexpr (FORCED) {
        Fx = __ldg(F + n);
        Fy = __ldg(F + (plane + n));
    }
    collide_node<TC, TL, FORCED>(q, Fx, Fy, p);
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        qout[(I)c * plane + n] = to_storage<TS, TC>(q[c]);
    });
}

// Moments of the state the next collision sees: eps, v (FP64, compact
// nx*ny), and per-block FP64 partial sums of (T^00, T^0x, T^0y) for the
// global conservation totals (warp shuffles, then one partial per block in
// `partials`, reduced in a fixed order by k_reduce_partials).  The frame is
// FP64-accurate: TL = double solves it by FP64 Newton; TL = float (the FP32
// and 16-bit forms, whose moments are FP32 sums) solves it by FP32 Newton
// refined by one double-float Newton step (landau_refine_df), and forms
// eps and v from the refined pairs in FP64.
template <typename TS, typename TC, typename TL, int SM>
__global__ void __launch_bounds__(256) k_moments(const TS *__restrict__ qin, StepParams p, double *__restrict__ eps,
                                                 double *__restrict__ vx, double *__restrict__ vy,
                                                 double *__restrict__ partials, int *__restrict__ bad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double sE = 0.0, sMx = 0.0, sMy = 0.0;
    if (x < p.nx && y < p.ny) {
        TC q[NC];
        gather_node<TS, TC, long long, SM>(qin, p, x, y, q);
        const NodeMoments<TC> m = node_moments<TC>(q, par_scale<TC>(p));
        double e64, vx64, vy64;
        bool ok;
        if constexpr (std::is_same<TL, float>::value) {
            float delta;
            Frame<float> fr = landau_solve<float>(p.eps0_f, m.dE, m.Mx, m.My, m.dSxx, m.dSxy, m.dSyy, 4.0 / 3.0,
                                                  &delta);
            FramePairs<float> pr;
            landau_refine_df<float>(p.alpha_hi_f, p.alpha_lo_f, p.eps0_f, m.dE, m.Mx, m.My, m.dSxx, m.dSxy, m.dSyy,
                                    delta, fr, &pr);
            // one refinement squares the FP32 solve's relative error (a few ulp, about 1e-13 after);
            // close to the light cone (|v| above about 0.95) the FP32 solve is off by more than
            // 1e-6 and the refined frame would be too: solve those nodes by FP64 Newton instead
            const float tol = 1e-6f;
            const bool fine = fabsf(pr.delta_lo) <= tol * fabsf(pr.delta_hi) + 1e-30f &&
                              fabsf(pr.vx_lo) + fabsf(pr.vy_lo) <= tol * (fabsf(pr.vx_hi) + fabsf(pr.vy_hi)) + 1e-30f;
            if (fine) {
                e64 = p.eps0 + ((double)m.dE - ((double)pr.delta_hi + (double)pr.delta_lo));
                vx64 = (double)pr.vx_hi + (double)pr.vx_lo;
                vy64 = (double)pr.vy_hi + (double)pr.vy_lo;
            } else {
                const Frame<double> f64 = landau_solve<double>(p.eps0, (double)m.dE, (double)m.Mx, (double)m.My,
                                                               (double)m.dSxx, (double)m.dSxy, (double)m.dSyy);
                e64 = f64.eps;
                vx64 = f64.vx;
                vy64 = f64.vy;
            }
            ok = (fmadd(vx64, vx64, vy64 * vy64) < 1.0) && (e64 > 0.0) && isfinite(e64) && isfinite(vx64) &&
                 isfinite(vy64);
        } else {
            const Frame<TL> fr = landau_solve<TL>(par_eps0<TL>(p), (TL)m.dE, (TL)m.Mx, (TL)m.My, (TL)m.dSxx,
                                                  (TL)m.dSxy, (TL)m.dSyy);
            e64 = (double)fr.eps;
            vx64 = (double)fr.vx;
            vy64 = (double)fr.vy;
            ok = (fr.v2 < (TL)1) && (fr.eps > (TL)0) && isfinite((double)fr.eps);
        }
        const long long n = (long long)y * p.nx + x;
        if (!ok) atomicAdd(bad, 1);
        if (eps) eps[n] = ok ? e64 : __longlong_as_double(0x7ff8000000000000LL);
        if (vx) vx[n] = ok ? vx64 : __longlong_as_double(0x7ff8000000000000LL);
        if (vy) vy[n] = ok ? vy64 : __longlong_as_double(0x7ff8000000000000LL);
        sE = (double)m.dE;  // eps0 * nodes is added on the host side of the reduction
        sMx = (double)m.Mx;
        sMy = (double)m.My;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sE += __shfl_down_sync(0xffffffffu, sE, o);
        sMx += __shfl_down_sync(0xffffffffu, sMx, o);
        sMy += __shfl_down_sync(0xffffffffu, sMy, o);
    }
    __shared__ double red[3][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        red[0][warp] = sE;
        red[1][warp] = sMx;
        red[2][warp] = sMy;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x * blockDim.y + 31) >> 5;
        double a = lane < nw ? red[0][lane] : 0.0;
        double b = lane < nw ? red[1][lane] : 0.0;
        double c = lane < nw ? red[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
            c += __shfl_down_sync(0xffffffffu, c, o);
        }
        if (lane == 0) {
            const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
            partials[3 * blk + 0] = a;
            partials[3 * blk + 1] = b;
            partials[3 * blk + 2] = c;
        }
    }
}

}  // namespace rlbk
