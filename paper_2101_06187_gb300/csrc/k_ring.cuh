// k_ring.cuh -- the genuinely two-dimensional massless variant: momenta in
// the plane on an 8-direction ring (v_k at 45 degree steps, weight 1/8),
// ideal-gas pressure P = eps/2, sound speed c_s^2 = 1/2.  Same step as the
// spherical node (pull-stream with bilinear interpolation, moments, Landau
// frame, truncated equilibrium, Anderson-Witting relaxation, driving term),
// with the circle's angular polynomials P^(0) = 1, P^(1) = v,
// P^(2) = v v - I/2 (norms 1, 2, 4):
//   f_eq,k = W eps [1 + gamma^2 (3 xi + 6 xi^2 - 3/2 |v|^2)],  xi = v_k . v,
//   G_k = W [-F.M + 2 E (F.v_k) + 8 (F.v_k)(v_k.M) - 4 F_a v_k^b v_k^c Q^abc],
// the projection carrying sum G = F.M, sum G v = F E, sum G v v = F M + M F -
// F.Q.  Stored as q_k = (f_k - W eps0) / (W s).
#pragma once

#include "k_step_vec.cuh"
#include "packed.cuh"
#include "rlbm_device.cuh"

namespace rlbk {

constexpr int NR = 8;
constexpr double kRingW = 1.0 / 8.0;

RLBM_HD constexpr double ring_cx(int k) {
    return k == 0 ? 1.0 : k == 1 ? kA : k == 2 ? 0.0 : k == 3 ? -kA : k == 4 ? -1.0 : k == 5 ? -kA : k == 6 ? 0.0 : kA;
}
RLBM_HD constexpr double ring_cy(int k) {
    return k == 0 ? 0.0 : k == 1 ? kA : k == 2 ? 1.0 : k == 3 ? kA : k == 4 ? 0.0 : k == 5 ? -kA : k == 6 ? -1.0 : -kA;
}
RLBM_HD constexpr int ring_ox(int k) { return floor_int(-ring_cx(k)); }
RLBM_HD constexpr int ring_oy(int k) { return floor_int(-ring_cy(k)); }
RLBM_HD constexpr double ring_tx(int k) { return -ring_cx(k) - (double)ring_ox(k); }
RLBM_HD constexpr double ring_ty(int k) { return -ring_cy(k) - (double)ring_oy(k); }

template <int k, typename TS, typename TC>
__device__ __forceinline__ TC ring_gather(const TS *__restrict__ qin, int cbase, const int (&rowoff)[3],
                                          const int (&cols)[3]) {
    constexpr int ox = ring_ox(k), oy = ring_oy(k);
    constexpr double tx = ring_tx(k), ty = ring_ty(k);
    const int r0 = cbase + rowoff[oy + 1];
    TC v = (TC)((1.0 - tx) * (1.0 - ty)) * load_q<TS, TC>(qin + (r0 + cols[ox + 1]));
    if constexpr (tx != 0.0) v += (TC)(tx * (1.0 - ty)) * load_q<TS, TC>(qin + (r0 + cols[ox + 2]));
    if constexpr (ty != 0.0) {
        const int r1 = cbase + rowoff[oy + 2];
        v += (TC)((1.0 - tx) * ty) * load_q<TS, TC>(qin + (r1 + cols[ox + 1]));
        if constexpr (tx != 0.0) v += (TC)(tx * ty) * load_q<TS, TC>(qin + (r1 + cols[ox + 2]));
    }
    return v;
}

// Ring moments (deviation form) over the 4 opposite pairs (k, k+4).
template <typename TC>
__device__ __forceinline__ NodeMoments<TC> ring_moments(const TC (&q)[NR], TC s) {
    TC e = 0, mx = 0, my = 0, sxx = 0, sxy = 0, syy = 0, qxxx = 0, qxxy = 0, qxyy = 0, qyyy = 0;
    static_for<0, 4>([&](auto K) {
        constexpr int k = decltype(K)::value;
        constexpr double w = kRingW, cx = ring_cx(k), cy = ring_cy(k);
        const TC sp = q[k] + q[k + 4];
        const TC dp = q[k] - q[k + 4];
        e = fmadd((TC)w, sp, e);
        if constexpr (cx != 0.0) {
            mx = fmadd((TC)(w * cx), dp, mx);
            sxx = fmadd((TC)(w * cx * cx), sp, sxx);
            qxxx = fmadd((TC)(w * cx * cx * cx), dp, qxxx);
        }
        if constexpr (cy != 0.0) {
            my = fmadd((TC)(w * cy), dp, my);
            syy = fmadd((TC)(w * cy * cy), sp, syy);
            qyyy = fmadd((TC)(w * cy * cy * cy), dp, qyyy);
        }
        if constexpr (cx != 0.0 && cy != 0.0) {
            sxy = fmadd((TC)(w * cx * cy), sp, sxy);
            qxxy = fmadd((TC)(w * cx * cx * cy), dp, qxxy);
            qxyy = fmadd((TC)(w * cx * cy * cy), dp, qxyy);
        }
    });
    NodeMoments<TC> m;
    m.dE = s * e;
    m.Mx = s * mx;
    m.My = s * my;
    m.dSxx = s * sxx;
    m.dSxy = s * sxy;
    m.dSyy = s * syy;
    m.Qxxx = s * qxxx;
    m.Qxxy = s * qxxy;
    m.Qxyy = s * qxyy;
    m.Qyyy = s * qyyy;
    return m;
}

// Collision of one ring node: per class q' = q (1 - om + om xi) + om (1 - xi) q_eq
// + G / (W s), split into the part even in v_k (a quadratic form) and the odd part.
template <typename TC, typename TL, bool FORCED>
__device__ __forceinline__ Frame<TL> ring_collide(TC (&q)[NR], TC Fx, TC Fy, const StepParams &p) {
    const TC s = par_scale<TC>(p);
    const NodeMoments<TC> m = ring_moments<TC>(q, s);
    const Frame<TL> fr = landau_solve<TL>(par_eps0<TL>(p), (TL)m.dE, (TL)m.Mx, (TL)m.My, (TL)m.dSxx, (TL)m.dSxy,
                                          (TL)m.dSyy, 1.5);
    const TC inv_s = par_inv_scale<TC>(p);
    const TL eg2 = fr.eps * fr.g2;
    const TC P0 = (TC)(fmadd((TL)(-1.5) * eg2, fr.v2, fr.ddelta_eps)) * inv_s;
    const TC P1 = (TC)((TL)3 * eg2) * inv_s;
    const TC P2 = (TC)((TL)6 * eg2) * inv_s;
    const TC vx = (TC)fr.vx, vy = (TC)fr.vy;
    const TC om = (TC)(fr.gamma * par_inv_tau<TL>(p));
    const TC e2 = om * (P2 - P1);
    TC K0 = om * P0, Kxx = e2 * vx * vx, Kxy = (TC)2 * e2 * vx * vy, Kyy = e2 * vy * vy;
    const TC o1 = om * (P1 - P0), no3 = (TC)0 - om * P2;
    TC G1 = 0;
    if constexpr (FORCED) {
        const TC E = par_eps0<TC>(p) + m.dE;
        const TC G0 = (TC)(-1.0) * inv_s * fmadd(Fx, m.Mx, Fy * m.My);
        G1 = (TC)2 * inv_s * E;
        const TC G3 = (TC)8 * inv_s;
        const TC c4 = (TC)(-4.0) * inv_s;
        const TC Pxx = c4 * fmadd(Fx, m.Qxxx, Fy * m.Qxxy);
        const TC Pxy = c4 * fmadd(Fx, m.Qxxy, Fy * m.Qxyy);
        const TC Pyy = c4 * fmadd(Fx, m.Qxyy, Fy * m.Qyyy);
        K0 = K0 + G0;
        Kxx = fmadd(G3 * Fx, m.Mx, Kxx + Pxx);
        Kxy = fmadd(G3, fmadd(Fx, m.My, Fy * m.Mx), Kxy + (TC)2 * Pxy);
        Kyy = fmadd(G3 * Fy, m.My, Kyy + Pyy);
    }
    const TC a0 = (TC)1 - om;
    static_for<0, 4>([&](auto K) {
        constexpr int k = decltype(K)::value;
        constexpr double cx = ring_cx(k), cy = ring_cy(k);
        TC xi = 0;
        [[maybe_unused]] TC Fc = 0;
        TC even = K0;
        if constexpr (cx != 0.0) {
            xi = (TC)cx * vx;
            even = fmadd((TC)(cx * cx), Kxx, even);
            if constexpr (FORCED) Fc = (TC)cx * Fx;
        }
        if constexpr (cy != 0.0) {
            xi = fmadd((TC)cy, vy, xi);
            even = fmadd((TC)(cy * cy), Kyy, even);
            if constexpr (FORCED) Fc = fmadd((TC)cy, Fy, Fc);
        }
        if constexpr (cx != 0.0 && cy != 0.0) even = fmadd((TC)(cx * cy), Kxy, even);
        TC odd = xi * fmadd(no3, xi * xi, o1);
        if constexpr (FORCED) odd = fmadd(G1, Fc, odd);
        const TC oxi = om * xi;
        const TC qp = q[k], qn = q[k + 4];
        q[k] = fmadd(qp, a0 + oxi, even + odd);
        q[k + 4] = fmadd(qn, a0 - oxi, even - odd);
    });
    return fr;
}

template <typename TS, typename TC>
__device__ __forceinline__ void ring_gather_node(const TS *__restrict__ qin, const StepParams &p, int x, int y,
                                                 TC (&q)[NR]) {
    const int ym = (y == 0) ? p.ny - 1 : y - 1;
    const int yp = (y == p.ny - 1) ? 0 : y + 1;
    const int xm = (x == 0) ? p.nx - 1 : x - 1;
    const int xp = (x == p.nx - 1) ? 0 : x + 1;
    const int rowoff[3] = {ym * p.pitch, y * p.pitch, yp * p.pitch};
    const int cols[3] = {xm, x, xp};
    const int plane = (int)p.plane;
    static_for<0, NR>([&](auto K) {
        constexpr int k = decltype(K)::value;
        q[k] = ring_gather<k, TS, TC>(qin, k * plane, rowoff, cols);
    });
}

// Fused ring step, one node per thread (indices fit 32 bits: 8 planes).
template <typename TS, typename TC, typename TL, bool FORCED>
__global__ void __launch_bounds__(256) k_ring_step(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                   const TC *__restrict__ F, StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    TC q[NR];
    ring_gather_node<TS, TC>(qin, p, x, y, q);
    const int n = y * p.pitch + x;
    TC Fx = 0, Fy = 0;
    if constexpr (FORCED) {
        Fx = __ldg(F + n);
        Fy = __ldg(F + ((int)p.plane + n));
    }
    ring_collide<TC, TL, FORCED>(q, Fx, Fy, p);
    static_for<0, NR>([&](auto K) {
        constexpr int k = decltype(K)::value;
        qout[k * (int)p.plane + n] = to_storage<TS, TC>(q[k]);
    });
}

// Packed-lane ring step: two x-adjacent nodes per thread in pairs of FP32
// lanes (packed.cuh); each source row of a direction is read once for the
// pair (columns x0-1 .. x0+2 as the direction needs).  nx even.
template <int k, typename TS>
__device__ __forceinline__ pf2 ring_gather_pair(const TS *__restrict__ qin, long long cbase, const long long (&rowoff)[3],
                                                int x0, int xl, int xr) {
    constexpr int ox = ring_ox(k), oy = ring_oy(k);
    constexpr double tx = ring_tx(k), ty = ring_ty(k);
    auto row = [&](const TS *r, float (&a)[4]) {
        load_run<TS, float, 2>(r + x0, &a[1]);
        if constexpr (ox == -1) a[0] = load_q<TS, float>(r + xl);
        if constexpr (ox == 1 || (ox == 0 && tx != 0.0)) a[3] = load_q<TS, float>(r + xr);
    };
    float a[4];
    row(qin + (cbase + rowoff[oy + 1]), a);
    pf2 v = pf2((float)((1.0 - tx) * (1.0 - ty))) * pf2(a[ox + 1], a[ox + 2]);
    if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * (1.0 - ty))), pf2(a[ox + 2], a[ox + 3]), v);
    if constexpr (ty != 0.0) {
        float b[4];
        row(qin + (cbase + rowoff[oy + 2]), b);
        v = fmadd(pf2((float)((1.0 - tx) * ty)), pf2(b[ox + 1], b[ox + 2]), v);
        if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * ty)), pf2(b[ox + 2], b[ox + 3]), v);
    }
    return v;
}

template <typename TS, bool FORCED>
__global__ void __launch_bounds__(256) k_ring_step_pair(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                        const float *__restrict__ F, StepParams p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
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

template <typename TS, typename TC>
__global__ void __launch_bounds__(256) k_ring_moments(const TS *__restrict__ qin, StepParams p,
                                                      double *__restrict__ eps, double *__restrict__ vx,
                                                      double *__restrict__ vy, double *__restrict__ partials,
                                                      int *__restrict__ bad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double sE = 0.0, sMx = 0.0, sMy = 0.0;
    if (x < p.nx && y < p.ny) {
        TC q[NR];
        ring_gather_node<TS, TC>(qin, p, x, y, q);
        const NodeMoments<TC> m = ring_moments<TC>(q, par_scale<TC>(p));
        const Frame<double> fr = landau_solve<double>(p.eps0, (double)m.dE, (double)m.Mx, (double)m.My,
                                                      (double)m.dSxx, (double)m.dSxy, (double)m.dSyy, 1.5);
        const long long n = (long long)y * p.nx + x;
        const bool ok = (fr.v2 < 1.0) && (fr.eps > 0.0) && isfinite(fr.eps);
        if (!ok) atomicAdd(bad, 1);
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        if (eps) eps[n] = ok ? fr.eps : nan;
        if (vx) vx[n] = ok ? fr.vx : nan;
        if (vy) vy[n] = ok ? fr.vy : nan;
        sE = (double)m.dE;
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

// f_eq of the given fields in deviation form:
// q_k = [eps - eps0 + eps gamma^2 (3 xi + 6 xi^2 - 3/2 |v|^2)] / s.
template <typename TS, typename TC>
__global__ void k_ring_init(TS *q, StepParams p, const double *eps, const double *vx, const double *vy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long i = (long long)y * p.nx + x;
    const TC de = eps ? (TC)(eps[i] - p.eps0) : (TC)0;
    const TC e = par_eps0<TC>(p) + de;
    const TC a = vx ? (TC)vx[i] : (TC)0, b = vy ? (TC)vy[i] : (TC)0;
    const TC v2 = a * a + b * b;
    const TC eg2 = e / ((TC)1 - v2);
    const TC inv_s = par_inv_scale<TC>(p);
    const long long n = (long long)y * p.pitch + x;
    static_for<0, NR>([&](auto K) {
        constexpr int k = decltype(K)::value;
        const TC xi = (TC)ring_cx(k) * a + (TC)ring_cy(k) * b;
        const TC qk = (de + eg2 * ((TC)3 * xi + (TC)6 * xi * xi - (TC)1.5 * v2)) * inv_s;
        q[(long long)k * p.plane + n] = to_storage<TS, TC>(qk);
    });
}

}  // namespace rlbk
