// k_lattice3d.cuh -- the paper's node on a three-dimensional periodic lattice
// (the three-dimensional model its conclusion names as the next test): all
// 26 directions of the spherical rule stored (no merging), pull-streaming
// with trilinear interpolation from x - v_i (Sec. 3.2's linear interpolation
// in 3D, CFL 1), moments with the full in-space tensors, the Landau frame as
// a 3x3 problem, and the same equilibrium, relaxation and driving term as the
// one-layer lattice (collide_node in rlbm_device.cuh) without the z-mirror
// reductions.
//
// Direction order on the device: k = 0..12 and k + 13 = its opposite:
//   0..2   faces (1,0,0), (0,1,0), (0,0,1)                     W = 1/21
//   3..8   edges (a,a,0), (a,-a,0), (a,0,a), (a,0,-a),
//                (0,a,a), (0,a,-a), a = 1/sqrt2                W = 4/105
//   9..12  corners (b,b,b), (b,b,-b), (b,-b,b), (b,-b,-b),
//                b = 1/sqrt3                                   W = 9/280
// Stored value q_k = (f_k - W_k eps0) / (W_k s); layout q[k][z][y][pitch].
#pragma once

#include "forcing.cuh"
#include "k_step_vec.cuh"
#include "packed.cuh"
#include "rlbm_device.cuh"

namespace rlbk {

constexpr int N3 = 26;
constexpr int NP3 = 13;

RLBM_HD constexpr double d3c(int k, int axis) {
    // components of the first 13 directions; the rest are their negatives
    constexpr double a = kA, b = 0.57735026918962576451;
    const int j = k < NP3 ? k : k - NP3;
    const double sgn = k < NP3 ? 1.0 : -1.0;
    double v = 0.0;
    switch (j) {
    case 0: v = axis == 0 ? 1.0 : 0.0; break;
    case 1: v = axis == 1 ? 1.0 : 0.0; break;
    case 2: v = axis == 2 ? 1.0 : 0.0; break;
    case 3: v = axis == 0 ? a : axis == 1 ? a : 0.0; break;
    case 4: v = axis == 0 ? a : axis == 1 ? -a : 0.0; break;
    case 5: v = axis == 0 ? a : axis == 2 ? a : 0.0; break;
    case 6: v = axis == 0 ? a : axis == 2 ? -a : 0.0; break;
    case 7: v = axis == 1 ? a : axis == 2 ? a : 0.0; break;
    case 8: v = axis == 1 ? a : axis == 2 ? -a : 0.0; break;
    case 9: v = b; break;
    case 10: v = axis == 2 ? -b : b; break;
    case 11: v = axis == 1 ? -b : b; break;
    default: v = axis == 0 ? b : -b; break;
    }
    return sgn * v;
}
RLBM_HD constexpr double d3w(int k) {
    const int j = k < NP3 ? k : k - NP3;
    return j < 3 ? 1.0 / 21.0 : j < 9 ? 4.0 / 105.0 : 9.0 / 280.0;
}
// pull source x - v: corner offset floor(-c) and fractional part per axis
RLBM_HD constexpr int d3o(int k, int axis) { return floor_int(-d3c(k, axis)); }
RLBM_HD constexpr double d3t(int k, int axis) { return -d3c(k, axis) - (double)d3o(k, axis); }

// Neighbour offsets of a node: zoff/yoff/cols[0..2] = z-1, z, z+1 (periodic)
// as element offsets of the slab, row and column.
template <typename I>
struct Nbr3 {
    I zoff[3], yoff[3], cols[3];
};

template <typename I>
__device__ __forceinline__ Nbr3<I> nbr3(const StepParams &p, int x, int y, int z) {
    Nbr3<I> n;
    const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
    const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
    const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
    n.zoff[0] = (I)zm * (I)p.slab;
    n.zoff[1] = (I)z * (I)p.slab;
    n.zoff[2] = (I)zp * (I)p.slab;
    n.yoff[0] = (I)ym * (I)p.pitch;
    n.yoff[1] = (I)y * (I)p.pitch;
    n.yoff[2] = (I)yp * (I)p.pitch;
    n.cols[0] = (I)xm;
    n.cols[1] = (I)x;
    n.cols[2] = (I)xp;
    return n;
}

// Trilinear pull of direction k (1, 2, 4 or 8 sources, weights fixed at
// compile time).
template <int k, typename TS, typename TC, typename I>
__device__ __forceinline__ TC gather3(const TS *__restrict__ qin, I base, const Nbr3<I> &nb) {
    constexpr int ox = d3o(k, 0), oy = d3o(k, 1), oz = d3o(k, 2);
    constexpr double tx = d3t(k, 0), ty = d3t(k, 1), tz = d3t(k, 2);
    TC v = 0;
    static_for<0, 8>([&](auto D) {
        constexpr int d = decltype(D)::value;
        constexpr int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
        constexpr double w = (dx ? tx : 1.0 - tx) * (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
        if constexpr (w != 0.0) {
            const I off = base + nb.zoff[oz + 1 + dz] + nb.yoff[oy + 1 + dy] + nb.cols[ox + 1 + dx];
            if constexpr (w == 1.0) v = load_q<TS, TC>(qin + off);
            else v = fmadd((TC)w, load_q<TS, TC>(qin + off), v);
        }
    });
    return v;
}

template <typename TS, typename TC, typename I>
__device__ __forceinline__ void gather3_node(const TS *__restrict__ qin, const StepParams &p, int x, int y, int z,
                                             TC (&q)[N3]) {
    const Nbr3<I> nb = nbr3<I>(p, x, y, z);
    const I plane = (I)p.plane;
    static_for<0, N3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        q[k] = gather3<k, TS, TC, I>(qin, (I)k * plane, nb);
    });
}

// Moments of the post-stream node in deviation form (the 3D counterpart of
// node_moments): dE = s sum W q, M = s sum W q c, dS = s sum W q c c,
// Q = s sum W q c c c, over the 13 opposite pairs (sum for even moments,
// difference for odd ones).
template <typename TC>
struct Moments3 {
    TC dE, M[3], dS[6], Q[10];  // dS: xx yy zz xy xz yz; Q: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
};

RLBM_HD constexpr int sym2(int a, int b) {
    return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
}
// index of Q^{abc} (a <= b <= c) in the list above
RLBM_HD constexpr int sym3(int a, int b, int c) {
    return a == 0 ? (b == 0 ? c : (b == 1 ? 2 + c : 5)) : (a == 1 ? (b == 1 ? 5 + c : 8) : 9);
}

template <typename TC>
__device__ __forceinline__ Moments3<TC> moments3(const TC (&q)[N3], TC s) {
    Moments3<TC> m;
    TC e = 0, M[3] = {0, 0, 0}, S[6] = {0, 0, 0, 0, 0, 0}, Q[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    static_for<0, NP3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        constexpr double w = d3w(k);
        const TC sp = q[k] + q[k + NP3];
        const TC dp = q[k] - q[k + NP3];
        e = fmadd((TC)w, sp, e);
        static_for<0, 3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            constexpr double ca = d3c(k, a);
            if constexpr (ca != 0.0) {
                M[a] = fmadd((TC)(w * ca), dp, M[a]);
                static_for<a, 3>([&](auto B) {
                    constexpr int b = decltype(B)::value;
                    constexpr double cb = d3c(k, b);
                    if constexpr (cb != 0.0) {
                        S[sym2(a, b)] = fmadd((TC)(w * ca * cb), sp, S[sym2(a, b)]);
                        static_for<b, 3>([&](auto C) {
                            constexpr int c = decltype(C)::value;
                            constexpr double cc = d3c(k, c);
                            if constexpr (cc != 0.0)
                                Q[sym3(a, b, c)] = fmadd((TC)(w * ca * cb * cc), dp, Q[sym3(a, b, c)]);
                        });
                    }
                });
            }
        });
    });
    m.dE = s * e;
    for (int a = 0; a < 3; ++a) m.M[a] = s * M[a];
    for (int i = 0; i < 6; ++i) m.dS[i] = s * S[i];
    for (int i = 0; i < 10; ++i) m.Q[i] = s * Q[i];
    return m;
}

// Landau frame in 3D: (S + eps I) v = M, delta = E - eps = M . v, solved as
// in landau_solve (Newton on delta from the series start, fast reciprocals
// inside the iteration, correctly rounded ones for the final frame), with
// the 3x3 symmetric system solved by its adjugate.
template <typename TL>
struct Frame3 {
    TL ddelta_eps, eps, v[3], v2, g2, gamma;
};

template <typename TL>
__device__ __forceinline__ Frame3<TL> landau3(TL eps0, TL dE, const TL (&M)[3], const TL (&dS)[6]) {
    const TL a0 = (TL)(4.0 / 3.0) * eps0 + dE;
    constexpr bool dbl = std::is_same<TL, double>::value;
    const TL tol = dbl ? (TL)4e-16 : (TL)1e-7;
    TL v[3];
    auto velocity = [&](TL d, bool exact) {
        const TL a = a0 - d;
        const TL b00 = a + dS[0], b11 = a + dS[1], b22 = a + dS[2];
        const TL b01 = dS[3], b02 = dS[4], b12 = dS[5];
        const TL c00 = b11 * b22 - b12 * b12, c01 = b02 * b12 - b01 * b22, c02 = b01 * b12 - b02 * b11;
        const TL c11 = b00 * b22 - b02 * b02, c12 = b01 * b02 - b00 * b12, c22 = b00 * b11 - b01 * b01;
        const TL det = b00 * c00 + b01 * c01 + b02 * c02;
        const TL inv = exact ? frame_recip(det) : fast_recip(det);
        v[0] = (c00 * M[0] + c01 * M[1] + c02 * M[2]) * inv;
        v[1] = (c01 * M[0] + c11 * M[1] + c12 * M[2]) * inv;
        v[2] = (c02 * M[0] + c12 * M[1] + c22 * M[2]) * inv;
    };
    velocity((TL)0, false);
    const TL m1 = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
    const TL m2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    TL delta = m1 * fast_recip((TL)1 - m2);
    TL step = 0;
    auto newton = [&]() {
        velocity(delta, false);
        const TL g = delta - (M[0] * v[0] + M[1] * v[1] + M[2] * v[2]);
        const TL gp = (TL)1 - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        step = g * fast_recip(gp);
        delta = delta - step;
    };
    newton();
    for (int it = 1; it < (dbl ? 24 : 12); ++it) {
        if (!(step * step > tol * absval(delta))) break;
        newton();
    }
    velocity(delta, true);
    Frame3<TL> fr;
    fr.ddelta_eps = dE - delta;
    fr.eps = eps0 + fr.ddelta_eps;
    for (int a = 0; a < 3; ++a) fr.v[a] = v[a];
    fr.v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if constexpr (is_f32_lane<TL>::value) {
        fr.gamma = frame_rsqrt((TL)1 - fr.v2);
        fr.g2 = fr.gamma * fr.gamma;
    } else {
        fr.g2 = recip((TL)1 - fr.v2);
        fr.gamma = sqrt_(fr.g2);
    }
    return fr;
}

// Collision of one 3D node in place (the same equilibrium, Anderson-Witting
// rate and driving term as collide_node, with every tensor component kept):
// per direction q' = q (1 - om + om xi) + om (1 - xi) q_eq + G / (W s),
// even part K0 + K_ab c_a c_b, odd part xi (o1 - om P2 xi^2) + G1 (F . c).
template <typename TC, typename TL, bool FORCED>
__device__ __forceinline__ Frame3<TL> collide3(TC (&q)[N3], const TC (&F)[3], const StepParams &p) {
    const TC s = par_scale<TC>(p);
    const Moments3<TC> m = moments3<TC>(q, s);
    const TL Ml[3] = {(TL)m.M[0], (TL)m.M[1], (TL)m.M[2]};
    const TL Sl[6] = {(TL)m.dS[0], (TL)m.dS[1], (TL)m.dS[2], (TL)m.dS[3], (TL)m.dS[4], (TL)m.dS[5]};
    const Frame3<TL> fr = landau3<TL>(par_eps0<TL>(p), (TL)m.dE, Ml, Sl);
    const TC inv_s = par_inv_scale<TC>(p);
    const TL eg2 = fr.eps * fr.g2;
    const TC P0 = (TC)(fmadd((TL)(-2) * eg2, fr.v2, fr.ddelta_eps)) * inv_s;
    const TC P1 = (TC)((TL)4 * eg2) * inv_s;
    const TC P2 = (TC)((TL)10 * eg2) * inv_s;
    const TC v[3] = {(TC)fr.v[0], (TC)fr.v[1], (TC)fr.v[2]};
    TL inv_tau = par_inv_tau<TL>(p);
    if (p.eta_k_f > 0.0f) inv_tau = par_eta_k<TL>(p) * sqrt_(sqrt_(fr.eps));
    const TC om = (TC)(fr.gamma * inv_tau);
    const TC e2 = om * (P2 - P1);
    // K[sym2(a, b)]: coefficient of c_a c_b (a < b terms carry both orders)
    TC K[6];
    for (int a = 0; a < 3; ++a) K[a] = e2 * v[a] * v[a];
    K[3] = (TC)2 * e2 * v[0] * v[1];
    K[4] = (TC)2 * e2 * v[0] * v[2];
    K[5] = (TC)2 * e2 * v[1] * v[2];
    TC K0 = om * P0;
    const TC o1 = om * (P1 - P0), no3 = (TC)0 - om * P2;
    TC G1 = 0;
    if constexpr (FORCED) {
        const TC E = par_eps0<TC>(p) + m.dE;
        const TC c6 = (TC)(-6.0) * inv_s;
        const TC FM = F[0] * m.M[0] + F[1] * m.M[1] + F[2] * m.M[2];
        K0 = K0 + c6 * (TC)0.25 * FM;
        G1 = c6 * (TC)(-0.5) * E;
        const TC G3 = c6 * (TC)(-2.5);
        const TC c54 = c6 * (TC)1.25;
        // (F.c)(c.M) = F_a M_b c_a c_b ; F_a c_b c_c Q^abc = P_bc c_b c_c, P_bc = F_a Q^abc
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = b; c < 3; ++c) {
                const int i = sym2(b, c);
                TC Pbc = 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int lo = a, mid = b, hi = c;  // sort (a, b, c)
                    if (lo > mid) { int t = lo; lo = mid; mid = t; }
                    if (mid > hi) { int t = mid; mid = hi; hi = t; }
                    if (lo > mid) { int t = lo; lo = mid; mid = t; }
                    Pbc = fmadd(F[a], m.Q[sym3(lo, mid, hi)], Pbc);
                }
                const TC FMbc = (b == c) ? F[b] * m.M[b] : F[b] * m.M[c] + F[c] * m.M[b];
                K[i] = fmadd(G3, FMbc, fmadd(c54 * (b == c ? (TC)1 : (TC)2), Pbc, K[i]));
            }
    }
    const TC a0 = (TC)1 - om;
    static_for<0, NP3>([&](auto Kk) {
        constexpr int k = decltype(Kk)::value;
        constexpr double cx = d3c(k, 0), cy = d3c(k, 1), cz = d3c(k, 2);
        TC xi = 0, even = K0;
        [[maybe_unused]] TC Fc = 0;
        if constexpr (cx != 0.0) {
            xi = fmadd((TC)cx, v[0], xi);
            even = fmadd((TC)(cx * cx), K[0], even);
            if constexpr (FORCED) Fc = fmadd((TC)cx, F[0], Fc);
        }
        if constexpr (cy != 0.0) {
            xi = fmadd((TC)cy, v[1], xi);
            even = fmadd((TC)(cy * cy), K[1], even);
            if constexpr (FORCED) Fc = fmadd((TC)cy, F[1], Fc);
        }
        if constexpr (cz != 0.0) {
            xi = fmadd((TC)cz, v[2], xi);
            even = fmadd((TC)(cz * cz), K[2], even);
            if constexpr (FORCED) Fc = fmadd((TC)cz, F[2], Fc);
        }
        if constexpr (cx != 0.0 && cy != 0.0) even = fmadd((TC)(cx * cy), K[3], even);
        if constexpr (cx != 0.0 && cz != 0.0) even = fmadd((TC)(cx * cz), K[4], even);
        if constexpr (cy != 0.0 && cz != 0.0) even = fmadd((TC)(cy * cz), K[5], even);
        TC odd = xi * fmadd(no3, xi * xi, o1);
        if constexpr (FORCED) odd = fmadd(G1, Fc, odd);
        const TC oxi = om * xi;
        const TC qp = q[k], qn = q[k + NP3];
        q[k] = fmadd(qp, a0 + oxi, even + odd);
        q[k + NP3] = fmadd(qn, a0 - oxi, even - odd);
    });
    return fr;
}

// Fused 3D step, one node per thread; block (bx, by), grid (x, y, z).
template <typename TS, typename TC, typename TL, bool FORCED, typename I>
__global__ void __launch_bounds__(256) k_step3(const TS *__restrict__ qin, TS *__restrict__ qout,
                                               const TC *__restrict__ F, StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    TC q[N3];
    gather3_node<TS, TC, I>(qin, p, x, y, z, q);
    const I n = (I)z * (I)p.slab + (I)y * (I)p.pitch + (I)x;
    TC Fv[3] = {0, 0, 0};
    if constexpr (FORCED) {
        Fv[0] = __ldg(F + n);
        Fv[1] = __ldg(F + ((I)p.plane + n));
        Fv[2] = __ldg(F + ((I)2 * (I)p.plane + n));
    }
    collide3<TC, TL, FORCED>(q, Fv, p);
    static_for<0, N3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        qout[(I)k * (I)p.plane + n] = to_storage<TS, TC>(q[k]);
    });
}

// Packed-lane form of k_step3: two x-adjacent nodes per thread whose whole
// arithmetic runs in pairs of FP32 lanes (packed.cuh), one instruction per
// operation for both nodes.  Each source row of a direction is read once
// for the pair: columns x0-1 .. x0+2 as the direction's x corner needs.
template <int ox, bool TXNZ, typename TS, typename I>
__device__ __forceinline__ void load_row_pair(const TS *__restrict__ row, int x0, int xl, int xr, float (&a)[4]) {
    load_run<TS, float, 2>(row + x0, &a[1]);
    if constexpr (ox == -1) a[0] = load_q<TS, float>(row + xl);
    if constexpr (ox == 1 || (ox == 0 && TXNZ)) a[3] = load_q<TS, float>(row + xr);
}

template <int k, typename TS, typename I>
__device__ __forceinline__ pf2 gather3_pair(const TS *__restrict__ qin, I base, const I (&zoff)[3], const I (&yoff)[3],
                                            int x0, int xl, int xr) {
    constexpr int ox = d3o(k, 0), oy = d3o(k, 1), oz = d3o(k, 2);
    constexpr double tx = d3t(k, 0), ty = d3t(k, 1), tz = d3t(k, 2);
    pf2 v = 0.0f;
    static_for<0, 4>([&](auto D) {
        constexpr int d = decltype(D)::value;
        constexpr int dy = d & 1, dz = (d >> 1) & 1;
        constexpr double wyz = (dy ? ty : 1.0 - ty) * (dz ? tz : 1.0 - tz);
        if constexpr (wyz != 0.0) {
            float a[4];
            load_row_pair<ox, tx != 0.0, TS, I>(qin + (base + zoff[oz + 1 + dz] + yoff[oy + 1 + dy]), x0, xl, xr, a);
            v = fmadd(pf2((float)(wyz * (1.0 - tx))), pf2(a[ox + 1], a[ox + 2]), v);
            if constexpr (tx != 0.0) v = fmadd(pf2((float)(wyz * tx)), pf2(a[ox + 2], a[ox + 3]), v);
        }
    });
    return v;
}

// MINB: minimum resident 256-thread blocks per SM asked of the register
// allocator (1: unconstrained; 2: at most 128 registers per thread).
template <typename TS, bool FORCED, typename I, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step3_pair(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                          const float *__restrict__ F, StepParams p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x0 >= p.nx || y >= p.ny) return;
    const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
    const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
    const int xl = x0 == 0 ? p.nx - 1 : x0 - 1, xr = x0 + 2 == p.nx ? 0 : x0 + 2;
    const I zoff[3] = {(I)zm * (I)p.slab, (I)z * (I)p.slab, (I)zp * (I)p.slab};
    const I yoff[3] = {(I)ym * (I)p.pitch, (I)y * (I)p.pitch, (I)yp * (I)p.pitch};
    pf2 q[N3];
    static_for<0, N3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        q[k] = gather3_pair<k, TS, I>(qin, (I)k * (I)p.plane, zoff, yoff, x0, xl, xr);
    });
    const I n0 = zoff[1] + yoff[1] + (I)x0;
    pf2 Fv[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (FORCED) {
        static_for<0, 3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            float f2[2];
            load_run<float, float, 2>(F + ((I)a * (I)p.plane + n0), f2);
            Fv[a] = pf2(f2[0], f2[1]);
        });
    }
    collide3<pf2, pf2, FORCED>(q, Fv, p);
    static_for<0, N3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        const float out[2] = {q[k].v.x, q[k].v.y};
        store_run<TS, float, 2>(qout + ((I)k * (I)p.plane + n0), out);
    });
}

// Moments of the state the next collision sees (FP64 frame): eps, v
// (compact [z][y][x]) and per-block partial sums of (T^00, T^0x, T^0y, T^0z).
template <typename TS, typename TC>
__global__ void __launch_bounds__(256) k_moments3(const TS *__restrict__ qin, StepParams p, double *__restrict__ eps,
                                                  double *__restrict__ vx, double *__restrict__ vy,
                                                  double *__restrict__ vz, double *__restrict__ partials,
                                                  int *__restrict__ bad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (x < p.nx && y < p.ny) {
        TC q[N3];
        gather3_node<TS, TC, long long>(qin, p, x, y, z, q);
        const Moments3<TC> m = moments3<TC>(q, par_scale<TC>(p));
        const double Ml[3] = {(double)m.M[0], (double)m.M[1], (double)m.M[2]};
        const double Sl[6] = {(double)m.dS[0], (double)m.dS[1], (double)m.dS[2],
                              (double)m.dS[3], (double)m.dS[4], (double)m.dS[5]};
        const Frame3<double> fr = landau3<double>(p.eps0, (double)m.dE, Ml, Sl);
        const long long n = ((long long)z * p.ny + y) * p.nx + x;
        const bool ok = (fr.v2 < 1.0) && (fr.eps > 0.0) && isfinite(fr.eps);
        if (!ok) atomicAdd(bad, 1);
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        if (eps) eps[n] = ok ? fr.eps : nan;
        if (vx) vx[n] = ok ? fr.v[0] : nan;
        if (vy) vy[n] = ok ? fr.v[1] : nan;
        if (vz) vz[n] = ok ? fr.v[2] : nan;
        acc[0] = (double)m.dE;
        for (int a = 0; a < 3; ++a) acc[a + 1] = Ml[a];
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int i = 0; i < 4; ++i) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], o);
    __shared__ double red[4][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
        for (int i = 0; i < 4; ++i) red[i][warp] = acc[i];
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x * blockDim.y + 31) >> 5;
        double r[4];
        for (int i = 0; i < 4; ++i) r[i] = lane < nw ? red[i][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1)
            for (int i = 0; i < 4; ++i) r[i] += __shfl_down_sync(0xffffffffu, r[i], o);
        if (lane == 0) {
            const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            for (int i = 0; i < 4; ++i) partials[4 * blk + i] = r[i];
        }
    }
}

// f_eq of the given fields in deviation form:
// q_k = [eps - eps0 + eps gamma^2 (4 xi + 10 xi^2 - 2 |v|^2)] / s, xi = c_k . v.
template <typename TS, typename TC>
__global__ void k_init3(TS *q, StepParams p, const double *eps, const double *vx, const double *vy,
                        const double *vz) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long i = ((long long)z * p.ny + y) * p.nx + x;
    const TC de = eps ? (TC)(eps[i] - p.eps0) : (TC)0;
    const TC e = par_eps0<TC>(p) + de;
    const TC a = vx ? (TC)vx[i] : (TC)0, b = vy ? (TC)vy[i] : (TC)0, c = vz ? (TC)vz[i] : (TC)0;
    const TC v2 = a * a + b * b + c * c;
    const TC eg2 = e / ((TC)1 - v2);
    const TC inv_s = par_inv_scale<TC>(p);
    const long long n = (long long)z * p.slab + (long long)y * p.pitch + x;
    static_for<0, N3>([&](auto K) {
        constexpr int k = decltype(K)::value;
        const TC xi = (TC)d3c(k, 0) * a + (TC)d3c(k, 1) * b + (TC)d3c(k, 2) * c;
        const TC qk = (de + eg2 * ((TC)4 * xi + (TC)10 * xi * xi - (TC)2 * v2)) * inv_s;
        q[(long long)k * p.plane + n] = to_storage<TS, TC>(qk);
    });
}

// ---------------------------------------------------------------- 3D stirring
// Mode m (host-enumerated integer k on the 3D shell) of epoch e draws
// Philox({e, m, 0, 0}) -> r, phi and Philox({e, m, 1, 0}) -> azimuth, mu;
// direction (sqrt(1 - mu^2) cos az, sqrt(1 - mu^2) sin az, mu).  Stored per
// mode: A_a cos(phi) and A_a sin(phi) with A = 2 r amp d, so that
// F_a(x) = sum_m A_a cos(psi + phi) = sum_m [A_a cos phi cos psi - A_a sin phi sin psi].
struct Mode3 {
    int kx, ky, kz;
};

template <typename TC>
struct C6 {
    TC ac[3], as[3];
};

template <typename TC>
__global__ void k_draw_modes3(const Mode3 *__restrict__ modes, C6<TC> *coef, int nmodes, double amp,
                              unsigned long long seed, unsigned long long epoch) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmodes) return;
    const unsigned int k0 = (unsigned int)(seed & 0xffffffffull), k1 = (unsigned int)(seed >> 32);
    const U4 o0 = philox4x32_10(U4{{(unsigned int)epoch, (unsigned int)m, 0u, 0u}}, k0, k1);
    const U4 o1 = philox4x32_10(U4{{(unsigned int)epoch, (unsigned int)m, 1u, 0u}}, k0, k1);
    const double r = amp * u01_53(o0.w[0], o0.w[1]);
    const double ph = 2.0 * M_PI * u01_53(o0.w[2], o0.w[3]);
    const double az = 2.0 * M_PI * u01_53(o1.w[0], o1.w[1]);
    const double mu = 2.0 * u01_53(o1.w[2], o1.w[3]) - 1.0;
    const double sn = sqrt(1.0 - mu * mu);
    double saz, caz, sph, cph;
    sincos(az, &saz, &caz);
    sincos(ph, &sph, &cph);
    const double d[3] = {sn * caz, sn * saz, mu};
    C6<TC> c;
    for (int a = 0; a < 3; ++a) {
        c.ac[a] = (TC)(2.0 * r * d[a] * cph);
        c.as[a] = (TC)(2.0 * r * d[a] * sph);
    }
    coef[m] = c;
}

// Per-mode phase tables along one axis: T[m][i] = e^{2 pi i k_m i / n}, the
// phase index reduced in integers.
template <typename TC>
__global__ void k_mode_tables3(C2<TC> *T, const Mode3 *__restrict__ modes, int nmodes, const C2<TC> *__restrict__ tw,
                               int n, int axis) {
    const int m = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmodes || i >= n) return;
    const int km = axis == 0 ? modes[m].kx : axis == 1 ? modes[m].ky : modes[m].kz;
    const long long k = ((long long)km % n + n) % n;
    T[(long long)m * n + i] = tw[(k * i) % n];
}

template <typename TC>
__global__ void k_synth_force3(TC *F, const C6<TC> *__restrict__ coef, int nmodes, const C2<TC> *__restrict__ X,
                               const C2<TC> *__restrict__ Y, const C2<TC> *__restrict__ Z, StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    TC f[3] = {0, 0, 0};
    for (int m = 0; m < nmodes; ++m) {
        const C6<TC> c = coef[m];
        const C2<TC> a = X[(long long)m * p.nx + x];
        const C2<TC> b = Y[(long long)m * p.ny + y];
        const C2<TC> g = Z[(long long)m * p.nz + z];
        const TC cxy = a.c * b.c - a.s * b.s;
        const TC sxy = a.s * b.c + a.c * b.s;
        const TC cp = cxy * g.c - sxy * g.s;
        const TC sp = sxy * g.c + cxy * g.s;
        for (int k = 0; k < 3; ++k) f[k] += c.ac[k] * cp - c.as[k] * sp;
    }
    const long long n = (long long)z * p.slab + (long long)y * p.pitch + x;
    for (int k = 0; k < 3; ++k) F[(long long)k * p.plane + n] = f[k];
}

}  // namespace rlbk
