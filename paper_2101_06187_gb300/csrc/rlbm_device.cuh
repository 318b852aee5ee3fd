// rlbm_device.cuh -- per-node arithmetic of the RLBM stream-collide step
// (Watson, arXiv:2101.06187), shared by the fused step kernels and the
// moments kernel.
//
// Stored state: 17 in-plane classes c of the 26-direction spherical node
// (Sec. 5, "spherical D3Q27" with one lattice node in z).  A class merges
// the z-mirror pair (v_x, v_y, +v_z) / (v_x, v_y, -v_z): on a one-layer
// periodic lattice both stream by (v_x, v_y) and collide alike, so only
// their sum f_c is evolved.  Each class is stored as the scaled deviation
//     q_c = (f_c - W_c eps0) / (W_c s)
// from the rest equilibrium, which keeps the low-order digits that FP32 and
// 16-bit storage would otherwise lose to the constant W_c eps0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cmath>
#include <type_traits>

namespace rlbk {

#define RLBM_HD __host__ __device__

constexpr int NC = 17;

// 1/sqrt(2) and 1/sqrt(3): in-plane components of the edge and corner directions.
constexpr double kA = 0.70710678118654752440084436210484904;
constexpr double kB = 0.57735026918962576450914878050195746;

// Class table (in-plane velocity, merged weight W_c, v_z^2 of the class).
// Rest (0,0,+-1): W = 2 * 1/21.  Axis faces: 1/21.  (a,0)-type edges with a
// z component: 2 * 4/105.  In-plane diagonal edges: 4/105.  Corners:
// 2 * 9/280.  Sum of W = 1.
__host__ __device__ constexpr double cls_cx(int c) {
    return c == 1 ? 1.0 : c == 2 ? -1.0 : c == 5 ? kA : c == 6 ? -kA : c == 9 ? kA : c == 10 ? -kA
         : c == 11 ? kA : c == 12 ? -kA : c == 13 ? kB : c == 14 ? -kB : c == 15 ? kB : c == 16 ? -kB : 0.0;
}
__host__ __device__ constexpr double cls_cy(int c) {
    return c == 3 ? 1.0 : c == 4 ? -1.0 : c == 7 ? kA : c == 8 ? -kA : c == 9 ? kA : c == 10 ? kA
         : c == 11 ? -kA : c == 12 ? -kA : c == 13 ? kB : c == 14 ? kB : c == 15 ? -kB : c == 16 ? -kB : 0.0;
}
__host__ __device__ constexpr double cls_w(int c) {
    return c == 0 ? 2.0 / 21.0 : c <= 4 ? 1.0 / 21.0 : c <= 8 ? 8.0 / 105.0 : c <= 12 ? 4.0 / 105.0 : 9.0 / 140.0;
}
__host__ __device__ constexpr double cls_vz2(int c) {
    return c == 0 ? 1.0 : c <= 4 ? 0.0 : c <= 8 ? 0.5 : c <= 12 ? 0.0 : 1.0 / 3.0;
}

// Pull streaming with linear interpolation (Sec. 3.2): the class-c value at
// node x is the bilinear interpolation of the post-collision field at the
// off-lattice point x - c.  Source corner offset o = floor(-c) and
// fractional part t = -c - o, per axis; both depend only on the class.
__host__ __device__ constexpr int floor_int(double x) {
    return (x >= 0.0) ? (int)x : ((double)(int)x == x ? (int)x : (int)x - 1);
}
__host__ __device__ constexpr int cls_ox(int c) { return floor_int(-cls_cx(c)); }
__host__ __device__ constexpr int cls_oy(int c) { return floor_int(-cls_cy(c)); }
__host__ __device__ constexpr double cls_tx(int c) { return -cls_cx(c) - (double)cls_ox(c); }
__host__ __device__ constexpr double cls_ty(int c) { return -cls_cy(c) - (double)cls_oy(c); }

template <int I, int N, class F>
RLBM_HD inline void static_for(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// ---------------------------------------------------------------- storage conversion
template <typename TS, typename TC>
__device__ __forceinline__ TC load_q(const TS *p) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) {
        return (TC)__bfloat162float(__ldg(p));
    } else if constexpr (std::is_same<TS, __half>::value) {
        return (TC)__half2float(__ldg(p));
    } else {
        return (TC)__ldg(p);
    }
}

template <typename TS, typename TC>
__device__ __forceinline__ TS to_storage(TC x) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) {
        return __float2bfloat16_rn((float)x);
    } else if constexpr (std::is_same<TS, __half>::value) {
        return __float2half_rn((float)x);
    } else {
        return (TS)x;
    }
}

// ---------------------------------------------------------------- parameters
struct StepParams {
    int nx, ny, pitch;
    long long plane;  // elements per class plane = nz * ny * pitch
    int nz;           // layers (1 for the one-layer lattice)
    long long slab;   // elements per z layer = ny * pitch
    double inv_tau;   // 1/tau (Delta t = 1)
    double eps0;      // reference energy density of the deviation
    double scale;     // s
    double inv_scale; // 1/s
    // FP32 copies, so the FP32 kernels never touch the (slow) FP64 pipe
    float inv_tau_f, eps0_f, scale_f, inv_scale_f;
    // (4/3) eps0, the diagonal of S + eps I at rest, as an unevaluated sum
    // of two floats (for the frame refined to FP64 accuracy on FP32 lanes)
    float alpha_hi_f, alpha_lo_f;
    // eta/s mode (eta_k > 0): 1/tau = eta_k eps^{1/4}, from tau_R = 5 (eta/s)/T,
    // eps = 3 T^4/pi^2, in steps of dt: eta_k = (pi^2/3)^{1/4} dt / (5 eta/s)
    double eta_k;
    float eta_k_f;
    // CFL number (streaming displacement cfl * v_i per step) and, for
    // cfl != 1, the bilinear weights (w00, w10, w01, w11) of each class's
    // pull and the classes whose corner lies two cells away (cfl > 1):
    // bit c of far_x / far_y is set when cfl |c_x| > 1 (cfl |c_y| > 1)
    double cfl;
    double wt[17][4];
    float wt_f[17][4];
    unsigned far_x, far_y;
    // always 0: added to the state pointer of a second gather pass, so the
    // compiler cannot merge its loads with the first pass's (re-reading is
    // what frees the registers of the two-pass kernels)
    int reload_offset;
    // 1: stochastic rounding of 16-bit stores (packed kernels), else nearest
    int round_sr;
    int *err;         // device error word (bounded-wait / failure reporting)
};

// Arithmetic type of one node's lane: float and double here; packed.cuh
// adds a pair of FP32 lanes (two nodes per instruction).
template <typename T>
struct is_f32_lane : std::is_same<T, float> {};

// How the fused step streams: CFL 1 (compile-time corners and weights),
// 0 < cfl < 1 (compile-time corners, runtime weights), 1 < cfl < 2 (corners
// one or two cells away, chosen per class at run time: halo 2).
enum : int { kStreamCfl1 = 0, kStreamSub1 = 1, kStreamHalo2 = 2 };

inline int stream_mode(double cfl) { return cfl == 1.0 ? kStreamCfl1 : cfl < 1.0 ? kStreamSub1 : kStreamHalo2; }

// Fill the derived fields of a StepParams from inv_tau, eps0, scale, eta_k
// and cfl.  Pull source of class c: x - cfl c, per axis the corner offset
// o = floor(-cfl c) and fractional part t = -cfl c - o: for 0 < cfl < 1,
// o = -1 where c > 0 and 0 otherwise (t = 1 - cfl c or cfl |c|); for
// 1 < cfl < 2 the offset moves one cell further (-2 or +1) on the axes
// where cfl |c| > 1.
RLBM_HD inline void finish_params(StepParams &p) {
    p.reload_offset = 0;
    p.inv_scale = 1.0 / p.scale;
    p.inv_tau_f = (float)p.inv_tau;
    p.eps0_f = (float)p.eps0;
    p.scale_f = (float)p.scale;
    p.inv_scale_f = (float)p.inv_scale;
    p.eta_k_f = (float)p.eta_k;
    {
        const double alpha = 4.0 / 3.0 * p.eps0;
        p.alpha_hi_f = (float)alpha;
        p.alpha_lo_f = (float)(alpha - (double)p.alpha_hi_f);
    }
    p.far_x = p.far_y = 0u;
    for (int c = 0; c < 17; ++c) {
        const double sx = -p.cfl * cls_cx(c), sy = -p.cfl * cls_cy(c);
        const double ox = floor(sx), oy = floor(sy);
        const double tx = sx - ox, ty = sy - oy;
        if (ox == -2.0 || ox == 1.0) p.far_x |= 1u << c;
        if (oy == -2.0 || oy == 1.0) p.far_y |= 1u << c;
        p.wt[c][0] = (1.0 - tx) * (1.0 - ty);
        p.wt[c][1] = tx * (1.0 - ty);
        p.wt[c][2] = (1.0 - tx) * ty;
        p.wt[c][3] = tx * ty;
        for (int k = 0; k < 4; ++k) p.wt_f[c][k] = (float)p.wt[c][k];
    }
}

template <typename T>
RLBM_HD inline T par_wt(const StepParams &p, int c, int k) {
    if constexpr (is_f32_lane<T>::value) return T(p.wt_f[c][k]);
    else return p.wt[c][k];
}
template <typename T>
RLBM_HD inline T par_eta_k(const StepParams &p) {
    if constexpr (is_f32_lane<T>::value) return T(p.eta_k_f);
    else return p.eta_k;
}

template <typename T>
RLBM_HD inline T par_eps0(const StepParams &p) {
    if constexpr (is_f32_lane<T>::value) return T(p.eps0_f);
    else return p.eps0;
}
template <typename T>
RLBM_HD inline T par_scale(const StepParams &p) {
    if constexpr (is_f32_lane<T>::value) return T(p.scale_f);
    else return p.scale;
}
template <typename T>
RLBM_HD inline T par_inv_scale(const StepParams &p) {
    if constexpr (is_f32_lane<T>::value) return T(p.inv_scale_f);
    else return p.inv_scale;
}
template <typename T>
RLBM_HD inline T par_inv_tau(const StepParams &p) {
    if constexpr (is_f32_lane<T>::value) return T(p.inv_tau_f);
    else return p.inv_tau;
}

// a * b + c (one fused instruction); overloaded for packed lanes.
template <typename T>
RLBM_HD inline T fmadd(T a, T b, T c) { return a * b + c; }
template <typename T>
RLBM_HD inline T sqrt_(T x) { return std::sqrt(x); }

// One lattice of an ensemble step (k_step_batch): its buffers, parameters
// and its range in the flat tile list.
struct BatchRun {
    const void *qin;
    void *qout;
    const void *F;  // NULL: unforced
    StepParams p;
    int tiles_x;    // tiles along x
    int tile0;      // first global tile index of this lattice
};

// Moments of the post-stream node (deviation form), Eq. energyMomentumIntegral
// discretised: with f_c = W_c (eps0 + s q_c),
//   E = eps0 + dE, dE = s sum W q;  M^a = s sum W q c^a;
//   S^ab = eps0 delta^ab / 3 + dS^ab, dS^ab = s sum W q c^a c^b (in-plane);
//   Q^abc = s sum W q c^a c^b c^c (in-plane); Q^azz = M^a - Q^axx - Q^ayy.
template <typename TC>
struct NodeMoments {
    TC dE, Mx, My, dSxx, dSxy, dSyy, Qxxx, Qxxy, Qxyy, Qyyy;
};

// The 16 moving classes form 8 opposite pairs (c, -c) of equal weight.
RLBM_HD constexpr int pair_pos(int k) { return k == 0 ? 1 : k == 1 ? 3 : k == 2 ? 5 : k == 3 ? 7 : k == 4 ? 9 : k == 5 ? 10 : k == 6 ? 13 : 14; }
RLBM_HD constexpr int pair_neg(int k) { return k == 0 ? 2 : k == 1 ? 4 : k == 2 ? 6 : k == 3 ? 8 : k == 4 ? 12 : k == 5 ? 11 : k == 6 ? 16 : 15; }
constexpr int NPAIR = 8;

// Moments from pair sums s = q_c + q_-c (even moments E, S) and differences
// d = q_c - q_-c (odd moments M, Q), accumulated pair by pair (so a kernel
// may gather one pair at a time) and scaled by s at the end.
template <typename TC>
struct MomentSums {
    TC e, mx, my, sxx, sxy, syy, qxxx, qxxy, qxyy, qyyy;
};

template <typename TC>
RLBM_HD inline MomentSums<TC> moments_begin(TC q0) {
    MomentSums<TC> a;
    a.e = (TC)cls_w(0) * q0;
    a.mx = a.my = a.sxx = a.sxy = a.syy = a.qxxx = a.qxxy = a.qxyy = a.qyyy = (TC)0;
    return a;
}

template <int k, typename TC>
RLBM_HD inline void moments_add_pair(MomentSums<TC> &a, TC qp, TC qn) {
    constexpr int c = pair_pos(k);
    constexpr double w = cls_w(c), cx = cls_cx(c), cy = cls_cy(c);
    const TC sp = qp + qn;
    const TC dp = qp - qn;
    a.e = fmadd((TC)w, sp, a.e);
    if constexpr (cx != 0.0) {
        a.mx = fmadd((TC)(w * cx), dp, a.mx);
        a.sxx = fmadd((TC)(w * cx * cx), sp, a.sxx);
        a.qxxx = fmadd((TC)(w * cx * cx * cx), dp, a.qxxx);
    }
    if constexpr (cy != 0.0) {
        a.my = fmadd((TC)(w * cy), dp, a.my);
        a.syy = fmadd((TC)(w * cy * cy), sp, a.syy);
        a.qyyy = fmadd((TC)(w * cy * cy * cy), dp, a.qyyy);
    }
    if constexpr (cx != 0.0 && cy != 0.0) {
        a.sxy = fmadd((TC)(w * cx * cy), sp, a.sxy);
        a.qxxy = fmadd((TC)(w * cx * cx * cy), dp, a.qxxy);
        a.qxyy = fmadd((TC)(w * cx * cy * cy), dp, a.qxyy);
    }
}

// Opposite pairs k and k + 1 whose positive classes are (a, a) and (-a, a)
// (the in-plane diagonals, a = 1/sqrt2, and the corners, a = 1/sqrt3), of
// equal weight w.  With s_P, d_P and s_Q, d_Q the pairs' sums and
// differences, S = s_P + s_Q, D = s_P - s_Q, U = d_P + d_Q, V = d_P - d_Q:
//   E += w S,  S^xx, S^yy += w a^2 S,  S^xy += w a^2 D,
//   M^x += w a V,  M^y += w a U,  Q^xxx, Q^xyy += w a^3 V,  Q^xxy, Q^yyy += w a^3 U
// (the same sums as two moments_add_pair calls, in ten multiply-adds
// instead of twenty).
template <int k, typename TC>
RLBM_HD inline void moments_add_diag(MomentSums<TC> &a, TC pp, TC pn, TC qp, TC qn) {
    constexpr int cP = pair_pos(k), cQ = pair_pos(k + 1);
    constexpr double w = cls_w(cP), c = cls_cx(cP);
    static_assert(c > 0.0 && cls_cy(cP) == c && cls_cx(cQ) == -c && cls_cy(cQ) == c && cls_w(cQ) == w,
                  "pairs k, k + 1 are the diagonal classes (a, a), (-a, a)");
    const TC sP = pp + pn, dP = pp - pn, sQ = qp + qn, dQ = qp - qn;
    const TC S = sP + sQ, D = sP - sQ, U = dP + dQ, V = dP - dQ;
    a.e = fmadd((TC)w, S, a.e);
    a.sxx = fmadd((TC)(w * c * c), S, a.sxx);
    a.syy = fmadd((TC)(w * c * c), S, a.syy);
    a.sxy = fmadd((TC)(w * c * c), D, a.sxy);
    a.mx = fmadd((TC)(w * c), V, a.mx);
    a.my = fmadd((TC)(w * c), U, a.my);
    a.qxxx = fmadd((TC)(w * c * c * c), V, a.qxxx);
    a.qxyy = fmadd((TC)(w * c * c * c), V, a.qxyy);
    a.qxxy = fmadd((TC)(w * c * c * c), U, a.qxxy);
    a.qyyy = fmadd((TC)(w * c * c * c), U, a.qyyy);
}

// UNIT: the deviation scale s is 1 (FP32 and FP64 storage), so the sums
// are the moments and the multiplies are skipped (multiplying by 1 is exact:
// the results are the same bits either way).
template <typename TC, bool UNIT = false>
RLBM_HD inline NodeMoments<TC> moments_end(const MomentSums<TC> &a, TC s) {
    if constexpr (UNIT) {
        return NodeMoments<TC>{a.e, a.mx, a.my, a.sxx, a.sxy, a.syy, a.qxxx, a.qxxy, a.qxyy, a.qyyy};
    }
    NodeMoments<TC> m;
    m.dE = s * a.e;
    m.Mx = s * a.mx;
    m.My = s * a.my;
    m.dSxx = s * a.sxx;
    m.dSxy = s * a.sxy;
    m.dSyy = s * a.syy;
    m.Qxxx = s * a.qxxx;
    m.Qxxy = s * a.qxxy;
    m.Qxyy = s * a.qxyy;
    m.Qyyy = s * a.qyyy;
    return m;
}

template <typename TC, bool UNIT = false>
RLBM_HD inline NodeMoments<TC> node_moments(const TC (&q)[NC], TC s) {
    MomentSums<TC> a = moments_begin<TC>(q[0]);
    // the axis classes pair by pair, the diagonal and corner classes two pairs at a time
    static_for<0, 4>([&](auto K) {
        constexpr int k = decltype(K)::value;
        moments_add_pair<k, TC>(a, q[pair_pos(k)], q[pair_neg(k)]);
    });
    moments_add_diag<4, TC>(a, q[pair_pos(4)], q[pair_neg(4)], q[pair_pos(5)], q[pair_neg(5)]);
    moments_add_diag<6, TC>(a, q[pair_pos(6)], q[pair_neg(6)], q[pair_pos(7)], q[pair_neg(7)]);
    return moments_end<TC, UNIT>(a, s);
}

template <typename T>
RLBM_HD inline T absval(T x) { return x < (T)0 ? -x : x; }

template <typename T>
RLBM_HD inline T recip(T x) {
#ifdef __CUDA_ARCH__
    if constexpr (std::is_same<T, float>::value) return __frcp_rn(x);
#endif
    return (T)1 / x;
}

// Landau-Lifshitz frame (the eigenvalue problem closing Sec. 3.2):
// T^{mu nu} u_nu = -eps u^mu.  With v = u/u^0 and delta = E - eps this is
//   (S + eps I) v = M,  delta = M . v.
// In deviation variables S + eps I = A0 - delta I with A0 = (4 eps0/3 + dE) I
// + dS (the z row decouples: M_z = S_xz = S_yz = 0, so v_z = 0).  Newton on
//   g(delta) = delta - M . (A0 - delta I)^{-1} M,   g'(delta) = 1 - |v|^2.
// g is increasing and concave (g'' = -2 v.(A0 - delta I)^{-1} v), so Newton
// from below rises monotonically onto the physical root (eps > 0, |v| < 1).
// Start: expanding (A0 - delta I)^{-1} in delta gives delta = m1 + m2 delta +
// O(delta^2) with m1 = M.A0^{-1}M, m2 = |A0^{-1}M|^2, so delta0 = m1/(1 - m2)
// is already second-order accurate; one Newton step then reaches FP32
// round-off for typical |v| and further steps run only where needed.  The
// iterations use fast reciprocals (Newton corrects them); the final frame
// uses correctly rounded ones, because the equilibrium must carry the
// frame's energy-momentum to round-off or the collision stops conserving.
template <typename TL>
struct Frame {
    TL ddelta_eps;  // eps - eps0 = dE - delta
    TL eps;         // eps0 + dE - delta
    TL vx, vy;      // 3-velocity
    TL v2, g2;      // |v|^2, gamma^2 = 1/(1 - |v|^2)
    TL gamma;
};

// The hardware's approximate reciprocal and reciprocal square root (PTX
// rcp.approx.ftz.f32, rsqrt.approx.ftz.f32: one instruction each, a few
// units in the last place; arguments here are normal, positive numbers, so
// flushing subnormals changes nothing).  The Landau iteration corrects
// their error, and the final frame refines them by one Newton step.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename T>
RLBM_HD inline T fast_recip(T x) {
#ifdef __CUDA_ARCH__
    if constexpr (std::is_same<T, float>::value) return rcp_approx(x);
#endif
    return (T)1 / x;
}

template <typename T>
RLBM_HD inline T fast_rsqrt(T x) {
#ifdef __CUDA_ARCH__
    if constexpr (std::is_same<T, float>::value) return rsqrt_approx(x);
#endif
    return (T)1 / std::sqrt(x);
}

// Reciprocal and reciprocal square root of the final Landau frame.  FP32
// lanes: the hardware estimate refined by one step of Newton's method,
// y <- y + y (1 - x y) for 1/x and y <- y + (y/2) (1 - x y^2) for x^(-1/2),
// which squares the estimate's relative error, so the result is within
// about one unit in the last place (checked against IEEE division and
// square root by the numerics test); FP64 lanes: IEEE division and square
// root.
template <typename T>
RLBM_HD inline T frame_recip(T x) {
    if constexpr (is_f32_lane<T>::value) {
        const T y = fast_recip(x);
        const T e = fmadd((T)0 - x, y, T(1.0f));
        return fmadd(y, e, y);
    } else {
        return (T)1 / x;
    }
}

template <typename T>
RLBM_HD inline T frame_rsqrt(T x) {
    if constexpr (is_f32_lane<T>::value) {
        const T y = fast_rsqrt(x);
        const T e = fmadd((T)0 - x * y, y, T(1.0f));
        return fmadd(y * T(0.5f), e, y);
    } else {
        return (T)1 / sqrt_(x);
    }
}

// rest_a: (S + eps I) at rest in units of eps0 -- 4/3 for the spherical node
// (P = eps/3), 3/2 for the 2D ring (P = eps/2).
template <typename TL>
RLBM_HD inline Frame<TL> landau_solve(TL eps0, TL dE, TL Mx, TL My, TL dSxx, TL dSxy, TL dSyy,
                                      double rest_a = 4.0 / 3.0, TL *delta_out = nullptr) {
    const TL a0 = (TL)rest_a * eps0 + dE;
    constexpr bool dbl = std::is_same<TL, double>::value;
    const TL tol = dbl ? (TL)4e-16 : (TL)1e-7;
    TL vx, vy;
    const TL nMx = (TL)0 - Mx, nMy = (TL)0 - My, nSxy = (TL)0 - dSxy;
    // the delta-independent products of the 2 x 2 solve, formed once
    const TL nSxy2 = nSxy * dSxy, nSxyMy = nSxy * My, nSxyMx = nSxy * Mx;
    auto velocity = [&](TL d, bool exact) {
        const TL a = a0 - d;
        const TL axx = a + dSxx, ayy = a + dSyy;
        const TL det = fmadd(axx, ayy, nSxy2);
        const TL inv_det = exact ? frame_recip(det) : fast_recip(det);
        vx = fmadd(ayy, Mx, nSxyMy) * inv_det;
        vy = fmadd(axx, My, nSxyMx) * inv_det;
    };
    velocity((TL)0, false);
    const TL m1 = fmadd(Mx, vx, My * vy);
    const TL m2 = fmadd(vx, vx, vy * vy);
    TL delta = m1 * fast_recip((TL)1 - m2);
    TL step;
    auto newton = [&]() {
        velocity(delta, false);
        const TL g = fmadd(nMx, vx, fmadd(nMy, vy, delta));
        const TL gp = fmadd((TL)0 - vx, vx, fmadd((TL)0 - vy, vy, (TL)1));
        step = g * fast_recip(gp);
        delta = delta - step;
    };
    newton();
    // near the root the error after a step is ~ step^2 |v|^2 / a0, so the
    // iteration has converged once step^2 <= tol |delta| (exits on NaN too)
    for (int it = 1; it < (dbl ? 24 : 12); ++it) {
        if (!(step * step > tol * absval(delta))) break;
        newton();
    }
    if (delta_out) *delta_out = delta;
    velocity(delta, true);
    Frame<TL> fr;
    fr.ddelta_eps = dE - delta;
    fr.eps = eps0 + fr.ddelta_eps;
    fr.vx = vx;
    fr.vy = vy;
    fr.v2 = fmadd(vx, vx, vy * vy);
    if constexpr (is_f32_lane<TL>::value) {
        fr.gamma = frame_rsqrt((TL)1 - fr.v2);
        fr.g2 = fr.gamma * fr.gamma;
    } else {
        fr.g2 = recip((TL)1 - fr.v2);
        fr.gamma = sqrt_(fr.g2);
    }
    return fr;
}

// ---------------------------------------------------------------- frame to FP64 accuracy on FP32 lanes
// Rounded single operations that the compiler may neither contract into a
// fused multiply-add nor reassociate: the error-free transformations below
// rely on each rounding happening exactly as written.  (Overloads for the
// packed lanes live in packed.cuh, whose operators are such operations.)
__device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float xsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// s + e = a + b exactly (Knuth's branch-free TwoSum).
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = xadd(a, b);
    const T bb = xsub(s, a);
    e = xadd(xsub(a, xsub(s, bb)), xsub(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker's Fast2Sum).
template <typename T>
__device__ __forceinline__ void fast_two_sum(T a, T b, T &s, T &e) {
    s = xadd(a, b);
    e = xsub(b, xsub(s, a));
}
// p + e = a * b exactly (the rounding error of a product is one FMA away).
template <typename T>
__device__ __forceinline__ void two_prod(T a, T b, T &p, T &e) {
    p = xmul(a, b);
    e = xfma(a, b, xsub(T(0.0f), p));
}

// The Landau frame of the FP32 Newton solve (delta, v), refined by one
// Newton step of the coupled system
//     F1 = M - (A - delta I) v = 0,   F2 = M . v - delta = 0
// (the frame condition in the deviation variables of landau_solve) whose
// residuals are evaluated in double-float arithmetic: each product and sum
// of the residual is carried as an unevaluated pair of floats with its
// rounding error, so the residuals come out with about 48 significant
// bits although each input is an FP32 number.  The correction itself
// needs only FP32: with B = A - delta I, w = B^-1 F1 and u = B^-1 v,
//     d_delta = (F2 + M . w) / (1 - M . u),   d_v = w + d_delta u,
// where M . u = (B^-1 M) . v = |v|^2 to the order kept (B is symmetric), so
// 1 / (1 - M . u) is the frame's gamma^2.  The FP32 solve has converged to
// a few units in the last place, so the step's quadratic convergence
// leaves (delta + d_delta, v + d_v) within about 1e-14 of the exact frame
// of the stored moments: an FP64-accurate solve on the FP32 pipes (the
// FP64 units of this GPU run at 1/58 of the FP32 rate).  The frame's FP32
// fields are then the refined values rounded once; the collision consumes
// them in FP32, as it consumes an FP64 solve's.
// The refined frame as unevaluated sums hi + lo (for accuracy checks).
template <typename TL>
struct FramePairs {
    TL delta_hi, delta_lo, vx_hi, vx_lo, vy_hi, vy_lo;
};

template <typename TL>
__device__ __forceinline__ void landau_refine_df(TL alpha_hi, TL alpha_lo, TL eps0, TL dE, TL Mx, TL My, TL dSxx,
                                                 TL dSxy, TL dSyy, TL delta, Frame<TL> &fr,
                                                 FramePairs<TL> *pairs = nullptr) {
    const TL vx = fr.vx, vy = fr.vy, zero = TL(0.0f);
    const TL ndelta = xsub(zero, delta);
    // a = alpha + dE - delta (pair ah + al); bxx = a + dSxx, byy = a + dSyy
    TL s1, e1, ah, e2;
    two_sum(alpha_hi, dE, s1, e1);
    fast_two_sum(s1, ndelta, ah, e2);  // |s1| = E + eps0/3 > delta = M . v
    const TL al = xadd(alpha_lo, xadd(e1, e2));
    TL bxh, e3, byh, e4;
    two_sum(ah, dSxx, bxh, e3);
    two_sum(ah, dSyy, byh, e4);
    const TL bxl = xadd(al, e3), byl = xadd(al, e4);
    // F1x = Mx - bxx vx - dSxy vy,  F1y = My - dSxy vx - byy vy
    auto residual = [&](TL Ma, TL bh, TL bl, TL va, TL vb) {
        TL p1, q1, p2, q2, t1, f1, t2, f2;
        two_prod(bh, va, p1, q1);
        q1 = xfma(bl, va, q1);
        two_prod(dSxy, vb, p2, q2);
        two_sum(Ma, xsub(zero, p1), t1, f1);
        two_sum(t1, xsub(zero, p2), t2, f2);
        return xadd(t2, xsub(xadd(f1, f2), xadd(q1, q2)));
    };
    const TL rx = residual(Mx, bxh, bxl, vx, vy);
    const TL ry = residual(My, byh, byl, vy, vx);
    // F2 = Mx vx + My vy - delta
    TL p5, q5, p6, q6, t5, f5, t6, f6;
    two_prod(Mx, vx, p5, q5);
    two_prod(My, vy, p6, q6);
    two_sum(p5, p6, t5, f5);
    two_sum(t5, ndelta, t6, f6);
    const TL r2 = xadd(t6, xadd(xadd(f5, f6), xadd(q5, q6)));
    // the FP32 Newton correction
    const TL nSxy = zero - dSxy;
    const TL inv_det = fast_recip(fmadd(bxh, byh, nSxy * dSxy));
    const TL wx = fmadd(byh, rx, nSxy * ry) * inv_det;
    const TL wy = fmadd(bxh, ry, nSxy * rx) * inv_det;
    const TL ux = fmadd(byh, vx, nSxy * vy) * inv_det;
    const TL uy = fmadd(bxh, vy, nSxy * vx) * inv_det;
    const TL dd = fmadd(Mx, wx, fmadd(My, wy, r2)) * fr.g2;
    const TL dvx = fmadd(dd, ux, wx), dvy = fmadd(dd, uy, wy);
    if (pairs) *pairs = FramePairs<TL>{delta, dd, vx, dvx, vy, dvy};
    // refined frame, rounded once to FP32: eps - eps0 = dE - delta - dd
    TL h, e;
    two_sum(dE, ndelta, h, e);
    fr.ddelta_eps = xadd(h, xsub(e, dd));
    fr.eps = eps0 + fr.ddelta_eps;
    fr.vx = xadd(vx, dvx);
    fr.vy = xadd(vy, dvy);
    fr.v2 = fmadd(fr.vx, fr.vx, fr.vy * fr.vy);
    fr.gamma = frame_rsqrt(TL(1.0f) - fr.v2);
    fr.g2 = fr.gamma * fr.gamma;
}

// Fused collision of one node (steps (c)-(e) of Sec. 3.3) on the gathered
// deviations q[c] (in place), returning the frame for diagnostics.
//
// Equilibrium (Eqs. rel_pdf_exp, rel_pdf_exp_coef with T_eq of Eq.
// stressEnergyT, P = eps/3, App. A norms): f_eq,i = w_i [-(3/2) T00 + 3 v_i.M_eq
// + (15/2) v_i S_eq v_i]; for |v_i| = 1 and xi = v_i . v this is
//   f_eq,c = W_c eps [3 - 2 gamma^2 + gamma^2 (4 xi + 10 xi^2)],
// so q_eq,c = P0 + P1 xi + P2 xi^2 with P0 = [eps - eps0 - 2 eps gamma^2 |v|^2]/s,
// P1 = 4 eps gamma^2 / s, P2 = 10 eps gamma^2 / s.
// Relaxation (Eq. boltzmanneq_rel, Anderson-Witting): rate
// (u^0 - v_c . u)/tau = om (1 - xi), om = gamma/tau.
// Driving term (Eq. forceTerm, App. B), F^mu = (0, F_x, F_y, 0), prefactor
// -6 so that sum G = F.M and sum G v = F E:
//   G_c = -6 W_c [ F.M/4 - (F.c) E/2 + (5/4) F_a c_b c_c Q^abc - (5/2)(F.c)(c.M) ]
// with the moments of the post-stream populations, and Q^azz = M^a - Q^axx - Q^ayy,
// v_z^2 = 1 - c_x^2 - c_y^2.
//
// Per class the update q' = q (1 - om + om xi) + om (1 - xi) q_eq + G/(W s)
// is a cubic polynomial in (c_x, c_y); splitting it into the part even in c
//   K0 + Kxx c_x^2 + Kxy c_x c_y + Kyy c_y^2
// and the odd part  xi [om (P1 - P0) - om P2 xi^2] + G1 (F.c)
// lets each opposite pair (c, -c) share one evaluation.
// Coefficients of the per-class update of one node (below).
// vs = vx + vy, vd = vy - vx, KS = Kxx + Kyy, Gs = G1 (Fx + Fy), Gd =
// G1 (Fy - Fx): the terms the diagonal classes (a, a), (-a, a) share.
template <typename TC>
struct CollideCoef {
    TC K0, Kxx, Kxy, Kyy, o1, no3, G1, om, nom, a0, vx, vy, Fx, Fy;
    TC vs, vd, KS, Gs, Gd;
};

// Frame and update coefficients of a node from its moments.  DFL: refine
// the FP32 frame to FP64 accuracy (landau_refine_df; FP32 lanes only).
template <typename TC, typename TL, bool FORCED, bool DFL = false, bool UNIT = false>
RLBM_HD inline Frame<TL> collide_coef(const NodeMoments<TC> &m, TC Fx, TC Fy, const StepParams &p,
                                      CollideCoef<TC> &k) {
    TL delta;
    Frame<TL> fr = landau_solve<TL>(par_eps0<TL>(p), (TL)m.dE, (TL)m.Mx, (TL)m.My, (TL)m.dSxx, (TL)m.dSxy,
                                    (TL)m.dSyy, 4.0 / 3.0, DFL ? &delta : nullptr);
    if constexpr (DFL) {
        static_assert(is_f32_lane<TL>::value, "the double-float refinement runs on FP32 lanes");
#ifdef __CUDA_ARCH__
        landau_refine_df<TL>(TL(p.alpha_hi_f), TL(p.alpha_lo_f), par_eps0<TL>(p), (TL)m.dE, (TL)m.Mx, (TL)m.My,
                             (TL)m.dSxx, (TL)m.dSxy, (TL)m.dSyy, delta, fr);
#endif
    }
    const TC inv_s = par_inv_scale<TC>(p);
    // times 1/s, skipped where s = 1 (exact either way)
    auto unscale = [&](TC x) {
        if constexpr (UNIT) return x;
        else return x * inv_s;
    };
    const TL eg2 = fr.eps * fr.g2;
    const TC P0 = unscale((TC)(fmadd((TL)(-2) * eg2, fr.v2, fr.ddelta_eps)));
    const TC P1 = unscale((TC)((TL)4 * eg2));
    const TC P2 = unscale((TC)((TL)10 * eg2));
    const TC vx = (TC)fr.vx, vy = (TC)fr.vy;
    // relaxation rate: 1/tau, or in eta/s mode T(eps) dt / (5 eta/s)
    TL inv_tau = par_inv_tau<TL>(p);
    if (p.eta_k_f > 0.0f) inv_tau = par_eta_k<TL>(p) * sqrt_(sqrt_(fr.eps));
    const TC om = (TC)(fr.gamma * inv_tau);

    // even part K0 + Kxx cx^2 + Kxy cx cy + Kyy cy^2, odd part coefficients
    const TC e2 = om * (P2 - P1);
    TC K0 = om * P0, Kxx = e2 * vx * vx, Kxy = (TC)2 * e2 * vx * vy, Kyy = e2 * vy * vy;
    const TC o1 = om * (P1 - P0), no3 = (TC)0 - om * P2;
    TC G1 = 0;
    if constexpr (FORCED) {
        const TC E = par_eps0<TC>(p) + m.dE;
        const TC c6 = unscale((TC)(-6.0));
        const TC G0 = c6 * (TC)0.25 * fmadd(Fx, m.Mx, Fy * m.My);
        G1 = c6 * (TC)(-0.5) * E;
        const TC G3 = c6 * (TC)(-2.5);
        const TC c54 = c6 * (TC)1.25;
        const TC Qxzz = m.Mx - m.Qxxx - m.Qxyy;
        const TC Qyzz = m.My - m.Qxxy - m.Qyyy;
        const TC Pxx = c54 * fmadd(Fx, m.Qxxx, Fy * m.Qxxy);
        const TC Pxy = c54 * fmadd(Fx, m.Qxxy, Fy * m.Qxyy);
        const TC Pyy = c54 * fmadd(Fx, m.Qxyy, Fy * m.Qyyy);
        const TC Pzz = c54 * fmadd(Fx, Qxzz, Fy * Qyzz);
        K0 = K0 + (G0 + Pzz);
        Kxx = fmadd(G3 * Fx, m.Mx, Kxx + (Pxx - Pzz));
        Kxy = fmadd(G3, fmadd(Fx, m.My, Fy * m.Mx), Kxy + (TC)2 * Pxy);
        Kyy = fmadd(G3 * Fy, m.My, Kyy + (Pyy - Pzz));
    }
    k.K0 = K0;
    k.Kxx = Kxx;
    k.Kxy = Kxy;
    k.Kyy = Kyy;
    k.o1 = o1;
    k.no3 = no3;
    k.G1 = G1;
    k.om = om;
    k.nom = (TC)0 - om;
    k.a0 = (TC)1 - om;
    k.vx = vx;
    k.vy = vy;
    k.Fx = Fx;
    k.Fy = Fy;
    k.vs = vx + vy;
    k.vd = vy - vx;
    k.KS = Kxx + Kyy;
    k.Gs = 0;
    k.Gd = 0;
    if constexpr (FORCED) {
        k.Gs = G1 * (Fx + Fy);
        k.Gd = G1 * (Fy - Fx);
    }
    return fr;
}

// The rest class: q' = q (1 - om) + K0.
template <typename TC>
RLBM_HD inline TC collide_rest(TC q0, const CollideCoef<TC> &k) {
    return fmadd(q0, k.a0, k.K0);
}

// Opposite pair k: (q_c, q_-c) -> updated values.  The relaxation factors
// a0 +- om xi are single fused multiply-adds; components of c equal to 1
// (the axis classes) enter without a multiply.
template <int kp, typename TC, bool FORCED>
RLBM_HD inline void collide_pair(TC &qp, TC &qn, const CollideCoef<TC> &k) {
    constexpr int c = pair_pos(kp);
    constexpr double cx = cls_cx(c), cy = cls_cy(c);
    TC xi = 0;
    [[maybe_unused]] TC Fc = 0;
    TC even = k.K0;
    if constexpr (cx != 0.0) {
        if constexpr (cx == 1.0) {
            xi = k.vx;
            even = even + k.Kxx;
            if constexpr (FORCED) Fc = k.Fx;
        } else {
            xi = (TC)cx * k.vx;
            even = fmadd((TC)(cx * cx), k.Kxx, even);
            if constexpr (FORCED) Fc = (TC)cx * k.Fx;
        }
    }
    if constexpr (cy != 0.0) {
        if constexpr (cy == 1.0 && cx == 0.0) {
            xi = k.vy;
            even = even + k.Kyy;
            if constexpr (FORCED) Fc = k.Fy;
        } else {
            xi = fmadd((TC)cy, k.vy, xi);
            even = fmadd((TC)(cy * cy), k.Kyy, even);
            if constexpr (FORCED) Fc = fmadd((TC)cy, k.Fy, Fc);
        }
    }
    if constexpr (cx != 0.0 && cy != 0.0) even = fmadd((TC)(cx * cy), k.Kxy, even);
    TC odd = xi * fmadd(k.no3, xi * xi, k.o1);
    if constexpr (FORCED) odd = fmadd(k.G1, Fc, odd);
    const TC ap = fmadd(k.om, xi, k.a0), an = fmadd(k.nom, xi, k.a0);
    const TC p0 = qp, n0 = qn;
    qp = fmadd(p0, ap, even + odd);
    qn = fmadd(n0, an, even - odd);
}

// Opposite pairs kp and kp + 1 with positive classes (a, a) and (-a, a)
// (see moments_add_diag): xi = a vs and a vd, the even parts K0 + a^2 KS
// +- a^2 Kxy, the forcing a Gs and a Gd -- collide_pair's update of the four
// classes with the terms the two pairs share formed once.
template <int kp, typename TC, bool FORCED>
RLBM_HD inline void collide_diag(TC &pp, TC &pn, TC &qp, TC &qn, const CollideCoef<TC> &k) {
    constexpr int cP = pair_pos(kp), cQ = pair_pos(kp + 1);
    constexpr double c = cls_cx(cP);
    static_assert(c > 0.0 && cls_cy(cP) == c && cls_cx(cQ) == -c && cls_cy(cQ) == c,
                  "pairs kp, kp + 1 are the diagonal classes (a, a), (-a, a)");
    const TC xiP = (TC)c * k.vs, xiQ = (TC)c * k.vd;
    const TC base = fmadd((TC)(c * c), k.KS, k.K0);
    const TC evenP = fmadd((TC)(c * c), k.Kxy, base), evenQ = fmadd((TC)(-c * c), k.Kxy, base);
    TC oddP = xiP * fmadd(k.no3, xiP * xiP, k.o1);
    TC oddQ = xiQ * fmadd(k.no3, xiQ * xiQ, k.o1);
    if constexpr (FORCED) {
        oddP = fmadd((TC)c, k.Gs, oddP);
        oddQ = fmadd((TC)c, k.Gd, oddQ);
    }
    const TC aPp = fmadd(k.om, xiP, k.a0), aPn = fmadd(k.nom, xiP, k.a0);
    const TC aQp = fmadd(k.om, xiQ, k.a0), aQn = fmadd(k.nom, xiQ, k.a0);
    const TC p0 = pp, p1 = pn, q0 = qp, q1 = qn;
    pp = fmadd(p0, aPp, evenP + oddP);
    pn = fmadd(p1, aPn, evenP - oddP);
    qp = fmadd(q0, aQp, evenQ + oddQ);
    qn = fmadd(q1, aQn, evenQ - oddQ);
}

template <typename TC, typename TL, bool FORCED, bool DFL = false, bool UNIT = false>
RLBM_HD inline Frame<TL> collide_node(TC (&q)[NC], TC Fx, TC Fy, const StepParams &p) {
    const NodeMoments<TC> m = node_moments<TC, UNIT>(q, par_scale<TC>(p));
    CollideCoef<TC> k;
    const Frame<TL> fr = collide_coef<TC, TL, FORCED, DFL, UNIT>(m, Fx, Fy, p, k);
    q[0] = collide_rest<TC>(q[0], k);
    static_for<0, 4>([&](auto K) {
        constexpr int kp = decltype(K)::value;
        collide_pair<kp, TC, FORCED>(q[pair_pos(kp)], q[pair_neg(kp)], k);
    });
    collide_diag<4, TC, FORCED>(q[pair_pos(4)], q[pair_neg(4)], q[pair_pos(5)], q[pair_neg(5)], k);
    collide_diag<6, TC, FORCED>(q[pair_pos(6)], q[pair_neg(6)], q[pair_pos(7)], q[pair_neg(7)], k);
    return fr;
}

}  // namespace rlbk
