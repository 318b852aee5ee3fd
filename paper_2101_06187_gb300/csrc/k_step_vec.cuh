// k_step_vec.cuh -- fused stream + collide + force step with a run of V
// x-adjacent nodes per thread.  Each class row is fetched as one aligned
// vector load (16 bytes for FP32 and FP64, 8 bytes for 16-bit storage)
// plus at most one scalar neighbour on the side the class streams from, so
// a thread issues about a quarter of the loads, address arithmetic and
// stores of the one-node kernel.  Needs nx % V == 0 (rows start aligned
// because the pitch is a multiple of 32 elements).
#pragma once

#include "rlbm_device.cuh"

namespace rlbk {

// Default run length per storage type (16-byte runs for FP32/FP64, 8-byte
// runs for 16-bit storage).
template <typename TS>
struct VecOf {
    static constexpr int V = std::is_same<TS, double>::value ? 2 : 4;
};

// Aligned vector load of V consecutive stored values, converted to TC.
template <typename TS, typename TC, int V>
__device__ __forceinline__ void load_run(const TS *__restrict__ p, TC *out) {
    if constexpr (std::is_same<TS, float>::value && V == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    } else if constexpr (std::is_same<TS, float>::value && V == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        out[0] = v.x;
        out[1] = v.y;
    } else if constexpr (std::is_same<TS, double>::value && V == 2) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        out[0] = v.x;
        out[1] = v.y;
    } else if constexpr (std::is_same<TS, __nv_bfloat16>::value || std::is_same<TS, __half>::value) {
        using T2 = typename std::conditional<std::is_same<TS, __half>::value, __half2, __nv_bfloat162>::type;
        auto cvt = [](const T2 &h) -> float2 {
            if constexpr (std::is_same<TS, __half>::value) return __half22float2(h);
            else return __bfloat1622float2(h);
        };
        if constexpr (V == 4) {
            const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(p));
            const float2 a = cvt(*reinterpret_cast<const T2 *>(&raw.x));
            const float2 b = cvt(*reinterpret_cast<const T2 *>(&raw.y));
            out[0] = a.x;
            out[1] = a.y;
            out[2] = b.x;
            out[3] = b.y;
        } else {
            const unsigned int raw = __ldg(reinterpret_cast<const unsigned int *>(p));
            const float2 a = cvt(*reinterpret_cast<const T2 *>(&raw));
            out[0] = a.x;
            out[1] = a.y;
        }
    } else {
        static_assert(V == 4 || V == 2, "unsupported run length");
    }
}

template <typename TS, typename TC, int V>
__device__ __forceinline__ void store_run(TS *__restrict__ p, const TC *in) {
    if constexpr (std::is_same<TS, float>::value && V == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(in[0], in[1], in[2], in[3]);
    } else if constexpr (std::is_same<TS, float>::value && V == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(in[0], in[1]);
    } else if constexpr (std::is_same<TS, double>::value && V == 2) {
        *reinterpret_cast<double2 *>(p) = make_double2(in[0], in[1]);
    } else if constexpr (std::is_same<TS, __nv_bfloat16>::value || std::is_same<TS, __half>::value) {
        auto pack = [](float a, float b) -> unsigned int {
            if constexpr (std::is_same<TS, __half>::value) {
                const __half2 h = __floats2half2_rn(a, b);
                return *reinterpret_cast<const unsigned int *>(&h);
            } else {
                const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                return *reinterpret_cast<const unsigned int *>(&h);
            }
        };
        if constexpr (V == 4) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(pack((float)in[0], (float)in[1]), pack((float)in[2], (float)in[3]));
        } else {
            *reinterpret_cast<unsigned int *>(p) = pack((float)in[0], (float)in[1]);
        }
    }
}

// One class row around the run: r[0] = column x0-1, r[1..V] = x0..x0+V-1,
// r[V+1] = x0+V (periodic); only the side the class pulls from is loaded.
template <int c, typename TS, typename TC, int V>
__device__ __forceinline__ void load_class_row(const TS *__restrict__ row, int x0, int xl, int xr, TC (&r)[V + 2]) {
    constexpr int ox = cls_ox(c);
    constexpr double tx = cls_tx(c);
    load_run<TS, TC, V>(row + x0, &r[1]);
    if constexpr (ox == -1) r[0] = load_q<TS, TC>(row + xl);
    if constexpr (ox == 1 || (ox == 0 && tx != 0.0)) r[V + 1] = load_q<TS, TC>(row + xr);
}

// The fused step for the run of V nodes starting at (x0, y).
template <typename TS, typename TC, typename TL, bool FORCED, int V>
__device__ __forceinline__ void step_run(const TS *__restrict__ qin, TS *__restrict__ qout, const TC *__restrict__ F,
                                         const StepParams &p, int x0, int y) {
    const int ym = (y == 0) ? p.ny - 1 : y - 1;
    const int yp = (y == p.ny - 1) ? 0 : y + 1;
    const int xl = (x0 == 0) ? p.nx - 1 : x0 - 1;
    const int xr = (x0 + V == p.nx) ? 0 : x0 + V;
    const long long rowoff[3] = {(long long)ym * p.pitch, (long long)y * p.pitch, (long long)yp * p.pitch};

    TC q[V][NC];
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        constexpr int ox = cls_ox(c), oy = cls_oy(c);
        constexpr double tx = cls_tx(c), ty = cls_ty(c);
        const TS *plane = qin + (long long)c * p.plane;
        TC a[V + 2];
        load_class_row<c, TS, TC, V>(plane + rowoff[oy + 1], x0, xl, xr, a);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            TC v = (TC)((1.0 - tx) * (1.0 - ty)) * a[i + ox + 1];
            if constexpr (tx != 0.0) v += (TC)(tx * (1.0 - ty)) * a[i + ox + 2];
            q[i][c] = v;
        }
        if constexpr (ty != 0.0) {
            TC b[V + 2];
            load_class_row<c, TS, TC, V>(plane + rowoff[oy + 2], x0, xl, xr, b);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                TC v = (TC)((1.0 - tx) * ty) * b[i + ox + 1];
                if constexpr (tx != 0.0) v += (TC)(tx * ty) * b[i + ox + 2];
                q[i][c] += v;
            }
        }
    });

    TC Fx[V], Fy[V];
    const long long n0 = (long long)y * p.pitch + x0;
    if constexpr (FORCED) {
        load_run<TC, TC, V>(F + n0, Fx);
        load_run<TC, TC, V>(F + p.plane + n0, Fy);
    }
#pragma unroll
    for (int i = 0; i < V; ++i) collide_node<TC, TL, FORCED>(q[i], FORCED ? Fx[i] : (TC)0, FORCED ? Fy[i] : (TC)0, p);

    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        TC out[V];
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = q[i][c];
        store_run<TS, TC, V>(qout + (long long)c * p.plane + n0, out);
    });
}

template <typename TS, typename TC, typename TL, bool FORCED, int V>
__global__ void __launch_bounds__(256) k_step_vec(const TS *__restrict__ qin, TS *__restrict__ qout,
                                                  const TC *__restrict__ F, StepParams p) {
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= p.nx || y >= p.ny) return;
    step_run<TS, TC, TL, FORCED, V>(qin, qout, F, p, x0, y);
}

// Ensemble of independent lattices advanced by one launch: a flat list of
// tiles (one thread block's worth of runs, blockDim.x * V columns by
// blockDim.y rows) over all lattices; each block walks the list with a grid
// stride, so the grid can be sized to the GPU (a multiple of the SM count)
// rather than to the work.
template <typename TS, typename TC, typename TL>
__global__ void __launch_bounds__(256) k_step_batch(const BatchRun *__restrict__ runs, int nruns, int ntiles) {
    constexpr int V = VecOf<TS>::V;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        // binary search of the lattice owning tile t
        int lo = 0, hi = nruns - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (runs[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchRun &r = runs[lo];
        const int local = t - r.tile0;
        const int tx = local % r.tiles_x, ty = local / r.tiles_x;
        const int x0 = (tx * blockDim.x + threadIdx.x) * V;
        const int y = ty * blockDim.y + threadIdx.y;
        if (x0 < r.p.nx && y < r.p.ny) {
            if (r.F)
                step_run<TS, TC, TL, true, V>(static_cast<const TS *>(r.qin), static_cast<TS *>(r.qout),
                                              static_cast<const TC *>(r.F), r.p, x0, y);
            else
                step_run<TS, TC, TL, false, V>(static_cast<const TS *>(r.qin), static_cast<TS *>(r.qout), nullptr,
                                               r.p, x0, y);
        }
    }
}

}  // namespace rlbk
