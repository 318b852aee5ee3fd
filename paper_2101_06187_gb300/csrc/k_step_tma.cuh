// k_step_tma.cuh -- the fused step with the populations staged in shared
// memory by the tensor-memory accelerator (TMA) in a double-buffered,
// persistent pipeline: FP32 storage, packed FP32 lanes (two x-adjacent nodes
// per thread), FP32 Landau solve, CFL 1.
//
// Each CTA walks tiles of TW x TH nodes (grid stride).  One thread issues a
// single 3D bulk tensor copy per tile: the 17 class planes of the tile with
// a halo of one row above and below and four columns left and right (the
// TMA x coordinate has to start on a 16-byte boundary, so the one-column
// halo is widened to four), plus a second copy of the tile's force field.
// While the CTA computes tile k from one stage, the copy of tile k+1 lands
// in the other, so the number of bytes in flight no longer depends on how
// many warps the register budget allows.  The periodic wrap of the lattice
// edges (the TMA fills out-of-range cells with zeros) is patched with plain
// loads for the tiles that touch an edge.  Results go straight from
// registers to global memory (coalesced 8-byte stores).
//
// Every wait on a shared-memory barrier is bounded; a wait that gives up
// sets the launch's error word, lets the copies already issued land (again
// with a bound) and leaves the kernel.
#pragma once

#include <cuda.h>

#include "k_step_vec.cuh"
#include "packed.cuh"

namespace rlbk {

constexpr int kTmaTW = 64;  // tile width (nodes); 32 threads x 2 nodes
constexpr int kTmaTH = 8;   // tile height (rows); 8 warps
constexpr int kTmaSW = kTmaTW + 8;  // staged row width: 4 halo columns each side
constexpr int kTmaSH = kTmaTH + 2;  // staged rows: 1 halo row each side
constexpr int kTmaPlane = kTmaSW * kTmaSH;  // floats per staged class plane
constexpr int kTmaQBytes = NC * kTmaPlane * 4;                   // one bulk copy
constexpr int kTmaQRegion = ((kTmaQBytes + 127) / 128) * 128;     // force copy starts 128-byte aligned
constexpr int kTmaFBytes = 2 * kTmaTW * kTmaTH * 4;
constexpr int kTmaStageBytes = ((kTmaQRegion + kTmaFBytes + 127) / 128) * 128;
constexpr int kTmaSmemBytes = 128 + 2 * kTmaStageBytes + 16;  // alignment slack, two stages, two barriers
constexpr int kTmaThreads = (kTmaTW / 2) * kTmaTH;
constexpr unsigned long long kTmaWaitNs = 1000000000ull;  // a wait gives up after one second
constexpr int kTmaErrTimeout = 1;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity to complete: gives up
// (returns false) once kTmaWaitNs of global time have passed.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kTmaWaitNs) return false;
    }
}

// 3D tiled bulk tensor copy global -> shared, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

struct TmaTile {
    int x0, y0;
};

__device__ __forceinline__ TmaTile tma_tile(int t, int tiles_x) {
    return TmaTile{(t % tiles_x) * kTmaTW, (t / tiles_x) * kTmaTH};
}

// Issue the copies of tile t into stage s (one thread).
template <bool FORCED>
__device__ __forceinline__ void tma_issue(unsigned char *stage, unsigned bar, const CUtensorMap *mq,
                                          const CUtensorMap *mf, int t, int tiles_x) {
    const TmaTile tl = tma_tile(t, tiles_x);
    mbar_expect_tx(bar, kTmaQBytes + (FORCED ? kTmaFBytes : 0));
    tma_load_3d(smem_addr(stage), mq, tl.x0 - 4, tl.y0 - 1, 0, bar);
    if constexpr (FORCED) tma_load_3d(smem_addr(stage + kTmaQRegion), mf, tl.x0, tl.y0, 0, bar);
}

// The staged cells whose lattice position lies across a periodic edge
// (x = -1 or nx, y = -1 or ny) hold the TMA's zero fill: list them per
// class -- whole staged rows across a y edge, staged columns across an x
// edge -- and load their wrapped values.
struct TmaFix {
    int rows[2], nrows, cols[2], ncols, per_class;
};

__device__ __forceinline__ TmaFix tma_fix_list(const TmaTile &tl, int nx, int ny) {
    TmaFix f;
    f.nrows = f.ncols = 0;
    if (tl.y0 == 0) f.rows[f.nrows++] = 0;
    if (tl.y0 + kTmaTH >= ny) f.rows[f.nrows++] = ny - tl.y0 + 1;
    if (tl.x0 == 0) f.cols[f.ncols++] = 3;
    if (tl.x0 + kTmaTW >= nx) f.cols[f.ncols++] = nx - tl.x0 + 4;
    f.per_class = f.nrows * (kTmaTW + 2) + f.ncols * kTmaSH;
    return f;
}

// Item u of the fix list -> staged offset (class plane + row + column) and
// source element of the wrapped lattice.
__device__ __forceinline__ void tma_fix_item(const TmaFix &f, const TmaTile &tl, int u, const StepParams &p,
                                             int *soff, long long *goff) {
    const int c = u / f.per_class;
    int r = u - c * f.per_class;
    int i, j;
    const int nr = f.nrows * (kTmaTW + 2);
    if (r < nr) {
        i = f.rows[r / (kTmaTW + 2)];
        j = 3 + r % (kTmaTW + 2);
    } else {
        r -= nr;
        j = f.cols[r / kTmaSH];
        i = r % kTmaSH;
    }
    int gx = tl.x0 - 4 + j, gy = tl.y0 - 1 + i;
    gx = (gx + p.nx) % p.nx;
    gy = (gy + p.ny) % p.ny;
    *soff = c * kTmaPlane + i * kTmaSW + j;
    *goff = (long long)c * p.plane + (long long)gy * p.pitch + gx;
}

// One staged class row around the node pair at staged column j (even):
// a[k] = row[j - 1 + k], k = 0..3.
template <int c>
__device__ __forceinline__ void smem_class_row(const float *row, int j, float (&a)[4]) {
    constexpr int ox = cls_ox(c);
    constexpr double tx = cls_tx(c);
    const float2 mid = *reinterpret_cast<const float2 *>(row + j);
    a[1] = mid.x;
    a[2] = mid.y;
    if constexpr (ox == -1) a[0] = row[j - 1];
    if constexpr (ox == 1 || (ox == 0 && tx != 0.0)) a[3] = row[j + 2];
}

template <bool FORCED>
__device__ __forceinline__ void step_pair_staged(const float *st, const float *Fst, float *__restrict__ qout,
                                                 const StepParams &p, int lx, int ly, int x, int y) {
    pf2 q[NC];
    const int j = lx + 4;
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        constexpr int ox = cls_ox(c), oy = cls_oy(c);
        constexpr double tx = cls_tx(c), ty = cls_ty(c);
        const float *plane = st + c * kTmaPlane;
        float a[4];
        smem_class_row<c>(plane + (ly + 1 + oy) * kTmaSW, j, a);
        pf2 v = pf2((float)((1.0 - tx) * (1.0 - ty))) * pf2(a[ox + 1], a[ox + 2]);
        if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * (1.0 - ty))), pf2(a[ox + 2], a[ox + 3]), v);
        if constexpr (ty != 0.0) {
            float b[4];
            smem_class_row<c>(plane + (ly + 2 + oy) * kTmaSW, j, b);
            v = fmadd(pf2((float)((1.0 - tx) * ty)), pf2(b[ox + 1], b[ox + 2]), v);
            if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * ty)), pf2(b[ox + 2], b[ox + 3]), v);
        }
        q[c] = v;
    });
    pf2 Fx = 0.0f, Fy = 0.0f;
    if constexpr (FORCED) {
        const float2 fx = *reinterpret_cast<const float2 *>(Fst + ly * kTmaTW + lx);
        const float2 fy = *reinterpret_cast<const float2 *>(Fst + (kTmaTH + ly) * kTmaTW + lx);
        Fx = pf2(fx);
        Fy = pf2(fy);
    }
    collide_node<pf2, pf2, FORCED>(q, Fx, Fy, p);
    const long long n0 = (long long)y * p.pitch + x;
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        *reinterpret_cast<float2 *>(qout + (long long)c * p.plane + n0) = q[c].v;
    });
}

// Persistent TMA-pipelined fused step.  Block (32, 8); grid = resident CTAs.
// mq: 3D map of the input state (x: nx, y: ny, class: 17; box 72 x 10 x 17);
// mf: 3D map of the force (x: nx, y: ny, component: 2; box 64 x 8 x 2).
// unarmed: failure-detection test only -- the CTAs issue no tile copies, so
// their first wait runs out after kTmaWaitNs and the error word is set
// (nothing is in flight, nothing faults).
template <bool FORCED>
__global__ void __launch_bounds__(kTmaThreads, 2)
    k_step_tma(const __grid_constant__ CUtensorMap mq, const __grid_constant__ CUtensorMap mf,
               const float *__restrict__ qin, float *__restrict__ qout, StepParams p, int unarmed) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    unsigned char *const stage0 = smem;
    const unsigned bar0 = smem_addr(smem + 2 * kTmaStageBytes);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int tiles_x = (p.nx + kTmaTW - 1) / kTmaTW;
    const int ntiles = tiles_x * ((p.ny + kTmaTH - 1) / kTmaTH);
    const int G = gridDim.x;

    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&mq)) : "memory");
        for (int s = 0; s < 2 && !unarmed; ++s) {
            const int t = blockIdx.x + s * G;
            if (t < ntiles) tma_issue<FORCED>(stage0 + s * kTmaStageBytes, bar0 + 8 * s, &mq, &mf, t, tiles_x);
        }
    }
    __syncthreads();

    const int lx = 2 * threadIdx.x, ly = threadIdx.y;
    bool ok = true;
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, ++k) {
        const int s = k & 1;
        unsigned char *const stage = stage0 + s * kTmaStageBytes;
        const unsigned bar = bar0 + 8 * s;
        const TmaTile tl = tma_tile(t, tiles_x);
        const TmaFix fix = tma_fix_list(tl, p.nx, p.ny);
        const int nfix = NC * fix.per_class;
        // the wrapped cells' loads go out before the wait, so their latency
        // overlaps the tile copy
        constexpr int kPre = 2;
        float pre[kPre];
        int pre_off[kPre];
#pragma unroll
        for (int r = 0; r < kPre; ++r) {
            const int u = tid + r * kTmaThreads;
            pre_off[r] = -1;
            pre[r] = 0.0f;
            if (u < nfix) {
                long long g;
                tma_fix_item(fix, tl, u, p, &pre_off[r], &g);
                pre[r] = __ldg(qin + g);
            }
        }
        const bool landed = mbar_wait(bar, (k >> 1) & 1);
        if (!__syncthreads_and(landed)) {  // one decision for the whole CTA
            ok = false;
            break;
        }
        if (nfix > 0) {
            float *st = reinterpret_cast<float *>(stage);
#pragma unroll
            for (int r = 0; r < kPre; ++r)
                if (pre_off[r] >= 0) st[pre_off[r]] = pre[r];
            for (int u = tid + kPre * kTmaThreads; u < nfix; u += kTmaThreads) {
                int so;
                long long g;
                tma_fix_item(fix, tl, u, p, &so, &g);
                st[so] = __ldg(qin + g);
            }
            __syncthreads();
        }
        const int x = tl.x0 + lx, y = tl.y0 + ly;
        if (x < p.nx && y < p.ny)
            step_pair_staged<FORCED>(reinterpret_cast<const float *>(stage),
                                     reinterpret_cast<const float *>(stage + kTmaQRegion), qout, p, lx, ly, x, y);
        __syncthreads();  // every thread is done with this stage
        if (tid == 0 && t + 2 * G < ntiles) {
            // order this CTA's generic-proxy accesses of the stage before the
            // async-proxy writes of the next copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_issue<FORCED>(stage, bar, &mq, &mf, t + 2 * G, tiles_x);
        }
    }
    if (!ok) {
        if (tid == 0) {
            if (p.err) atomicOr(p.err, kTmaErrTimeout);
            // let the copies this CTA issued land before it leaves: tiles k
            // and k + 1 (where they exist) are the outstanding ones
            int kk = k;
            for (int t = blockIdx.x + k * G; t < ntiles && kk < k + 2 && !unarmed; t += G, ++kk)
                mbar_wait(bar0 + 8 * (kk & 1), (kk >> 1) & 1);
        }
        __syncthreads();
    }
}

}  // namespace rlbk
