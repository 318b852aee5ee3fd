// k_step_fused2.cuh -- two time steps per launch (temporal blocking) of the
// fused stream + collide + force update, in packed FP32 lanes.
//
// A CTA owns a TW x TH tile of output nodes.  Step t -> t+1 is computed on
// the tile grown by the one-cell pull halo of the next step (Sec. 3.2: at
// cfl <= 1 a class pulls from the 3 x 3 neighbourhood), i.e. on (TW + 4) x
// (TH + 2) nodes -- two extra columns a side, so every node pair starts on
// an even column and loads stay 8-byte aligned -- and kept in shared memory
// in the storage type; step t+1 -> t+2 then pulls from shared memory and
// writes the tile.  Per two steps the state is read from and written to HBM
// once: half the traffic of two single-step launches, for 10-20% more
// arithmetic (the halo nodes are updated by every tile that needs them: 16%
// for 64 x 8 tiles).  Both steps run the same per-node arithmetic as
// k_step_pair in the same streaming mode (CFL 1, or 0 < cfl < 1 with the
// launch's weights), and the intermediate state is rounded to the storage
// type exactly as a single step stores it, so two steps here equal two
// single steps bit for bit.  The force field is the same for both steps:
// the host launches this kernel only for step pairs inside one forcing
// epoch.
#pragma once

#include "k_step_pair.cuh"

namespace rlbk {

// Shared-memory reads of the storage type (no read-only-cache path there).
template <typename TS>
__device__ __forceinline__ void lds_run2(const TS *p, float *o) {
    if constexpr (std::is_same<TS, float>::value) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        o[0] = v.x;
        o[1] = v.y;
    } else if constexpr (std::is_same<TS, __half>::value) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        o[0] = v.x;
        o[1] = v.y;
    } else {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
        o[0] = v.x;
        o[1] = v.y;
    }
}
template <typename TS>
__device__ __forceinline__ float lds1(const TS *p) {
    if constexpr (std::is_same<TS, float>::value) return *p;
    else if constexpr (std::is_same<TS, __half>::value) return __half2float(*p);
    else return __bfloat162float(*p);
}

// Pull of the node pair (x0, x0 + 1) from a state laid out as NC planes of
// `plane` elements: rows[k] is the offset of row y - 1 + k, xl and xr the
// columns x0 - 1 and x0 + 2.  SHARED selects shared-memory reads.  SM is
// kStreamCfl1 (corners and weights fixed at compile time) or kStreamSub1
// (0 < cfl < 1: each moving class between its near corner and the cell it
// streams from, with the launch's weights); the same taps, weights and
// operation order as step_pair in that mode.
template <typename TS, typename I, bool SHARED, int SM>
__device__ __forceinline__ void pull_pair(const TS *__restrict__ src, const StepParams &p, I plane,
                                          const I (&rows)[3], I x0, I xl, I xr, pf2 (&q)[NC]) {
    static_assert(SM == kStreamCfl1 || SM == kStreamSub1, "halo-1 streaming modes only");
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        // the class row around the pair: a[1], a[2] = columns x0, x0 + 1; a[0] = x0 - 1 if LEFT;
        // a[3] = x0 + 2 if RIGHT
        auto row = [&](I r, float (&a)[4], auto left, auto right) {
            const TS *base = src + ((I)c * plane + r);
            if constexpr (SHARED) {
                lds_run2<TS>(base + x0, &a[1]);
                if constexpr (decltype(left)::value) a[0] = lds1<TS>(base + xl);
                if constexpr (decltype(right)::value) a[3] = lds1<TS>(base + xr);
            } else {
                load_run<TS, float, 2>(base + x0, &a[1]);
                if constexpr (decltype(left)::value) a[0] = load_q<TS, float>(base + xl);
                if constexpr (decltype(right)::value) a[3] = load_q<TS, float>(base + xr);
            }
        };
        if constexpr (SM == kStreamCfl1) {
            constexpr int ox = cls_ox(c), oy = cls_oy(c);
            constexpr double tx = cls_tx(c), ty = cls_ty(c);
            using L = std::integral_constant<bool, ox == -1>;
            using R = std::integral_constant<bool, ox == 1 || (ox == 0 && tx != 0.0)>;
            float a[4];  // columns x0-1 .. x0+2
            row(rows[oy + 1], a, L{}, R{});
            // a whole-cell shift (weight 1) needs no multiply: 1 * a is a exactly
            pf2 v = (tx == 0.0 && ty == 0.0) ? pf2(a[ox + 1], a[ox + 2])
                                              : pf2((float)((1.0 - tx) * (1.0 - ty))) * pf2(a[ox + 1], a[ox + 2]);
            if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * (1.0 - ty))), pf2(a[ox + 2], a[ox + 3]), v);
            if constexpr (ty != 0.0) {
                float b[4];
                row(rows[oy + 2], b, L{}, R{});
                v = fmadd(pf2((float)((1.0 - tx) * ty)), pf2(b[ox + 1], b[ox + 2]), v);
                if constexpr (tx != 0.0) v = fmadd(pf2((float)(tx * ty)), pf2(b[ox + 2], b[ox + 3]), v);
            }
            q[c] = v;
        } else {
            // near corner (the class's own cell on an axis where it does not move)
            constexpr double cx = cls_cx(c), cy = cls_cy(c);
            constexpr int nx_ = cx > 0 ? -1 : 0, ny_ = cy > 0 ? -1 : 0;
            constexpr bool mx = cx != 0.0, my = cy != 0.0;
            using L = std::integral_constant<bool, mx && nx_ == -1>;
            using R = std::integral_constant<bool, mx && nx_ == 0>;
            float a[4];  // columns x0-1 .. x0+2
            row(rows[ny_ + 1], a, L{}, R{});
            if constexpr (!mx && !my) {
                q[c] = pf2(a[1], a[2]);
            } else {
                pf2 v = pf2(par_wt<float>(p, c, 0)) * pf2(a[nx_ + 1], a[nx_ + 2]);
                if constexpr (mx) v = fmadd(pf2(par_wt<float>(p, c, 1)), pf2(a[nx_ + 2], a[nx_ + 3]), v);
                if constexpr (my) {
                    float b[4];
                    row(rows[ny_ + 2], b, L{}, R{});
                    v = fmadd(pf2(par_wt<float>(p, c, 2)), pf2(b[nx_ + 1], b[nx_ + 2]), v);
                    if constexpr (mx) v = fmadd(pf2(par_wt<float>(p, c, 3)), pf2(b[nx_ + 2], b[nx_ + 3]), v);
                }
                q[c] = v;
            }
        }
    });
}

template <typename I, bool FORCED>
__device__ __forceinline__ void force_pair(const float *__restrict__ F, I plane, I n0, pf2 &Fx, pf2 &Fy) {
    if constexpr (FORCED) {
        float fx[2], fy[2];
        load_run<float, float, 2>(F + n0, fx);
        load_run<float, float, 2>(F + (plane + n0), fy);
        Fx = pf2(fx[0], fx[1]);
        Fy = pf2(fy[0], fy[1]);
    } else {
        Fx = 0.0f;
        Fy = 0.0f;
    }
}

// Shared-memory footprint of one tile's intermediate state.
template <typename TS, int TW, int TH>
constexpr int fused2_smem_bytes() {
    return NC * (TW + 4) * (TH + 2) * (int)sizeof(TS);
}

// a mod n for the window coordinates: one conditional add or subtract for
// a in [-n, 2n), the integer remainder only for lattices narrower than the
// window (where the window wraps more than once).
__device__ __forceinline__ int wrap_window(int a, int n) {
    if (a < 0) a += n;
    else if (a >= n) a -= n;
    if ((unsigned)a < (unsigned)n) return a;
    const int r = a % n;
    return r < 0 ? r + n : r;
}

// Two steps of the TW x TH tile whose first node is (tx0, ty0), by the NT
// threads of a CTA, through the shared window S.  Needs nx even and a
// halo-1 streaming mode SM (cfl <= 1); nodes of the tile past the lattice
// edge are not written.
template <typename TS, bool FORCED, int TW, int TH, int NT, typename I, int SM = kStreamCfl1, bool DFL = false>
__device__ __forceinline__ void fused2_tile(const TS *__restrict__ qin, TS *__restrict__ qout,
                                            const float *__restrict__ F, const StepParams &p, int tx0, int ty0,
                                            TS *__restrict__ S) {
    static_assert(TW % 2 == 0, "tiles hold whole node pairs");
    constexpr int SW = TW + 4, SH = TH + 2, SPLANE = SW * SH;
    constexpr int PW1 = SW / 2, NP1 = PW1 * SH;  // node pairs of the first step
    constexpr int PW2 = TW / 2, NP2 = PW2 * TH;  // node pairs of the second step
    const I plane = (I)p.plane;

    // step t -> t+1 on the window: local (lr, lc) <-> node
    // ((tx0 - 2 + lc) mod nx, (ty0 - 1 + lr) mod ny)
    for (int i = threadIdx.x; i < NP1; i += NT) {
        const int lr = i / PW1, lc = (i - lr * PW1) * 2;
        const int x0 = wrap_window(tx0 - 2 + lc, p.nx), y = wrap_window(ty0 - 1 + lr, p.ny);
        const int ym = (y == 0) ? p.ny - 1 : y - 1;
        const int yp = (y == p.ny - 1) ? 0 : y + 1;
        const int xl = (x0 == 0) ? p.nx - 1 : x0 - 1;
        const int xr = (x0 + 2 == p.nx) ? 0 : x0 + 2;
        const I rows[3] = {(I)ym * (I)p.pitch, (I)y * (I)p.pitch, (I)yp * (I)p.pitch};
        pf2 q[NC];
        pull_pair<TS, I, false, SM>(qin, p, plane, rows, (I)x0, (I)xl, (I)xr, q);
        pf2 Fx, Fy;
        force_pair<I, FORCED>(F, plane, rows[1] + (I)x0, Fx, Fy);
        collide_node<pf2, pf2, FORCED, DFL, std::is_same<TS, float>::value>(q, Fx, Fy, p);
        const unsigned seed =
            rounds_sr<TS>(p) ? sr_pair_seed((unsigned)y * (unsigned)p.nx + (unsigned)x0, q[0].v.x, q[0].v.y) : 0u;
        static_for<0, NC>([&](auto C) {
            constexpr int c = decltype(C)::value;
            store_pair<TS, c>(S + (c * SPLANE + lr * SW + lc), q[c].v.x, q[c].v.y, p, seed);
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
        pf2 q[NC];
        pull_pair<TS, int, true, SM>(S, p, SPLANE, rows, lc, lc - 1, lc + 2, q);
        const I n0 = (I)y * (I)p.pitch + (I)x0;
        pf2 Fx, Fy;
        force_pair<I, FORCED>(F, plane, n0, Fx, Fy);
        collide_node<pf2, pf2, FORCED, DFL, std::is_same<TS, float>::value>(q, Fx, Fy, p);
        const unsigned seed =
            rounds_sr<TS>(p) ? sr_pair_seed((unsigned)y * (unsigned)p.nx + (unsigned)x0, q[0].v.x, q[0].v.y) : 0u;
        static_for<0, NC>([&](auto C) {
            constexpr int c = decltype(C)::value;
            store_pair<TS, c>(qout + ((I)c * plane + n0), q[c].v.x, q[c].v.y, p, seed);
        });
    }
}

// Two steps of the lattice, one TW x TH tile per CTA (blockIdx.x, blockIdx.y).
// DFL: the Landau frame refined to FP64 accuracy (see step_pair).
template <typename TS, bool FORCED, int TW, int TH, int NT, int MINB, typename I, int SM = kStreamCfl1,
          bool DFL = false>
__global__ void __launch_bounds__(NT, MINB)
    k_step_fused2(const TS *__restrict__ qin, TS *__restrict__ qout, const float *__restrict__ F, StepParams p) {
    extern __shared__ __align__(16) unsigned char fused2_smem[];
    fused2_tile<TS, FORCED, TW, TH, NT, I, SM, DFL>(qin, qout, F, p, blockIdx.x * TW, blockIdx.y * TH,
                                                    reinterpret_cast<TS *>(fused2_smem));
}

// Ensemble form: a grid-stride walk over the flat tile list of all members
// (BatchRun descriptors, tiles of TW x TH nodes).  TWO: two steps per tile
// through shared memory, as k_step_fused2; else one step of the tile's node
// pairs with the packed body (the odd step of an odd count).  Members hold
// fewer than 2^31 / 17 elements per plane: 32-bit offsets.
template <typename TS, int TW, int TH, int NT, int MINB, bool TWO>
__global__ void __launch_bounds__(NT, MINB)
    k_step_batch_fused2(const BatchRun *__restrict__ runs, int nruns, int ntiles) {
    extern __shared__ __align__(16) unsigned char fused2_smem[];
    TS *S = reinterpret_cast<TS *>(fused2_smem);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int lo = 0, hi = nruns - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (runs[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchRun &r = runs[lo];
        const int local = t - r.tile0;
        const int tx0 = (local % r.tiles_x) * TW, ty0 = (local / r.tiles_x) * TH;
        const TS *qin = static_cast<const TS *>(r.qin);
        TS *qout = static_cast<TS *>(r.qout);
        const float *F = static_cast<const float *>(r.F);
        if constexpr (TWO) {
            if (F) fused2_tile<TS, true, TW, TH, NT, int>(qin, qout, F, r.p, tx0, ty0, S);
            else fused2_tile<TS, false, TW, TH, NT, int>(qin, qout, nullptr, r.p, tx0, ty0, S);
            __syncthreads();  // the next tile's first step overwrites the window
        } else {
            for (int i = threadIdx.x; i < (TW / 2) * TH; i += NT) {
                const int rr = i / (TW / 2);
                const int x0 = tx0 + (i - rr * (TW / 2)) * 2, y = ty0 + rr;
                if (x0 >= r.p.nx || y >= r.p.ny) continue;
                if (F) step_pair<TS, true, int>(qin, qout, F, r.p, x0, y);
                else step_pair<TS, false, int>(qin, qout, nullptr, r.p, x0, y);
            }
        }
    }
}

}  // namespace rlbk
