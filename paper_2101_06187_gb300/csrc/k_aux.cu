// k_aux.cu -- kernels off the per-step path: initialisation (step (a) of
// Sec. 3.3), the global conservation reduction, the stirring-force draw and
// synthesis (Sec. 5), population encode/decode, and the energy spectrum
// (Sec. 4).
#include <math.h>

#include <algorithm>

#include "forcing.cuh"
#include "rlbm_internal.h"

namespace rlbk {

size_t storage_bytes(int dtype) { return dtype == RLBM_F64 ? 8 : dtype == RLBM_F32 ? 4 : 2; }
size_t compute_bytes(int dtype) { return dtype == RLBM_F64 ? 8 : 4; }

template <typename TS>
__device__ __forceinline__ double load_any(const TS *p) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) return (double)__bfloat162float(*p);
    else if constexpr (std::is_same<TS, __half>::value) return (double)__half2float(*p);
    else return (double)*p;
}

template <typename TS>
__device__ __forceinline__ TS store_any(double x) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) return __float2bfloat16_rn((float)x);
    else if constexpr (std::is_same<TS, __half>::value) return __float2half_rn((float)x);
    else return (TS)x;
}

#define RLBM_DISPATCH_STORAGE(dtype, TS, ...)            \
    switch (dtype) {                                       \
    case RLBM_F64: { using TS = double; __VA_ARGS__; break; }        \
    case RLBM_F32: { using TS = float; __VA_ARGS__; break; }         \
    case RLBM_BF16: { using TS = __nv_bfloat16; __VA_ARGS__; break; } \
    default: { using TS = __half; __VA_ARGS__; break; }              \
    }

// ---------------------------------------------------------------- initialisation
// f_c = f_eq,c(eps, v) in deviation form (see collide_node):
// q_c = [eps - eps0 + eps gamma^2 (4 xi + 10 xi^2 - 2 |v|^2)] / s, xi = c . v.
template <typename TS, typename TC>
__global__ void k_init(TS *q, StepParams p, const double *eps, const double *vx, const double *vy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long i = (long long)y * p.nx + x;
    const TC de = eps ? (TC)(eps[i] - p.eps0) : (TC)0;  // deviation formed in FP64, then rounded once
    const TC e = par_eps0<TC>(p) + de;
    const TC a = vx ? (TC)vx[i] : (TC)0, b = vy ? (TC)vy[i] : (TC)0;
    const TC v2 = a * a + b * b;
    const TC eg2 = e / ((TC)1 - v2);
    const TC inv_s = par_inv_scale<TC>(p);
    const long long n = (long long)y * p.pitch + x;
    static_for<0, NC>([&](auto C) {
        constexpr int c = decltype(C)::value;
        const TC xi = (TC)cls_cx(c) * a + (TC)cls_cy(c) * b;
        const TC qc = (de + eg2 * ((TC)4 * xi + (TC)10 * xi * xi - (TC)2 * v2)) * inv_s;
        q[(long long)c * p.plane + n] = to_storage<TS, TC>(qc);
    });
}

cudaError_t launch_init(int dtype, void *q, const StepParams &p, const double *eps, const double *vx,
                        const double *vy, cudaStream_t s) {
    dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
    if (dtype == RLBM_F64)
        k_init<double, double><<<g, b, 0, s>>>(static_cast<double *>(q), p, eps, vx, vy);
    else if (dtype == RLBM_F32)
        k_init<float, float><<<g, b, 0, s>>>(static_cast<float *>(q), p, eps, vx, vy);
    else if (dtype == RLBM_BF16)
        k_init<__nv_bfloat16, float><<<g, b, 0, s>>>(static_cast<__nv_bfloat16 *>(q), p, eps, vx, vy);
    else
        k_init<__half, float><<<g, b, 0, s>>>(static_cast<__half *>(q), p, eps, vx, vy);
    return cudaGetLastError();
}

// Count initial-field entries with no physical frame: eps <= 0 or not
// finite, |v| >= 1 or not finite (any pointer may be NULL: default value).
__global__ void k_check_fields(const double *eps, const double *vx, const double *vy, long long n, int *bad) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double e = eps ? eps[i] : 1.0;
    const double a = vx ? vx[i] : 0.0, b = vy ? vy[i] : 0.0;
    const bool ok = isfinite(e) && e > 0.0 && isfinite(a) && isfinite(b) && (a * a + b * b < 1.0);
    if (!ok) atomicAdd(bad, 1);
}

cudaError_t launch_check_fields(const double *eps, const double *vx, const double *vy, long long n, int *bad,
                                cudaStream_t s) {
    k_check_fields<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(eps, vx, vy, n, bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- conservation totals
// Fixed-order, compensated FP64 reduction of the per-block partials: thread
// t sums partials t, t+256, ... with Neumaier's compensated summation (the
// rounding error of every addition is carried in a second accumulator),
// then a tree over the 256 threads on (sum, compensation) pairs.
struct KSum {
    double s, c;
};

__device__ __forceinline__ KSum ksum_add(KSum a, double x) {
    const double t = a.s + x;
    const double e = (fabs(a.s) >= fabs(x)) ? (a.s - t) + x : (x - t) + a.s;
    return {t, a.c + e};
}

__device__ __forceinline__ KSum ksum_merge(KSum a, KSum b) {
    KSum r = ksum_add(a, b.s);
    r.c += b.c;
    return r;
}

__global__ void k_reduce_partials(const double *partials, int nblocks, double base_E, double *totals) {
    __shared__ KSum red[3][256];
    const int t = threadIdx.x;
    KSum a[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    for (int i = t; i < nblocks; i += 256)
        for (int j = 0; j < 3; ++j) a[j] = ksum_add(a[j], partials[3 * i + j]);
    for (int j = 0; j < 3; ++j) red[j][t] = a[j];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h)
            for (int j = 0; j < 3; ++j) red[j][t] = ksum_merge(red[j][t], red[j][t + h]);
        __syncthreads();
    }
    if (t == 0) {
        const KSum e = ksum_add(red[0][0], base_E);
        totals[0] = e.s + e.c;
        totals[1] = red[1][0].s + red[1][0].c;
        totals[2] = red[2][0].s + red[2][0].c;
    }
}

cudaError_t launch_reduce_partials(const double *partials, int nblocks, double base_E, double *totals,
                                   cudaStream_t s) {
    k_reduce_partials<<<1, 256, 0, s>>>(partials, nblocks, base_E, totals);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- stirring force
template <typename TC>
struct C4 {
    TC ax, bx, ay, by;
};

// Mode m of epoch `epoch`: magnitude, phase and in-plane direction from two
// Philox4x32-10 blocks keyed by the seed (Sec. 5's random stirring).
template <typename TC>
__device__ __forceinline__ void draw_mode(Mode *modes, C4<TC> *coef, int m, double amp, unsigned long long seed,
                                          unsigned long long epoch) {
    const unsigned int k0 = (unsigned int)(seed & 0xffffffffull), k1 = (unsigned int)(seed >> 32);
    U4 c0 = {{(unsigned int)epoch, (unsigned int)m, 0u, 0u}};
    U4 c1 = {{(unsigned int)epoch, (unsigned int)m, 1u, 0u}};
    const U4 o0 = philox4x32_10(c0, k0, k1);
    const U4 o1 = philox4x32_10(c1, k0, k1);
    const double r = amp * u01_53(o0.w[0], o0.w[1]);
    const double ph = 2.0 * M_PI * u01_53(o0.w[2], o0.w[3]);
    const double th = 2.0 * M_PI * u01_53(o1.w[0], o1.w[1]);
    double sph, cph, sth, cth;
    sincos(ph, &sph, &cph);
    sincos(th, &sth, &cth);
    Mode md = modes[m];
    md.ax = 2.0 * r * cth * cph;
    md.bx = 2.0 * r * cth * sph;
    md.ay = 2.0 * r * sth * cph;
    md.by = 2.0 * r * sth * sph;
    modes[m] = md;
    coef[m] = C4<TC>{(TC)md.ax, (TC)md.bx, (TC)md.ay, (TC)md.by};
}

template <typename TC>
__global__ void k_draw_modes(Mode *modes, C4<TC> *coef, int nmodes, double amp, unsigned long long seed,
                             unsigned long long epoch) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmodes) return;
    draw_mode<TC>(modes, coef, m, amp, seed, epoch);
}

cudaError_t launch_draw_modes(int dtype, Mode *modes, void *coef, int nmodes, double amp, unsigned long long seed,
                              unsigned long long epoch, cudaStream_t s) {
    if (nmodes <= 0) return cudaSuccess;
    if (dtype == RLBM_F64)
        k_draw_modes<double><<<(nmodes + 127) / 128, 128, 0, s>>>(modes, static_cast<C4<double> *>(coef), nmodes, amp,
                                                                  seed, epoch);
    else
        k_draw_modes<float><<<(nmodes + 127) / 128, 128, 0, s>>>(modes, static_cast<C4<float> *>(coef), nmodes, amp,
                                                                 seed, epoch);
    return cudaGetLastError();
}


// tw[j] = (cos, sin)(2 pi j / n), j < n.
template <typename TC>
__global__ void k_twiddles(C2<TC> *tw, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sv, cv;
    sincospi(2.0 * (double)j / (double)n, &sv, &cv);
    tw[j].c = (TC)cv;
    tw[j].s = (TC)sv;
}

cudaError_t launch_twiddles(int dtype, void *tw, int n, cudaStream_t s) {
    if (dtype == RLBM_F64)
        k_twiddles<double><<<(n + 255) / 256, 256, 0, s>>>(static_cast<C2<double> *>(tw), n);
    else
        k_twiddles<float><<<(n + 255) / 256, 256, 0, s>>>(static_cast<C2<float> *>(tw), n);
    return cudaGetLastError();
}

// Per-mode phase tables: X[m][x] = e^{2 pi i kx_m (x + x0) / nxg} and
// Y[m][y] = e^{2 pi i ky_m (y + y0) / nyg}, read from the twiddle tables of
// the global sizes nxg, nyg with the phase index reduced in integers
// ((k (x + x0)) mod nxg), so the argument is exact at any lattice size.  A
// whole lattice has x0 = y0 = 0 and nxg, nyg its own sizes; a slab of a
// decomposed lattice its global offset (y0 may be negative: halo rows) and
// the global sizes.  Built once per lattice (or force frame).
template <typename TC>
__global__ void k_mode_tables(C2<TC> *X, C2<TC> *Y, const Mode *__restrict__ modes, int nmodes,
                              const C2<TC> *__restrict__ twx, const C2<TC> *__restrict__ twy, int nx, int ny,
                              int nxg, int nyg, int x0, int y0) {
    const int m = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmodes) return;
    if (i < nx) {
        const long long k = ((long long)modes[m].kx % nxg + nxg) % nxg;
        const long long g = (((long long)i + x0) % nxg + nxg) % nxg;
        X[(long long)m * nx + i] = twx[(k * g) % nxg];
    }
    if (i < ny) {
        const long long k = ((long long)modes[m].ky % nyg + nyg) % nyg;
        const long long g = (((long long)i + y0) % nyg + nyg) % nyg;
        Y[(long long)m * ny + i] = twy[(k * g) % nyg];
    }
}

cudaError_t launch_mode_tables(int dtype, void *X, void *Y, const Mode *modes, int nmodes, const void *twx,
                               const void *twy, int nx, int ny, int nxg, int nyg, int x0, int y0, cudaStream_t s) {
    if (nmodes <= 0) return cudaSuccess;
    const dim3 g((std::max(nx, ny) + 255) / 256, nmodes, 1);
    if (dtype == RLBM_F64)
        k_mode_tables<double><<<g, 256, 0, s>>>(static_cast<C2<double> *>(X), static_cast<C2<double> *>(Y), modes,
                                                nmodes, static_cast<const C2<double> *>(twx),
                                                static_cast<const C2<double> *>(twy), nx, ny, nxg, nyg, x0, y0);
    else
        k_mode_tables<float><<<g, 256, 0, s>>>(static_cast<C2<float> *>(X), static_cast<C2<float> *>(Y), modes,
                                               nmodes, static_cast<const C2<float> *>(twx),
                                               static_cast<const C2<float> *>(twy), nx, ny, nxg, nyg, x0, y0);
    return cudaGetLastError();
}

// F(x) = sum_m [a cos psi - b sin psi] = Re sum_m (a + i b) e^{i psi},
// psi = 2 pi (kx x/nx + ky y/ny), e^{i psi} = X[m][x] Y[m][y].  The modes
// come in runs of equal ky (enumerated ky ascending), which share Y, so the
// synthesis is separable: per run j and column x the row sums
//     G_j(x) = sum_{m in run j} (a_m + i b_m) X[m][x]      (k_force_rows)
// and per node F = Re sum_j G_j(x) Y_j(y)                   (k_synth_force):
// 4 multiply-adds per run and node instead of 12 per mode and node.
template <typename TC>
__device__ __forceinline__ void force_row(C4<TC> *G, const C4<TC> *__restrict__ coef,
                                          const int *__restrict__ run_start, const C2<TC> *__restrict__ X, int nx,
                                          int x, int j) {
    TC xr = 0, xi = 0, yr = 0, yi = 0;
    for (int m = run_start[j]; m < run_start[j + 1]; ++m) {
        const C4<TC> c = coef[m];
        const C2<TC> a = X[(long long)m * nx + x];
        xr += c.ax * a.c - c.bx * a.s;
        xi += c.ax * a.s + c.bx * a.c;
        yr += c.ay * a.c - c.by * a.s;
        yi += c.ay * a.s + c.by * a.c;
    }
    G[(long long)j * nx + x] = C4<TC>{xr, xi, yr, yi};
}

template <typename TC>
__global__ void k_force_rows(C4<TC> *G, const C4<TC> *__restrict__ coef, const int *__restrict__ run_start,
                             const C2<TC> *__restrict__ X, int nx) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    force_row<TC>(G, coef, run_start, X, nx, x, blockIdx.y);
}

// One thread per column x and SYNTH_ROWS consecutive rows: the row sums
// G_j(x) are read once per run and reused for every row of the strip.
constexpr int SYNTH_ROWS = 8;

template <typename TC>
__device__ __forceinline__ void synth_strip(TC *F, const C4<TC> *__restrict__ G, const int *__restrict__ run_start,
                                            int nruns, const C2<TC> *__restrict__ Y, const StepParams &p, int x,
                                            int y0) {
    const int rows = min(SYNTH_ROWS, p.ny - y0);
    TC fx[SYNTH_ROWS], fy[SYNTH_ROWS];
#pragma unroll
    for (int r = 0; r < SYNTH_ROWS; ++r) fx[r] = fy[r] = 0;
    for (int j = 0; j < nruns; ++j) {
        const C4<TC> g = G[(long long)j * p.nx + x];
        const C2<TC> *Yj = Y + (long long)run_start[j] * p.ny + y0;
#pragma unroll
        for (int r = 0; r < SYNTH_ROWS; ++r) {
            if (r < rows) {
                const C2<TC> b = Yj[r];
                fx[r] += g.ax * b.c - g.bx * b.s;
                fy[r] += g.ay * b.c - g.by * b.s;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < SYNTH_ROWS; ++r) {
        if (r < rows) {
            const long long n = (long long)(y0 + r) * p.pitch + x;
            F[n] = fx[r];
            F[p.plane + n] = fy[r];
        }
    }
}

template <typename TC>
__global__ void k_synth_force(TC *F, const C4<TC> *__restrict__ G, const int *__restrict__ run_start, int nruns,
                              const C2<TC> *__restrict__ Y, StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * SYNTH_ROWS;
    if (x >= p.nx || y0 >= p.ny) return;
    synth_strip<TC>(F, G, run_start, nruns, Y, p, x, y0);
}

cudaError_t launch_synth_force(int dtype, void *F, const void *coef, int nmodes, const int *run_start, int nruns,
                               void *G, const void *X, const void *Y, const StepParams &p, cudaStream_t s) {
    if (nmodes <= 0 || nruns <= 0) return cudaSuccess;
    const dim3 gr((p.nx + 255) / 256, nruns, 1);
    const dim3 block(32, 8, 1);
    const dim3 grid((p.nx + 31) / 32, (p.ny + 8 * SYNTH_ROWS - 1) / (8 * SYNTH_ROWS), 1);
    if (dtype == RLBM_F64) {
        k_force_rows<double><<<gr, 256, 0, s>>>(static_cast<C4<double> *>(G), static_cast<const C4<double> *>(coef),
                                                run_start, static_cast<const C2<double> *>(X), p.nx);
        k_synth_force<double><<<grid, block, 0, s>>>(static_cast<double *>(F), static_cast<const C4<double> *>(G),
                                                     run_start, nruns, static_cast<const C2<double> *>(Y), p);
    } else {
        k_force_rows<float><<<gr, 256, 0, s>>>(static_cast<C4<float> *>(G), static_cast<const C4<float> *>(coef),
                                               run_start, static_cast<const C2<float> *>(X), p.nx);
        k_synth_force<float><<<grid, block, 0, s>>>(static_cast<float *>(F), static_cast<const C4<float> *>(G),
                                                    run_start, nruns, static_cast<const C2<float> *>(Y), p);
    }
    return cudaGetLastError();
}

// Ensemble-wide synthesis: the kernels above for every job whose redraw
// period divides `step` (job = blockIdx.y for the draw, blockIdx.z for the
// other two), each on its own lattice's sizes, so a member's force is the
// one launch_draw_modes + launch_synth_force give it.
__device__ __forceinline__ bool job_redraws(const ForceJob &j, long long step) { return step % j.period == 0; }

template <typename TC>
__global__ void k_draw_modes_jobs(const ForceJob *__restrict__ jobs, long long step) {
    const ForceJob &j = jobs[blockIdx.y];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= j.nmodes || !job_redraws(j, step)) return;
    draw_mode<TC>(j.modes, static_cast<C4<TC> *>(j.coef), m, j.amp, j.seed, (unsigned long long)(step / j.period));
}

template <typename TC>
__global__ void k_force_rows_jobs(const ForceJob *__restrict__ jobs, long long step) {
    const ForceJob &j = jobs[blockIdx.z];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= j.p.nx || (int)blockIdx.y >= j.nruns || !job_redraws(j, step)) return;
    force_row<TC>(static_cast<C4<TC> *>(j.G), static_cast<const C4<TC> *>(j.coef), j.run_start,
                  static_cast<const C2<TC> *>(j.X), j.p.nx, x, blockIdx.y);
}

template <typename TC>
__global__ void k_synth_force_jobs(const ForceJob *__restrict__ jobs, long long step) {
    const ForceJob &j = jobs[blockIdx.z];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * SYNTH_ROWS;
    if (x >= j.p.nx || y0 >= j.p.ny || !job_redraws(j, step)) return;
    synth_strip<TC>(static_cast<TC *>(j.F), static_cast<const C4<TC> *>(j.G), j.run_start, j.nruns,
                    static_cast<const C2<TC> *>(j.Y), j.p, x, y0);
}

cudaError_t launch_force_jobs(int dtype, const ForceJob *jobs, int njobs, int max_nmodes, int max_nruns, int max_nx,
                              int max_ny, long long step, cudaStream_t s) {
    if (njobs <= 0 || max_nmodes <= 0 || max_nruns <= 0) return cudaSuccess;
    if (njobs > 65535 || max_nruns > 65535) return cudaErrorInvalidValue;
    const dim3 gd((max_nmodes + 127) / 128, njobs, 1);
    const dim3 gr((max_nx + 255) / 256, max_nruns, njobs);
    const dim3 block(32, 8, 1);
    const dim3 gs((max_nx + 31) / 32, (max_ny + 8 * SYNTH_ROWS - 1) / (8 * SYNTH_ROWS), njobs);
    if (dtype == RLBM_F64) {
        k_draw_modes_jobs<double><<<gd, 128, 0, s>>>(jobs, step);
        k_force_rows_jobs<double><<<gr, 256, 0, s>>>(jobs, step);
        k_synth_force_jobs<double><<<gs, block, 0, s>>>(jobs, step);
    } else {
        k_draw_modes_jobs<float><<<gd, 128, 0, s>>>(jobs, step);
        k_force_rows_jobs<float><<<gr, 256, 0, s>>>(jobs, step);
        k_synth_force_jobs<float><<<gs, block, 0, s>>>(jobs, step);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- population encode / decode
template <typename TS>
__global__ void k_decode_class(const TS *q, int c, StepParams p, double W, double *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const double qc = load_any<TS>(q + (long long)c * p.plane + (long long)y * p.pitch + x);
    out[(long long)y * p.nx + x] = W * (p.eps0 + p.scale * qc);
}

template <typename TS>
__global__ void k_encode_class(TS *q, int c, StepParams p, double W, const double *in) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const double f = in[(long long)y * p.nx + x];
    q[(long long)c * p.plane + (long long)y * p.pitch + x] = store_any<TS>((f / W - p.eps0) / p.scale);
}

cudaError_t launch_decode_class(int dtype, const void *q, int c, double W, const StepParams &p, double *out,
                                cudaStream_t s) {
    dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
    RLBM_DISPATCH_STORAGE(dtype, TS, k_decode_class<TS><<<g, b, 0, s>>>(static_cast<const TS *>(q), c, p, W, out));
    return cudaGetLastError();
}

cudaError_t launch_encode_class(int dtype, void *q, int c, double W, const StepParams &p, const double *in,
                                cudaStream_t s) {
    dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
    RLBM_DISPATCH_STORAGE(dtype, TS, k_encode_class<TS><<<g, b, 0, s>>>(static_cast<TS *>(q), c, p, W, in));
    return cudaGetLastError();
}

template <typename TC>
__global__ void k_force_to_f64(const TC *F, int comp, StepParams p, double *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    out[(long long)y * p.nx + x] = (double)F[comp * p.plane + (long long)y * p.pitch + x];
}

cudaError_t launch_force_to_f64(int dtype, const void *F, int comp, const StepParams &p, double *out,
                                cudaStream_t s) {
    dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
    if (dtype == RLBM_F64)
        k_force_to_f64<double><<<g, b, 0, s>>>(static_cast<const double *>(F), comp, p, out);
    else
        k_force_to_f64<float><<<g, b, 0, s>>>(static_cast<const float *>(F), comp, p, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- energy spectrum
// z = v_x + i v_y is transformed once (2D DFT, FP64); since every shell is
// symmetric under k -> -k, sum_shell |X|^2 + |Y|^2 = sum_shell |Z|^2 with
// X, Y the transforms of v_x, v_y, so E(n) = 1/2 sum_shell |Z|^2 / (nx ny)^2.
// Lines of length 2^m <= 8192 use an in-shared-memory radix-2 FFT; other
// lengths a direct DFT with an integer-reduced twiddle index.
struct Z2 {
    double re, im;
};

__device__ __forceinline__ Z2 zmul(Z2 a, Z2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Forward twiddles w[k] = exp(-2 pi i k / n), k < n.
__global__ void k_dft_twiddles(Z2 *w, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    w[k] = {c, -s};
}

__global__ void k_pack_z(const double *vx, const double *vy, Z2 *z, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) z[i] = {vx[i], vy[i]};
}

// One line per block: elements line*ls + j*es, j < n.
__global__ void k_fft_lines(Z2 *data, int n, int log2n, long long es, long long ls, const Z2 *__restrict__ w) {
    extern __shared__ Z2 sh[];
    Z2 *base = data + (long long)blockIdx.x * ls;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int r = (int)(__brev((unsigned int)j) >> (32 - log2n));
        sh[r] = base[(long long)j * es];
    }
    __syncthreads();
    for (int h = 1; h < n; h <<= 1) {
        const int stride = n / (2 * h);
        for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
            const int k = i % h;
            const int pos = (i / h) * 2 * h + k;
            const Z2 a = sh[pos];
            const Z2 b = zmul(sh[pos + h], w[k * stride]);
            sh[pos] = {a.re + b.re, a.im + b.im};
            sh[pos + h] = {a.re - b.re, a.im - b.im};
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) base[(long long)j * es] = sh[j];
}

__global__ void k_dft_lines(Z2 *data, int n, long long es, long long ls, const Z2 *__restrict__ w) {
    extern __shared__ Z2 sh[];
    Z2 *base = data + (long long)blockIdx.x * ls;
    for (int j = threadIdx.x; j < n; j += blockDim.x) sh[j] = base[(long long)j * es];
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        Z2 acc = {0.0, 0.0};
        long long idx = 0;
        for (int j = 0; j < n; ++j) {
            const Z2 t = zmul(sh[j], w[idx]);
            acc.re += t.re;
            acc.im += t.im;
            idx += k;
            if (idx >= n) idx -= n;
        }
        base[(long long)k * es] = acc;  // reads come from sh only
    }
}

__global__ void k_shell_bin(const Z2 *z, int nx, int ny, int nshells, double *Ek) {
    extern __shared__ double hist[];
    for (int i = threadIdx.x; i < nshells; i += blockDim.x) hist[i] = 0.0;
    __syncthreads();
    const long long count = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const int jy = (int)(i / nx), jx = (int)(i % nx);
        const double kx = (jx < (nx + 1) / 2) ? jx : jx - nx;
        const double ky = (jy < (ny + 1) / 2) ? jy : jy - ny;
        const int sh = (int)floor(sqrt(kx * kx + ky * ky) + 0.5);
        if (sh < nshells) atomicAdd(&hist[sh], z[i].re * z[i].re + z[i].im * z[i].im);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nshells; i += blockDim.x)
        if (hist[i] != 0.0) atomicAdd(&Ek[i], hist[i]);
}

// Sum of |Z(k)|^2 over the modes with |k| < kf (signed integer wavenumbers).
__global__ void k_band_sum(const Z2 *z, int nx, int ny, double kf, double *out) {
    __shared__ double red[256];
    double acc = 0.0;
    const long long count = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const int jy = (int)(i / nx), jx = (int)(i % nx);
        const double kx = (jx < (nx + 1) / 2) ? jx : jx - nx;
        const double ky = (jy < (ny + 1) / 2) ? jy : jy - ny;
        if (kx * kx + ky * ky < kf * kf) acc += z[i].re * z[i].re + z[i].im * z[i].im;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// Per-shell running sums of E and E^2 for time statistics of the spectrum.
__global__ void k_accumulate(const double *E, int n, double *sum, double *sq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        sum[i] += E[i];
        sq[i] += E[i] * E[i];
    }
}

cudaError_t launch_accumulate(const double *E, int n, double *sum, double *sq, cudaStream_t s) {
    k_accumulate<<<(n + 255) / 256, 256, 0, s>>>(E, n, sum, sq);
    return cudaGetLastError();
}

__global__ void k_scale(double *a, int n, double f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] *= f;
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
static int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

size_t spectrum_work_doubles(int nx, int ny) { return 2 * ((size_t)nx * ny + (size_t)nx + (size_t)ny); }

static cudaError_t transform_lines(Z2 *z, int n, int lines, long long es, long long ls, Z2 *w, cudaStream_t s) {
    const size_t smem = (size_t)n * sizeof(Z2);
    k_dft_twiddles<<<(n + 255) / 256, 256, 0, s>>>(w, n);
    cudaError_t e;
    if (is_pow2(n)) {
        e = cudaFuncSetAttribute(k_fft_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_fft_lines<<<lines, 512, smem, s>>>(z, n, ilog2(n), es, ls, w);
    } else {
        e = cudaFuncSetAttribute(k_dft_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_dft_lines<<<lines, 256, smem, s>>>(z, n, es, ls, w);
    }
    return cudaGetLastError();
}

static cudaError_t transform_2d(const double *vx, const double *vy, int nx, int ny, double *work, cudaStream_t s) {
    Z2 *z = reinterpret_cast<Z2 *>(work);
    Z2 *wx = z + (size_t)nx * ny;
    Z2 *wy = wx + nx;
    const long long count = (long long)nx * ny;
    k_pack_z<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(vx, vy, z, count);
    cudaError_t e = transform_lines(z, nx, ny, 1, nx, wx, s);  // rows
    if (e != cudaSuccess) return e;
    return transform_lines(z, ny, nx, nx, 1, wy, s);  // columns
}

// Mean square of the velocity with every mode |k| >= kf removed:
// <|v_f|^2> = sum_{|k| < kf} |v_hat(k)|^2 = sum_{|k| < kf} |Z(k)|^2 / (nx ny)^2
// (the set |k| < kf is symmetric under k -> -k, as for the shells).
cudaError_t launch_band_power(const double *vx, const double *vy, int nx, int ny, double kf, double *work,
                              double *out, cudaStream_t s) {
    cudaError_t e = transform_2d(vx, vy, nx, ny, work, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(out, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_band_sum<<<304, 256, 0, s>>>(reinterpret_cast<const Z2 *>(work), nx, ny, kf, out);
    const double count = (double)nx * ny;
    k_scale<<<1, 32, 0, s>>>(out, 1, 1.0 / (count * count));
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const double *vx, const double *vy, int nx, int ny, int nshells, double *work,
                            double *Ek, cudaStream_t s) {
    Z2 *z = reinterpret_cast<Z2 *>(work);
    const long long count = (long long)nx * ny;
    cudaError_t e = transform_2d(vx, vy, nx, ny, work, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(Ek, 0, sizeof(double) * nshells, s);
    if (e != cudaSuccess) return e;
    k_shell_bin<<<304, 256, sizeof(double) * nshells, s>>>(z, nx, ny, nshells, Ek);
    const double f = 0.5 / ((double)count * (double)count);
    k_scale<<<(nshells + 255) / 256, 256, 0, s>>>(Ek, nshells, f);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- 3D spectra
// The three velocity components as two complex fields Z1 = vx + i vy and
// Z2 = vz, each transformed along x, y and z; over a shell (symmetric under
// k -> -k) the sum of |Z1|^2 + |Z2|^2 is the sum of |v_hat_x|^2 + |v_hat_y|^2
// + |v_hat_z|^2, times vol^2.
__global__ void k_pack_z3(const double *vx, const double *vy, const double *vz, Z2 *z1, Z2 *z2, long long count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        z1[i] = {vx[i], vy[i]};
        z2[i] = {vz[i], 0.0};
    }
}

__device__ __forceinline__ double signed_k(int j, int n) { return (j < (n + 1) / 2) ? j : j - n; }

__global__ void k_shell_bin3(const Z2 *z1, const Z2 *z2, int nx, int ny, int nz, int nshells, double *Ek) {
    extern __shared__ double hist[];
    for (int i = threadIdx.x; i < nshells; i += blockDim.x) hist[i] = 0.0;
    __syncthreads();
    const long long count = (long long)nx * ny * nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const int jx = (int)(i % nx), jy = (int)((i / nx) % ny), jz = (int)(i / ((long long)nx * ny));
        const double kx = signed_k(jx, nx), ky = signed_k(jy, ny), kz = signed_k(jz, nz);
        const int sh = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);
        if (sh < nshells)
            atomicAdd(&hist[sh], z1[i].re * z1[i].re + z1[i].im * z1[i].im + z2[i].re * z2[i].re + z2[i].im * z2[i].im);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nshells; i += blockDim.x)
        if (hist[i] != 0.0) atomicAdd(&Ek[i], hist[i]);
}

__global__ void k_band_sum3(const Z2 *z1, const Z2 *z2, int nx, int ny, int nz, double kf, double *out) {
    __shared__ double red[256];
    double acc = 0.0;
    const long long count = (long long)nx * ny * nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const int jx = (int)(i % nx), jy = (int)((i / nx) % ny), jz = (int)(i / ((long long)nx * ny));
        const double kx = signed_k(jx, nx), ky = signed_k(jy, ny), kz = signed_k(jz, nz);
        if (kx * kx + ky * ky + kz * kz < kf * kf)
            acc += z1[i].re * z1[i].re + z1[i].im * z1[i].im + z2[i].re * z2[i].re + z2[i].im * z2[i].im;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

size_t spectrum_work_doubles3(int nx, int ny, int nz) {
    return 2 * (2 * (size_t)nx * ny * nz + (size_t)nx + (size_t)ny + (size_t)nz);
}

static cudaError_t transform_3d_one(Z2 *z, int nx, int ny, int nz, Z2 *w, cudaStream_t s) {
    const long long slab = (long long)nx * ny;
    cudaError_t e = transform_lines(z, nx, ny * nz, 1, nx, w, s);  // x lines
    for (int k = 0; k < nz && e == cudaSuccess; ++k)                  // y lines, slab by slab
        e = transform_lines(z + k * slab, ny, nx, nx, 1, w + nx, s);
    if (e == cudaSuccess) e = transform_lines(z, nz, (int)slab, slab, 1, w + nx + ny, s);  // z lines
    return e;
}

static cudaError_t transform_3d(const double *vx, const double *vy, const double *vz, int nx, int ny, int nz,
                                double *work, cudaStream_t s) {
    const long long count = (long long)nx * ny * nz;
    Z2 *z1 = reinterpret_cast<Z2 *>(work);
    Z2 *z2 = z1 + count;
    Z2 *w = z2 + count;
    k_pack_z3<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(vx, vy, vz, z1, z2, count);
    cudaError_t e = transform_3d_one(z1, nx, ny, nz, w, s);
    if (e == cudaSuccess) e = transform_3d_one(z2, nx, ny, nz, w, s);
    return e;
}

cudaError_t launch_spectrum3(const double *vx, const double *vy, const double *vz, int nx, int ny, int nz, int nshells,
                             double *work, double *Ek, cudaStream_t s) {
    const long long count = (long long)nx * ny * nz;
    cudaError_t e = transform_3d(vx, vy, vz, nx, ny, nz, work, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(Ek, 0, sizeof(double) * nshells, s);
    if (e != cudaSuccess) return e;
    const Z2 *z1 = reinterpret_cast<const Z2 *>(work);
    k_shell_bin3<<<304, 256, sizeof(double) * nshells, s>>>(z1, z1 + count, nx, ny, nz, nshells, Ek);
    k_scale<<<(nshells + 255) / 256, 256, 0, s>>>(Ek, nshells, 0.5 / ((double)count * (double)count));
    return cudaGetLastError();
}

cudaError_t launch_band_power3(const double *vx, const double *vy, const double *vz, int nx, int ny, int nz, double kf,
                               double *work, double *out, cudaStream_t s) {
    const long long count = (long long)nx * ny * nz;
    cudaError_t e = transform_3d(vx, vy, vz, nx, ny, nz, work, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(out, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    const Z2 *z1 = reinterpret_cast<const Z2 *>(work);
    k_band_sum3<<<304, 256, 0, s>>>(z1, z1 + count, nx, ny, nz, kf, out);
    k_scale<<<1, 32, 0, s>>>(out, 1, 1.0 / ((double)count * (double)count));
    return cudaGetLastError();
}

}  // namespace rlbk
