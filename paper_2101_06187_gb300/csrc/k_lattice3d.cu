// Launchers of the three-dimensional lattice (k_lattice3d.cuh) for every
// storage form.
#include <algorithm>

#include "k_lattice3d.cuh"
#include "rlbm_internal.h"

namespace rlbk {

// Fixed-order FP64 reduction of the 4-wide block partials, with Neumaier's
// compensated summation (error of each addition carried separately).
__device__ __forceinline__ void ksum4_add(double &s, double &c, double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
}

__global__ void k_reduce_partials4(const double *partials, long long nblocks, double base_E, double *totals) {
    __shared__ double rs[4][256], rc[4][256];
    const int t = threadIdx.x;
    double s[4] = {0.0, 0.0, 0.0, 0.0}, c[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = t; i < nblocks; i += 256)
        for (int j = 0; j < 4; ++j) ksum4_add(s[j], c[j], partials[4 * i + j]);
    for (int j = 0; j < 4; ++j) {
        rs[j][t] = s[j];
        rc[j][t] = c[j];
    }
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h)
            for (int j = 0; j < 4; ++j) {
                ksum4_add(rs[j][t], rc[j][t], rs[j][t + h]);
                rc[j][t] += rc[j][t + h];
            }
        __syncthreads();
    }
    if (t == 0) {
        ksum4_add(rs[0][0], rc[0][0], base_E);
        for (int j = 0; j < 4; ++j) totals[j] = rs[j][0] + rc[j][0];
    }
}

// Count initial-field entries with no physical frame (3D).
__global__ void k_check_fields3(const double *eps, const double *vx, const double *vy, const double *vz, long long n,
                                int *bad) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double e = eps ? eps[i] : 1.0;
    const double a = vx ? vx[i] : 0.0, b = vy ? vy[i] : 0.0, c = vz ? vz[i] : 0.0;
    const bool ok = isfinite(e) && e > 0.0 && isfinite(a) && isfinite(b) && isfinite(c) && (a * a + b * b + c * c < 1.0);
    if (!ok) atomicAdd(bad, 1);
}


#define RLBM3_FORMS(dtype, landau, CALL)                                         \
    switch (dtype) {                                                             \
    case RLBM_F64: CALL(double, double, double); break;                          \
    case RLBM_F32:                                                               \
        if (landau == RLBM_LANDAU_FP32) CALL(float, float, float);               \
        else CALL(float, float, double);                                         \
        break;                                                                   \
    case RLBM_BF16:                                                              \
        if (landau == RLBM_LANDAU_FP32) CALL(__nv_bfloat16, float, float);       \
        else CALL(__nv_bfloat16, float, double);                                 \
        break;                                                                   \
    default:                                                                     \
        if (landau == RLBM_LANDAU_FP32) CALL(__half, float, float);              \
        else CALL(__half, float, double);                                        \
    }

template <typename TS, typename TC, typename TL>
static cudaError_t launch_step3_t(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,
                                  const StepParams &p, cudaStream_t s) {
    const dim3 block(cfg.bx, cfg.by, 1);
    const bool idx32 = (long long)N3 * p.plane < (1ll << 31) - 1;
    const TS *in = static_cast<const TS *>(qin);
    TS *out = static_cast<TS *>(qout);
    const TC *f = static_cast<const TC *>(F);
    if (cfg.kernel == RLBM_KERNEL_PACKED) {
        if constexpr (std::is_same<TC, float>::value && std::is_same<TL, float>::value) {
            if (p.nx % 2 != 0) return cudaErrorInvalidValue;
            const dim3 g2((p.nx / 2 + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, p.nz);
#define RLBM3_PAIR(MB)                                                                           \
    do {                                                                                         \
        if (idx32) {                                                                             \
            if (forced) k_step3_pair<TS, true, int, MB><<<g2, block, 0, s>>>(in, out, f, p);     \
            else k_step3_pair<TS, false, int, MB><<<g2, block, 0, s>>>(in, out, f, p);           \
        } else {                                                                                 \
            if (forced) k_step3_pair<TS, true, long long, MB><<<g2, block, 0, s>>>(in, out, f, p); \
            else k_step3_pair<TS, false, long long, MB><<<g2, block, 0, s>>>(in, out, f, p);     \
        }                                                                                        \
    } while (0)
            if (cfg.minb >= 2) RLBM3_PAIR(2);
            else RLBM3_PAIR(1);
#undef RLBM3_PAIR
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;  // packed lanes: FP32 compute with the FP32 Landau solve
        }
    }
    const dim3 grid((p.nx + cfg.bx - 1) / cfg.bx, (p.ny + cfg.by - 1) / cfg.by, p.nz);
    if (idx32) {
        if (forced) k_step3<TS, TC, TL, true, int><<<grid, block, 0, s>>>(in, out, f, p);
        else k_step3<TS, TC, TL, false, int><<<grid, block, 0, s>>>(in, out, f, p);
    } else {
        if (forced) k_step3<TS, TC, TL, true, long long><<<grid, block, 0, s>>>(in, out, f, p);
        else k_step3<TS, TC, TL, false, long long><<<grid, block, 0, s>>>(in, out, f, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_step3(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                         const void *F, const StepParams &p, cudaStream_t s) {
    if (cfg.bx < 1 || cfg.by < 1 || cfg.bx * cfg.by > 256 || p.nz > 65535) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaSuccess;
#define RLBM3_STEP(TS, TC, TL) e = launch_step3_t<TS, TC, TL>(cfg, forced, qin, qout, F, p, s)
    RLBM3_FORMS(dtype, landau, RLBM3_STEP)
#undef RLBM3_STEP
    return e;
}

static dim3 block3() { return dim3(32, 8, 1); }
static dim3 grid3(const StepParams &p) { return dim3((p.nx + 31) / 32, (p.ny + 7) / 8, p.nz); }

long long moments3_blocks(const StepParams &p) {
    const dim3 g = grid3(p);
    return (long long)g.x * g.y * g.z;
}

cudaError_t launch_moments3(int dtype, const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                            double *vz, double *partials, int *bad, cudaStream_t s) {
#define RLBM3_MOM(TS, TC, TL)                                                                                   \
    k_moments3<TS, TC><<<grid3(p), block3(), 0, s>>>(static_cast<const TS *>(qin), p, eps, vx, vy, vz, partials, \
                                                     bad)
    RLBM3_FORMS(dtype, RLBM_LANDAU_FP64, RLBM3_MOM)
#undef RLBM3_MOM
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials4(const double *partials, long long nblocks, double base_E, double *totals,
                                    cudaStream_t s) {
    k_reduce_partials4<<<1, 256, 0, s>>>(partials, nblocks, base_E, totals);
    return cudaGetLastError();
}

cudaError_t launch_init3(int dtype, void *q, const StepParams &p, const double *eps, const double *vx,
                         const double *vy, const double *vz, cudaStream_t s) {
#define RLBM3_INIT(TS, TC, TL) k_init3<TS, TC><<<grid3(p), block3(), 0, s>>>(static_cast<TS *>(q), p, eps, vx, vy, vz)
    RLBM3_FORMS(dtype, RLBM_LANDAU_FP32, RLBM3_INIT)
#undef RLBM3_INIT
    return cudaGetLastError();
}

cudaError_t launch_check_fields3(const double *eps, const double *vx, const double *vy, const double *vz, long long n,
                                 int *bad, cudaStream_t s) {
    k_check_fields3<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(eps, vx, vy, vz, n, bad);
    return cudaGetLastError();
}

size_t mode3_bytes() { return sizeof(Mode3); }
size_t coef3_bytes(int dtype) { return dtype == RLBM_F64 ? sizeof(C6<double>) : sizeof(C6<float>); }

cudaError_t launch_draw_modes3(int dtype, const void *modes, void *coef, int nmodes, double amp,
                               unsigned long long seed, unsigned long long epoch, cudaStream_t s) {
    if (nmodes <= 0) return cudaSuccess;
    const Mode3 *m = static_cast<const Mode3 *>(modes);
    if (dtype == RLBM_F64)
        k_draw_modes3<double><<<(nmodes + 127) / 128, 128, 0, s>>>(m, static_cast<C6<double> *>(coef), nmodes, amp,
                                                                   seed, epoch);
    else
        k_draw_modes3<float><<<(nmodes + 127) / 128, 128, 0, s>>>(m, static_cast<C6<float> *>(coef), nmodes, amp,
                                                                  seed, epoch);
    return cudaGetLastError();
}

cudaError_t launch_mode_tables3(int dtype, void *T, const void *modes, int nmodes, const void *tw, int n, int axis,
                                cudaStream_t s) {
    if (nmodes <= 0) return cudaSuccess;
    const dim3 g((n + 255) / 256, nmodes, 1);
    const Mode3 *m = static_cast<const Mode3 *>(modes);
    if (dtype == RLBM_F64)
        k_mode_tables3<double><<<g, 256, 0, s>>>(static_cast<C2<double> *>(T), m, nmodes,
                                                 static_cast<const C2<double> *>(tw), n, axis);
    else
        k_mode_tables3<float><<<g, 256, 0, s>>>(static_cast<C2<float> *>(T), m, nmodes,
                                                static_cast<const C2<float> *>(tw), n, axis);
    return cudaGetLastError();
}

cudaError_t launch_synth_force3(int dtype, void *F, const void *coef, int nmodes, const void *X, const void *Y,
                                const void *Z, const StepParams &p, cudaStream_t s) {
    if (dtype == RLBM_F64)
        k_synth_force3<double><<<grid3(p), block3(), 0, s>>>(
            static_cast<double *>(F), static_cast<const C6<double> *>(coef), nmodes, static_cast<const C2<double> *>(X),
            static_cast<const C2<double> *>(Y), static_cast<const C2<double> *>(Z), p);
    else
        k_synth_force3<float><<<grid3(p), block3(), 0, s>>>(
            static_cast<float *>(F), static_cast<const C6<float> *>(coef), nmodes, static_cast<const C2<float> *>(X),
            static_cast<const C2<float> *>(Y), static_cast<const C2<float> *>(Z), p);
    return cudaGetLastError();
}

void host_mode3(void *dst, int i, int kx, int ky, int kz) { static_cast<Mode3 *>(dst)[i] = Mode3{kx, ky, kz}; }

double class_weight3(int k) { return d3w(k); }
void class_vector3(int k, double *c) {
    for (int a = 0; a < 3; ++a) c[a] = d3c(k, a);
}

}  // namespace rlbk
