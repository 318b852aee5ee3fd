// The stochastic rounding of 16-bit stores (cvt_pair_sr, sr_pair_seed and
// the per-class mixing of store_pair in k_step_pair.cuh): every result is
// one of the two 16-bit neighbours of the FP32 value, and over many nodes
// (the hash's inputs) the mean of the rounded values equals the FP32 value
// to within its sampling error, for BF16 and FP16, in both halves of the
// pair.  Prints one JSON line.  Test infrastructure only.
#include <cstdio>

#include "../../paper_2101_06187_gb300/csrc/k_step_pair.cuh"

using namespace rlbk;

constexpr int NVAL = 64, NDRAW = 1 << 14;

template <typename TS>
__device__ float to_f(unsigned short u) {
    TS h;
    *reinterpret_cast<unsigned short *>(&h) = u;
    if constexpr (std::is_same<TS, __half>::value) return __half2float(h);
    else return __bfloat162float(h);
}

// value v: a spread of magnitudes and signs; block b draws NDRAW nodes
template <typename TS>
__global__ void k_sr(double *mean_err, int *outside) {
    const int v = blockIdx.x;
    const float x = (v % 2 ? -1.0f : 1.0f) * (0.013f + 0.37f * (float)v) * (1.0f + 0.001f * (float)(v * v));
    const float y = 0.5f * x + 0.125f;
    // the two round-to-zero neighbours and the next ones away from zero
    double sx = 0.0, sy = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < NDRAW; i += blockDim.x) {
        // the random bits of class 5 of node pair i, with the pair's rest values varying too
        const unsigned seed = sr_pair_seed((unsigned)i, 1.0f + 1e-3f * (float)(i % 97), -2e-3f * (float)(i % 89));
        const unsigned d = cvt_pair_sr<TS>(x, y, (seed ^ __float_as_uint(x)) * sr_class_mult(5));
        const float rx = to_f<TS>((unsigned short)(d & 0xFFFFu));
        const float ry = to_f<TS>((unsigned short)(d >> 16));
        sx += rx;
        sy += ry;
        // neighbours: round-down and round-up of x in the 16-bit type
        TS lo, hi;
        if constexpr (std::is_same<TS, __half>::value) {
            lo = __float2half_rd(x);
            hi = __float2half_ru(x);
        } else {
            lo = __float2bfloat16_rd(x);
            hi = __float2bfloat16_ru(x);
        }
        const float flo = std::is_same<TS, __half>::value ? __half2float(*(__half *)&lo) : __bfloat162float(*(__nv_bfloat16 *)&lo);
        const float fhi = std::is_same<TS, __half>::value ? __half2float(*(__half *)&hi) : __bfloat162float(*(__nv_bfloat16 *)&hi);
        if (rx != flo && rx != fhi) ++bad;
    }
    __shared__ double rsx[256], rsy[256];
    __shared__ int rb[256];
    rsx[threadIdx.x] = sx;
    rsy[threadIdx.x] = sy;
    rb[threadIdx.x] = bad;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            rsx[threadIdx.x] += rsx[threadIdx.x + h];
            rsy[threadIdx.x] += rsy[threadIdx.x + h];
            rb[threadIdx.x] += rb[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // error of the mean in units of the gap between the neighbours
        TS lo, hi;
        if constexpr (std::is_same<TS, __half>::value) {
            lo = __float2half_rd(x);
            hi = __float2half_ru(x);
        } else {
            lo = __float2bfloat16_rd(x);
            hi = __float2bfloat16_ru(x);
        }
        const double flo = std::is_same<TS, __half>::value ? __half2float(*(__half *)&lo) : __bfloat162float(*(__nv_bfloat16 *)&lo);
        const double fhi = std::is_same<TS, __half>::value ? __half2float(*(__half *)&hi) : __bfloat162float(*(__nv_bfloat16 *)&hi);
        const double gap = fhi > flo ? fhi - flo : 1.0;
        mean_err[2 * v] = (rsx[0] / NDRAW - (double)x) / gap;
        TS ylo, yhi;
        if constexpr (std::is_same<TS, __half>::value) {
            ylo = __float2half_rd(y);
            yhi = __float2half_ru(y);
        } else {
            ylo = __float2bfloat16_rd(y);
            yhi = __float2bfloat16_ru(y);
        }
        const double gl = std::is_same<TS, __half>::value ? __half2float(*(__half *)&ylo) : __bfloat162float(*(__nv_bfloat16 *)&ylo);
        const double gh = std::is_same<TS, __half>::value ? __half2float(*(__half *)&yhi) : __bfloat162float(*(__nv_bfloat16 *)&yhi);
        const double gy = gh > gl ? gh - gl : 1.0;
        mean_err[2 * v + 1] = (rsy[0] / NDRAW - (double)y) / gy;
        outside[v] = rb[0];
    }
}

template <typename TS>
static int run(const char *name, double *d_err, int *d_out, bool last) {
    k_sr<TS><<<NVAL, 256>>>(d_err, d_out);
    double err[2 * NVAL];
    int out[NVAL];
    if (cudaMemcpy(err, d_err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    if (cudaMemcpy(out, d_out, sizeof out, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    double m = 0.0;
    int bad = 0;
    for (int i = 0; i < 2 * NVAL; ++i) m = m > fabs(err[i]) ? m : fabs(err[i]);
    for (int i = 0; i < NVAL; ++i) bad += out[i];
    std::printf("\"%s_max_mean_err_gaps\": %.5f, \"%s_outside\": %d%s", name, m, name, bad, last ? "" : ", ");
    return 0;
}

int main() {
    double *d_err;
    int *d_out;
    if (cudaMalloc(&d_err, sizeof(double) * 2 * NVAL) != cudaSuccess) return 1;
    if (cudaMalloc(&d_out, sizeof(int) * NVAL) != cudaSuccess) return 1;
    std::printf("{\"draws\": %d, ", NDRAW);
    if (run<__nv_bfloat16>("bf16", d_err, d_out, false)) return 1;
    if (run<__half>("f16", d_err, d_out, true)) return 1;
    std::printf("}\n");
    cudaFree(d_err);
    cudaFree(d_out);
    return 0;
}
