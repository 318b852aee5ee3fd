// Accuracy of the Landau frame's FP32 reciprocal and reciprocal square root
// (frame_recip, frame_rsqrt in rlbm_device.cuh / packed.cuh) against the
// exact values computed in FP64, over the ranges the frame meets (the 2x2
// determinant near (4/3)^2 eps^2 and 1 - |v|^2 in (0, 1]), for the scalar
// FP32 lane and the packed pair of lanes.  Prints the largest errors in
// units in the last place as one JSON line.  Test infrastructure only.
#include <cmath>
#include <cstdio>

#include "../../paper_2101_06187_gb300/csrc/packed.cuh"

using namespace rlbk;

__global__ void k_check(int n, double *out_recip, double *out_rsqrt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // deterministic spread of arguments: a in [0.05, 8), w in (1e-3, 1]
    const float a = 0.05f + 7.95f * ((float)i / (float)n);
    const float w = 1e-3f + (1.0f - 1e-3f) * ((float)(((long long)i * 7919) % n) / (float)n);
    const float r1 = frame_recip(a);
    const float s1 = frame_rsqrt(w);
    const pf2 r2 = frame_recip(pf2(a, w));
    const pf2 s2 = frame_rsqrt(pf2(w, a));
    auto ulp_err = [](float got, double exact) {
        const float e = (float)exact;
        const double ulp = (double)nextafterf(fabsf(e), INFINITY) - (double)fabsf(e);
        return fabs((double)got - exact) / ulp;
    };
    const double er = fmax(fmax(ulp_err(r1, 1.0 / (double)a), ulp_err(r2.v.x, 1.0 / (double)a)),
                           ulp_err(r2.v.y, 1.0 / (double)w));
    const double es = fmax(fmax(ulp_err(s1, 1.0 / sqrt((double)w)), ulp_err(s2.v.x, 1.0 / sqrt((double)w))),
                           ulp_err(s2.v.y, 1.0 / sqrt((double)a)));
    out_recip[i] = er;
    out_rsqrt[i] = es;
}

int main() {
    const int n = 1 << 22;
    double *r, *s;
    if (cudaMallocManaged(&r, n * sizeof(double)) != cudaSuccess || cudaMallocManaged(&s, n * sizeof(double)) != cudaSuccess)
        return 2;
    k_check<<<(n + 255) / 256, 256>>>(n, r, s);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    double mr = 0, ms = 0, sr = 0, ss = 0;
    for (int i = 0; i < n; ++i) {
        mr = fmax(mr, r[i]);
        ms = fmax(ms, s[i]);
        sr += r[i];
        ss += s[i];
    }
    printf("{\"recip_max_ulp\": %.4f, \"rsqrt_max_ulp\": %.4f, \"recip_mean_ulp\": %.4f, \"rsqrt_mean_ulp\": %.4f}\n",
           mr, ms, sr / n, ss / n);
    return 0;
}
