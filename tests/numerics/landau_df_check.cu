// Accuracy of the Landau frame refined to FP64 accuracy on FP32 lanes
// (landau_refine_df in rlbm_device.cuh, packed lanes of packed.cuh) against
// the library's FP64 Newton solve of the same FP32 moments, over moments of
// fluid states with |v| up to argv[1] (default 0.6) and energy deviations
// up to 30%: the refined pairs (delta, v) agree with the FP64 frame to about
// 1e-13 at |v| <= 0.6, the FP32 Newton solve alone to about 1e-7.  Prints
// one JSON line.  Test infrastructure only.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "../../paper_2101_06187_gb300/csrc/packed.cuh"

using namespace rlbk;

// a deterministic spread of node moments: an ideal fluid (eps, v) in the
// deviation variables of the moments kernel, plus a non-equilibrium part
__device__ void sample_moments(int i, int n, double vmax, float &dE, float &Mx, float &My, float &Sxx, float &Sxy,
                               float &Syy) {
    const double t = (double)i / n;
    const double eps = 0.7 + 0.6 * fmod(t * 7.31, 1.0);
    const double sp = vmax * fmod(t * 3.17 + 0.13, 1.0);
    const double th = 6.283185307179586 * fmod(t * 11.7, 1.0);
    const double vx = sp * cos(th), vy = sp * sin(th);
    const double g2 = 1.0 / (1.0 - vx * vx - vy * vy);
    const double w = 4.0 / 3.0 * eps * g2;  // (eps + P) gamma^2, P = eps / 3
    const double ne = 1e-3 * sin(17.0 * t);  // a non-equilibrium shear part
    dE = (float)(w - eps / 3.0 - 1.0);
    Mx = (float)(w * vx);
    My = (float)(w * vy);
    Sxx = (float)(w * vx * vx + eps / 3.0 - 1.0 / 3.0 + ne);
    Sxy = (float)(w * vx * vy + 0.5 * ne);
    Syy = (float)(w * vy * vy + eps / 3.0 - 1.0 / 3.0 - ne);
}

__global__ void k_check(int n, double vmax, double *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float dE, Mx, My, Sxx, Sxy, Syy;
    sample_moments(i, n, vmax, dE, Mx, My, Sxx, Sxy, Syy);
    double d64;
    const Frame<double> f64 = landau_solve<double>(1.0, dE, Mx, My, Sxx, Sxy, Syy, 4.0 / 3.0, &d64);
    float d32;
    const Frame<float> f32 = landau_solve<float>(1.0f, dE, Mx, My, Sxx, Sxy, Syy, 4.0 / 3.0, &d32);
    pf2 dp;
    Frame<pf2> fp = landau_solve<pf2>(pf2(1.0f), pf2(dE), pf2(Mx), pf2(My), pf2(Sxx), pf2(Sxy), pf2(Syy), 4.0 / 3.0,
                                      &dp);
    const double alpha = 4.0 / 3.0;
    const float ah = (float)alpha, al = (float)(alpha - (double)ah);
    FramePairs<pf2> pr;
    landau_refine_df<pf2>(pf2(ah), pf2(al), pf2(1.0f), pf2(dE), pf2(Mx), pf2(My), pf2(Sxx), pf2(Sxy), pf2(Syy), dp,
                          fp, &pr);
    const double vn = fmax(sqrt(f64.v2), 1e-30);
    const double dn = fmax(fabs(d64), 1e-30);
    // refined pairs, both lanes
    double e_df = 0.0, e_32 = 0.0, e_round = 0.0;
    for (int l = 0; l < 2; ++l) {
        const double dh = l ? pr.delta_hi.v.y : pr.delta_hi.v.x, dl = l ? pr.delta_lo.v.y : pr.delta_lo.v.x;
        const double xh = l ? pr.vx_hi.v.y : pr.vx_hi.v.x, xl = l ? pr.vx_lo.v.y : pr.vx_lo.v.x;
        const double yh = l ? pr.vy_hi.v.y : pr.vy_hi.v.x, yl = l ? pr.vy_lo.v.y : pr.vy_lo.v.x;
        e_df = fmax(e_df, fabs(dh + dl - d64) / dn);
        e_df = fmax(e_df, fmax(fabs(xh + xl - f64.vx), fabs(yh + yl - f64.vy)) / vn);
        // the FP32 fields: the refined values rounded once (within an ulp)
        const float fe = l ? fp.eps.v.y : fp.eps.v.x;
        const float fx = l ? fp.vx.v.y : fp.vx.v.x;
        e_round = fmax(e_round, fabs((double)fe - f64.eps) / (ldexp(1.0, ilogb(f64.eps) - 23)));
        e_round = fmax(e_round, fabs((double)fx - f64.vx) / fmax(ldexp(1.0, ilogb(fabs(f64.vx)) - 23), 1e-40));
    }
    e_32 = fmax(fabs((double)d32 - d64) / dn, fmax(fabs((double)f32.vx - f64.vx), fabs((double)f32.vy - f64.vy)) / vn);
    err[3 * i + 0] = e_df;
    err[3 * i + 1] = e_32;
    err[3 * i + 2] = e_round;
}

int main(int argc, char **argv) {
    const int n = 1 << 16;
    const double vmax = argc > 1 ? std::atof(argv[1]) : 0.6;  // largest |v| of the sampled fluid states
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * 3 * n) != cudaSuccess) return 1;
    k_check<<<(n + 127) / 128, 128>>>(n, vmax, d);
    double *h = new double[3 * n];
    if (cudaMemcpy(h, d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    double m[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) m[k] = fmax(m[k], h[3 * i + k]);
    std::printf("{\"vmax\": %.3f, \"df_max_rel\": %.3e, \"fp32_max_rel\": %.3e, \"fp32_fields_max_ulp\": %.3f, "
                "\"n\": %d}\n", vmax, m[0], m[1], m[2], n);
    cudaFree(d);
    delete[] h;
    return 0;
}
