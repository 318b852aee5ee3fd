// rlbm_api.cu -- the extern "C" boundary declared in include/rlbm.h: handle
// life cycle, device memory, the step loop (direct launches or CUDA-graph
// replay), diagnostics.
#include <math.h>

#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rlbm_internal.h"
#include "k_ring.cuh"

namespace rlbk {

cudaError_t launch_step_f64(const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout,
                            const void *F, const StepParams &p, cudaStream_t s);
cudaError_t launch_step_f32(const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout,
                            const void *F, const StepParams &p, cudaStream_t s);
cudaError_t launch_step_h16(int dtype, const LaunchCfg &cfg, int landau, bool forced, const void *qin, void *qout,
                            const void *F, const StepParams &p, cudaStream_t s);
cudaError_t launch_batch_f64(const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns, int ntiles,
                             cudaStream_t s);
cudaError_t launch_batch_f32(const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns, int ntiles,
                             cudaStream_t s);
cudaError_t launch_batch_h16(int dtype, const LaunchCfg &cfg, int landau, int grid, const void *runs, int nruns,
                             int ntiles, cudaStream_t s);
cudaError_t launch_moments_f64(int landau, const void *qin, const StepParams &p, double *eps, double *vx,
                               double *vy, double *partials, int *bad, cudaStream_t s);
cudaError_t launch_moments_f32(int landau, const void *qin, const StepParams &p, double *eps, double *vx,
                               double *vy, double *partials, int *bad, cudaStream_t s);
cudaError_t launch_moments_h16(int dtype, int landau, const void *qin, const StepParams &p, double *eps,
                               double *vx, double *vy, double *partials, int *bad, cudaStream_t s);

cudaError_t launch_step(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                        const void *F, const StepParams &p, cudaStream_t s) {
    switch (dtype) {
    case RLBM_F64: return launch_step_f64(cfg, landau, forced, qin, qout, F, p, s);
    case RLBM_F32: return launch_step_f32(cfg, landau, forced, qin, qout, F, p, s);
    default: return launch_step_h16(dtype, cfg, landau, forced, qin, qout, F, p, s);
    }
}

cudaError_t launch_moments(int dtype, int landau, const void *qin, const StepParams &p, double *eps, double *vx,
                           double *vy, double *partials, int *bad, cudaStream_t s) {
    switch (dtype) {
    case RLBM_F64: return launch_moments_f64(landau, qin, p, eps, vx, vy, partials, bad, s);
    case RLBM_F32: return launch_moments_f32(landau, qin, p, eps, vx, vy, partials, bad, s);
    default: return launch_moments_h16(dtype, landau, qin, p, eps, vx, vy, partials, bad, s);
    }
}

cudaError_t launch_batch(int dtype, int landau, const LaunchCfg &cfg, int grid, const void *runs, int nruns,
                         int ntiles, cudaStream_t s) {
    switch (dtype) {
    case RLBM_F64: return launch_batch_f64(cfg, landau, grid, runs, nruns, ntiles, s);
    case RLBM_F32: return launch_batch_f32(cfg, landau, grid, runs, nruns, ntiles, s);
    default: return launch_batch_h16(dtype, cfg, landau, grid, runs, nruns, ntiles, s);
    }
}

int run_length(int dtype) { return dtype == RLBM_F64 ? 2 : 4; }

int moments_blocks(const StepParams &p) { return ((p.nx + 31) / 32) * ((p.ny + 7) / 8); }

}  // namespace rlbk

using namespace rlbk;

// ---------------------------------------------------------------- helpers
// NVTX range over a library call (visible in Nsight timelines; free when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static rlbm_status fail(rlbm_t *h, rlbm_status st, const char *fmt, ...) {
    if (!h) return st;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->msg = buf;
    if (st == RLBM_ERR_CUDA || st == RLBM_ERR_TIMEOUT) h->status = st;  // sticky
    return st;
}

#define CUDA_TRY(h, call)                                                                                 \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail(h, RLBM_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                           \
    } while (0)

#define CHECK_HANDLE(h)                                  \
    do {                                                 \
        if (!(h)) return RLBM_ERR_ARG;                   \
        if ((h)->status != RLBM_OK) return (h)->status;  \
        if (cudaSetDevice((h)->device) != cudaSuccess) return fail(h, RLBM_ERR_CUDA, "cudaSetDevice failed"); \
    } while (0)

static void *dev_alloc(rlbm_t *h, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (h->opts.alloc) {
        p = h->opts.alloc(bytes, h->opts.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) h->device_bytes += bytes;
    return p;
}

static void dev_free(rlbm_t *h, void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (h->opts.alloc) {
        if (h->opts.free) h->opts.free(p, bytes, h->opts.alloc_ctx);
    } else {
        cudaFree(p);
    }
}

static StepParams params_of(const rlbm_t *h) {
    StepParams p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.pitch = h->pitch;
    p.slab = (long long)h->ny * h->pitch;
    p.nz = h->nz;
    p.plane = p.slab * h->nz;
    p.inv_tau = 1.0 / h->tau;
    p.eps0 = h->opts.eps0;
    p.scale = h->opts.scale;
    p.cfl = h->opts.cfl;
    // eta/s mode: 1/tau = T dt / (5 eta/s), T = (pi^2 eps / 3)^{1/4}
    p.eta_k = h->opts.eta_s > 0.0 ? std::pow(M_PI * M_PI / 3.0, 0.25) * h->opts.dt / (5.0 * h->opts.eta_s) : 0.0;
    p.err = h->errword;
    finish_params(p);
    p.round_sr = h->opts.rounding == RLBM_ROUND_STOCHASTIC ? 1 : 0;  // resolved at create (16-bit forms only)
    return p;
}

static size_t nodes_of(const rlbm_t *h) { return (size_t)h->nx * h->ny * h->nz; }
static size_t q_bytes(const rlbm_t *h) {
    return (size_t)h->ncls * h->nz * h->ny * h->pitch * storage_bytes(h->opts.dtype);
}
static size_t F_bytes(const rlbm_t *h) {
    return (size_t)(h->d3 ? 3 : 2) * h->nz * h->ny * h->pitch * compute_bytes(h->opts.dtype);
}
static size_t tw_bytes(const rlbm_t *h, int n) { return (size_t)n * 2 * compute_bytes(h->opts.dtype); }
static size_t fields_bytes(const rlbm_t *h) { return (size_t)(h->d3 ? 4 : 3) * nodes_of(h) * sizeof(double); }
static size_t partials_bytes(const rlbm_t *h) {
    return h->d3 ? (size_t)4 * moments3_blocks(params_of(h)) * sizeof(double)
                 : (size_t)3 * moments_blocks(params_of(h)) * sizeof(double);
}
static size_t gtab_bytes(const rlbm_t *h) { return (size_t)h->nky * h->nx * 4 * compute_bytes(h->opts.dtype); }
static size_t coef_bytes(const rlbm_t *h) {
    return h->d3 ? coef3_bytes(h->opts.dtype) * h->nmodes : 4 * compute_bytes(h->opts.dtype) * h->nmodes;
}

// Class weight W_c of stored class c (spherical node or 2D ring).
static double class_weight(const rlbm_t *h, int c) {
    if (h->ring) return 1.0 / 8.0;
    if (h->d3) return class_weight3(c);
    return c == 0 ? 2.0 / 21.0 : c <= 4 ? 1.0 / 21.0 : c <= 8 ? 8.0 / 105.0 : c <= 12 ? 4.0 / 105.0 : 9.0 / 140.0;
}

static cudaError_t launch_step_h(const rlbm_t *h, const LaunchCfg &cfg, const void *qin, void *qout,
                                 const StepParams &p) {
    if (h->ring) return launch_ring_step(h->opts.dtype, h->opts.landau, cfg, h->forced, qin, qout, h->F, p, h->stream);
    if (h->d3) return launch_step3(h->opts.dtype, h->opts.landau, cfg, h->forced, qin, qout, h->F, p, h->stream);
    // FP32 / 16-bit storage with the FP64 Landau solve on the packed kernels: the frame refined to FP64
    // accuracy on the FP32 lanes
    const bool dfl = h->opts.landau == RLBM_LANDAU_FP64 && h->opts.dtype != RLBM_F64;
    if (cfg.kernel == RLBM_KERNEL_FUSED2) {
        if (dfl) return launch_step_fused2_dfl(h->opts.dtype, cfg, h->forced, qin, qout, h->F, p, h->stream);
        return launch_step_fused2(h->opts.dtype, h->opts.landau, cfg, h->forced, qin, qout, h->F, p, h->stream);
    }
    if (cfg.kernel == RLBM_KERNEL_PACKED && dfl)
        return launch_step_pair_dfl(h->opts.dtype, cfg, h->forced, qin, qout, h->F, p, h->stream);
    if (cfg.kernel == RLBM_KERNEL_PACKED4) {
        switch (h->opts.dtype) {
        case RLBM_F32:
            return (dfl ? launch_step_quad_dfl_f32 : launch_step_quad_f32)(cfg, h->forced, qin, qout, h->F, p,
                                                                          h->stream);
        case RLBM_BF16:
            return (dfl ? launch_step_quad_dfl_bf16 : launch_step_quad_bf16)(cfg, h->forced, qin, qout, h->F, p,
                                                                            h->stream);
        case RLBM_F16:
            return (dfl ? launch_step_quad_dfl_f16 : launch_step_quad_f16)(cfg, h->forced, qin, qout, h->F, p,
                                                                          h->stream);
        default: return cudaErrorInvalidValue;
        }
    }
    if (cfg.kernel == RLBM_KERNEL_TMA) {
        if (!h->tm_ready) return cudaErrorNotSupported;
        const CUtensorMap &mq = (qin == h->q[0]) ? h->tm_q[0] : h->tm_q[1];
        return launch_step_tma(cfg, h->forced, mq, h->tm_F, qin, qout, p, h->stream, h->opts.test_unarmed_wait);
    }
    return launch_step(h->opts.dtype, h->opts.landau, cfg, h->forced, qin, qout, h->F, p, h->stream);
}

static int enumerate_modes(int kmin, int kmax, std::vector<Mode> *out) {
    int m = 0;
    for (int ky = 0; ky <= kmax; ++ky)
        for (int kx = -kmax; kx <= kmax; ++kx) {
            if (ky == 0 && kx <= 0) continue;
            const int k2 = kx * kx + ky * ky;
            if (k2 < kmin * kmin || k2 > kmax * kmax) continue;
            if (out) out->push_back(Mode{kx, ky, 0.0, 0.0, 0.0, 0.0});
            ++m;
        }
    return m;
}

// Make F hold the force of the epoch containing step `step`.
static rlbm_status ensure_force(rlbm_t *h) {
    if (!h->forced) return RLBM_OK;
    const long long e = h->step / h->forcing.redraw_period;
    if (e == h->force_epoch) return RLBM_OK;
    NvtxRange range("rlbm_force_epoch");
    const StepParams p = params_of(h);
    if (h->d3) {
        CUDA_TRY(h, launch_draw_modes3(h->opts.dtype, h->modes3, h->coef, h->nmodes, h->forcing.amp,
                                       (unsigned long long)h->forcing.seed, (unsigned long long)e, h->stream));
        CUDA_TRY(h, launch_synth_force3(h->opts.dtype, h->F, h->coef, h->nmodes, h->tabx, h->taby, h->tabz, p,
                                        h->stream));
        h->force_epoch = e;
        return RLBM_OK;
    }
    CUDA_TRY(h, launch_draw_modes(h->opts.dtype, h->modes, h->coef, h->nmodes, h->forcing.amp,
                                  (unsigned long long)h->forcing.seed, (unsigned long long)e, h->stream));
    CUDA_TRY(h, launch_synth_force(h->opts.dtype, h->F, h->coef, h->nmodes, h->ky_start, h->nky, h->gtab, h->tabx,
                                   h->taby, p, h->stream));
    h->force_epoch = e;
    return RLBM_OK;
}

// Lattice steps one launch of `cfg` advances.
static int steps_per_launch(const LaunchCfg &cfg) { return cfg.kernel == RLBM_KERNEL_FUSED2 ? 2 : 1; }

// Launches that advance n steps: two-step launches, then single steps for
// what is left (the packed single step after two-step launches).
static int launches_for(const LaunchCfg &cfg, int n) { return steps_per_launch(cfg) == 2 ? n / 2 + n % 2 : n; }

static rlbm_status launch_steps(rlbm_t *h, int n) {
    const StepParams p = params_of(h);
    int i = 0;
    LaunchCfg one = h->cfg;
    if (steps_per_launch(h->cfg) == 2) {
        for (; i + 2 <= n; i += 2) {
            CUDA_TRY(h, launch_step_h(h, h->cfg, h->q[h->cur], h->q[h->cur ^ 1], p));
            h->cur ^= 1;
        }
        one = LaunchCfg{RLBM_KERNEL_PACKED, 128, 1, 2};
    }
    for (; i < n; ++i) {
        CUDA_TRY(h, launch_step_h(h, one, h->q[h->cur], h->q[h->cur ^ 1], p));
        h->cur ^= 1;
    }
    return RLBM_OK;
}

// Run `n` steps inside one epoch: replay a captured graph of the even part
// of n (keyed by that count and the buffer it starts from; it leaves the
// state in the buffer its launch count implies), then a last single step.
// An even part of one launch (two steps of a two-step kernel) is launched
// directly: a graph saves host work only over several launches, and a
// one-node graph starts its kernel later on the GPU than a plain launch
// (about 1.8 us at 1024^2, measured with CUDA events).
static rlbm_status run_chunk(rlbm_t *h, int n) {
    const int even = n & ~1;
    const bool graphs = h->opts.use_graphs && h->stream != nullptr && n >= 2 && launches_for(h->cfg, even) >= 2;
    if (!graphs) return launch_steps(h, n);
    auto key = std::make_pair(even, h->cur);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        const int cur0 = h->cur;
        CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        rlbm_status st = launch_steps(h, even);
        cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
        h->cur = cur0;
        if (st != RLBM_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ec != cudaSuccess) return fail(h, RLBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) return fail(h, RLBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
        it = h->graphs.emplace(key, ge).first;
    }
    CUDA_TRY(h, cudaGraphLaunch(it->second, h->stream));
    h->cur ^= launches_for(h->cfg, even) & 1;
    if (even != n) return launch_steps(h, 1);
    return RLBM_OK;
}

// The spectrum work area (complex lattice + twiddles + shell sums), made on
// first use.
static size_t spectrum_doubles(const rlbm_t *h) {
    return h->d3 ? spectrum_work_doubles3(h->nx, h->ny, h->nz) : spectrum_work_doubles(h->nx, h->ny);
}

static rlbm_status ensure_spectrum_work(rlbm_t *h) {
    if (std::max(std::max(h->nx, h->ny), h->nz) > 8192)
        return fail(h, RLBM_ERR_ARG, "spectra support lattice sides up to 8192");
    if (!h->spec_work) {
        const size_t need = spectrum_doubles(h) * sizeof(double) + 4096 * sizeof(double);
        h->spec_work = static_cast<double *>(dev_alloc(h, need));
        if (!h->spec_work) return fail(h, RLBM_ERR_ALLOC, "spectrum work area");
        h->spec_work_bytes = need;
    }
    return RLBM_OK;
}

// Launch configurations tried by rlbm_autotune, and the winners per
// (nx, ny, dtype, landau, forced), shared by all handles of the process.
static const LaunchCfg kCandidates[] = {
    {RLBM_KERNEL_GATHER_VEC, 32, 4}, {RLBM_KERNEL_GATHER_VEC, 64, 2}, {RLBM_KERNEL_GATHER_VEC, 128, 1},
    {RLBM_KERNEL_GATHER_VEC, 32, 8}, {RLBM_KERNEL_GATHER_VEC, 64, 4}, {RLBM_KERNEL_GATHER_VEC, 128, 2},
    {RLBM_KERNEL_GATHER_VEC, 256, 1}, {RLBM_KERNEL_GATHER_VEC, 32, 2}, {RLBM_KERNEL_GATHER_VEC, 64, 1},
    {RLBM_KERNEL_GATHER_VEC2, 32, 4}, {RLBM_KERNEL_GATHER_VEC2, 64, 2}, {RLBM_KERNEL_GATHER_VEC2, 128, 1},
    {RLBM_KERNEL_GATHER_VEC2, 32, 8}, {RLBM_KERNEL_GATHER_VEC2, 64, 4}, {RLBM_KERNEL_GATHER_VEC2, 128, 2},
    {RLBM_KERNEL_PACKED, 32, 4}, {RLBM_KERNEL_PACKED, 64, 2}, {RLBM_KERNEL_PACKED, 128, 1},
    {RLBM_KERNEL_PACKED, 32, 8}, {RLBM_KERNEL_PACKED, 64, 4}, {RLBM_KERNEL_PACKED, 128, 2},
    {RLBM_KERNEL_PACKED, 64, 2, 2}, {RLBM_KERNEL_PACKED, 128, 1, 2}, {RLBM_KERNEL_PACKED, 128, 2, 2},
    {RLBM_KERNEL_PACKED, 64, 2, 3}, {RLBM_KERNEL_PACKED, 128, 1, 3}, {RLBM_KERNEL_PACKED, 128, 2, 3},
    {RLBM_KERNEL_PACKED, 64, 4, 3}, {RLBM_KERNEL_PACKED, 32, 8, 3},
    {RLBM_KERNEL_PACKED, 64, 2, 5}, {RLBM_KERNEL_PACKED, 128, 1, 5}, {RLBM_KERNEL_PACKED, 32, 4, 5},
    {RLBM_KERNEL_TMA, 32, 8, 2}, {RLBM_KERNEL_TMA, 32, 8, 1},
    {RLBM_KERNEL_TWOPASS, 64, 2, 2}, {RLBM_KERNEL_TWOPASS, 128, 1, 2}, {RLBM_KERNEL_TWOPASS, 32, 8, 2},
    {RLBM_KERNEL_TWOPASS, 64, 2, 3}, {RLBM_KERNEL_TWOPASS, 128, 1, 3}, {RLBM_KERNEL_TWOPASS, 32, 8, 3},
    {RLBM_KERNEL_TWOPASS, 64, 4, 3}, {RLBM_KERNEL_TWOPASS, 64, 2, 4}, {RLBM_KERNEL_TWOPASS, 128, 1, 4},
    {RLBM_KERNEL_TWOPASS, 32, 8, 4},
    {RLBM_KERNEL_GATHER, 32, 8}, {RLBM_KERNEL_GATHER, 64, 4}, {RLBM_KERNEL_GATHER, 128, 2},
    {RLBM_KERNEL_GATHER, 256, 1}, {RLBM_KERNEL_GATHER, 32, 4}, {RLBM_KERNEL_GATHER, 128, 1},
    {RLBM_KERNEL_FUSED2, 64, 16, 2}, {RLBM_KERNEL_FUSED2, 64, 8, 4}, {RLBM_KERNEL_FUSED2, 32, 16, 4},
    {RLBM_KERNEL_FUSED2, 128, 8, 2},
    {RLBM_KERNEL_PACKED4, 128, 1, 4}, {RLBM_KERNEL_PACKED4, 64, 2, 4}, {RLBM_KERNEL_PACKED4, 32, 4, 4},
    {RLBM_KERNEL_PACKED4, 128, 1, 3}, {RLBM_KERNEL_PACKED4, 64, 2, 3}, {RLBM_KERNEL_PACKED4, 32, 4, 3},
};
// Whether launch shape c can run this lattice (the launchers reject the
// remaining misfits: storage form, Landau precision, nx parity).
static bool candidate_applies(const rlbm_t *h, const LaunchCfg &c) {
    if (h->opts.cfl != 1.0 && c.kernel != RLBM_KERNEL_GATHER &&
        !(c.kernel == RLBM_KERNEL_PACKED && c.minb <= 2 && !h->ring && !h->d3) &&
        !(c.kernel == RLBM_KERNEL_FUSED2 && h->opts.cfl < 1.0 && !h->ring && !h->d3))
        return false;
    if ((h->d3 || h->ring) && c.kernel != RLBM_KERNEL_GATHER && c.kernel != RLBM_KERNEL_PACKED &&
        !(h->ring && c.kernel == RLBM_KERNEL_FUSED2))
        return false;
    if (c.kernel == RLBM_KERNEL_TMA && !h->tm_ready) return false;
    if (h->opts.rounding == RLBM_ROUND_STOCHASTIC && c.kernel != RLBM_KERNEL_PACKED &&
        c.kernel != RLBM_KERNEL_FUSED2 && c.kernel != RLBM_KERNEL_PACKED4)
        return false;  // the other kernels round to nearest
    return true;
}

static std::map<std::tuple<int, int, int, int, int, int, int, int>, LaunchCfg> g_tuned;
static std::mutex g_tuned_mu;

static std::tuple<int, int, int, int, int, int, int, int> tune_key(const rlbm_t *h) {
    return std::make_tuple(h->nx, h->ny, h->opts.dtype, h->opts.landau, h->forced ? 1 : 0,
                           h->ring ? 1 : (h->d3 ? 2 + h->nz : 0), stream_mode(h->opts.cfl), h->opts.rounding);
}


// The device error word of the bounded waits (synchronises): a wait that
// gave up leaves the state of that step undefined, so the error is sticky.
static rlbm_status check_errword(rlbm_t *h) {
    int *w = reinterpret_cast<int *>(h->host_small) + 64;
    CUDA_TRY(h, cudaMemcpyAsync(w, h->errword, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (*w) return fail(h, RLBM_ERR_TIMEOUT, "a bounded wait on a tile copy gave up (error word %d)", *w);
    return RLBM_OK;
}

static void drop_graphs(rlbm_t *h) {
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
}

extern "C" {

const char *rlbm_status_string(rlbm_status s) {
    switch (s) {
    case RLBM_OK: return "ok";
    case RLBM_ERR_ARG: return "invalid argument";
    case RLBM_ERR_ALLOC: return "device allocation failed";
    case RLBM_ERR_CUDA: return "CUDA error";
    case RLBM_ERR_TIMEOUT: return "device wait timed out";
    case RLBM_ERR_NAN: return "non-finite or non-physical state";
    case RLBM_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

void rlbm_opts_default(rlbm_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->dtype = RLBM_F32;
    o->landau = RLBM_LANDAU_FP32;
    o->kernel = RLBM_KERNEL_AUTO;
    o->use_graphs = 1;
    o->eps0 = 1.0;
    o->scale = 0.0;
    o->stream = nullptr;
    o->device = -1;
    o->cfl = 1.0;
    o->eta_s = 0.0;
    o->dt = 1.0;
}

void rlbm_destroy(rlbm_t *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    drop_graphs(h);
    dev_free(h, h->q[0], q_bytes(h));
    dev_free(h, h->q[1], q_bytes(h));
    if (h->F) dev_free(h, h->F, F_bytes(h));
    if (h->twx) dev_free(h, h->twx, tw_bytes(h, h->fnx));
    if (h->twy) dev_free(h, h->twy, tw_bytes(h, h->fny));
    if (h->coef) dev_free(h, h->coef, coef_bytes(h));
    if (h->twz) dev_free(h, h->twz, tw_bytes(h, h->nz));
    if (h->tabz) dev_free(h, h->tabz, tw_bytes(h, h->nz) * h->nmodes);
    if (h->modes3) dev_free(h, h->modes3, mode3_bytes() * h->nmodes);
    if (h->tabx) dev_free(h, h->tabx, tw_bytes(h, h->nx) * h->nmodes);
    if (h->taby) dev_free(h, h->taby, tw_bytes(h, h->ny) * h->nmodes);
    if (h->modes) dev_free(h, h->modes, sizeof(Mode) * h->nmodes);
    if (h->ky_start) dev_free(h, h->ky_start, sizeof(int) * (h->nky + 1));
    if (h->gtab) dev_free(h, h->gtab, gtab_bytes(h));
    dev_free(h, h->fields, fields_bytes(h));
    dev_free(h, h->partials, partials_bytes(h));
    dev_free(h, h->totals, 4 * sizeof(double));
    dev_free(h, h->bad, sizeof(int) * 4);
    dev_free(h, h->errword, sizeof(int) * 4);
    if (h->spec_work) dev_free(h, h->spec_work, h->spec_work_bytes);
    if (h->spec_acc) dev_free(h, h->spec_acc, 2 * 4096 * sizeof(double));
    if (h->host_small) cudaFreeHost(h->host_small);
    delete h;
}

}  // extern "C"

// The 3D mode list: integer k on the shell, one per pair +-k, the
// representative with kz > 0, or kz = 0 and ky > 0, or kz = ky = 0 and
// kx > 0, in the order kz = 0..kmax, ky = -kmax..kmax, kx = -kmax..kmax.
static int enumerate_modes3(int kmin, int kmax, std::vector<int> *out) {
    int m = 0;
    for (int kz = 0; kz <= kmax; ++kz)
        for (int ky = -kmax; ky <= kmax; ++ky)
            for (int kx = -kmax; kx <= kmax; ++kx) {
                if (kz == 0 && (ky < 0 || (ky == 0 && kx <= 0))) continue;
                const int k2 = kx * kx + ky * ky + kz * kz;
                if (k2 < kmin * kmin || k2 > kmax * kmax) continue;
                if (out) {
                    out->push_back(kx);
                    out->push_back(ky);
                    out->push_back(kz);
                }
                ++m;
            }
    return m;
}

static rlbm_status create_impl(int nx, int ny, int nz, bool d3, rlbm_stencil stencil, double tau,
                               const rlbm_forcing *forcing, const rlbm_opts *opts, rlbm_t **out) {
    if (!out) return RLBM_ERR_ARG;
    *out = nullptr;
    if (stencil != RLBM_STENCIL_SPH26_SLAB && stencil != RLBM_STENCIL_RING8_2D) return RLBM_ERR_ARG;
    const bool ring = stencil == RLBM_STENCIL_RING8_2D;
    if (d3 && (ring || nz < 4)) return RLBM_ERR_ARG;
    if (!d3) nz = 1;
    if (nx < 4 || ny < 4 || (long long)nx * ny * nz > (1ll << 31)) return RLBM_ERR_ARG;
    if (ny > 65535 || nz > 65535) return RLBM_ERR_ARG;  // rows and layers span launch-grid y and z
    if (!(tau > 0.5) || !isfinite(tau)) return RLBM_ERR_ARG;
    rlbm_opts o;
    rlbm_opts_default(&o);
    if (opts) o = *opts;
    if (o.dtype < RLBM_F64 || o.dtype > RLBM_F16) return RLBM_ERR_ARG;
    if (o.landau != RLBM_LANDAU_FP64 && o.landau != RLBM_LANDAU_FP32) return RLBM_ERR_ARG;
    if (o.kernel < RLBM_KERNEL_AUTO || o.kernel > RLBM_KERNEL_PACKED4) return RLBM_ERR_ARG;
    if (o.kernel == RLBM_KERNEL_TMA && (nx % 2 != 0 || o.dtype != RLBM_F32 || o.landau != RLBM_LANDAU_FP32))
        return RLBM_ERR_ARG;
    if ((o.kernel == RLBM_KERNEL_PACKED || o.kernel == RLBM_KERNEL_TWOPASS || o.kernel == RLBM_KERNEL_FUSED2) &&
        (nx % 2 != 0 || o.dtype == RLBM_F64))
        return RLBM_ERR_ARG;
    if (o.kernel == RLBM_KERNEL_PACKED4 && (nx % 4 != 0 || o.dtype == RLBM_F64 || ring || d3 ||
                                            !(o.cfl == 0.0 || o.cfl == 1.0)))
        return RLBM_ERR_ARG;  // four nodes per thread: aligned runs of four, CFL 1, the one-layer lattice
    // the FP64 Landau solve on the packed kernels is the frame refined on the FP32 lanes: one-layer lattice, CFL 1
    if (o.landau != RLBM_LANDAU_FP32 &&
        (o.kernel == RLBM_KERNEL_TWOPASS ||
         ((o.kernel == RLBM_KERNEL_PACKED || o.kernel == RLBM_KERNEL_FUSED2) &&
          (ring || d3 || !(o.cfl == 0.0 || o.cfl == 1.0)))))
        return RLBM_ERR_ARG;
    if (o.kernel == RLBM_KERNEL_GATHER_VEC && nx % (o.dtype == RLBM_F64 ? 2 : 4) != 0) return RLBM_ERR_ARG;
    if (o.kernel == RLBM_KERNEL_GATHER_VEC2 && nx % 2 != 0) return RLBM_ERR_ARG;
    if (o.eps0 == 0.0) o.eps0 = 1.0;
    if (!(o.eps0 > 0.0) || !isfinite(o.eps0)) return RLBM_ERR_ARG;
    if (o.scale == 0.0) o.scale = (o.dtype == RLBM_BF16 || o.dtype == RLBM_F16) ? 1.0 / 64.0 : 1.0;
    if (!(o.scale > 0.0) || !isfinite(o.scale)) return RLBM_ERR_ARG;
    // FP32 and FP64 storage keep the deviation unscaled (a scale buys floating point nothing)
    if ((o.dtype == RLBM_F32 || o.dtype == RLBM_F64) && o.scale != 1.0) return RLBM_ERR_ARG;
    if (o.alloc && !o.free) return RLBM_ERR_ARG;
    if (o.cfl == 0.0) o.cfl = 1.0;
    if (o.dt == 0.0) o.dt = 1.0;
    if (!(o.cfl > 0.0 && o.cfl < 2.0) || !(o.eta_s >= 0.0) || !isfinite(o.eta_s) || !(o.dt > 0.0) || !isfinite(o.dt))
        return RLBM_ERR_ARG;
    if (o.cfl != 1.0 && (o.kernel == RLBM_KERNEL_GATHER_VEC || o.kernel == RLBM_KERNEL_GATHER_VEC2 ||
                         o.kernel == RLBM_KERNEL_TMA || o.kernel == RLBM_KERNEL_TWOPASS))
        return RLBM_ERR_ARG;  // the vector kernels stream at CFL 1 only
    if (o.cfl > 1.0 && o.kernel == RLBM_KERNEL_FUSED2) return RLBM_ERR_ARG;  // two steps per launch: halo 1
    if (o.rounding < RLBM_ROUND_DEFAULT || o.rounding > RLBM_ROUND_STOCHASTIC) return RLBM_ERR_ARG;
    const bool h16 = o.dtype == RLBM_BF16 || o.dtype == RLBM_F16;
    const bool sr_kernel = o.kernel == RLBM_KERNEL_AUTO || o.kernel == RLBM_KERNEL_PACKED ||
                           o.kernel == RLBM_KERNEL_FUSED2 || o.kernel == RLBM_KERNEL_PACKED4;
    if (o.rounding == RLBM_ROUND_DEFAULT)  // BF16: stochastic where the kernel can, else nearest
        o.rounding = (o.dtype == RLBM_BF16 && !ring && !d3 && sr_kernel && nx % 2 == 0) ? RLBM_ROUND_STOCHASTIC
                                                                                           : RLBM_ROUND_NEAREST;
    if (!h16) o.rounding = RLBM_ROUND_NEAREST;
    // stochastic rounding of 16-bit stores: the packed kernels of the one-layer lattice
    if (o.rounding == RLBM_ROUND_STOCHASTIC && (ring || d3 || !sr_kernel || nx % 2 != 0)) return RLBM_ERR_ARG;
    if (o.dtype == RLBM_F64) o.landau = RLBM_LANDAU_FP64;
    // the ring runs the one-node-per-thread kernel, at CFL 1 with a fixed tau
    if (ring && ((o.kernel != RLBM_KERNEL_AUTO && o.kernel != RLBM_KERNEL_GATHER && o.kernel != RLBM_KERNEL_PACKED &&
                  o.kernel != RLBM_KERNEL_FUSED2) ||
                 o.cfl != 1.0 || o.eta_s != 0.0))
        return RLBM_ERR_ARG;
    // the 3D lattice runs the one-node-per-thread or the packed-lane kernel at CFL 1
    if (d3 && ((o.kernel != RLBM_KERNEL_AUTO && o.kernel != RLBM_KERNEL_GATHER && o.kernel != RLBM_KERNEL_PACKED) ||
               o.cfl != 1.0))
        return RLBM_ERR_ARG;

    rlbm_forcing fz{};
    bool forced = false;
    if (forcing) {
        fz = *forcing;
        if (!(fz.amp >= 0.0) || !isfinite(fz.amp)) return RLBM_ERR_ARG;
        if (fz.amp > 0.0 && fz.kmax > 0) {
            if (fz.kmin < 1 || fz.kmin > fz.kmax || 2 * fz.kmax >= std::min(nx, ny)) return RLBM_ERR_ARG;
            if (d3 && 2 * fz.kmax >= nz) return RLBM_ERR_ARG;
            if (fz.redraw_period < 1) return RLBM_ERR_ARG;
            forced = true;
        }
    }

    rlbm_t *h = new rlbm_t();
    h->nx = nx;
    h->ny = ny;
    h->pitch = (nx + 31) & ~31;
    h->tau = tau;
    h->opts = o;
    h->forcing = fz;
    h->forced = forced;
    h->ring = ring;
    h->d3 = d3;
    h->nz = nz;
    h->ncls = ring ? NR : d3 ? 26 : NC;  // 3D: all 26 directions stored
    if (o.device >= 0) {
        if (cudaSetDevice(o.device) != cudaSuccess) {
            delete h;
            return RLBM_ERR_ARG;
        }
        h->device = o.device;
    } else if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return RLBM_ERR_CUDA;
    }
    h->stream = static_cast<cudaStream_t>(o.stream);
    // the two-step kernels keep more than 48 KB of shared memory per CTA
    if (!ring && !d3 && o.dtype != RLBM_F64 &&
        (o.landau == RLBM_LANDAU_FP32 ? fused2_prepare() : fused2_dfl_prepare()) != cudaSuccess) {
        cudaGetLastError();
        if (o.kernel == RLBM_KERNEL_FUSED2) {
            delete h;
            return RLBM_ERR_CUDA;
        }
    }
    if (o.kernel == RLBM_KERNEL_AUTO) {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        auto it = g_tuned.find(tune_key(h));
        if (it != g_tuned.end()) {
            h->cfg = it->second;
            h->tuned = true;
        }
    } else {
        h->cfg.kernel = o.kernel;
        if (o.kernel == RLBM_KERNEL_TMA) h->cfg.minb = 2;  // two CTAs per SM
        if (o.kernel == RLBM_KERNEL_PACKED && !d3) {     // the shape the autotuner usually picks
            h->cfg.bx = 128;
            h->cfg.by = 1;
            h->cfg.minb = 2;
        }
        if (o.kernel == RLBM_KERNEL_TWOPASS) {
            h->cfg.bx = 64;
            h->cfg.by = 2;
            h->cfg.minb = 3;
        }
        if (o.kernel == RLBM_KERNEL_PACKED4) {  // 128 threads per block, four blocks per SM
            h->cfg.bx = 128;
            h->cfg.by = 1;
            h->cfg.minb = 4;
        }
        if (o.kernel == RLBM_KERNEL_FUSED2) {  // 64 x 16 output tiles, two CTAs per SM
            h->cfg.bx = 64;
            h->cfg.by = 16;
            h->cfg.minb = 2;
            if (o.landau == RLBM_LANDAU_FP64 && o.dtype != RLBM_F64 && !ring) {
                h->cfg.by = 8;  // the refined-frame kernel comes in 64 x 8 tiles, four CTAs per SM
                h->cfg.minb = 4;
            }
        }
    }
    if (!h->tuned && o.kernel == RLBM_KERNEL_AUTO) {
        h->cfg.kernel = RLBM_KERNEL_GATHER;
        h->cfg.bx = 128;
        h->cfg.by = 2;
        if (o.rounding == RLBM_ROUND_STOCHASTIC) {
            h->cfg.kernel = RLBM_KERNEL_PACKED;  // the kernels that round stochastically
            h->cfg.bx = 128;
            h->cfg.by = 1;
            h->cfg.minb = 2;
        }
    }

    std::vector<Mode> modes;
    std::vector<int> ky_runs;  // first mode of each run of equal ky, then nmodes
    std::vector<int> modes3;
    if (forced) h->nmodes = d3 ? enumerate_modes3(fz.kmin, fz.kmax, &modes3) : enumerate_modes(fz.kmin, fz.kmax, &modes);
    if (forced && h->nmodes == 0) {
        delete h;
        return RLBM_ERR_ARG;
    }

    h->q[0] = dev_alloc(h, q_bytes(h));
    h->q[1] = dev_alloc(h, q_bytes(h));
    h->fields = static_cast<double *>(dev_alloc(h, fields_bytes(h)));
    h->partials = static_cast<double *>(dev_alloc(h, partials_bytes(h)));
    h->totals = static_cast<double *>(dev_alloc(h, 4 * sizeof(double)));
    h->bad = static_cast<int *>(dev_alloc(h, sizeof(int) * 4));
    h->errword = static_cast<int *>(dev_alloc(h, sizeof(int) * 4));
    bool ok = h->q[0] && h->q[1] && h->fields && h->partials && h->totals && h->bad && h->errword;
    if (forced) {
        h->F = dev_alloc(h, F_bytes(h));
        h->fnx = nx;
        h->fny = ny;
        h->twx = dev_alloc(h, tw_bytes(h, nx));
        h->twy = dev_alloc(h, tw_bytes(h, ny));
        h->coef = dev_alloc(h, coef_bytes(h));
        h->tabx = dev_alloc(h, tw_bytes(h, nx) * h->nmodes);
        h->taby = dev_alloc(h, tw_bytes(h, ny) * h->nmodes);
        ok = ok && h->F && h->twx && h->twy && h->coef && h->tabx && h->taby;
        if (d3) {
            h->modes3 = dev_alloc(h, mode3_bytes() * h->nmodes);
            h->twz = dev_alloc(h, tw_bytes(h, nz));
            h->tabz = dev_alloc(h, tw_bytes(h, nz) * h->nmodes);
            ok = ok && h->modes3 && h->twz && h->tabz;
        } else {
            h->modes = static_cast<Mode *>(dev_alloc(h, sizeof(Mode) * h->nmodes));
            for (int m = 0; m < h->nmodes; ++m)
                if (m == 0 || modes[m].ky != modes[m - 1].ky) ky_runs.push_back(m);
            ky_runs.push_back(h->nmodes);
            h->nky = (int)ky_runs.size() - 1;
            h->ky_start = static_cast<int *>(dev_alloc(h, sizeof(int) * ky_runs.size()));
            h->gtab = dev_alloc(h, gtab_bytes(h));
            ok = ok && h->modes && h->ky_start && h->gtab;
        }
    }
    if (!ok || cudaMallocHost(&h->host_small, 4096) != cudaSuccess) {
        cudaGetLastError();
        h->host_small = nullptr;
        rlbm_destroy(h);
        return RLBM_ERR_ALLOC;
    }
    rlbm_status st = RLBM_OK;
    if (forced && d3) {
        std::vector<unsigned char> hm(mode3_bytes() * h->nmodes);
        for (int m = 0; m < h->nmodes; ++m) host_mode3(hm.data(), m, modes3[3 * m], modes3[3 * m + 1], modes3[3 * m + 2]);
        cudaError_t e = cudaMemcpyAsync(h->modes3, hm.data(), hm.size(), cudaMemcpyHostToDevice, h->stream);
        void *tw[3] = {h->twx, h->twy, h->twz}, *tab[3] = {h->tabx, h->taby, h->tabz};
        const int n3[3] = {nx, ny, nz};
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
            e = launch_twiddles(o.dtype, tw[a], n3[a], h->stream);
            if (e == cudaSuccess) e = launch_mode_tables3(o.dtype, tab[a], h->modes3, h->nmodes, tw[a], n3[a], a, h->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = RLBM_ERR_CUDA;
    } else if (forced) {
        cudaError_t e = cudaMemcpyAsync(h->modes, modes.data(), sizeof(Mode) * h->nmodes, cudaMemcpyHostToDevice,
                                        h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->ky_start, ky_runs.data(), sizeof(int) * ky_runs.size(), cudaMemcpyHostToDevice,
                                h->stream);
        if (e == cudaSuccess) e = launch_twiddles(o.dtype, h->twx, nx, h->stream);
        if (e == cudaSuccess) e = launch_twiddles(o.dtype, h->twy, ny, h->stream);
        if (e == cudaSuccess)
            e = launch_mode_tables(o.dtype, h->tabx, h->taby, h->modes, h->nmodes, h->twx, h->twy, nx, ny, nx, ny, 0,
                                   0, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = RLBM_ERR_CUDA;
    }
    if (st == RLBM_OK && cudaMemsetAsync(h->errword, 0, sizeof(int) * 4, h->stream) != cudaSuccess) st = RLBM_ERR_CUDA;
    // tensor maps for the TMA kernel where it applies (a host-side encoding)
    if (st == RLBM_OK && !ring && !d3 && o.dtype == RLBM_F32 && o.landau == RLBM_LANDAU_FP32 && nx % 2 == 0 &&
        o.cfl == 1.0) {
        const StepParams p = params_of(h);
        bool enc = tma_encode_state(&h->tm_q[0], h->q[0], p) == cudaSuccess &&
                   tma_encode_state(&h->tm_q[1], h->q[1], p) == cudaSuccess;
        if (enc && forced) enc = tma_encode_force(&h->tm_F, h->F, p) == cudaSuccess;
        else if (enc) h->tm_F = h->tm_q[0];  // never read by the unforced kernel
        h->tm_ready = enc;
        cudaGetLastError();
        if (!enc && o.kernel == RLBM_KERNEL_TMA) st = RLBM_ERR_CUDA;
    }
    if (st == RLBM_OK) st = rlbm_init_fields_device(h, nullptr, nullptr, nullptr);
    if (st == RLBM_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = RLBM_ERR_CUDA;
    if (st != RLBM_OK) {
        rlbm_destroy(h);
        return st;
    }
    *out = h;
    return RLBM_OK;
}

extern "C" {

rlbm_status rlbm_create(int nx, int ny, rlbm_stencil stencil, double tau, const rlbm_forcing *forcing,
                        const rlbm_opts *opts, rlbm_t **out) {
    return create_impl(nx, ny, 1, false, stencil, tau, forcing, opts, out);
}

rlbm_status rlbm_create3d(int nx, int ny, int nz, double tau, const rlbm_forcing *forcing, const rlbm_opts *opts,
                          rlbm_t **out) {
    return create_impl(nx, ny, nz, true, RLBM_STENCIL_SPH26_SLAB, tau, forcing, opts, out);
}

}  // extern "C"

// Write f_eq of the given device fields into the current buffer.  A plain
// handle restarts its clock (step 0, current buffer 0); an ensemble member
// keeps the ensemble's clock and buffer parity.
static rlbm_status init_device_impl(rlbm_t *h, const double *d_eps, const double *d_vx, const double *d_vy,
                                    bool keep_clock, const double *d_vz = nullptr) {
    if (!keep_clock) {
        h->cur = 0;
        h->step = 0;
        h->force_epoch = -1;
    }
    if (h->d3)
        CUDA_TRY(h, launch_init3(h->opts.dtype, h->q[h->cur], params_of(h), d_eps, d_vx, d_vy, d_vz, h->stream));
    else if (h->ring)
        CUDA_TRY(h, launch_ring_init(h->opts.dtype, h->q[h->cur], params_of(h), d_eps, d_vx, d_vy, h->stream));
    else CUDA_TRY(h, launch_init(h->opts.dtype, h->q[h->cur], params_of(h), d_eps, d_vx, d_vy, h->stream));
    return RLBM_OK;
}

// The host fields are copied straight from the caller's memory, checked on
// the device (no host pass over the arrays), and only then turned into
// populations, so invalid fields leave the state untouched.
static rlbm_status init_host_impl(rlbm_t *h, const double *eps, const double *vx, const double *vy, bool keep_clock,
                                  const double *vz = nullptr) {
    const size_t n = nodes_of(h);
    const double *src[4] = {eps, vx, vy, vz};
    double *dptr[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < (h->d3 ? 4 : 3); ++k) {
        if (!src[k]) continue;
        dptr[k] = h->fields + k * n;
        CUDA_TRY(h, cudaMemcpyAsync(dptr[k], src[k], n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    int *bad_host = reinterpret_cast<int *>(h->host_small);
    CUDA_TRY(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->stream));
    if (h->d3) CUDA_TRY(h, launch_check_fields3(dptr[0], dptr[1], dptr[2], dptr[3], (long long)n, h->bad, h->stream));
    else CUDA_TRY(h, launch_check_fields(dptr[0], dptr[1], dptr[2], (long long)n, h->bad, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(bad_host, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (*bad_host) return fail(h, RLBM_ERR_ARG, "%d initial-field entries have eps <= 0, |v| >= 1 or non-finite values",
                               *bad_host);
    rlbm_status st = init_device_impl(h, dptr[0], dptr[1], dptr[2], keep_clock, dptr[3]);
    if (st != RLBM_OK) return st;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return RLBM_OK;
}

extern "C" {

rlbm_status rlbm_init_fields_device(rlbm_t *h, const double *d_eps, const double *d_vx, const double *d_vy) {
    CHECK_HANDLE(h);
    return init_device_impl(h, d_eps, d_vx, d_vy, false);  // a 3D handle: v_z = 0
}

rlbm_status rlbm_init_fields(rlbm_t *h, const double *eps, const double *vx, const double *vy) {
    CHECK_HANDLE(h);
    if (h->d3) return fail(h, RLBM_ERR_STATE, "3D lattice: use rlbm_init_fields3d");
    return init_host_impl(h, eps, vx, vy, false);
}

rlbm_status rlbm_init_fields3d(rlbm_t *h, const double *eps, const double *vx, const double *vy, const double *vz) {
    CHECK_HANDLE(h);
    if (!h->d3) return fail(h, RLBM_ERR_STATE, "not a 3D lattice");
    return init_host_impl(h, eps, vx, vy, false, vz);
}

rlbm_status rlbm_step(rlbm_t *h, int n) {
    CHECK_HANDLE(h);
    NvtxRange range("rlbm_step");
    if (n < 0) return fail(h, RLBM_ERR_ARG, "negative step count");
    while (n > 0) {
        int chunk = n;
        if (h->forced) {
            rlbm_status st = ensure_force(h);
            if (st != RLBM_OK) return st;
            const int left = h->forcing.redraw_period - (int)(h->step % h->forcing.redraw_period);
            chunk = std::min(n, left);
        }
        rlbm_status st = run_chunk(h, chunk);
        if (st != RLBM_OK) return st;
        h->step += chunk;
        n -= chunk;
    }
    return RLBM_OK;
}

rlbm_status rlbm_moments_device(rlbm_t *h, double *d_eps, double *d_vx, double *d_vy, double *d_totals) {
    CHECK_HANDLE(h);
    if (h->d3) return fail(h, RLBM_ERR_STATE, "3D lattice: use rlbm_moments3d");
    const StepParams p = params_of(h);
    CUDA_TRY(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->stream));
    if (h->ring)
        CUDA_TRY(h, launch_ring_moments(h->opts.dtype, h->q[h->cur], p, d_eps, d_vx, d_vy, h->partials, h->bad,
                                        h->stream));
    else
        CUDA_TRY(h, launch_moments(h->opts.dtype, h->opts.landau, h->q[h->cur], p, d_eps, d_vx, d_vy, h->partials,
                                   h->bad, h->stream));
    if (d_totals)
        CUDA_TRY(h, launch_reduce_partials(h->partials, moments_blocks(p), h->opts.eps0 * (double)h->nx * h->ny,
                                           d_totals, h->stream));
    return RLBM_OK;
}

rlbm_status rlbm_moments3d(rlbm_t *h, double *eps, double *vx, double *vy, double *vz, double totals[4]) {
    CHECK_HANDLE(h);
    if (!h->d3) return fail(h, RLBM_ERR_STATE, "not a 3D lattice");
    const size_t n = nodes_of(h);
    const StepParams p = params_of(h);
    double *dst[4] = {eps, vx, vy, vz};
    double *dev[4];
    for (int k = 0; k < 4; ++k) dev[k] = dst[k] ? h->fields + k * n : nullptr;
    CUDA_TRY(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->stream));
    CUDA_TRY(h, launch_moments3(h->opts.dtype, h->q[h->cur], p, dev[0], dev[1], dev[2], dev[3], h->partials, h->bad,
                                h->stream));
    if (totals)
        CUDA_TRY(h, launch_reduce_partials4(h->partials, moments3_blocks(p), h->opts.eps0 * (double)n, h->totals,
                                            h->stream));
    for (int k = 0; k < 4; ++k)
        if (dst[k]) CUDA_TRY(h, cudaMemcpyAsync(dst[k], dev[k], n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int *bad_host = reinterpret_cast<int *>(h->host_small);
    double *tot_host = h->host_small + 8;
    CUDA_TRY(h, cudaMemcpyAsync(bad_host, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (totals) CUDA_TRY(h, cudaMemcpyAsync(tot_host, h->totals, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (totals)
        for (int k = 0; k < 4; ++k) totals[k] = tot_host[k];
    rlbm_status st = check_errword(h);
    if (st != RLBM_OK) return st;
    if (*bad_host) return fail(h, RLBM_ERR_NAN, "%d nodes have no physical Landau frame", *bad_host);
    return RLBM_OK;
}

rlbm_status rlbm_moments(rlbm_t *h, double *eps, double *vx, double *vy, double totals[3]) {
    CHECK_HANDLE(h);
    NvtxRange range("rlbm_moments");
    const size_t n = (size_t)h->nx * h->ny;
    rlbm_status st = rlbm_moments_device(h, eps ? h->fields : nullptr, vx ? h->fields + n : nullptr,
                                         vy ? h->fields + 2 * n : nullptr, totals ? h->totals : nullptr);
    if (st != RLBM_OK) return st;
    double *dst[3] = {eps, vx, vy};
    for (int k = 0; k < 3; ++k)
        if (dst[k])
            CUDA_TRY(h, cudaMemcpyAsync(dst[k], h->fields + k * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                                        h->stream));
    int *bad_host = reinterpret_cast<int *>(h->host_small);
    double *tot_host = h->host_small + 8;
    CUDA_TRY(h, cudaMemcpyAsync(bad_host, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (totals)
        CUDA_TRY(h, cudaMemcpyAsync(tot_host, h->totals, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (totals)
        for (int k = 0; k < 3; ++k) totals[k] = tot_host[k];
    st = check_errword(h);
    if (st != RLBM_OK) return st;
    if (*bad_host) return fail(h, RLBM_ERR_NAN, "%d nodes have no physical Landau frame", *bad_host);
    return RLBM_OK;
}

}  // extern "C"

// Velocity components of the state the next collision sees into the fields
// buffer (vx at n, vy at 2n, vz at 3n for a 3D lattice), on the stream.
static rlbm_status velocity_to_fields(rlbm_t *h) {
    const size_t n = nodes_of(h);
    CUDA_TRY(h, cudaMemsetAsync(h->bad, 0, sizeof(int), h->stream));
    const StepParams p = params_of(h);
    if (h->d3)
        CUDA_TRY(h, launch_moments3(h->opts.dtype, h->q[h->cur], p, nullptr, h->fields + n, h->fields + 2 * n,
                                    h->fields + 3 * n, h->partials, h->bad, h->stream));
    else if (h->ring)
        CUDA_TRY(h, launch_ring_moments(h->opts.dtype, h->q[h->cur], p, nullptr, h->fields + n, h->fields + 2 * n,
                                        h->partials, h->bad, h->stream));
    else
        CUDA_TRY(h, launch_moments(h->opts.dtype, h->opts.landau, h->q[h->cur], p, nullptr, h->fields + n,
                                   h->fields + 2 * n, h->partials, h->bad, h->stream));
    return RLBM_OK;
}

// E(k) of the current velocity into dEk (device, nshells doubles).
static rlbm_status spectrum_on_device(rlbm_t *h, int nshells, double *dEk) {
    rlbm_status st = velocity_to_fields(h);
    if (st != RLBM_OK) return st;
    const size_t n = nodes_of(h);
    if (h->d3)
        CUDA_TRY(h, launch_spectrum3(h->fields + n, h->fields + 2 * n, h->fields + 3 * n, h->nx, h->ny, h->nz, nshells,
                                     h->spec_work, dEk, h->stream));
    else
        CUDA_TRY(h, launch_spectrum(h->fields + n, h->fields + 2 * n, h->nx, h->ny, nshells, h->spec_work, dEk,
                                    h->stream));
    return RLBM_OK;
}

extern "C" {

rlbm_status rlbm_energy_spectrum(rlbm_t *h, int nshells, double *Ek) {
    CHECK_HANDLE(h);
    NvtxRange range("rlbm_energy_spectrum");
    if (nshells < 1 || nshells > 4096 || !Ek) return fail(h, RLBM_ERR_ARG, "nshells must be in [1, 4096]");
    rlbm_status st0 = ensure_spectrum_work(h);
    if (st0 != RLBM_OK) return st0;
    double *dEk = h->spec_work + spectrum_doubles(h);
    rlbm_status st = spectrum_on_device(h, nshells, dEk);
    if (st != RLBM_OK) return st;
    int *bad_host = reinterpret_cast<int *>(h->host_small);
    CUDA_TRY(h, cudaMemcpyAsync(bad_host, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(Ek, dEk, nshells * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (*bad_host) return fail(h, RLBM_ERR_NAN, "%d nodes have no physical Landau frame", *bad_host);
    return RLBM_OK;
}

rlbm_status rlbm_filtered_velocity(rlbm_t *h, double kf, double *rms) {
    CHECK_HANDLE(h);
    if (!rms || !(kf >= 0.0)) return fail(h, RLBM_ERR_ARG, "kf must be >= 0 and rms non-NULL");
    rlbm_status st = ensure_spectrum_work(h);
    if (st != RLBM_OK) return st;
    const size_t n = nodes_of(h);
    st = velocity_to_fields(h);
    if (st != RLBM_OK) return st;
    double *dout = h->spec_work + spectrum_doubles(h);
    if (h->d3)
        CUDA_TRY(h, launch_band_power3(h->fields + n, h->fields + 2 * n, h->fields + 3 * n, h->nx, h->ny, h->nz, kf,
                                       h->spec_work, dout, h->stream));
    else
        CUDA_TRY(h, launch_band_power(h->fields + n, h->fields + 2 * n, h->nx, h->ny, kf, h->spec_work, dout,
                                      h->stream));
    double *host = h->host_small + 16;
    int *bad_host = reinterpret_cast<int *>(h->host_small);
    CUDA_TRY(h, cudaMemcpyAsync(host, dout, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(bad_host, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (*bad_host) return fail(h, RLBM_ERR_NAN, "%d nodes have no physical Landau frame", *bad_host);
    *rms = std::sqrt(*host);
    return RLBM_OK;
}

rlbm_status rlbm_spectrum_reset(rlbm_t *h) {
    CHECK_HANDLE(h);
    if (h->spec_acc) CUDA_TRY(h, cudaMemsetAsync(h->spec_acc, 0, 2 * 4096 * sizeof(double), h->stream));
    h->spec_count = 0;
    h->spec_nshells = 0;
    return RLBM_OK;
}

rlbm_status rlbm_spectrum_sample(rlbm_t *h, int nshells) {
    CHECK_HANDLE(h);
    if (nshells < 1 || nshells > 4096) return fail(h, RLBM_ERR_ARG, "nshells must be in [1, 4096]");
    if (h->spec_count > 0 && nshells != h->spec_nshells)
        return fail(h, RLBM_ERR_STATE, "sampling %d shells into a record of %d (reset first)", nshells,
                    h->spec_nshells);
    rlbm_status st = ensure_spectrum_work(h);
    if (st != RLBM_OK) return st;
    if (!h->spec_acc) {
        h->spec_acc = static_cast<double *>(dev_alloc(h, 2 * 4096 * sizeof(double)));
        if (!h->spec_acc) return fail(h, RLBM_ERR_ALLOC, "spectrum accumulators");
        CUDA_TRY(h, cudaMemsetAsync(h->spec_acc, 0, 2 * 4096 * sizeof(double), h->stream));
    }
    double *dEk = h->spec_work + spectrum_doubles(h);
    st = spectrum_on_device(h, nshells, dEk);
    if (st != RLBM_OK) return st;
    CUDA_TRY(h, launch_accumulate(dEk, nshells, h->spec_acc, h->spec_acc + 4096, h->stream));
    h->spec_count += 1;
    h->spec_nshells = nshells;
    return RLBM_OK;
}

rlbm_status rlbm_spectrum_stats(rlbm_t *h, int nshells, double *mean, double *sem, int *count) {
    CHECK_HANDLE(h);
    if (count) *count = h->spec_count;
    if (h->spec_count == 0) return fail(h, RLBM_ERR_STATE, "no spectrum samples");
    if (nshells < 1 || nshells > h->spec_nshells) return fail(h, RLBM_ERR_ARG, "nshells out of range");
    std::vector<double> sum(nshells), sq(nshells);
    CUDA_TRY(h, cudaMemcpyAsync(sum.data(), h->spec_acc, nshells * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(sq.data(), h->spec_acc + 4096, nshells * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const double m = (double)h->spec_count;
    for (int i = 0; i < nshells; ++i) {
        const double mu = sum[i] / m;
        if (mean) mean[i] = mu;
        if (sem) {
            const double var = (m > 1) ? std::max(0.0, (sq[i] - m * mu * mu) / (m - 1)) : 0.0;
            sem[i] = std::sqrt(var / m);
        }
    }
    return RLBM_OK;
}

rlbm_status rlbm_get_populations(rlbm_t *h, double *f) {
    CHECK_HANDLE(h);
    if (!f) return RLBM_ERR_ARG;
    const size_t layer = (size_t)h->nx * h->ny, n = nodes_of(h);
    const StepParams p = params_of(h);
    const size_t sb = storage_bytes(h->opts.dtype);
    for (int c = 0; c < h->ncls; ++c) {
        for (int z = 0; z < h->nz; ++z) {
            const void *qz = static_cast<const char *>(h->q[h->cur]) + (size_t)z * p.slab * sb;
            CUDA_TRY(h, launch_decode_class(h->opts.dtype, qz, c, class_weight(h, c), p, h->fields + z * layer,
                                            h->stream));
        }
        CUDA_TRY(h, cudaMemcpyAsync(f + c * n, h->fields, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    return RLBM_OK;
}

rlbm_status rlbm_set_populations(rlbm_t *h, const double *f) {
    CHECK_HANDLE(h);
    if (!f) return RLBM_ERR_ARG;
    const size_t layer = (size_t)h->nx * h->ny, n = nodes_of(h);
    const StepParams p = params_of(h);
    const size_t sb = storage_bytes(h->opts.dtype);
    for (int c = 0; c < h->ncls; ++c) {
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        CUDA_TRY(h, cudaMemcpyAsync(h->fields, f + c * n, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        for (int z = 0; z < h->nz; ++z) {
            void *qz = static_cast<char *>(h->q[h->cur]) + (size_t)z * p.slab * sb;
            CUDA_TRY(h, launch_encode_class(h->opts.dtype, qz, c, class_weight(h, c), p, h->fields + z * layer,
                                            h->stream));
        }
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return RLBM_OK;
}

rlbm_status rlbm_get_force3d(rlbm_t *h, double *Fx, double *Fy, double *Fz) {
    CHECK_HANDLE(h);
    if (!h->d3) return fail(h, RLBM_ERR_STATE, "not a 3D lattice");
    const size_t n = nodes_of(h), layer = (size_t)h->nx * h->ny;
    double *dst[3] = {Fx, Fy, Fz};
    if (!h->forced) {
        for (int k = 0; k < 3; ++k)
            if (dst[k]) memset(dst[k], 0, n * sizeof(double));
        return RLBM_OK;
    }
    rlbm_status st = ensure_force(h);
    if (st != RLBM_OK) return st;
    const StepParams p = params_of(h);
    const size_t cb = compute_bytes(h->opts.dtype);
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        for (int z = 0; z < h->nz; ++z) {
            // component k of layer z, read as the first component of a one-layer force array
            const void *Fk = static_cast<const char *>(h->F) + ((size_t)k * p.plane + (size_t)z * p.slab) * cb;
            CUDA_TRY(h, launch_force_to_f64(h->opts.dtype, Fk, 0, p, h->fields + z * layer, h->stream));
        }
        CUDA_TRY(h, cudaMemcpyAsync(dst[k], h->fields, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    return RLBM_OK;
}

rlbm_status rlbm_get_force(rlbm_t *h, double *Fx, double *Fy) {
    CHECK_HANDLE(h);
    if (h->d3) return fail(h, RLBM_ERR_STATE, "3D lattice: use rlbm_get_force3d");
    const size_t n = (size_t)h->nx * h->ny;
    if (!h->forced) {
        if (Fx) memset(Fx, 0, n * sizeof(double));
        if (Fy) memset(Fy, 0, n * sizeof(double));
        return RLBM_OK;
    }
    rlbm_status st = ensure_force(h);
    if (st != RLBM_OK) return st;
    const StepParams p = params_of(h);
    double *dst[2] = {Fx, Fy};
    for (int k = 0; k < 2; ++k) {
        if (!dst[k]) continue;
        CUDA_TRY(h, launch_force_to_f64(h->opts.dtype, h->F, k, p, h->fields, h->stream));
        CUDA_TRY(h, cudaMemcpyAsync(dst[k], h->fields, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    return RLBM_OK;
}

rlbm_status rlbm_set_force_frame(rlbm_t *h, int nx_global, int ny_global, int x0, int y0) {
    CHECK_HANDLE(h);
    if (h->d3) return fail(h, RLBM_ERR_STATE, "3D lattice: no force frame");
    if (nx_global < 4 || ny_global < 4 || x0 <= -nx_global || x0 >= nx_global || y0 <= -ny_global ||
        y0 >= ny_global)
        return fail(h, RLBM_ERR_ARG, "force frame %dx%d at (%d, %d) is not valid", nx_global, ny_global, x0, y0);
    if (h->forced && !(h->forcing.kmax < std::min(nx_global, ny_global) / 2))
        return fail(h, RLBM_ERR_ARG, "forcing shell kmax %d needs a frame wider than %d", h->forcing.kmax,
                    2 * h->forcing.kmax);
    if (!h->forced) return RLBM_OK;  // nothing is drawn
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (nx_global != h->fnx || ny_global != h->fny) {
        void *tx = dev_alloc(h, tw_bytes(h, nx_global)), *ty = dev_alloc(h, tw_bytes(h, ny_global));
        if (!tx || !ty) {
            if (tx) dev_free(h, tx, tw_bytes(h, nx_global));
            if (ty) dev_free(h, ty, tw_bytes(h, ny_global));
            return fail(h, RLBM_ERR_ALLOC, "force frame twiddles");
        }
        dev_free(h, h->twx, tw_bytes(h, h->fnx));
        dev_free(h, h->twy, tw_bytes(h, h->fny));
        h->twx = tx;
        h->twy = ty;
        h->fnx = nx_global;
        h->fny = ny_global;
        CUDA_TRY(h, launch_twiddles(h->opts.dtype, h->twx, nx_global, h->stream));
        CUDA_TRY(h, launch_twiddles(h->opts.dtype, h->twy, ny_global, h->stream));
    }
    h->fx0 = x0;
    h->fy0 = y0;
    CUDA_TRY(h, launch_mode_tables(h->opts.dtype, h->tabx, h->taby, h->modes, h->nmodes, h->twx, h->twy, h->nx, h->ny,
                                   h->fnx, h->fny, x0, y0, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->force_epoch = -1;  // the next step synthesises the force in the new frame
    return RLBM_OK;
}

// Rows [row, row + nrows) of every class plane, with their pitch padding:
// one 2D copy of ncls blocks of nrows * pitch elements.
static rlbm_status halo_copy(rlbm_t *h, int row, int nrows, void *d_buf, bool pack) {
    CHECK_HANDLE(h);
    if (h->d3) return fail(h, RLBM_ERR_STATE, "3D lattice: no halo rows");
    if (!d_buf || nrows < 1 || row < 0 || row + nrows > h->ny)
        return fail(h, RLBM_ERR_ARG, "halo rows [%d, %d) outside 0..%d", row, row + nrows, h->ny);
    const size_t es = storage_bytes(h->opts.dtype);
    const size_t width = (size_t)nrows * h->pitch * es, plane = (size_t)h->ny * h->pitch * es;
    char *state = static_cast<char *>(h->q[h->cur]) + (size_t)row * h->pitch * es;
    if (pack)
        CUDA_TRY(h, cudaMemcpy2DAsync(d_buf, width, state, plane, width, h->ncls, cudaMemcpyDeviceToDevice, h->stream));
    else
        CUDA_TRY(h, cudaMemcpy2DAsync(state, plane, d_buf, width, width, h->ncls, cudaMemcpyDeviceToDevice, h->stream));
    return RLBM_OK;
}

rlbm_status rlbm_halo_pack(rlbm_t *h, int row, int nrows, void *d_buf) { return halo_copy(h, row, nrows, d_buf, true); }

rlbm_status rlbm_halo_unpack(rlbm_t *h, int row, int nrows, const void *d_buf) {
    return halo_copy(h, row, nrows, const_cast<void *>(d_buf), false);
}

rlbm_status rlbm_get_info(rlbm_t *h, rlbm_info_t *info) {
    if (!h || !info) return RLBM_ERR_ARG;
    info->nx = h->nx;
    info->ny = h->ny;
    info->pitch = h->pitch;
    info->nclasses = h->ncls;
    info->nz = h->nz;
    info->launch_budget = h->cfg.minb;
    info->dtype = h->opts.dtype;
    info->kernel = h->cfg.kernel;
    info->block_x = h->cfg.bx;
    info->block_y = h->cfg.by;
    info->nmodes = h->forced ? h->nmodes : 0;
    info->step = h->step;
    info->tau = h->tau;
    info->eps0 = h->opts.eps0;
    info->scale = h->opts.scale;
    info->steps_per_launch = steps_per_launch(h->cfg);
    info->bytes_per_node = ((size_t)2 * h->ncls * storage_bytes(h->opts.dtype) +
                            (h->forced ? (h->d3 ? 3 : 2) * compute_bytes(h->opts.dtype) : 0)) /
                           (size_t)info->steps_per_launch;
    info->device_bytes = h->device_bytes;
    info->populations = h->q[h->cur];
    return RLBM_OK;
}

rlbm_status rlbm_autotune(rlbm_t *h, int reps, int *chosen_kernel, int *block_x, int *block_y) {
    CHECK_HANDLE(h);
    NvtxRange range("rlbm_autotune");
    if (reps < 1) reps = 20;
    rlbm_status st = ensure_force(h);
    if (st != RLBM_OK) return st;
    const StepParams p = params_of(h);
    cudaEvent_t a = nullptr, b = nullptr;
    CUDA_TRY(h, cudaEventCreate(&a));
    CUDA_TRY(h, cudaEventCreate(&b));
    float best_ms = 1e30f;
    LaunchCfg best = h->cfg;
    for (const LaunchCfg &c : kCandidates) {
        if (h->opts.kernel != RLBM_KERNEL_AUTO && c.kernel != h->opts.kernel) continue;
        if (!candidate_applies(h, c)) continue;
        // the trial steps read the current state and overwrite only the spare buffer
        bool ok = true;
        for (int i = 0; i < 2 + reps && ok; ++i) {
            if (i == 2) ok = cudaEventRecord(a, h->stream) == cudaSuccess;
            ok = ok && launch_step_h(h, c, h->q[h->cur], h->q[h->cur ^ 1], p) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            continue;
        }
        CUDA_TRY(h, cudaEventRecord(b, h->stream));
        CUDA_TRY(h, cudaEventSynchronize(b));
        float ms = 0.f;
        CUDA_TRY(h, cudaEventElapsedTime(&ms, a, b));
        ms /= (float)steps_per_launch(c);  // per lattice step
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->cfg = best;
    h->tuned = true;
    drop_graphs(h);
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        g_tuned[tune_key(h)] = best;
    }
    if (chosen_kernel) *chosen_kernel = best.kernel;
    if (block_x) *block_x = best.bx;
    if (block_y) *block_y = best.by;
    return RLBM_OK;
}

}  // extern "C"

extern "C" {
rlbm_status rlbm_set_launch(rlbm_t *h, int kernel, int block_x, int block_y, int launch_budget) {
    CHECK_HANDLE(h);
    if (h->opts.kernel != RLBM_KERNEL_AUTO && kernel != h->opts.kernel)
        return fail(h, RLBM_ERR_ARG, "the handle was created for kernel %d", h->opts.kernel);
    for (const LaunchCfg &c : kCandidates) {
        if (c.kernel != kernel || c.bx != block_x || c.by != block_y || c.minb != launch_budget) continue;
        if (!candidate_applies(h, c)) break;
        // one trial launch into the spare buffer: the launcher's own checks
        const StepParams p = params_of(h);
        rlbm_status st = ensure_force(h);
        if (st != RLBM_OK) return st;
        if (launch_step_h(h, c, h->q[h->cur], h->q[h->cur ^ 1], p) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, RLBM_ERR_ARG, "launch shape does not fit this lattice");
        }
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        h->cfg = c;
        drop_graphs(h);
        return RLBM_OK;
    }
    return fail(h, RLBM_ERR_ARG, "no such launch shape for this lattice");
}
}  // extern "C"

// Checkpoint layout: this header, then the current state buffer verbatim
// (ncls planes of nz * ny * pitch elements of the storage type).
struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t nx, ny, nz, pitch, ncls, dtype, kind, forced;
    double tau, eps0, scale, cfl, eta_s, dt;
    int32_t kmin, kmax, redraw_period, rounding;
    double amp;
    uint64_t seed;
    int64_t step;
    uint64_t state_bytes;
};
static const char kCkptMagic[8] = {'R', 'L', 'B', 'M', 'C', 'K', 'P', 'T'};

static CkptHeader ckpt_header_of(const rlbm_t *h) {
    CkptHeader c;
    memset(&c, 0, sizeof c);
    memcpy(c.magic, kCkptMagic, 8);
    c.version = 1;
    c.header_bytes = sizeof(CkptHeader);
    c.nx = h->nx;
    c.ny = h->ny;
    c.nz = h->nz;
    c.pitch = h->pitch;
    c.ncls = h->ncls;
    c.dtype = h->opts.dtype;
    c.kind = h->ring ? 1 : (h->d3 ? 2 : 0);
    c.forced = h->forced ? 1 : 0;
    c.tau = h->tau;
    c.eps0 = h->opts.eps0;
    c.scale = h->opts.scale;
    c.cfl = h->opts.cfl;
    c.eta_s = h->opts.eta_s;
    c.dt = h->opts.dt;
    if (h->forced) {
        c.kmin = h->forcing.kmin;
        c.kmax = h->forcing.kmax;
        c.redraw_period = h->forcing.redraw_period;
        c.amp = h->forcing.amp;
        c.seed = h->forcing.seed;
    }
    c.rounding = h->opts.rounding;
    c.step = h->step;
    c.state_bytes = q_bytes(h);
    return c;
}

extern "C" {

rlbm_status rlbm_checkpoint_size(rlbm_t *h, size_t *bytes) {
    CHECK_HANDLE(h);
    if (!bytes) return RLBM_ERR_ARG;
    *bytes = sizeof(CkptHeader) + q_bytes(h);
    return RLBM_OK;
}

rlbm_status rlbm_checkpoint_save(rlbm_t *h, void *buf, size_t len) {
    CHECK_HANDLE(h);
    const size_t need = sizeof(CkptHeader) + q_bytes(h);
    if (!buf || len < need) return fail(h, RLBM_ERR_ARG, "checkpoint needs %zu bytes, got %zu", need, len);
    const CkptHeader c = ckpt_header_of(h);
    memcpy(buf, &c, sizeof c);
    CUDA_TRY(h, cudaMemcpyAsync(static_cast<char *>(buf) + sizeof c, h->q[h->cur], q_bytes(h), cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return check_errword(h);
}

rlbm_status rlbm_checkpoint_load(rlbm_t *h, const void *buf, size_t len) {
    CHECK_HANDLE(h);
    if (!buf || len < sizeof(CkptHeader)) return fail(h, RLBM_ERR_ARG, "not a checkpoint (too short)");
    CkptHeader c;
    memcpy(&c, buf, sizeof c);
    CkptHeader mine = ckpt_header_of(h);
    if (memcmp(c.magic, kCkptMagic, 8) != 0 || c.version != 1 || c.header_bytes != sizeof(CkptHeader))
        return fail(h, RLBM_ERR_ARG, "not a checkpoint of this library version");
    mine.step = c.step;  // the only field that may differ
    if (memcmp(&c, &mine, sizeof c) != 0)
        return fail(h, RLBM_ERR_ARG, "checkpoint of a different lattice configuration");
    if (len < sizeof c + c.state_bytes) return fail(h, RLBM_ERR_ARG, "checkpoint truncated");
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->q[0], static_cast<const char *>(buf) + sizeof c, c.state_bytes,
                                cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->step = c.step;
    h->force_epoch = -1;
    return RLBM_OK;
}

rlbm_status rlbm_synchronize(rlbm_t *h) {
    CHECK_HANDLE(h);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return check_errword(h);
}

rlbm_status rlbm_last_error(rlbm_t *h, char *buf, size_t len) {
    if (!h || !buf || len == 0) return RLBM_ERR_ARG;
    snprintf(buf, len, "%s", h->msg.c_str());
    return RLBM_OK;
}


}  // extern "C"

// ---------------------------------------------------------------- ensemble
// An ensemble keeps one ordinary handle per lattice (buffers, force field,
// diagnostics) on a shared stream and advances all of them with one
// k_step_batch launch per step over a flat tile list.
struct rlbm_batch {
    std::vector<rlbm_t *> runs;
    rlbm_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0;
    LaunchCfg cfg;         // tile = cfg.bx * run_length columns x cfg.by rows
    int grid = 0;          // blocks of the persistent launch
    int ntiles = 0;
    BatchRun *desc[2] = {nullptr, nullptr};  // device descriptors for parity 0 / 1
    ForceJob *jobs = nullptr;  // device: the forced members' force synthesis, for epoch starts in three launches
    int njobs = 0, job_nmodes = 0, job_nruns = 0, job_nx = 0, job_ny = 0;  // count and grid extents
    int cur = 0;
    long long step = 0;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    rlbm_status status = RLBM_OK;
    std::string msg;
};

static rlbm_status bfail(rlbm_batch_t *b, rlbm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->msg = buf;
    if (st == RLBM_ERR_CUDA || st == RLBM_ERR_TIMEOUT) b->status = st;
    return st;
}

#define BCUDA_TRY(b, call)                                                                                  \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return bfail(b, RLBM_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                            __FILE__, __LINE__);                                            \
    } while (0)

#define CHECK_BATCH(b)                                   \
    do {                                                 \
        if (!(b)) return RLBM_ERR_ARG;                   \
        if ((b)->status != RLBM_OK) return (b)->status;  \
        if (cudaSetDevice((b)->device) != cudaSuccess) return bfail(b, RLBM_ERR_CUDA, "cudaSetDevice failed"); \
    } while (0)

static void batch_drop_graphs(rlbm_batch_t *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Host copy of the descriptors for a launch shape; returns the tile count.
static int batch_descriptors(const rlbm_batch_t *b, const LaunchCfg &cfg, int parity, std::vector<BatchRun> *out) {
    // columns per tile unit: node pairs (packed), whole nodes (two-step tiles of bx x by nodes), runs
    const int V = (cfg.kernel == RLBM_KERNEL_PACKED) ? 2 : (cfg.kernel == RLBM_KERNEL_FUSED2) ? 1 : run_length(b->opts.dtype);
    int t0 = 0;
    out->clear();
    for (rlbm_t *h : b->runs) {
        BatchRun r;
        r.qin = h->q[parity];
        r.qout = h->q[parity ^ 1];
        r.F = h->forced ? h->F : nullptr;
        r.p = params_of(h);
        const int cols = h->nx / V;
        r.tiles_x = (cols + cfg.bx - 1) / cfg.bx;
        const int tiles_y = (h->ny + cfg.by - 1) / cfg.by;
        r.tile0 = t0;
        t0 += r.tiles_x * tiles_y;
        out->push_back(r);
    }
    return t0;
}

static rlbm_status batch_upload(rlbm_batch_t *b, const LaunchCfg &cfg) {
    std::vector<BatchRun> d[2];
    int nt = 0;
    for (int par = 0; par < 2; ++par) nt = batch_descriptors(b, cfg, par, &d[par]);
    BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
    for (int par = 0; par < 2; ++par)
        BCUDA_TRY(b, cudaMemcpy(b->desc[par], d[par].data(), sizeof(BatchRun) * d[par].size(), cudaMemcpyHostToDevice));
    b->ntiles = nt;
    return RLBM_OK;
}

static int sm_count(int device) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

// One launch of the ensemble step with launch shape c: two steps (two-step
// tiles, two != 0) or one.
static cudaError_t batch_launch(const rlbm_batch_t *b, const LaunchCfg &c, int grid, int two) {
    if (c.kernel == RLBM_KERNEL_FUSED2)
        return launch_batch_fused2(b->opts.dtype, b->opts.landau, c, grid, b->desc[b->cur], (int)b->runs.size(),
                                   b->ntiles, two, b->stream);
    return launch_batch(b->opts.dtype, b->opts.landau, c, grid, b->desc[b->cur], (int)b->runs.size(), b->ntiles,
                        b->stream);
}

static rlbm_status batch_launch_steps(rlbm_batch_t *b, int n) {
    const int spl = steps_per_launch(b->cfg);
    for (int i = 0; i < n; i += spl) {
        const int two = (spl == 2 && i + 2 <= n) ? 1 : 0;
        BCUDA_TRY(b, batch_launch(b, b->cfg, b->grid, two));
        b->cur ^= 1;
        if (spl == 2 && !two) break;  // the odd last step
    }
    return RLBM_OK;
}

// As run_chunk: graphs for even parts of several launches only.
static rlbm_status batch_run_chunk(rlbm_batch_t *b, int n) {
    const int even = n & ~1;
    const bool graphs = b->opts.use_graphs && b->stream != nullptr && n >= 2 && launches_for(b->cfg, even) >= 2;
    if (!graphs) return batch_launch_steps(b, n);
    auto key = std::make_pair(even, b->cur);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        const int cur0 = b->cur;
        BCUDA_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        rlbm_status st = batch_launch_steps(b, even);
        cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
        b->cur = cur0;
        if (st != RLBM_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ec != cudaSuccess) return bfail(b, RLBM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) return bfail(b, RLBM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
        it = b->graphs.emplace(key, ge).first;
    }
    BCUDA_TRY(b, cudaGraphLaunch(it->second, b->stream));
    b->cur ^= launches_for(b->cfg, even) & 1;
    if (even != n) return batch_launch_steps(b, 1);
    return RLBM_OK;
}

// Bring an ensemble member's own bookkeeping in line with the ensemble.
static void batch_sync_member(const rlbm_batch_t *b, rlbm_t *h) {
    h->cur = b->cur;
    h->step = b->step;
}

static rlbm_status batch_member(rlbm_batch_t *b, int run, rlbm_t **h) {
    if (run < 0 || run >= (int)b->runs.size()) return bfail(b, RLBM_ERR_ARG, "run index %d out of range", run);
    *h = b->runs[run];
    batch_sync_member(b, *h);
    return RLBM_OK;
}

static rlbm_status from_member(rlbm_batch_t *b, rlbm_t *h, rlbm_status st) {
    if (st != RLBM_OK) {
        b->msg = h->msg;
        if (st == RLBM_ERR_CUDA || st == RLBM_ERR_TIMEOUT) b->status = st;
    }
    return st;
}

// The forced members' force synthesis as one job list on the device (what
// ensure_force launches per member), built once at create.
static rlbm_status batch_build_jobs(rlbm_batch_t *b) {
    std::vector<ForceJob> jobs;
    for (const rlbm_t *h : b->runs) {
        if (!h->forced || h->nmodes <= 0) continue;
        ForceJob j;
        j.modes = h->modes;
        j.coef = h->coef;
        j.run_start = h->ky_start;
        j.G = h->gtab;
        j.X = h->tabx;
        j.Y = h->taby;
        j.F = h->F;
        j.amp = h->forcing.amp;
        j.seed = (unsigned long long)h->forcing.seed;
        j.period = h->forcing.redraw_period;
        j.nmodes = h->nmodes;
        j.nruns = h->nky;
        j.p = params_of(h);
        jobs.push_back(j);
        b->job_nmodes = std::max(b->job_nmodes, h->nmodes);
        b->job_nruns = std::max(b->job_nruns, h->nky);
        b->job_nx = std::max(b->job_nx, h->nx);
        b->job_ny = std::max(b->job_ny, h->ny);
    }
    if (jobs.empty() || jobs.size() > 65535 || b->job_nruns > 65535) return RLBM_OK;  // member by member (grid limits)
    b->jobs = static_cast<ForceJob *>(dev_alloc(b->runs[0], sizeof(ForceJob) * jobs.size()));
    if (!b->jobs) return RLBM_ERR_ALLOC;
    b->njobs = (int)jobs.size();
    BCUDA_TRY(b, cudaMemcpy(b->jobs, jobs.data(), sizeof(ForceJob) * jobs.size(), cudaMemcpyHostToDevice));
    return RLBM_OK;
}

// Bring every forced member's force to the epoch of the ensemble's step.
// Where each member that needs a new force starts an epoch at this step (a
// run stepped from its start), one ensemble-wide synthesis in three launches
// redraws every member that starts an epoch here (a member already holding
// that epoch's force gets the same values again); otherwise member by member
// (192 launches for 64 members).
static rlbm_status batch_ensure_forces(rlbm_batch_t *b) {
    bool any = false, aligned = true;
    for (rlbm_t *h : b->runs) {
        if (!h->forced) continue;
        batch_sync_member(b, h);
        if (b->step / h->forcing.redraw_period == h->force_epoch) continue;
        any = true;
        if (b->step % h->forcing.redraw_period != 0) aligned = false;
    }
    if (!any) return RLBM_OK;
    if (aligned && b->njobs > 0) {
        NvtxRange range("rlbm_force_epoch");
        BCUDA_TRY(b, launch_force_jobs(b->opts.dtype, b->jobs, b->njobs, b->job_nmodes, b->job_nruns, b->job_nx,
                                       b->job_ny, b->step, b->stream));
        for (rlbm_t *h : b->runs)
            if (h->forced && h->nmodes > 0 && b->step % h->forcing.redraw_period == 0)
                h->force_epoch = b->step / h->forcing.redraw_period;
        return RLBM_OK;
    }
    for (rlbm_t *h : b->runs) {
        if (!h->forced) continue;
        rlbm_status st = from_member(b, h, ensure_force(h));
        if (st != RLBM_OK) return st;
    }
    return RLBM_OK;
}

extern "C" {

void rlbm_batch_destroy(rlbm_batch_t *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    batch_drop_graphs(b);
    if (!b->runs.empty()) {
        for (int par = 0; par < 2; ++par)
            dev_free(b->runs[0], b->desc[par], sizeof(BatchRun) * b->runs.size());
        if (b->jobs) dev_free(b->runs[0], b->jobs, sizeof(ForceJob) * b->njobs);
    }
    for (rlbm_t *h : b->runs) rlbm_destroy(h);
    delete b;
}

rlbm_status rlbm_batch_create(int nruns, const rlbm_run_desc *runs, const rlbm_opts *opts, rlbm_batch_t **out) {
    if (!out) return RLBM_ERR_ARG;
    *out = nullptr;
    if (nruns < 1 || !runs) return RLBM_ERR_ARG;
    rlbm_opts o;
    rlbm_opts_default(&o);
    if (opts) o = *opts;
    if (o.dtype < RLBM_F64 || o.dtype > RLBM_F16) return RLBM_ERR_ARG;
    // body of the ensemble step: the vector kernel (AUTO starts there), packed lanes, or two steps per launch
    const int bk = o.kernel;
    if (bk != RLBM_KERNEL_AUTO && bk != RLBM_KERNEL_GATHER_VEC && bk != RLBM_KERNEL_PACKED &&
        bk != RLBM_KERNEL_FUSED2)
        return RLBM_ERR_ARG;
    const bool lanes = bk == RLBM_KERNEL_PACKED || bk == RLBM_KERNEL_FUSED2;
    if (lanes && (o.dtype == RLBM_F64 || o.landau != RLBM_LANDAU_FP32)) return RLBM_ERR_ARG;
    // ensembles round to nearest unless asked otherwise; stochastic rounding needs a packed-lane body
    if (o.rounding < RLBM_ROUND_DEFAULT || o.rounding > RLBM_ROUND_STOCHASTIC) return RLBM_ERR_ARG;
    if (o.rounding == RLBM_ROUND_DEFAULT || (o.dtype != RLBM_BF16 && o.dtype != RLBM_F16))
        o.rounding = RLBM_ROUND_NEAREST;
    if (o.rounding == RLBM_ROUND_STOCHASTIC && !lanes) return RLBM_ERR_ARG;
    const int V = lanes ? 2 : run_length(o.dtype);
    for (int r = 0; r < nruns; ++r) {
        if (runs[r].nx % V != 0) return RLBM_ERR_ARG;  // the ensemble kernel works on runs of V nodes
        if (lanes && (long long)NC * runs[r].ny * ((runs[r].nx + 31) & ~31) >= (1ll << 31) - 1)
            return RLBM_ERR_ARG;  // the packed ensemble bodies index with 32-bit offsets
    }
    if (!(o.cfl == 0.0 || o.cfl == 1.0)) return RLBM_ERR_ARG;  // and streams at CFL 1
    rlbm_batch_t *b = new rlbm_batch_t();
    b->opts = o;
    b->stream = static_cast<cudaStream_t>(o.stream);
    rlbm_opts member = o;
    member.kernel = lanes ? RLBM_KERNEL_PACKED : RLBM_KERNEL_GATHER_VEC;  // validates the member's shape
    for (int r = 0; r < nruns; ++r) {
        rlbm_t *h = nullptr;
        rlbm_status st = rlbm_create(runs[r].nx, runs[r].ny, RLBM_STENCIL_SPH26_SLAB, runs[r].tau, &runs[r].forcing,
                                     &member, &h);
        if (st != RLBM_OK) {
            rlbm_batch_destroy(b);
            return st;
        }
        b->runs.push_back(h);
    }
    b->device = b->runs[0]->device;
    b->opts.landau = b->runs[0]->opts.landau;
    for (int par = 0; par < 2; ++par) {
        b->desc[par] = static_cast<BatchRun *>(dev_alloc(b->runs[0], sizeof(BatchRun) * nruns));
        if (!b->desc[par]) {
            rlbm_batch_destroy(b);
            return RLBM_ERR_ALLOC;
        }
    }
    rlbm_status stj = batch_build_jobs(b);
    if (stj != RLBM_OK) {
        rlbm_batch_destroy(b);
        return stj;
    }
    if (bk == RLBM_KERNEL_PACKED) b->cfg = LaunchCfg{RLBM_KERNEL_PACKED, 64, 2, 1};
    else if (bk == RLBM_KERNEL_FUSED2) b->cfg = LaunchCfg{RLBM_KERNEL_FUSED2, 64, 8, 4};
    else b->cfg = LaunchCfg{RLBM_KERNEL_GATHER_VEC, 64, 2, 1};
    rlbm_status st = batch_upload(b, b->cfg);
    if (st != RLBM_OK) {
        rlbm_batch_destroy(b);
        return st;
    }
    b->grid = std::min(b->ntiles, 8 * sm_count(b->device));
    *out = b;
    return RLBM_OK;
}

rlbm_status rlbm_create_batch(int nruns, const rlbm_run_desc *runs, const rlbm_opts *opts, rlbm_batch_t **out) {
    return rlbm_batch_create(nruns, runs, opts, out);
}

rlbm_status rlbm_batch_init_fields(rlbm_batch_t *b, int run, const double *eps, const double *vx, const double *vy) {
    CHECK_BATCH(b);
    rlbm_t *h = nullptr;
    rlbm_status st = batch_member(b, run, &h);
    if (st != RLBM_OK) return st;
    return from_member(b, h, init_host_impl(h, eps, vx, vy, true));
}

rlbm_status rlbm_batch_step(rlbm_batch_t *b, int n) {
    CHECK_BATCH(b);
    if (n < 0) return bfail(b, RLBM_ERR_ARG, "negative step count");
    while (n > 0) {
        int chunk = n;
        rlbm_status st0 = batch_ensure_forces(b);
        if (st0 != RLBM_OK) return st0;
        for (rlbm_t *h : b->runs) {
            if (!h->forced) continue;
            const int left = h->forcing.redraw_period - (int)(b->step % h->forcing.redraw_period);
            chunk = std::min(chunk, left);
        }
        rlbm_status st = batch_run_chunk(b, chunk);
        if (st != RLBM_OK) return st;
        b->step += chunk;
        n -= chunk;
    }
    for (rlbm_t *h : b->runs) batch_sync_member(b, h);
    return RLBM_OK;
}

rlbm_status rlbm_batch_moments(rlbm_batch_t *b, int run, double *eps, double *vx, double *vy, double totals[3]) {
    CHECK_BATCH(b);
    rlbm_t *h = nullptr;
    rlbm_status st = batch_member(b, run, &h);
    if (st != RLBM_OK) return st;
    return from_member(b, h, rlbm_moments(h, eps, vx, vy, totals));
}

rlbm_status rlbm_batch_energy_spectrum(rlbm_batch_t *b, int run, int nshells, double *Ek) {
    CHECK_BATCH(b);
    rlbm_t *h = nullptr;
    rlbm_status st = batch_member(b, run, &h);
    if (st != RLBM_OK) return st;
    return from_member(b, h, rlbm_energy_spectrum(h, nshells, Ek));
}

rlbm_status rlbm_batch_get_populations(rlbm_batch_t *b, int run, double *f) {
    CHECK_BATCH(b);
    rlbm_t *h = nullptr;
    rlbm_status st = batch_member(b, run, &h);
    if (st != RLBM_OK) return st;
    return from_member(b, h, rlbm_get_populations(h, f));
}

rlbm_status rlbm_batch_autotune(rlbm_batch_t *b, int reps, int *block_x, int *block_y, int *grid) {
    CHECK_BATCH(b);
    if (reps < 1) reps = 10;
    rlbm_status st0 = batch_ensure_forces(b);
    if (st0 != RLBM_OK) return st0;
    static const int shapes[][2] = {{32, 4}, {64, 2}, {128, 1}, {32, 8}, {64, 4}, {128, 2}, {32, 2}, {64, 1}};
    // two-step tiles (bx x by nodes) and their launch budgets
    static const int tiles2[][3] = {{64, 8, 4}, {64, 16, 2}, {32, 16, 4}, {128, 8, 2}};
    // body: the vector kernel, the packed-lane kernel (FP32 compute, FP32 Landau), or two steps per
    // launch with the packed body
    bool packed_ok = b->opts.dtype != RLBM_F64 && b->opts.landau == RLBM_LANDAU_FP32;
    for (const rlbm_t *h : b->runs)  // the packed ensemble body indexes with 32-bit offsets
        if ((long long)NC * h->ny * h->pitch >= (1ll << 31) - 1) packed_ok = false;
    static const int bodies[][2] = {{RLBM_KERNEL_GATHER_VEC, 1}, {RLBM_KERNEL_PACKED, 1}, {RLBM_KERNEL_PACKED, 3},
                                    {RLBM_KERNEL_FUSED2, 0}};
    const int sms = sm_count(b->device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCUDA_TRY(b, cudaEventCreate(&e0));
    BCUDA_TRY(b, cudaEventCreate(&e1));
    float best_ms = 1e30f;
    LaunchCfg best = b->cfg;
    int best_grid = b->grid;
    for (const auto &body : bodies)
    for (int si = 0; si < 8; ++si) {
        if (b->opts.kernel != RLBM_KERNEL_AUTO && body[0] != b->opts.kernel) continue;
        if ((body[0] == RLBM_KERNEL_PACKED || body[0] == RLBM_KERNEL_FUSED2) && !packed_ok) continue;
        if (body[0] == RLBM_KERNEL_FUSED2 && si >= 4) continue;
        LaunchCfg c;
        c.kernel = body[0];
        c.minb = body[0] == RLBM_KERNEL_FUSED2 ? tiles2[si][2] : body[1];
        c.bx = body[0] == RLBM_KERNEL_FUSED2 ? tiles2[si][0] : shapes[si][0];
        c.by = body[0] == RLBM_KERNEL_FUSED2 ? tiles2[si][1] : shapes[si][1];
        rlbm_status st = batch_upload(b, c);
        if (st != RLBM_OK) return st;
        const int grids[] = {sms, 2 * sms, 4 * sms, 8 * sms, 16 * sms, b->ntiles};
        for (int g : grids) {
            g = std::min(g, b->ntiles);
            // trial launches read the current state and overwrite only the spare buffers
            bool ok = true;
            for (int i = 0; i < 1 + reps && ok; ++i) {
                if (i == 1) ok = cudaEventRecord(e0, b->stream) == cudaSuccess;
                ok = ok && batch_launch(b, c, g, 1) == cudaSuccess;
            }
            if (!ok) {
                cudaGetLastError();
                continue;
            }
            BCUDA_TRY(b, cudaEventRecord(e1, b->stream));
            BCUDA_TRY(b, cudaEventSynchronize(e1));
            float ms = 0.f;
            BCUDA_TRY(b, cudaEventElapsedTime(&ms, e0, e1));
            ms /= (float)steps_per_launch(c);  // per ensemble step
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
                best_grid = g;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cfg = best;
    rlbm_status st = batch_upload(b, best);
    if (st != RLBM_OK) return st;
    b->grid = std::min(best_grid, b->ntiles);
    batch_drop_graphs(b);
    if (block_x) *block_x = best.bx;
    if (block_y) *block_y = best.by;
    if (grid) *grid = b->grid;
    return RLBM_OK;
}

rlbm_status rlbm_batch_get_info(rlbm_batch_t *b, rlbm_batch_info_t *info) {
    if (!b || !info) return RLBM_ERR_ARG;
    info->nruns = (int)b->runs.size();
    info->dtype = b->opts.dtype;
    info->block_x = b->cfg.bx;
    info->block_y = b->cfg.by;
    info->grid = b->grid;
    info->kernel = b->cfg.kernel;
    info->steps_per_launch = steps_per_launch(b->cfg);
    info->ntiles = b->ntiles;
    info->step = b->step;
    long long nodes = 0;
    size_t bytes = 0, dev = 0;
    for (rlbm_t *h : b->runs) {
        nodes += (long long)h->nx * h->ny;
        bytes += ((size_t)2 * NC * storage_bytes(h->opts.dtype) + (h->forced ? 2 * compute_bytes(h->opts.dtype) : 0)) *
                 (size_t)h->nx * h->ny;
        dev += h->device_bytes;
    }
    info->nodes = nodes;
    info->bytes_per_step = bytes / (size_t)steps_per_launch(b->cfg);
    info->device_bytes = dev;
    return RLBM_OK;
}

rlbm_status rlbm_batch_synchronize(rlbm_batch_t *b) {
    CHECK_BATCH(b);
    BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
    return RLBM_OK;
}

rlbm_status rlbm_batch_last_error(rlbm_batch_t *b, char *buf, size_t len) {
    if (!b || !buf || len == 0) return RLBM_ERR_ARG;
    snprintf(buf, len, "%s", b->msg.c_str());
    return RLBM_OK;
}
}  // extern "C"
