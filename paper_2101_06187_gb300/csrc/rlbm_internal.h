// rlbm_internal.h -- handle layout and kernel launchers shared by the
// translation units of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>

#include "../../include/rlbm.h"
#include "rlbm_device.cuh"

namespace rlbk {

// One forcing mode: integer wavevector and the four synthesis coefficients
// F_x += ax cos(psi) - bx sin(psi), F_y += ay cos(psi) - by sin(psi),
// psi = 2 pi (kx x/nx + ky y/ny): ax = 2 r amp cos(th) cos(ph),
// bx = 2 r amp cos(th) sin(ph), ay, by likewise with sin(th).
struct Mode {
    int kx, ky;
    double ax, bx, ay, by;
};

// One lattice's stirring force in an ensemble-wide synthesis: what
// launch_draw_modes and launch_synth_force take for that lattice, plus its
// redraw period (a lattice redraws at steps divisible by it, epoch = step /
// period).  Device pointers; p is the lattice's step parameters.
struct ForceJob {
    Mode *modes;
    void *coef;
    const int *run_start;  // first mode of each run of equal ky, then nmodes [nruns + 1]
    void *G;               // per-run row sums [nruns][nx] x 4
    const void *X, *Y;     // per-mode phase tables [nmodes][nx], [nmodes][ny]
    void *F;
    double amp;
    unsigned long long seed;
    long long period;
    int nmodes, nruns;
    StepParams p;
};

// Launch shape of the fused step: kernel variant, thread-block shape and a
// launch budget -- for the packed kernels the minimum resident blocks per SM
// asked of the register allocator (1, 2, 3; 5 = five 128-thread blocks),
// for the two-pass kernel 2..4, for the TMA kernel the CTAs per SM.
struct LaunchCfg {
    int kernel = RLBM_KERNEL_GATHER;
    int bx = 32, by = 8;
    int minb = 1;
};

// Step launchers (defined in the per-form translation units).

cudaError_t launch_step(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                        const void *F, const StepParams &p, cudaStream_t s);
// One launch of the ensemble step over `runs` (a device array of BatchRun
// descriptors, k_step_vec.cuh) with `grid` blocks walking `ntiles` tiles.
cudaError_t launch_batch(int dtype, int landau, const LaunchCfg &cfg, int grid, const void *runs, int nruns,
                         int ntiles, cudaStream_t s);
int run_length(int dtype);

cudaError_t launch_moments(int dtype, int landau, const void *qin, const StepParams &p, double *eps, double *vx,
                           double *vy, double *partials, int *bad, cudaStream_t s);
int moments_blocks(const StepParams &p);

// The TMA-pipelined step (k_step_tma.cu): tensor maps of a state buffer
// and of the force, and the launch (FP32 storage, FP32 Landau, CFL 1).
cudaError_t tma_encode_state(CUtensorMap *map, const void *q, const StepParams &p);
cudaError_t tma_encode_force(CUtensorMap *map, const void *F, const StepParams &p);
cudaError_t launch_step_tma(const LaunchCfg &cfg, bool forced, const CUtensorMap &mq, const CUtensorMap &mf,
                            const void *qin, void *qout, const StepParams &p, cudaStream_t s, int unarmed = 0);

// Two steps per launch (k_step_fused2.cu): cfg.bx x cfg.by is the output
// tile; FP32 / BF16 / FP16 storage with the FP32 Landau solve, CFL 1, nx
// even.  fused2_prepare raises the shared-memory limit of its kernels on the
// current device (once per device, before any launch or stream capture).
cudaError_t fused2_prepare();
cudaError_t launch_step_fused2(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                               const void *F, const StepParams &p, cudaStream_t s);
// The packed single step and the two-step kernel (64 x 8 tiles) with the
// Landau frame refined to FP64 accuracy on the FP32 lanes (k_step_dfl.cu):
// RLBM_LANDAU_FP64 for FP32 / BF16 / FP16 storage on those kernels, CFL 1,
// nx even, launch budgets 1 and 2 for the single step.  fused2_dfl_prepare
// as fused2_prepare.
cudaError_t launch_step_pair_dfl(int dtype, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                                 const void *F, const StepParams &p, cudaStream_t s);
cudaError_t fused2_dfl_prepare();
cudaError_t launch_step_fused2_dfl(int dtype, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                                   const void *F, const StepParams &p, cudaStream_t s);
// Four nodes per thread (k_quad_*.cu, k_quad_dfl_*.cu): the packed body for
// two node pairs per thread, FP32 / BF16 / FP16 storage, the FP32 Landau
// frame or (_dfl_) the frame refined to FP64 accuracy on the FP32 lanes,
// CFL 1, nx divisible by 4; cfg.bx x cfg.by <= 128 threads, cfg.minb 3 or 4.
#define RLBM_QUAD_ENTRY(NAME)                                                                               \
    cudaError_t NAME(const LaunchCfg &cfg, bool forced, const void *qin, void *qout, const void *F,         \
                     const StepParams &p, cudaStream_t s);
RLBM_QUAD_ENTRY(launch_step_quad_f32)
RLBM_QUAD_ENTRY(launch_step_quad_bf16)
RLBM_QUAD_ENTRY(launch_step_quad_f16)
RLBM_QUAD_ENTRY(launch_step_quad_dfl_f32)
RLBM_QUAD_ENTRY(launch_step_quad_dfl_bf16)
RLBM_QUAD_ENTRY(launch_step_quad_dfl_f16)
#undef RLBM_QUAD_ENTRY
// Ensemble form over `runs` (BatchRun descriptors with TW x TH tiles, cfl 1
// members): two steps per launch (two != 0) or one packed step.
cudaError_t launch_batch_fused2(int dtype, int landau, const LaunchCfg &cfg, int grid, const void *runs, int nruns,
                                int ntiles, int two, cudaStream_t s);

// The three-dimensional lattice (k_lattice3d.cu).
cudaError_t launch_step3(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                         const void *F, const StepParams &p, cudaStream_t s);
long long moments3_blocks(const StepParams &p);
cudaError_t launch_moments3(int dtype, const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                            double *vz, double *partials, int *bad, cudaStream_t s);
cudaError_t launch_reduce_partials4(const double *partials, long long nblocks, double base_E, double *totals,
                                    cudaStream_t s);
cudaError_t launch_init3(int dtype, void *q, const StepParams &p, const double *eps, const double *vx,
                         const double *vy, const double *vz, cudaStream_t s);
cudaError_t launch_check_fields3(const double *eps, const double *vx, const double *vy, const double *vz, long long n,
                                 int *bad, cudaStream_t s);
size_t mode3_bytes();
size_t coef3_bytes(int dtype);
void host_mode3(void *dst, int i, int kx, int ky, int kz);
cudaError_t launch_draw_modes3(int dtype, const void *modes, void *coef, int nmodes, double amp,
                               unsigned long long seed, unsigned long long epoch, cudaStream_t s);
cudaError_t launch_mode_tables3(int dtype, void *T, const void *modes, int nmodes, const void *tw, int n, int axis,
                                cudaStream_t s);
cudaError_t launch_synth_force3(int dtype, void *F, const void *coef, int nmodes, const void *X, const void *Y,
                                const void *Z, const StepParams &p, cudaStream_t s);
double class_weight3(int k);
void class_vector3(int k, double *c);

// Spectra of a 3D lattice (k_aux.cu): work area of spectrum_work_doubles3
// doubles; Ek[nshells] and the band power on the device.
size_t spectrum_work_doubles3(int nx, int ny, int nz);
cudaError_t launch_spectrum3(const double *vx, const double *vy, const double *vz, int nx, int ny, int nz, int nshells,
                             double *work, double *Ek, cudaStream_t s);
cudaError_t launch_band_power3(const double *vx, const double *vy, const double *vz, int nx, int ny, int nz, double kf,
                               double *work, double *out, cudaStream_t s);

// The 2D ring variant (k_ring.cu).
cudaError_t launch_ring_step(int dtype, int landau, const LaunchCfg &cfg, bool forced, const void *qin, void *qout,
                             const void *F, const StepParams &p, cudaStream_t s);
cudaError_t launch_ring_moments(int dtype, const void *qin, const StepParams &p, double *eps, double *vx, double *vy,
                                double *partials, int *bad, cudaStream_t s);
cudaError_t launch_ring_init(int dtype, void *q, const StepParams &p, const double *eps, const double *vx,
                             const double *vy, cudaStream_t s);

// Auxiliary kernels (k_aux.cu).
cudaError_t launch_init(int dtype, void *q, const StepParams &p, const double *eps, const double *vx,
                        const double *vy, cudaStream_t s);
cudaError_t launch_check_fields(const double *eps, const double *vx, const double *vy, long long n, int *bad,
                                cudaStream_t s);
cudaError_t launch_reduce_partials(const double *partials, int nblocks, double base_E, double *totals,
                                   cudaStream_t s);
cudaError_t launch_twiddles(int dtype, void *tw, int n, cudaStream_t s);
cudaError_t launch_draw_modes(int dtype, Mode *modes, void *coef, int nmodes, double amp, unsigned long long seed,
                              unsigned long long epoch, cudaStream_t s);
cudaError_t launch_mode_tables(int dtype, void *X, void *Y, const Mode *modes, int nmodes, const void *twx,
                               const void *twy, int nx, int ny, int nxg, int nyg, int x0, int y0, cudaStream_t s);
// F from the mode coefficients, separably: per run of equal ky (ky_start,
// nky runs) the row sums G over the x tables X, then per node the sum over
// runs with the run's y table (Y of its first mode); G is [nky][nx] x 4.
cudaError_t launch_synth_force(int dtype, void *F, const void *coef, int nmodes, const int *ky_start, int nky,
                               void *G, const void *X, const void *Y, const StepParams &p, cudaStream_t s);
// The force of every job in `jobs` (device array of njobs) whose period
// divides `step`, in three launches for all of them; max_*: the largest
// mode count, run count and sides among the jobs (the grid).  Per job the
// arithmetic of launch_draw_modes + launch_synth_force, so the force is the
// same bit for bit.
cudaError_t launch_force_jobs(int dtype, const ForceJob *jobs, int njobs, int max_nmodes, int max_nruns, int max_nx,
                              int max_ny, long long step, cudaStream_t s);
cudaError_t launch_decode_class(int dtype, const void *q, int c, double W, const StepParams &p, double *out,
                                cudaStream_t s);
cudaError_t launch_encode_class(int dtype, void *q, int c, double W, const StepParams &p, const double *in,
                                cudaStream_t s);
cudaError_t launch_force_to_f64(int dtype, const void *F, int comp, const StepParams &p, double *out,
                                cudaStream_t s);
cudaError_t launch_spectrum(const double *vx, const double *vy, int nx, int ny, int nshells, double *work,
                            double *Ek, cudaStream_t s);
size_t spectrum_work_doubles(int nx, int ny);
cudaError_t launch_band_power(const double *vx, const double *vy, int nx, int ny, double kf, double *work,
                              double *out, cudaStream_t s);
cudaError_t launch_accumulate(const double *E, int n, double *sum, double *sq, cudaStream_t s);

size_t storage_bytes(int dtype);
size_t compute_bytes(int dtype);

}  // namespace rlbk

struct rlbm {
    int nx = 0, ny = 0, pitch = 0;
    double tau = 0;
    rlbm_opts opts{};
    rlbm_forcing forcing{};
    bool forced = false;
    int nmodes = 0;
    int ncls = rlbk::NC;  // stored classes: 17 (spherical node) or 8 (2D ring)
    bool ring = false;
    // tensor maps of the two state buffers and of the force (TMA kernel)
    CUtensorMap tm_q[2];
    CUtensorMap tm_F;
    bool tm_ready = false;
    int *errword = nullptr;  // device error word of the bounded waits
    // three-dimensional lattice: nz layers, 26 stored directions, 3 force
    // components, mode table of integer 3-vectors, z phase tables
    bool d3 = false;
    int nz = 1;
    void *modes3 = nullptr;
    void *twz = nullptr, *tabz = nullptr;
    rlbk::LaunchCfg cfg;
    bool tuned = false;
    cudaStream_t stream = nullptr;
    int device = 0;

    void *q[2] = {nullptr, nullptr};  // ping-pong population buffers [17][ny][pitch]
    int cur = 0;                      // index of the current (post-collision) state
    void *F = nullptr;                // force field [2][ny][pitch] (compute type)
    void *twx = nullptr, *twy = nullptr;  // twiddles of the force frame's global sizes [fnx], [fny]
    int fnx = 0, fny = 0, fx0 = 0, fy0 = 0;  // force frame: global sizes and this lattice's offset in it
    void *tabx = nullptr, *taby = nullptr;  // per-mode phase tables [nmodes][nx], [nmodes][ny]
    rlbk::Mode *modes = nullptr;
    void *coef = nullptr;             // per-mode synthesis coefficients (ax, bx, ay, by) in the compute type
    int nky = 0;                      // runs of modes with equal ky (the modes are enumerated ky ascending)
    int *ky_start = nullptr;          // first mode of each run, and nmodes at the end [nky + 1]
    void *gtab = nullptr;             // per-run row sums of the synthesis [nky][nx] (4 values, compute type)
    double *fields = nullptr;         // 3 * nx * ny doubles: staging for init / moments outputs
    double *partials = nullptr;       // per-block partial sums of the moments kernel
    double *totals = nullptr;         // 3 doubles
    int *bad = nullptr;               // device counter of failed nodes
    double *spec_work = nullptr;      // spectrum work area
    size_t spec_work_bytes = 0;
    double *spec_acc = nullptr;       // running sums of E and E^2 per shell (2 x 4096)
    int spec_count = 0, spec_nshells = 0;
    double *host_small = nullptr;     // small pinned buffer for counters and totals
    size_t device_bytes = 0;

    long long step = 0;
    long long force_epoch = -1;  // epoch whose force is in F

    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (steps, parity) -> graph

    rlbm_status status = RLBM_OK;
    std::string msg;
};
