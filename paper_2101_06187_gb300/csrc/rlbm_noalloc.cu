// rlbm_noalloc.cu -- a moments/totals entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need
// the macroscopic fields: code running under a memory budget fixed up front
// (an embedding application that hands the library only pre-sized buffers),
// callers that must not trigger the implicit device synchronisation and
// allocator locks of cudaMalloc in their time-stepping loop, and hosts whose
// device memory is owned by another framework's pool.  rlbm_moments_static
// serves them: it takes the population array and the output buffers from
// the caller and keeps its only scratch -- the per-block FP64 partial sums
// of the conservation totals and the failed-node counter -- in a file-scope
// device array of fixed size, so neither it nor anything it calls allocates.
#include <mutex>

#include "rlbm_internal.h"

namespace {

// Scratch: RLBM_STATIC_MAX_BLOCKS moments blocks (32 x 8 nodes each) of three
// FP64 partial sums, plus one int counter at the end.  1.5 MiB per device,
// held until the process exits by every GPU on which this module is loaded
// (with CUDA's lazy module loading, the default, on the first use of the
// module on that device: the first call of rlbm_moments_static, or any
// earlier kernel launch of the library there).
constexpr int kMaxBlocks = RLBM_STATIC_MAX_BLOCKS;
constexpr size_t kScratchBytes = (size_t)3 * kMaxBlocks * sizeof(double) + 256;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once per device with
// that device current (in host code the name g_scratch is only a host-side
// stand-in; a kernel handed it would read the wrong memory).
constexpr int kMaxDevices = 64;
static void *g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

rlbm_status scratch_for_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RLBM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RLBM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RLBM_OK;
}

}  // namespace

extern "C" RLBM_API rlbm_status rlbm_moments_static(int stencil, int dtype, const void *d_q, int nx, int ny,
                                                    int pitch, double eps0, double scale, double cfl, double *d_eps,
                                                    double *d_vx, double *d_vy, double *d_totals, int *d_bad,
                                                    void *stream) {
    // only the 17-class one-layer state of the paper's node: the ring's 8
    // planes or the 3D lattice's 26 would be read as something they are not
    if (stencil != RLBM_STENCIL_SPH26_SLAB) return RLBM_ERR_ARG;
    if (!d_q || nx < 4 || ny < 4 || pitch < nx || dtype < RLBM_F64 || dtype > RLBM_F16) return RLBM_ERR_ARG;
    if (!(eps0 > 0.0) || !(scale > 0.0) || !(cfl > 0.0 && cfl < 2.0)) return RLBM_ERR_ARG;
    rlbk::StepParams p{};
    p.nx = nx;
    p.ny = ny;
    p.pitch = pitch;
    p.plane = (long long)ny * pitch;
    p.slab = p.plane;
    p.nz = 1;
    p.inv_tau = 1.0;  // unused by the moments kernel
    p.eps0 = eps0;
    p.scale = scale;
    p.eta_k = 0.0;
    p.cfl = cfl;  // the pull of the last stream before the moments: cfl v_i cells
    p.err = nullptr;
    rlbk::finish_params(p);
    const int nblocks = rlbk::moments_blocks(p);
    if (nblocks > kMaxBlocks) return RLBM_ERR_ARG;  // lattice exceeds the static scratch
    void *scratch = nullptr;
    rlbm_status st = scratch_for_current_device(&scratch);
    if (st != RLBM_OK) return st;
    double *partials = static_cast<double *>(scratch);
    int *bad = reinterpret_cast<int *>(static_cast<unsigned char *>(scratch) + (size_t)3 * kMaxBlocks * sizeof(double));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) return RLBM_ERR_CUDA;
    if (rlbk::launch_moments(dtype, RLBM_LANDAU_FP64, d_q, p, d_eps, d_vx, d_vy, partials, bad, s) != cudaSuccess)
        return RLBM_ERR_CUDA;
    if (d_totals &&
        rlbk::launch_reduce_partials(partials, nblocks, eps0 * (double)nx * ny, d_totals, s) != cudaSuccess)
        return RLBM_ERR_CUDA;
    if (d_bad && cudaMemcpyAsync(d_bad, bad, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return RLBM_ERR_CUDA;
    return RLBM_OK;
}
