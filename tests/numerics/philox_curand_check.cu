// Philox4x32-10 on the GPU two ways: cuRAND's block function
// (curand_Philox4x32_10, a library routine) and the library's own device
// generator (rlbk::philox4x32_10, the one the stirring force draws with).
// Reads n counters (n x 4 uint32) and keys (n x 2 uint32) from the binary
// files argv[1], argv[2] and writes both outputs (n x 4 uint32 each) to
// argv[3] and argv[4].  Test infrastructure only.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include <curand_kernel.h>

#include "../../paper_2101_06187_gb300/csrc/forcing.cuh"

__global__ void k_philox_both(int n, const uint4 *ctr, const uint2 *key, uint4 *out_curand, uint4 *out_lib) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    const uint2 k = key[i];
    out_curand[i] = curand_Philox4x32_10(c, k);
    rlbk::U4 u;
    u.w[0] = c.x;
    u.w[1] = c.y;
    u.w[2] = c.z;
    u.w[3] = c.w;
    const rlbk::U4 r = rlbk::philox4x32_10(u, k.x, k.y);
    out_lib[i] = make_uint4(r.w[0], r.w[1], r.w[2], r.w[3]);
}

static std::vector<unsigned char> slurp(const char *path) {
    std::vector<unsigned char> b;
    FILE *f = std::fopen(path, "rb");
    if (!f) return b;
    unsigned char buf[65536];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) b.insert(b.end(), buf, buf + got);
    std::fclose(f);
    return b;
}

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));              \
            return 1;                                                                  \
        }                                                                              \
    } while (0)

int main(int argc, char **argv) {
    if (argc != 5) return 2;
    const std::vector<unsigned char> c = slurp(argv[1]), k = slurp(argv[2]);
    if (c.empty() || c.size() % 16 != 0 || k.size() * 2 != c.size()) return 2;
    const int n = (int)(c.size() / 16);
    uint4 *dc, *d1, *d2;
    uint2 *dk;
    CK(cudaMalloc(&dc, c.size()));
    CK(cudaMalloc(&dk, k.size()));
    CK(cudaMalloc(&d1, c.size()));
    CK(cudaMalloc(&d2, c.size()));
    CK(cudaMemcpy(dc, c.data(), c.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dk, k.data(), k.size(), cudaMemcpyHostToDevice));
    k_philox_both<<<(n + 255) / 256, 256>>>(n, dc, dk, d1, d2);
    CK(cudaGetLastError());
    std::vector<unsigned char> o1(c.size()), o2(c.size());
    CK(cudaMemcpy(o1.data(), d1, c.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(o2.data(), d2, c.size(), cudaMemcpyDeviceToHost));
    for (int j = 0; j < 2; ++j) {
        FILE *f = std::fopen(argv[3 + j], "wb");
        if (!f) return 3;
        const std::vector<unsigned char> &o = j ? o2 : o1;
        if (std::fwrite(o.data(), 1, o.size(), f) != o.size()) return 3;
        std::fclose(f);
    }
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(d1);
    cudaFree(d2);
    return 0;
}
