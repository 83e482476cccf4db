// Test-only probe: evaluates libsmp's device Philox4x32-10 and cuRAND's curand_Philox4x32_10 on the same
// (counter, key) pairs so a GPU test can pin both the CUDA path's and the oracle's generator to an independent
// implementation. Every thread reads 4 + 2 words and writes 4 + 4 words at its own index (< n).
#include <cstdint>
#include <curand_kernel.h>

#include "../../paper_1610_06656_gb300/csrc/common.cuh"

__global__ void philox_pair_kernel(const uint32_t* ctr, const uint32_t* key, int n, uint32_t* mine, uint32_t* ref) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
    const uint4 r = curand_Philox4x32_10(c, k);
    const smp::U32x4 m = smp::philox4x32_10(c.x, c.y, c.z, c.w, k.x, k.y);
    ref[4 * i] = r.x;
    ref[4 * i + 1] = r.y;
    ref[4 * i + 2] = r.z;
    ref[4 * i + 3] = r.w;
    mine[4 * i] = m.x;
    mine[4 * i + 1] = m.y;
    mine[4 * i + 2] = m.z;
    mine[4 * i + 3] = m.w;
}

extern "C" int philox_pair(const uint32_t* ctr, const uint32_t* key, int n, uint32_t* mine, uint32_t* ref) {
    if (n <= 0) return 0;
    philox_pair_kernel<<<(n + 127) / 128, 128>>>(ctr, key, n, mine, ref);
    return (int)cudaDeviceSynchronize();
}
