// Test helper: runs cuRAND's device Philox4x32-10 block function on given
// counters, so that the library's and the oracle's Philox bit patterns can be
// checked against an independent implementation.  Built by the GPU tests.
#include <cstdint>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4* ctr, uint32_t k0, uint32_t k1, int64_t n, uint4* out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = curand_Philox4x32_10(ctr[i], make_uint2(k0, k1));
}

extern "C" int curand_philox_ref(const void* ctr, uint32_t k0, uint32_t k1, int64_t n, void* out)
{
    if (n <= 0) return 0;
    curand_philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>((const uint4*)ctr, k0, k1, n, (uint4*)out);
    return (int)cudaDeviceSynchronize();
}
