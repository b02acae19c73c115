// Test-only probe: the largest absolute error of the fast hardware sine and
// cosine at the arguments the steppers form, over every binary32 angle theta
// with |theta| <= pi/2:
//   err[0] = max |__sincosf(2 theta).sin - sin(2 theta)|   (q = 2, exact product)
//   err[1] = max |__sincosf(2 theta).cos - cos(2 theta)|
//   err[2] = max |__sinf(fl(2.5 theta)) - sin(fl(2.5 theta))| (p = 2.5; the
//            rounding of the product is accounted for separately)
//   err[3] = max |__cosf(fl(2.5 theta)) - cos(fl(2.5 theta))|
// against the double-precision sin and cos of the same binary32 argument.
// Errors are non-negative floats, so their bit patterns order like integers.
#include <cstdint>
#include <cuda_runtime.h>

__global__ void sweep(uint32_t n_pos, unsigned* err)
{
    unsigned m[4] = {0u, 0u, 0u, 0u};
    const uint64_t total = 2ull * n_pos;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t bits = (uint32_t)(i >> 1) | ((uint32_t)(i & 1) << 31);  // +-, magnitude order
        const float t = __uint_as_float(bits);
        const float x = __fmul_rn(2.0f, t);
        float s, c;
        __sincosf(x, &s, &c);
        const float y = __fmul_rn(2.5f, t);
        const float sp = __sinf(y), cp = __cosf(y);
        const double e[4] = {fabs((double)s - sin((double)x)), fabs((double)c - cos((double)x)),
                             fabs((double)sp - sin((double)y)), fabs((double)cp - cos((double)y))};
        for (int k = 0; k < 4; ++k) {
            const unsigned u = __float_as_uint(__double2float_ru(e[k]));  // rounded up: still a bound
            m[k] = u > m[k] ? u : m[k];
        }
    }
    for (int k = 0; k < 4; ++k) atomicMax(&err[k], m[k]);
}

// n_pos: number of non-negative binary32 values swept (bit patterns 0 .. n_pos - 1);
// err_out: host float[4].  Returns 0 or the CUDA error code.
extern "C" int intrinsic_error(uint32_t n_pos, float* err_out)
{
    unsigned* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(d, 0, 4 * sizeof(unsigned));
    if (e == cudaSuccess) {
        sweep<<<152 * 8, 256>>>(n_pos, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(err_out, d, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return (int)e;
}
