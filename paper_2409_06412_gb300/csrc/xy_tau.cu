// xy_tau.cu -- integrated autocorrelation time and error of the mean of
// recorded observable series (arXiv 2409.06412, App. B: Eq.
// Autocorrelation-Function, Eq. Autocorrelation-Time, Eq. Time-Series-Var).
//
// For one series f_0 .. f_{n-1} (one lattice's records):
//   C(m)   = 1/(n - m) sum_s (f_s - f_bar)(f_{s+m} - f_bar),  C(0) = sigma_f^2
//   tau(M) = 1/2 + sum_{m=1}^{M} C(m) / C(0)                   (record units)
//   tau_C  = tau(M) at the smallest M >= 1 with M >= c tau(M) (the
//            self-consistent window), or at M = floor(n/2) (the paper's
//            tau_s / 2 taken literally) when half_window is set
//   sigma_mean = sqrt(2 tau_C sigma_f^2 / n)
// One block per series.  The mean and C(0) are FP64; the lag sums multiply
// FP32 deviations (relative 1e-7) and add 1024-term FP32 runs into FP64.
// Lags are formed 256 at a time and the window is checked after each batch,
// so a series with a short autocorrelation time costs one batch.
#include "xy_device.cuh"

namespace xy {

namespace {

__device__ __forceinline__ double transform_value(double v, int transform)
{
    switch (transform) {
    case 1: return v * v;
    case 2: return (v * v) * (v * v);
    case 3: return fabs(v);
    default: return v;
    }
}

__device__ double block_sum(double v, double* s_red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    return t;
}

// sum_{s=0}^{n-m-1} d[s] d[s+m]
__device__ double lag_sum(const float* d, int n, int m)
{
    double total = 0.0;
    const int len = n - m;
    for (int s0 = 0; s0 < len; s0 += 1024) {
        const int s1 = min(len, s0 + 1024);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int s = s0;
        for (; s + 3 < s1; s += 4) {
            a0 = fmaf(d[s], d[s + m], a0);
            a1 = fmaf(d[s + 1], d[s + 1 + m], a1);
            a2 = fmaf(d[s + 2], d[s + 2 + m], a2);
            a3 = fmaf(d[s + 3], d[s + 3 + m], a3);
        }
        for (; s < s1; ++s) a0 = fmaf(d[s], d[s + m], a0);
        total += (double)((a0 + a1) + (a2 + a3));
    }
    return total;
}

}  // namespace

__global__ void __launch_bounds__(256) autocorr_kernel(const double2* rec, int64_t R, int component, int transform,
                                                       int64_t skip, int n, float* scratch, double c_win,
                                                       int half_window, double* out)
{
    __shared__ double s_red[8];
    __shared__ double s_C[256];
    __shared__ int s_done;
    const int b = blockIdx.x;
    const double2* series = rec + (int64_t)b * R + skip;
    float* d = scratch + (int64_t)b * n;
    double acc = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const double2 r = series[s];
        acc += transform_value(component ? r.y : r.x, transform);
    }
    const double mean = block_sum(acc, s_red) / n;
    acc = 0.0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const double2 r = series[s];
        const double dv = transform_value(component ? r.y : r.x, transform) - mean;
        d[s] = (float)dv;
        acc += dv * dv;
    }
    const double C0 = block_sum(acc, s_red) / n;  // also orders the writes of d before the lag sums
    const int M_max = n / 2;
    double tau = 0.5;
    if (threadIdx.x == 0) s_done = C0 > 0.0 ? 0 : 1;
    __syncthreads();
    for (int m0 = 1; m0 <= M_max && !s_done; m0 += blockDim.x) {
        const int m = m0 + threadIdx.x;
        s_C[threadIdx.x] = m <= M_max ? lag_sum(d, n, m) / (double)(n - m) : 0.0;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < (int)blockDim.x && m0 + i <= M_max; ++i) {
                tau += s_C[i] / C0;
                if (!half_window && (double)(m0 + i) >= c_win * tau) {
                    s_done = 1;
                    break;
                }
            }
            if (m0 + (int)blockDim.x > M_max) s_done = 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[4 * b + 0] = mean;
        out[4 * b + 1] = C0;
        out[4 * b + 2] = tau;
        out[4 * b + 3] = sqrt(2.0 * tau * C0 / n);
    }
}

cudaError_t launch_autocorr(const double2* rec, int64_t n_series, int64_t R, int component, int transform,
                            int64_t skip, int n, double c_win, int half_window, double* out, cudaStream_t st)
{
    if (n_series == 0) return cudaSuccess;
    float* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, sizeof(float) * (size_t)n_series * n, st);
    if (e != cudaSuccess) return e;
    autocorr_kernel<<<(unsigned)n_series, 256, 0, st>>>(rec, R, component, transform, skip, n, scratch, c_win,
                                                        half_window, out);
    e = cudaGetLastError();
    cudaFreeAsync(scratch, st);
    return e;
}

}  // namespace xy
