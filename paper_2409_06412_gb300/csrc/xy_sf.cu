// xy_sf.cu -- structure factors S_par(k), S_perp(k) of the rotor lattice for
// the correlation-length extraction of arXiv 2409.06412, App. C.
//
// With rotors s = (cos(r theta), sin(r theta)) (the paper's definition is
// r = 1) on an N_par x N_perp lattice (x along the dimer rows, y across),
// Eq. S-as-lattice-FT reads
//   S_perp(k) = 1 / (N_perp N_par^2) sum_l sum_kappa |s~^kappa_{k,l}|^2,
// s~ the 2-D DFT of one rotor component.  Summing |.|^2 over l is, by
// Parseval, N_par times the sum over columns x of the 1-D DFT along y:
//   S_perp(k) = 1 / (N_perp N_par) sum_x sum_kappa |sum_y s^kappa_{x,y} e^{-2 pi i k y / N_perp}|^2,
// and likewise S_par(k) from the 1-D DFTs of the rows along x.  Only the
// wavenumbers k < K near the peak at k = 0 (Eq. Lorentzian-Peak) are formed,
// each as a direct sum with twiddles from a per-block table, in one pass over
// theta per group of 8 wavenumbers: no 2-D transform is needed.
//
// Per-line DFT sums are FP32 (at most 4096 unit-bounded terms); the squared
// moduli are summed in FP64 per block and the blocks of a lattice in a fixed
// order by sf_finish_kernel (deterministic).
#include <vector>

#include "xy_device.cuh"

namespace xy {

namespace {

constexpr int kKC = 8;          // wavenumbers per pass
constexpr int kRowsPerBlock = 64;
constexpr int kColsPerBlock = 256;
constexpr unsigned kFullS = 0xFFFFFFFFu;

struct SfLattice {
    int64_t offset;  // first site of the lattice in the state buffer
    int Lx, Ly;
};

// twiddles W[m] = (cos 2 pi m / N, sin 2 pi m / N), m < N
__device__ void build_twiddles(float2* W, int N)
{
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)m / (float)N, &s, &c);
        W[m] = make_float2(c, s);
    }
    __syncthreads();
}

}  // namespace

// S_par partials: block (b, row chunk, k chunk); warp w takes rows
// y0 + w, y0 + w + 8, ... of the chunk; lane l the sites x = l, l + 32, ...
// part[(b * n_kc + kc) * n_rc + rc][k - k0] = sum over the chunk's rows of sum_kappa |b_k(y)|^2
__global__ void __launch_bounds__(256) sf_rows_kernel(const float* theta, const SfLattice* lats, int K, float r,
                                                      double* part, int n_rc)
{
    extern __shared__ float2 W[];
    const SfLattice lt = lats[blockIdx.x];
    const int rc = blockIdx.y, kc = blockIdx.z;
    const int n_kc = gridDim.z;
    const int Lx = lt.Lx, Ly = lt.Ly;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    build_twiddles(W, Lx);
    const int k0 = kc * kKC;
    const float* th = theta + lt.offset;
    // per wavenumber: twiddle index of this lane's first site and its step per 32 sites
    int idx0[kKC], step[kKC];
#pragma unroll
    for (int q = 0; q < kKC; ++q) {
        const int k = k0 + q < K ? k0 + q : 0;
        idx0[q] = (int)(((int64_t)k * lane) % Lx);
        step[q] = (int)(((int64_t)k * 32) % Lx);
    }
    double acc = 0.0;  // lane q < kKC: wavenumber k0 + q
    const int y_end = min(Ly, (rc + 1) * kRowsPerBlock);
    for (int y = rc * kRowsPerBlock + warp; y < y_end; y += 8) {
        // v[c * kKC + q]: c = 0 re cos, 1 im cos, 2 re sin, 3 im sin
        float v[4 * kKC];
#pragma unroll
        for (int i = 0; i < 4 * kKC; ++i) v[i] = 0.f;
        int idx[kKC];
#pragma unroll
        for (int q = 0; q < kKC; ++q) idx[q] = idx0[q];
        const float* row = th + (int64_t)y * Lx;
        // one site of this lane: its rotor against the kKC twiddles, in x order
        auto site = [&](float t) {
            float sn, cs;
            sincosf(r * t, &sn, &cs);
#pragma unroll
            for (int q = 0; q < kKC; ++q) {
                const float2 w = W[idx[q]];
                v[q] = fmaf(cs, w.x, v[q]);
                v[kKC + q] = fmaf(cs, w.y, v[kKC + q]);
                v[2 * kKC + q] = fmaf(sn, w.x, v[2 * kKC + q]);
                v[3 * kKC + q] = fmaf(sn, w.y, v[3 * kKC + q]);
                idx[q] += step[q];
                if (idx[q] >= Lx) idx[q] -= Lx;
            }
        };
        int x = lane;
        for (; x + 96 < Lx; x += 128) {  // four loads in flight, then the four sites in order
            float t4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) t4[u] = row[x + 32 * u];
#pragma unroll
            for (int u = 0; u < 4; ++u) site(t4[u]);
        }
        for (; x < Lx; x += 32) site(row[x]);
        // reduce-scatter butterfly: afterwards lane i holds the warp total of v[i]
#pragma unroll
        for (int o = 16, n = 32; o >= 1; o >>= 1, n >>= 1) {
            const bool hi = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (i < n / 2) {
                    const float send = hi ? v[i] : v[i + n / 2];
                    const float keep = hi ? v[i + n / 2] : v[i];
                    v[i] = keep + __shfl_xor_sync(kFullS, send, o);
                }
            }
        }
        // lanes q, q + 8, q + 16, q + 24 hold the four parts of wavenumber k0 + q
        float p = v[0] * v[0];
        p += __shfl_xor_sync(kFullS, p, 8);
        p += __shfl_xor_sync(kFullS, p, 16);
        acc += (double)p;
    }
    __shared__ double s_acc[8][kKC];
    if (lane < kKC) s_acc[warp][lane] = acc;
    __syncthreads();
    if (threadIdx.x < kKC) {
        double t = 0.0;
        for (int w2 = 0; w2 < 8; ++w2) t += s_acc[w2][threadIdx.x];
        part[((int64_t)blockIdx.x * n_kc + kc) * n_rc * kKC + (int64_t)rc * kKC + threadIdx.x] = t;
    }
}

// S_perp partials: block (b, column chunk, k chunk); thread t takes column
// x = x0 + t and walks down all rows; the twiddles of a row are the same for
// every thread (shared-memory broadcast).
__global__ void __launch_bounds__(256) sf_cols_kernel(const float* theta, const SfLattice* lats, int K, float r,
                                                      double* part, int n_cc)
{
    extern __shared__ float2 W[];
    const SfLattice lt = lats[blockIdx.x];
    const int cc = blockIdx.y, kc = blockIdx.z;
    const int n_kc = gridDim.z;
    const int Lx = lt.Lx, Ly = lt.Ly;
    build_twiddles(W, Ly);
    const int k0 = kc * kKC;
    const int x = cc * kColsPerBlock + threadIdx.x;
    const bool live = x < Lx;
    int step[kKC], idx[kKC];
#pragma unroll
    for (int q = 0; q < kKC; ++q) {
        step[q] = k0 + q < K ? k0 + q : 0;
        idx[q] = 0;
    }
    float v[4 * kKC];
#pragma unroll
    for (int i = 0; i < 4 * kKC; ++i) v[i] = 0.f;
    const float* col = theta + lt.offset + (live ? x : 0);
    // one site of this column: its rotor against the kKC twiddles, in y order
    auto site = [&](float t) {
        float sn = 0.f, cs = 0.f;
        if (live) sincosf(r * t, &sn, &cs);
#pragma unroll
        for (int q = 0; q < kKC; ++q) {
            const float2 w = W[idx[q]];
            v[q] = fmaf(cs, w.x, v[q]);
            v[kKC + q] = fmaf(cs, w.y, v[kKC + q]);
            v[2 * kKC + q] = fmaf(sn, w.x, v[2 * kKC + q]);
            v[3 * kKC + q] = fmaf(sn, w.y, v[3 * kKC + q]);
            idx[q] += step[q];
            if (idx[q] >= Ly) idx[q] -= Ly;
        }
    };
    int y = 0;
    for (; y + 3 < Ly; y += 4) {  // four loads in flight, then the four sites in order
        float t4[4] = {0.f, 0.f, 0.f, 0.f};
        if (live) {
#pragma unroll
            for (int u = 0; u < 4; ++u) t4[u] = col[(int64_t)(y + u) * Lx];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) site(t4[u]);
    }
    for (; y < Ly; ++y) site(live ? col[(int64_t)y * Lx] : 0.f);
    // |a_k(x)|^2 per thread, summed over the block's columns in a fixed order
    __shared__ double s_acc[kKC][256 / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kKC; ++q) {
        double p = (double)(v[q] * v[q] + v[kKC + q] * v[kKC + q] + v[2 * kKC + q] * v[2 * kKC + q] +
                            v[3 * kKC + q] * v[3 * kKC + q]);
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(kFullS, p, o);
        if (lane == 0) s_acc[q][warp] = p;
    }
    __syncthreads();
    if (threadIdx.x < kKC) {
        double t = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += s_acc[threadIdx.x][w2];
        part[((int64_t)blockIdx.x * n_kc + kc) * n_cc * kKC + (int64_t)cc * kKC + threadIdx.x] = t;
    }
}

// S[b][k] = (sum over chunks of part) / (Lx Ly), k < K
__global__ void sf_finish_kernel(const double* part, const SfLattice* lats, int n_lat, int K, int n_kc, int n_chunks,
                                 double* S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_lat * K) return;
    const int b = i / K, k = i - b * K;
    const int kc = k / kKC, q = k - kc * kKC;
    const double* p = part + ((int64_t)b * n_kc + kc) * n_chunks * kKC + q;
    double t = 0.0;
    for (int c = 0; c < n_chunks; ++c) t += p[(int64_t)c * kKC];
    S[i] = t / ((double)lats[b].Lx * (double)lats[b].Ly);
}

cudaError_t launch_structure_factor(const float* theta, const int64_t* offsets, const int* Lx, const int* Ly,
                                    int n_lat, int K, float r, double* S_par, double* S_perp, int* n_launches,
                                    cudaStream_t st)
{
    if (n_lat == 0) return cudaSuccess;
    int max_x = 0, max_y = 0;
    for (int b = 0; b < n_lat; ++b) {
        max_x = Lx[b] > max_x ? Lx[b] : max_x;
        max_y = Ly[b] > max_y ? Ly[b] : max_y;
    }
    const int n_kc = (K + kKC - 1) / kKC;
    const int n_rc = (max_y + kRowsPerBlock - 1) / kRowsPerBlock;
    const int n_cc = (max_x + kColsPerBlock - 1) / kColsPerBlock;
    std::vector<SfLattice> h((size_t)n_lat);
    for (int b = 0; b < n_lat; ++b) h[(size_t)b] = SfLattice{offsets[b], Lx[b], Ly[b]};
    SfLattice* d_lats = nullptr;
    double *p_rows = nullptr, *p_cols = nullptr;
    const size_t n_rows_part = (size_t)n_lat * n_kc * n_rc * kKC, n_cols_part = (size_t)n_lat * n_kc * n_cc * kKC;
    cudaError_t e = cudaMallocAsync(&d_lats, sizeof(SfLattice) * n_lat, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&p_rows, sizeof(double) * n_rows_part, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&p_cols, sizeof(double) * n_cols_part, st);
    // chunks past a smaller lattice's rows or columns contribute zero
    if (e == cudaSuccess) e = cudaMemsetAsync(p_rows, 0, sizeof(double) * n_rows_part, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p_cols, 0, sizeof(double) * n_cols_part, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_lats, h.data(), sizeof(SfLattice) * n_lat, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && max_x * sizeof(float2) > 48 * 1024)
        e = cudaFuncSetAttribute(sf_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(max_x * sizeof(float2)));
    if (e == cudaSuccess && max_y * sizeof(float2) > 48 * 1024)
        e = cudaFuncSetAttribute(sf_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(max_y * sizeof(float2)));
    if (e == cudaSuccess) {
        sf_rows_kernel<<<dim3((unsigned)n_lat, (unsigned)n_rc, (unsigned)n_kc), 256, max_x * sizeof(float2), st>>>(
            theta, d_lats, K, r, p_rows, n_rc);
        sf_cols_kernel<<<dim3((unsigned)n_lat, (unsigned)n_cc, (unsigned)n_kc), 256, max_y * sizeof(float2), st>>>(
            theta, d_lats, K, r, p_cols, n_cc);
        const int nt = n_lat * K;
        sf_finish_kernel<<<(nt + 255) / 256, 256, 0, st>>>(p_rows, d_lats, n_lat, K, n_kc, n_rc, S_par);
        sf_finish_kernel<<<(nt + 255) / 256, 256, 0, st>>>(p_cols, d_lats, n_lat, K, n_kc, n_cc, S_perp);
        e = cudaGetLastError();
        *n_launches += 4;
    }
    cudaFreeAsync(d_lats, st);
    cudaFreeAsync(p_rows, st);
    cudaFreeAsync(p_cols, st);
    return e;
}

}  // namespace xy
