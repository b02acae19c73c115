// xy_ccl.cu -- labelling of frozen domains after a quench (paper: frozen
// domains and their size distribution, abstract and Fig. 6; Sec. IV.C).
//
// A site's Ising projection is spin = (theta >= 0), the sign of
// s = sin(2 theta) on [-pi/2, pi/2) (Sec. IV.A).  Domains are the connected
// components of equal spin under 4-neighbour adjacency with periodic wrap.
// Each site gets the smallest site index of its component, which makes the
// labels unique and comparable bit for bit.
//
// Union-find in three passes (block-local union-find in shared memory, then
// a global merge across tile borders and a flattening pass; unions always
// link the larger root under the smaller, so every root is its component's
// minimum), followed by a per-component size count and an ordered compaction
// of the size histogram into (size, count) pairs.
#include <cstdint>

#include "xy_internal.h"

namespace xy {

namespace {

constexpr int kMaxUnionIters = 1 << 22;

}  // namespace

// Upper bound on the steps of one root search and on the link retries of one
// union in global memory (per device).  xy_debug_set_union_limit() lowers it
// so that tests can run the timeout path: a loop that reaches the bound sets
// XY_ETIMEOUT and returns, and since links only ever point at smaller
// indices the forest stays acyclic and every index stays in range.
__device__ int g_union_limit = kMaxUnionIters;

namespace {

__device__ __forceinline__ bool spin_of(float t) { return t >= 0.0f; }

__device__ __forceinline__ int find_root_global(const int32_t* L, int x, int limit, int* err)
{
    int p = *(volatile const int32_t*)&L[x];
    for (int it = 0; p != x; ++it) {
        if (it >= limit) {
            atomicExch(err, XY_ETIMEOUT);
            return x;
        }
        x = p;
        p = *(volatile const int32_t*)&L[x];
    }
    return x;
}

// Link the components of a and b (global indices inside one lattice's label
// array L): the larger root is pointed at the smaller with atomicMin; a failed
// link (the root changed meanwhile) retries from the value it found.
__device__ void union_global(int32_t* L, int a, int b, int limit, int* err)
{
    for (int it = 0; it < limit; ++it) {
        a = find_root_global(L, a, limit, err);
        b = find_root_global(L, b, limit, err);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&L[a], b);
        if (old == a) return;
        a = old;
    }
    atomicExch(err, XY_ETIMEOUT);
}

__device__ __forceinline__ int find_root_shared(const int* L, int x)
{
    int p = L[x];
    while (p != x) {
        x = p;
        p = L[x];
    }
    return x;
}

__device__ void union_shared(int* L, int a, int b)
{
    for (int it = 0; it < 4096 * 4; ++it) {
        a = find_root_shared(L, a);
        b = find_root_shared(L, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&L[a], b);
        if (old == a) return;
        a = old;
    }
}

}  // namespace

// Pass 1: one block per TW x TH tile, one thread per site; union-find on
// tile-local indices (row-major in the tile, hence ordered like global
// indices), result written as the global index of the local root.
__global__ void ccl_local_kernel(const float* theta, int Lx, int Ly, int TW, int TH, int32_t* labels)
{
    extern __shared__ int s_lab[];
    const int tiles_x = Lx / TW, tiles_y = Ly / TH;
    const int tiles = tiles_x * tiles_y;
    const int lat = blockIdx.x / tiles;
    const int tile = blockIdx.x - lat * tiles;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int lid = threadIdx.x;
    const int ly = lid / TW, lx = lid - ly * TW;
    const int gx = tx * TW + lx, gy = ty * TH + ly;
    const int64_t N = (int64_t)Lx * Ly;
    const float* th = theta + (int64_t)lat * N;
    const bool sp = spin_of(th[(int64_t)gy * Lx + gx]);
    s_lab[lid] = lid;
    __syncthreads();
    if (lx + 1 < TW && spin_of(th[(int64_t)gy * Lx + gx + 1]) == sp) union_shared(s_lab, lid, lid + 1);
    if (ly + 1 < TH && spin_of(th[(int64_t)(gy + 1) * Lx + gx]) == sp) union_shared(s_lab, lid, lid + TW);
    __syncthreads();
    const int root = find_root_shared(s_lab, lid);
    const int rly = root / TW, rlx = root - rly * TW;
    labels[(int64_t)lat * N + (int64_t)gy * Lx + gx] = (int32_t)((ty * TH + rly) * Lx + tx * TW + rlx);
}

// Pass 2: merge across the right and bottom border of every tile (periodic).
__global__ void ccl_border_kernel(const float* theta, int Lx, int Ly, int TW, int TH, int n_lat, int32_t* labels,
                                  int* err)
{
    const int64_t N = (int64_t)Lx * Ly;
    const int64_t per_lat = N;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= per_lat * n_lat) return;
    const int lat = (int)(i / per_lat);
    const int s = (int)(i - (int64_t)lat * per_lat);
    const int y = s / Lx, x = s - y * Lx;
    const bool right_border = (x % TW) == TW - 1;
    const bool bottom_border = (y % TH) == TH - 1;
    if (!right_border && !bottom_border) return;
    const float* th = theta + (int64_t)lat * N;
    int32_t* L = labels + (int64_t)lat * N;
    const bool sp = spin_of(th[s]);
    const int limit = g_union_limit;
    if (right_border) {
        const int n = y * Lx + (x + 1 == Lx ? 0 : x + 1);
        if (spin_of(th[n]) == sp) union_global(L, s, n, limit, err);
    }
    if (bottom_border) {
        const int n = (y + 1 == Ly ? 0 : y + 1) * Lx + x;
        if (spin_of(th[n]) == sp) union_global(L, s, n, limit, err);
    }
}

// Pass 3: every site points straight at its root; count component sizes.
__global__ void ccl_flatten_kernel(int64_t N, int n_lat, int32_t* labels, int32_t* sizes, int* err)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * n_lat) return;
    const int lat = (int)(i / N);
    const int s = (int)(i - (int64_t)lat * N);
    int32_t* L = labels + (int64_t)lat * N;
    const int r = find_root_global(L, s, g_union_limit, err);
    atomicAdd(&sizes[(int64_t)lat * N + r], 1);
    // the final write happens after every find of this pass may have read L[s]
    // as an intermediate node; writing the root keeps the forest valid.
    L[s] = r;
}

// Pass 4: histogram of component sizes: count[size] over roots.
__global__ void ccl_size_hist_kernel(int64_t N, int n_lat, const int32_t* labels, const int32_t* sizes,
                                     int32_t* counts)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N * n_lat) return;
    const int lat = (int)(i / N);
    const int s = (int)(i - (int64_t)lat * N);
    if (labels[(int64_t)lat * N + s] != s) return;
    const int sz = sizes[(int64_t)lat * N + s];
    atomicAdd(&counts[(int64_t)lat * (N + 1) + sz], 1);
}

// Pass 5: ordered compaction of the nonzero counts into (size, count) pairs,
// one block per lattice, ascending size.
__global__ void __launch_bounds__(1024) ccl_compact_kernel(int64_t N, const int32_t* counts, int64_t* hist,
                                                           int64_t hist_cap, int64_t* n_sizes, int* err)
{
    __shared__ int s_warp[32];
    __shared__ int64_t s_base;
    const int lat = blockIdx.x;
    const int32_t* cnt = counts + (int64_t)lat * (N + 1);
    int64_t* out = hist ? hist + (int64_t)lat * hist_cap * 2 : nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int64_t c0 = 1; c0 <= N; c0 += blockDim.x) {
        const int64_t sz = c0 + threadIdx.x;
        const int v = sz <= N ? cnt[sz] : 0;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, v != 0);
        const int before = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        int woff = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) woff += s_warp[w];
            total += s_warp[w];
        }
        const int64_t pos = s_base + woff + before;
        if (v != 0 && out) {
            if (pos < hist_cap) {
                out[2 * pos] = sz;
                out[2 * pos + 1] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (n_sizes) n_sizes[lat] = s_base;
        if (out && s_base > hist_cap) atomicExch(err, XY_EINVAL);
    }
}

static int gcd_int(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

cudaError_t launch_ccl(const float* theta, int Lx, int Ly, int n_lat, int32_t* labels, int32_t* size_scratch,
                       int32_t* count_scratch, int64_t* hist, int64_t hist_cap, int64_t* n_sizes, int* err,
                       cudaStream_t st)
{
    const int64_t N = (int64_t)Lx * Ly;
    int TW = gcd_int(Lx, 32), TH = gcd_int(Ly, 32);
    cudaError_t e;
    if ((e = cudaMemsetAsync(size_scratch, 0, sizeof(int32_t) * N * n_lat, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(count_scratch, 0, sizeof(int32_t) * (N + 1) * n_lat, st)) != cudaSuccess) return e;
    const int tiles = (Lx / TW) * (Ly / TH);
    ccl_local_kernel<<<(unsigned)(tiles * n_lat), TW * TH, TW * TH * sizeof(int), st>>>(theta, Lx, Ly, TW, TH,
                                                                                        labels);
    const int64_t total = N * n_lat;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    ccl_border_kernel<<<blocks, 256, 0, st>>>(theta, Lx, Ly, TW, TH, n_lat, labels, err);
    ccl_flatten_kernel<<<blocks, 256, 0, st>>>(N, n_lat, labels, size_scratch, err);
    ccl_size_hist_kernel<<<blocks, 256, 0, st>>>(N, n_lat, labels, size_scratch, count_scratch);
    ccl_compact_kernel<<<n_lat, 1024, 0, st>>>(N, count_scratch, hist, hist_cap, n_sizes, err);
    return cudaGetLastError();
}

}  // namespace xy

// Diagnostics: bound of the union-find loops on the current device
// (iters <= 0 restores the default 2^22).
extern "C" int xy_debug_set_union_limit(int iters)
{
    const int v = iters > 0 ? iters : xy::kMaxUnionIters;
    const cudaError_t e = cudaMemcpyToSymbol(xy::g_union_limit, &v, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return xy::report_error(XY_ECUDA, cudaGetErrorString(e));
    }
    return XY_OK;
}
