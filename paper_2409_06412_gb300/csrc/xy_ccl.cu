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

// Link in shared memory, with a bound on the retries: every failed atomicMin
// means another thread lowered the same label, so the loop ends long before
// the bound in practice; reaching it sets XY_ETIMEOUT like the global loops
// (the tile's forest stays valid, links only point at smaller indices).
__device__ void union_shared(int* L, int a, int b, int* err)
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
    atomicExch(err, XY_ETIMEOUT);
}

}  // namespace

// Pass 1: one block per TW x TH tile, one thread per site; union-find on
// tile-local indices (row-major in the tile, hence ordered like global
// indices), result written as the global index of the local root.
__global__ void ccl_local_kernel(const float* theta, int Lx, int Ly, int TW, int TH, int32_t* labels,
                                 int* err)
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
    if (TW == 32) {
        // a warp is one tile row: every site points at the first site of its
        // run of equal spins (the run's smallest index), found with one
        // ballot, and only vertical contacts need unions, one per pair of
        // runs touching side by side
        constexpr unsigned kAll = 0xFFFFFFFFu;
        const bool spL = __shfl_up_sync(kAll, sp, 1);
        const bool horiz = lx > 0 && sp == spL;  // same run as the left site
        const unsigned starts = __ballot_sync(kAll, !horiz);
        const unsigned upto = lx == 31 ? starts : (starts & ((2u << lx) - 1u));
        s_lab[lid] = ly * 32 + (31 - __clz(upto));
        __syncthreads();
        if (ly + 1 < TH) {  // uniform in the warp
            const bool vert = spin_of(th[(int64_t)(gy + 1) * Lx + gx]) == sp;
            const bool vertL = __shfl_up_sync(kAll, vert, 1);
            if (vert && !(horiz && vertL)) union_shared(s_lab, lid, lid + 32, err);
        }
    } else {
        s_lab[lid] = lid;
        __syncthreads();
        if (lx + 1 < TW && spin_of(th[(int64_t)gy * Lx + gx + 1]) == sp) union_shared(s_lab, lid, lid + 1, err);
        if (ly + 1 < TH && spin_of(th[(int64_t)(gy + 1) * Lx + gx]) == sp) union_shared(s_lab, lid, lid + TW, err);
    }
    __syncthreads();
    const int root = find_root_shared(s_lab, lid);
    const int rly = root / TW, rlx = root - rly * TW;
    labels[(int64_t)lat * N + (int64_t)gy * Lx + gx] = (int32_t)((ty * TH + rly) * Lx + tx * TW + rlx);
}

// Pass 2: merge across the right and bottom border of every tile (periodic).
// One thread per border site: the TH sites of a tile's right column (each
// linked to its right neighbour) and the TW sites of its bottom row (each
// linked to the site below); the corner does both.
__global__ void ccl_border_kernel(const float* theta, int Lx, int Ly, int TW, int TH, int n_lat, int32_t* labels,
                                  int* err)
{
    const int64_t N = (int64_t)Lx * Ly;
    const int tiles_x = Lx / TW, tiles = tiles_x * (Ly / TH), per_tile = TH + TW;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_lat * tiles * per_tile) return;
    const int lat = (int)(i / ((int64_t)tiles * per_tile));
    const int rem = (int)(i - (int64_t)lat * tiles * per_tile);
    const int tile = rem / per_tile, k = rem - tile * per_tile;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const bool right = k < TH;
    const int y = right ? ty * TH + k : ty * TH + TH - 1;
    const int x = right ? tx * TW + TW - 1 : tx * TW + (k - TH);
    const int s = y * Lx + x;
    const float* th = theta + (int64_t)lat * N;
    int32_t* L = labels + (int64_t)lat * N;
    const bool sp = spin_of(th[s]);
    const int limit = g_union_limit;
    const int n = right ? y * Lx + (x + 1 == Lx ? 0 : x + 1) : (y + 1 == Ly ? 0 : y + 1) * Lx + x;
    if (spin_of(th[n]) == sp) union_global(L, s, n, limit, err);
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
    // lanes that found the same root of the same lattice add their count
    // once (a large domain would otherwise serialise on one address)
    const unsigned long long key = ((unsigned long long)(unsigned)lat << 32) | (unsigned)r;
    const unsigned grp = __match_any_sync(__activemask(), key);
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&sizes[(int64_t)lat * N + r], __popc(grp));
    // the final write happens after every find of this pass may have read L[s]
    // as an intermediate node; writing the root keeps the forest valid.
    L[s] = r;
}

// Pass 4: histogram of component sizes: count[size] over roots.  One thread
// per quad of sites (Lx is a multiple of 4); the label buffer may be the
// caller's and only 4-byte aligned, so the quad is read as four words.
__global__ void ccl_size_hist_kernel(int64_t N, int n_lat, const int32_t* labels, const int32_t* sizes,
                                     int32_t* counts)
{
    const int64_t nq = N / 4;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq * n_lat) return;
    const int lat = (int)(i / nq);
    const int s0 = (int)(4 * (i - (int64_t)lat * nq));
    const int32_t* lp = labels + (int64_t)lat * N + s0;
    const int l4[4] = {lp[0], lp[1], lp[2], lp[3]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (l4[k] != s0 + k) continue;
        const int sz = sizes[(int64_t)lat * N + s0 + k];
        atomicAdd(&counts[(int64_t)lat * (N + 1) + sz], 1);
    }
}

// Pass 5: ordered compaction of the nonzero counts into (size, count) pairs,
// one block per lattice, ascending size.  Warp w owns a contiguous slice of
// the sizes 1..N and reads it 32 consecutive entries at a time, so the order
// of the slices is the order of the sizes: each warp counts its nonzero
// entries, one block-wide prefix over the warps places them, and a second
// pass writes them with ballot ranks.
__global__ void __launch_bounds__(1024) ccl_compact_kernel(int64_t N, const int32_t* __restrict__ counts,
                                                           int64_t* hist, int64_t hist_cap, int64_t* n_sizes, int* err)
{
    __shared__ int64_t s_warp[32];
    const int lat = blockIdx.x;
    const int32_t* cnt = counts + (int64_t)lat * (N + 1);
    int64_t* out = hist ? hist + (int64_t)lat * hist_cap * 2 : nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t per = ((N + nw - 1) / nw + 31) / 32 * 32;  // whole rounds of 32 per warp
    const int64_t lo = 1 + (int64_t)warp * per;
    const int64_t hi = lo + per < N + 1 ? lo + per : N + 1;
    int64_t mine = 0;  // nonzero entries of this warp's slice (same in every lane)
    constexpr int kU = 8;  // rounds of 32 loaded before their ballots: eight loads in flight
    for (int64_t z0 = lo; z0 < hi; z0 += 32 * kU) {
        int v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t z = z0 + 32 * u + lane;
            v[u] = z < hi ? cnt[z] : 0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) mine += __popc(__ballot_sync(0xFFFFFFFFu, v[u] != 0));
    }
    if (lane == 0) s_warp[warp] = mine;
    __syncthreads();
    int64_t pos = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) pos += s_warp[w];
        total += s_warp[w];
    }
    if (out && mine > 0) {
        for (int64_t z0 = lo; z0 < hi; z0 += 32 * kU) {
            int v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t z = z0 + 32 * u + lane;
                v[u] = z < hi ? cnt[z] : 0;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const unsigned m = __ballot_sync(0xFFFFFFFFu, v[u] != 0);
                const int64_t at = pos + __popc(m & ((1u << lane) - 1u));
                if (v[u] != 0 && at < hist_cap) {
                    out[2 * at] = z0 + 32 * u + lane;
                    out[2 * at + 1] = v[u];
                }
                pos += __popc(m);
            }
        }
    }
    if (threadIdx.x == 0) {
        if (n_sizes) n_sizes[lat] = total;
        if (out && total > hist_cap) atomicExch(err, XY_EINVAL);
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
                                                                                        labels, err);
    const int64_t total = N * n_lat;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    const int64_t border = (int64_t)n_lat * tiles * (TW + TH);
    ccl_border_kernel<<<(unsigned)((border + 255) / 256), 256, 0, st>>>(theta, Lx, Ly, TW, TH, n_lat, labels, err);
    ccl_flatten_kernel<<<blocks, 256, 0, st>>>(N, n_lat, labels, size_scratch, err);
    ccl_size_hist_kernel<<<(unsigned)((total / 4 + 255) / 256), 256, 0, st>>>(N, n_lat, labels, size_scratch,
                                                                              count_scratch);
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
