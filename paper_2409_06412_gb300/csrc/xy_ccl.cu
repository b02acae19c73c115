// xy_ccl.cu -- labelling of frozen domains after a quench (paper: frozen
// domains and their size distribution, abstract and Fig. 6; Sec. IV.C).
//
// A site's Ising projection is spin = (theta >= 0), the sign of
// s = sin(2 theta) on [-pi/2, pi/2) (Sec. IV.A).  Domains are the connected
// components of equal spin under 4-neighbour adjacency with periodic wrap.
// Each site gets the smallest site index of its component, which makes the
// labels unique and comparable bit for bit.
//
// Passes (unions always link the larger root under the smaller, so every
// root is its component's minimum):
//   tile    one warp per 32 x 32 tile: the rows' spins as 32-bit masks, runs
//           of equal spin, union-find over the runs in shared memory; every
//           site gets its tile root, and each piece its tile-local size.
//           A piece that does not reach the tile's edge is a whole domain and
//           goes into the size histogram at once; one that does goes on a
//           short list (batch index, local size) for the merge.
//   border  one warp per tile, from the spins and tile roots of the edge sites
//           that the tile pass kept: one union in global memory per pair of
//           runs that touch across the tile's right and bottom edges.
//   sizes   the listed pieces add their local sizes at their domain's root's
//           entry of the list (and point their tile roots at the root); the
//           roots' entries then enter the histogram.
//   flatten one warp per tile: every site points straight at its root.
//   compact the histogram's nonzero entries become (size, count) pairs in
//           ascending order: sizes below 64 are summed over the copies their
//           counts are spread over, larger ones are found through a bitmap
//           with one bit per size.
// The histogram counts, their copies and the bitmap are zero between calls:
// the passes clear every entry they set, so no pass reads or clears memory in
// proportion to the lattice beyond the labels themselves.
#include <algorithm>
#include <cstdint>

#include "xy_internal.h"

namespace xy {

namespace {

constexpr int kMaxUnionIters = 1 << 22;
constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr int kTileWarps = 4;      // tiles (warps) per block of the tile pass
constexpr int kSmallSizes = 64;    // sizes counted in shared memory before the global histogram
constexpr int kEdgeFlag = 1 << 16;  // added to a piece's size count for each of its runs on the tile edge

}  // namespace

// Upper bound on the steps of one root search and on the link retries of one
// union in global memory (per device).  xy_debug_set_union_limit() lowers it
// so that tests can run the timeout path: a loop that reaches the bound sets
// XY_ETIMEOUT and returns, and since links only ever point at smaller
// indices the forest stays acyclic and every index stays in range.
__device__ int g_union_limit = kMaxUnionIters;

namespace {

__device__ __forceinline__ bool spin_of(float t) { return t >= 0.0f; }

// Bit x set where a run of equal bits starts in the row mask m (bit 0 always),
// over the tile's columns vm.
__device__ __forceinline__ unsigned run_starts(unsigned m, unsigned vm) { return ((m ^ (m << 1)) | 1u) & vm; }

// Column of the start of the run that holds column x.
__device__ __forceinline__ int run_of(unsigned starts, int x) { return 31 - __clz(starts & ((2u << x) - 1u)); }

// Root of x in the forest L (global memory), halving the path on the way:
// each visited node is pointed at its grandparent, an ancestor, so concurrent
// searches and links stay valid.
__device__ __forceinline__ int find_root_global(int32_t* L, int x, int limit, int* err)
{
    int p = *(volatile const int32_t*)&L[x];
    for (int it = 0; p != x; ++it) {
        if (it >= limit) {
            atomicExch(err, XY_ETIMEOUT);
            return x;
        }
        const int g = *(volatile const int32_t*)&L[p];
        if (g == p) return p;
        L[x] = g;
        x = g;
        p = *(volatile const int32_t*)&L[x];
    }
    return x;
}

// The same search without writes (used while the owners of nodes point them
// at their roots: a halving step could replace such a pointer with an older
// ancestor).
__device__ __forceinline__ int find_root_global_ro(const int32_t* L, int x, int limit, int* err)
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

// Tile-local site i = y * 32 + x lives at shared-memory word i + y (rows
// padded to 33 words): lanes that each own a row and touch the same column
// then hit 32 different banks.  Indices keep the site order; only the
// address is padded.
__device__ __forceinline__ int ph(int i) { return i + (i >> 5); }

// Root of x in a tile's forest (padded layout), halving the path.
__device__ __forceinline__ int find_root_tile(int* L, int x)
{
    int p = L[ph(x)];
    while (p != x) {
        const int g = L[ph(p)];
        if (g == p) return p;
        L[ph(x)] = g;
        x = g;
        p = L[ph(x)];
    }
    return x;
}

// The same search without writes: while lanes point their own run starts at
// their roots, a halving step elsewhere could replace such a pointer with an
// older ancestor.
__device__ __forceinline__ int find_root_tile_ro(const int* L, int x)
{
    int p = L[ph(x)];
    while (p != x) {
        x = p;
        p = L[ph(x)];
    }
    return x;
}

// Link in a tile's forest (padded layout), with a bound on the retries:
// every failed atomicMin means another lane lowered the same entry, so the
// loop ends long before the bound in practice; reaching it sets XY_ETIMEOUT
// like the global loops (the forest stays valid, links only point at
// smaller indices).
__device__ void union_tile(int* L, int a, int b, int* err)
{
    for (int it = 0; it < 4096 * 4; ++it) {
        a = find_root_tile(L, a);
        b = find_root_tile(L, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&L[ph(a)], b);
        if (old == a) return;
        a = old;
    }
    atomicExch(err, XY_ETIMEOUT);
}

// how_many more domains of size sz in lattice lat's histogram.  Small sizes
// are hot (every tile has some): their counts are spread over s.copies
// copies per lattice, picked by tile, and the compaction adds the copies.  A
// larger size is marked in the bitmap by the first add that finds its count
// at zero, so no lane reads a shared word.
__device__ __forceinline__ void count_size(const CclScratch& s, int64_t N, int lat, int sz, int how_many, int tile)
{
    if (sz < kSmallSizes) {
        atomicAdd(s.small + ((int64_t)lat * s.copies + tile % s.copies) * kSmallSizes + sz, how_many);
    } else if (atomicAdd(s.counts + (int64_t)lat * (N + 1) + sz, how_many) == 0) {
        atomicOr(s.bits + (int64_t)lat * s.words + (sz >> 5), 1u << (sz & 31));
    }
}

// Shared memory of one tile: the forest over run starts (tile-local index
// y * 32 + x at word ph(i); other entries unused), and the counts of small
// sizes.  Once the forest is final, a root's own entry holds
// -1 - (size + kEdgeFlag * edge runs) of its piece: every other run start
// then points straight at its root, so the entry is free.
struct TileSmem {
    int P[32 * 33];
    int H[kSmallSizes];
};

}  // namespace

// Pass 1: one warp per tile of up to 32 x 32 sites (the last tile of a row or
// column of tiles may be narrower).  Tile-local indices y * 32 + x order like
// global indices, so a tile root is its piece's smallest site.
__global__ void __launch_bounds__(32 * kTileWarps, 12) ccl_tile_kernel(const float* __restrict__ theta, int Lx, int Ly,
                                                                     int n_lat, int32_t* __restrict__ labels,
                                                                     CclScratch s, int* err)
{
    __shared__ TileSmem sm[kTileWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int tiles_x = (Lx + 31) >> 5, tiles_y = (Ly + 31) >> 5;
    const int tiles = tiles_x * tiles_y;  // the batch has fewer than 2^31 sites
    const int t = blockIdx.x * kTileWarps + wib;
    if (t >= tiles * n_lat) return;  // a whole warp
    const int lat = t / tiles;
    const int tile = t - lat * tiles;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int gx0 = tx * 32, gy0 = ty * 32;
    const int tw = min(32, Lx - gx0), thh = min(32, Ly - gy0);
    const unsigned vm = tw == 32 ? kAll : ((1u << tw) - 1u);
    const int64_t N = (int64_t)Lx * Ly;
    const float* th = theta + (int64_t)lat * N + gy0 * Lx + gx0;
    int32_t* lab = labels + (int64_t)lat * N + gy0 * Lx + gx0;
    int* P = sm[wib].P;
    int* H = sm[wib].H;

    // the rows' spins as masks (lane y keeps row y); 16 loads in flight per lane
    unsigned row = 0;
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
        float v[16];
#pragma unroll
        for (int y = 0; y < 16; ++y) v[y] = (h + y < thh && lane < tw) ? th[(h + y) * Lx + lane] : 0.0f;
#pragma unroll
        for (int y = 0; y < 16; ++y) {
            const unsigned m = __ballot_sync(kAll, spin_of(v[y])) & vm;
            if (lane == h + y) row = m;
        }
    }
    const unsigned st = run_starts(row, vm);  // lane y: the run starts of row y

    // every run start is a root
    for (unsigned b = st; b; b &= b - 1) {
        const int i = lane * 32 + __ffs(b) - 1;
        P[ph(i)] = i;
    }
    H[lane] = 0;
    H[lane + 32] = 0;
    __syncwarp();

    // vertical contacts between rows y and y + 1 (lane y): one union per pair
    // of runs, at the first column where they touch
    {
        const unsigned below = __shfl_down_sync(kAll, row, 1);
        const unsigned sb = __shfl_down_sync(kAll, st, 1);
        if (lane + 1 < thh) {
            const unsigned c = ~(row ^ below) & vm;
            unsigned u = c & ~((c << 1) & c & ~st & ~sb);
            while (u) {
                const int x = __ffs(u) - 1;
                u &= u - 1;
                union_tile(P, lane * 32 + run_of(st, x), (lane + 1) * 32 + run_of(sb, x), err);
            }
        }
    }
    __syncwarp();

    // every run start points straight at its root: each lane writes only its
    // own run starts, and only roots; the searches write nothing
    unsigned roots = 0;  // lane y: the tile roots of row y
    if (lane < thh) {
        for (unsigned b = st; b; b &= b - 1) {
            const int i = lane * 32 + __ffs(b) - 1;
            const int r = find_root_tile_ro(P, i);
            if (r != i)
                P[ph(i)] = r;
            else
                roots |= 1u << (i & 31);
        }
    }
    __syncwarp();
    // a root's entry becomes its piece's count: -1 - (size + kEdgeFlag * edge runs)
    for (unsigned b = roots; b; b &= b - 1) P[ph(lane * 32 + __ffs(b) - 1)] = -1;
    __syncwarp();
    if (lane < thh) {
        for (unsigned b = st; b; b &= b - 1) {
            const int x = __ffs(b) - 1;
            const int i = lane * 32 + x;
            const int q = P[ph(i)];
            const int r = q < 0 ? i : q;
            const unsigned later = b & (b - 1);
            const int end = later ? __ffs(later) - 1 : tw;
            const bool edge = lane == 0 || lane == thh - 1 || x == 0 || end == tw;
            atomicSub(&P[ph(r)], (end - x) + (edge ? kEdgeFlag : 0));
        }
    }
    __syncwarp();

    // labels, a row at a time (coalesced): each site's root through its run
    // start; the tile roots and spins of the edge sites go to the border pass
    uint16_t* er = s.edge_root + (int64_t)t * 128;  // top row, bottom row, left column, right column
#pragma unroll 4
    for (int y = 0; y < thh; ++y) {
        const unsigned sy = __shfl_sync(kAll, st, y);
        if (lane < tw) {
            const int i = y * 32 + run_of(sy, lane);
            const int q = P[y * 33 + (i & 31)];
            const int r = q < 0 ? i : q;
            lab[y * Lx + lane] = (gy0 + (r >> 5)) * Lx + gx0 + (r & 31);
            if (y == 0) er[lane] = (uint16_t)r;
            if (y == thh - 1) er[32 + lane] = (uint16_t)r;
            if (lane == 0) er[64 + y] = (uint16_t)r;
            if (lane == tw - 1) er[96 + y] = (uint16_t)r;
        }
    }
    {
        const unsigned left = __ballot_sync(kAll, lane < thh && (row & 1u));
        const unsigned right = __ballot_sync(kAll, lane < thh && ((row >> (tw - 1)) & 1u));
        const unsigned top = __shfl_sync(kAll, row, 0), bottom = __shfl_sync(kAll, row, thh - 1);
        if (lane == 0) s.edge_spin[t] = make_uint4(top, bottom, left, right);
    }

    // the pieces: whole domains into the histogram, edge pieces onto the list
    int n_edge = 0;
    for (unsigned b = roots; b; b &= b - 1) n_edge += -1 - P[lane * 33 + __ffs(b) - 1] >= kEdgeFlag;
    int before = n_edge;  // inclusive prefix over the lanes
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(kAll, before, d);
        if (lane >= d) before += o;
    }
    const int total = __shfl_sync(kAll, before, 31);
    int base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(s.list_n, total);
    base = __shfl_sync(kAll, base, 31) + before - n_edge;
    for (unsigned b = roots; b; b &= b - 1) {
        const int x = __ffs(b) - 1;
        const int c = -1 - P[lane * 33 + x];
        const int sz = c & (kEdgeFlag - 1);
        if (c >= kEdgeFlag) {
            if (base < s.list_cap) {
                const int g = (gy0 + lane) * Lx + gx0 + x;
                s.list[base] = make_int2((int)((int64_t)lat * N + g), sz);
                s.aux[base] = make_int2(-1, 0);
                s.entry[(int64_t)lat * N + g] = base;
            } else {
                atomicExch(err, XY_ENOMEM);  // not reached: the capacity bounds the pieces on tile edges
            }
            ++base;
        } else if (sz < kSmallSizes) {
            atomicAdd(&H[sz], 1);
        } else {
            count_size(s, N, lat, sz, 1, tile);
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int sz = lane + 32 * k;
        if (H[sz] > 0) count_size(s, N, lat, sz, H[sz], tile);
    }
}

// Pass 2: merge across the right and bottom edge of every tile (periodic).
// One warp per tile; lane k takes the k-th site of the right edge (against
// the first column of the next tile) and of the bottom edge (against the top
// row of the tile below).  The spins and tile roots of edge sites come from
// the tile pass (no angle or label is read along the edges).  Where the
// previous lane also touches and its site continues the run along the edge
// (then so does the neighbour's, which has the same spin), the pair of
// pieces is already linked: one union per pair of touching runs.  The roots'
// entries are read at once for both edges; two roots are then linked
// straight away, anything else goes through the general union.
__global__ void __launch_bounds__(256) ccl_border_kernel(int Lx, int Ly, int n_lat, int32_t* labels, CclScratch s,
                                                         int* err)
{
    const int lane = threadIdx.x & 31;
    const int tiles_x = (Lx + 31) >> 5, tiles_y = (Ly + 31) >> 5;
    const int tiles = tiles_x * tiles_y;
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= tiles * n_lat) return;  // a whole warp
    const int lat = t / tiles;
    const int tile = t - lat * tiles;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int gx0 = tx * 32, gy0 = ty * 32;
    const int tw = min(32, Lx - gx0), thh = min(32, Ly - gy0);
    const int txr = tx + 1 == tiles_x ? 0 : tx + 1, tyb = ty + 1 == tiles_y ? 0 : ty + 1;
    const int t0 = lat * tiles;
    const int tr = t0 + ty * tiles_x + txr, tb = t0 + tyb * tiles_x + tx;  // the tiles to the right and below
    int32_t* L = labels + (int64_t)lat * Lx * Ly;
    const int limit = g_union_limit;
    const uint4 me = s.edge_spin[t];
    const unsigned sp_right = me.w, sp_bottom = me.y;
    const unsigned sp_nleft = s.edge_spin[tr].z, sp_ntop = s.edge_spin[tb].x;
    const uint16_t* er = s.edge_root + (int64_t)t * 128;
    // edge 0: right (rows k < thh); edge 1: bottom (columns k < tw)
    int a[2], b[2];
    bool need[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const bool act = lane < (e == 0 ? thh : tw);
        const unsigned ms = e == 0 ? sp_right : sp_bottom, mn = e == 0 ? sp_nleft : sp_ntop;
        const bool sa = act && ((ms >> lane) & 1u);
        const bool touch = act && sa == (((mn >> lane) & 1u) != 0);
        const unsigned tm = __ballot_sync(kAll, touch);
        const bool prev_sa = __shfl_up_sync(kAll, sa, 1);
        need[e] = touch && !(lane > 0 && ((tm >> (lane - 1)) & 1u) && prev_sa == sa);
        a[e] = b[e] = 0;
        if (need[e]) {
            const int ra = er[(e == 0 ? 96 : 32) + lane];
            const int rb = s.edge_root[(int64_t)(e == 0 ? tr : tb) * 128 + (e == 0 ? 64 : 0) + lane];
            const int gxn = e == 0 ? txr * 32 : gx0, gyn = e == 0 ? gy0 : tyb * 32;
            a[e] = (gy0 + (ra >> 5)) * Lx + gx0 + (ra & 31);
            b[e] = (gyn + (rb >> 5)) * Lx + gxn + (rb & 31);
        }
    }
    int pa[2], pb[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        pa[e] = need[e] ? L[a[e]] : 0;
        pb[e] = need[e] ? L[b[e]] : 0;
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (!need[e]) continue;
        if (pa[e] == a[e] && pb[e] == b[e]) {  // two roots
            if (a[e] == b[e]) continue;
            const int hi = max(a[e], b[e]), lo = min(a[e], b[e]);
            const int old = atomicMin(&L[hi], lo);
            if (old != hi) union_global(L, old, lo, limit, err);  // hi was linked meanwhile
        } else {
            union_global(L, a[e], b[e], limit, err);
        }
    }
}

// Pass 3: each listed piece finds its domain's root, points its tile root
// there, and adds its tile-local size to the root's own entry of the list
// (the root is the tile root of a listed piece: a domain that spans tiles
// reaches the edge of each of its tiles; the tile pass recorded each listed
// tile root's entry).  Searches write nothing here, so afterwards every tile
// root of a merged piece points straight at its domain's root.  A block
// takes 256 consecutive entries from a few tiles; a domain spanning many
// tiles would get an atomic from nearly every entry, all on one address, so
// the pieces of the block's first entry's domain are summed in shared
// memory and added once.
__global__ void __launch_bounds__(256) ccl_list_size_kernel(int64_t N, int32_t* labels, CclScratch s, int* err)
{
    __shared__ int s_key;
    __shared__ int s_sum;
    const int n = min(*s.list_n, (int)s.list_cap);
    const int limit = g_union_limit;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int i = base + threadIdx.x;
        int key = -1, sz = 0;
        if (i < n) {
            const int2 e = s.list[i];
            const int lat = (int)(e.x / N);
            const int g = (int)(e.x - lat * N);
            int32_t* L = labels + (int64_t)lat * N;
            const int r = find_root_global_ro(L, g, limit, err);
            if (r != g) L[g] = r;  // every merged tile root now points at its domain's root
            key = r == g ? i : s.entry[(int64_t)lat * N + r];
            // the root's entry, checked (a search cut short by the bound ends
            // at a node that may not be listed)
            if (key < 0 || key >= n || s.list[key].x != (int)((int64_t)lat * N + r)) {
                atomicExch(err, XY_ETIMEOUT);
                key = -1;
            }
            s.aux[i].x = key;
            sz = e.y;
        }
        if (threadIdx.x == 0) {
            s_key = key;
            s_sum = 0;
        }
        __syncthreads();
        const int k0 = s_key;
        if (key >= 0) {
            if (key == k0)
                atomicAdd(&s_sum, sz);
            else
                atomicAdd(&s.aux[key].y, sz);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_sum > 0) atomicAdd(&s.aux[k0].y, s_sum);
        __syncthreads();
    }
}

// Pass 3b: the listed pieces whose tile root is their domain's root enter the
// histogram with the domain's size.  A block takes 256 consecutive entries,
// from a few tiles of one lattice: small sizes of that lattice are counted
// in shared memory and added with one atomic per size.
__global__ void __launch_bounds__(256) ccl_list_hist_kernel(int64_t N, CclScratch s, int* err)
{
    __shared__ int bins[kSmallSizes];
    __shared__ int blat;
    const int n = min(*s.list_n, (int)s.list_cap);
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        if (threadIdx.x < kSmallSizes) bins[threadIdx.x] = 0;
        if (threadIdx.x == 0) blat = (int)(s.list[base].x / N);
        __syncthreads();
        const int i = base + threadIdx.x;
        if (i < n) {
            const int2 a = s.aux[i];
            if (a.x == i && (a.y < 1 || a.y > N)) {
                atomicExch(err, XY_ETIMEOUT);  // only after a search was cut short
            } else if (a.x == i) {
                const int l = (int)(s.list[i].x / N);
                if (l == blat && a.y < kSmallSizes)
                    atomicAdd(&bins[a.y], 1);
                else
                    count_size(s, N, l, a.y, 1, blockIdx.x);
            }
        }
        __syncthreads();
        if (threadIdx.x < kSmallSizes && bins[threadIdx.x] > 0)
            count_size(s, N, blat, threadIdx.x, bins[threadIdx.x], blockIdx.x);
        __syncthreads();
    }
}

// Pass 4: every site points straight at its root; one warp per tile, lane =
// column.  A site's label is its tile root, a site of the same tile (the
// tile root's own entry is the exception: after a merge it points outside),
// and after pass 3 the tile root's own entry is the domain's root (or
// itself): so the warp reads the tile's labels once (16 rows at a time per
// lane), keeps them in shared memory, and looks every tile root up there.  A
// site whose tile root is still a root is final and is not written.
__global__ void __launch_bounds__(256, 4) ccl_flatten_kernel(int Lx, int Ly, int n_lat, float inv_lx, int32_t* labels)
{
    __shared__ int T[8][32 * 33];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int tiles_x = (Lx + 31) >> 5, tiles_y = (Ly + 31) >> 5;
    const int tiles = tiles_x * tiles_y;
    const int t = blockIdx.x * 8 + wib;
    if (t >= tiles * n_lat) return;  // a whole warp
    const int lat = t / tiles;
    const int tile = t - lat * tiles;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int gx0 = tx * 32, gy0 = ty * 32;
    const int tw = min(32, Lx - gx0), thh = min(32, Ly - gy0);
    const bool in = lane < tw;
    int32_t* L = labels + (int64_t)lat * Lx * Ly;
    const int base = gy0 * Lx + gx0;
    int* Tw = T[wib];
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
        int l[16];
#pragma unroll
        for (int y = 0; y < 16; ++y) l[y] = (in && h + y < thh) ? L[base + (h + y) * Lx + lane] : 0;
#pragma unroll
        for (int y = 0; y < 16; ++y) Tw[(h + y) * 33 + lane] = l[y];
    }
    __syncwarp();
    if (!in) return;
#pragma unroll 4
    for (int y = 0; y < thh; ++y) {
        const int li = Tw[y * 33 + lane];
        const int d = li - base;  // a site of the tile at row ry, column rx: d = ry * Lx + rx
        int ry = (int)((float)d * inv_lx);
        if (ry * Lx > d)
            --ry;
        else if ((ry + 1) * Lx <= d)
            ++ry;
        const int rx = d - ry * Lx;
        // a label outside the tile belongs to a tile root whose entry points
        // at its domain's root already: final
        if (ry >= 0 && ry < thh && rx >= 0 && rx < tw) {
            const int p = Tw[ry * 33 + rx];
            if (p != li) L[base + y * Lx + lane] = p;
        }
    }
}

// Pass 5: ordered compaction of the nonzero counts into (size, count) pairs,
// one block per lattice, ascending size; the rest of the lattice's hist_cap
// pairs is zeroed.  Sizes 1..63 are summed over their copies; larger ones
// are found through the bitmap, one bit per size, a word per thread per
// round in order: each round's set bits are placed by one block-wide prefix,
// and each thread writes its word's pairs and clears what it read.
__global__ void __launch_bounds__(1024) ccl_compact_kernel(int64_t N, CclScratch s, int64_t* hist, int64_t hist_cap,
                                                           int64_t* n_sizes, int* err)
{
    __shared__ int s_warp[32];
    __shared__ int s_small[kSmallSizes];
    __shared__ int64_t s_pos;
    const int lat = blockIdx.x;
    int32_t* cnt = s.counts + (int64_t)lat * (N + 1);
    uint32_t* bw = s.bits + (int64_t)lat * s.words;
    int64_t* out = hist ? hist + (int64_t)lat * hist_cap * 2 : nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_small = (int)(N < kSmallSizes - 1 ? N : kSmallSizes - 1);  // sizes 1..n_small
    if (threadIdx.x < kSmallSizes) s_small[threadIdx.x] = 0;
    __syncthreads();
    {
        // thread j adds copies j / 64, j / 64 + 16, ... of size j % 64: every
        // copy is read by one thread, at most two loads deep
        const int z = threadIdx.x & (kSmallSizes - 1);
        const int nk = (int)blockDim.x / kSmallSizes;
        int v = 0;
        if (z >= 1 && z <= n_small) {
            for (int k = (int)threadIdx.x / kSmallSizes; k < s.copies; k += nk) {
                int32_t* c = s.small + ((int64_t)lat * s.copies + k) * kSmallSizes + z;
                const int a = *c;
                if (a) {
                    v += a;
                    *c = 0;
                }
            }
        }
        if (v) atomicAdd(&s_small[z], v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t at = 0;
        for (int z = 1; z < kSmallSizes; ++z)
            if (s_small[z] != 0) {
                if (out && at < hist_cap) {
                    out[2 * at] = z;
                    out[2 * at + 1] = s_small[z];
                }
                ++at;
            }
        s_pos = at;
    }
    __syncthreads();
    // words holding sizes >= 64: round k of a chunk gives thread j the word
    // k * blockDim + j, so the order within a round is the order of the
    // threads; all 32 rounds' words are read at once
    const int64_t w0 = kSmallSizes / 32;
    const int nt = blockDim.x;
    for (int64_t wc = w0; wc < s.words; wc += 32 * (int64_t)nt) {
        uint32_t wd[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int64_t w = wc + (int64_t)k * nt + threadIdx.x;
            wd[k] = w < s.words ? bw[w] : 0u;
        }
#pragma unroll 1
        for (int k = 0; k < 32; ++k) {
            const uint32_t word = wd[k];
            if (!__syncthreads_or(word != 0u)) continue;  // uniform
            const int c = __popc(word);
            int before = c;  // inclusive prefix over the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(kAll, before, d);
                if (lane >= d) before += o;
            }
            if (lane == 31) s_warp[warp] = before;
            __syncthreads();
            int64_t at = s_pos + before - c;
            int round = 0;
            for (int w = 0; w < (nt >> 5); ++w) {
                if (w < warp) at += s_warp[w];
                round += s_warp[w];
            }
            const int64_t w = wc + (int64_t)k * nt + threadIdx.x;
            for (uint32_t b = word; b; b &= b - 1) {
                const int64_t z = (w << 5) + __ffs(b) - 1;
                if (out && at < hist_cap) {
                    out[2 * at] = z;
                    out[2 * at + 1] = cnt[z];
                }
                cnt[z] = 0;
                ++at;
            }
            if (word) bw[w] = 0;
            __syncthreads();  // every thread has read s_pos and s_warp
            if (threadIdx.x == 0) s_pos += round;
            __syncthreads();
        }
    }
    const int64_t total = s_pos;
    if (out)
        for (int64_t i = total + threadIdx.x; i < hist_cap; i += blockDim.x) {
            out[2 * i] = 0;
            out[2 * i + 1] = 0;
        }
    if (threadIdx.x == 0) {
        if (n_sizes) n_sizes[lat] = total;
        if (out && total > hist_cap) atomicExch(err, XY_EINVAL);
    }
}

namespace {

constexpr int64_t kAlign = 256;

int64_t round_up(int64_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Edge sites of one tile: a bound on the pieces of the tile that reach its edge.
int64_t edge_sites(int tw, int th) { return (tw <= 2 || th <= 2) ? (int64_t)tw * th : 2 * (int64_t)(tw + th) - 4; }

int64_t list_capacity(int Lx, int Ly, int n_lat)
{
    const int fx = Lx / 32, fy = Ly / 32, rx = Lx % 32, ry = Ly % 32;
    int64_t per = (int64_t)fx * fy * edge_sites(32, 32);
    if (rx) per += (int64_t)fy * edge_sites(rx, 32);
    if (ry) per += (int64_t)fx * edge_sites(32, ry);
    if (rx && ry) per += edge_sites(rx, ry);
    return per * n_lat;
}

}  // namespace

// Copies of the small-size counts per lattice: one per 32 tiles, at most 32.
int small_copies(int Lx, int Ly)
{
    const int64_t tiles = (int64_t)((Lx + 31) / 32) * ((Ly + 31) / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(32, tiles / 32));
}

int64_t ccl_scratch_bytes(int Lx, int Ly, int n_lat, int64_t* zeroed_bytes)
{
    const int64_t N = (int64_t)Lx * Ly;
    const int64_t words = (N + 1 + 31) / 32;
    const int64_t z = round_up(4 * (N + 1) * n_lat) + round_up(4 * words * n_lat) +
                      round_up((int64_t)4 * kSmallSizes * small_copies(Lx, Ly) * n_lat);
    if (zeroed_bytes) *zeroed_bytes = z;
    const int64_t cap = list_capacity(Lx, Ly, n_lat);
    const int64_t tiles = (int64_t)((Lx + 31) / 32) * ((Ly + 31) / 32) * n_lat;
    return z + round_up(4 * N * n_lat) + 2 * round_up(8 * cap) + round_up(256 * tiles) + round_up(16 * tiles) + kAlign;
}

CclScratch ccl_scratch_carve(void* base, int Lx, int Ly, int n_lat)
{
    const int64_t N = (int64_t)Lx * Ly;
    CclScratch s{};
    s.words = (N + 1 + 31) / 32;
    s.list_cap = list_capacity(Lx, Ly, n_lat);
    char* p = static_cast<char*>(base);
    s.counts = reinterpret_cast<int32_t*>(p);
    p += round_up(4 * (N + 1) * n_lat);
    s.bits = reinterpret_cast<uint32_t*>(p);
    p += round_up(4 * s.words * n_lat);
    s.copies = small_copies(Lx, Ly);
    s.small = reinterpret_cast<int32_t*>(p);
    p += round_up((int64_t)4 * kSmallSizes * s.copies * n_lat);
    s.entry = reinterpret_cast<int32_t*>(p);
    p += round_up(4 * N * n_lat);
    s.list = reinterpret_cast<int2*>(p);
    p += round_up(8 * s.list_cap);
    s.aux = reinterpret_cast<int2*>(p);
    p += round_up(8 * s.list_cap);
    const int64_t tiles = (int64_t)((Lx + 31) / 32) * ((Ly + 31) / 32) * n_lat;
    s.edge_root = reinterpret_cast<uint16_t*>(p);
    p += round_up(256 * tiles);
    s.edge_spin = reinterpret_cast<uint4*>(p);
    p += round_up(16 * tiles);
    s.list_n = reinterpret_cast<int*>(p);
    return s;
}

cudaError_t launch_ccl(const float* theta, int Lx, int Ly, int n_lat, int32_t* labels, const CclScratch& s,
                       int64_t* hist, int64_t hist_cap, int64_t* n_sizes, int* err, cudaStream_t st)
{
    // every pass runs whether or not sizes are asked for: the size pass also
    // points every merged tile root at its domain's root, which the flattening
    // relies on, and the compaction clears the counts for the next call
    const int64_t N = (int64_t)Lx * Ly;
    const int64_t tiles = (int64_t)((Lx + 31) / 32) * ((Ly + 31) / 32) * n_lat;
    cudaError_t e;
    if ((e = cudaMemsetAsync(s.list_n, 0, sizeof(int), st)) != cudaSuccess) return e;
    ccl_tile_kernel<<<(unsigned)((tiles + kTileWarps - 1) / kTileWarps), 32 * kTileWarps, 0, st>>>(
        theta, Lx, Ly, n_lat, labels, s, err);
    ccl_border_kernel<<<(unsigned)((tiles + 7) / 8), 256, 0, st>>>(Lx, Ly, n_lat, labels, s, err);
    const unsigned g = (unsigned)std::min<int64_t>((s.list_cap + 255) / 256, 152 * 8);
    ccl_list_size_kernel<<<g, 256, 0, st>>>(N, labels, s, err);
    ccl_list_hist_kernel<<<g, 256, 0, st>>>(N, s, err);
    ccl_flatten_kernel<<<(unsigned)((tiles + 7) / 8), 256, 0, st>>>(Lx, Ly, n_lat, 1.0f / (float)Lx, labels);
    ccl_compact_kernel<<<n_lat, 1024, 0, st>>>(N, s, hist, hist_cap, n_sizes, err);
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
