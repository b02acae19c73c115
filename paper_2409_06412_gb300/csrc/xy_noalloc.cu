// xy_noalloc.cu -- domain labelling for callers that must not allocate.
//
// xy_label_domains() takes its working memory (component sizes, the size
// histogram, the pieces to merge) from cudaMalloc, kept by the lattice
// object between calls.  Some callers
// cannot allow that: services that hand every byte of device memory to their
// own pool and forbid libraries from allocating behind its back, loops where
// an allocation and the device-wide synchronisation of cudaFree are not
// acceptable, and jobs near the memory limit that must not fail half-way on
// an allocation.  xy_label_domains_static() serves them: the caller passes the
// angles and the output buffers, and the working memory is one fixed array
// in this file, part of the library image, that every GPU which loads the
// library holds until the process exits.
#include <cstdint>
#include <mutex>

#include "xy_internal.h"

namespace {

// Working memory of one call (the size histogram and its bitmap, the pieces
// to merge and their list index by site; laid out by ccl_scratch_carve) and
// an error flag.  Bound for at most XY_STATIC_CCL_MAX_SITES sites in at most
// XY_STATIC_CCL_MAX_LATTICES lattices: 4 bytes per site and lattice of
// counts, 4 per 32 sizes and 8 per lattice of bitmap, 256 bytes per copy of
// the small size counts (one copy per 32 tiles of at least 32 sites, at least
// one per lattice), 4 per site of list index, at most 16 per site of list (a
// tile has no more pieces on its edge than sites), 272 per tile of edge data
// (ceil(Lx/32) ceil(Ly/32) <= N/1024 + Lx/32 + Ly/32 + 1 <= N/24 + 1 tiles per
// lattice, as Lx >= 4), and the alignment of each part.  The call checks its
// own layout against this size.
constexpr int64_t kSites = XY_STATIC_CCL_MAX_SITES;
constexpr int64_t kLats = XY_STATIC_CCL_MAX_LATTICES;
constexpr int64_t kScratchBytes = 4 * (kSites + kLats) + 4 * (kSites / 32 + 2 * kLats) +
                                  256 * (kSites / 1024 + kLats) + 4 * kSites + 16 * kSites +
                                  272 * (kSites / 24 + kLats) + 10 * 256;
constexpr int64_t kScratchWords = kScratchBytes / 4 + 64;

static __device__ __align__(256) int32_t g_ccl_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_scratch_addr[kMaxDevices] = {};

int fail_static(int code, const char* msg) { return xy::report_error(code, msg); }

// True for memory the current device's kernels can address (device or
// managed); host and foreign pointers would become illegal accesses on the GPU.
bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device.  In host code
// the array's name is only a stand-in, so the address is looked up once per
// device with that device current.
int scratch_address(int32_t** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail_static(XY_ECUDA, "xy_label_domains_static: no current CUDA device");
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_ccl_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail_static(XY_ECUDA, "xy_label_domains_static: cudaGetSymbolAddress failed");
        }
        g_scratch_addr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return XY_OK;
}

}  // namespace

extern "C" int xy_label_domains_static(const float* theta, int Lx, int Ly, int n_lattices, int32_t* labels,
                                       int64_t* hist, int64_t hist_cap, int64_t* n_sizes, void* cuda_stream)
{
    if (!theta || !labels) return fail_static(XY_EINVAL, "xy_label_domains_static: theta and labels are required");
    if (Lx < 4 || Lx % 4 != 0 || Ly < 1 || n_lattices < 1)
        return fail_static(XY_EINVAL, "xy_label_domains_static: need Lx a positive multiple of 4, Ly >= 1, "
                                      "n_lattices >= 1");
    if (hist && hist_cap <= 0) return fail_static(XY_EINVAL, "xy_label_domains_static: hist_cap must be > 0");
    if (!on_device(theta) || !on_device(labels) || (hist && !on_device(hist)) || (n_sizes && !on_device(n_sizes)))
        return fail_static(XY_EINVAL, "xy_label_domains_static: theta, labels, hist and n_sizes must be device memory");
    const int64_t N = (int64_t)Lx * Ly;
    if (n_lattices > XY_STATIC_CCL_MAX_LATTICES || N * n_lattices > XY_STATIC_CCL_MAX_SITES)
        return fail_static(XY_EINVAL, "xy_label_domains_static: more than XY_STATIC_CCL_MAX_SITES sites or "
                                      "XY_STATIC_CCL_MAX_LATTICES lattices in one call");
    int32_t* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    int64_t zeroed = 0;
    if (xy::ccl_scratch_bytes(Lx, Ly, n_lattices, &zeroed) > kScratchBytes)
        return fail_static(XY_EINVAL, "xy_label_domains_static: working memory exceeds the static array");
    const xy::CclScratch scratch = xy::ccl_scratch_carve(base, Lx, Ly, n_lattices);
    int* err = reinterpret_cast<int*>(base + kScratchBytes / 4);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the call reads its error flag back and synchronises the stream, which a
    // capturing stream does not allow (and the attempt would end the capture)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return fail_static(XY_EINVAL, "xy_label_domains_static: the stream cannot be queried");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return fail_static(XY_EINVAL, "xy_label_domains_static: the stream is capturing; the call synchronises it");
    // the array keeps the previous call's contents: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, zeroed, st);
    if (e == cudaSuccess)
        e = xy::launch_ccl(theta, Lx, Ly, n_lattices, labels, scratch, hist, hist ? hist_cap : 0, n_sizes, err, st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_static(XY_ECUDA, cudaGetErrorString(e));
    }
    if (herr == XY_EINVAL) return fail_static(XY_EINVAL, "xy_label_domains_static: more distinct sizes than hist_cap");
    if (herr == XY_ENOMEM)
        return fail_static(XY_ENOMEM, "xy_label_domains_static: the list of pieces on tile edges overflowed");
    if (herr) return fail_static(herr, "xy_label_domains_static: a bounded union loop ran out of iterations");
    return XY_OK;
}
