// xy_step.cu -- stepping kernels of the BBK Langevin integrator on the
// periodic Si(001) dimer-angle lattice (arXiv 2409.06412, Sec. III and App. A.1),
// with the per-step order-parameter and energy reductions (Sec. IV.A,
// Eq. lattice-average; App. B, Eq. ensemble-average-calculation).
//
// Three steppers share the per-site arithmetic of xy_device.cuh and give
// bit-identical states:
//   plain    one thread per quad (4 sites), neighbours from global memory/L2,
//            one launch per step per configuration (the reference path);
//   strip    one warp per 128-site column strip (or per full row when
//            Lx <= 128) sweeping down H rows with a sliding window of
//            (sin q t, cos q t) rows in registers; x neighbours by warp
//            shuffles, one force and one Philox call per quad per step;
//            all lattices of all configurations in one launch;
//   resident one thread block, or a thread-block cluster of up to 16
//            blocks sharing rows through distributed shared memory, per
//            whole lattice held in shared memory, stepping many steps per
//            launch (Lx <= 128).
#include <cstdio>

#include <cooperative_groups.h>

#include <type_traits>

#include "xy_device.cuh"

namespace cg = cooperative_groups;

namespace xy {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ void sc_of(float q, float th, float& s, float& c)
{
    __sincosf(__fmul_rn(q, th), &s, &c);
}

__device__ __forceinline__ float sinp_of(float p, float th) { return __sinf(__fmul_rn(p, th)); }
__device__ __forceinline__ float cosp_of(float p, float th) { return __cosf(__fmul_rn(p, th)); }

// Periodic index for offsets in (-n, 2n): one compare-and-add either way.
__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Neighbourhood of one quad (4 consecutive sites of a row) read from global memory.
struct QuadField {
    float th[4];
    float s[4], c[4];
    float sx[4], cx[4];  // sums over the two x neighbours
    float sy[4], cy[4];  // sums over the two y neighbours
    float sR[4], cR[4];  // forward x neighbour
    float sD[4], cD[4];  // forward y neighbour
};

__device__ __forceinline__ void quad_field(const float* lat, int Lx, int Ly, int x, int y, float q, QuadField& f)
{
    const float4 t = ld4(lat + (int64_t)y * Lx + x);
    const float4 tu = ld4(lat + (int64_t)wrapi(y - 1, Ly) * Lx + x);
    const float4 td = ld4(lat + (int64_t)wrapi(y + 1, Ly) * Lx + x);
    const float tl = lat[(int64_t)y * Lx + wrapi(x - 1, Lx)];
    const float tr = lat[(int64_t)y * Lx + wrapi(x + 4, Lx)];
    float su[4], cu[4], sl, cl, sr, cr;
    f.th[0] = t.x; f.th[1] = t.y; f.th[2] = t.z; f.th[3] = t.w;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        sc_of(q, f.th[i], f.s[i], f.c[i]);
        sc_of(q, f4get(tu, i), su[i], cu[i]);
        sc_of(q, f4get(td, i), f.sD[i], f.cD[i]);
    }
    sc_of(q, tl, sl, cl);
    sc_of(q, tr, sr, cr);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float sLi = i == 0 ? sl : f.s[i - 1];
        const float cLi = i == 0 ? cl : f.c[i - 1];
        f.sR[i] = i == 3 ? sr : f.s[i + 1];
        f.cR[i] = i == 3 ? cr : f.c[i + 1];
        f.sx[i] = __fadd_rn(sLi, f.sR[i]);
        f.cx[i] = __fadd_rn(cLi, f.cR[i]);
        f.sy[i] = __fadd_rn(su[i], f.sD[i]);
        f.cy[i] = __fadd_rn(cu[i], f.cD[i]);
    }
}

// FP64 warp sum in a fixed butterfly order (deterministic).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// FP32 warp sum in the same order.  A warp's partial covers at most a few
// thousand sites, each term of magnitude O(1), so FP32 keeps it to ~1e-6
// relative; the partials of different warps and blocks are combined in FP64.
// (FP64 issues at a small fraction of the FP32 rate on this GPU, so a double
// butterfly per warp and per step is not free.)
__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Commit one unit's (M, E) partial of lattice b; the unit that arrives last
// sums all partials of the lattice in a fixed order and writes the record.
// Must be called by a whole warp (lane 0 holds the partial).
__device__ void commit_partial(Partials pa, int64_t b, int unit, int n_units, double pm, double pe,
                               double2* rec_slot, int64_t N, double e_ref)
{
    const int lane = threadIdx.x & 31;
    int last = 0;
    if (lane == 0) {
        pa.part[b * pa.max_units + unit] = make_double2(pm, pe);
        __threadfence();
        const unsigned old = atomicAdd(&pa.count[b], 1u);
        last = (old == (unsigned)(n_units - 1));
    }
    last = __shfl_sync(kFull, last, 0);
    if (!last) return;
    __threadfence();
    double sm = 0.0, se = 0.0;
    for (int u = lane; u < n_units; u += 32) {
        const double2 p = __ldcg(&pa.part[b * pa.max_units + u]);
        sm += p.x;
        se += p.y;
    }
    sm = warp_sum(sm);
    se = warp_sum(se);
    if (lane == 0) {
        *rec_slot = make_double2(sm / (double)N, se / (double)N + e_ref);
        pa.count[b] = 0u;
    }
}

}  // namespace

// ===========================================================================
// Initial state
// ===========================================================================
__global__ void init_kernel(const DevCfg* cfgs, int c, int mode, float* theta, float* omega)
{
    const DevCfg& cf = cfgs[c];
    const int64_t nq_lat = cf.N / 4;
    const int64_t nq = nq_lat * cf.n_rep;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int rep = (int)(i / nq_lat);
        const int64_t quad = i - (int64_t)rep * nq_lat;
        const int64_t base = cf.offset + (int64_t)rep * cf.N + 4 * quad;
        float4 t;
        if (mode == XY_INIT_UNIFORM) {
            const uint4 w = philox4x32_10(
                noise_counter((uint32_t)quad, ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + rep), 0, 1u), cf.key0,
                cf.key1);
            const float kTwoPi = 6.28318530717958648f;
            t.x = wrap_angle(__fmul_rn(kTwoPi, uniform01(w.x)));
            t.y = wrap_angle(__fmul_rn(kTwoPi, uniform01(w.y)));
            t.z = wrap_angle(__fmul_rn(kTwoPi, uniform01(w.z)));
            t.w = wrap_angle(__fmul_rn(kTwoPi, uniform01(w.w)));
        } else {
            const float o = 1.25663706143591730f;  // 2 pi / 5
            t = make_float4(o, o, o, o);
        }
        st4(theta + base, t);
        st4(omega + base, make_float4(0.f, 0.f, 0.f, 0.f));
    }
}

cudaError_t launch_init(const DevCfg* d_cfg, const DevCfg& h, int init_mode, float* theta, float* omega,
                        cudaStream_t st)
{
    if (init_mode == XY_INIT_USER) return cudaSuccess;
    const int64_t nq = h.N / 4 * h.n_rep;
    const int threads = 256;
    const int blocks = (int)((nq + threads - 1) / threads < 65536 ? (nq + threads - 1) / threads : 65536);
    init_kernel<<<blocks, threads, 0, st>>>(d_cfg, h.slot, init_mode, theta, omega);
    return cudaGetLastError();
}

// ===========================================================================
// Per-quad kernels with global-memory neighbours: prime, full-step omega,
// plain stepper.
// ===========================================================================

// Convert a full-step omega_0 (in omega) into the stored leapfrog velocity
// v_0 = (1 + eta dt / 2) omega_0 - g_0 so that the first step reproduces
// Eq. (BBK-1) exactly: omega_0 = (v_0 + g_0) / (1 + eta dt / 2).
__global__ void prime_kernel(const DevCfg* cfgs, int c, float* theta, float* omega)
{
    const DevCfg& cf = cfgs[c];
    __shared__ float s_c;
    if (threadIdx.x == 0) s_c = noise_amp(cf, cf.k_start);
    __syncthreads();
    const StepConst K = step_const_k(cf, cf.k_start, s_c);
    const int64_t nq_lat = cf.N / 4;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq_lat * cf.n_rep) return;
    const int rep = (int)(i / nq_lat);
    const int64_t quad = i - (int64_t)rep * nq_lat;
    const int y = (int)(4 * quad / cf.Lx), x = (int)(4 * quad - (int64_t)y * cf.Lx);
    const float* lat = theta + cf.offset + (int64_t)rep * cf.N;
    float* om = omega + cf.offset + (int64_t)rep * cf.N + 4 * quad;
    QuadField f;
    quad_field(lat, cf.Lx, cf.Ly, x, y, K.q, f);
    const uint4 w = philox4x32_10(noise_counter((uint32_t)quad, ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + rep),
                                                cf.k_start, 0u), cf.key0, cf.key1);
    const float4 cn = gauss4_scaled(w, K.c);
    const float4 w0 = ld4(om);
    float out[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float F = site_force(K, f.s[s], f.c[s], f.sx[s], f.cx[s], f.sy[s], f.cy[s], sinp_of(K.p, f.th[s]));
        const float g = fmaf(K.hdt, F, f4get(cn, s));
        out[s] = __fadd_rn(__fdiv_rn(f4get(w0, s), K.inv1pa), -g);
    }
    st4(om, make_float4(out[0], out[1], out[2], out[3]));
}

cudaError_t launch_prime(const DevCfg* d_cfg, const DevCfg& h, float* theta, float* omega, cudaStream_t st)
{
    const int64_t nq = h.N / 4 * h.n_rep;
    prime_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(d_cfg, h.slot, theta, omega);
    return cudaGetLastError();
}

// omega_k = (v_k + g_k) / (1 + eta dt / 2) of replicas [rep_first, rep_first + rep_count).
__global__ void omega_full_kernel(const DevCfg* cfgs, int c, int rep_first, int rep_count, const float* theta,
                                  const float* omega, float* out)
{
    const DevCfg& cf = cfgs[c];
    __shared__ float s_c;
    if (threadIdx.x == 0) s_c = noise_amp(cf, cf.k_start);
    __syncthreads();
    const StepConst K = step_const_k(cf, cf.k_start, s_c);
    const int64_t nq_lat = cf.N / 4;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq_lat * rep_count) return;
    const int rr = (int)(i / nq_lat);
    const int rep = rep_first + rr;
    const int64_t quad = i - (int64_t)rr * nq_lat;
    const int y = (int)(4 * quad / cf.Lx), x = (int)(4 * quad - (int64_t)y * cf.Lx);
    const float* lat = theta + cf.offset + (int64_t)rep * cf.N;
    QuadField f;
    quad_field(lat, cf.Lx, cf.Ly, x, y, K.q, f);
    const uint4 w = philox4x32_10(noise_counter((uint32_t)quad, ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + rep),
                                                cf.k_start, 0u), cf.key0, cf.key1);
    const float4 cn = gauss4_scaled(w, K.c);
    const float4 v = ld4(omega + cf.offset + (int64_t)rep * cf.N + 4 * quad);
    float o[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float F = site_force(K, f.s[s], f.c[s], f.sx[s], f.cx[s], f.sy[s], f.cy[s], sinp_of(K.p, f.th[s]));
        const SiteOut so = site_update(K, f.th[s], f4get(v, s), F, f4get(cn, s));
        o[s] = so.omega;
    }
    st4(out + (int64_t)rr * cf.N + 4 * quad, make_float4(o[0], o[1], o[2], o[3]));
}

cudaError_t launch_omega_full(const DevCfg* d_cfg, const DevCfg& h, int rep_first, int rep_count,
                              const float* theta, const float* omega, float* out, cudaStream_t st)
{
    const int64_t nq = h.N / 4 * rep_count;
    omega_full_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(d_cfg, h.slot, rep_first, rep_count,
                                                                     theta, omega, out);
    return cudaGetLastError();
}

// One step of one configuration, one thread per quad.  Blocks never straddle
// two lattices: block index = rep * blocks_per_lattice + unit.
__global__ void __launch_bounds__(256) plain_step_kernel(const DevCfg* cfgs, int c, int64_t j_local, Buffers buf,
                                                         const CallArgs* cap, Partials pa, int write_state)
{
    const DevCfg& cf = cfgs[c];
    const CallArgs ca = *cap;
    const int64_t j = ca.j_base + j_local;
    if (j >= cf.n_call) return;
    __shared__ float s_c;
    __shared__ double s_red[2][8];
    const int64_t k = cf.k_start + j + ca.k_shift;
    if (threadIdx.x == 0) s_c = noise_amp(cf, k);
    __syncthreads();
    const StepConst K = step_const_k(cf, k, s_c);
    const int64_t nq_lat = cf.N / 4;
    const int bpl = (int)((nq_lat + blockDim.x - 1) / blockDim.x);
    const int rep = blockIdx.x / bpl;
    const int unit = blockIdx.x - rep * bpl;
    const int64_t quad = (int64_t)unit * blockDim.x + threadIdx.x;
    const bool odd = !ca.fixed_parity && (j & 1) != 0;
    const int64_t lat_off = cf.offset + (int64_t)rep * cf.N;
    const float* thS = (odd ? buf.thB : buf.thA) + lat_off;
    const float* omS = (odd ? buf.omB : buf.omA) + lat_off;
    float* thD = (odd ? buf.thA : buf.thB) + lat_off;
    float* omD = (odd ? buf.omA : buf.omB) + lat_off;
    const bool rec = ca.record_every > 0 && (k % ca.record_every) == 0;
    float pm = 0.f, pe = 0.f;
    if (quad < nq_lat) {
        const int y = (int)(4 * quad / cf.Lx), x = (int)(4 * quad - (int64_t)y * cf.Lx);
        QuadField f;
        quad_field(thS, cf.Lx, cf.Ly, x, y, K.q, f);
        const uint4 w = philox4x32_10(
            noise_counter((uint32_t)quad, ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + rep), k, 0u), cf.key0, cf.key1);
        const float4 cn = gauss4_scaled(w, K.c);
        const float4 v = ld4(omS + 4 * quad);
        float to[4], vo[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float F =
                site_force(K, f.s[s], f.c[s], f.sx[s], f.cx[s], f.sy[s], f.cy[s], sinp_of(K.p, f.th[s]));
            const SiteOut so = site_update(K, f.th[s], f4get(v, s), F, f4get(cn, s));
            to[s] = so.theta;
            vo[s] = so.v;
            if (rec) {
                const float sigma = (cf.stag && ((x + s + y) & 1)) ? -1.f : 1.f;
                pm = fmaf(sigma, f.s[s], pm);
                if (!ca.m_only)
                    pe = __fadd_rn(pe, site_energy(cf, couplings_at(cf, k), field_h(cf, k), so.omega, f.s[s], f.c[s],
                                                   f.sR[s], f.cR[s],
                                                   f.sD[s], f.cD[s], cosp_of(K.p, f.th[s])));
            }
        }
        if (write_state) {
            st4(thD + 4 * quad, make_float4(to[0], to[1], to[2], to[3]));
            st4(omD + 4 * quad, make_float4(vo[0], vo[1], vo[2], vo[3]));
        }
    }
    if (!rec) return;
    // block partial: per-warp FP32 butterfly, then warp 0 sums the warps in FP64 in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double wm = warp_sumf(pm), we = warp_sumf(pe);
    if (lane == 0) {
        s_red[0][warp] = wm;
        s_red[1][warp] = we;
    }
    __syncthreads();
    if (warp == 0) {
        double bm = 0.0, be = 0.0;
        if (lane == 0)
            for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) {
                bm += s_red[0][w2];
                be += s_red[1][w2];
            }
        const int64_t b = cf.b_first + rep;
        const int64_t r = (k - cf.rec_first) / ca.record_every;
        commit_partial(pa, b, unit, bpl, bm, be, ca.rec_dev + b * ca.rec_stride + r, cf.N,
                       ca.m_only ? 0.0 : (double)cf.e_ref);
    }
}

cudaError_t launch_plain_step(const DevCfg* d_cfg, const DevCfg& h, int64_t j_local, Buffers buf,
                              const CallArgs* ca, Partials pa, int write_state, cudaStream_t st)
{
    const int64_t nq_lat = h.N / 4;
    const int bpl = (int)((nq_lat + 255) / 256);
    plain_step_kernel<<<(unsigned)(bpl * h.n_rep), 256, 0, st>>>(d_cfg, h.slot, j_local, buf, ca, pa,
                                                                  write_state);
    return cudaGetLastError();
}

// ===========================================================================
// Strip stepper: one warp sweeps H rows of a column strip.
// ===========================================================================
namespace {

// One row of a strip as seen by one lane: the raw angles of its quad and of
// its edge column, and their (sin q t, cos q t).
struct RowBuf {
    float4 th;
    float te;
    float s[4], c[4];
};

__device__ __forceinline__ void rowbuf_sc(float q, RowBuf& r)
{
    sc_of(q, r.th.x, r.s[0], r.c[0]);
    sc_of(q, r.th.y, r.s[1], r.c[1]);
    sc_of(q, r.th.z, r.s[2], r.c[2]);
    sc_of(q, r.th.w, r.s[3], r.c[3]);
}

// Everything one lane needs to update its quad in every row of its unit.
struct StripCtx {
    const float* __restrict__ thS;
    const float* __restrict__ omS;
    float* __restrict__ thD;
    float* __restrict__ omD;
    int Lx, Ly, x, xe, srcL, srcR, lg;
    bool multi, rec;
    uint32_t cfgrep;
    int64_t k;
    StepConst K;
    float Jx, Jy, hF, eref;  // energy constants in registers (stores may alias the descriptor)
    bool stag;
    float pm, pe;
};

// All rows of the unit, one row per iteration with a sliding window of three
// rows of (sin q t, cos q t); the raw angles run two rows ahead.  Row
// pointers advance by Lx per row and wrap at the lattice end.
// Rows staged by cp.async: slot i of a lane holds theta of row y_i + 2 (with
// the strip's edge column) and v of row y_i, issued kStages - 1 rows ahead,
// so that three rows of every warp are in flight while one is computed (four
// stages reach the same bandwidth as five; three give 1 % less).
constexpr int kStages = 4;
struct StripStage {
    float4 th[kStages][32];
    float4 v[kStages][32];
    float te[kStages][32];
};

template <int REC>
__device__ __forceinline__ void strip_rows(StripCtx& X, const DevCfg& cf, const PhiloxKeys& keys, int ybeg, int H,
                                           StripStage& stg)
{
    const int64_t Lx = X.Lx;
    const int64_t Nsites = Lx * X.Ly;
    int yp = ybeg - 1;
    if (yp < 0) yp += X.Ly;
    int yn = ybeg + 1;
    if (yn >= X.Ly) yn -= X.Ly;
    int ynn = yn + 1;
    if (ynn >= X.Ly) ynn -= X.Ly;
    RowBuf P, C, N;
    P.th = ld4(X.thS + yp * Lx + X.x);
    C.th = ld4(X.thS + (int64_t)ybeg * Lx + X.x);
    C.te = X.thS[(int64_t)ybeg * Lx + X.xe];
    N.th = ld4(X.thS + yn * Lx + X.x);
    N.te = X.thS[yn * Lx + X.xe];
    rowbuf_sc(X.K.q, P);
    rowbuf_sc(X.K.q, C);
    float* p_to = X.thD + (int64_t)ybeg * Lx;
    float* p_vo = X.omD + (int64_t)ybeg * Lx;
    uint32_t quad = (uint32_t)(((int64_t)ybeg * Lx + X.x) >> 2);
    const uint32_t dquad = (uint32_t)(Lx >> 2);
    const int ln = (int)(threadIdx.x & 31);
    const bool edge = X.multi && (X.lg == 0 || X.lg == 31);
    const float* q_nn = X.thS + ynn * Lx;  // theta row of the next issue (y_i + 2)
    int s_use = 0;                         // slot of row r; row i sits in slot i % kStages
    // issue row i (theta of y_i + 2, v of y_i) into its slot; an empty group
    // past the last row keeps the group count uniform
    auto issue = [&](int i, int slot) {
        if (i < H) {
            cp_async16(&stg.th[slot][ln], q_nn + X.x);
            cp_async16(&stg.v[slot][ln], X.omS + (int64_t)(ybeg + i) * Lx + X.x);
            if (edge) cp_async4(&stg.te[slot][ln], q_nn + X.xe);
            q_nn += Lx;
            if (q_nn >= X.thS + Nsites) q_nn -= Nsites;
        }
        cp_async_commit();
    };
    for (int i = 0; i < kStages - 1; ++i) issue(i, i);
    for (int r = 0; r < H; ++r) {
        const int y = ybeg + r;
        issue(r + kStages - 1, s_use == 0 ? kStages - 1 : s_use - 1);
        cp_async_wait<kStages - 1>();  // this lane's copies of row y have landed
        const float4 th_nn = stg.th[s_use][ln];
        const float te_nn = edge ? stg.te[s_use][ln] : 0.f;
        const float4 v = stg.v[s_use][ln];
        s_use = s_use + 1 == kStages ? 0 : s_use + 1;
        rowbuf_sc(X.K.q, N);
        float sL = __shfl_sync(kFull, C.s[3], X.srcL);
        float cL = __shfl_sync(kFull, C.c[3], X.srcL);
        float sR = __shfl_sync(kFull, C.s[0], X.srcR);
        float cR = __shfl_sync(kFull, C.c[0], X.srcR);
        if (X.multi) {
            // the strip's edge column (lane 0: x0 - 1, lane 31: x0 + 128)
            float se, ce;
            sc_of(X.K.q, C.te, se, ce);
            if (X.lg == 0) { sL = se; cL = ce; }
            if (X.lg == 31) { sR = se; cR = ce; }
        }
        const float4 cn = gauss4_scaled(philox4x32_10_rk(noise_counter(quad, X.cfgrep, X.k, 0u), keys), X.K.c);
        float to[4], vo[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float sl = s == 0 ? sL : C.s[s - 1];
            const float cl = s == 0 ? cL : C.c[s - 1];
            const float sr = s == 3 ? sR : C.s[s + 1];
            const float cr = s == 3 ? cR : C.c[s + 1];
            const float sx = __fadd_rn(sl, sr), cx = __fadd_rn(cl, cr);
            const float sy = __fadd_rn(P.s[s], N.s[s]), cy = __fadd_rn(P.c[s], N.c[s]);
            const float th = f4get(C.th, s);
            const float F = site_force(X.K, C.s[s], C.c[s], sx, cx, sy, cy, sinp_of(X.K.p, th));
            const SiteOut so = site_update(X.K, th, f4get(v, s), F, f4get(cn, s));
            to[s] = so.theta;
            vo[s] = so.v;
            if (REC == 2) {
                const float bx = fmaf(C.c[s], cr, __fmul_rn(C.s[s], sr));
                const float by = fmaf(C.c[s], N.c[s], __fmul_rn(C.s[s], N.s[s]));
                X.pe = __fadd_rn(X.pe, site_energy_rel(so.omega, bx, by, cosp_of(X.K.p, th), X.Jx, X.Jy, X.hF,
                                                       X.eref));
            }
        }
        if (REC) {
            // order parameter of the row: sites x + 0, x + 2 have the parity of
            // y (x is a multiple of 4), sites x + 1, x + 3 the other one
            const float ev = __fadd_rn(C.s[0], C.s[2]), od = __fadd_rn(C.s[1], C.s[3]);
            const float m = !X.stag ? __fadd_rn(ev, od) : ((y & 1) ? __fadd_rn(od, -ev) : __fadd_rn(ev, -od));
            X.pm = __fadd_rn(X.pm, m);
        }
        st4_stream(p_to + X.x, make_float4(to[0], to[1], to[2], to[3]));
        st4_stream(p_vo + X.x, make_float4(vo[0], vo[1], vo[2], vo[3]));
        P = C;
        C = N;
        N.th = th_nn;
        N.te = te_nn;
        p_to += Lx;
        p_vo += Lx;
        quad += dquad;
    }
}

}  // namespace

// REC: 0 = the launch records nothing, 1 = it may record M, 2 = M and E.
// Each kernel carries only the recording code (and registers) it needs.
// SCHED: some configuration of the launch has a field or coupling schedule;
// without one the step's constants are the configuration's own, and the
// kernel carries none of the knot searches (1.7 % of the batch's step time).
template <int MINB, int REC, bool SCHED>
__global__ void __launch_bounds__(256, MINB) strip_step_kernel(const DevCfg* cfgs, const StripTask* tasks, int H,
                                                               int64_t j_local, Buffers buf, const CallArgs* cap,
                                                               Partials pa, PhiloxKeys keys)
{
    const CallArgs ca = *cap;
    const int lane = threadIdx.x & 31, warp = (int)(threadIdx.x >> 5);
    const StripTask task = tasks[blockIdx.x];  // block-uniform
    const int unit = task.unit0 + warp;
    const bool live = unit < task.n_units;     // the lattice's last block may have idle warps
    __shared__ StripStage s_stage[8];          // one per warp of the 256-thread block
    const DevCfg& cf = cfgs[task.cfg];
    const int64_t j = ca.j_base + j_local;
    if (j >= cf.n_call) return;
    StripCtx X;
    X.k = cf.k_start + j + ca.k_shift;
    X.K = SCHED ? step_const_k(cf, X.k, noise_amp(cf, X.k)) : step_const(cf, noise_amp(cf, X.k));
    X.Lx = cf.Lx;
    X.Ly = cf.Ly;
    const bool odd = !ca.fixed_parity && (j & 1) != 0;
    const int64_t lat_off = cf.offset + (int64_t)task.rep * cf.N;
    X.thS = (odd ? buf.thB : buf.thA) + lat_off;
    X.omS = (odd ? buf.omB : buf.omA) + lat_off;
    X.thD = (odd ? buf.thA : buf.thB) + lat_off;
    X.omD = (odd ? buf.omA : buf.omB) + lat_off;

    const int G = X.Lx >= 128 ? 32 : (X.Lx >> 2);  // lanes per row
    const int groups = 32 / G;
    const int strips = X.Lx >= 128 ? (X.Lx >> 7) : 1;
    const int seg = unit / strips;
    const int x0 = (unit - seg * strips) * 128;
    const int grp = lane / G;
    X.lg = lane - grp * G;
    X.multi = X.Lx > 128;
    X.x = x0 + 4 * X.lg;
    const int ybeg = seg * H * groups + grp * H;
    // edge column: lane 0 of a strip needs x0 - 1, lane 31 needs x0 + 128
    X.xe = X.multi ? (X.lg == 0 ? wrapi(x0 - 1, X.Lx) : wrapi(x0 + 128, X.Lx)) : X.x;
    X.srcL = grp * G + (X.lg + G - 1) % G;
    X.srcR = grp * G + (X.lg + 1) % G;
    X.rec = ca.record_every > 0 && (X.k % ca.record_every) == 0;
    X.cfgrep = ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + task.rep);
    X.pm = 0.f;
    X.pe = 0.f;
    if (REC > 0 && X.rec) {  // block-uniform
        const float2 Jk = SCHED ? couplings_at(cf, X.k) : make_float2(cf.Jx, cf.Jy);
        X.Jx = Jk.x;
        X.Jy = Jk.y;
        X.hF = SCHED ? field_h(cf, X.k) : cf.h;
        X.eref = cf.e_ref;
        X.stag = cf.stag != 0;
        if (live) strip_rows<REC>(X, cf, keys, ybeg, H, s_stage[warp]);
        // one partial per block: warp sums, then the block's warps in order
        __shared__ double2 s_part[8];
        const double wm = warp_sumf(X.pm), we = warp_sumf(X.pe);
        if (lane == 0) s_part[warp] = make_double2(wm, we);
        __syncthreads();
        if (warp == 0) {
            const int nw = (int)(blockDim.x >> 5);
            double bm = 0.0, be = 0.0;
            for (int w = 0; w < nw; ++w) {
                bm += s_part[w].x;
                be += s_part[w].y;
            }
            // task, descriptor and call arguments read again here rather than
            // kept in registers across the row loop (which would spill there)
            const StripTask t2 = tasks[blockIdx.x];
            const DevCfg& c2 = cfgs[t2.cfg];
            const CallArgs a2 = *cap;
            const int64_t k2 = c2.k_start + a2.j_base + j_local + a2.k_shift;
            const int64_t b = c2.b_first + t2.rep;
            const int64_t r = (k2 - c2.rec_first) / a2.record_every;
            commit_partial(pa, b, t2.unit0 >> 3, (t2.n_units + 7) >> 3, bm, be, a2.rec_dev + b * a2.rec_stride + r,
                           c2.N,
                           REC == 2 ? (double)c2.e_ref : 0.0);
        }
    } else if (live) {
        strip_rows<0>(X, cf, keys, ybeg, H, s_stage[warp]);
    }
}

// Units (warps) per lattice for the strip stepper with H rows per row group.
int strip_units_per_lattice(int Lx, int Ly, int H)
{
    if (Lx >= 128) return (Lx / 128) * (Ly / H);
    const int groups = 32 / (Lx / 4);
    return Ly / (H * groups);
}

// variant = resident blocks per SM the registers are capped for (2, 3 or 4).
// Every task of one launch uses the noise key `seed`.
cudaError_t launch_strip_step(const DevCfg* d_cfg, const StripTask* tasks, int n_tasks, int H, int variant,
                              int rec, bool sched, uint64_t seed, int64_t j_local, Buffers buf, const CallArgs* ca,
                              Partials pa, cudaStream_t st)
{
    if (n_tasks == 0) return cudaSuccess;
    const PhiloxKeys keys = philox_round_keys(seed);
    using Kern = void (*)(const DevCfg*, const StripTask*, int, int64_t, Buffers, const CallArgs*, Partials,
                          PhiloxKeys);
    // Launches that record run at most 3 blocks per SM: capped at 64
    // registers the recording code spills inside the row loop.
    static const Kern table[2][3][3] = {
        {
            {strip_step_kernel<2, 0, false>, strip_step_kernel<2, 1, false>, strip_step_kernel<2, 2, false>},
            {strip_step_kernel<3, 0, false>, strip_step_kernel<3, 1, false>, strip_step_kernel<3, 2, false>},
            {strip_step_kernel<4, 0, false>, strip_step_kernel<3, 1, false>, strip_step_kernel<3, 2, false>},
        },
        {
            {strip_step_kernel<2, 0, true>, strip_step_kernel<2, 1, true>, strip_step_kernel<2, 2, true>},
            {strip_step_kernel<3, 0, true>, strip_step_kernel<3, 1, true>, strip_step_kernel<3, 2, true>},
            {strip_step_kernel<4, 0, true>, strip_step_kernel<3, 1, true>, strip_step_kernel<3, 2, true>},
        },
    };
    const int vi = variant >= 4 ? 2 : (variant == 3 ? 1 : 0);
    const Kern kern = table[sched ? 1 : 0][vi][rec < 0 ? 0 : (rec > 2 ? 2 : rec)];
    kern<<<(unsigned)n_tasks, 256, 0, st>>>(d_cfg, tasks, H, j_local, buf, ca, pa, keys);
    return cudaGetLastError();
}


// ===========================================================================
// Two steps per pass (temporal blocking over K_t = 2 steps)
// ===========================================================================
// A block owns a band of H rows across the whole lattice width (Lx / 128
// warps side by side, 256 <= Lx <= 1024) and sweeps it once for two steps:
// iteration i loads row y = y0 - 2 + i of theta_k (and v_k of row y - 1),
// advances row a = y - 1 to step k + 1 (level 1, rows y0 - 1 .. y0 + H) and
// row b = y - 2 to step k + 2 (level 2, rows y0 .. y0 + H - 1), which is the
// only row written back: 8 bytes per site-update instead of 16.  The two
// extra level-1 rows are recomputed by the neighbouring bands too (2 / H
// more level-1 work).  Columns next to a warp's strip come from the
// neighbouring warp through shared memory (one barrier per row, the lattice's
// periodic wrap inside the block); the per-site arithmetic is that of every
// other stepper, so states are bit-identical to two single steps.
namespace {

constexpr int kB2Stages = 4;
struct B2Stage {
    float4 th[kB2Stages][32];  // theta_k of the row loaded by an iteration
    float4 v[kB2Stages][32];   // v_k of the row above it
};
struct R0 {  // a level-0 row: theta_k and its (sin q t, cos q t)
    float4 th;
    float s[4], c[4];
};
struct R1 {  // a level-1 row: theta_{k+1}, v_{k+1} and (sin q t, cos q t)
    float4 th, v;
    float s[4], c[4];
};

__device__ __forceinline__ void sc_row(float q, const float4& t, float* s, float* c)
{
    sc_of(q, t.x, s[0], c[0]);
    sc_of(q, t.y, s[1], c[1]);
    sc_of(q, t.z, s[2], c[2]);
    sc_of(q, t.w, s[3], c[3]);
}

// One row of one level: the update of the center row C from its rows above
// (P) and below (N); sL.. are the x neighbours of the row's first and last
// site of this lane (shuffles, or the neighbouring warp's edge for lanes 0, 31).
__device__ __forceinline__ void b2_update(const StepConst& K, const float* Ps, const float* Pc, const float4& th,
                                          const float* Cs, const float* Cc, const float* Ns, const float* Nc,
                                          const float4& v, float sL, float cL, float sR, float cR, const float4& cn,
                                          float4& th_out, float4& v_out)
{
    float to[4], vo[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float sl = s == 0 ? sL : Cs[s - 1];
        const float cl = s == 0 ? cL : Cc[s - 1];
        const float sr = s == 3 ? sR : Cs[s + 1];
        const float cr = s == 3 ? cR : Cc[s + 1];
        const float sx = __fadd_rn(sl, sr), cx = __fadd_rn(cl, cr);
        const float sy = __fadd_rn(Ps[s], Ns[s]), cy = __fadd_rn(Pc[s], Nc[s]);
        const float t = f4get(th, s);
        const float F = site_force(K, Cs[s], Cc[s], sx, cx, sy, cy, sinp_of(K.p, t));
        const SiteOut so = site_update(K, t, f4get(v, s), F, f4get(cn, s));
        to[s] = so.theta;
        vo[s] = so.v;
    }
    th_out = make_float4(to[0], to[1], to[2], to[3]);
    v_out = make_float4(vo[0], vo[1], vo[2], vo[3]);
}

}  // namespace

template <int MINB>
__global__ void __launch_bounds__(256, MINB) band2_step_kernel(const DevCfg* cfgs, const BandTask* tasks, int H,
                                                               int64_t j_local, Buffers buf, const CallArgs* cap,
                                                               PhiloxKeys keys)
{
    extern __shared__ B2Stage s_b2stage[];  // one per warp
    __shared__ float2 s_edge[2][2][8][2];  // [slot][level][warp][first, last site]: (sin q t, cos q t)
    const CallArgs ca = *cap;
    const int lane = threadIdx.x & 31, warp = (int)(threadIdx.x >> 5), nw = (int)(blockDim.x >> 5);
    const BandTask task = tasks[blockIdx.x];
    const DevCfg& cf = cfgs[task.cfg];
    const int64_t j = ca.j_base + j_local;
    if (j >= cf.n_call) return;
    if (j + 1 >= cf.n_call) {  // the host never pairs a last single step; say so if it ever did
        if (threadIdx.x == 0) atomicExch(&((CallArgs*)cap)->err, XY_EINVAL);
        return;
    }
    const int64_t k = cf.k_start + j + ca.k_shift;
    const StepConst K1 = step_const_k(cf, k, noise_amp(cf, k));
    const float c2 = noise_amp(cf, k + 1);
    const StepConst K2c = step_const_k(cf, k + 1, c2);  // the field and couplings of step k + 1
    const int Lx = cf.Lx, Ly = cf.Ly;
    const int64_t lat_off = cf.offset + (int64_t)task.rep * cf.N;
    // a batch of steps holds an even number of pairs: pair p = j_local / 2 of it
    // reads the buffer the single-step convention gives for step j, flipped when
    // p is odd, and writes the other
    const bool rd_b = ca.fixed_parity ? false : (((j & 1) != 0) != (((j_local >> 1) & 1) != 0));
    const float* thS = (rd_b ? buf.thB : buf.thA) + lat_off;
    const float* omS = (rd_b ? buf.omB : buf.omA) + lat_off;
    float* thD = (rd_b ? buf.thA : buf.thB) + lat_off;
    float* omD = (rd_b ? buf.omA : buf.omB) + lat_off;
    const int x = warp * 128 + 4 * lane;
    const int y0 = task.band0 * H;
    const int wl = warp == 0 ? nw - 1 : warp - 1, wr = warp + 1 == nw ? 0 : warp + 1;
    const int srcL = (lane + 31) & 31, srcR = (lane + 1) & 31;
    const uint32_t cfgrep = ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + task.rep);
    B2Stage& stg = s_b2stage[warp];
    const int n_it = H + 4;
    // prefetch: iteration ii loads theta_k of row y0 - 2 + ii and (ii >= 2) v_k of row y0 - 3 + ii
    auto issue = [&](int ii) {
        if (ii < n_it) {
            const int sl = ii % kB2Stages;
            cp_async16(&stg.th[sl][lane], thS + (int64_t)wrapi(y0 - 2 + ii, Ly) * Lx + x);
            if (ii >= 2) cp_async16(&stg.v[sl][lane], omS + (int64_t)wrapi(y0 - 3 + ii, Ly) * Lx + x);
        }
        cp_async_commit();
    };
    for (int ii = 0; ii < kB2Stages - 1; ++ii) issue(ii);
    // neighbours in x of a row of this lane: shuffles inside the warp, the
    // neighbouring warps' edge sites (published the iteration before) for lanes 0 and 31
    auto x_nbrs = [&](const float* Cs, const float* Cc, int slot, int lev, float& sL, float& cL, float& sR, float& cR) {
        sL = __shfl_sync(kFull, Cs[3], srcL);
        cL = __shfl_sync(kFull, Cc[3], srcL);
        sR = __shfl_sync(kFull, Cs[0], srcR);
        cR = __shfl_sync(kFull, Cc[0], srcR);
        // every lane reads the two edge words (a broadcast) and lanes 0 and 31
        // select them: no divergent branch in the row loop
        const float2 el = s_edge[slot][lev][wl][1], er = s_edge[slot][lev][wr][0];
        sL = lane == 0 ? el.x : sL;
        cL = lane == 0 ? el.y : cL;
        sR = lane == 31 ? er.x : sR;
        cR = lane == 31 ? er.y : cR;
    };
    auto publish = [&](const float* Cs, const float* Cc, int slot, int lev) {
        if (lane == 0) s_edge[slot][lev][warp][0] = make_float2(Cs[0], Cc[0]);
        if (lane == 31) s_edge[slot][lev][warp][1] = make_float2(Cs[3], Cc[3]);
    };
    R0 a0, b0, c0;
    R1 a1, b1, c1;
    // iteration i: P0, C0, N0 = level-0 rows y - 2, y - 1, y; P1, C1, N1 =
    // level-1 rows b - 1, b, a (N1 computed here)
    auto body = [&](int i, R0& P0, R0& C0, R0& N0, R1& P1, R1& C1, R1& N1) {
        issue(i + kB2Stages - 1);
        cp_async_wait<kB2Stages - 1>();  // this lane's copies of iteration i have landed
        const int sl = i % kB2Stages;
        const int slot = i & 1, prev = slot ^ 1;
        N0.th = stg.th[sl][lane];
        sc_row(K1.q, N0.th, N0.s, N0.c);
        publish(N0.s, N0.c, slot, 0);
        if (i >= 2) {  // level 1 on row a = y - 1
            const int a = wrapi(y0 - 3 + i, Ly);
            const float4 va = stg.v[sl][lane];
            float sL, cL, sR, cR;
            x_nbrs(C0.s, C0.c, prev, 0, sL, cL, sR, cR);
            const uint32_t quad = (uint32_t)(((int64_t)a * Lx + x) >> 2);
            const float4 cn = gauss4_scaled(philox4x32_10_rk(noise_counter(quad, cfgrep, k, 0u), keys), K1.c);
            b2_update(K1, P0.s, P0.c, C0.th, C0.s, C0.c, N0.s, N0.c, va, sL, cL, sR, cR, cn, N1.th, N1.v);
            sc_row(K1.q, N1.th, N1.s, N1.c);
            publish(N1.s, N1.c, slot, 1);
        }
        if (i >= 4) {  // level 2 on row b = y - 2
            const int b = wrapi(y0 - 4 + i, Ly);
            float sL, cL, sR, cR;
            x_nbrs(C1.s, C1.c, prev, 1, sL, cL, sR, cR);
            const uint32_t quad = (uint32_t)(((int64_t)b * Lx + x) >> 2);
            const StepConst K2 = K2c;
            const float4 cn = gauss4_scaled(philox4x32_10_rk(noise_counter(quad, cfgrep, k + 1, 0u), keys), c2);
            float4 to, vo;
            b2_update(K2, P1.s, P1.c, C1.th, C1.s, C1.c, N1.s, N1.c, C1.v, sL, cL, sR, cR, cn, to, vo);
            st4_stream(thD + (int64_t)b * Lx + x, to);
            st4_stream(omD + (int64_t)b * Lx + x, vo);
        }
        __syncthreads();  // edges of this iteration visible; the slot read here free for the next
    };
    for (int i = 0; i < n_it; i += 3) {
        body(i, a0, b0, c0, a1, b1, c1);
        if (i + 1 < n_it) body(i + 1, b0, c0, a0, b1, c1, a1);
        if (i + 2 < n_it) body(i + 2, c0, a0, b0, c1, a1, b1);
    }
    cp_async_wait<0>();
}

// Bands of the two-step kernel: H (dividing Ly) is the tuner's to choose;
// threads = Lx / 4, one warp per 128 columns.
cudaError_t launch_band2_step(const DevCfg* d_cfg, const BandTask* tasks, int n_tasks, int Lx, int H, int variant,
                              uint64_t seed, int64_t j_local, Buffers buf, const CallArgs* ca, cudaStream_t st)
{
    if (n_tasks == 0) return cudaSuccess;
    if (Lx < 256 || Lx > 1024 || Lx % 128 != 0) return cudaErrorInvalidValue;
    // variant = resident 256-thread blocks per SM the registers are capped for:
    // 2 (no spills) or 3 (a few spilled words, more warps to hide latency)
    using Kern = void (*)(const DevCfg*, const BandTask*, int, int64_t, Buffers, const CallArgs*, PhiloxKeys);
    const Kern kern = variant >= 3 ? band2_step_kernel<3> : band2_step_kernel<2>;
    const size_t smem = sizeof(B2Stage) * (size_t)(Lx / 128);
    kern<<<(unsigned)n_tasks, Lx / 4, smem, st>>>(d_cfg, tasks, H, j_local, buf, ca, philox_round_keys(seed));
    return cudaGetLastError();
}

namespace {
struct SC4 {
    float s[4], c[4];
};

__device__ __forceinline__ void sc4_from_theta(const float4& t, float q, SC4& r)
{
    sc_of(q, t.x, r.s[0], r.c[0]);
    sc_of(q, t.y, r.s[1], r.c[1]);
    sc_of(q, t.z, r.s[2], r.c[2]);
    sc_of(q, t.w, r.s[3], r.c[3]);
}

__device__ __forceinline__ void sc4_load(const float2* p, SC4& r)
{
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 2);
    r.s[0] = a.x; r.c[0] = a.y; r.s[1] = a.z; r.c[1] = a.w;
    r.s[2] = b.x; r.c[2] = b.y; r.s[3] = b.z; r.c[3] = b.w;
}

__device__ __forceinline__ void sc4_store(float2* p, const SC4& r)
{
    *reinterpret_cast<float4*>(p) = make_float4(r.s[0], r.c[0], r.s[1], r.c[1]);
    *reinterpret_cast<float4*>(p + 2) = make_float4(r.s[2], r.c[2], r.s[3], r.c[3]);
}
}  // namespace

size_t resident_smem_bytes(int Lx, int Ly, int threads, int csize);

// Threads of a resident block when a cluster of `csize` blocks holds the
// lattice (csize = 1: one block): the largest power of two <= 1024 that is a
// multiple of G = Lx / 4, gives whole bands of the block's Ly / csize rows
// and keeps the block's shared memory within max_smem bytes.
int resident_threads(int Lx, int Ly, int csize, size_t max_smem)
{
    if (Lx % 4 != 0 || Lx > 128 || csize < 1 || Ly % csize != 0) return 0;
    const int G = Lx / 4;
    if (32 % G != 0) return 0;
    const int Lr = Ly / csize;
    for (int nt = 1024; nt >= 32; nt >>= 1) {
        if (nt % G != 0) continue;
        const int NB = nt / G;
        if (NB <= Lr && Lr % NB == 0 && resident_smem_bytes(Lx, Ly, nt, csize) <= max_smem) return nt;
    }
    return 0;
}

// Dynamic shared memory of one resident block: theta and v of its rows, the
// (sin q t, cos q t) exports of its bands' first and last rows for two step
// parities, and the record partials for two step parities.
size_t resident_smem_bytes(int Lx, int Ly, int threads, int csize)
{
    const int G = Lx / 4;
    const int NB = threads / G;
    const int Lr = Ly / csize;
    return (size_t)Lx * Lr * 8 + (size_t)4 * NB * Lx * 8 + 2 * 64 * sizeof(double) + 16;
}

// ===========================================================================
// Resident stepper: a thread-block cluster of C blocks (C = 1: one block)
// holds one whole lattice in shared memory, block r owning rows
// [r Ly / C, (r + 1) Ly / C), and runs many steps per launch.  Thread t owns
// the quad column x = 4 (t % G) of band t / G, a band being R consecutive
// rows; G = Lx / 4 <= 32 lanes span a row, so x neighbours come from warp
// shuffles of width G.  Each step:
//   phase 1: every band exports (sin q t, cos q t) of its first and last row
//            to its block's shared memory (buffers alternate with the step
//            parity), then the cluster synchronises once;
//   phase 2: every band sweeps its rows with a sliding window, taking the
//            rows above / below the band from the neighbouring bands'
//            exports -- in the block's own shared memory, or in a
//            neighbouring block's through distributed shared memory -- and
//            updates theta and v in place (no thread reads another thread's
//            theta).
// The parity-alternating exports make one cluster barrier per step enough:
// an export buffer is rewritten two steps after it was read, and every
// reader has passed the barrier in between.
// ===========================================================================
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// Every lattice of one launch uses the noise key whose round keys are `keys`.
// ONE_ROW: the launch's bands are one row high (R = 1), the specialisation
// whose quads stay in registers; the other instantiation serves R > 1.
template <int MAXT, bool ONE_ROW>
__global__ void __launch_bounds__(MAXT, 1) resident_step_kernel(const DevCfg* cfgs, const ResidentTask* tasks,
                                                                int64_t j_local, int n_steps, Buffers buf,
                                                                const CallArgs* cap, PhiloxKeys keys)
{
    extern __shared__ float4 smem4[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const CallArgs ca = *cap;
    const ResidentTask task = tasks[blockIdx.x / C];
    const DevCfg& cf = cfgs[task.cfg];
    const int64_t j0 = ca.j_base + j_local;
    const int64_t j1 = (j0 + n_steps < cf.n_call) ? j0 + n_steps : cf.n_call;
    if (j0 >= j1) return;  // uniform over the cluster
    const int Lx = cf.Lx, Ly = cf.Ly;
    const int N = Lx * Ly;
    const int Lr = Ly / C;  // rows of this block
    const int G = Lx >> 2;
    const int NT = blockDim.x;
    const int NB = NT / G, R = Lr / NB, NBt = NB * C;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int band = tid / G, lg = tid - band * G;
    const int x = 4 * lg;
    const int gb = (lane / G) * G;
    const int srcL = gb + (lg + G - 1) % G, srcR = gb + (lg + 1) % G;
    constexpr bool R1 = ONE_ROW;  // a band's first and last rows coincide
    if ((R == 1) != ONE_ROW) return;  // the host launches the matching instantiation (uniform)

    float* s_th = reinterpret_cast<float*>(smem4);
    float* s_om = s_th + Lr * Lx;
    float2* s_exp = reinterpret_cast<float2*>(s_om + Lr * Lx);  // [parity][top, bottom][NB][Lx]
    double* s_red = reinterpret_cast<double*>(s_exp + 4 * NB * Lx);  // [parity][64]

    const int64_t lat_off = cf.offset + (int64_t)task.rep * cf.N;
    const int y_base = rank * Lr;
    {
        const bool odd = !ca.fixed_parity && (j0 & 1) != 0;
        const float* thS = (odd ? buf.thB : buf.thA) + lat_off + (int64_t)y_base * Lx;
        const float* omS = (odd ? buf.omB : buf.omA) + lat_off + (int64_t)y_base * Lx;
        for (int i = tid; i < Lr * Lx / 4; i += NT) {
            st4(s_th + 4 * i, ld4(thS + 4 * i));
            st4(s_om + 4 * i, ld4(omS + 4 * i));
        }
    }
    const uint32_t cfgrep = ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + task.rep);
    const int ytop = band * R, ybot = band * R + R - 1;  // rows within the block
    // neighbouring bands (cluster-wide numbering) and the blocks holding them
    const int gband = rank * NB + band;
    const int up = (gband + NBt - 1) % NBt, dn = (gband + 1) % NBt;
    const int rank_up = up / NB, lb_up = up - rank_up * NB;
    const int rank_dn = dn / NB, lb_dn = dn - rank_dn * NB;
    const StepConst K0 = step_const(cf, 0.f);
    const bool const_T = cf.sched_kind == 0 && cf.n_knots <= 1;
    const float c_const = noise_amp(cf, 0);
    // without a field or coupling schedule h, h p and the couplings are the
    // configuration's own for every step: read once here, not from the
    // descriptor after every cluster barrier
    const bool const_h = cf.f_n_knots == 0 && cf.c_n_knots == 0;
    const float h0 = cf.h;
    const float2 J0 = make_float2(cf.Jx, cf.Jy);
    // (each step loop below is compiled twice, with and without the schedules'
    // code, and the block takes one of them: without a schedule the loop
    // carries none of the knot searches' registers)
    const bool stag = cf.stag != 0;
    const int64_t kbase = cf.k_start + ca.k_shift;
    // noise of the band's single row (R = 1) at step k, computed one step
    // ahead between the arrival at the cluster barrier and the wait on it
    const uint32_t quad1 = (uint32_t)(((y_base + ytop) * Lx + x) >> 2);
    auto noise1 = [&](int64_t k) {
        return gauss4_scaled(philox4x32_10_rk(noise_counter(quad1, cfgrep, k, 0u), keys),
                             const_T ? c_const : noise_amp(cf, k));
    };
    float4 cn1 = R1 ? noise1(kbase + j0) : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();  // the block's rows are in shared memory

    if (R1) {
        // one row per band: the thread's quad stays in registers for the
        // whole launch; shared memory carries only the exported (s, c) rows
        const int y = ytop;
        const int gy = y_base + y;
        float4 th4 = ld4(s_th + y * Lx + x);
        float4 v4 = ld4(s_om + y * Lx + x);
        const float2* up_base = cl.map_shared_rank(s_exp + lb_up * Lx + x, rank_up);
        const float2* dn_base = cl.map_shared_rank(s_exp + lb_dn * Lx + x, rank_dn);
        auto steps = [&](auto fs) {
        constexpr bool FS = decltype(fs)::value;
        for (int64_t j = j0; j < j1; ++j) {
            const int64_t k = kbase + j;
            StepConst K = K0;
            K.c = const_T ? c_const : noise_amp(cf, k);
            if constexpr (FS) {
                const StepConst Kk = step_const_k(cf, k, K.c);
                K.hp = Kk.hp;
                K.nqJx = Kk.nqJx;
                K.nqJy = Kk.nqJy;
            }
            const bool rec = ca.record_every > 0 && (k % ca.record_every) == 0;
            const int par = (int)(j & 1);
            const size_t poff = (size_t)(2 * par) * NB * Lx;
            SC4 cur, prev, nxt;
            sc4_from_theta(th4, K.q, cur);
            sc4_store(s_exp + poff + band * Lx + x, cur);
            cluster_arrive();
            cluster_wait();
            sc4_load(up_base + poff, prev);
            sc4_load(dn_base + poff, nxt);
            // next step's noise: independent of the state, interleaved by the
            // compiler with this step's update
            float4 cn_next = cn1;
            if (j + 1 < j1) cn_next = noise1(k + 1);
            const float sL = __shfl_sync(kFull, cur.s[3], srcL), cL = __shfl_sync(kFull, cur.c[3], srcL);
            const float sR = __shfl_sync(kFull, cur.s[0], srcR), cR = __shfl_sync(kFull, cur.c[0], srcR);
            float to[4], vo[4];
            float pm = 0.f, pe = 0.f;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float sl = s == 0 ? sL : cur.s[s - 1];
                const float cl_ = s == 0 ? cL : cur.c[s - 1];
                const float sr = s == 3 ? sR : cur.s[s + 1];
                const float cr = s == 3 ? cR : cur.c[s + 1];
                const float sx = __fadd_rn(sl, sr), cx = __fadd_rn(cl_, cr);
                const float sy = __fadd_rn(prev.s[s], nxt.s[s]), cy = __fadd_rn(prev.c[s], nxt.c[s]);
                const float th = f4get(th4, s);
                const float F = site_force(K, cur.s[s], cur.c[s], sx, cx, sy, cy, sinp_of(K.p, th));
                const SiteOut so = site_update(K, th, f4get(v4, s), F, f4get(cn1, s));
                to[s] = so.theta;
                vo[s] = so.v;
                if (rec) {
                    const float sigma = (stag && ((x + s + gy) & 1)) ? -1.f : 1.f;
                    pm = fmaf(sigma, cur.s[s], pm);
                    if (!ca.m_only)
                        pe = __fadd_rn(pe, site_energy(cf, FS ? couplings_at(cf, k) : J0, FS ? field_h(cf, k) : h0, so.omega, cur.s[s], cur.c[s], sr, cr,
                                                       nxt.s[s], nxt.c[s], cosp_of(K.p, th)));
                }
            }
            th4 = make_float4(to[0], to[1], to[2], to[3]);
            v4 = make_float4(vo[0], vo[1], vo[2], vo[3]);
            cn1 = cn_next;
            if (rec) {
                double* red = s_red + 64 * par;
                const double wm = warp_sumf(pm), we = warp_sumf(pe);
                if (lane == 0) {
                    red[warp] = wm;
                    red[32 + warp] = we;
                }
                cl.sync();
                if (rank == 0 && tid == 0) {
                    double bm = 0.0, be = 0.0;
                    for (int rb = 0; rb < C; ++rb) {
                        const double* rr = cl.map_shared_rank(red, rb);
                        for (int w2 = 0; w2 < NT / 32; ++w2) {
                            bm += rr[w2];
                            be += rr[32 + w2];
                        }
                    }
                    const int64_t b = cf.b_first + task.rep;
                    const int64_t ri = (k - cf.rec_first) / ca.record_every;
                    ca.rec_dev[b * ca.rec_stride + ri] =
                        make_double2(bm / (double)N, ca.m_only ? 0.0 : be / (double)N + (double)cf.e_ref);
                }
            }
        }
        };
        if (const_h) steps(std::false_type{}); else steps(std::true_type{});
        st4(s_th + y * Lx + x, th4);
        st4(s_om + y * Lx + x, v4);
    } else {
        auto steps = [&](auto fs) {
        constexpr bool FS = decltype(fs)::value;
        for (int64_t j = j0; j < j1; ++j) {
            const int64_t k = kbase + j;
            StepConst K = K0;
            K.c = const_T ? c_const : noise_amp(cf, k);
            if constexpr (FS) {
                const StepConst Kk = step_const_k(cf, k, K.c);
                K.hp = Kk.hp;
                K.nqJx = Kk.nqJx;
                K.nqJy = Kk.nqJy;
            }
            const bool rec = ca.record_every > 0 && (k % ca.record_every) == 0;
            const int par = (int)(j & 1);
            float2* e_top = s_exp + (size_t)(2 * par) * NB * Lx;
            float2* e_bot = R1 ? e_top : e_top + (size_t)NB * Lx;
            // phase 1
            {
                SC4 a;
                sc4_from_theta(ld4(s_th + ytop * Lx + x), K.q, a);
                sc4_store(e_top + band * Lx + x, a);
                if (!R1) {
                    sc4_from_theta(ld4(s_th + ybot * Lx + x), K.q, a);
                    sc4_store(e_bot + band * Lx + x, a);
                }
            }
            cluster_arrive();
            float4 cn_next = cn1;
            if (R1 && j + 1 < j1) cn_next = noise1(k + 1);
            cluster_wait();
            // phase 2
            SC4 prev, cur, nxt;
            sc4_load(cl.map_shared_rank(e_bot + lb_up * Lx + x, rank_up), prev);
            sc4_load(e_top + band * Lx + x, cur);
            float pm = 0.f, pe = 0.f;
            for (int r = 0; r < R; ++r) {
                const int y = ytop + r;
                if (r == R - 1) sc4_load(cl.map_shared_rank(e_top + lb_dn * Lx + x, rank_dn), nxt);
                else if (r + 1 == R - 1) sc4_load(e_bot + band * Lx + x, nxt);
                else sc4_from_theta(ld4(s_th + (y + 1) * Lx + x), K.q, nxt);
                const float4 th4 = ld4(s_th + y * Lx + x);
                const float4 v4 = ld4(s_om + y * Lx + x);
                const float sL = __shfl_sync(kFull, cur.s[3], srcL), cL = __shfl_sync(kFull, cur.c[3], srcL);
                const float sR = __shfl_sync(kFull, cur.s[0], srcR), cR = __shfl_sync(kFull, cur.c[0], srcR);
                float4 cn = cn1;
                if (!R1) {
                    const uint32_t quad = (uint32_t)(((y_base + y) * Lx + x) >> 2);
                    cn = gauss4_scaled(philox4x32_10_rk(noise_counter(quad, cfgrep, k, 0u), keys), K.c);
                }
                float to[4], vo[4];
    #pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const float sl = s == 0 ? sL : cur.s[s - 1];
                    const float cl_ = s == 0 ? cL : cur.c[s - 1];
                    const float sr = s == 3 ? sR : cur.s[s + 1];
                    const float cr = s == 3 ? cR : cur.c[s + 1];
                    const float sx = __fadd_rn(sl, sr), cx = __fadd_rn(cl_, cr);
                    const float sy = __fadd_rn(prev.s[s], nxt.s[s]), cy = __fadd_rn(prev.c[s], nxt.c[s]);
                    const float th = f4get(th4, s);
                    const float F = site_force(K, cur.s[s], cur.c[s], sx, cx, sy, cy, sinp_of(K.p, th));
                    const SiteOut so = site_update(K, th, f4get(v4, s), F, f4get(cn, s));
                    to[s] = so.theta;
                    vo[s] = so.v;
                    if (rec) {
                        const float sigma = (stag && ((x + s + y_base + y) & 1)) ? -1.f : 1.f;
                        pm = fmaf(sigma, cur.s[s], pm);
                        if (!ca.m_only)
                            pe = __fadd_rn(pe, site_energy(cf, FS ? couplings_at(cf, k) : J0, FS ? field_h(cf, k) : h0, so.omega, cur.s[s], cur.c[s], sr, cr,
                                                           nxt.s[s], nxt.c[s], cosp_of(K.p, th)));
                    }
                }
                st4(s_th + y * Lx + x, make_float4(to[0], to[1], to[2], to[3]));
                st4(s_om + y * Lx + x, make_float4(vo[0], vo[1], vo[2], vo[3]));
                prev = cur;
                cur = nxt;
            }
            cn1 = cn_next;
            if (rec) {
                // warp partials of every block, summed by block 0 in (block, warp) order
                double* red = s_red + 64 * par;
                const double wm = warp_sumf(pm), we = warp_sumf(pe);
                if (lane == 0) {
                    red[warp] = wm;
                    red[32 + warp] = we;
                }
                cl.sync();
                if (rank == 0 && tid == 0) {
                    double bm = 0.0, be = 0.0;
                    for (int rb = 0; rb < C; ++rb) {
                        const double* rr = cl.map_shared_rank(red, rb);
                        for (int w2 = 0; w2 < NT / 32; ++w2) {
                            bm += rr[w2];
                            be += rr[32 + w2];
                        }
                    }
                    const int64_t b = cf.b_first + task.rep;
                    const int64_t ri = (k - cf.rec_first) / ca.record_every;
                    ca.rec_dev[b * ca.rec_stride + ri] =
                        make_double2(bm / (double)N, ca.m_only ? 0.0 : be / (double)N + (double)cf.e_ref);
                }
            }
        }
        };
        if (const_h) steps(std::false_type{}); else steps(std::true_type{});
    }
    // no block leaves while another may still read its shared memory
    cl.sync();
    {
        const bool odd = ca.fixed_parity ? true : (j1 & 1) != 0;
        float* thD = (odd ? buf.thB : buf.thA) + lat_off + (int64_t)y_base * Lx;
        float* omD = (odd ? buf.omB : buf.omA) + lat_off + (int64_t)y_base * Lx;
        for (int i = tid; i < Lr * Lx / 4; i += NT) {
            st4(thD + 4 * i, ld4(s_th + 4 * i));
            st4(omD + 4 * i, ld4(s_om + 4 * i));
        }
    }
}

namespace {
using ResidentFn = void (*)(const DevCfg*, const ResidentTask*, int64_t, int, Buffers, const CallArgs*, PhiloxKeys);

// the instantiation for a block size and band height (rows of a band: the
// block's Ly / csize rows over its threads / (Lx / 4) bands)
ResidentFn resident_fn(int Lx, int Ly, int threads, int csize)
{
    const int R = (Ly / csize) / (threads / (Lx / 4));
    if (threads > 512) return R == 1 ? resident_step_kernel<1024, true> : resident_step_kernel<1024, false>;
    return R == 1 ? resident_step_kernel<512, true> : resident_step_kernel<512, false>;
}

cudaLaunchConfig_t resident_config(int n_tasks, int threads, int csize, size_t smem, cudaStream_t st,
                                   cudaLaunchAttribute* at)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(n_tasks * csize));
    lc.blockDim = dim3((unsigned)threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return lc;
}
}  // namespace

cudaError_t launch_resident_step(const DevCfg* d_cfg, const ResidentTask* tasks, int n_tasks, int Lx, int Ly,
                                 int threads, int csize, uint64_t seed, int64_t j_local, int n_steps, Buffers buf,
                                 const CallArgs* ca, cudaStream_t st)
{
    if (n_tasks == 0) return cudaSuccess;
    const size_t smem = resident_smem_bytes(Lx, Ly, threads, csize);
    const PhiloxKeys keys = philox_round_keys(seed);
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t lc = resident_config(n_tasks, threads, csize, smem, st, at);
    const cudaError_t e =
        cudaLaunchKernelEx(&lc, resident_fn(Lx, Ly, threads, csize), d_cfg, tasks, j_local, n_steps, buf, ca, keys);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Opt in to the dynamic shared memory (and, above 8 blocks, the non-portable
// cluster size) of one resident shape, outside any capture.  *clusters, when
// given, receives how many such clusters fit on the device at once (0: the
// shape cannot run).
cudaError_t prepare_resident(int Lx, int Ly, int threads, int csize, int* clusters)
{
    const int smem = (int)resident_smem_bytes(Lx, Ly, threads, csize);
    const ResidentFn fn = resident_fn(Lx, Ly, threads, csize);
    // Several shapes (of one object or of several, and the tuner's
    // candidates) share a kernel instance, and the attribute belongs to the
    // instance: only ever raise it, so that no shape prepared earlier, or a
    // graph captured with it, loses the shared memory it launches with.
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)fn);
    if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < smem)
        e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && csize > 8)
        e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess || !clusters) return e;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t lc = resident_config(1, threads, csize, (size_t)smem, nullptr, at);
    *clusters = 0;
    e = cudaOccupancyMaxActiveClusters(clusters, (const void*)fn, &lc);
    if (e != cudaSuccess) {  // an unsupported cluster shape is "does not fit", not a failure
        cudaGetLastError();
        *clusters = 0;
        e = cudaSuccess;
    }
    return e;
}

// ===========================================================================
// Small kernels: chunk counter, moments, diagnostics.
// ===========================================================================
__global__ void advance_kernel(CallArgs* ca, int64_t by) { ca->j_base += by; }

cudaError_t launch_advance(CallArgs* ca, int64_t by, cudaStream_t st)
{
    advance_kernel<<<1, 1, 0, st>>>(ca, by);
    return cudaGetLastError();
}

__global__ void add_kshift_kernel(CallArgs* ca, int64_t by) { ca->k_shift += by; }

cudaError_t launch_add_kshift(CallArgs* ca, int64_t by, cudaStream_t st)
{
    add_kshift_kernel<<<1, 1, 0, st>>>(ca, by);
    return cudaGetLastError();
}

// Running FP64 moments of one configuration (App. B, Eq.
// ensemble-average-calculation): sums over replicas and recorded steps
// k >= t0 of (1, M^2, M^4, E, E^2, |M|), added to moments[c][0..5].  Fixed
// per-thread strides and a fixed tree make the sums deterministic.
__global__ void __launch_bounds__(256) moments_kernel(const DevCfg* cfgs, const CallArgs* cap, int64_t t0,
                                                      double* moments)
{
    const DevCfg& cf = cfgs[blockIdx.x];
    const CallArgs ca = *cap;
    __shared__ double s_acc[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const int re = ca.record_every;
    int64_t n_rec = 0;
    if (re > 0 && cf.n_call > 0 && cf.rec_first < cf.k_start + cf.n_call)
        n_rec = (cf.k_start + cf.n_call - 1 - cf.rec_first) / re + 1;
    const int64_t total = n_rec * cf.n_rep;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int64_t rep = i / n_rec, r = i - rep * n_rec;
        const int64_t k = cf.rec_first + r * re;
        if (k < t0) continue;
        const double2 me = ca.rec_dev[(cf.b_first + rep) * ca.rec_stride + r];
        const double m2 = me.x * me.x;
        acc[0] += 1.0;
        acc[1] += m2;
        acc[2] += m2 * m2;
        acc[3] += me.y;
        acc[4] += me.y * me.y;
        acc[5] += fabs(me.x);
    }
    for (int q = 0; q < 6; ++q) s_acc[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 6; ++q) s_acc[q][threadIdx.x] += s_acc[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) moments[6 * blockIdx.x + q] += s_acc[q][0];
}

cudaError_t launch_moments(const DevCfg* d_cfg, int n_cfg, const CallArgs* ca, int64_t t0, double* moments,
                           cudaStream_t st)
{
    moments_kernel<<<n_cfg, 256, 0, st>>>(d_cfg, ca, t0, moments);
    return cudaGetLastError();
}

__global__ void debug_noise_kernel(uint64_t seed, int cfg, int rep, int64_t k, int tag, int64_t n_quads,
                                   uint32_t* words, float* gauss)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_quads) return;
    const uint4 w = philox4x32_10(noise_counter((uint32_t)q, ((uint32_t)cfg << 16) | (uint32_t)rep, k, (uint32_t)tag),
                                  (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    if (words) *reinterpret_cast<uint4*>(words + 4 * q) = w;
    if (gauss) st4(gauss + 4 * q, gauss4_scaled(w, 1.0f));
}

cudaError_t launch_debug_noise(uint64_t seed, int cfg, int rep, int64_t k, int tag, int64_t n_quads,
                               uint32_t* words, float* gauss, cudaStream_t st)
{
    if (n_quads <= 0) return cudaSuccess;
    debug_noise_kernel<<<(unsigned)((n_quads + 255) / 256), 256, 0, st>>>(seed, cfg, rep, k, tag, n_quads, words,
                                                                          gauss);
    return cudaGetLastError();
}

__global__ void debug_gauss4_kernel(const uint32_t* words, int64_t n_quads, float c, float* out)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n_quads) return;
    st4(out + 4 * q, gauss4_scaled(*reinterpret_cast<const uint4*>(words + 4 * q), c));
}

cudaError_t launch_debug_gauss4(const uint32_t* words, int64_t n_quads, float c, float* out, cudaStream_t st)
{
    if (n_quads <= 0) return cudaSuccess;
    debug_gauss4_kernel<<<(unsigned)((n_quads + 255) / 256), 256, 0, st>>>(words, n_quads, c, out);
    return cudaGetLastError();
}

__global__ void debug_philox_kernel(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = *reinterpret_cast<const uint4*>(ctr + 4 * i);
    *reinterpret_cast<uint4*>(out + 4 * i) = philox4x32_10(c, k0, k1);
}

cudaError_t launch_debug_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                                cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    debug_philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, k0, k1, n, out);
    return cudaGetLastError();
}

}  // namespace xy
