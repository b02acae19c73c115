// xy_adjoint.cu -- reverse sweep of the pathwise adjoint of the BBK
// trajectory (App. A.1) with the noise held fixed.
//
// Forward map of one step in the stored leapfrog variables (theta_k,
// v_k = omega_{k-1/2}), with b = 1 / (1 + a), a = eta dt / 2:
//   F_k = F(theta_k),  g_k = (dt/2) F_k + c_k n_k,  omega_k = (v_k + g_k) b,
//   v_{k+1} = (1 - a) omega_k + g_k,  theta_{k+1} = wrap(theta_k + dt v_{k+1}),
// observation O_k = w_E E_k(theta_k, omega_k) + w_M |M_k(theta_k)| for
// k0 < k <= k0 + n.  At k = k0 the full-step omega_{k0} is held fixed.
//
// Reverse of step k, given the adjoints (tb, vb) of (theta_{k+1}, v_{k+1}):
//   phase A (site-local):  vb' = vb + dt tb,  omega-bar = (1-a) vb',
//     g-bar = vb',  a-bar -= omega_k vb';  observation terms;
//     if k > k0:  v-bar_k = b omega-bar,  g-bar += b omega-bar,
//                 b-bar += (v_k + g_k) omega-bar;
//     F-bar = (dt/2) g-bar,  c-bar += g-bar n_k,  parameter terms of F;
//   phase B (stencil):  tb += (dF/dtheta)^T F-bar, i.e.
//     tb_j += q^2 sum_n J_n cos q(t_j - t_n) (Fb_n - Fb_j) + h p^2 cos(p t_j) Fb_j.
// d/d eta = (dt/2)(a-bar - b^2 b-bar) + sum_k c-bar_k c_k / (2 eta).
#include "xy_device.cuh"

namespace xy {

namespace {

constexpr unsigned kFullA = 0xFFFFFFFFu;

// Periodic index for offsets in (-n, 2n): one compare-and-add either way.
__device__ __forceinline__ int wrapa(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void sc_q(float q, float th, float& s, float& c) { __sincosf(__fmul_rn(q, th), &s, &c); }

struct Nbr4 {
    float t[4];           // own
    float tl, tr;         // x-1 of site 0, x+4
    float tu[4], td[4];   // y-1, y+1
};

__device__ __forceinline__ void load_nbr(const float* lat, int Lx, int Ly, int x, int y, Nbr4& n)
{
    const float4 a = ld4(lat + (int64_t)y * Lx + x);
    const float4 u = ld4(lat + (int64_t)wrapa(y - 1, Ly) * Lx + x);
    const float4 d = ld4(lat + (int64_t)wrapa(y + 1, Ly) * Lx + x);
    n.t[0] = a.x; n.t[1] = a.y; n.t[2] = a.z; n.t[3] = a.w;
    n.tu[0] = u.x; n.tu[1] = u.y; n.tu[2] = u.z; n.tu[3] = u.w;
    n.td[0] = d.x; n.td[1] = d.y; n.td[2] = d.z; n.td[3] = d.w;
    n.tl = lat[(int64_t)y * Lx + wrapa(x - 1, Lx)];
    n.tr = lat[(int64_t)y * Lx + wrapa(x + 4, Lx)];
}

__device__ __forceinline__ double warp_sum_a(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullA, v, o);
    return v;
}

}  // namespace

int adjoint_blocks(const DevCfg& h)
{
    const int64_t nq_lat = h.N / 4;
    return (int)((nq_lat + 255) / 256) * h.n_rep;
}

__global__ void __launch_bounds__(256) adjoint_phase_a_kernel(const DevCfg* cfgs, int c, int block_base, AdjArgs A)
{
    const DevCfg& cf = cfgs[c];
    __shared__ float s_c;
    __shared__ double s_red[kGacc][8];
    const int64_t k = A.k;
    if (threadIdx.x == 0) s_c = noise_amp(cf, k);
    __syncthreads();
    const StepConst K = step_const(cf, s_c);
    const int64_t nq_lat = cf.N / 4;
    const int bpl = (int)((nq_lat + blockDim.x - 1) / blockDim.x);
    const int rep = blockIdx.x / bpl;
    const int unit = blockIdx.x - rep * bpl;
    const int64_t quad = (int64_t)unit * blockDim.x + threadIdx.x;
    const int64_t lat_off = cf.offset + (int64_t)rep * cf.N;
    const bool observe = k > A.k0;
    const bool first = k == A.k0;
    const float invN = 1.0f / (float)cf.N;
    float aJx = 0.f, aJy = 0.f, ah = 0.f, abar = 0.f, bbar = 0.f, cbar = 0.f, eacc = 0.f;
    if (quad < nq_lat) {
        const int y = (int)(4 * quad / cf.Lx), x = (int)(4 * quad - (int64_t)y * cf.Lx);
        Nbr4 n;
        load_nbr(A.theta + lat_off, cf.Lx, cf.Ly, x, y, n);
        float s[4], co[4], su[4], cu[4], sd[4], cd[4], sl, cl, sr, cr;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            sc_q(K.q, n.t[i], s[i], co[i]);
            sc_q(K.q, n.tu[i], su[i], cu[i]);
            sc_q(K.q, n.td[i], sd[i], cd[i]);
        }
        sc_q(K.q, n.tl, sl, cl);
        sc_q(K.q, n.tr, sr, cr);
        const uint4 w = philox4x32_10(
            noise_counter((uint32_t)quad, ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + rep), k, 0u), cf.key0, cf.key1);
        const float4 nz = gauss4_scaled(w, 1.0f);     // n_k (unit Gaussians)
        const float4 cn = gauss4_scaled(w, K.c);      // c_k n_k exactly as in the forward step
        const float4 v = ld4(A.omega + lat_off + 4 * quad);
        const float4 tb4 = ld4(A.tb + lat_off + 4 * quad);
        const float4 vb4 = ld4(A.vb + lat_off + 4 * quad);
        float sgnM = 0.f;
        if (observe && A.wM != 0.0) {
            const double M = A.rec[(int64_t)(cf.b_first + rep) * A.rec_stride + (k - A.k0)].x;
            sgnM = M > 0.0 ? 1.f : (M < 0.0 ? -1.f : 0.f);
        }
        const float wE = (float)A.wE, wM = (float)A.wM;
        float tbo[4], vbo[4], fbo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float sL = i == 0 ? sl : s[i - 1], cL = i == 0 ? cl : co[i - 1];
            const float sR = i == 3 ? sr : s[i + 1], cR = i == 3 ? cr : co[i + 1];
            const float sx = __fadd_rn(sL, sR), cx = __fadd_rn(cL, cR);
            const float sy = __fadd_rn(su[i], sd[i]), cy = __fadd_rn(cu[i], cd[i]);
            const float sinp = __sinf(__fmul_rn(K.p, n.t[i]));
            const float F = site_force(K, s[i], co[i], sx, cx, sy, cy, sinp);
            const SiteOut so = site_update(K, n.t[i], f4get(v, i), F, f4get(cn, i));
            const float om = so.omega;
            const float vbt = fmaf(K.dt, f4get(tb4, i), f4get(vb4, i));
            float omb = __fmul_rn(K.oma, vbt);
            float gb = vbt;
            abar = fmaf(-om, vbt, abar);
            float tbi = f4get(tb4, i);
            if (observe) {
                omb = fmaf(wE * invN, om, omb);
                // dE/dtheta = -F / N ; d|M|/dtheta = sgn(M) sigma q cos(q theta) / N
                tbi = fmaf(-wE * invN, F, tbi);
                const float sigma = (cf.stag && ((x + i + y) & 1)) ? -1.f : 1.f;
                tbi = fmaf(wM * invN * sgnM * sigma * K.q, co[i], tbi);
                // explicit parameter dependence of E (forward bonds)
                const float bx = fmaf(co[i], cR, s[i] * sR);
                const float by = fmaf(co[i], cd[i], s[i] * sd[i]);
                const float cp = __cosf(__fmul_rn(K.p, n.t[i]));
                aJx = fmaf(-wE * invN, bx, aJx);
                aJy = fmaf(-wE * invN, by, aJy);
                ah = fmaf(wE * invN, cp, ah);
                float e = __fmul_rn(0.5f, __fmul_rn(om, om));
                e = fmaf(-cf.Jx, bx, e);
                e = fmaf(-cf.Jy, by, e);
                e = fmaf(cf.h, cp, e);
                eacc = fmaf(wE * invN, e, eacc);
            }
            float vbk = 0.f;
            if (!first) {
                vbk = __fmul_rn(K.inv1pa, omb);
                gb = fmaf(K.inv1pa, omb, gb);
                bbar = fmaf(__fadd_rn(f4get(v, i), fmaf(K.hdt, F, f4get(cn, i))), omb, bbar);
            }
            const float fb = __fmul_rn(K.hdt, gb);
            cbar = fmaf(gb, f4get(nz, i), cbar);
            // parameter dependence of F: dF/dJx = -q (s cx - c sx), dF/dJy likewise, dF/dh = p sin(p t)
            aJx = fmaf(fb, -K.q * fmaf(s[i], cx, -co[i] * sx), aJx);
            aJy = fmaf(fb, -K.q * fmaf(s[i], cy, -co[i] * sy), aJy);
            ah = fmaf(fb, K.p * sinp, ah);
            tbo[i] = tbi;
            vbo[i] = vbk;
            fbo[i] = fb;
        }
        st4(A.tb + lat_off + 4 * quad, make_float4(tbo[0], tbo[1], tbo[2], tbo[3]));
        st4(A.vb + lat_off + 4 * quad, make_float4(vbo[0], vbo[1], vbo[2], vbo[3]));
        st4(A.Fb + lat_off + 4 * quad, make_float4(fbo[0], fbo[1], fbo[2], fbo[3]));
    }
    // block sums in FP64, fixed order; per-block accumulators across steps
    const double ceta = cf.eta_d > 0.0 ? (double)K.c / (2.0 * cf.eta_d) : 0.0;  // d c_k / d eta = c_k / (2 eta)
    double vals[kGacc] = {aJx, aJy, ah, abar, bbar, (double)cbar * ceta, eacc};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kGacc; ++q) {
        const double w = warp_sum_a(vals[q]);
        if (lane == 0) s_red[q][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < kGacc) {
        double acc = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) acc += s_red[threadIdx.x][w2];
        A.gacc[(int64_t)(block_base + blockIdx.x) * kGacc + threadIdx.x] += acc;
    }
}

__global__ void __launch_bounds__(256) adjoint_phase_b_kernel(const DevCfg* cfgs, int c, AdjArgs A)
{
    const DevCfg& cf = cfgs[c];
    const int64_t nq_lat = cf.N / 4;
    const int bpl = (int)((nq_lat + blockDim.x - 1) / blockDim.x);
    const int rep = blockIdx.x / bpl;
    const int unit = blockIdx.x - rep * bpl;
    const int64_t quad = (int64_t)unit * blockDim.x + threadIdx.x;
    if (quad >= nq_lat) return;
    const int64_t lat_off = cf.offset + (int64_t)rep * cf.N;
    const int Lx = cf.Lx, Ly = cf.Ly;
    const int y = (int)(4 * quad / Lx), x = (int)(4 * quad - (int64_t)y * Lx);
    const float q = cf.q, q2 = __fmul_rn(cf.q, cf.q);
    Nbr4 t, f;
    load_nbr(A.theta + lat_off, Lx, Ly, x, y, t);
    load_nbr(A.Fb + lat_off, Lx, Ly, x, y, f);
    float s[4], co[4], su[4], cu[4], sd[4], cd[4], sl, cl, sr, cr;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        sc_q(q, t.t[i], s[i], co[i]);
        sc_q(q, t.tu[i], su[i], cu[i]);
        sc_q(q, t.td[i], sd[i], cd[i]);
    }
    sc_q(q, t.tl, sl, cl);
    sc_q(q, t.tr, sr, cr);
    const float4 tb4 = ld4(A.tb + lat_off + 4 * quad);
    float out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float sL = i == 0 ? sl : s[i - 1], cL = i == 0 ? cl : co[i - 1];
        const float sR = i == 3 ? sr : s[i + 1], cR = i == 3 ? cr : co[i + 1];
        const float fL = i == 0 ? f.tl : f.t[i - 1];
        const float fR = i == 3 ? f.tr : f.t[i + 1];
        const float fj = f.t[i];
        const float kL = fmaf(co[i], cL, s[i] * sL), kR = fmaf(co[i], cR, s[i] * sR);
        const float kU = fmaf(co[i], cu[i], s[i] * su[i]), kD = fmaf(co[i], cd[i], s[i] * sd[i]);
        const float hx = fmaf(kL, fL - fj, kR * (fR - fj));
        const float hy = fmaf(kU, f.tu[i] - fj, kD * (f.td[i] - fj));
        float acc = q2 * fmaf(cf.Jx, hx, cf.Jy * hy);
        acc = fmaf(cf.hp * cf.p, __cosf(__fmul_rn(cf.p, t.t[i])) * fj, acc);
        out[i] = __fadd_rn(f4get(tb4, i), acc);
    }
    st4(A.tb + lat_off + 4 * quad, make_float4(out[0], out[1], out[2], out[3]));
}

cudaError_t launch_adjoint_phase_a(const DevCfg* d_cfg, const DevCfg& h, int block_base, AdjArgs a, cudaStream_t st)
{
    adjoint_phase_a_kernel<<<adjoint_blocks(h), 256, 0, st>>>(d_cfg, h.slot, block_base, a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_phase_b(const DevCfg* d_cfg, const DevCfg& h, AdjArgs a, cudaStream_t st)
{
    adjoint_phase_b_kernel<<<adjoint_blocks(h), 256, 0, st>>>(d_cfg, h.slot, a);
    return cudaGetLastError();
}


// ===========================================================================
// Fused reverse step on the strip decomposition of the forward stepper.
//
// One launch performs phase B of step kB = kA + 1 (the Hessian stencil on
// F-bar_{kB}, reading theta_{kB}) and phase A of step kA (site-local,
// reading theta_{kA}, v_{kA}) on the same rows: tb and vb are touched only at
// their own site, so they are updated in place; F-bar of step kA goes to a
// second buffer because phase B of the next launch reads it with its
// neighbours.  Each warp walks its unit's rows with sliding windows of
// (sin q t, cos q t) of both time levels and of F-bar; x neighbours come by
// shuffles and the strip's edge columns from global memory, as in the
// forward stepper.  Either phase can be switched off (segment ends).
// ===========================================================================
namespace {

struct RevRow {
    float4 th;
    float te;
    float s[4], c[4];
};

__device__ __forceinline__ void rev_sc(float q, RevRow& r)
{
    sc_q(q, r.th.x, r.s[0], r.c[0]);
    sc_q(q, r.th.y, r.s[1], r.c[1]);
    sc_q(q, r.th.z, r.s[2], r.c[2]);
    sc_q(q, r.th.w, r.s[3], r.c[3]);
}

__device__ __forceinline__ void rev_load(const float* lat, int64_t row, int x, int xe, RevRow& r)
{
    r.th = ld4(lat + row + x);
    r.te = lat[row + xe];
}

}  // namespace

template <int MINB, bool DOA, bool DOB>
__global__ void __launch_bounds__(256, MINB) adjoint_strip_kernel(const DevCfg* cfgs, const StripTask* tasks, int H,
                                                                  RevArgs R, PhiloxKeys keys)
{
    __shared__ double s_red[kGacc][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const StripTask task = tasks[blockIdx.x];
    const int unit = task.unit0 + warp;
    const bool active = unit < task.n_units;
    const DevCfg& cf = cfgs[task.cfg];
    const int Lx = cf.Lx, Ly = cf.Ly;
    const int64_t lat_off = cf.offset + (int64_t)task.rep * cf.N;
    const float q = cf.q, q2 = __fmul_rn(cf.q, cf.q), hp2 = __fmul_rn(cf.hp, cf.p);
    const StepConst KA = step_const(cf, noise_amp(cf, R.kA));
    const float invN = 1.0f / (float)cf.N;
    const float wE = R.wE, wM = R.wM;
    const bool observe = R.kA > R.k0, first = R.kA == R.k0;
    float aJx = 0.f, aJy = 0.f, ah = 0.f, abar = 0.f, bbar = 0.f, cbar = 0.f, eacc = 0.f;
    if (active) {
        const int G = Lx >= 128 ? 32 : (Lx >> 2);
        const int groups = 32 / G;
        const int strips = Lx >= 128 ? (Lx >> 7) : 1;
        const int seg = unit / strips;
        const int x0 = (unit - seg * strips) * 128;
        const int grp = lane / G, lg = lane - grp * G;
        const bool multi = Lx > 128;
        const int x = x0 + 4 * lg;
        const int ybeg = seg * H * groups + grp * H;
        const int xe = multi ? (lg == 0 ? wrapa(x0 - 1, Lx) : wrapa(x0 + 128, Lx)) : x;
        const int srcL = grp * G + (lg + G - 1) % G;
        const int srcR = grp * G + (lg + 1) % G;
        const uint32_t cfgrep = ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + task.rep);
        const float* thB = R.thB + lat_off;
        const float* FbI = R.FbIn + lat_off;
        const float* thA = R.thA + lat_off;
        const float* vA = R.vA + lat_off;
        float* tb = R.tb + lat_off;
        float* vb = R.vb + lat_off;
        float* FbO = R.FbOut + lat_off;
        float sgnM = 0.f;
        if (DOA && observe && R.wM != 0.f) {
            const double M = R.rec[(int64_t)(cf.b_first + task.rep) * R.rec_stride + (R.kA - R.k0)].x;
            sgnM = M > 0.0 ? 1.f : (M < 0.0 ? -1.f : 0.f);
        }
        RevRow PB, CB, NB, PA, CA, NA;
        float4 FP, FC, FN;
        const int yp = wrapa(ybeg - 1, Ly);
        if (DOB) {
            rev_load(thB, (int64_t)yp * Lx, x, xe, PB);
            rev_load(thB, (int64_t)ybeg * Lx, x, xe, CB);
            rev_sc(q, PB);
            rev_sc(q, CB);
            FP = ld4(FbI + (int64_t)yp * Lx + x);
            FC = ld4(FbI + (int64_t)ybeg * Lx + x);
        }
        if (DOA) {
            rev_load(thA, (int64_t)yp * Lx, x, xe, PA);
            rev_load(thA, (int64_t)ybeg * Lx, x, xe, CA);
            rev_sc(KA.q, PA);
            rev_sc(KA.q, CA);
        }
        for (int r = 0; r < H; ++r) {
            const int y = ybeg + r;
            const int yn = wrapa(y + 1, Ly);
            const int64_t row = (int64_t)y * Lx, rown = (int64_t)yn * Lx;
            float4 tb4 = ld4(tb + row + x);
            // ---------------- phase B of step kB at row y
            if (DOB) {
                rev_load(thB, rown, x, xe, NB);
                FN = ld4(FbI + rown + x);
                const float fe = FbI[row + xe];
                rev_sc(q, NB);
                float sL = __shfl_sync(kFullA, CB.s[3], srcL), cL = __shfl_sync(kFullA, CB.c[3], srcL);
                float sR = __shfl_sync(kFullA, CB.s[0], srcR), cR = __shfl_sync(kFullA, CB.c[0], srcR);
                float fL = __shfl_sync(kFullA, FC.w, srcL), fR = __shfl_sync(kFullA, FC.x, srcR);
                if (multi) {
                    float se, ce;
                    sc_q(q, CB.te, se, ce);
                    if (lg == 0) { sL = se; cL = ce; fL = fe; }
                    if (lg == 31) { sR = se; cR = ce; fR = fe; }
                }
                float out[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float sl = i == 0 ? sL : CB.s[i - 1], cl = i == 0 ? cL : CB.c[i - 1];
                    const float sr = i == 3 ? sR : CB.s[i + 1], cr = i == 3 ? cR : CB.c[i + 1];
                    const float fl = i == 0 ? fL : f4get(FC, i - 1), fr = i == 3 ? fR : f4get(FC, i + 1);
                    const float fj = f4get(FC, i);
                    const float kl = fmaf(CB.c[i], cl, CB.s[i] * sl), kr = fmaf(CB.c[i], cr, CB.s[i] * sr);
                    const float ku = fmaf(CB.c[i], PB.c[i], CB.s[i] * PB.s[i]);
                    const float kd = fmaf(CB.c[i], NB.c[i], CB.s[i] * NB.s[i]);
                    const float hx = fmaf(kl, fl - fj, kr * (fr - fj));
                    const float hy = fmaf(ku, f4get(FP, i) - fj, kd * (f4get(FN, i) - fj));
                    float acc = q2 * fmaf(cf.Jx, hx, cf.Jy * hy);
                    acc = fmaf(hp2, __cosf(__fmul_rn(cf.p, f4get(CB.th, i))) * fj, acc);
                    out[i] = __fadd_rn(f4get(tb4, i), acc);
                }
                tb4 = make_float4(out[0], out[1], out[2], out[3]);
                PB = CB;
                CB = NB;
                FP = FC;
                FC = FN;
            }
            // ---------------- phase A of step kA at row y
            if (DOA) {
                rev_load(thA, rown, x, xe, NA);
                const float4 v = ld4(vA + row + x);
                const float4 vb4 = ld4(vb + row + x);
                rev_sc(KA.q, NA);
                float sL = __shfl_sync(kFullA, CA.s[3], srcL), cL = __shfl_sync(kFullA, CA.c[3], srcL);
                float sR = __shfl_sync(kFullA, CA.s[0], srcR), cR = __shfl_sync(kFullA, CA.c[0], srcR);
                if (multi) {
                    float se, ce;
                    sc_q(KA.q, CA.te, se, ce);
                    if (lg == 0) { sL = se; cL = ce; }
                    if (lg == 31) { sR = se; cR = ce; }
                }
                const uint32_t quad = (uint32_t)((row + x) >> 2);
                const float4 nz = gauss4_scaled(philox4x32_10_rk(noise_counter(quad, cfgrep, R.kA, 0u), keys), 1.0f);
                float tbo[4], vbo[4], fbo[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float sl = i == 0 ? sL : CA.s[i - 1], cl = i == 0 ? cL : CA.c[i - 1];
                    const float sr = i == 3 ? sR : CA.s[i + 1], cr = i == 3 ? cR : CA.c[i + 1];
                    const float sx = __fadd_rn(sl, sr), cx = __fadd_rn(cl, cr);
                    const float sy = __fadd_rn(PA.s[i], NA.s[i]), cy = __fadd_rn(PA.c[i], NA.c[i]);
                    const float th = f4get(CA.th, i);
                    const float sinp = __sinf(__fmul_rn(KA.p, th));
                    const float F = site_force(KA, CA.s[i], CA.c[i], sx, cx, sy, cy, sinp);
                    const float cn = __fmul_rn(KA.c, f4get(nz, i));
                    const float g = fmaf(KA.hdt, F, cn);
                    const float om = __fmul_rn(__fadd_rn(f4get(v, i), g), KA.inv1pa);
                    const float vbt = fmaf(KA.dt, f4get(tb4, i), f4get(vb4, i));
                    float omb = __fmul_rn(KA.oma, vbt);
                    float gb = vbt;
                    abar = fmaf(-om, vbt, abar);
                    float tbi = f4get(tb4, i);
                    if (observe) {
                        omb = fmaf(wE * invN, om, omb);
                        tbi = fmaf(-wE * invN, F, tbi);
                        const float sigma = (cf.stag && ((x + i + y) & 1)) ? -1.f : 1.f;
                        tbi = fmaf(wM * invN * sgnM * sigma * KA.q, CA.c[i], tbi);
                        const float bx = fmaf(CA.c[i], cr, CA.s[i] * sr);
                        const float by = fmaf(CA.c[i], NA.c[i], CA.s[i] * NA.s[i]);
                        const float cp = __cosf(__fmul_rn(KA.p, th));
                        aJx = fmaf(-wE * invN, bx, aJx);
                        aJy = fmaf(-wE * invN, by, aJy);
                        ah = fmaf(wE * invN, cp, ah);
                        // the objective's energy term: w_E E_kA summed over sites (E linear in the sum)
                        float e = __fmul_rn(0.5f, __fmul_rn(om, om));
                        e = fmaf(-cf.Jx, bx, e);
                        e = fmaf(-cf.Jy, by, e);
                        e = fmaf(cf.h, cp, e);
                        eacc = fmaf(wE * invN, e, eacc);
                    }
                    float vbk = 0.f;
                    if (!first) {
                        vbk = __fmul_rn(KA.inv1pa, omb);
                        gb = fmaf(KA.inv1pa, omb, gb);
                        bbar = fmaf(__fadd_rn(f4get(v, i), g), omb, bbar);
                    }
                    const float fb = __fmul_rn(KA.hdt, gb);
                    cbar = fmaf(gb, f4get(nz, i), cbar);
                    aJx = fmaf(fb, -KA.q * fmaf(CA.s[i], cx, -CA.c[i] * sx), aJx);
                    aJy = fmaf(fb, -KA.q * fmaf(CA.s[i], cy, -CA.c[i] * sy), aJy);
                    ah = fmaf(fb, KA.p * sinp, ah);
                    tbo[i] = tbi;
                    vbo[i] = vbk;
                    fbo[i] = fb;
                }
                st4(tb + row + x, make_float4(tbo[0], tbo[1], tbo[2], tbo[3]));
                st4(vb + row + x, make_float4(vbo[0], vbo[1], vbo[2], vbo[3]));
                st4(FbO + row + x, make_float4(fbo[0], fbo[1], fbo[2], fbo[3]));
                PA = CA;
                CA = NA;
            } else {
                st4(tb + row + x, tb4);
            }
        }
    }
    // per-block FP64 accumulators in a fixed order (only phase A contributes)
    if (!DOA) return;
    const double ceta = cf.eta_d > 0.0 ? (double)KA.c / (2.0 * cf.eta_d) : 0.0;  // d c_k / d eta = c_k / (2 eta)
    double vals[kGacc] = {aJx, aJy, ah, abar, bbar, (double)cbar * ceta, eacc};
#pragma unroll
    for (int k = 0; k < kGacc; ++k) {
        const double w = warp_sum_a(vals[k]);
        if (lane == 0) s_red[k][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < kGacc) {
        double acc = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) acc += s_red[threadIdx.x][w2];
        R.gacc[(int64_t)(R.block_base + blockIdx.x) * kGacc + threadIdx.x] += acc;
    }
}

// R.doA / R.doB select the phases; split = true runs phase B and phase A as
// two launches (fewer registers each) instead of one fused launch.
cudaError_t launch_adjoint_strip(const DevCfg* d_cfg, const StripTask* tasks, int n_tasks, int H, uint64_t seed,
                                 RevArgs R, bool split, cudaStream_t st)
{
    if (n_tasks == 0) return cudaSuccess;
    const PhiloxKeys keys = philox_round_keys(seed);
    if (R.doA && R.doB && !split) {
        adjoint_strip_kernel<2, true, true><<<(unsigned)n_tasks, 256, 0, st>>>(d_cfg, tasks, H, R, keys);
        return cudaGetLastError();
    }
    if (R.doB) adjoint_strip_kernel<4, false, true><<<(unsigned)n_tasks, 256, 0, st>>>(d_cfg, tasks, H, R, keys);
    if (R.doA) adjoint_strip_kernel<2, true, false><<<(unsigned)n_tasks, 256, 0, st>>>(d_cfg, tasks, H, R, keys);
    return cudaGetLastError();
}

}  // namespace xy
