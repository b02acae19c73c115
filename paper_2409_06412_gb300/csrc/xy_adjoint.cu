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

__device__ __forceinline__ float warp_sumf_a(float v)
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
    const StepConst K = step_const_k(cf, k, s_c);
    const float hk = field_h(cf, k);
    const float2 Jk = couplings_at(cf, k), abk = coupling_scales(cf, k);
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
                e = fmaf(-Jk.x, bx, e);
                e = fmaf(-Jk.y, by, e);
                e = fmaf(hk, cp, e);
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
    // with schedules the field of step k is h s(k) and the couplings J a(k),
    // J b(k): d/dh and d/dJ of their terms carry s(k), a(k), b(k)
    double vals[kGacc] = {(double)aJx * abk.x, (double)aJy * abk.y, (double)ah * field_scale(cf, k), abar, bbar,
                          (double)cbar * ceta, eacc};
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
    const float2 Jk = couplings_at(cf, A.k);
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
        float acc = q2 * fmaf(Jk.x, hx, Jk.y * hy);
        acc = fmaf(field_hp(cf, A.k) * cf.p, __cosf(__fmul_rn(cf.p, t.t[i])) * fj, acc);
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
// Reverse step on row bands: phase A and phase B of the SAME step in one
// launch.  A thread block owns a band of H rows over the full width of one
// lattice (Lx / 128 warps side by side, each a 128-column strip), or, when
// Lx <= 128, each group of Lx / 4 lanes owns a band of its own.  Row t:
// phase A on row t (F-bar, the site-local adjoint, v-bar), then phase B on
// row t - 1 (the Hessian stencil, which needs F-bar of rows t - 2 .. t).
// F-bar and (sin q t, cos q t) live in register windows; the strips of a row
// exchange their edge columns through shared memory, one barrier per row.
// Phase A also runs on the halo rows y0 - 1 and y0 + H (its F-bar feeds the
// band's edge rows) without storing anything there, so the adjoint state is
// read from one buffer pair and written to another.
// ===========================================================================
namespace {

constexpr int kMaxBandWarps = 16;  // Lx <= 2048



struct BandSC {
    float s[4], c[4];
};

__device__ __forceinline__ void band_sc(float q, const float4& t, BandSC& r)
{
    sc_q(q, t.x, r.s[0], r.c[0]);
    sc_q(q, t.y, r.s[1], r.c[1]);
    sc_q(q, t.z, r.s[2], r.c[2]);
    sc_q(q, t.w, r.s[3], r.c[3]);
}

}  // namespace

// WIDE: Lx > 128 (a block spans one band of Lx / 128 strips); OBS: k > k0
// (the step is observed; k = k0 holds omega_{k0} fixed instead).
// NZ: regenerate the noise n_k from the counter-based stream.  Without it the
// step's noise term comes from the stored half-step velocities: in the BBK
// leapfrog omega_k = (v_k + v_{k+1}) / 2 exactly, g_k = v_{k+1} - (1 - a)
// omega_k and c_k n_k = g_k - (dt/2) F_k, which costs one more row read and
// saves the Philox rounds and the Box-Muller transform of every site.
template <bool WIDE, bool OBS, bool NZ>
__global__ void __launch_bounds__(512, 1) adjoint_band_kernel(const DevCfg* cfgs, const BandTask* tasks, int H,
                                                              BandArgs R, PhiloxKeys keys)
{
    // per warp, two stages of [theta(t+1), v(t), tb(t), vb(t), v_{k+1}(t)] for its 32 lanes
    extern __shared__ float4 s_stage[];
    // edge exchange: [slot][warp][side]  side 0 = left edge (site x0), 1 = right edge (site x0 + 127)
    // edge slots of the wide bands, four rows deep: a slot last read in phase B
    // of row t + 1 is rewritten for row t + 4, in the phase A of a warp that has
    // passed the barrier of row t + 2, after every warp's phase B of row t + 1
    __shared__ float2 s_sc[4][kMaxBandWarps][2];
    __shared__ float s_fb[4][kMaxBandWarps][2];
    __shared__ double s_red[kGacc][kMaxBandWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const BandTask task = tasks[blockIdx.x];
    const DevCfg& cf = cfgs[task.cfg];
    const int Lx = cf.Lx, Ly = cf.Ly;
    constexpr bool wide = WIDE;
    const int G = Lx >= 128 ? 32 : (Lx >> 2);
    const int groups = 32 / G;
    const int grp = lane / G, lg = lane - grp * G;
    const int band_raw = wide ? task.band0 : task.band0 + warp * groups + grp;
    // lane groups past the last band recompute the last band (so every shuffle
    // and barrier runs converged) and store nothing
    const bool active = band_raw < task.n_bands;
    const int band = active ? band_raw : task.n_bands - 1;
    const int x = (wide ? warp * 128 : 0) + 4 * lg;
    const int y0 = band * H;
    const int srcL = grp * G + (lg + G - 1) % G, srcR = grp * G + (lg + 1) % G;
    const int wl = (warp + n_warps - 1) % n_warps, wr = (warp + 1) % n_warps;  // neighbour strips (wide)
    const int64_t lat_off = cf.offset + (int64_t)task.rep * cf.N;
    const float* th = R.theta + lat_off;
    const float* vv = R.omega + lat_off;
    const float* tbI = R.tb_in + lat_off;
    const float* vbI = R.vb_in + lat_off;
    float* tbO = R.tb_out + lat_off;
    float* vbO = R.vb_out + lat_off;
    const StepConst K = step_const_k(cf, R.k, noise_amp(cf, R.k));
    const float q2 = __fmul_rn(K.q, K.q), hp2 = __fmul_rn(K.hp, cf.p);
    const float invN = 1.0f / (float)cf.N, wE = R.wE, wM = R.wM;
    constexpr bool observe = OBS, first = !OBS;
    const uint32_t cfgrep = ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + task.rep);
    float sgnM = 0.f;
    if (observe && R.wM != 0.f) {
        const double M = R.rec[(int64_t)(cf.b_first + task.rep) * R.rec_stride + (R.k - R.k0)].x;
        sgnM = M > 0.0 ? 1.f : (M < 0.0 ? -1.f : 0.f);
    }
    // configuration constants in registers (the cp.async statements clobber
    // memory, which would otherwise reload them from the descriptor every row)
    const float2 Jk = couplings_at(cf, R.k), abk = coupling_scales(cf, R.k);
    const float Jx = Jk.x, Jy = Jk.y, hF = field_h(cf, R.k);
    const float q2Jx = q2 * Jx, q2Jy = q2 * Jy;
    const bool stag = cf.stag != 0;
    const float wEn = wE * invN, wMs = wM * invN * sgnM * K.q;
    // per-thread sums of the step: F-bar against dF/dJ_par = -q a_x,
    // dF/dJ_perp = -q a_y, dF/dh = p sin(p t) (the factors -q, p applied at
    // the end); a-bar, b-bar, c-bar; and the observed site terms omega^2, the
    // bonds cos q(t - t_{x+1}), cos q(t - t_{y+1}) and cos(p t), from which
    // the energy and its parameter derivatives are formed at the end
    float aJx = 0.f, aJy = 0.f, ah = 0.f, abar = 0.f, bbar = 0.f, cbar = 0.f;
    float sw2 = 0.f, sbx = 0.f, sby = 0.f, scp = 0.f;

    // window: S0 = row t-2, S1 = t-1, S2 = t, S3 = t+1; F0 = F-bar(t-2), F1 = t-1
    BandSC S0, S1, S2, S3;
    float4 F0 = make_float4(0.f, 0.f, 0.f, 0.f), F1 = F0;
    float4 th2, tbp1 = F0, cp1 = F0;  // raw theta of row t; tb partial and cos(p theta) of row t-1
    // row offsets of rows t - 1, t, t + 1, t + 2 (advanced by Lx per row, periodic)
    const int Nl = Lx * Ly;
    auto rowp = [&](int y) { return wrapa(y, Ly) * Lx; };
    auto adv = [&](int r) { return r + Lx == Nl ? 0 : r + Lx; };
    int r_m1 = rowp(y0 - 2), r_0 = rowp(y0 - 1), r_p1 = rowp(y0), r_p2 = rowp(y0 + 1);
    // slots of the edge exchange: rows t - 1, t, t + 1 modulo 3
    // slot of row y: (y - y0 + 8) & 3 (the block's rows share y0 in the wide layout)
    int sl_m1 = 2, sl_0 = 3, sl_p1 = 0;
    auto publish_sc = [&](int slot, const BandSC& S) {
        if (!wide) return;
        if (lane == 0) s_sc[slot][warp][0] = make_float2(S.s[0], S.c[0]);
        if (lane == 31) s_sc[slot][warp][1] = make_float2(S.s[3], S.c[3]);
    };
    // x neighbours of the quad's outer sites for one row of (s, c)
    auto nbr_sc = [&](int slot, const BandSC& S, float& sL, float& cL, float& sR, float& cR) {
        sL = __shfl_sync(kFullA, S.s[3], srcL);
        cL = __shfl_sync(kFullA, S.c[3], srcL);
        sR = __shfl_sync(kFullA, S.s[0], srcR);
        cR = __shfl_sync(kFullA, S.c[0], srcR);
        if (wide) {
            if (lane == 0) { const float2 e = s_sc[slot][wl][1]; sL = e.x; cL = e.y; }
            if (lane == 31) { const float2 e = s_sc[slot][wr][0]; sR = e.x; cR = e.y; }
        }
    };
    constexpr int kStage = (NZ ? 4 : 5) * 32;  // float4 per warp and stage
    const float* vN = NZ ? nullptr : R.vnext + lat_off;
    float4* my_stage = s_stage + (size_t)warp * 2 * kStage;
    // theta of row offset rt and v, tb, vb (v_{k+1}) of row offset rv into stage st
    auto prefetch = [&](int st, int rt, int rv) {
        float4* p = my_stage + st * kStage;
        cp_async16(p + 0 * 32 + lane, th + rt + x);
        cp_async16(p + 1 * 32 + lane, vv + rv + x);
        cp_async16(p + 2 * 32 + lane, tbI + rv + x);
        cp_async16(p + 3 * 32 + lane, vbI + rv + x);
        if (!NZ) cp_async16(p + 4 * 32 + lane, vN + rv + x);
        cp_async_commit();
    };
    band_sc(K.q, ld4(th + r_m1 + x), S1);
    th2 = ld4(th + r_0 + x);
    band_sc(K.q, th2, S2);
    publish_sc(sl_0, S2);
    prefetch(0, r_p1, r_0);
    if (wide) __syncthreads(); else __syncwarp();
    for (int t = y0 - 1; t <= y0 + H; ++t) {
        const bool own_a = active && t >= y0 && t < y0 + H;  // phase A results stored / accumulated
        const bool do_b = t - 1 >= y0;                      // phase B on row t-1
        const int st = (t - y0 + 1) & 1;
        prefetch(st ^ 1, r_p2, r_p1);
        cp_async_wait<1>();  // this lane's copies of stage st have landed
        const float4* sp = my_stage + st * kStage;
        const float4 th3 = sp[0 * 32 + lane];
        band_sc(K.q, th3, S3);
        publish_sc(sl_p1, S3);
        // ---------------- phase A on row t
        float4 Fn = make_float4(0.f, 0.f, 0.f, 0.f), tbpn = Fn, cpn = Fn;
        {
            const float4 v = sp[1 * 32 + lane];
            const float4 tb4 = sp[2 * 32 + lane];
            const float4 vb4 = sp[3 * 32 + lane];
            float sL, cL, sR, cR;
            nbr_sc(sl_0, S2, sL, cL, sR, cR);
            float4 nz, v1;
            if (NZ) {
                const uint32_t quad = (uint32_t)((r_0 + x) >> 2);
                nz = gauss4_scaled(philox4x32_10_rk(noise_counter(quad, cfgrep, R.k, 0u), keys), K.c);
            } else {
                v1 = sp[4 * 32 + lane];
            }
            float tbo[4], vbo[4], fbo[4], cpo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float s_ = S2.s[i], c_ = S2.c[i];
                const float sl = i == 0 ? sL : S2.s[i - 1], cl = i == 0 ? cL : S2.c[i - 1];
                const float sr = i == 3 ? sR : S2.s[i + 1], cr = i == 3 ? cR : S2.c[i + 1];
                const float sx = sl + sr, cx = cl + cr;
                const float sy = S1.s[i] + S3.s[i], cy = S1.c[i] + S3.c[i];
                const float tht = f4get(th2, i);
                const float sinp = __sinf(K.p * tht);
                const float cp = __cosf(K.p * tht);
                // F = -q J_par a_x - q J_perp a_y + h p sin(p t)
                const float ax = fmaf(s_, cx, -c_ * sx), ay = fmaf(s_, cy, -c_ * sy);
                const float F = fmaf(K.nqJx, ax, fmaf(K.nqJy, ay, K.hp * sinp));
                float cn, g, om;  // c_k n_k, g_k, omega_k
                if (NZ) {
                    cn = f4get(nz, i);
                    g = fmaf(K.hdt, F, cn);
                    om = (f4get(v, i) + g) * K.inv1pa;
                } else {
                    om = 0.5f * (f4get(v, i) + f4get(v1, i));
                    g = f4get(v1, i) - K.oma * om;
                    cn = g - K.hdt * F;
                }
                const float vbt = fmaf(K.dt, f4get(tb4, i), f4get(vb4, i));
                float omb = K.oma * vbt;
                float gb = vbt;
                float tbi = f4get(tb4, i);
                if (observe) {
                    omb = fmaf(wEn, om, omb);
                    tbi = fmaf(-wEn, F, tbi);
                    const float sigma = (stag && ((x + i + t) & 1)) ? -wMs : wMs;
                    tbi = fmaf(sigma, c_, tbi);
                    if (own_a) {
                        sw2 = fmaf(om, om, sw2);
                        sbx += fmaf(c_, cr, s_ * sr);
                        sby += fmaf(c_, S3.c[i], s_ * S3.s[i]);
                        scp += cp;
                    }
                }
                float vbk = 0.f;
                if (!first) {
                    vbk = K.inv1pa * omb;
                    gb += vbk;
                    if (own_a) bbar = fmaf(f4get(v, i) + g, omb, bbar);
                }
                const float fb = K.hdt * gb;
                if (own_a) {
                    aJx = fmaf(fb, ax, aJx);
                    aJy = fmaf(fb, ay, aJy);
                    ah = fmaf(fb, sinp, ah);
                    abar = fmaf(-om, vbt, abar);
                    cbar = fmaf(gb, cn, cbar);
                }
                tbo[i] = tbi;
                vbo[i] = vbk;
                fbo[i] = fb;
                cpo[i] = cp;
            }
            if (own_a) st4(vbO + r_0 + x, make_float4(vbo[0], vbo[1], vbo[2], vbo[3]));
            Fn = make_float4(fbo[0], fbo[1], fbo[2], fbo[3]);
            tbpn = make_float4(tbo[0], tbo[1], tbo[2], tbo[3]);
            cpn = make_float4(cpo[0], cpo[1], cpo[2], cpo[3]);
            if (wide) {
                if (lane == 0) s_fb[(t - y0 + 8) & 3][warp][0] = Fn.x;
                if (lane == 31) s_fb[(t - y0 + 8) & 3][warp][1] = Fn.w;
            }
        }
        if (wide) __syncthreads(); else __syncwarp();
        // ---------------- phase B on row t - 1 (needs F-bar of rows t - 2, t - 1, t)
        if (do_b) {
            float sL, cL, sR, cR;
            nbr_sc(sl_m1, S1, sL, cL, sR, cR);
            float fL = __shfl_sync(kFullA, F1.w, srcL), fR = __shfl_sync(kFullA, F1.x, srcR);
            if (wide) {
                if (lane == 0) fL = s_fb[(t - 1 - y0 + 8) & 3][wl][1];
                if (lane == 31) fR = s_fb[(t - 1 - y0 + 8) & 3][wr][0];
            }
            float out[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float sl = i == 0 ? sL : S1.s[i - 1], cl = i == 0 ? cL : S1.c[i - 1];
                const float sr = i == 3 ? sR : S1.s[i + 1], cr = i == 3 ? cR : S1.c[i + 1];
                const float fl = i == 0 ? fL : f4get(F1, i - 1), fr = i == 3 ? fR : f4get(F1, i + 1);
                const float fj = f4get(F1, i);
                const float kl = fmaf(S1.c[i], cl, S1.s[i] * sl), kr = fmaf(S1.c[i], cr, S1.s[i] * sr);
                const float ku = fmaf(S1.c[i], S0.c[i], S1.s[i] * S0.s[i]);
                const float kd = fmaf(S1.c[i], S2.c[i], S1.s[i] * S2.s[i]);
                const float hx = fmaf(kl, fl - fj, kr * (fr - fj));
                const float hy = fmaf(ku, f4get(F0, i) - fj, kd * (f4get(Fn, i) - fj));
                float acc = fmaf(q2Jx, hx, q2Jy * hy);
                acc = fmaf(hp2, f4get(cp1, i) * fj, acc);
                out[i] = f4get(tbp1, i) + acc;
            }
            if (active) st4(tbO + r_m1 + x, make_float4(out[0], out[1], out[2], out[3]));
        }
        // shift the windows
        S0 = S1;
        S1 = S2;
        S2 = S3;
        th2 = th3;
        F0 = F1;
        F1 = Fn;
        tbp1 = tbpn;
        cp1 = cpn;
        r_m1 = r_0;
        r_0 = r_p1;
        r_p1 = r_p2;
        r_p2 = adv(r_p2);
        sl_m1 = sl_0;
        sl_0 = sl_p1;
        sl_p1 = (sl_p1 + 1) & 3;
    }
    // per-block accumulators: FP32 warp butterflies (a warp covers a few
    // thousand sites), the warps and the steps combined in FP64 in a fixed order
    const float vals[kGacc] = {
        fmaf(-K.q, aJx, -wEn * sbx) * abk.x,                                // d/d J_par (J_par(k) = J_par a(k))
        fmaf(-K.q, aJy, -wEn * sby) * abk.y,                                // d/d J_perp (J_perp b(k))
        fmaf(K.p, ah, wEn * scp) * field_scale(cf, R.k),                    // d/d h (h_k = h s(k))
        abar, bbar, cbar,
        wEn * fmaf(0.5f, sw2, fmaf(-Jx, sbx, fmaf(-Jy, sby, hF * scp))),  // w_E E / N
    };
#pragma unroll
    for (int k = 0; k < kGacc; ++k) {
        const float w = warp_sumf_a(vals[k]);
        if (lane == 0) s_red[k][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < kGacc) {
        double acc = 0.0;
        for (int w2 = 0; w2 < n_warps; ++w2) acc += s_red[threadIdx.x][w2];
        // c-bar (summed against c_k n_k) enters the eta gradient through
        // d c_k / d eta = c_k / (2 eta)
        if (threadIdx.x == 5) acc *= cf.eta_d > 0.0 ? 1.0 / (2.0 * cf.eta_d) : 0.0;
        R.gacc[(int64_t)(R.block_base + blockIdx.x) * kGacc + threadIdx.x] += acc;
    }
}

// ===========================================================================
// Order parameter of every state of a recomputed segment:
//   M_k = (1/N) sum_i sigma_i sin(q theta_i)   (sigma_i = (-1)^(x+y) when
// staggered, else 1), the quantity whose sign the |M| term of the objective
// differentiates.  Block (b, i) reduces lattice b of segment slot i: FP32 over
// runs of 16 quads per thread, FP64 across runs and threads, in a fixed order.
// ===========================================================================
__global__ void __launch_bounds__(256) segment_m_kernel(const DevCfg* cfgs, int n_cfg, const float* seg, int64_t T,
                                                        double2* rec, int64_t rec_stride, int64_t r0)
{
    const int b = blockIdx.x;
    const int i = blockIdx.y;
    int c = 0;
    while (c + 1 < n_cfg && b >= cfgs[c + 1].b_first) ++c;
    const DevCfg& cf = cfgs[c];
    const int rep = b - cf.b_first;
    const int Lx = cf.Lx;
    const int64_t nq = cf.N / 4;
    const float q = cf.q;
    const bool stag = cf.stag != 0;
    const float* th = seg + 2 * T * (int64_t)i + cf.offset + (int64_t)rep * cf.N;
    double acc = 0.0;
    float run = 0.f;
    int in_run = 0;
    for (int64_t u = threadIdx.x; u < nq; u += blockDim.x) {
        const float4 t = ld4(th + 4 * u);
        const float s0 = __sinf(__fmul_rn(q, t.x)), s1 = __sinf(__fmul_rn(q, t.y));
        const float s2 = __sinf(__fmul_rn(q, t.z)), s3 = __sinf(__fmul_rn(q, t.w));
        const float ev = s0 + s2, od = s1 + s3;  // x is a multiple of 4: sites 0, 2 share the parity of y
        const int y = (int)(4 * u / Lx);
        run += !stag ? ev + od : ((y & 1) ? od - ev : ev - od);
        if (++in_run == 16) {
            acc += run;
            run = 0.f;
            in_run = 0;
        }
    }
    acc += run;
    __shared__ double s_acc[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    acc = warp_sum_a(acc);
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m += s_acc[w];
        rec[(int64_t)b * rec_stride + r0 + i] = make_double2(m / (double)cf.N, 0.0);
    }
}

cudaError_t launch_segment_m(const DevCfg* d_cfg, int n_cfg, int64_t B, const float* seg, int64_t T, int n_states,
                             double2* rec, int64_t rec_stride, int64_t r0, cudaStream_t st)
{
    if (B == 0 || n_states == 0) return cudaSuccess;
    for (int i0 = 0; i0 < n_states; i0 += 65535) {  // grid.y limit
        const int n = n_states - i0 < 65535 ? n_states - i0 : 65535;
        segment_m_kernel<<<dim3((unsigned)B, (unsigned)n), 256, 0, st>>>(d_cfg, n_cfg, seg + 2 * T * (int64_t)i0, T, rec,
                                                                         rec_stride, r0 + i0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_adjoint_band(const DevCfg* d_cfg, const BandTask* tasks, int n_tasks, int Lx, int H, uint64_t seed,
                                BandArgs R, cudaStream_t st)
{
    if (n_tasks == 0) return cudaSuccess;
    const bool wide = Lx > 128;
    const int threads = wide ? (Lx / 128) * 32 : 256;
    const bool nz = R.vnext == nullptr;
    const int smem = (threads / 32) * 2 * (nz ? 4 : 5) * 32 * (int)sizeof(float4);
    const bool obs = R.k > R.k0;
    using Kern = void (*)(const DevCfg*, const BandTask*, int, BandArgs, PhiloxKeys);
    static const Kern table[2][2][2] = {
        {{adjoint_band_kernel<false, false, false>, adjoint_band_kernel<false, false, true>},
         {adjoint_band_kernel<false, true, false>, adjoint_band_kernel<false, true, true>}},
        {{adjoint_band_kernel<true, false, false>, adjoint_band_kernel<true, false, true>},
         {adjoint_band_kernel<true, true, false>, adjoint_band_kernel<true, true, true>}},
    };
    const Kern kern = table[wide][obs][nz];
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)n_tasks, threads, smem, st>>>(d_cfg, tasks, H, R, philox_round_keys(seed));
    return cudaGetLastError();
}

}  // namespace xy
