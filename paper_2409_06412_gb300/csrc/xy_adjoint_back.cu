// xy_adjoint_back.cu -- reverse sweep of the pathwise adjoint with the states
// of each checkpoint segment integrated backward in time inside the reverse
// kernel (App. A.1 run in reverse), instead of being recomputed forward and
// stored.
//
// The BBK step in leapfrog variables (theta_k, v_k = omega_{k-1/2}) with
// a = eta dt / 2 and g_k = (dt/2) F(theta_k) + c_k n_k,
//   omega_k = (v_k + g_k) / (1 + a),  v_{k+1} = (1 - a) omega_k + g_k,
//   theta_{k+1} = wrap(theta_k + dt v_{k+1}),
// is inverted site by site once the noise n_k is regenerated from its
// counter:
//   theta_k = wrap(theta_{k+1} - dt v_{k+1}),
//   omega_k = (v_{k+1} - g_k) / (1 - a),  v_k = (1 + a) omega_k - g_k,
// where g_k needs F(theta_k), i.e. the recovered angles of the four
// neighbours.  A launch for step k reads the state of step k + 1 and the
// adjoints of step k + 1, writes the state of step k and the adjoints of
// step k, and does the reverse of step k (phase A: site-local adjoint, phase
// B: Hessian stencil) exactly as the band reverse kernel of xy_adjoint.cu.
// Each segment starts from the exact checkpoint (or final state) at its end,
// so rounding of the inversion does not carry across segments.
//
// The |M_k| term of the objective needs sign(M_k), a sum over the whole
// lattice of the angles recovered in the same launch.  Its contribution
// w_M sign(M_k) sigma q cos(q theta_k) / N to the adjoint of theta_k enters
// nothing else of step k, so it is added by the next launch (step k - 1)
// when it reads that adjoint: every launch writes per-block partial sums of
// M_k into a two-slot ring, and the next one sums them in a fixed order,
// records M_k and applies the deferred term.
#include "xy_device.cuh"

namespace xy {

namespace {

constexpr unsigned kFullB = 0xFFFFFFFFu;
constexpr int kMaxBackWarps = 16;  // Lx <= 2048

__device__ __forceinline__ int wrapb(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void sc_b(float q, float th, float& s, float& c) { __sincosf(__fmul_rn(q, th), &s, &c); }

struct SCb {
    float s[4], c[4];
};

__device__ __forceinline__ void scb4(float q, const float4& t, SCb& r)
{
    sc_b(q, t.x, r.s[0], r.c[0]);
    sc_b(q, t.y, r.s[1], r.c[1]);
    sc_b(q, t.z, r.s[2], r.c[2]);
    sc_b(q, t.w, r.s[3], r.c[3]);
}

// theta_k = wrap(theta_{k+1} - dt v_{k+1}): the drift of step k undone, with
// one explicit rounding so that every block recovering a row gets its bits
__device__ __forceinline__ float4 undrift(const float4& t1, const float4& v1, float dt)
{
    return make_float4(wrap_angle(fmaf(-dt, v1.x, t1.x)), wrap_angle(fmaf(-dt, v1.y, t1.y)),
                       wrap_angle(fmaf(-dt, v1.z, t1.z)), wrap_angle(fmaf(-dt, v1.w, t1.w)));
}

__device__ __forceinline__ float warp_sumf_b(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullB, v, o);
    return v;
}

}  // namespace

// WIDE: Lx > 128 (a block spans one band of Lx / 128 strips); OBS: k > k0;
// BACK: the state of step k is recovered from that of step k + 1 (every
// launch but the first, which reads the final state itself); SCHED: some
// configuration of the launch has a field or coupling schedule (without one
// the step's constants are the configuration's own and no knot is searched).  At 128
// registers an SM partition holds four warps (16 per SM), enough for bands
// of 16 rows on 64 lattices of 256 x 256 to run in one wave.
template <bool WIDE, bool OBS, bool BACK, bool SCHED>
__global__ void __launch_bounds__(512, 1) adjoint_back_kernel(const DevCfg* cfgs, const BandTask* tasks, int H,
                                                              BackArgs R, PhiloxKeys keys)
{
    // per warp, two stages of [theta_in(t+1), v_in, tb(t), vb(t)] for its 32 lanes
    extern __shared__ float4 s_stage[];
    // edge slots of the wide bands, four rows deep: a slot last read in phase B
    // of row t + 1 is rewritten for row t + 4, in the phase A of a warp that has
    // passed the barrier of row t + 2, after every warp's phase B of row t + 1
    __shared__ float2 s_sc[4][kMaxBackWarps][2];
    __shared__ float s_fb[4][kMaxBackWarps][2];
    __shared__ float s_bx[4][kMaxBackWarps];  // bond cosine of a strip's last site to the next strip
    __shared__ double s_red[kGacc + 1][kMaxBackWarps];
    __shared__ float s_wm1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const BandTask task = tasks[blockIdx.x];
    const DevCfg& cf = cfgs[task.cfg];
    const int Lx = cf.Lx, Ly = cf.Ly;
    constexpr bool wide = WIDE;
    const int G = Lx >= 128 ? 32 : (Lx >> 2);
    const int groups = 32 / G;
    const int grp = lane / G, lg = lane - grp * G;
    const int per_block = wide ? 1 : n_warps * groups;  // bands per block
    const int band_raw = wide ? task.band0 : task.band0 + warp * groups + grp;
    // lane groups past the last band recompute the last band (so every shuffle
    // and barrier runs converged) and store nothing
    const bool active = band_raw < task.n_bands;
    const int band = active ? band_raw : task.n_bands - 1;
    const int x = (wide ? warp * 128 : 0) + 4 * lg;
    const int y0 = band * H;
    const int srcL = grp * G + (lg + G - 1) % G, srcR = grp * G + (lg + 1) % G;
    const int wl = (warp + n_warps - 1) % n_warps, wr = (warp + 1) % n_warps;  // neighbour strips (wide)
    const int64_t b = cf.b_first + task.rep;
    const int64_t lat_off = cf.offset + (int64_t)task.rep * cf.N;
    const int slot_j = task.band0 / per_block;  // this block's partial of M
    const int n_parts = (task.n_bands + per_block - 1) / per_block;
    const float* thI = R.th_in + lat_off;
    const float* vI = R.v_in + lat_off;
    float* thO = BACK ? R.th_out + lat_off : nullptr;
    float* vO = BACK ? R.v_out + lat_off : nullptr;
    const float* tbI = R.tb_in + lat_off;
    const float* vbI = R.vb_in + lat_off;
    float* tbO = R.tb_out + lat_off;
    float* vbO = R.vb_out + lat_off;
    const StepConst K = SCHED ? step_const_k(cf, R.k, noise_amp(cf, R.k)) : step_const(cf, noise_amp(cf, R.k));
    const float q2 = K.q * K.q, hp2 = K.hp * cf.p;
    const float invN = 1.0f / (float)cf.N, wE = R.wE;
    constexpr bool observe = OBS, first = !OBS;
    const uint32_t cfgrep = ((uint32_t)cf.noise_cfg << 16) | (uint32_t)(cf.rep0 + task.rep);
    // M_{k+1} from the previous launch's partials (fixed order), recorded by
    // the lattice's first block; its sign weights the deferred |M| term
    if (threadIdx.x == 0) {
        float w = 0.f;
        if (BACK) {
            const double* mp = R.mpart + (b * 2 + ((R.k + 1) & 1)) * R.P;
            double m = 0.0;
            for (int j = 0; j < n_parts; ++j) m += mp[j];
            m /= (double)cf.N;
            if (slot_j == 0) R.rec[b * R.rec_stride + (R.k + 1 - R.k0)].x = m;
            const float wq = R.wM * invN * K.q;
            w = m > 0.0 ? wq : (m < 0.0 ? -wq : 0.f);
        }
        s_wm1 = w;
    }
    // configuration constants in registers (the cp.async statements clobber
    // memory, which would otherwise reload them from the descriptor every row)
    const float2 Jk = SCHED ? couplings_at(cf, R.k) : make_float2(cf.Jx, cf.Jy);
    const float2 abk = SCHED ? coupling_scales(cf, R.k) : make_float2(1.f, 1.f);
    const float Jx = Jk.x, Jy = Jk.y, hF = SCHED ? field_h(cf, R.k) : cf.h;
    const float q2Jx = q2 * Jx, q2Jy = q2 * Jy;
    const bool stag = cf.stag != 0;
    const float wEn = wE * invN;
    const float inv_oma = 1.0f / K.oma, opa = 2.0f - K.oma;  // 1 / (1 - a), 1 + a
    float aJx = 0.f, aJy = 0.f, ah = 0.f, abar = 0.f, bbar = 0.f, cbar = 0.f;
    float sw2 = 0.f, sbx = 0.f, sby = 0.f, scp = 0.f, pm = 0.f;

    // window: S1 = row t-1, S2 = t, S3 = t+1 (of theta_k); F0 = F-bar(t-2), F1 = t-1;
    // Bm2, Bm1: bond cosines cos q(theta_y - theta_{y+1}) of rows t-2 and t-1,
    // formed in phase A and reused by the stencil of phase B
    SCb S1, S2, S3;
    float4 Bm2, Bm1;
    float4 Bx1 = make_float4(0.f, 0.f, 0.f, 0.f);  // cos q(theta_x - theta_{x+1}) of row t-1
    float4 F0 = make_float4(0.f, 0.f, 0.f, 0.f), F1 = F0;
    float4 th2, tbp1 = F0;  // theta_k of row t; tb partial of row t-1 (site-local terms of phase B folded in)
    float4 t1c = F0, v1c = F0;        // BACK: theta_{k+1}, v_{k+1} of row t
    const int Nl = Lx * Ly;
    auto rowp = [&](int y) { return wrapb(y, Ly) * Lx; };
    auto adv = [&](int r) { return r + Lx == Nl ? 0 : r + Lx; };
    int r_m1 = rowp(y0 - 2), r_0 = rowp(y0 - 1), r_p1 = rowp(y0), r_p2 = rowp(y0 + 1);
    // slot of row y: (y - y0 + 8) & 3 (the block's rows share y0 in the wide layout)
    int sl_0 = 3, sl_p1 = 0;
    auto publish_sc = [&](int slot, const SCb& S) {
        if (!wide) return;
        if (lane == 0) s_sc[slot][warp][0] = make_float2(S.s[0], S.c[0]);
        if (lane == 31) s_sc[slot][warp][1] = make_float2(S.s[3], S.c[3]);
    };
    auto nbr_sc = [&](int slot, const SCb& S, float& sL, float& cL, float& sR, float& cR) {
        sL = __shfl_sync(kFullB, S.s[3], srcL);
        cL = __shfl_sync(kFullB, S.c[3], srcL);
        sR = __shfl_sync(kFullB, S.s[0], srcR);
        cR = __shfl_sync(kFullB, S.c[0], srcR);
        if (wide) {
            if (lane == 0) { const float2 e = s_sc[slot][wl][1]; sL = e.x; cL = e.y; }
            if (lane == 31) { const float2 e = s_sc[slot][wr][0]; sR = e.x; cR = e.y; }
        }
    };
    constexpr int kStage = 4 * 32;  // float4 per warp and stage
    float4* my_stage = s_stage + (size_t)warp * 2 * kStage;
    // stage st: theta_in of row offset rt, v_in of row offset rvin (BACK: row
    // t + 1, else row t), tb and vb of row offset rv
    auto prefetch = [&](int st, int rt, int rvin, int rv) {
        float4* p = my_stage + st * kStage;
        cp_async16(p + 0 * 32 + lane, thI + rt + x);
        cp_async16(p + 1 * 32 + lane, vI + rvin + x);
        cp_async16(p + 2 * 32 + lane, tbI + rv + x);
        cp_async16(p + 3 * 32 + lane, vbI + rv + x);
        cp_async_commit();
    };
    if (BACK) {
        scb4(K.q, undrift(ld4(thI + r_m1 + x), ld4(vI + r_m1 + x), K.dt), S1);
        t1c = ld4(thI + r_0 + x);
        v1c = ld4(vI + r_0 + x);
        th2 = undrift(t1c, v1c, K.dt);
        prefetch(0, r_p1, r_p1, r_0);
    } else {
        scb4(K.q, ld4(thI + r_m1 + x), S1);
        th2 = ld4(thI + r_0 + x);
        prefetch(0, r_p1, r_0, r_0);
    }
    scb4(K.q, th2, S2);
    publish_sc(sl_0, S2);
    Bm1 = make_float4(fmaf(S1.c[0], S2.c[0], S1.s[0] * S2.s[0]), fmaf(S1.c[1], S2.c[1], S1.s[1] * S2.s[1]),
                      fmaf(S1.c[2], S2.c[2], S1.s[2] * S2.s[2]), fmaf(S1.c[3], S2.c[3], S1.s[3] * S2.s[3]));
    Bm2 = Bm1;
    __syncthreads();  // s_wm1, and the edge slots of the first rows
    const float wM1 = s_wm1;
    for (int t = y0 - 1; t <= y0 + H; ++t) {
        const bool own_a = active && t >= y0 && t < y0 + H;  // phase A results stored / accumulated
        const bool do_b = t - 1 >= y0;                      // phase B on row t-1
        const int st = (t - y0 + 1) & 1;
        const int yw = wrapb(t, Ly);
        if (BACK) prefetch(st ^ 1, r_p2, r_p2, r_p1);
        else prefetch(st ^ 1, r_p2, r_p1, r_p1);
        cp_async_wait<1>();  // this lane's copies of stage st have landed
        const float4* sp = my_stage + st * kStage;
        const float4 in3 = sp[0 * 32 + lane];
        const float4 vin = sp[1 * 32 + lane];
        float4 th3, v1n = vin;
        if (BACK) th3 = undrift(in3, vin, K.dt);
        else th3 = in3;
        scb4(K.q, th3, S3);
        publish_sc(sl_p1, S3);
        // ---------------- phase A on row t
        float4 Fn = make_float4(0.f, 0.f, 0.f, 0.f), tbpn = Fn, Bn = Fn, Bxn = Fn;
        {
            float4 tb4 = sp[2 * 32 + lane];
            const float4 vb4 = sp[3 * 32 + lane];
            if (BACK) {
                // deferred |M_{k+1}| term of the adjoint of theta_{k+1} (step
                // k + 1 > k0 is always observed); sites 0, 2 of a quad share
                // the staggered sign of (x + y), sites 1, 3 take the other
                const float wa = (stag && ((x + yw) & 1)) ? -wM1 : wM1;
                const float wb = stag ? -wa : wa;
                tb4.x = fmaf(wa, __cosf(K.q * t1c.x), tb4.x);
                tb4.y = fmaf(wb, __cosf(K.q * t1c.y), tb4.y);
                tb4.z = fmaf(wa, __cosf(K.q * t1c.z), tb4.z);
                tb4.w = fmaf(wb, __cosf(K.q * t1c.w), tb4.w);
            }
            float sL, cL, sR, cR;
            nbr_sc(sl_0, S2, sL, cL, sR, cR);
            const uint32_t quad = (uint32_t)((r_0 + x) >> 2);
            const float4 nz = gauss4_scaled(philox4x32_10_rk(noise_counter(quad, cfgrep, R.k, 0u), keys), K.c);
            float tbo[4], vbo[4], fbo[4], vko[4], byo[4], bxo[4];
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
                const float ax = fmaf(s_, cx, -c_ * sx), ay = fmaf(s_, cy, -c_ * sy);
                const float F = fmaf(K.nqJx, ax, fmaf(K.nqJy, ay, K.hp * sinp));
                const float cn = f4get(nz, i);
                const float g = fmaf(K.hdt, F, cn);
                float om, vk;  // omega_k, v_k
                if (BACK) {
                    om = (f4get(v1c, i) - g) * inv_oma;
                    vk = fmaf(opa, om, -g);
                } else {
                    vk = f4get(vin, i);
                    om = (vk + g) * K.inv1pa;
                }
                byo[i] = fmaf(c_, S3.c[i], s_ * S3.s[i]);  // bond to row t + 1
                bxo[i] = fmaf(c_, cr, s_ * sr);            // bond to column x + 1
                const float vbt = fmaf(K.dt, f4get(tb4, i), f4get(vb4, i));
                float omb = K.oma * vbt;
                float gb = vbt;
                float tbi = f4get(tb4, i);
                if (observe) {
                    omb = fmaf(wEn, om, omb);
                    tbi = fmaf(-wEn, F, tbi);
                    if (own_a) {
                        sw2 = fmaf(om, om, sw2);
                        sbx += bxo[i];
                        sby += byo[i];
                        scp += cp;
                    }
                }
                if (own_a) pm += (stag && ((x + i + yw) & 1)) ? -s_ : s_;
                float vbk = 0.f;
                if (!first) {
                    vbk = K.inv1pa * omb;
                    gb += vbk;
                    if (own_a) bbar = fmaf(vk + g, omb, bbar);
                }
                const float fb = K.hdt * gb;
                if (own_a) {
                    aJx = fmaf(fb, ax, aJx);
                    aJy = fmaf(fb, ay, aJy);
                    ah = fmaf(fb, sinp, ah);
                    abar = fmaf(-om, vbt, abar);
                    cbar = fmaf(gb, cn, cbar);
                }
                // the field's diagonal Hessian term of phase B, h p^2 cos(p t) F-bar, is site-local
                tbo[i] = fmaf(hp2 * cp, fb, tbi);
                vbo[i] = vbk;
                fbo[i] = fb;
                vko[i] = vk;
            }
            if (own_a) {
                st4(vbO + r_0 + x, make_float4(vbo[0], vbo[1], vbo[2], vbo[3]));
                if (BACK) {
                    st4(thO + r_0 + x, th2);
                    st4(vO + r_0 + x, make_float4(vko[0], vko[1], vko[2], vko[3]));
                }
            }
            Fn = make_float4(fbo[0], fbo[1], fbo[2], fbo[3]);
            Bn = make_float4(byo[0], byo[1], byo[2], byo[3]);
            Bxn = make_float4(bxo[0], bxo[1], bxo[2], bxo[3]);
            tbpn = make_float4(tbo[0], tbo[1], tbo[2], tbo[3]);
            if (wide) {
                if (lane == 0) s_fb[(t - y0 + 8) & 3][warp][0] = Fn.x;
                if (lane == 31) {
                    s_fb[(t - y0 + 8) & 3][warp][1] = Fn.w;
                    s_bx[(t - y0 + 8) & 3][warp] = Bxn.w;
                }
            }
        }
        if (wide) __syncthreads(); else __syncwarp();
        // ---------------- phase B on row t - 1 (needs F-bar of rows t - 2, t - 1, t)
        if (do_b) {
            float fL = __shfl_sync(kFullB, F1.w, srcL), fR = __shfl_sync(kFullB, F1.x, srcR);
            float kl0 = __shfl_sync(kFullB, Bx1.w, srcL);  // bond of the site to its left
            if (wide) {
                if (lane == 0) {
                    fL = s_fb[(t - 1 - y0 + 8) & 3][wl][1];
                    kl0 = s_bx[(t - 1 - y0 + 8) & 3][wl];
                }
                if (lane == 31) fR = s_fb[(t - 1 - y0 + 8) & 3][wr][0];
            }
            float out[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float fl = i == 0 ? fL : f4get(F1, i - 1), fr = i == 3 ? fR : f4get(F1, i + 1);
                const float fj = f4get(F1, i);
                const float kl = i == 0 ? kl0 : f4get(Bx1, i - 1), kr = f4get(Bx1, i);
                const float ku = f4get(Bm2, i), kd = f4get(Bm1, i);
                const float hx = fmaf(kl, fl - fj, kr * (fr - fj));
                const float hy = fmaf(ku, f4get(F0, i) - fj, kd * (f4get(Fn, i) - fj));
                out[i] = f4get(tbp1, i) + fmaf(q2Jx, hx, q2Jy * hy);
            }
            if (active) st4(tbO + r_m1 + x, make_float4(out[0], out[1], out[2], out[3]));
        }
        // shift the windows
        Bm2 = Bm1;
        Bm1 = Bn;
        Bx1 = Bxn;
        S1 = S2;
        S2 = S3;
        th2 = th3;
        t1c = in3;
        v1c = v1n;
        F0 = F1;
        F1 = Fn;
        tbp1 = tbpn;
        r_m1 = r_0;
        r_0 = r_p1;
        r_p1 = r_p2;
        r_p2 = adv(r_p2);
        sl_0 = sl_p1;
        sl_p1 = (sl_p1 + 1) & 3;
    }
    // per-block accumulators: FP32 warp butterflies, the warps and the steps
    // combined in FP64 in a fixed order; the partial of M_k goes to the ring
    const float vals[kGacc + 1] = {
        fmaf(-K.q, aJx, -wEn * sbx) * abk.x,                                // d/d J_par (J_par(k) = J_par a(k))
        fmaf(-K.q, aJy, -wEn * sby) * abk.y,                                // d/d J_perp (J_perp b(k))
        fmaf(K.p, ah, wEn * scp) * (SCHED ? field_scale(cf, R.k) : 1.f),    // d/d h (h_k = h s(k))
        abar, bbar, cbar,
        wEn * fmaf(0.5f, sw2, fmaf(-Jx, sbx, fmaf(-Jy, sby, hF * scp))),  // w_E E / N
        pm,                                                                 // sum of sigma sin(q theta_k)
    };
#pragma unroll
    for (int k = 0; k < kGacc + 1; ++k) {
        const float w = warp_sumf_b(vals[k]);
        if (lane == 0) s_red[k][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < kGacc + 1) {
        double acc = 0.0;
        for (int w2 = 0; w2 < n_warps; ++w2) acc += s_red[threadIdx.x][w2];
        if (threadIdx.x == kGacc) {
            R.mpart[(b * 2 + (R.k & 1)) * R.P + slot_j] = acc;
        } else {
            // c-bar (summed against c_k n_k) enters the eta gradient through
            // d c_k / d eta = c_k / (2 eta)
            if (threadIdx.x == 5) acc *= cf.eta_d > 0.0 ? 1.0 / (2.0 * cf.eta_d) : 0.0;
            R.gacc[(int64_t)(R.block_base + blockIdx.x) * kGacc + threadIdx.x] += acc;
        }
    }
}

cudaError_t launch_adjoint_back(const DevCfg* d_cfg, const BandTask* tasks, int n_tasks, int Lx, int H, uint64_t seed,
                                bool back, BackArgs R, cudaStream_t st)
{
    if (n_tasks == 0) return cudaSuccess;
    const bool wide = Lx > 128;
    const int threads = wide ? (Lx / 128) * 32 : 256;
    const int smem = (threads / 32) * 2 * 4 * 32 * (int)sizeof(float4);
    const bool obs = R.k > R.k0;
    using Kern = void (*)(const DevCfg*, const BandTask*, int, BackArgs, PhiloxKeys);
    static const Kern table[2][2][2][2] = {
        {{{adjoint_back_kernel<false, false, false, false>, adjoint_back_kernel<false, false, true, false>},
          {adjoint_back_kernel<false, true, false, false>, adjoint_back_kernel<false, true, true, false>}},
         {{adjoint_back_kernel<true, false, false, false>, adjoint_back_kernel<true, false, true, false>},
          {adjoint_back_kernel<true, true, false, false>, adjoint_back_kernel<true, true, true, false>}}},
        {{{adjoint_back_kernel<false, false, false, true>, adjoint_back_kernel<false, false, true, true>},
          {adjoint_back_kernel<false, true, false, true>, adjoint_back_kernel<false, true, true, true>}},
         {{adjoint_back_kernel<true, false, false, true>, adjoint_back_kernel<true, false, true, true>},
          {adjoint_back_kernel<true, true, false, true>, adjoint_back_kernel<true, true, true, true>}}},
    };
    const Kern kern = table[R.sched != 0][wide][obs][back];
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)n_tasks, threads, smem, st>>>(d_cfg, tasks, H, R, philox_round_keys(seed));
    return cudaGetLastError();
}

}  // namespace xy
