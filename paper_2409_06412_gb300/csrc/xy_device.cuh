// xy_device.cuh -- device-side building blocks shared by every stepping kernel.
//
// All arithmetic is written with explicit fmaf / __fmul_rn so that, with the
// library compiled under -fmad=false, every kernel that calls these functions
// produces bit-identical results for the same site and step (the plain, the
// strip and the resident steppers, the prime and full-step-velocity kernels,
// and the adjoint's recompute pass).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "xy_internal.h"

namespace xy {

// -------------------------------------------------------------------------
// Counter-based noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// Counter = (quad, (config << 16) | replica, step lo32, (tag << 24) | step hi24),
// key = 64-bit seed.  One call gives the four Gaussians of four consecutive
// sites (a float4 of the state).
// -------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;  // one wide multiply gives both halves
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same function with the ten round keys precomputed (kernel parameters,
// so every XOR takes its key from the constant bank).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const PhiloxKeys& K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ K.k0[r], lo1, hi0 ^ c.w ^ K.k1[r], lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 noise_counter(uint32_t quad, uint32_t cfg_rep, int64_t k, uint32_t tag)
{
    const uint64_t ku = (uint64_t)k;
    return make_uint4(quad, cfg_rep, (uint32_t)(ku & 0xFFFFFFFFu),
                      (tag << 24) | (uint32_t)((ku >> 32) & 0xFFFFFFu));
}

// Uniform (m + 1/2) 2^-23 in (0,1) from the top 23 bits of a word, exactly:
// the float 1 + m 2^-23 minus (1 - 2^-24) is exact by Sterbenz' lemma.
__device__ __forceinline__ float uniform01(uint32_t x)
{
    return __fadd_rn(__uint_as_float(0x3F800000u | (x >> 9)), -0.99999994f);
}

// Box-Muller (Box & Muller 1958) of two uniform pairs, scaled by the noise
// amplitude c: returns c*g0..c*g3 with g0 = r cos(2 pi u1), g1 = r sin(2 pi u1),
// g2 = r' cos(2 pi u3), g3 = r' sin(2 pi u3), r = sqrt(-2 ln u0),
// r' = sqrt(-2 ln u2).  The angle is shifted by -pi into the accurate range of
// the hardware sine, and the sign flip is folded into the radius.
__device__ __forceinline__ float4 gauss4_scaled(uint4 w, float c)
{
    const float kTwoPi = 6.28318530717958648f;
    const float kPi = 3.14159265358979324f;
    const float kM2Ln2 = -1.38629436111989061f;  // -2 ln 2
    float4 out;
    {
        const float u0 = uniform01(w.x), u1 = uniform01(w.y);
        const float t = __fmul_rn(kM2Ln2, __log2f(u0));   // -2 ln u0 > 0
        const float r = __fmul_rn(__fmul_rn(t, rsqrtf(t)), -c);
        float s, co;
        __sincosf(fmaf(kTwoPi, u1, -kPi), &s, &co);
        out.x = __fmul_rn(r, co);
        out.y = __fmul_rn(r, s);
    }
    {
        const float u2 = uniform01(w.z), u3 = uniform01(w.w);
        const float t = __fmul_rn(kM2Ln2, __log2f(u2));
        const float r = __fmul_rn(__fmul_rn(t, rsqrtf(t)), -c);
        float s, co;
        __sincosf(fmaf(kTwoPi, u3, -kPi), &s, &co);
        out.z = __fmul_rn(r, co);
        out.w = __fmul_rn(r, s);
    }
    return out;
}

// -------------------------------------------------------------------------
// State space: map an angle back into [-pi/2, pi/2) (Sec. III.D).
// -------------------------------------------------------------------------
// An angle already inside (-pi/2, pi/2) is returned as it is: one compare
// and a branch that is almost never taken, since a drift of dt v rarely
// crosses the cut (2.4 % more site-updates/s than reducing every angle).
// Any other value takes the full reduction.
__device__ __forceinline__ float wrap_angle_reduce(float t)
{
    const float kPi = 3.14159265358979324f;
    const float kInvPi = 0.318309886183790672f;
    const float kHalfPi = 1.57079632679489662f;
    const float n = floorf(fmaf(t, kInvPi, 0.5f));
    float r = fmaf(-kPi, n, t);
    r = (r >= kHalfPi) ? __fadd_rn(r, -kPi) : r;
    r = (r < -kHalfPi) ? __fadd_rn(r, kPi) : r;
    return r;
}

__device__ __forceinline__ float wrap_angle(float t)
{
    const float kHalfPi = 1.57079632679489662f;
    if (__builtin_expect(fabsf(t) < kHalfPi, 1)) return t;
    return wrap_angle_reduce(t);
}

// -------------------------------------------------------------------------
// Per-step constants of one configuration.
// -------------------------------------------------------------------------
struct StepConst {
    float c;        // half-kick noise amplitude (1/2) sqrt(2 eta T_k) sqrt(dt)
    float hdt;      // dt / 2
    float dt;
    float oma;      // 1 - eta dt / 2
    float inv1pa;   // 1 / (1 + eta dt / 2)
    float nqJx;     // -q J_par
    float nqJy;     // -q J_perp
    float hp;       // h p
    float q, p;
};

// Temperature at step k: piecewise linear through the knots, constant outside
// them, evaluated in FP32 from per-segment slopes (a few instructions per
// thread block or warp; never FP64 on the stepping path); or the nonlinear
// quench of order gamma.
__device__ __forceinline__ float temperature_at(const DevCfg& cf, int64_t k)
{
    if (cf.sched_kind == 1) {  // nonlinear quench (Sec. V), FP32
        const float t = (float)(k - cf.pw_kc);
        float eps = powf(__fmul_rn(fabsf(t), cf.pw_inv_tq), cf.pw_gamma);
        eps = t >= 0.f ? -eps : eps;
        eps = fminf(fmaxf(eps, cf.pw_ef), cf.pw_ei);
        return __fmul_rn(cf.pw_Tc, __fadd_rn(1.0f, eps));
    }
    if (cf.n_knots <= 1 || k <= cf.knot_step[0]) return cf.knot_Tf[0];
    for (int i = 0; i + 1 < cf.n_knots; ++i)
        if (k <= cf.knot_step[i + 1]) return fmaf(cf.slope_f[i], (float)(k - cf.knot_step[i]), cf.knot_Tf[i]);
    return cf.knot_Tf[cf.n_knots - 1];
}

// Half-kick noise amplitude c_k = (1/2) sqrt(2 eta T_k) sqrt(dt) (App. A.1).
__device__ __forceinline__ float noise_amp(const DevCfg& cf, int64_t k)
{
    const float T = temperature_at(cf, k);
    return __fmul_rn(cf.amp_pref, __fsqrt_rn(T > 0.f ? T : 0.f));
}

// Field schedule s(k) of the orthogonal quench: h_k = h s(k) (1 without one).
__device__ __forceinline__ float field_scale(const DevCfg& cf, int64_t k)
{
    if (cf.f_n_knots <= 1 || k <= cf.f_knot_step[0]) return cf.f_n_knots == 0 ? 1.0f : cf.f_knot_s[0];
    for (int i = 0; i + 1 < cf.f_n_knots; ++i)
        if (k <= cf.f_knot_step[i + 1]) return fmaf(cf.f_slope[i], (float)(k - cf.f_knot_step[i]), cf.f_knot_s[i]);
    return cf.f_knot_s[cf.f_n_knots - 1];
}

// h p and h at step k: the configuration's constants themselves without a
// schedule (the same bits as before schedules existed), else scaled by s(k)
__device__ __forceinline__ float field_hp(const DevCfg& cf, int64_t k)
{
    return cf.f_n_knots == 0 ? cf.hp : __fmul_rn(cf.hp, field_scale(cf, k));
}
__device__ __forceinline__ float field_h(const DevCfg& cf, int64_t k)
{
    return cf.f_n_knots == 0 ? cf.h : __fmul_rn(cf.h, field_scale(cf, k));
}

__device__ __forceinline__ StepConst step_const(const DevCfg& cf, float c)
{
    StepConst s;
    s.c = c;
    s.hdt = cf.hdt;
    s.dt = cf.dt;
    s.oma = cf.oma;
    s.inv1pa = cf.inv1pa;
    s.nqJx = cf.nqJx;
    s.nqJy = cf.nqJy;
    s.hp = cf.hp;
    s.q = cf.q;
    s.p = cf.p;
    return s;
}

// Coupling profiles of the anisotropic quench: J_par(k) = J_par a(k),
// J_perp(k) = J_perp b(k), piecewise linear through one knot grid and
// constant outside it, in FP32 like T(k); (1, 1) without a schedule.
__device__ __forceinline__ float2 coupling_scales(const DevCfg& cf, int64_t k)
{
    const int n = cf.c_n_knots;
    if (n <= 1 || k <= cf.c_knot_step[0])
        return n == 0 ? make_float2(1.f, 1.f) : make_float2(cf.c_knot_a[0], cf.c_knot_b[0]);
    for (int i = 0; i + 1 < n; ++i)
        if (k <= cf.c_knot_step[i + 1]) {
            const float dk = (float)(k - cf.c_knot_step[i]);
            return make_float2(fmaf(cf.c_slope_a[i], dk, cf.c_knot_a[i]), fmaf(cf.c_slope_b[i], dk, cf.c_knot_b[i]));
        }
    return make_float2(cf.c_knot_a[n - 1], cf.c_knot_b[n - 1]);
}

// J_par(k), J_perp(k): the configuration's own without a schedule (the same
// bits as before schedules existed), else scaled by the profiles
__device__ __forceinline__ float2 couplings_at(const DevCfg& cf, int64_t k)
{
    if (cf.c_n_knots == 0) return make_float2(cf.Jx, cf.Jy);
    const float2 ab = coupling_scales(cf, k);
    return make_float2(__fmul_rn(cf.Jx, ab.x), __fmul_rn(cf.Jy, ab.y));
}

// The constants of step k: noise amplitude c_k, the field's h_k p, and the
// couplings' -q J_par(k), -q J_perp(k).
__device__ __forceinline__ StepConst step_const_k(const DevCfg& cf, int64_t k, float c)
{
    StepConst s = step_const(cf, c);
    s.hp = field_hp(cf, k);
    if (cf.c_n_knots != 0) {
        const float2 ab = coupling_scales(cf, k);
        s.nqJx = __fmul_rn(cf.nqJx, ab.x);
        s.nqJy = __fmul_rn(cf.nqJy, ab.y);
    }
    return s;
}

// -------------------------------------------------------------------------
// One site of the merged BBK step (App. A.1) in leapfrog form.
// Stored state: theta_k and v_k = omega_{k-1/2}.  With g = (dt/2) F_k + c_k n_k:
//   omega_k     = (v_k + g) / (1 + eta dt / 2)          (end of Eq. BBK-2 of step k-1)
//   v_{k+1}     = (1 - eta dt / 2) omega_k + g           (Eq. BBK-1 of step k)
//   theta_{k+1} = wrap(theta_k + dt v_{k+1})             (drift + modulo)
// -------------------------------------------------------------------------

// Force on one site from its own (s, c) = (sin q t, cos q t), the sums of the
// neighbours' (s, c) along x and y, and sin(p t):
//   F = -q J_par (s (cL + cR) - c (sL + sR)) - q J_perp (s (cU + cD) - c (sU + sD)) + h p sin(p t)
__device__ __forceinline__ float site_force(const StepConst& K, float s, float c, float sx, float cx,
                                            float sy, float cy, float sinp)
{
    const float ax = fmaf(s, cx, -__fmul_rn(c, sx));
    const float ay = fmaf(s, cy, -__fmul_rn(c, sy));
    return fmaf(K.nqJx, ax, fmaf(K.nqJy, ay, __fmul_rn(K.hp, sinp)));
}

struct SiteOut {
    float theta, v, omega;
};

__device__ __forceinline__ SiteOut site_update(const StepConst& K, float theta, float v, float F, float cn)
{
    SiteOut o;
    const float g = fmaf(K.hdt, F, cn);
    o.omega = __fmul_rn(__fadd_rn(v, g), K.inv1pa);
    o.v = fmaf(K.oma, o.omega, g);
    o.theta = wrap_angle(fmaf(K.dt, o.v, theta));
    return o;
}

// Energy of one site with its forward bonds (x+1, y+1), per Eq. (XY-Hamilton-Kinetic),
// relative to the reference e_ref <= the potential part at every step:
//   omega^2 / 2 - J_par cos q(t - t_{x+1}) - J_perp cos q(t - t_{y+1}) + h cos(p t) - e_ref
// with cos q(a - b) = c_a c_b + s_a s_b, bx, by those bond cosines.  The
// potential terms are added to the small h cos(p t) - e_ref first, so every
// rounding is relative to the (small) result; the caller adds N e_ref back in FP64.
__device__ __forceinline__ float site_energy_rel(float omega, float bx, float by, float cosp, float Jx, float Jy,
                                                 float h, float e_ref)
{
    float e = fmaf(h, cosp, -e_ref);
    e = fmaf(-Jx, bx, e);
    e = fmaf(-Jy, by, e);
    return fmaf(__fmul_rn(0.5f, omega), omega, e);
}

// Jk: the couplings (couplings_at) and hk the field (field_h) of the recorded step
__device__ __forceinline__ float site_energy(const DevCfg& cf, float2 Jk, float hk, float omega, float s, float c,
                                             float sR, float cR, float sD, float cD, float cosp)
{
    const float bx = fmaf(c, cR, __fmul_rn(s, sR));
    const float by = fmaf(c, cD, __fmul_rn(s, sD));
    return site_energy_rel(omega, bx, by, cosp, Jk.x, Jk.y, hk, cf.e_ref);
}

// Asynchronous global -> shared copies (cp.async), issued by one lane for its
// own slot and read back by the same lane after cp_async_wait<N>() (this
// lane's groups but the newest N have landed): rows of the next iterations are
// in flight while the current one is computed, without a barrier.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 ld4_stream(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4_stream(float* p, float4 v) { __stcs(reinterpret_cast<float4*>(p), v); }

__device__ __forceinline__ float f4get(const float4& v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

}  // namespace xy
