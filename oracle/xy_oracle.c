/*
 * xy_oracle.c -- plain FP64 CPU oracle for the Langevin (BBK) dynamics of the
 * symmetry-broken XY model of Si(001) dimer angles (arXiv 2409.06412).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline call this file.  It shares no code, header or constant table with
 * the CUDA library; each side implements the counter-based noise generator on
 * its own from the published definition.
 *
 * Everything here is written for a reader who checks it against the paper by
 * eye: one loop per equation, no blocking, no fusion, doubles throughout.
 *
 *   Hamiltonian          Sec. III.A, Eq. (XY-Hamilton-Field); q = 2, p = 2.5 (Sec. III.C)
 *   kinetic term         Sec. III.D, Eq. (XY-Hamilton-Kinetic), I = 1
 *   Langevin equations   Sec. III.D, Eqs. (Si-Langevin-theta/omega)
 *   modulo wrap          Sec. III.D (after every integration step), Fig. 3b
 *   BBK integrator       App. A.1, Eqs. (BBK-1), drift, (BBK-2)
 *   order parameter      Sec. IV.A, Eq. (lattice-average), s_i = sin(q theta_i)
 *   benchmark 1 (MSD)    App. A.2, Eq. (MSD-HO)
 *   quench schedule      Sec. II.B, Eq. (Linear-Quench)
 *   field schedule       h_k = h s(k), the orthogonal quench named in Sec. V
 *
 * Readings where the paper is silent (noise keying, sharing of one Gaussian per
 * time point between the two half-kicks, periodic boundaries, domain labels,
 * the adjoint objective) are listed with the build's design notes.
 *
 * Parity: every function below is pinned by the CPU test suite (closed forms,
 * quadrature of the canonical distribution, brute force on tiny inputs,
 * finite differences).  The Philox integer stream is pinned only statistically
 * on the CPU; its bit pattern is pinned against a library implementation on the
 * GPU.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define XYO_PI 3.14159265358979323846

/* Parameter vector layout shared with the Python wrapper of this file. */
enum { P_JPAR = 0, P_JPERP, P_H, P_P, P_Q, P_ETA, P_DT, P_STAG, P_COUNT };

/* ------------------------------------------------------------------------- */
/* Counter-based noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).     */
/* ------------------------------------------------------------------------- */

/* One call: 10 rounds of the Philox-4x32 S-box; the key is bumped by the two
 * Weyl increments between rounds. */
void xyo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from the top 23 bits of one Philox word: (m + 1/2) 2^-23.
 * Exact in binary32 and binary64. */
double xyo_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Counter of one Philox call: word 0 = quad index (site >> 2) inside the
 * lattice, word 1 = (config << 16) | replica, words 2,3 = 56-bit step with an
 * 8-bit stream tag on top (tag 0: dynamics noise n(t), tag 1: initial angles).
 * Key = the 64-bit seed. */
static void noise_words(uint64_t seed, int cfg, int rep, uint64_t quad, int64_t k, int tag,
                        uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)quad;
    ctr[1] = ((uint32_t)cfg << 16) | ((uint32_t)rep & 0xFFFFu);
    ctr[2] = (uint32_t)((uint64_t)k & 0xFFFFFFFFu);
    ctr[3] = ((uint32_t)tag << 24) | (uint32_t)(((uint64_t)k >> 32) & 0xFFFFFFu);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    xyo_philox4x32_10(ctr, key, out);
}

/* Four standard normal samples of one quad by the Box-Muller transform
 * (Box & Muller 1958): (u0,u1) -> g0,g1 and (u2,u3) -> g2,g3. */
void xyo_gauss_quad(uint64_t seed, int cfg, int rep, uint64_t quad, int64_t k, int tag, double g[4])
{
    uint32_t w[4];
    noise_words(seed, cfg, rep, quad, k, tag, w);
    for (int pair = 0; pair < 2; ++pair) {
        double u_r = xyo_uniform(w[2 * pair]);
        double u_a = xyo_uniform(w[2 * pair + 1]);
        double r = sqrt(-2.0 * log(u_r));
        g[2 * pair] = r * cos(2.0 * XYO_PI * u_a);
        g[2 * pair + 1] = r * sin(2.0 * XYO_PI * u_a);
    }
}

/* n(t) of one site: the Gaussian of slot (site & 3) of its quad's call. */
double xyo_gauss_site(uint64_t seed, int cfg, int rep, uint64_t site, int64_t k, int tag)
{
    double g[4];
    xyo_gauss_quad(seed, cfg, rep, site >> 2, k, tag, g);
    return g[site & 3];
}

/* All n(t) of one lattice (N sites) at step k. */
static void gauss_field(uint64_t seed, int cfg, int rep, int64_t N, int64_t k, double* out)
{
    for (int64_t s = 0; s < N; ++s)
        out[s] = xyo_gauss_site(seed, cfg, rep, (uint64_t)s, k, 0);
}

/* ------------------------------------------------------------------------- */
/* State space and schedule                                                  */
/* ------------------------------------------------------------------------- */

/* Map an angle back into [-pi/2, pi/2) (Sec. III.D; Fig. 3 caption). */
double xyo_wrap(double t)
{
    double r = t - XYO_PI * floor((t + 0.5 * XYO_PI) / XYO_PI);
    if (r >= 0.5 * XYO_PI) r -= XYO_PI;
    if (r < -0.5 * XYO_PI) r += XYO_PI;
    return r;
}

/* Nonlinear quench of order gamma (Sec. V, the proposed extension
 * eps(t) = t^gamma / tau_Q^gamma): T(k) = T_c (1 + eps(k)) with
 * eps(k) = -sign(t) |t / tau_Q|^gamma, t = k - k_cross, held within
 * [eps_f, eps_i] (eps_i above, eps_f below the critical point).  gamma = 1 is
 * the linear quench eps(t) = -t / tau_Q of Eq. (Linear-Quench). */
double xyo_temperature_power(int64_t k, double T_c, double k_cross, double tau_Q, double gamma, double eps_i,
                             double eps_f)
{
    const double t = (double)k - k_cross;
    double eps = -(t >= 0.0 ? 1.0 : -1.0) * pow(fabs(t) / tau_Q, gamma);
    if (eps > eps_i) eps = eps_i;
    if (eps < eps_f) eps = eps_f;
    return T_c * (1.0 + eps);
}

/* Piecewise-linear temperature T(k) through the knots (step_i, T_i), constant
 * outside them; a linear ramp is the quench of Eq. (Linear-Quench).  A
 * negative n_knots selects the nonlinear quench above with
 * Ts = {T_c, k_cross, tau_Q, gamma, eps_i, eps_f} (ks unused). */
double xyo_temperature(int64_t k, int n_knots, const int64_t* ks, const double* Ts)
{
    if (n_knots < 0) return xyo_temperature_power(k, Ts[0], Ts[1], Ts[2], Ts[3], Ts[4], Ts[5]);
    if (n_knots == 0) return 0.0;
    if (k <= ks[0]) return Ts[0];
    for (int i = 0; i + 1 < n_knots; ++i) {
        if (k <= ks[i + 1]) {
            double f = (double)(k - ks[i]) / (double)(ks[i + 1] - ks[i]);
            return Ts[i] + (Ts[i + 1] - Ts[i]) * f;
        }
    }
    return Ts[n_knots - 1];
}

/* A parameter profile: the field schedule of the orthogonal quench (Sec. V
 * proposes quenches orthogonal to the phase boundary T_c(h) of App. D; Sec.
 * IV.C the quench angle), h_k = h s(k), and the coupling profiles of the anisotropic quench.
 * Piecewise linear through (ks[i], ss[i]) and constant outside them; n = 0
 * means 1. */
double xyo_field_scale(int64_t k, int n, const int64_t* ks, const double* ss)
{
    if (n <= 0) return 1.0;
    if (k <= ks[0]) return ss[0];
    for (int i = 0; i + 1 < n; ++i)
        if (k <= ks[i + 1]) {
            double f = (double)(k - ks[i]) / (double)(ks[i + 1] - ks[i]);
            return ss[i] + (ss[i + 1] - ss[i]) * f;
        }
    return ss[n - 1];
}

/* Schedules of the parameters beside T(k): the field profile s(k) of the
 * orthogonal quench, and the anisotropic quench's profiles a(k), b(k) of the
 * two directional couplings, J_par(k) = J_par a(k), J_perp(k) = J_perp b(k)
 * (the quench moves the two coupling directions of App. D's coupling space
 * at different rates).  Each is piecewise linear through its knots and
 * constant outside them (xyo_field_scale); n = 0 means 1. */
typedef struct {
    int nf;
    const int64_t* fks;
    const double* fss;
    int nc;
    const int64_t* cks;
    const double* cpar;
    const double* cperp;
} xyo_sched;

/* The parameter vector of time point k: h, J_par and J_perp scaled by their
 * profiles. */
static void params_at(const double* prm, int64_t k, const xyo_sched* sc, double* out)
{
    memcpy(out, prm, sizeof(double) * P_COUNT);
    out[P_H] = prm[P_H] * xyo_field_scale(k, sc->nf, sc->fks, sc->fss);
    out[P_JPAR] = prm[P_JPAR] * xyo_field_scale(k, sc->nc, sc->cks, sc->cpar);
    out[P_JPERP] = prm[P_JPERP] * xyo_field_scale(k, sc->nc, sc->cks, sc->cperp);
}

static double half_kick_amp(double eta, double T, double dt)
{
    return 0.5 * sqrt(2.0 * eta * T) * sqrt(dt);
}

/* Initial angles: mode 0 = uniform theta in [0, 2pi) then wrapped (tag 1,
 * step 0); mode 1 = ordered, every theta = +2pi/5 (a minimum of cos(p theta)
 * at p = 2.5); any other mode leaves theta untouched. */
void xyo_init_theta(int Lx, int Ly, int cfg, int rep, uint64_t seed, int mode, double* theta)
{
    int64_t N = (int64_t)Lx * Ly;
    for (int64_t s = 0; s < N; ++s) {
        if (mode == 0) {
            uint32_t w[4];
            noise_words(seed, cfg, rep, (uint64_t)s >> 2, 0, 1, w);
            theta[s] = xyo_wrap(2.0 * XYO_PI * xyo_uniform(w[s & 3]));
        } else if (mode == 1) {
            theta[s] = 2.0 * XYO_PI / 5.0;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Model: force and observables on a periodic Lx x Ly lattice                 */
/* site s = y*Lx + x; x runs along the dimer rows (J_par), y across (J_perp).  */
/* ------------------------------------------------------------------------- */

static int64_t nb(int Lx, int Ly, int x, int y, int dx, int dy)
{
    int xx = (x + dx + Lx) % Lx;
    int yy = (y + dy + Ly) % Ly;
    return (int64_t)yy * Lx + xx;
}

/* F_i = -dV/dtheta_i of Eq. (XY-Hamilton-Field):
 *   -q J_par  [sin q(t_i - t_{x+1}) + sin q(t_i - t_{x-1})]
 *   -q J_perp [sin q(t_i - t_{y+1}) + sin q(t_i - t_{y-1})]
 *   + h p sin(p t_i)                                                           */
void xyo_force(int Lx, int Ly, const double* prm, const double* th, double* F)
{
    double Jx = prm[P_JPAR], Jy = prm[P_JPERP], h = prm[P_H], p = prm[P_P], q = prm[P_Q];
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int64_t i = (int64_t)y * Lx + x;
            double t = th[i];
            double fx = sin(q * (t - th[nb(Lx, Ly, x, y, 1, 0)])) + sin(q * (t - th[nb(Lx, Ly, x, y, -1, 0)]));
            double fy = sin(q * (t - th[nb(Lx, Ly, x, y, 0, 1)])) + sin(q * (t - th[nb(Lx, Ly, x, y, 0, -1)]));
            F[i] = -q * Jx * fx - q * Jy * fy + h * p * sin(p * t);
        }
}

/* Lattice averages at one time point: M = (1/N) sum sigma_i sin(q t_i)
 * (Eq. lattice-average; sigma_i = (-1)^(x+y) when the staggered reading is
 * requested, else 1) and E = H / N with H of Eq. (XY-Hamilton-Kinetic), each
 * bond counted once through its forward neighbour. */
void xyo_observe(int Lx, int Ly, const double* prm, const double* th, const double* om,
                 double* M_out, double* E_out)
{
    double Jx = prm[P_JPAR], Jy = prm[P_JPERP], h = prm[P_H], p = prm[P_P], q = prm[P_Q];
    int stag = prm[P_STAG] != 0.0;
    double N = (double)Lx * (double)Ly;
    double sm = 0.0, se = 0.0;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int64_t i = (int64_t)y * Lx + x;
            double sigma = (stag && ((x + y) & 1)) ? -1.0 : 1.0;
            sm += sigma * sin(q * th[i]);
            se += 0.5 * om[i] * om[i]
                - Jx * cos(q * (th[i] - th[nb(Lx, Ly, x, y, 1, 0)]))
                - Jy * cos(q * (th[i] - th[nb(Lx, Ly, x, y, 0, 1)]))
                + h * cos(p * th[i]);
        }
    *M_out = sm / N;
    *E_out = se / N;
}

/* ------------------------------------------------------------------------- */
/* BBK integrator (App. A.1)                                                  */
/* ------------------------------------------------------------------------- */

typedef void (*force_fn)(const void* ctx, const double* x, double* F);

/* One BBK step for n coordinates.  On entry F = F(x(t)); on exit F = F(x(t+dt)).
 * nz0, nz1 are n(t) and n(t+dt); amp0, amp1 the half-kick noise amplitudes at
 * t and t+dt.  The same sample n(t+dt) also enters the first half-kick of the
 * next step (one Gaussian per time point).  wh is scratch of length n. */
static void bbk_step(int64_t n, double* x, double* w, double* F, const double* nz0, const double* nz1,
                     double amp0, double amp1, double eta, double dt, int wrap,
                     force_fn force, const void* ctx, double* wh)
{
    /* Eq. (BBK-1): half-kick */
    for (int64_t i = 0; i < n; ++i)
        wh[i] = (1.0 - 0.5 * eta * dt) * w[i] + 0.5 * dt * F[i] + amp0 * nz0[i];
    /* drift, then the modulo map back into the allowed interval */
    for (int64_t i = 0; i < n; ++i) {
        x[i] = x[i] + wh[i] * dt;
        if (wrap) x[i] = xyo_wrap(x[i]);
    }
    /* force at the new position */
    force(ctx, x, F);
    /* Eq. (BBK-2): second half-kick */
    for (int64_t i = 0; i < n; ++i)
        w[i] = (wh[i] + 0.5 * dt * F[i] + amp1 * nz1[i]) / (1.0 + 0.5 * eta * dt);
}

typedef struct { int Lx, Ly; const double* prm; } lattice_ctx;

static void lattice_force_cb(const void* ctx, const double* x, double* F)
{
    const lattice_ctx* c = (const lattice_ctx*)ctx;
    xyo_force(c->Lx, c->Ly, c->prm, x, F);
}

/* Advance one lattice (config cfg, replica rep) from step k0 by n BBK steps.
 * theta, omega: the state (theta_k, omega_k) at integer time k, updated in
 * place.  Whenever record_every > 0 and k % record_every == 0 the observables
 * (M_k, E_k) of the state at the start of step k are appended to rec (pairs).
 * Returns the number of records written. */
int64_t xyo_run_lattice(int Lx, int Ly, int cfg, int rep, uint64_t seed, const double* prm,
                        int n_knots, const int64_t* knot_step, const double* knot_T,
                        const xyo_sched* sc,
                        int64_t k0, int64_t n, double* theta, double* omega,
                        int record_every, double* rec)
{
    int64_t N = (int64_t)Lx * Ly;
    double eta = prm[P_ETA], dt = prm[P_DT];
    double* F = (double*)malloc(sizeof(double) * N);
    double* nz0 = (double*)malloc(sizeof(double) * N);
    double* nz1 = (double*)malloc(sizeof(double) * N);
    double* wh = (double*)malloc(sizeof(double) * N);
    double prm_k[P_COUNT], prm_next[P_COUNT];  /* the field of time points k and k + 1 */
    lattice_ctx ctx = { Lx, Ly, prm_next };
    int64_t nrec = 0;

    params_at(prm, k0, sc, prm_k);
    xyo_force(Lx, Ly, prm_k, theta, F);
    gauss_field(seed, cfg, rep, N, k0, nz0);
    for (int64_t j = 0; j < n; ++j) {
        int64_t k = k0 + j;
        params_at(prm, k, sc, prm_k);
        if (record_every > 0 && k % record_every == 0) {
            xyo_observe(Lx, Ly, prm_k, theta, omega, &rec[2 * nrec], &rec[2 * nrec + 1]);
            ++nrec;
        }
        gauss_field(seed, cfg, rep, N, k + 1, nz1);
        double amp0 = half_kick_amp(eta, xyo_temperature(k, n_knots, knot_step, knot_T), dt);
        double amp1 = half_kick_amp(eta, xyo_temperature(k + 1, n_knots, knot_step, knot_T), dt);
        /* the force at the new position belongs to time point k + 1 */
        params_at(prm, k + 1, sc, prm_next);
        bbk_step(N, theta, omega, F, nz0, nz1, amp0, amp1, eta, dt, 1, lattice_force_cb, &ctx, wh);
        double* t = nz0; nz0 = nz1; nz1 = t;
    }
    free(F); free(nz0); free(nz1); free(wh);
    return nrec;
}

/* ------------------------------------------------------------------------- */
/* One row strip of a lattice (the lattice split over workers along y)        */
/* ------------------------------------------------------------------------- */

/* Force on local row i of a strip buffer of R rows.  x is periodic; the rows
 * above and below are the buffer's own rows i - 1 and i + 1, so rows 0 and
 * R - 1, which lack one of them, get NaN.  The sum is taken in the order of
 * xyo_force. */
static void strip_force(int Lx, int R, const double* prm, const double* th, double* F)
{
    double jpar = prm[P_JPAR], jperp = prm[P_JPERP], hk = prm[P_H], p = prm[P_P], q = prm[P_Q];
    for (int i = 0; i < R; ++i)
        for (int x = 0; x < Lx; ++x) {
            int64_t s = (int64_t)i * Lx + x;
            if (i == 0 || i == R - 1) { F[s] = NAN; continue; }
            const double* row = th + (int64_t)i * Lx;
            double t = row[x];
            double right = row[(x + 1) % Lx], left = row[(x + Lx - 1) % Lx];
            double below = th[s + Lx], above = th[s - Lx];
            double fx = sin(q * (t - right)) + sin(q * (t - left));
            double fy = sin(q * (t - below)) + sin(q * (t - above));
            F[s] = -q * jpar * fx - q * jperp * fy + hk * p * sin(p * t);
        }
}

/* Advance one strip of an Lx x Ly lattice by n BBK steps.  Local row i of the
 * buffers theta, omega, F (R rows of Lx) holds global row (y0 + i) mod Ly.
 * Every site takes the noise of its global index and the arithmetic of
 * xyo_run_lattice, so a site whose dependencies lie inside the buffer gets the
 * bits of the whole-lattice run.  The state between steps is
 * (theta_k, omega_k, F_k = F(theta_k)), the three arrays xyo_run_lattice
 * carries from one step to the next; F must hold F_{k0} on entry.  Each step
 * loses one row at either end (NaN, see strip_force): started from a buffer
 * exact everywhere, after n steps omega and F are exact on local rows
 * [n, R - n) and theta on [n - 1, R - n + 1).  With record_every > 0 the raw
 * sums over local rows [r0, r1) of sigma_i sin(q t_i) and of the site energy
 * (bonds to the forward neighbours x + 1 and y + 1, as xyo_observe counts
 * them) are appended to rec as pairs at every step k with
 * k % record_every == 0, before the step.  Returns the number of records. */
int64_t xyo_run_strip(int Lx, int Ly, int y0, int R, int cfg, int rep, uint64_t seed, const double* prm,
                      int n_knots, const int64_t* knot_step, const double* knot_T,
                      const xyo_sched* sc,
                      int64_t k0, int64_t n, double* theta, double* omega, double* F,
                      int r0, int r1, int record_every, double* rec)
{
    int64_t M = (int64_t)R * Lx;
    double eta = prm[P_ETA], dt = prm[P_DT];
    double* nz0 = (double*)malloc(sizeof(double) * M);
    double* nz1 = (double*)malloc(sizeof(double) * M);
    double* wh = (double*)malloc(sizeof(double) * M);
    double prm_k[P_COUNT];
    int64_t nrec = 0;

    for (int64_t j = 0; j < n; ++j) {
        int64_t k = k0 + j;
        params_at(prm, k, sc, prm_k);
        if (record_every > 0 && k % record_every == 0) {
            int stag = prm_k[P_STAG] != 0.0;
            double sm = 0.0, se = 0.0;
            for (int i = r0; i < r1; ++i) {
                int gy = (int)(((int64_t)y0 + i) % Ly);
                for (int x = 0; x < Lx; ++x) {
                    int64_t s = (int64_t)i * Lx + x;
                    double sigma = (stag && ((x + gy) & 1)) ? -1.0 : 1.0;
                    double t = theta[s];
                    sm += sigma * sin(prm_k[P_Q] * t);
                    se += 0.5 * omega[s] * omega[s]
                        - prm_k[P_JPAR] * cos(prm_k[P_Q] * (t - theta[(int64_t)i * Lx + (x + 1) % Lx]))
                        - prm_k[P_JPERP] * cos(prm_k[P_Q] * (t - theta[s + Lx]))
                        + prm_k[P_H] * cos(prm_k[P_P] * t);
                }
            }
            rec[2 * nrec] = sm;
            rec[2 * nrec + 1] = se;
            ++nrec;
        }
        /* n(t) and n(t + dt) of the global sites held here */
        for (int i = 0; i < R; ++i) {
            int64_t g0 = (((int64_t)y0 + i) % Ly) * Lx;
            for (int x = 0; x < Lx; ++x) {
                nz0[(int64_t)i * Lx + x] = xyo_gauss_site(seed, cfg, rep, (uint64_t)(g0 + x), k, 0);
                nz1[(int64_t)i * Lx + x] = xyo_gauss_site(seed, cfg, rep, (uint64_t)(g0 + x), k + 1, 0);
            }
        }
        double amp0 = half_kick_amp(eta, xyo_temperature(k, n_knots, knot_step, knot_T), dt);
        double amp1 = half_kick_amp(eta, xyo_temperature(k + 1, n_knots, knot_step, knot_T), dt);
        /* Eq. (BBK-1), the drift with the wrap, the force of time point k + 1,
         * Eq. (BBK-2) */
        for (int64_t s = 0; s < M; ++s)
            wh[s] = (1.0 - 0.5 * eta * dt) * omega[s] + 0.5 * dt * F[s] + amp0 * nz0[s];
        for (int64_t s = 0; s < M; ++s)
            theta[s] = xyo_wrap(theta[s] + wh[s] * dt);
        params_at(prm, k + 1, sc, prm_k);
        strip_force(Lx, R, prm_k, theta, F);
        for (int64_t s = 0; s < M; ++s)
            omega[s] = (wh[s] + 0.5 * dt * F[s] + amp1 * nz1[s]) / (1.0 + 0.5 * eta * dt);
    }
    free(nz0); free(nz1); free(wh);
    return nrec;
}

/* ------------------------------------------------------------------------- */
/* Benchmark 1 of App. A.2: thermal harmonic oscillators, V = w2 x^2 / 2      */
/* ------------------------------------------------------------------------- */

typedef struct { double w2; int64_t n; } harmonic_ctx;

static void harmonic_force_cb(const void* ctx, const double* x, double* F)
{
    const harmonic_ctx* c = (const harmonic_ctx*)ctx;
    for (int64_t i = 0; i < c->n; ++i) F[i] = -c->w2 * x[i];
}

/* n_paths independent oscillators from x = 0, v = 0 (m = 1), integrated with
 * the same BBK step as the lattice (no wrap); noise of path i is site i of the
 * generator.  msd[j] = <x^2> over the paths after j steps, j = 0..n_steps. */
void xyo_harmonic_msd(int64_t n_paths, int64_t n_steps, double dt, double eta, double T, double w2,
                      uint64_t seed, double* msd)
{
    double* x = (double*)calloc(n_paths, sizeof(double));
    double* w = (double*)calloc(n_paths, sizeof(double));
    double* F = (double*)calloc(n_paths, sizeof(double));
    double* nz0 = (double*)malloc(sizeof(double) * n_paths);
    double* nz1 = (double*)malloc(sizeof(double) * n_paths);
    double* wh = (double*)malloc(sizeof(double) * n_paths);
    harmonic_ctx ctx = { w2, n_paths };
    double amp = half_kick_amp(eta, T, dt);

    harmonic_force_cb(&ctx, x, F);
    msd[0] = 0.0;
    gauss_field(seed, 0, 0, n_paths, 0, nz0);
    for (int64_t j = 0; j < n_steps; ++j) {
        gauss_field(seed, 0, 0, n_paths, j + 1, nz1);
        bbk_step(n_paths, x, w, F, nz0, nz1, amp, amp, eta, dt, 0, harmonic_force_cb, &ctx, wh);
        double s = 0.0;
        for (int64_t i = 0; i < n_paths; ++i) s += x[i] * x[i];
        msd[j + 1] = s / (double)n_paths;
        double* t = nz0; nz0 = nz1; nz1 = t;
    }
    free(x); free(w); free(F); free(nz0); free(nz1); free(wh);
}

/* ------------------------------------------------------------------------- */
/* Frozen domains: connected components of equal Ising projection             */
/* ------------------------------------------------------------------------- */

/* spin_i = (theta_i >= 0), the sign of s_i = sin(2 theta_i) on [-pi/2, pi/2).
 * Components under 4-neighbour adjacency with periodic wrap, found by
 * breadth-first flood fill started from every unvisited site in row-major
 * order, so each label is the smallest site index of its component.
 * Returns the number of components. */
int64_t xyo_ccl(int Lx, int Ly, const float* theta, int32_t* labels)
{
    int64_t N = (int64_t)Lx * Ly;
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    int64_t ncomp = 0;
    for (int64_t s = 0; s < N; ++s) labels[s] = -1;
    for (int64_t s = 0; s < N; ++s) {
        if (labels[s] >= 0) continue;
        int spin = theta[s] >= 0.0f;
        int64_t head = 0, tail = 0;
        labels[s] = (int32_t)s;
        queue[tail++] = s;
        while (head < tail) {
            int64_t c = queue[head++];
            int x = (int)(c % Lx), y = (int)(c / Lx);
            int64_t nbs[4] = { nb(Lx, Ly, x, y, 1, 0), nb(Lx, Ly, x, y, -1, 0),
                               nb(Lx, Ly, x, y, 0, 1), nb(Lx, Ly, x, y, 0, -1) };
            for (int d = 0; d < 4; ++d) {
                int64_t m = nbs[d];
                if (labels[m] < 0 && (theta[m] >= 0.0f) == spin) {
                    labels[m] = (int32_t)s;
                    queue[tail++] = m;
                }
            }
        }
        ++ncomp;
    }
    free(queue);
    return ncomp;
}

/* ------------------------------------------------------------------------- */
/* Pathwise adjoint of the BBK trajectory with the noise held fixed           */
/* ------------------------------------------------------------------------- */

/* Partial derivatives of F_i with respect to (J_par, J_perp, h) at theta. */
static void force_param_derivs(int Lx, int Ly, const double* prm, const double* th, int64_t i,
                               double d[3])
{
    double p = prm[P_P], q = prm[P_Q];
    int x = (int)(i % Lx), y = (int)(i / Lx);
    double t = th[i];
    d[0] = -q * (sin(q * (t - th[nb(Lx, Ly, x, y, 1, 0)])) + sin(q * (t - th[nb(Lx, Ly, x, y, -1, 0)])));
    d[1] = -q * (sin(q * (t - th[nb(Lx, Ly, x, y, 0, 1)])) + sin(q * (t - th[nb(Lx, Ly, x, y, 0, -1)])));
    d[2] = p * sin(p * t);
}

/* out += (dF/dtheta)^T v, entry by entry of the Jacobian of xyo_force:
 *   dF_i/dtheta_i = -q^2 sum_n J_n cos q(t_i - t_n) + h p^2 cos(p t_i)
 *   dF_i/dtheta_n = +q^2 J_n cos q(t_i - t_n)       (n a neighbour of i)      */
static void force_jacobian_T(int Lx, int Ly, const double* prm, const double* th, const double* v,
                             double* out)
{
    double Jx = prm[P_JPAR], Jy = prm[P_JPERP], h = prm[P_H], p = prm[P_P], q = prm[P_Q];
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int64_t i = (int64_t)y * Lx + x;
            double t = th[i];
            int64_t nbr[4] = { nb(Lx, Ly, x, y, 1, 0), nb(Lx, Ly, x, y, -1, 0),
                               nb(Lx, Ly, x, y, 0, 1), nb(Lx, Ly, x, y, 0, -1) };
            double J[4] = { Jx, Jx, Jy, Jy };
            out[i] += v[i] * h * p * p * cos(p * t);
            for (int d = 0; d < 4; ++d) {
                double cq = q * q * J[d] * cos(q * (t - th[nbr[d]]));
                out[i] += -v[i] * cq;
                out[nbr[d]] += v[i] * cq;
            }
        }
}

/* Gradient of one observation w_E E + w_M |M| with respect to theta and omega
 * (added into tb, wb) and to (J_par, J_perp, h) (added into gp).  sign(0) = 0. */
static void observation_grad(int Lx, int Ly, const double* prm, const double* th, const double* om,
                             double wE, double wM, double* tb, double* wb, double gp[3])
{
    double Jx = prm[P_JPAR], Jy = prm[P_JPERP], h = prm[P_H], p = prm[P_P], q = prm[P_Q];
    int stag = prm[P_STAG] != 0.0;
    double N = (double)Lx * (double)Ly;
    double M, E;
    xyo_observe(Lx, Ly, prm, th, om, &M, &E);
    double sgn = (M > 0.0) ? 1.0 : ((M < 0.0) ? -1.0 : 0.0);
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
            int64_t i = (int64_t)y * Lx + x;
            int64_t ix = nb(Lx, Ly, x, y, 1, 0), iy = nb(Lx, Ly, x, y, 0, 1);
            double dx = th[i] - th[ix], dy = th[i] - th[iy];
            double sigma = (stag && ((x + y) & 1)) ? -1.0 : 1.0;
            /* energy: kinetic, forward bonds, field */
            wb[i] += wE * om[i] / N;
            tb[i] += wE * Jx * q * sin(q * dx) / N;
            tb[ix] -= wE * Jx * q * sin(q * dx) / N;
            tb[i] += wE * Jy * q * sin(q * dy) / N;
            tb[iy] -= wE * Jy * q * sin(q * dy) / N;
            tb[i] += -wE * h * p * sin(p * th[i]) / N;
            gp[0] += -wE * cos(q * dx) / N;
            gp[1] += -wE * cos(q * dy) / N;
            gp[2] += wE * cos(p * th[i]) / N;
            /* order parameter */
            tb[i] += wM * sgn * sigma * q * cos(q * th[i]) / N;
        }
}

/* Forward n BBK steps of one lattice from the full-step state (theta0, omega0)
 * at step k0, held fixed, with the noise of the generator; objective
 *   obj = sum_{k=k0+1}^{k0+n} [ w_E E_k + w_M |M_k| ]
 * and its gradient grad[0..3] with respect to (J_par, J_perp, h, eta), by
 * reverse accumulation through the three stages of App. A.1.  The wrap has
 * derivative 1 and the kink of the periodically continued field potential at
 * +-pi/2 contributes nothing (derivative taken almost everywhere).
 * theta_out/omega_out (nullable) receive the final state. */
void xyo_adjoint_lattice(int Lx, int Ly, int cfg, int rep, uint64_t seed, const double* prm,
                         int n_knots, const int64_t* knot_step, const double* knot_T,
                         const xyo_sched* sc,
                         int64_t k0, int64_t n, const double* theta0, const double* omega0,
                         double wE, double wM, double* obj_out, double* grad,
                         double* theta_out, double* omega_out)
{
    int64_t N = (int64_t)Lx * Ly;
    double eta = prm[P_ETA], dt = prm[P_DT];
    double a = 0.5 * eta * dt, b = 1.0 / (1.0 + a);
    /* trajectory storage, index j = k - k0 in 0..n */
    double* th = (double*)malloc(sizeof(double) * N * (n + 1));
    double* om = (double*)malloc(sizeof(double) * N * (n + 1));
    double* F = (double*)malloc(sizeof(double) * N * (n + 1));
    double* nz = (double*)malloc(sizeof(double) * N * (n + 1));
    double* wh = (double*)malloc(sizeof(double) * N * (n > 0 ? n : 1));
    double* amp = (double*)malloc(sizeof(double) * (n + 1));

    /* the parameters of every time point k0 .. k0 + n (the field h s(k)) */
    double* prmj = (double*)malloc(sizeof(double) * P_COUNT * (n + 1));
    for (int64_t j = 0; j <= n; ++j) params_at(prm, k0 + j, sc, prmj + P_COUNT * j);
    memcpy(th, theta0, sizeof(double) * N);
    memcpy(om, omega0, sizeof(double) * N);
    xyo_force(Lx, Ly, prmj, th, F);
    for (int64_t j = 0; j <= n; ++j) {
        gauss_field(seed, cfg, rep, N, k0 + j, nz + N * j);
        amp[j] = half_kick_amp(eta, xyo_temperature(k0 + j, n_knots, knot_step, knot_T), dt);
    }
    double obj = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double *t0 = th + N * j, *w0 = om + N * j, *F0 = F + N * j, *z0 = nz + N * j;
        double *t1 = th + N * (j + 1), *w1 = om + N * (j + 1), *F1 = F + N * (j + 1), *z1 = nz + N * (j + 1);
        double* h = wh + N * j;
        for (int64_t i = 0; i < N; ++i) h[i] = (1.0 - a) * w0[i] + 0.5 * dt * F0[i] + amp[j] * z0[i];
        for (int64_t i = 0; i < N; ++i) t1[i] = xyo_wrap(t0[i] + h[i] * dt);
        xyo_force(Lx, Ly, prmj + P_COUNT * (j + 1), t1, F1);
        for (int64_t i = 0; i < N; ++i) w1[i] = (h[i] + 0.5 * dt * F1[i] + amp[j + 1] * z1[i]) / (1.0 + a);
        double M, E;
        xyo_observe(Lx, Ly, prmj + P_COUNT * (j + 1), t1, w1, &M, &E);
        obj += wE * E + wM * fabs(M);
    }

    /* reverse sweep */
    double* tb = (double*)calloc(N, sizeof(double));   /* adjoint of theta_{j+1} */
    double* wb = (double*)calloc(N, sizeof(double));   /* adjoint of omega_{j+1} */
    double* Fb = (double*)calloc(N, sizeof(double));   /* adjoint of F_{j+1}     */
    double* hb = (double*)calloc(N, sizeof(double));
    double gJx = 0.0, gJy = 0.0, gh = 0.0, abar = 0.0, bbar = 0.0, geta_amp = 0.0;
    for (int64_t j = n - 1; j >= 0; --j) {
        double *t0 = th + N * j, *w0 = om + N * j, *z0 = nz + N * j;
        double *t1 = th + N * (j + 1), *w1 = om + N * (j + 1), *z1 = nz + N * (j + 1);
        double gp[3] = { 0.0, 0.0, 0.0 };
        const double* p1 = prmj + P_COUNT * (j + 1);  /* parameters of time point j + 1 */
        /* d h_{j+1} / d h, d J_par(j+1) / d J_par, d J_perp(j+1) / d J_perp */
        double s1 = xyo_field_scale(k0 + j + 1, sc->nf, sc->fks, sc->fss);
        double a1 = xyo_field_scale(k0 + j + 1, sc->nc, sc->cks, sc->cpar);
        double b1 = xyo_field_scale(k0 + j + 1, sc->nc, sc->cks, sc->cperp);
        /* observation at j+1 */
        observation_grad(Lx, Ly, p1, t1, w1, wE, wM, tb, wb, gp);
        gJx += gp[0] * a1; gJy += gp[1] * b1; gh += gp[2] * s1;
        /* omega_{j+1} = b (wh_j + dt/2 F_{j+1} + amp_{j+1} n_{j+1}) */
        double ampb = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            hb[i] = b * wb[i];
            Fb[i] += 0.5 * dt * b * wb[i];
            ampb += b * wb[i] * z1[i];
            bbar += (w1[i] / b) * wb[i];
        }
        geta_amp += ampb * (eta > 0.0 ? amp[j + 1] / (2.0 * eta) : 0.0);
        /* F_{j+1} = F(theta_{j+1}) */
        force_jacobian_T(Lx, Ly, p1, t1, Fb, tb);
        for (int64_t i = 0; i < N; ++i) {
            double d[3];
            force_param_derivs(Lx, Ly, p1, t1, i, d);
            gJx += Fb[i] * d[0] * a1; gJy += Fb[i] * d[1] * b1; gh += Fb[i] * d[2] * s1;
        }
        /* theta_{j+1} = wrap(theta_j + dt wh_j) */
        for (int64_t i = 0; i < N; ++i) hb[i] += dt * tb[i];
        /* wh_j = (1-a) omega_j + dt/2 F_j + amp_j n_j */
        ampb = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            abar += -w0[i] * hb[i];
            ampb += hb[i] * z0[i];
            Fb[i] = 0.5 * dt * hb[i];
            wb[i] = (1.0 - a) * hb[i];
        }
        geta_amp += ampb * (eta > 0.0 ? amp[j] / (2.0 * eta) : 0.0);
        (void)t0;
    }
    /* F_{k0} = F(theta_{k0}; params): theta_{k0} is fixed, the parameters are not */
    double s0 = xyo_field_scale(k0, sc->nf, sc->fks, sc->fss);
    double a0 = xyo_field_scale(k0, sc->nc, sc->cks, sc->cpar);
    double b0 = xyo_field_scale(k0, sc->nc, sc->cks, sc->cperp);
    for (int64_t i = 0; i < N; ++i) {
        double d[3];
        force_param_derivs(Lx, Ly, prmj, th, i, d);
        gJx += Fb[i] * d[0] * a0; gJy += Fb[i] * d[1] * b0; gh += Fb[i] * d[2] * s0;
    }
    grad[0] = gJx;
    grad[1] = gJy;
    grad[2] = gh;
    grad[3] = 0.5 * dt * (abar - b * b * bbar) + geta_amp;
    *obj_out = obj;
    if (theta_out) memcpy(theta_out, th + N * n, sizeof(double) * N);
    if (omega_out) memcpy(omega_out, om + N * n, sizeof(double) * N);
    free(th); free(om); free(F); free(nz); free(wh); free(amp); free(prmj);
    free(tb); free(wb); free(Fb); free(hb);
}

/* ------------------------------------------------------------------------- */
/* First-order sensitivity of one final angle to perturbations along the path */
/* ------------------------------------------------------------------------- */

/* Forward n BBK steps of one lattice from the full-step state (theta0, omega0)
 * at step k0 (the three stages of App. A.1, as in xyo_run_lattice), then, for
 * each target site t, one reverse sweep of the linearised step (the same
 * Jacobian as xyo_adjoint_lattice, with the final angle theta_t(k0 + n) as the
 * objective and the parameters fixed).  It yields
 *   lt_s(j) = d theta_t(k0+n) / d theta_s(k0+j),  j = 1..n  (a perturbation of
 *             the angle after the drift of step j-1, including its effect on
 *             the force F_j and everything after it),
 *   lv_s(j) = d theta_t(k0+n) / d wh_s(j),        j = 0..n-1 (a perturbation of
 *             the half-step velocity of Eq. (BBK-1) of step j, before its
 *             drift).
 * With per-site weights wt[j-1][s] (j = 1..n) on the angles and wv[j][s]
 * (j = 0..n-1) on the half-step velocities (nullable: all 1),
 *   out[2 t]     = sum_j sum_s |lt_s(j)| wt[j-1][s] + sum_j sum_s |lv_s(j)| wv[j][s]
 *   out[2 t + 1] = sqrt(sum_j sum_s lt_s(j)^2 wt[j-1][s]^2 + sum_j sum_s lv_s(j)^2 wv[j][s]^2)
 * so that local perturbations bounded by the weights move theta_t(k0+n) by at
 * most out[2 t] to first order, and independent ones spread it by a root mean
 * square at most out[2 t + 1] / sqrt(3) when each is uniform within its bound.
 * The wrap has derivative 1 (its kink is ignored, as in the adjoint).
 * traj_theta, traj_omega (nullable): [n + 1][N] receive the trajectory theta_j,
 * omega_j; lt_out, lv_out (nullable, used on tiny lattices by the tests): the
 * fields of the first target, [n][N] each, lt_out[j - 1] and lv_out[j]. */
void xyo_theta_sensitivity(int Lx, int Ly, int cfg, int rep, uint64_t seed, const double* prm,
                           int n_knots, const int64_t* knot_step, const double* knot_T,
                           const xyo_sched* sc,
                           int64_t k0, int64_t n, const double* theta0, const double* omega0,
                           int n_targets, const int64_t* targets, const double* wt, const double* wv,
                           double* out, double* traj_theta, double* traj_omega,
                           double* lt_out, double* lv_out)
{
    int64_t N = (int64_t)Lx * Ly;
    double eta = prm[P_ETA], dt = prm[P_DT];
    double a = 0.5 * eta * dt, b = 1.0 / (1.0 + a);
    double* th = (double*)malloc(sizeof(double) * N * (n + 1));
    double* om = (double*)malloc(sizeof(double) * N * (n + 1));
    double* F = (double*)malloc(sizeof(double) * N);
    double* F1 = (double*)malloc(sizeof(double) * N);
    double* z0 = (double*)malloc(sizeof(double) * N);
    double* z1 = (double*)malloc(sizeof(double) * N);
    double* wh = (double*)malloc(sizeof(double) * N);

    double* prmj = (double*)malloc(sizeof(double) * P_COUNT * (n + 1));
    for (int64_t j = 0; j <= n; ++j) params_at(prm, k0 + j, sc, prmj + P_COUNT * j);
    memcpy(th, theta0, sizeof(double) * N);
    memcpy(om, omega0, sizeof(double) * N);
    xyo_force(Lx, Ly, prmj, th, F);
    gauss_field(seed, cfg, rep, N, k0, z0);
    for (int64_t j = 0; j < n; ++j) {
        double *t0 = th + N * j, *w0 = om + N * j, *t1 = th + N * (j + 1), *w1 = om + N * (j + 1);
        double amp0 = half_kick_amp(eta, xyo_temperature(k0 + j, n_knots, knot_step, knot_T), dt);
        double amp1 = half_kick_amp(eta, xyo_temperature(k0 + j + 1, n_knots, knot_step, knot_T), dt);
        gauss_field(seed, cfg, rep, N, k0 + j + 1, z1);
        for (int64_t i = 0; i < N; ++i) wh[i] = (1.0 - a) * w0[i] + 0.5 * dt * F[i] + amp0 * z0[i];
        for (int64_t i = 0; i < N; ++i) t1[i] = xyo_wrap(t0[i] + wh[i] * dt);
        xyo_force(Lx, Ly, prmj + P_COUNT * (j + 1), t1, F1);
        for (int64_t i = 0; i < N; ++i) w1[i] = (wh[i] + 0.5 * dt * F1[i] + amp1 * z1[i]) / (1.0 + a);
        double* tmp = F; F = F1; F1 = tmp;
        tmp = z0; z0 = z1; z1 = tmp;
    }
    if (traj_theta) memcpy(traj_theta, th, sizeof(double) * N * (n + 1));
    if (traj_omega) memcpy(traj_omega, om, sizeof(double) * N * (n + 1));

    double* tb = (double*)malloc(sizeof(double) * N);
    double* wb = (double*)malloc(sizeof(double) * N);
    double* Fb = (double*)malloc(sizeof(double) * N);
    double* hb = (double*)malloc(sizeof(double) * N);
    for (int t = 0; t < n_targets; ++t) {
        double s1 = 0.0, s2 = 0.0;
        memset(tb, 0, sizeof(double) * N);
        memset(wb, 0, sizeof(double) * N);
        memset(Fb, 0, sizeof(double) * N);
        tb[targets[t]] = 1.0;
        for (int64_t j = n - 1; j >= 0; --j) {
            double* t1 = th + N * (j + 1);
            /* omega_{j+1} = b (wh_j + dt/2 F_{j+1} + amp n): its adjoint wb passes
             * to wh_j and to F_{j+1} */
            for (int64_t i = 0; i < N; ++i) {
                hb[i] = wb[i] * b;
                Fb[i] += wb[i] * b * 0.5 * dt;
            }
            /* F_{j+1} = F(theta_{j+1}): tb is now the whole adjoint of theta_{j+1} */
            force_jacobian_T(Lx, Ly, prmj + P_COUNT * (j + 1), t1, Fb, tb);
            for (int64_t i = 0; i < N; ++i) {
                double w = wt ? wt[N * j + i] : 1.0;
                s1 += fabs(tb[i]) * w;
                s2 += tb[i] * tb[i] * w * w;
            }
            if (t == 0 && lt_out) memcpy(lt_out + N * j, tb, sizeof(double) * N);
            /* theta_{j+1} = wrap(theta_j + dt wh_j): hb is now the whole adjoint of wh_j */
            for (int64_t i = 0; i < N; ++i) hb[i] += tb[i] * dt;
            for (int64_t i = 0; i < N; ++i) {
                double w = wv ? wv[N * j + i] : 1.0;
                s1 += fabs(hb[i]) * w;
                s2 += hb[i] * hb[i] * w * w;
            }
            if (t == 0 && lv_out) memcpy(lv_out + N * j, hb, sizeof(double) * N);
            /* wh_j = (1 - a) omega_j + dt/2 F_j + amp n_j; tb carries on as the
             * adjoint of theta_j (the drift has derivative 1) */
            for (int64_t i = 0; i < N; ++i) {
                Fb[i] = hb[i] * 0.5 * dt;   /* F_j enters wh_j with dt/2 */
                wb[i] = hb[i] * (1.0 - a);  /* omega_j enters wh_j with 1 - a */
            }
        }
        out[2 * t] = s1;
        out[2 * t + 1] = sqrt(s2);
    }
    free(th); free(om); free(F); free(F1); free(z0); free(z1); free(wh); free(prmj);
    free(tb); free(wb); free(Fb); free(hb);
}

/* ------------------------------------------------------------------------- */
/* Batch helpers for the tests (loops over the functions above)               */
/* ------------------------------------------------------------------------- */

void xyo_philox_batch(int64_t n, const uint32_t* ctrs, const uint32_t key[2], uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) xyo_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

void xyo_gauss_batch(uint64_t seed, int cfg, int rep, int64_t n_sites, int64_t k, int tag, double* out)
{
    for (int64_t s = 0; s < n_sites; ++s) out[s] = xyo_gauss_site(seed, cfg, rep, (uint64_t)s, k, tag);
}

void xyo_wrap_batch(int64_t n, const double* in, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = xyo_wrap(in[i]);
}
