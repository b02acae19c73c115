/*
 * xy_lattice.h -- C ABI of the GB300 (sm_103a) Langevin stepper for the
 * symmetry-broken XY model of Si(001) dimer angles (arXiv 2409.06412).
 *
 * The model (paper, Sec. III):
 *   H = sum_ij omega_ij^2 / 2                                    Eq. (XY-Hamilton-Kinetic)
 *     - J_par  sum cos q(theta_ij - theta_i+1,j)
 *     - J_perp sum cos q(theta_ij - theta_i,j+1)
 *     + h sum cos(p theta_ij)                                    Eq. (XY-Hamilton-Field)
 * with theta in [-pi/2, pi/2) (Sec. III.C), q = 2, p = 2.5, and the Langevin
 * equations of Sec. III.D integrated by the BBK scheme of App. A.1, the angle
 * mapped back into [-pi/2, pi/2) after every step.
 *
 * Conventions for every call below.
 *  - A lattice object holds n_cfg configurations; configuration c has
 *    n_replicas independent periodic Lx x Ly lattices.  All lattices of all
 *    configurations are stored back to back, configuration after
 *    configuration, replica after replica, row-major inside a lattice
 *    (site s = y * Lx + x; x runs along the dimer rows, the J_par direction).
 *    "Lattice b" below is the flattened (configuration, replica) index.
 *  - theta and omega are caller-owned DEVICE buffers of float (FP32), one value
 *    per site; the library borrows them for the lifetime of the object and
 *    keeps the live state in them between calls.  omega holds the leapfrog
 *    half-step angular velocity omega_{k-1/2} of the state at integer step k;
 *    xy_omega_full() returns the full-step omega_k of the paper's scheme.
 *  - Every call returns XY_OK (0) or a negative XY_E* code; xy_last_error()
 *    then gives a message (thread-local, valid until the next call on that
 *    thread).  No call throws or aborts.
 *  - Calls are asynchronous on the stream given at creation unless stated
 *    otherwise.  Output pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; a host pointer makes the call synchronous.
 *    Internally a call may fork work from that stream onto the object's own
 *    streams (concurrent lattice slices); it joins them back before anything
 *    later on the creation stream runs, so stream order is as if all of it ran
 *    there.
 *  - Thread safety: one lattice object must not be used from two threads at
 *    once.  Distinct objects are independent.
 */
#ifndef XY_LATTICE_H
#define XY_LATTICE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XY_OK 0
#define XY_EINVAL (-1)   /* bad argument, shape or state; nothing was launched */
#define XY_ENOMEM (-2)   /* a device or host allocation failed */
#define XY_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define XY_ETIMEOUT (-4) /* a bounded device-side loop ran out of iterations */
#define XY_ENAN (-5)     /* a non-finite observable was produced */

#define XY_INIT_UNIFORM 0 /* theta = wrap(2 pi u), u uniform from the noise generator (stream tag 1), omega = 0 */
#define XY_INIT_ORDERED 1 /* theta = +2 pi / 5 everywhere (a field minimum at p = 2.5), omega = 0 */
#define XY_INIT_USER 2    /* theta and the FULL-STEP omega_0 are taken from the caller's buffers */

#define XY_PATH_BATCHED 0 /* tuned kernels, all configurations per launch, CUDA-graph chunks */
#define XY_PATH_PLAIN 1   /* one plain launch per step per configuration (reference path) */

#define XY_MAX_KNOTS 16

typedef struct xy_lattice xy_lattice;

/* One configuration: Lx % 4 == 0, Lx >= 4, Ly >= 1, 1 <= n_replicas <= 65535,
 * at most 65536 configurations per object.  seed keys the Philox4x32-10
 * noise; the configuration id and the replica id enter its counter, so
 * configurations that share a seed still draw independent noise.
 * cfg_id = -1 uses the position of the configuration in the array; replica r
 * of this object has replica id replica0 + r (< 65536).  A run split over
 * several objects (or GPUs) that keeps the ids reproduces the unsplit run
 * bit for bit. */
typedef struct {
    int32_t Lx;
    int32_t Ly;
    int32_t n_replicas;
    int32_t init_mode;
    uint64_t seed;
    int32_t cfg_id;
    int32_t replica0;
} xy_config_desc;

/* Model and integrator parameters of one configuration (Sec. III, App. A.1;
 * the paper's production values are J_par = 10, J_perp = 0.1, h = 1, p = 2.5,
 * q = 2, eta = 1, with dt = 0.01).  staggered_M != 0 measures the order
 * parameter with the sign (-1)^(x+y) (antiferromagnetic reading of Sec. III.B). */
typedef struct {
    double J_par;
    double J_perp;
    double h;
    double p;
    double q;
    double eta;
    double dt;
    int32_t staggered_M;
    int32_t reserved;
} xy_params;

/* Create a lattice object on `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream).  theta/omega: device buffers of sum_c n_replicas*Lx*Ly
 * floats, 16-byte aligned.  Initialises theta/omega per init_mode on the
 * stream.  Allocates the second state buffer of the double-buffered stepper
 * (8 bytes per site) and small tables.  *out receives the object. */
int xy_lattice_create(const xy_config_desc* cfg, int n_cfg, float* theta, float* omega,
                      void* cuda_stream, xy_lattice** out);

/* Set the parameters of configuration cfg (must precede the first step): the
 * couplings and field of the Hamiltonian of Sec. III.A,
 * Eq. (XY-Hamilton-Field), the damping of the Langevin equations of
 * Sec. III.D and the time step of the BBK integrator of App. A.1.
 * Requires dt > 0, eta >= 0. */
int xy_set_params(xy_lattice* lat, int cfg, const xy_params* params);

/* Temperature schedule of configuration cfg: T(k) piecewise linear through
 * the knots (step_knots[i], T_knots[i]) (strictly increasing steps, T >= 0),
 * constant outside them; a linear ramp is the quench eps(t) = -t / tau_Q of
 * Sec. II.B, Eq. (Linear-Quench).  n_steps_total bounds the run of this
 * configuration: stepping stops there (uneven run lengths in one batch). */
int xy_set_schedule(xy_lattice* lat, int cfg, const int64_t* step_knots, const double* T_knots,
                    int n_knots, int64_t n_steps_total);

/* Advance every configuration by min(n, n_steps_total - step) BBK steps.
 * record_every > 0: at every step k of this call with k % record_every == 0
 * the lattice averages M_k = (1/N) sum sin(q theta_i) (Sec. IV.A, Eq.
 * lattice-average) and E_k = H_k / N of the state at step k are evaluated;
 * those with k >= t0_discard enter the FP64 running moments (xy_observe).
 * rec (nullable; host or device): double[B][R][2] with B the total number of
 * lattices and R = n / record_every + 1; entry r of lattice b holds (M, E) of
 * the r-th recorded step of its configuration in this call (unfilled entries
 * are left untouched). */
int xy_step_n(xy_lattice* lat, int64_t n, int record_every, double* rec, int64_t t0_discard);

/* Running FP64 moments per configuration (synchronous):
 * moments[c][0..5] = sums over replicas and recorded steps >= t0 of
 * (1, M^2, M^4, E, E^2, |M|); the paper's Binder ratio (Eq. Def-Binder-Cum) is
 * U = (m[2]/m[0]) / (m[1]/m[0])^2.  step_now[c] (nullable) = current step.
 * Returns XY_ENAN if any moment is not finite. */
int xy_observe(xy_lattice* lat, double* moments, int64_t* step_now);

/* Clear the running moments of every configuration. */
int xy_reset_moments(xy_lattice* lat);

/* Full-step angular velocity omega_k of lattices [b_first, b_first+b_count)
 * into out (device, b_count*Lx*Ly floats, same layout as the state): the
 * omega(t) of the three-stage BBK scheme of App. A.1 (Eq. BBK-2), which the
 * stored half-step velocity v_k and the noise of step k determine. */
int xy_omega_full(xy_lattice* lat, int b_first, int b_count, float* out);

/* Frozen-domain labelling: the domains of equal buckling left by a quench
 * (abstract; Sec. IV.C, Fig. 6), as connected components of the Ising
 * projection spin = (theta >= 0), 4-neighbour adjacency, periodic, of lattices
 * [b_first, b_first+b_count), which must all have the same Lx, Ly.
 * labels (nullable; host or device): int32[b_count][Ly*Lx], label = smallest
 * site index of the component.  hist (nullable; host or device):
 * int64[b_count][hist_cap][2] of (size, count) pairs in ascending size,
 * zero-padded; n_sizes (nullable; host or device): int64[b_count] number of
 * distinct sizes.  Returns XY_EINVAL (after writing labels) if a lattice has
 * more than hist_cap distinct sizes.  The working memory (about 8.5 bytes per
 * site of the call, 4 more when labels go to host memory) is allocated on the
 * first call that needs more than the lattice object holds and kept until
 * xy_lattice_destroy; XY_ENOMEM if it cannot be allocated.  Synchronous. */
int xy_label_domains(xy_lattice* lat, int b_first, int b_count, int32_t* labels, int64_t* hist,
                     int64_t hist_cap, int64_t* n_sizes);

/* Domain labelling without allocation (synchronous).  The same labels, size
 * histogram and counts as xy_label_domains, for callers that must not
 * allocate device memory: services whose memory pool owns every byte of the
 * GPU and forbids libraries from allocating on their own, loops that cannot
 * afford an allocation and the device-wide synchronisation of cudaFree, and
 * jobs running close to the memory limit that must not fail half-way on an
 * allocation (this working memory is reserved when the library loads).
 * The paper has no counterpart; this is a property of the library only.
 *   theta: device float[n_lattices][Ly*Lx] (the layout of the state);
 *   labels: device int32[n_lattices][Ly*Lx]; hist (nullable): device
 *   int64[n_lattices][hist_cap][2]; n_sizes (nullable): device
 *   int64[n_lattices]; cuda_stream: the stream the work runs on.
 * Working memory is one fixed array inside the library image, sized for the
 * worst lattice shape within the limits below (about 105 MB: narrow lattices
 * cut into many small tiles), that every GPU which loads the library holds
 * until the process exits.  A call with more than XY_STATIC_CCL_MAX_SITES sites or
 * XY_STATIC_CCL_MAX_LATTICES lattices returns XY_EINVAL without launching
 * anything.  Every call shares that array and it keeps the previous call's
 * contents (each call clears what must start at zero), so calls whose work
 * overlaps on the GPU (other streams, other threads) race: issue them one
 * after another.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress).  Every call reads its error flag back and
 * synchronises cuda_stream, so no call may be issued on a capturing stream:
 * such a call returns XY_EINVAL without touching the stream.  theta, labels
 * and the non-null hist and n_sizes must be device (or managed) memory, else
 * XY_EINVAL.  No call allocates memory (no cudaMalloc or cudaFree). */
#define XY_STATIC_CCL_MAX_SITES 2097152
#define XY_STATIC_CCL_MAX_LATTICES 65536
int xy_label_domains_static(const float* theta, int Lx, int Ly, int n_lattices, int32_t* labels, int64_t* hist,
                            int64_t hist_cap, int64_t* n_sizes, void* cuda_stream);

/* Pathwise adjoint (synchronous) of the BBK trajectory of App. A.1 (the
 * paper has no adjoint; the objective's E_k and M_k are those of xy_step_n,
 * Eq. (XY-Hamilton-Kinetic) and Eq. (lattice-average)).  Runs n BBK steps
 * from the current state (which advances by n) with the noise held fixed and
 * returns
 *   objective = (1 / (B n)) sum_b sum_{k=k0+1}^{k0+n} [w_E E_k + w_M |M_k|]
 * (B = number of lattices, k0 = current step; every configuration must be at
 * the same step with n steps left) and grads[c][0..3] = d objective /
 * d(J_par, J_perp, h, eta) of configuration c.  The full-step state at k0 is
 * held fixed; the wrap has derivative 1; the kink of the field potential at
 * +-pi/2 contributes nothing (derivative almost everywhere).  The state is
 * checkpointed every checkpoint_every steps; the reverse sweep gets the states
 * of each segment as xy_set_adjoint_mode() selects.  objective, grads: host.
 * The working memory (the checkpoints, 8 bytes per site per segment, plus
 * 32 bytes per site of segment and adjoint states; the stored recompute
 * 8 bytes per site per step of a segment instead) is allocated by the first
 * call that needs more than the lattice object holds and kept until
 * xy_lattice_destroy; XY_ENOMEM if it cannot be allocated. */
int xy_adjoint_step_n(xy_lattice* lat, int64_t n, int checkpoint_every, double w_E, double w_M,
                      double* objective, double* grads);

/* Field schedule of configuration cfg: the orthogonal quench, in which the
 * symmetry-breaking field changes in time beside (or instead of) the
 * temperature, crossing the phase boundary T_c(h) of App. D (Fig. 10) at an
 * angle (Sec. V proposes such quenches; Sec. IV.C the quench angle).  The field of step k
 * is h_k = h s(k), with h from xy_set_params and s piecewise linear through
 * the knots (step_knots[i], scale_knots[i]) (steps strictly increasing,
 * scales finite) and constant outside them, evaluated in FP32 like T(k).
 * h_k replaces h in the force of time point k (both half-kicks that touch k)
 * and in E_k of Eq. (XY-Hamilton-Kinetic).  The adjoint's d/dh is the
 * derivative with respect to h at a fixed profile s.  n_knots = 0 removes
 * the schedule (s = 1: the same bits as a configuration that never had one).
 * Carried by xy_save/xy_load.  XY_EINVAL for bad knots. */
int xy_set_field_schedule(xy_lattice* lat, int cfg, const int64_t* step_knots, const double* scale_knots,
                          int n_knots);

/* Coupling profiles of configuration cfg: the anisotropic quench, in which
 * the two directional couplings move at different rates (Sec. V names
 * anisotropic quenches as an extension; in the coupling space of App. D the
 * path then leaves the temperature ray).  The couplings of step k are
 * J_par(k) = J_par a(k) and J_perp(k) = J_perp b(k), with J_par, J_perp from
 * xy_set_params and a, b piecewise linear through the knots
 * (step_knots[i], par_scales[i], perp_scales[i]) (steps strictly increasing,
 * scales finite) and constant outside them, evaluated in FP32 like T(k).
 * They replace J_par, J_perp in the force of time point k and in E_k of
 * Eq. (XY-Hamilton-Kinetic).  The adjoint's d/dJ_par and d/dJ_perp are the
 * derivatives at fixed profiles.  n_knots = 0 removes the schedule (the same
 * bits as a configuration that never had one).  Carried by xy_save/xy_load.
 * XY_EINVAL for bad knots. */
int xy_set_coupling_schedule(xy_lattice* lat, int cfg, const int64_t* step_knots, const double* par_scales,
                             const double* perp_scales, int n_knots);

/* Temporal blocking of the batched stepper (the paper steps one time step
 * per pass; this is a property of the library).  Lattices with
 * 256 <= Lx <= 1024 (Lx a multiple of 128, Ly a multiple of 8) can advance two
 * BBK steps per launch: a thread block sweeps a band of H rows across the
 * lattice width, carrying the intermediate step in registers, so the state
 * crosses HBM once per two steps (8 bytes per site-update instead of 16); the
 * two bands' boundary rows of the intermediate step are computed twice.
 * States are bit-identical either way.  Two-step launches run only over
 * stretches of steps that record nothing, in batches of a multiple of four
 * steps, and only for shapes whose configurations all run the whole call.
 *   kt = 0 (default): the autotuner times one and two steps per launch (and
 *          the band height H in {8, 16, 32, 64}) per lattice shape and keeps
 *          two only if at least 5 % faster per step;
 *   kt = 1: one step per launch everywhere;
 *   kt = 2: two steps per launch wherever the shape allows (the tuner's
 *          fastest band height, else the largest of 32, 16, 8 dividing Ly).
 * XY_EINVAL for any other value. */
int xy_set_temporal_blocking(xy_lattice* lat, int kt);

/* How the reverse sweep of xy_adjoint_step_n() gets the states of a
 * checkpoint segment (the paper has no adjoint; this is the schedule of the
 * pathwise derivative of the App. A.1 integrator):
 *   XY_ADJOINT_RECOMPUTE: recomputed forward from the checkpoint at the
 *     segment's start and stored (K + 1 states, 8 B per site each); the
 *     gradient is that of the forward trajectory to rounding of the sums.
 *   XY_ADJOINT_BACKWARD: integrated backward inside the reverse kernel from
 *     the checkpoint at the segment's end, theta_k = wrap(theta_{k+1} - dt
 *     v_{k+1}), omega_k = (v_{k+1} - g_k) / (1 - eta dt / 2), with the noise
 *     regenerated; no segment storage and no separate recompute pass.  FP32
 *     inversion recovers the forward states to ~1e-6 rad near equilibrium;
 *     far from it (random starts) unstable bonds amplify that to ~1e-3 rad
 *     at a few sites by the segment's start.  Needs the shapes of the band
 *     kernels (Lx a multiple of 128 up to 2048, or Lx <= 128 with Lx / 4
 *     dividing 32; Ly >= 2): XY_EINVAL at the adjoint call otherwise.
 *     Undoing the damping amplifies the rounding of the recovered states by
 *     about exp(eta dt K) over a segment of K steps: measured against the
 *     recompute at T_c with K = 100, the eta gradient agrees to 1e-5
 *     relative at eta dt K = 5 and only to 2e-3 at eta dt K = 10.
 *   XY_ADJOINT_AUTO (default): backward where every shape allows it and
 *     eta dt min(K, n) <= 5 for every configuration, else recompute. */
#define XY_ADJOINT_AUTO 0
#define XY_ADJOINT_RECOMPUTE 1
#define XY_ADJOINT_BACKWARD 2
int xy_set_adjoint_mode(xy_lattice* lat, int mode);

/* Structure factors of the rotor lattice (App. C, Eq. FT-Corr-delta and
 * Eq. S-as-lattice-FT), the input of the Lorentzian correlation-length fit of
 * Eq. Lorentzian-Peak.  With rotors s = (cos(r theta), sin(r theta)) of the
 * current state (the paper's rotors are r = 1), for lattices
 * b = b_first .. b_first + b_count - 1 and wavenumbers k = 0 .. K - 1:
 *   S_par[b - b_first][k]  = 1/(Lx Ly) sum_y sum_kappa |sum_x s^kappa_{x,y} e^{-2 pi i k x / Lx}|^2
 *   S_perp[b - b_first][k] = 1/(Lx Ly) sum_x sum_kappa |sum_y s^kappa_{x,y} e^{-2 pi i k y / Ly}|^2
 * which equal the paper's sums over the 2-D transform (Parseval over the
 * other wavenumber).  x runs along the dimer rows (the J_par direction).
 * S_par and S_perp: host or device, b_count * K doubles each, row-major.
 * Requires 1 <= K <= min(Lx, Ly) and Lx, Ly <= 8192 for every lattice of
 * the range (XY_EINVAL otherwise).  Synchronous when an output is on the
 * host.  Lattices of different shapes may share one call. */
int xy_structure_factor(xy_lattice* lat, int b_first, int b_count, int K, double rotor, double* S_par,
                        double* S_perp);

/* Integrated autocorrelation time and error of the mean of recorded series
 * (App. B: Eq. Autocorrelation-Function, Eq. Autocorrelation-Time,
 * Eq. Time-Series-Var), the input of the adaptive sampling interval
 * ds ~ tau_C / 10.  rec: DEVICE records as written by xy_step_n,
 * [n_series][R] pairs (M, E) of doubles, 16-byte aligned.  For each series b
 * the values f_s = g(rec[b][skip + s][component]), s < n, with g = identity,
 * square, fourth power or absolute value for transform 0, 1, 2, 3, give
 *   out[b] = { f_bar, sigma_f^2 = C(0), tau_C (in records), sigma_mean }
 * with C(m) = 1/(n - m) sum_s (f_s - f_bar)(f_{s+m} - f_bar),
 * tau(M) = 1/2 + sum_{m=1}^{M} C(m)/C(0), and sigma_mean^2 = 2 tau_C C(0) / n.
 * c_window > 0: tau_C = tau(M) at the smallest M >= 1 with M >= c_window tau(M)
 * (self-consistent window; 6 is customary).  c_window <= 0: M = floor(n/2),
 * the paper's integration to tau_s / 2 taken literally.
 * out: host or device, 4 * n_series doubles; synchronous when on the host.
 * Requires 2 <= n, 0 <= skip, skip + n <= R, component in {0, 1},
 * transform in {0, 1, 2, 3} (XY_EINVAL otherwise).  cuda_stream may be NULL. */
int xy_autocorr_time(const double* rec, int64_t n_series, int64_t R, int component, int transform, int64_t skip,
                     int64_t n, double c_window, double* out, void* cuda_stream);

/* Nonlinear quench (Sec. V, the extension eps(t) = t^gamma / tau_Q^gamma of
 * the linear quench of Eq. Linear-Quench) as the temperature schedule of
 * configuration cfg, replacing any xy_set_schedule():
 *   T(k) = T_c (1 + eps(k)),  eps(k) = -sign(t) |t / tau_Q|^gamma,  t = k - k_cross,
 * held within [eps_f, eps_i]: T = T_c (1 + eps_i) before the ramp and
 * T_c (1 + eps_f) after it; gamma = 1 is the linear quench.  The device
 * evaluates T(k) in FP32 once per step and block.  n_steps_total as in
 * xy_set_schedule.  Requires T_c > 0, tau_Q > 0, gamma > 0 and
 * -1 <= eps_f <= eps_i (XY_EINVAL otherwise). */
int xy_set_power_quench(xy_lattice* lat, int cfg, double T_c, int64_t k_cross, double tau_Q, double gamma,
                        double eps_i, double eps_f, int64_t n_steps_total);

/* Select the stepping path (XY_PATH_BATCHED default, or XY_PATH_PLAIN). */
int xy_set_path(xy_lattice* lat, int path);

/* Autotuner of the batched path (synchronous).  For every lattice shape it
 * times the strip stepper's rows per warp and register/occupancy variant, and
 * the resident stepper's block size, on the second state buffer (the live
 * state is untouched), and keeps the fastest; choices are cached per GPU name
 * and shape in the text file $XY_TUNE_CACHE (default
 * ~/.cache/xy_gb300_tune.txt).  Runs by itself at the first batched step
 * unless switched off with xy_set_autotune(lat, 0).  Every choice gives a
 * bit-identical state. */
int xy_autotune(xy_lattice* lat);
int xy_set_autotune(xy_lattice* lat, int on);

/* Snapshot of the complete state (synchronous): theta, omega, step counters,
 * moments, parameters and schedules.  host_buf NULL: *size receives the size
 * needed.  Resuming from a snapshot continues bit-identically. */
int xy_save(xy_lattice* lat, void* host_buf, size_t* size);
int xy_load(xy_lattice* lat, const void* host_buf, size_t size);

/* Wait for all work of the object. */
int xy_synchronize(xy_lattice* lat);

/* Number of this library's kernels launched on the object since creation
 * (graph replays count their kernel nodes). */
int64_t xy_kernel_launches(xy_lattice* lat);

#define XY_KCLASS_RESIDENT 0  /* resident stepper launches */
#define XY_KCLASS_STRIP 1     /* strip stepper launches */
#define XY_KCLASS_PLAIN 2     /* plain stepper launches */
#define XY_KCLASS_ADJ_FWD 3   /* adjoint: forward pass with checkpoints and records (one span per call) */
#define XY_KCLASS_ADJ_RECOMP 4 /* adjoint: recompute of the checkpoint segments (one span per call) */
#define XY_KCLASS_ADJ_REV 5   /* adjoint: reverse sweep kernels (one span per call) */
#define XY_KCLASS_STRIP2 6    /* two-step band launches (temporal blocking; each launch is two steps) */
#define XY_KCLASS_LABELS 7    /* domain labelling: the passes of one chunk of xy_label_domains (one span each) */
#define XY_KCLASS_COUNT 8

/* Kernel timing.  on != 0: the batched path launches its kernels directly
 * (no graph replay) and brackets every stepper launch with CUDA events on the
 * object's stream, the adjoint brackets its three phases (the spans include
 * the kernels of every class inside them) and xy_label_domains the passes of
 * each chunk (from the first pass to the last, host copies excluded); nothing
 * is skipped.  on == 0 (default): graphs, no events.
 * Switching clears the accumulated times. */
int xy_set_kernel_timing(xy_lattice* lat, int on);

/* Synchronous: accumulated device time in milliseconds (ms[XY_KCLASS_COUNT])
 * and launch counts (launches[XY_KCLASS_COUNT]) of the timed stepper launches
 * since timing was switched on. */
int xy_kernel_timing(xy_lattice* lat, double* ms, int64_t* launches);

void xy_lattice_destroy(xy_lattice* lat);
const char* xy_last_error(void);

/* Diagnostics: the device noise generator.  For lattice site s of
 * (cfg, replica) at step k and stream tag: words (nullable, device
 * uint32[n_quads][4]) = raw Philox4x32-10 output of quads 0..n_quads-1;
 * gauss (nullable, device float[4*n_quads]) = the unit Gaussians n(t) of the
 * sites.  Asynchronous on cuda_stream. */
int xy_debug_noise(uint64_t seed, int cfg, int replica, int64_t k, int tag, int64_t n_quads,
                   uint32_t* words, float* gauss, void* cuda_stream);

/* Diagnostics: bound on the steps of one root search and on the link
 * retries of one union in the domain labelling (xy_label_domains,
 * xy_label_domains_static) on the current device; iters <= 0 restores the
 * default 2^22.  A search or union that reaches the bound stops, and the call
 * returns XY_ETIMEOUT with incomplete labels (indices stay in range, nothing
 * faults).  For testing the timeout path; the paper has no counterpart. */
int xy_debug_set_union_limit(int iters);

/* Diagnostics: the Box-Muller map of the steppers (App. A.1 noise) applied to
 * given Philox words: words (device uint32[n_quads][4], 16-byte aligned) ->
 * out (device float[4*n_quads], 16-byte aligned) = c*g0..c*g3 exactly as a
 * stepping kernel forms the scaled noise of the quad's four sites from its
 * Philox output.  Lets tests sweep every uniform the generator can produce.
 * Asynchronous on cuda_stream. */
int xy_debug_gauss4(const uint32_t* words, int64_t n_quads, float c, float* out, void* cuda_stream);

/* Diagnostics: raw Philox4x32-10 of n arbitrary counters (device
 * uint32[n][4]) with key (k0, k1) into out (device uint32[n][4]). */
int xy_debug_philox(const uint32_t* counters, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                    void* cuda_stream);

/* Diagnostics: the plan of the concurrent lattice slices that a captured
 * chunk of steps (one branch per slice) and the adjoint's reverse sweep run
 * on their own streams.  Host only: no device call, no GPU needed.
 *
 * xy_debug_slice_parts: n_lat[n_groups] = lattices per kernel group;
 * fixed = branches that are not split (resident groups, the plain
 * configurations); budget = most branches in all (the stepper uses 9).  Each
 * group gets min(4, n_lat) slices (at least 1), fewer, the groups with the
 * most slices first, while fixed + the total exceeds budget.  parts[n_groups]
 * receives the counts.  XY_EINVAL on a null array, a negative count, fixed < 0
 * or budget < 1.
 *
 * xy_debug_slice_cuts: lattice_of_task[n_tasks] = the lattice of each block
 * task of a group (grouped by lattice, ascending).  cuts (room for parts + 1
 * ints) receives the first task of each slice followed by n_tasks, *n_cuts
 * their number (at most parts + 1).  Interior cuts fall on the first task of
 * a lattice, each the one nearest n_tasks * p / parts past the previous cut;
 * where no lattice start is left, fewer slices result.  XY_EINVAL on null
 * pointers, parts < 1 or tasks out of lattice order. */
int xy_debug_slice_parts(const int64_t* n_lat, int n_groups, int fixed, int budget, int* parts);
int xy_debug_slice_cuts(const int32_t* lattice_of_task, int n_tasks, int parts, int* cuts, int* n_cuts);

#ifdef __cplusplus
}
#endif
#endif /* XY_LATTICE_H */
