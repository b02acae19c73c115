// xy_internal.h -- data shared between the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/xy_lattice.h"

namespace xy {

// Per-configuration record in device memory (read by every kernel).
// One configuration's constants on the device.  The fields every launch
// reads at its start (geometry, noise ids, the step's FP32 constants, the
// call's step range and whether schedules are set) share the first 128-byte
// line; records are line-aligned, so a block's first reads touch few lines.
struct alignas(128) DevCfg {
    int32_t Lx, Ly, n_rep, slot;  // slot: index of this record in the device table
    int32_t noise_cfg;  // configuration id in the noise counter
    int32_t rep0;       // replica id of replica 0 in the noise counter
    int64_t offset;     // first site of replica 0 in the state buffers
    int64_t N;          // Lx * Ly
    uint32_t key0, key1;
    int32_t b_first;    // flattened lattice index of replica 0
    int32_t stag;
    // FP32 constants of the step
    float Jx, Jy, h, p, q, dt, hdt, oma, inv1pa, nqJx, nqJy, hp;
    // per call
    int64_t k_start;    // step at the start of the current call
    int64_t n_call;     // steps this configuration takes in the current call
    int32_t f_n_knots;  // knots of the field schedule (0: none)
    int32_t c_n_knots;  // knots of the coupling profiles (0: none)
    // ---- temperature schedule
    int32_t n_knots;
    int32_t sched_kind;  // 0: knots below; 1: nonlinear quench (pw_* fields)
    float amp_pref;      // (1/2) sqrt(2 eta dt): noise amplitude c_k = amp_pref sqrt(T_k)
    float e_ref;         // -(|J_par| + |J_perp| + |h|): site energies are summed relative to it
    // FP32 schedule used on the device: T(k) = knot_Tf[i] + slope_f[i] (k - knot_step[i])
    float knot_Tf[XY_MAX_KNOTS];
    float slope_f[XY_MAX_KNOTS];
    int64_t knot_step[XY_MAX_KNOTS];
    double knot_T[XY_MAX_KNOTS];
    int64_t rec_first;  // first step of this call with k % record_every == 0
    double eta_d, dt_d;
    // nonlinear quench: T(k) = pw_Tc (1 + eps), eps = -sign(t) (|t| / tau_Q)^gamma, t = k - pw_kc,
    // held within [pw_ef, pw_ei]
    int64_t pw_kc;
    float pw_Tc, pw_inv_tq, pw_gamma, pw_ei, pw_ef, pad2;
    int64_t n_total;
    // field schedule (the orthogonal quench): h_k = h s(k), s piecewise linear
    // through (f_knot_step[i], f_knot_s[i]) and constant outside them, in FP32
    // from per-segment slopes like T(k); f_n_knots = 0: s = 1 (no schedule)
    int64_t f_knot_step[XY_MAX_KNOTS];
    float f_knot_s[XY_MAX_KNOTS];
    float f_slope[XY_MAX_KNOTS];
    // coupling profiles (the anisotropic quench): J_par(k) = J_par a(k),
    // J_perp(k) = J_perp b(k), piecewise linear through one knot grid, in FP32
    // from per-segment slopes; c_n_knots = 0: a = b = 1 (no schedule)
    int64_t c_knot_step[XY_MAX_KNOTS];
    float c_knot_a[XY_MAX_KNOTS];
    float c_knot_b[XY_MAX_KNOTS];
    float c_slope_a[XY_MAX_KNOTS];
    float c_slope_b[XY_MAX_KNOTS];
};
static_assert(offsetof(DevCfg, c_n_knots) + sizeof(int32_t) <= 128, "hot fields in the first line");

// Per-call settings read by the stepping kernels.
// Lives in device memory so that captured CUDA graphs stay valid across calls.
struct CallArgs {
    int64_t j_base;     // steps already done in this call (advanced by a graph node)
    int64_t rec_stride; // R: records per lattice in rec_dev
    double2* rec_dev;   // [B][R] (M, E)
    int64_t k_shift;    // added to the step index (segment recompute of the adjoint)
    int record_every;   // 0: no observables
    int fixed_parity;   // 1: always read buffers A and write buffers B
    int err;            // device error flag
    int m_only;         // 1: records carry M only (E left 0)
};

// One thread block of the strip stepper: up to 8 consecutive units of one
// lattice, one per warp.  A unit is a 128-wide column strip (or the full row
// when Lx <= 128) over H rows per row group; unit u covers strip u % strips of
// row segment u / strips.  All warps of a block share the configuration, so
// its constants and noise key are block-uniform.
struct StripTask {
    int32_t cfg;
    int32_t rep;
    int32_t unit0;      // unit of warp 0
    int32_t n_units;    // units of the lattice
};

// One thread block of the resident stepper: one whole lattice.
struct ResidentTask {
    int32_t cfg;
    int32_t rep;
};

// Round keys of Philox4x32-10 for one seed: round r uses
// (k0 + r * 0x9E3779B9, k1 + r * 0xBB67AE85).
struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline PhiloxKeys philox_round_keys(uint64_t seed)
{
    PhiloxKeys k;
    uint32_t a = (uint32_t)(seed & 0xFFFFFFFFu), b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = a;
        k.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return k;
}

struct Buffers {
    float* thA;
    float* omA;
    float* thB;
    float* omB;
};

// Observable partial sums of one lattice assembled by "last unit" reduction.
struct Partials {
    double2* part;       // [B][max_units]
    unsigned* count;     // [B]
    int32_t max_units;
};

// ---- launchers (xy_step.cu)
cudaError_t launch_init(const DevCfg* d_cfg, const DevCfg& h_cfg, int init_mode, float* theta, float* omega,
                        cudaStream_t st);
cudaError_t launch_prime(const DevCfg* d_cfg, const DevCfg& h_cfg, float* theta, float* omega, cudaStream_t st);
cudaError_t launch_omega_full(const DevCfg* d_cfg, const DevCfg& h_cfg, int rep_first, int rep_count,
                              const float* theta, const float* omega, float* out, cudaStream_t st);
cudaError_t launch_plain_step(const DevCfg* d_cfg, const DevCfg& h_cfg, int64_t j_local, Buffers buf,
                              const CallArgs* ca, Partials pa, int write_state, cudaStream_t st);
// rec: 0 = no records in this launch, 1 = records of M only, 2 = M and E;
// sched: some configuration of the tasks has a field or coupling schedule
// (false selects kernels that read the configurations' constants only)
cudaError_t launch_strip_step(const DevCfg* d_cfg, const StripTask* tasks, int n_tasks, int H, int variant,
                              int rec, bool sched, uint64_t seed, int64_t j_local, Buffers buf, const CallArgs* ca,
                              Partials pa, cudaStream_t st);
// two steps per launch (k -> k + 2) on bands of H rows across the lattice
// width (256 <= Lx <= 1024); the launch at j_local takes steps j and j + 1 of
// the call; a batch of launches must hold an even number of such pairs
struct BandTask;
cudaError_t launch_band2_step(const DevCfg* d_cfg, const BandTask* tasks, int n_tasks, int Lx, int H, int variant,
                              uint64_t seed, int64_t j_local, Buffers buf, const CallArgs* ca, cudaStream_t st);
// every task of one launch uses the noise key `seed`
cudaError_t launch_resident_step(const DevCfg* d_cfg, const ResidentTask* tasks, int n_tasks, int Lx, int Ly,
                                 int threads, int csize, uint64_t seed, int64_t j_local, int n_steps, Buffers buf,
                                 const CallArgs* ca, cudaStream_t st);
cudaError_t prepare_resident(int Lx, int Ly, int threads, int csize, int* clusters);
cudaError_t launch_advance(CallArgs* ca, int64_t by, cudaStream_t st);
cudaError_t launch_add_kshift(CallArgs* ca, int64_t by, cudaStream_t st);
cudaError_t launch_moments(const DevCfg* d_cfg, int n_cfg, const CallArgs* ca, int64_t t0, double* moments,
                           cudaStream_t st);
int resident_threads(int Lx, int Ly, int csize, size_t max_smem);
size_t resident_smem_bytes(int Lx, int Ly, int threads, int csize);
int strip_units_per_lattice(int Lx, int Ly, int H);
cudaError_t launch_debug_noise(uint64_t seed, int cfg, int rep, int64_t k, int tag, int64_t n_quads,
                               uint32_t* words, float* gauss, cudaStream_t st);
cudaError_t launch_debug_gauss4(const uint32_t* words, int64_t n_quads, float c, float* out, cudaStream_t st);
cudaError_t launch_debug_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                                cudaStream_t st);

// ---- error channel of xy_last_error (xy_api.cu), for the other translation units
int report_error(int code, const char* msg);

// ---- domains (xy_ccl.cu)
// Working memory of a labelling call.  counts (int32 per possible size, N + 1
// per lattice), bits (one mark per size) and small (counts of sizes below
// 64, in `copies` copies per lattice) must be zero when a call starts and are
// zero again when it ends without error.  list holds up to list_cap pieces
// that reach their tile's edge (batch index of the tile root, local size),
// list_n their number, aux per piece (list index of its domain's root, the
// domain's size at the root's entry), and entry maps a listed tile root's
// site to its list index.
struct CclScratch {
    int32_t* counts;
    uint32_t* bits;
    int32_t* small;
    int32_t* entry;
    int2* list;
    int2* aux;
    uint16_t* edge_root;  // per tile: tile roots of the top row, bottom row, left and right columns (32 each)
    uint4* edge_spin;     // per tile: spin masks of the same (top, bottom, left, right)
    int* list_n;
    int64_t list_cap;
    int64_t words;  // bitmap words per lattice
    int copies;
};

// Bytes of the working memory for n_lat lattices of Lx x Ly; *zeroed_bytes
// (nullable) = the leading part that must start at zero.
int64_t ccl_scratch_bytes(int Lx, int Ly, int n_lat, int64_t* zeroed_bytes);
// The parts of a block of ccl_scratch_bytes() bytes (256-byte aligned).
CclScratch ccl_scratch_carve(void* base, int Lx, int Ly, int n_lat);
// Labels (device, n_lat * Lx * Ly), and the size histogram into hist and
// n_sizes where they are non-null.  The batch must have fewer than 2^31
// sites.
cudaError_t launch_ccl(const float* theta, int Lx, int Ly, int n_lat, int32_t* labels, const CclScratch& s,
                       int64_t* hist, int64_t hist_cap, int64_t* n_sizes, int* err, cudaStream_t st);

// ---- adjoint (xy_adjoint.cu)
struct AdjArgs {
    const float* theta;   // theta_k of all lattices (segment buffer slice)
    const float* omega;   // v_k = omega_{k-1/2}
    float* tb;            // adjoint of theta (in: theta_{k+1}, out: theta_k)
    float* vb;            // adjoint of v     (in: v_{k+1},     out: v_k)
    float* Fb;            // adjoint of F_k (scratch)
    const double2* rec;   // forward observables [B][R] (M_k, E_k) with R = n + 1
    int64_t rec_stride;
    int64_t k;            // step being reversed
    int64_t k0;           // first step of the adjoint window
    int64_t k_end;        // k0 + n
    double wE, wM, inv_norm;  // objective weights and 1/(B n)
    double* gacc;         // [n_blocks][7] per-block FP64 accumulators (J_par, J_perp, h, a-bar, b-bar, c-bar-eta, w_E E)
};
cudaError_t launch_adjoint_phase_a(const DevCfg* d_cfg, const DevCfg& h_cfg, int block_base, AdjArgs a,
                                   cudaStream_t st);
cudaError_t launch_adjoint_phase_b(const DevCfg* d_cfg, const DevCfg& h_cfg, AdjArgs a, cudaStream_t st);
int adjoint_blocks(const DevCfg& h_cfg);

constexpr int kGacc = 7;  // per-block accumulators of the reverse sweep

// Reverse step on row bands: phases A and B of step k in one launch.
struct BandTask {
    int32_t cfg, rep;
    int32_t band0;    // first band of the block
    int32_t n_bands;  // bands of the lattice
};
struct BandArgs {
    const float* theta;  // theta_k
    const float* omega;  // v_k
    const float* tb_in;  // adjoints of (theta_{k+1}, v_{k+1})
    const float* vb_in;
    float* tb_out;       // adjoints of (theta_k, v_k)
    float* vb_out;
    const float* vnext;  // v_{k+1}, or null: the noise of step k is regenerated
    const double2* rec;
    int64_t rec_stride;
    int64_t k, k0;
    float wE, wM;
    double* gacc;        // [blocks][kGacc]
    int block_base;
};
// Reverse step on row bands with the state of step k integrated backward
// from step k + 1 (xy_adjoint_back.cu).
struct BackArgs {
    const float* th_in;  // theta_{k+1} (backward launches) or theta_k (the first launch)
    const float* v_in;   // v_{k+1} or v_k
    float* th_out;       // theta_k, v_k recovered (backward launches; rows of the own bands)
    float* v_out;
    const float* tb_in;  // adjoints of (theta_{k+1}, v_{k+1}), without the |M_{k+1}| term
    const float* vb_in;
    float* tb_out;       // adjoints of (theta_k, v_k), without the |M_k| term
    float* vb_out;
    double* mpart;       // [B][2][P] per-block sums of sigma sin(q theta): slot k & 1 written
    int P;               // partial slots per lattice
    double2* rec;        // [B][rec_stride]: M_{k+1} written to .x of column k + 1 - k0
    int64_t rec_stride;
    int64_t k, k0;
    float wE, wM;
    double* gacc;        // [blocks][kGacc]
    int block_base;
    int sched;           // some configuration of the tasks has a field or coupling schedule
};
cudaError_t launch_adjoint_back(const DevCfg* d_cfg, const BandTask* tasks, int n_tasks, int Lx, int H, uint64_t seed,
                                bool back, BackArgs R, cudaStream_t st);
// M_k of slots [0, n_states) of a segment (slot stride 2 T floats) into
// rec[b * rec_stride + r0 + slot].x
cudaError_t launch_segment_m(const DevCfg* d_cfg, int n_cfg, int64_t B, const float* seg, int64_t T, int n_states,
                             double2* rec, int64_t rec_stride, int64_t r0, cudaStream_t st);
// Autocorrelation time of recorded series (xy_tau.cu); out: device, 4 * n_series doubles
cudaError_t launch_autocorr(const double2* rec, int64_t n_series, int64_t R, int component, int transform,
                            int64_t skip, int n, double c_win, int half_window, double* out, cudaStream_t st);
// Structure factors (xy_sf.cu) of n_lat lattices starting at theta +
// offsets[b], shapes Lx[b] x Ly[b]; S_par, S_perp: device, n_lat * K doubles
cudaError_t launch_structure_factor(const float* theta, const int64_t* offsets, const int* Lx, const int* Ly,
                                    int n_lat, int K, float r, double* S_par, double* S_perp, int* n_launches,
                                    cudaStream_t st);
cudaError_t launch_adjoint_band(const DevCfg* d_cfg, const BandTask* tasks, int n_tasks, int Lx, int H, uint64_t seed,
                                BandArgs R, cudaStream_t st);

}  // namespace xy
