// xy_api.cu -- the C ABI declared in include/xy_lattice.h: lattice objects,
// parameter and schedule tables, the stepping paths (plain per-configuration
// launches, or batched task tables replayed as CUDA graphs), observables,
// domain labelling, the pathwise adjoint and snapshots.
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "xy_internal.h"

using namespace xy;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(XY_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

struct CfgHost {
    xy_config_desc desc{};
    xy_params prm{};
    bool has_prm = false;
    bool has_sched = false;
    int sched_kind = 0;  // 0 knots, 1 nonlinear quench
    double pw[6] = {};   // T_c, k_cross, tau_Q, gamma, eps_i, eps_f
    int n_knots = 0;
    int64_t knot_step[XY_MAX_KNOTS] = {};
    double knot_T[XY_MAX_KNOTS] = {};
    int64_t n_total = 0;
    int64_t step = 0;
    bool primed = false;
    int f_n_knots = 0;  // field schedule s(k): h_k = h s(k)
    int64_t f_knot_step[XY_MAX_KNOTS] = {};
    double f_knot_s[XY_MAX_KNOTS] = {};
    int c_n_knots = 0;  // coupling profiles a(k), b(k): J_par a(k), J_perp b(k)
    int64_t c_knot_step[XY_MAX_KNOTS] = {};
    double c_knot_a[XY_MAX_KNOTS] = {};
    double c_knot_b[XY_MAX_KNOTS] = {};
    int kind = 2;   // 0 resident, 1 strip, 2 plain (inside the batched path)
    int H = 0;      // strip rows per row group
};

struct ResGroup {
    int Lx, Ly, threads;
    uint64_t seed;  // one noise key per group: the round keys become kernel parameters
    std::vector<ResidentTask> tasks;
    ResidentTask* d_tasks = nullptr;
    int csize = 1;  // blocks (a thread-block cluster) per lattice
};

// Autotuner cache: "gpu|kind|Lx|Ly|lattices" -> (a, b), in memory and in a
// text file (XY_TUNE_CACHE, default ~/.cache/xy_gb300_tune.txt).
struct TuneCache {
    std::vector<std::pair<std::string, std::pair<int, int>>> entries;
    bool loaded = false;
    std::string path()
    {
        const char* p = getenv("XY_TUNE_CACHE");
        if (p && *p) return p;
        const char* home = getenv("HOME");
        return std::string(home ? home : "/tmp") + "/.cache/xy_gb300_tune.txt";
    }
    void load()
    {
        if (loaded) return;
        loaded = true;
        FILE* f = fopen(path().c_str(), "r");
        if (!f) return;
        char key[512];
        int x, y;
        while (fscanf(f, "%511s %d %d", key, &x, &y) == 3) entries.push_back({key, {x, y}});
        fclose(f);
    }
    // the last entry of a key wins (put appends; a re-tuned choice overrides)
    bool get(const std::string& k, int* x, int* y)
    {
        load();
        for (auto it = entries.rbegin(); it != entries.rend(); ++it)
            if (it->first == k) {
                *x = it->second.first;
                *y = it->second.second;
                return true;
            }
        return false;
    }
    void put(const std::string& k, int x, int y)
    {
        load();
        entries.push_back({k, {x, y}});
        std::string p = path();
        const size_t slash = p.rfind('/');
        if (slash != std::string::npos) {
            std::string dir = p.substr(0, slash);
            std::string cmd_dir = dir;  // created best-effort below
            FILE* probe = fopen((dir + "/.probe").c_str(), "a");
            if (probe) {
                fclose(probe);
                remove((dir + "/.probe").c_str());
            } else {
                mkdir_p(cmd_dir);
            }
        }
        FILE* f = fopen(p.c_str(), "a");
        if (!f) return;
        fprintf(f, "%s %d %d\n", k.c_str(), x, y);
        fclose(f);
    }
    static void mkdir_p(const std::string& d)
    {
        std::string cur;
        for (size_t i = 0; i < d.size(); ++i) {
            cur += d[i];
            if (d[i] == '/' || i + 1 == d.size()) ::mkdir(cur.c_str(), 0755);
        }
    }
};
TuneCache g_tune;

// All strip-stepped lattices of one shape; H and the occupancy variant are
// chosen by the autotuner.
struct StripGroup {
    int Lx, Ly;
    uint64_t seed;  // one noise key per group: the round keys become kernel parameters
    int H;
    int variant;
    std::vector<int> cfgs;
    int64_t n_lat = 0;
    std::vector<StripTask> tasks;
    StripTask* d_tasks = nullptr;
    size_t d_cap = 0;
    int variant_rec = 0;  // occupancy variant of launches that record (0: derived from variant)
    // two steps per launch (temporal blocking): band height chosen by the
    // autotuner, 0 when one step per pass is faster or the shape does not fit
    int b2_H = 0;
    int b2_auto = 0;  // the tuner's choice (0: one step per pass)
    int b2_var = 2;   // occupancy variant of the two-step kernel (2 or 3 blocks per SM)
    int b2_best = 0;  // the fastest band height it timed, chosen or not
    std::vector<BandTask> b2_tasks;
    BandTask* d_b2_tasks = nullptr;
    size_t d_b2_cap = 0;
};

// Shapes the two-step band kernel takes: one warp per 128 columns, 2..8 warps.
bool b2_shape(int Lx, int Ly) { return Lx >= 256 && Lx <= 1024 && Lx % 128 == 0 && Ly >= 8 && Ly % 8 == 0; }

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Rows per warp of the strip stepper: the largest H <= 64 dividing the rows
// whose batch still gives at least `min_warps` warps (each warp walks its H
// rows serially, so small batches need short strips); 0 if unsupported.
int choose_strip_H(int Lx, int Ly, int64_t n_lattices_of_shape, int64_t min_warps)
{
    const bool full = Lx >= 128 ? (Lx % 128 == 0) : (Lx >= 4 && 32 % (Lx / 4) == 0);
    if (!full) return 0;
    const int groups = Lx >= 128 ? 1 : 32 / (Lx / 4);
    const int strips = Lx >= 128 ? Lx / 128 : 1;
    int best = 0;
    for (int H : {64, 32, 16, 8, 4, 2, 1}) {
        if (Ly % (H * groups) != 0) continue;
        if (best == 0) best = H;
        const int64_t warps = n_lattices_of_shape * strips * (Ly / (H * groups));
        if (warps >= min_warps) return H;
        if (H < 8) break;
        best = H;
    }
    return best;
}

}  // namespace

namespace xy {
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace xy

struct xy_lattice {
    int n_cfg = 0;
    int64_t B = 0;
    int64_t total_sites = 0;
    std::vector<CfgHost> cfg;
    std::vector<DevCfg> h_dev;
    DevCfg* d_cfg = nullptr;
    float *thA = nullptr, *omA = nullptr, *thB = nullptr, *omB = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    // branches of a captured chunk: one per stepper group (created at the
    // first capture that has more than one group)
    static constexpr int kBranches = 8;
    cudaStream_t aux[kBranches] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kBranches] = {};
    CallArgs* d_call = nullptr;
    static constexpr int kRing = 64;
    CallArgs* h_call = nullptr;  // pinned staging ring of kRing slots
    cudaEvent_t call_ev[kRing] = {};
    int call_next = 0;
    Partials pa{};
    double* d_moments = nullptr;
    double2* rec_buf = nullptr;
    size_t rec_cap = 0;
    int* d_err = nullptr;
    int path = XY_PATH_BATCHED;
    int adj_mode = XY_ADJOINT_AUTO;
    std::vector<ResGroup> res_groups;
    std::vector<StripGroup> strip_groups;
    std::vector<int> plain_cfgs;
    bool tuned = false;
    bool autotune = true;
    struct Graph {
        int chunk;
        int rec;
        uint32_t rec_mask;
        uint32_t kt2;
        std::vector<uint8_t> sched;  // sched_flags() at capture: the strip kernels chosen by schedule presence
        cudaGraphExec_t exec;
        int64_t kernels;
    };
    std::vector<Graph> graphs;  // captured chunks, by chunk length and recording
    int cur_rec = 0;            // records of the current window: 0 none, 1 M, 2 M and E
    int cur_re = 0;             // its record_every
    uint32_t cur_mask = ~0u;    // local steps of a chunk at which some strip-stepped lattice records
    uint32_t cur_kt2 = 0u;      // strip groups that take two steps per launch in this window
    int kt_mode = 0;            // xy_set_temporal_blocking: 0 tuner, 1 one step, 2 two steps per launch
    // kernel timing (direct launches bracketed by events)
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    std::vector<int> ev_class;
    size_t ev_used = 0;
    int64_t launches = 0;
    // working memory of the domain labelling, kept between calls (grown on
    // demand); its leading ccl_clean bytes are known to be zero
    void* ccl_buf = nullptr;
    int64_t ccl_bytes = 0;
    int64_t ccl_clean = 0;
    // working memory of the adjoint, kept between calls (each slot grown on
    // demand, all freed with the object): checkpoints, segment states,
    // adjoint states, records, gradient partials, partials of M, band tasks
    struct DevSlot {
        void* p = nullptr;
        size_t cap = 0;
    };
    enum { kAdjCk, kAdjSbuf, kAdjSeg, kAdjB, kAdjFb, kAdjRec, kAdjGacc, kAdjMpart, kAdjTasks, kAdjSlots };
    DevSlot adj_slot[kAdjSlots];
};

namespace {

Buffers state_buffers(const xy_lattice* L) { return Buffers{L->thA, L->omA, L->thB, L->omB}; }

int upload_cfg(xy_lattice* L)
{
    CK(cudaMemcpyAsync(L->d_cfg, L->h_dev.data(), sizeof(DevCfg) * L->n_cfg, cudaMemcpyHostToDevice, L->stream));
    return XY_OK;
}

int upload_call(xy_lattice* L, const CallArgs& ca)
{
    // a slot is reused only after the copy that read it has executed
    const int slot = L->call_next;
    L->call_next = (L->call_next + 1) % xy_lattice::kRing;
    CK(cudaEventSynchronize(L->call_ev[slot]));
    L->h_call[slot] = ca;
    CK(cudaMemcpyAsync(L->d_call, &L->h_call[slot], sizeof(CallArgs), cudaMemcpyHostToDevice, L->stream));
    CK(cudaEventRecord(L->call_ev[slot], L->stream));
    return XY_OK;
}

void fill_params(DevCfg& d, const xy_params& p)
{
    d.Jx = (float)p.J_par;
    d.Jy = (float)p.J_perp;
    d.h = (float)p.h;
    d.p = (float)p.p;
    d.q = (float)p.q;
    d.dt = (float)p.dt;
    d.hdt = (float)(0.5 * p.dt);
    d.oma = (float)(1.0 - 0.5 * p.eta * p.dt);
    d.inv1pa = (float)(1.0 / (1.0 + 0.5 * p.eta * p.dt));
    d.nqJx = (float)(-p.q * p.J_par);
    d.nqJy = (float)(-p.q * p.J_perp);
    d.hp = (float)(p.h * p.p);
    d.eta_d = p.eta;
    d.dt_d = p.dt;
    d.stag = p.staggered_M ? 1 : 0;
    d.amp_pref = (float)(0.5 * std::sqrt(2.0 * p.eta * p.dt));
    // a lower bound of a site's potential energy: sums of E_k run over the
    // site energies minus it, which at and below T_c are ~10x smaller than
    // the energies themselves, and so are their FP32 roundings
    d.e_ref = (float)(-(std::fabs(p.J_par) + std::fabs(p.J_perp) + std::fabs(p.h)));
}

// Largest |scale| of a profile (1 without one).
double profile_max(int n, const double* v)
{
    double m = n == 0 ? 1.0 : 0.0;
    for (int i = 0; i < n; ++i) m = std::max(m, std::fabs(v[i]));
    return m;
}

// The energy reference: the potential part of a site's energy is
// >= -(|J_par| max|a| + |J_perp| max|b| + |h| max|s|) at every step.
void fill_e_ref(DevCfg& d, const CfgHost& h)
{
    if (!h.has_prm) return;
    d.e_ref = (float)(-(std::fabs(h.prm.J_par) * profile_max(h.c_n_knots, h.c_knot_a) +
                        std::fabs(h.prm.J_perp) * profile_max(h.c_n_knots, h.c_knot_b) +
                        std::fabs(h.prm.h) * profile_max(h.f_n_knots, h.f_knot_s)));
}

// FP32 field schedule of the device record, and the energy reference.
void fill_field_f32(DevCfg& d, const CfgHost& h)
{
    d.f_n_knots = h.f_n_knots;
    for (int i = 0; i < XY_MAX_KNOTS; ++i) {
        const bool on = i < h.f_n_knots;
        d.f_knot_step[i] = on ? h.f_knot_step[i] : 0;
        d.f_knot_s[i] = on ? (float)h.f_knot_s[i] : 0.f;
        d.f_slope[i] = (i + 1 < h.f_n_knots)
                           ? (float)((h.f_knot_s[i + 1] - h.f_knot_s[i]) / (double)(h.f_knot_step[i + 1] - h.f_knot_step[i]))
                           : 0.f;
    }
    fill_e_ref(d, h);
}

// FP32 coupling profiles of the device record, and the energy reference.
void fill_coupling_f32(DevCfg& d, const CfgHost& h)
{
    d.c_n_knots = h.c_n_knots;
    for (int i = 0; i < XY_MAX_KNOTS; ++i) {
        const bool on = i < h.c_n_knots;
        const bool seg = i + 1 < h.c_n_knots;
        const double dk = seg ? (double)(h.c_knot_step[i + 1] - h.c_knot_step[i]) : 1.0;
        d.c_knot_step[i] = on ? h.c_knot_step[i] : 0;
        d.c_knot_a[i] = on ? (float)h.c_knot_a[i] : 0.f;
        d.c_knot_b[i] = on ? (float)h.c_knot_b[i] : 0.f;
        d.c_slope_a[i] = seg ? (float)((h.c_knot_a[i + 1] - h.c_knot_a[i]) / dk) : 0.f;
        d.c_slope_b[i] = seg ? (float)((h.c_knot_b[i + 1] - h.c_knot_b[i]) / dk) : 0.f;
    }
    fill_e_ref(d, h);
}

void fill_schedule_f32(DevCfg& d)
{
    for (int i = 0; i < XY_MAX_KNOTS; ++i) {
        d.knot_Tf[i] = (float)d.knot_T[i];
        d.slope_f[i] = (i + 1 < d.n_knots)
                           ? (float)((d.knot_T[i + 1] - d.knot_T[i]) / (double)(d.knot_step[i + 1] - d.knot_step[i]))
                           : 0.f;
    }
}

// FP32 parameters of the nonlinear quench for the device (or kind 0)
void fill_power_f32(DevCfg& d, const CfgHost& h)
{
    d.sched_kind = h.sched_kind;
    if (h.sched_kind != 1) return;
    d.pw_Tc = (float)h.pw[0];
    d.pw_kc = (int64_t)h.pw[1];
    d.pw_inv_tq = (float)(1.0 / h.pw[2]);
    d.pw_gamma = (float)h.pw[3];
    d.pw_ei = (float)h.pw[4];
    d.pw_ef = (float)h.pw[5];
}

int check_ready(xy_lattice* L)
{
    for (int c = 0; c < L->n_cfg; ++c) {
        if (!L->cfg[c].has_prm) return fail(XY_EINVAL, "configuration %d has no parameters (xy_set_params)", c);
        if (!L->cfg[c].has_sched) return fail(XY_EINVAL, "configuration %d has no schedule (xy_set_schedule)", c);
    }
    return XY_OK;
}

// Point every configuration's call window at its current step (no stepping).
void set_window_idle(xy_lattice* L)
{
    for (int c = 0; c < L->n_cfg; ++c) {
        L->h_dev[c].k_start = L->cfg[c].step;
        L->h_dev[c].n_call = 0;
        L->h_dev[c].rec_first = L->cfg[c].step;
    }
}

int prime_all(xy_lattice* L)
{
    bool any = false;
    for (int c = 0; c < L->n_cfg; ++c) any |= !L->cfg[c].primed;
    if (!any) return XY_OK;
    set_window_idle(L);
    int rc = upload_cfg(L);
    if (rc) return rc;
    for (int c = 0; c < L->n_cfg; ++c) {
        if (L->cfg[c].primed) continue;
        CK(launch_prime(L->d_cfg, L->h_dev[c], L->thA, L->omA, L->stream));
        ++L->launches;
        L->cfg[c].primed = true;
    }
    return XY_OK;
}

int ensure_rec(xy_lattice* L, size_t n)
{
    if (n <= L->rec_cap) return XY_OK;
    if (L->rec_buf) cudaFree(L->rec_buf);
    L->rec_buf = nullptr;
    L->rec_cap = 0;
    if (cudaMalloc(&L->rec_buf, n * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(XY_ENOMEM, "cannot allocate %zu records", n);
    }
    L->rec_cap = n;
    return XY_OK;
}

// Event pair of the next timed launch (pool grows on demand).
int timed_begin(xy_lattice* L, cudaStream_t st, int cls, cudaEvent_t* end)
{
    *end = nullptr;
    if (!L->timing || st != L->stream) return XY_OK;
    if (L->ev_used == L->ev_pool.size()) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        L->ev_pool.push_back({a, b});
        L->ev_class.push_back(0);
    }
    L->ev_class[L->ev_used] = cls;
    CK(cudaEventRecord(L->ev_pool[L->ev_used].first, st));
    *end = L->ev_pool[L->ev_used].second;
    ++L->ev_used;
    return XY_OK;
}

int timed_end(cudaEvent_t end, cudaStream_t st)
{
    if (end) CK(cudaEventRecord(end, st));
    return XY_OK;
}

// A timed span of the adjoint that contains other timed launches: its own
// event pair, recorded outside the per-launch pairs.
struct Span {
    xy_lattice* L;
    cudaEvent_t end = nullptr;
    int open(int cls) { return timed_begin(L, L->stream, cls, &end); }
    int close() { return timed_end(end, L->stream); }
};

// Whether some configuration in cfgs has a field or coupling schedule (the
// launches over them then take the kernels that evaluate them).
bool any_sched(const xy_lattice* L, const std::vector<int>& cfgs)
{
    for (int c : cfgs)
        if (L->h_dev[c].f_n_knots != 0 || L->h_dev[c].c_n_knots != 0) return true;
    return false;
}
bool group_sched(const xy_lattice* L, const StripGroup& g) { return any_sched(L, g.cfgs); }

// Entry g: strip group g has a schedule (part of a captured chunk's key).
std::vector<uint8_t> sched_flags(const xy_lattice* L)
{
    std::vector<uint8_t> f(L->strip_groups.size());
    for (size_t g = 0; g < f.size(); ++g) f[g] = group_sched(L, L->strip_groups[g]) ? 1 : 0;
    return f;
}

// Whether strip group g takes the local steps [jl0, jl0 + cnt) two per launch:
// the window allows it (cur_kt2: every configuration of the group runs the
// whole window), none of the steps records, and the batch holds an even number
// of pairs, so that after it the state is where single steps would leave it.
bool kt2_batch(const xy_lattice* L, int g, int64_t jl0, int cnt)
{
    // (groups past the 32 bits of cur_kt2 always take one step per launch)
    if (g >= 32 || !((L->cur_kt2 >> g) & 1u) || cnt % 4 != 0 || L->strip_groups[g].b2_H == 0) return false;
    if (L->cur_rec)
        for (int i = 0; i < cnt; ++i)
            if ((L->cur_mask >> ((jl0 + i) & 31)) & 1u) return false;
    return true;
}

// Launch the batched kernels for local steps [jl0, jl0 + cnt) of the current window.
int launch_batched_steps(xy_lattice* L, cudaStream_t st, int64_t jl0, int cnt, bool advance)
{
    const Buffers buf = state_buffers(L);
    cudaEvent_t end;
    int rc;
    for (auto& g : L->res_groups) {
        if ((rc = timed_begin(L, st, XY_KCLASS_RESIDENT, &end))) return rc;
        CK(launch_resident_step(L->d_cfg, g.d_tasks, (int)g.tasks.size(), g.Lx, g.Ly, g.threads, g.csize, g.seed, jl0, cnt, buf,
                                L->d_call, st));
        if ((rc = timed_end(end, st))) return rc;
        ++L->launches;
    }
    for (int i = 0; i < cnt; ++i) {
        for (auto& g : L->strip_groups) {
            if (kt2_batch(L, (int)(&g - L->strip_groups.data()), jl0, cnt)) {
                if (i & 1) continue;  // the launch at step i took step i + 1 too
                if ((rc = timed_begin(L, st, XY_KCLASS_STRIP2, &end))) return rc;
                CK(launch_band2_step(L->d_cfg, g.d_b2_tasks, (int)g.b2_tasks.size(), g.Lx, g.b2_H, g.b2_var, g.seed,
                                     jl0 + i, buf, L->d_call, st));
                if ((rc = timed_end(end, st))) return rc;
                ++L->launches;
                continue;
            }
            if ((rc = timed_begin(L, st, XY_KCLASS_STRIP, &end))) return rc;
            // only the steps that record run the recording kernel
            const int rec = (L->cur_rec && ((L->cur_mask >> ((jl0 + i) & 31)) & 1u)) ? L->cur_rec : 0;
            const int var = rec && g.variant_rec ? g.variant_rec : g.variant;
            CK(launch_strip_step(L->d_cfg, g.d_tasks, (int)g.tasks.size(), g.H, var, rec, group_sched(L, g),
                                 g.seed, jl0 + i, buf, L->d_call, L->pa, st));
            if ((rc = timed_end(end, st))) return rc;
            ++L->launches;
        }
        for (int c : L->plain_cfgs) {
            if ((rc = timed_begin(L, st, XY_KCLASS_PLAIN, &end))) return rc;
            CK(launch_plain_step(L->d_cfg, L->h_dev[c], jl0 + i, buf, L->d_call, L->pa, 1, st));
            if ((rc = timed_end(end, st))) return rc;
            ++L->launches;
        }
    }
    if (advance) {
        CK(launch_advance(L->d_call, cnt, st));
        ++L->launches;
    }
    return XY_OK;
}

// Concurrent slices of a set of kernel groups.  Lattices never read each
// other within a step, so a group's blocks may be cut into slices at lattice
// boundaries and each slice launched on its own stream, keeping only its own
// step order: when one slice's launch drains, the next slice's blocks fill
// the SMs it leaves idle, instead of every step waiting for the slowest SM.
// Each group with m lattices gets min(kMaxSlices, m) slices, fewer (largest
// counts first) while the total, with `fixed` unsplit branches, exceeds
// `budget`; cuts fall at the task nearest an even share of the group's tasks
// that starts a lattice.
constexpr int kMaxSlices = 4;

// Largest eta dt K (segment of K steps) at which XY_ADJOINT_AUTO integrates a
// segment's states backward (see xy_adjoint_step_n).
constexpr double kAutoBackMaxDamping = 5.0;

template <class Task>
std::vector<int> lattice_starts(const std::vector<Task>& tk)
{
    std::vector<int> st;
    for (int i = 0; i < (int)tk.size(); ++i)
        if (i == 0 || tk[i].cfg != tk[i - 1].cfg || tk[i].rep != tk[i - 1].rep) st.push_back(i);
    return st;
}

// Slices per group: the counts depend only on the groups' lattice counts
// (n_lat), so they are known before a group's tasks are built.
template <class Group>
std::vector<int> slice_parts(const std::vector<Group>& groups, int fixed, int budget)
{
    const size_t G = groups.size();
    std::vector<int> parts(G);
    int total = fixed;
    for (size_t g = 0; g < G; ++g) {
        parts[g] = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSlices, groups[g].n_lat));
        total += parts[g];
    }
    while (total > budget) {
        size_t big = G;
        for (size_t g = 0; g < G; ++g)
            if (parts[g] > 1 && (big == G || parts[g] > parts[big])) big = g;
        if (big == G) break;
        --parts[big];
        --total;
    }
    return parts;
}

// The first task of each of `parts` slices of tk, followed by tk's size.
template <class Task>
std::vector<int> cut_tasks(const std::vector<Task>& tk, int parts)
{
    const int nt = (int)tk.size();
    const std::vector<int> starts = lattice_starts(tk);
    std::vector<int> cuts{0};
    for (int p = 1; p < parts; ++p) {
        const int64_t want = (int64_t)nt * p / parts;
        int best = -1;
        for (int s : starts)
            if (s > cuts.back() && (best < 0 || std::llabs(s - want) < std::llabs(best - want))) best = s;
        if (best > 0 && best < nt) cuts.push_back(best);
    }
    cuts.push_back(nt);
    return cuts;
}

// cuts[g]: the first task of each slice of group g followed by the group's task count
template <class Group>
std::vector<std::vector<int>> slice_groups(const std::vector<Group>& groups, int fixed, int budget)
{
    const std::vector<int> parts = slice_parts(groups, fixed, budget);
    std::vector<std::vector<int>> cuts(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) cuts[g] = cut_tasks(groups[g].tasks, parts[g]);
    return cuts;
}

// The branch streams and their fork/join events, created on first use.
cudaError_t ensure_branch_streams(xy_lattice* L)
{
    if (L->fork_ev) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&L->fork_ev, cudaEventDisableTiming);
    for (int i = 0; i < xy_lattice::kBranches && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&L->aux[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->join_ev[i], cudaEventDisableTiming);
    }
    return e;
}

// fn(stream, task0, n_tasks) `reps` times for each slice of `cuts`, slice q
// on stream q (the object's stream, then its branch streams), forked from
// and joined back to the object's stream: the way a captured chunk runs a
// sliced group, so that the autotuner times its candidates that way too.
template <class F>
cudaError_t launch_sliced(xy_lattice* L, const std::vector<int>& cuts, int reps, F&& fn)
{
    const int ns = std::min((int)cuts.size() - 1, xy_lattice::kBranches + 1);
    cudaError_t e = cudaSuccess;
    if (ns <= 1) {
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = fn(L->stream, 0, cuts.back());
        return e;
    }
    if ((int)cuts.size() - 1 > ns) return cudaErrorInvalidValue;
    e = ensure_branch_streams(L);
    if (e == cudaSuccess) e = cudaEventRecord(L->fork_ev, L->stream);
    for (int q = 1; q < ns && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(L->aux[q - 1], L->fork_ev, 0);
    for (int q = 0; q < ns && e == cudaSuccess; ++q)
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = fn(q == 0 ? L->stream : L->aux[q - 1], cuts[q], cuts[q + 1] - cuts[q]);
    for (int q = 1; q < ns && e == cudaSuccess; ++q) {
        e = cudaEventRecord(L->join_ev[q - 1], L->aux[q - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(L->stream, L->join_ev[q - 1], 0);
    }
    return e;
}

// Branches of a captured chunk: each resident group, each slice of a strip
// group, and all plain configurations together.  Branches share no lattice,
// so a chunk's branches need no order among themselves.
struct Branch {
    int kind;  // 0 resident group, 1 strip group slice, 2 plain configurations
    int group;
    int task0, n_tasks;
    int b2_task0 = 0, b2_n_tasks = 0;  // the same lattices' tasks of the two-step kernel
};

// Index of the first two-step task of the lattice that strip task t starts
// (both task lists run lattice by lattice, every lattice of a group alike).
int b2_index_of(const StripGroup& g, int t)
{
    if (g.b2_H == 0 || g.tasks.empty()) return 0;
    if (t >= (int)g.tasks.size()) return (int)g.b2_tasks.size();
    const int per_strip = (int)(g.tasks.size() / g.n_lat);
    return (t / per_strip) * (g.Ly / g.b2_H);
}

std::vector<Branch> chunk_branches(const xy_lattice* L)
{
    std::vector<Branch> out;
    for (int r = 0; r < (int)L->res_groups.size(); ++r) out.push_back({0, r, 0, 0});
    const int fixed = (int)L->res_groups.size() + (L->plain_cfgs.empty() ? 0 : 1);
    const auto cuts = slice_groups(L->strip_groups, fixed, xy_lattice::kBranches + 1);
    for (int s = 0; s < (int)L->strip_groups.size(); ++s) {
        const StripGroup& g = L->strip_groups[s];
        for (size_t p = 0; p + 1 < cuts[s].size(); ++p) {
            Branch b{1, s, cuts[s][p], cuts[s][p + 1] - cuts[s][p]};
            b.b2_task0 = b2_index_of(g, cuts[s][p]);
            b.b2_n_tasks = b2_index_of(g, cuts[s][p + 1]) - b.b2_task0;
            out.push_back(b);
        }
    }
    if (!L->plain_cfgs.empty()) out.push_back({2, 0, 0, 0});
    return out;
}

cudaError_t launch_branch(xy_lattice* L, cudaStream_t st, const Branch& br, int64_t jl0, int cnt)
{
    const Buffers buf = state_buffers(L);
    cudaError_t e = cudaSuccess;
    if (br.kind == 0) {
        auto& g = L->res_groups[br.group];
        e = launch_resident_step(L->d_cfg, g.d_tasks, (int)g.tasks.size(), g.Lx, g.Ly, g.threads, g.csize, g.seed,
                                 jl0, cnt, buf, L->d_call, st);
        ++L->launches;
        return e;
    }
    const bool two = br.kind == 1 && kt2_batch(L, br.group, jl0, cnt);
    for (int i = 0; i < cnt && e == cudaSuccess; ++i) {
        if (two) {
            if (i & 1) continue;
            auto& g = L->strip_groups[br.group];
            e = launch_band2_step(L->d_cfg, g.d_b2_tasks + br.b2_task0, br.b2_n_tasks, g.Lx, g.b2_H, g.b2_var, g.seed,
                                  jl0 + i, buf, L->d_call, st);
            ++L->launches;
        } else if (br.kind == 1) {
            auto& g = L->strip_groups[br.group];
            const int rec = (L->cur_rec && ((L->cur_mask >> ((jl0 + i) & 31)) & 1u)) ? L->cur_rec : 0;
            const int var = rec && g.variant_rec ? g.variant_rec : g.variant;
            e = launch_strip_step(L->d_cfg, g.d_tasks + br.task0, br.n_tasks, g.H, var, rec, group_sched(L, g), g.seed,
                                  jl0 + i, buf, L->d_call, L->pa, st);
            ++L->launches;
        } else {
            for (int c : L->plain_cfgs) {
                if (e != cudaSuccess) break;
                e = launch_plain_step(L->d_cfg, L->h_dev[c], jl0 + i, buf, L->d_call, L->pa, 1, st);
                ++L->launches;
            }
        }
    }
    return e;
}

// Capture `chunk` batched steps (kernels + chunk counter) into a graph, or
// reuse the one captured before for that length.  The chunk forks into its
// branches (chunk_branches) and joins before the chunk counter advances, so
// their kernels overlap (one branch's launches fill the SMs another's leave
// idle as its launch drains) instead of taking turns every step.
int get_graph(xy_lattice* L, int chunk, xy_lattice::Graph** out)
{
    const std::vector<uint8_t> sm = sched_flags(L);
    for (auto& g : L->graphs)
        if (g.chunk == chunk && g.rec == L->cur_rec && g.rec_mask == L->cur_mask && g.kt2 == L->cur_kt2 &&
            g.sched == sm) {
            *out = &g;
            return XY_OK;
        }
    const std::vector<Branch> brs = chunk_branches(L);
    const int nb = (int)brs.size();
    const bool fork = nb >= 2 && nb <= xy_lattice::kBranches + 1;
    if (fork) {
        const cudaError_t e0 = ensure_branch_streams(L);
        if (e0 != cudaSuccess) return fail(XY_ECUDA, "branch streams: %s", cudaGetErrorString(e0));
    }
    const int64_t before = L->launches;
    CK(cudaStreamBeginCapture(L->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = XY_OK;
    if (fork) {
        cudaError_t e1 = cudaEventRecord(L->fork_ev, L->cap_stream);
        for (int b = 1; b < nb && e1 == cudaSuccess; ++b) e1 = cudaStreamWaitEvent(L->aux[b - 1], L->fork_ev, 0);
        for (int b = 0; b < nb && e1 == cudaSuccess; ++b)
            e1 = launch_branch(L, b == 0 ? L->cap_stream : L->aux[b - 1], brs[b], 0, chunk);
        for (int b = 1; b < nb && e1 == cudaSuccess; ++b) {
            e1 = cudaEventRecord(L->join_ev[b - 1], L->aux[b - 1]);
            if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(L->cap_stream, L->join_ev[b - 1], 0);
        }
        if (e1 == cudaSuccess) {
            e1 = launch_advance(L->d_call, chunk, L->cap_stream);
            ++L->launches;
        }
        if (e1 != cudaSuccess) rc = fail(XY_ECUDA, "graph capture of the branches: %s", cudaGetErrorString(e1));
    } else {
        rc = launch_batched_steps(L, L->cap_stream, 0, chunk, true);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(L->cap_stream, &g);
    const int64_t kernels = L->launches - before;
    L->launches = before;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(XY_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(XY_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    L->graphs.push_back({chunk, L->cur_rec, L->cur_mask, L->cur_kt2, sm, exec, kernels});
    *out = &L->graphs.back();
    return XY_OK;
}


int build_strip_tasks(xy_lattice* L, StripGroup& g);
int build_b2_tasks(xy_lattice* L, StripGroup& g, int H);

// ---- autotuner: per strip shape, time strip heights x occupancy variants;
// per resident shape, time the block sizes.  Candidates run one step from
// buffer A into buffer B (the scratch half of the double buffer), so the live
// state is untouched.
int time_window(xy_lattice* L, int64_t n_call)
{
    for (int c = 0; c < L->n_cfg; ++c) {
        L->h_dev[c].k_start = L->cfg[c].step;
        L->h_dev[c].n_call = n_call;
        L->h_dev[c].rec_first = L->cfg[c].step;
    }
    int rc = upload_cfg(L);
    if (rc) return rc;
    CallArgs ca{};
    ca.fixed_parity = 1;
    return upload_call(L, ca);
}

std::string gpu_name()
{
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        cudaGetLastError();
        return "gpu";
    }
    std::string s = p.name;
    for (auto& ch : s)
        if (ch == ' ' || ch == '|') ch = '_';
    return s;
}

// Band height of the two-step kernel per strip group under the current mode:
// the tuner's choice, none, or (forced) the tuner's fastest height, else the
// largest of 32, 16, 8 dividing Ly.
int apply_kt_mode(xy_lattice* L)
{
    for (auto& g : L->strip_groups) {
        int h = 0;
        if (L->kt_mode == 0) h = g.b2_auto;
        if (L->kt_mode == 2 && b2_shape(g.Lx, g.Ly)) {
            h = g.b2_best;
            for (int c : {32, 16, 8})
                if (h == 0 && g.Ly % c == 0) h = c;
        }
        if (h == g.b2_H) continue;
        g.b2_H = 0;
        if (h > 0) {
            int rc = build_b2_tasks(L, g, h);
            if (rc) return rc;
            g.b2_H = h;
        } else {
            for (auto& gr : L->graphs) cudaGraphExecDestroy(gr.exec);
            L->graphs.clear();
        }
    }
    return XY_OK;
}

int autotune_lattice(xy_lattice* L)
{
    if (L->tuned) return XY_OK;
    L->tuned = true;
    if (!L->autotune) return apply_kt_mode(L);
    const std::string gpu = gpu_name();
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = time_window(L, 8);
    const Buffers buf = state_buffers(L);
    // candidates run sliced the way the captured chunks run them
    const std::vector<int> parts =
        slice_parts(L->strip_groups, (int)L->res_groups.size() + (L->plain_cfgs.empty() ? 0 : 1),
                    xy_lattice::kBranches + 1);
    for (auto& g : L->strip_groups) {
        if (rc) break;
        if ((int64_t)g.Lx * g.Ly * g.n_lat < ((int64_t)1 << 21)) continue;  // too small to matter
        const int n_parts = parts[&g - L->strip_groups.data()];
        char key[256];
        snprintf(key, sizeof key, "%s|strip-sliced|%d|%d|%lld", gpu.c_str(), g.Lx, g.Ly, (long long)g.n_lat);
        int bh = 0, bv = 0;
        // a cached choice is used only if it satisfies the same constraints
        // as the candidates below (the cache is a plain text file)
        auto strip_ok = [&](int H, int v) {
            const int groups = g.Lx >= 128 ? 1 : 32 / (g.Lx / 4);
            return H >= 1 && H <= 64 && v >= 2 && v <= 4 && g.Ly % (H * groups) == 0 &&
                   (strip_units_per_lattice(g.Lx, g.Ly, H) + 7) / 8 <= L->pa.max_units;
        };
        if (g_tune.get(key, &bh, &bv) && !strip_ok(bh, bv)) bh = bv = 0;
        if (bh == 0) {
            // per candidate: the best of 5 timings, each over enough launches
            // to span about half a millisecond (single launches of a small
            // batch differ by less than their timing noise)
            float best = 1e30f;
            for (int H : {4, 8, 16, 32, 64}) {
                const int groups = g.Lx >= 128 ? 1 : 32 / (g.Lx / 4);
                if (g.Ly % (H * groups) != 0) continue;
                // one record partial per block of 8 units
                if ((strip_units_per_lattice(g.Lx, g.Ly, H) + 7) / 8 > L->pa.max_units) continue;
                g.H = H;
                if ((rc = build_strip_tasks(L, g))) break;
                const std::vector<int> cuts = cut_tasks(g.tasks, n_parts);
                float t_best[3] = {1e30f, 1e30f, 1e30f};
                int reps = 3;
                for (int round = 0; round < 5; ++round)
                    for (int vi = 0; vi < 3; ++vi) {
                        const int v = 2 + vi;
                        auto run = [&](cudaStream_t st, int t0, int cnt) {
                            return launch_strip_step(L->d_cfg, g.d_tasks + t0, cnt, H, v, 0, group_sched(L, g), g.seed,
                                                     0, buf, L->d_call, L->pa, st);
                        };
                        CK(launch_sliced(L, cuts, 1, run));
                        CK(cudaEventRecord(e0, L->stream));
                        CK(launch_sliced(L, cuts, reps, run));
                        CK(cudaEventRecord(e1, L->stream));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        L->launches += (int64_t)(1 + reps) * ((int)cuts.size() - 1);
                        t_best[vi] = std::min(t_best[vi], ms / reps);
                        if (round == 0 && vi == 0 && ms < 0.5f)
                            reps = std::min(64, (int)(0.5f / std::max(ms / reps, 1e-3f)) + 1);
                    }
                for (int vi = 0; vi < 3; ++vi)
                    if (t_best[vi] < best) {
                        best = t_best[vi];
                        bh = H;
                        bv = 2 + vi;
                    }
            }
            if (rc) break;
            if (bh > 0) g_tune.put(key, bh, bv);
        }
        if (bh > 0) {
            g.H = bh;
            g.variant = bv;
            if ((rc = build_strip_tasks(L, g))) break;
            // launches that record M (every step of the adjoint's recompute)
            // carry more live registers: their own variant at this H, among
            // those that do not spill
            char keyr[256];
            snprintf(keyr, sizeof keyr, "%s|striprec-sliced|%d|%d|%lld|%d", gpu.c_str(), g.Lx, g.Ly,
                     (long long)g.n_lat, bh);
            int rv = 0, unused = 0;
            if (g_tune.get(keyr, &rv, &unused) && (rv < 2 || rv > 4)) rv = 0;
            if (rv == 0) {
                double2* scratch = nullptr;
                CK(cudaMalloc(&scratch, sizeof(double2) * (size_t)L->B));
                CallArgs ca{};
                ca.fixed_parity = 1;
                ca.record_every = 1;
                ca.rec_dev = scratch;
                ca.rec_stride = 1;
                ca.m_only = 1;
                if ((rc = upload_call(L, ca))) {
                    cudaFree(scratch);
                    break;
                }
                const std::vector<int> cuts = cut_tasks(g.tasks, n_parts);
                float t_best[2] = {1e30f, 1e30f};
                int reps = 3;
                for (int round = 0; round < 5 && rc == XY_OK; ++round)
                    for (int vi = 0; vi < 2; ++vi) {
                        const int v = 2 + vi;
                        auto run = [&](cudaStream_t st, int t0, int cnt) {
                            return launch_strip_step(L->d_cfg, g.d_tasks + t0, cnt, bh, v, 1, group_sched(L, g),
                                                     g.seed, 0, buf, L->d_call, L->pa, st);
                        };
                        cudaError_t e = launch_sliced(L, cuts, 1, run);
                        if (e == cudaSuccess) e = cudaEventRecord(e0, L->stream);
                        if (e == cudaSuccess) e = launch_sliced(L, cuts, reps, run);
                        if (e == cudaSuccess) e = cudaEventRecord(e1, L->stream);
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                        if (e != cudaSuccess) {
                            cudaGetLastError();
                            rc = fail(XY_ECUDA, "autotune (recording launches): %s", cudaGetErrorString(e));
                            break;
                        }
                        L->launches += (int64_t)(1 + reps) * ((int)cuts.size() - 1);
                        t_best[vi] = std::min(t_best[vi], ms / reps);
                        if (round == 0 && vi == 0 && ms < 0.5f)
                            reps = std::min(64, (int)(0.5f / std::max(ms / reps, 1e-3f)) + 1);
                    }
                cudaStreamSynchronize(L->stream);
                cudaFree(scratch);
                if (rc) break;
                rv = t_best[1] < t_best[0] ? 3 : 2;
                g_tune.put(keyr, rv, 0);
                CallArgs ca0{};
                ca0.fixed_parity = 1;
                if ((rc = upload_call(L, ca0))) break;
            }
            g.variant_rec = rv;
        }
        // temporal blocking: two steps per launch on bands of H2 rows, timed
        // against one step per pass as chosen above, sliced alike; kept only
        // when at least 5 % faster per step
        if (rc == XY_OK && bh > 0 && b2_shape(g.Lx, g.Ly)) {
            char key2[256];
            snprintf(key2, sizeof key2, "%s|band2-sliced|%d|%d|%lld", gpu.c_str(), g.Lx, g.Ly, (long long)g.n_lat);
            int h2 = -1, unused = 0;
            if (g_tune.get(key2, &h2, &unused) && !(h2 == 0 || (h2 >= 8 && h2 <= 64 && g.Ly % h2 == 0))) h2 = -1;
            if (h2 < 0) {
                const std::vector<int> cuts1 = cut_tasks(g.tasks, n_parts);
                auto time_it = [&](const std::vector<int>& cuts, auto&& run, float& out) -> int {
                    int reps = 3;
                    out = 1e30f;
                    for (int round = 0; round < 5; ++round) {
                        CK(launch_sliced(L, cuts, 1, run));
                        CK(cudaEventRecord(e0, L->stream));
                        CK(launch_sliced(L, cuts, reps, run));
                        CK(cudaEventRecord(e1, L->stream));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        L->launches += (int64_t)(1 + reps) * ((int)cuts.size() - 1);
                        out = std::min(out, ms / reps);
                        if (round == 0 && ms < 0.5f) reps = std::min(64, (int)(0.5f / std::max(ms / reps, 1e-3f)) + 1);
                    }
                    return XY_OK;
                };
                float t1 = 1e30f;
                rc = time_it(cuts1, [&](cudaStream_t st, int t0, int cnt) {
                    return launch_strip_step(L->d_cfg, g.d_tasks + t0, cnt, g.H, g.variant, 0, group_sched(L, g),
                                             g.seed, 0, buf, L->d_call, L->pa, st);
                }, t1);
                float best2 = 1e30f;
                int bestH = 0, bestV = 2;
                for (int H2 : {8, 16, 32, 64}) {
                    if (rc || g.Ly % H2 != 0) continue;
                    if ((rc = build_b2_tasks(L, g, H2))) break;
                    g.b2_H = H2;
                    std::vector<int> cuts2;
                    for (int c1 : cuts1) cuts2.push_back(b2_index_of(g, c1));
                    for (int v2 : {2, 3}) {
                        float t2 = 1e30f;
                        rc = time_it(cuts2, [&](cudaStream_t st, int t0, int cnt) {
                            return launch_band2_step(L->d_cfg, g.d_b2_tasks + t0, cnt, g.Lx, H2, v2, g.seed, 0, buf,
                                                     L->d_call, st);
                        }, t2);
                        if (rc) break;
                        if (t2 / 2 < best2) {
                            best2 = t2 / 2;
                            bestH = H2;
                            bestV = v2;
                        }
                    }
                }
                g.b2_H = 0;
                if (rc) break;
                // a margin: isolated sliced timings overstate the two-step
                // kernel's gain inside a mixed batch (512^2 lattices of the
                // static-criticality batch: 2 % faster alone, 0.4 % slower in the batch)
                h2 = best2 < 0.95f * t1 ? bestH : 0;
                unused = bestH * 8 + bestV;  // height and variant of the fastest two-step candidate
                g_tune.put(key2, h2, unused);
            }
            g.b2_auto = h2;
            const int hb = unused / 8, vb = unused % 8;
            g.b2_best = (hb >= 8 && hb <= 64 && g.Ly % hb == 0) ? hb : 0;
            g.b2_var = (vb == 3) ? 3 : 2;
        }
    }
    if (rc == XY_OK) rc = apply_kt_mode(L);
    // resident shapes: block size x cluster size (1 = one block per lattice;
    // more blocks per lattice spread a small batch over more SMs)
    for (auto& g : L->res_groups) {
        if (rc) break;
        char key[256];
        snprintf(key, sizeof key, "%s|resident|%d|%d|%lld", gpu.c_str(), g.Lx, g.Ly, (long long)g.tasks.size());
        int bt = 0, bc = 0;
        const int G = g.Lx / 4;
        // block size nt and cluster size cs that tile the lattice into whole
        // bands and fit on the device
        auto res_ok = [&](int nt, int cs) {
            if (cs < 1 || cs > 16 || g.Ly % cs != 0 || nt < 32 || nt > 1024 || nt % G != 0) return false;
            const int Lr = g.Ly / cs;
            if (nt / G > Lr || Lr % (nt / G) != 0) return false;
            if (resident_smem_bytes(g.Lx, g.Ly, nt, cs) > 220 * 1024) return false;
            int fit = 0;
            return prepare_resident(g.Lx, g.Ly, nt, cs, &fit) == cudaSuccess && fit > 0;
        };
        if (g_tune.get(key, &bt, &bc)) {
            if (bc < 1) bc = 1;  // entries without a cluster size
            if (!res_ok(bt, bc)) bt = bc = 0;
        }
        if (bt == 0) {
            float best = 1e30f;
            const int n = (int)g.tasks.size();
            for (int cs : {1, 2, 4, 8, 16}) {
                for (int nt : {1024, 512, 256, 128, 64}) {
                    if (!res_ok(nt, cs)) continue;
                    float t_best = 1e30f;
                    for (int round = 0; round < 3; ++round) {
                        CK(launch_resident_step(L->d_cfg, g.d_tasks, n, g.Lx, g.Ly, nt, cs, g.seed, 0, 8, buf, L->d_call,
                                                L->stream));
                        CK(cudaEventRecord(e0, L->stream));
                        for (int i = 0; i < 3; ++i)
                            CK(launch_resident_step(L->d_cfg, g.d_tasks, n, g.Lx, g.Ly, nt, cs, g.seed, 0, 8, buf,
                                                    L->d_call, L->stream));
                        CK(cudaEventRecord(e1, L->stream));
                        CK(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        L->launches += 4;
                        t_best = std::min(t_best, ms);
                    }
                    if (t_best < best) {
                        best = t_best;
                        bt = nt;
                        bc = cs;
                    }
                }
            }
            if (bt > 0) g_tune.put(key, bt, bc);
        }
        if (bc < 1) bc = 1;
        if (bt > 0 && (bt != g.threads || bc != g.csize)) {
            g.threads = bt;
            g.csize = bc;
            CK(prepare_resident(g.Lx, g.Ly, bt, bc, nullptr));
            for (auto& gr : L->graphs) cudaGraphExecDestroy(gr.exec);
            L->graphs.clear();
        } else {
            CK(prepare_resident(g.Lx, g.Ly, g.threads, g.csize, nullptr));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_window_idle(L);
    if (rc == XY_OK) rc = upload_cfg(L);
    return rc;
}

// Advance every configuration by its n_call of the current window (already
// uploaded), recording into rec_dev with stride rec_stride.
int run_window(xy_lattice* L, int64_t n_max)
{
    if (n_max <= 0) return XY_OK;
    // two steps per launch for the strip groups the tuner gave a band height,
    // when every configuration of the group runs the whole window (a pair
    // never straddles the last step of one of them)
    L->cur_kt2 = 0u;
    for (int gi = 0; gi < (int)L->strip_groups.size() && gi < 32; ++gi) {
        const StripGroup& g = L->strip_groups[gi];
        bool all = g.b2_H > 0;
        for (int c : g.cfgs) all = all && L->h_dev[c].n_call == n_max;
        if (all) L->cur_kt2 |= 1u << gi;
    }
    if (L->path == XY_PATH_PLAIN) {
        for (int64_t j = 0; j < n_max; ++j)
            for (int c = 0; c < L->n_cfg; ++c) {
                if (j >= L->h_dev[c].n_call) continue;
                cudaEvent_t end;
                int rc = timed_begin(L, L->stream, XY_KCLASS_PLAIN, &end);
                if (rc) return rc;
                CK(launch_plain_step(L->d_cfg, L->h_dev[c], j, state_buffers(L), L->d_call, L->pa, 1, L->stream));
                if ((rc = timed_end(end, L->stream))) return rc;
                ++L->launches;
            }
        return XY_OK;
    }
    // Records further apart than a chunk: the stretches between recording
    // steps run as non-recording graph chunks, and each step at which some
    // strip configuration records runs alone with the recording kernel.
    if (L->cur_rec && L->cur_re > 32) {
        std::vector<int64_t> rec_steps;
        for (const auto& g : L->strip_groups)
            for (int c : g.cfgs) {
                const DevCfg& d = L->h_dev[c];
                const int64_t re = L->cur_re;
                for (int64_t j = ((re - d.k_start % re) % re); j < std::min(n_max, d.n_call); j += re)
                    rec_steps.push_back(j);
            }
        std::sort(rec_steps.begin(), rec_steps.end());
        rec_steps.erase(std::unique(rec_steps.begin(), rec_steps.end()), rec_steps.end());
        auto stretch = [&](int64_t cnt) -> int {
            L->cur_mask = 0u;
            const int ch = (int)std::min<int64_t>(32, cnt);
            const int64_t nf = (L->timing || ch < 2) ? 0 : cnt / ch;
            if (nf > 0) {
                xy_lattice::Graph* g = nullptr;
                int rc = get_graph(L, ch, &g);
                if (rc) return rc;
                for (int64_t i = 0; i < nf; ++i) {
                    CK(cudaGraphLaunch(g->exec, L->stream));
                    L->launches += g->kernels;
                }
            }
            for (int64_t done = nf * ch; done < cnt;) {
                const int k = (int)std::min<int64_t>(ch, cnt - done);
                int rc = launch_batched_steps(L, L->stream, 0, k, true);
                if (rc) return rc;
                done += k;
            }
            return XY_OK;
        };
        int64_t pos = 0;
        for (int64_t r : rec_steps) {
            int rc = r > pos ? stretch(r - pos) : XY_OK;
            if (rc) return rc;
            L->cur_mask = 1u;  // local step 0 of this one-step launch records
            if ((rc = launch_batched_steps(L, L->stream, 0, 1, true))) return rc;
            pos = r + 1;
        }
        return pos < n_max ? stretch(n_max - pos) : XY_OK;
    }
    // graph replays of 32-step chunks (or one chunk of the whole window when
    // it is shorter), then direct launches for the remainder.  When the
    // window records every re <= 32 steps, the chunk is a multiple of re, so
    // the local steps that record are the same in every chunk and only they
    // run the recording strip kernel (cur_mask); otherwise every step may.
    int chunk = (int)std::min<int64_t>(32, n_max);
    L->cur_mask = ~0u;
    if (L->cur_rec && L->cur_re > 0 && L->cur_re <= 32) {
        chunk = (int)std::min<int64_t>((32 / L->cur_re) * L->cur_re, n_max);
        uint32_t mask = 0;
        for (const auto& g : L->strip_groups)
            for (int c : g.cfgs) {
                const DevCfg& d = L->h_dev[c];
                for (int jl = 0; jl < chunk; ++jl)
                    if ((d.k_start + jl) % L->cur_re == 0) mask |= 1u << jl;
            }
        L->cur_mask = mask;
    }
    const int64_t n_full = (L->timing || chunk < 2) ? 0 : n_max / chunk;
    const int rem = (int)(n_max - n_full * chunk);
    if (n_full > 0) {
        xy_lattice::Graph* g = nullptr;
        int rc = get_graph(L, chunk, &g);
        if (rc) return rc;
        for (int64_t i = 0; i < n_full; ++i) {
            CK(cudaGraphLaunch(g->exec, L->stream));
            L->launches += g->kernels;
        }
    }
    for (int64_t done = 0; done < rem;) {
        // direct launches: at most one chunk per resident launch
        const int cnt = (int)std::min<int64_t>(chunk, rem - done);
        const bool more = done + cnt < rem;
        int rc = launch_batched_steps(L, L->stream, 0, cnt, more);
        if (rc) return rc;
        done += cnt;
    }
    return XY_OK;
}

// After a window: configurations that took an odd number of steps hold their
// state in buffer B; copy it back so that the caller's buffers are current.
int fixup_parity(xy_lattice* L)
{
    for (int c = 0; c < L->n_cfg; ++c) {
        if ((L->h_dev[c].n_call & 1) == 0) continue;
        const DevCfg& d = L->h_dev[c];
        const size_t bytes = sizeof(float) * (size_t)d.N * d.n_rep;
        CK(cudaMemcpyAsync(L->thA + d.offset, L->thB + d.offset, bytes, cudaMemcpyDeviceToDevice, L->stream));
        CK(cudaMemcpyAsync(L->omA + d.offset, L->omB + d.offset, bytes, cudaMemcpyDeviceToDevice, L->stream));
    }
    return XY_OK;
}

// Core of xy_step_n: n steps, records with stride rec_stride into rec_dev
// (nullable when record_every == 0), optional moments.
int advance_core(xy_lattice* L, int64_t n, int record_every, double2* rec_dev, int64_t rec_stride,
                 bool do_moments, int64_t t0, bool m_only = false)
{
    if (L->path == XY_PATH_BATCHED && !L->tuned) {
        int rc0 = autotune_lattice(L);
        if (rc0) return rc0;
    }
    int64_t n_max = 0;
    for (int c = 0; c < L->n_cfg; ++c) {
        CfgHost& h = L->cfg[c];
        DevCfg& d = L->h_dev[c];
        const int64_t left = h.n_total - h.step;
        d.k_start = h.step;
        d.n_call = std::max<int64_t>(0, std::min<int64_t>(n, left));
        d.rec_first = record_every > 0 ? ((h.step + record_every - 1) / record_every) * record_every : h.step;
        n_max = std::max(n_max, d.n_call);
    }
    int rc = upload_cfg(L);
    if (rc) return rc;
    CallArgs ca{};
    ca.j_base = 0;
    ca.rec_stride = rec_stride;
    ca.rec_dev = rec_dev;
    ca.k_shift = 0;
    ca.record_every = record_every;
    ca.fixed_parity = 0;
    ca.m_only = m_only ? 1 : 0;
    if ((rc = upload_call(L, ca))) return rc;
    L->cur_rec = record_every > 0 ? (m_only ? 1 : 2) : 0;
    L->cur_re = record_every;
    if ((rc = run_window(L, n_max))) return rc;
    if ((rc = fixup_parity(L))) return rc;
    if (do_moments && record_every > 0) {
        CK(launch_moments(L->d_cfg, L->n_cfg, L->d_call, t0, L->d_moments, L->stream));
        ++L->launches;
    }
    for (int c = 0; c < L->n_cfg; ++c) L->cfg[c].step += L->h_dev[c].n_call;
    return XY_OK;
}

int build_strip_tasks(xy_lattice* L, StripGroup& g)
{
    g.tasks.clear();
    const int nu = strip_units_per_lattice(g.Lx, g.Ly, g.H);
    for (int c : g.cfgs)
        for (int r = 0; r < L->cfg[c].desc.n_replicas; ++r)
            for (int u0 = 0; u0 < nu; u0 += 8) g.tasks.push_back(StripTask{c, r, u0, nu});
    if (g.tasks.size() > g.d_cap) {
        cudaFree(g.d_tasks);
        g.d_tasks = nullptr;
        g.d_cap = 0;
        CK(cudaMalloc(&g.d_tasks, sizeof(StripTask) * g.tasks.size()));
        g.d_cap = g.tasks.size();
    }
    CK(cudaMemcpy(g.d_tasks, g.tasks.data(), sizeof(StripTask) * g.tasks.size(), cudaMemcpyHostToDevice));
    for (auto& gr : L->graphs) cudaGraphExecDestroy(gr.exec);
    L->graphs.clear();
    return XY_OK;
}

// Tasks of the two-step band kernel: one block per band of H rows of every
// lattice of the group, lattice by lattice like the strip tasks.
int build_b2_tasks(xy_lattice* L, StripGroup& g, int H)
{
    g.b2_tasks.clear();
    const int nb = g.Ly / H;
    for (int c : g.cfgs)
        for (int r = 0; r < L->cfg[c].desc.n_replicas; ++r)
            for (int b = 0; b < nb; ++b) g.b2_tasks.push_back(BandTask{c, r, b, nb});
    if (g.b2_tasks.size() > g.d_b2_cap) {
        cudaFree(g.d_b2_tasks);
        g.d_b2_tasks = nullptr;
        g.d_b2_cap = 0;
        CK(cudaMalloc(&g.d_b2_tasks, sizeof(BandTask) * g.b2_tasks.size()));
        g.d_b2_cap = g.b2_tasks.size();
    }
    CK(cudaMemcpy(g.d_b2_tasks, g.b2_tasks.data(), sizeof(BandTask) * g.b2_tasks.size(), cudaMemcpyHostToDevice));
    for (auto& gr : L->graphs) cudaGraphExecDestroy(gr.exec);
    L->graphs.clear();
    return XY_OK;
}

// smallest strip height the autotuner may pick for a shape
int min_strip_H(int Lx, int Ly)
{
    const int groups = Lx >= 128 ? 1 : 32 / (Lx / 4);
    for (int H : {4, 8, 16, 32, 64, 2, 1})
        if (Ly % (H * groups) == 0) return H;
    return 1;
}

int classify(xy_lattice* L)
{
    // default kernel per configuration; see the design notes for the rules
    int max_units = 1;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    for (int c = 0; c < L->n_cfg; ++c) {
        CfgHost& h = L->cfg[c];
        const int Lx = h.desc.Lx, Ly = h.desc.Ly;
        const int64_t nq = (int64_t)Lx * Ly / 4;
        max_units = std::max<int>(max_units, (int)((nq + 255) / 256));
        const int rt = resident_threads(Lx, Ly, 1, 200 * 1024);
        int64_t same = 0;
        for (int c2 = 0; c2 < L->n_cfg; ++c2)
            if (L->cfg[c2].desc.Lx == Lx && L->cfg[c2].desc.Ly == Ly) same += L->cfg[c2].desc.n_replicas;
        const int H = choose_strip_H(Lx, Ly, same, (int64_t)sms * 16);
        if (rt > 0) {
            h.kind = 0;
        } else if (H > 0) {
            h.kind = 1;
            h.H = H;
            max_units = std::max(max_units, strip_units_per_lattice(Lx, Ly, std::min(H, min_strip_H(Lx, Ly))));
        } else {
            h.kind = 2;
        }
    }
    L->pa.max_units = max_units;
    // task tables
    for (int c = 0; c < L->n_cfg; ++c) {
        CfgHost& h = L->cfg[c];
        const int Lx = h.desc.Lx, Ly = h.desc.Ly;
        if (h.kind == 0) {
            const int rt = resident_threads(Lx, Ly, 1, 200 * 1024);
            ResGroup* g = nullptr;
            for (auto& gg : L->res_groups)
                if (gg.Lx == Lx && gg.Ly == Ly && gg.threads == rt && gg.seed == h.desc.seed) g = &gg;
            if (!g) {
                L->res_groups.push_back(ResGroup{Lx, Ly, rt, h.desc.seed, {}, nullptr});
                g = &L->res_groups.back();
            }
            for (int r = 0; r < h.desc.n_replicas; ++r) g->tasks.push_back(ResidentTask{c, r});
        } else if (h.kind == 1) {
            StripGroup* g = nullptr;
            for (auto& gg : L->strip_groups)
                if (gg.Lx == Lx && gg.Ly == Ly && gg.seed == h.desc.seed) g = &gg;
            if (!g) {
                L->strip_groups.push_back(StripGroup{Lx, Ly, h.desc.seed, h.H, 3, {}, 0, {}, nullptr, 0});
                g = &L->strip_groups.back();
            }
            g->cfgs.push_back(c);
            g->n_lat += h.desc.n_replicas;
        } else {
            L->plain_cfgs.push_back(c);
        }
    }
    for (auto& g : L->res_groups) {
        CK(cudaMalloc(&g.d_tasks, sizeof(ResidentTask) * g.tasks.size()));
        CK(cudaMemcpy(g.d_tasks, g.tasks.data(), sizeof(ResidentTask) * g.tasks.size(), cudaMemcpyHostToDevice));
        CK(prepare_resident(g.Lx, g.Ly, g.threads, g.csize, nullptr));
    }
    for (auto& g : L->strip_groups) {
        int rc = build_strip_tasks(L, g);
        if (rc) return rc;
    }
    return XY_OK;
}

void free_lattice(xy_lattice* L)
{
    if (!L) return;
    for (auto& g : L->graphs) cudaGraphExecDestroy(g.exec);
    for (auto& pr : L->ev_pool) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto& g : L->res_groups) cudaFree(g.d_tasks);
    for (auto& g : L->strip_groups) {
        cudaFree(g.d_tasks);
        cudaFree(g.d_b2_tasks);
    }
    cudaFree(L->thB);
    cudaFree(L->omB);
    cudaFree(L->d_cfg);
    cudaFree(L->d_call);
    if (L->h_call) cudaFreeHost(L->h_call);
    for (int i = 0; i < xy_lattice::kRing; ++i)
        if (L->call_ev[i]) cudaEventDestroy(L->call_ev[i]);
    cudaFree(L->pa.part);
    cudaFree(L->pa.count);
    cudaFree(L->d_moments);
    cudaFree(L->rec_buf);
    cudaFree(L->ccl_buf);
    for (auto& sl : L->adj_slot) cudaFree(sl.p);
    cudaFree(L->d_err);
    if (L->cap_stream) cudaStreamDestroy(L->cap_stream);
    for (int i = 0; i < xy_lattice::kBranches; ++i) {
        if (L->aux[i]) cudaStreamDestroy(L->aux[i]);
        if (L->join_ev[i]) cudaEventDestroy(L->join_ev[i]);
    }
    if (L->fork_ev) cudaEventDestroy(L->fork_ev);
    delete L;
}

}  // namespace

extern "C" {

const char* xy_last_error(void) { return g_err.c_str(); }

int xy_lattice_create(const xy_config_desc* cfg, int n_cfg, float* theta, float* omega, void* cuda_stream,
                      xy_lattice** out)
{
    if (!out) return fail(XY_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg || n_cfg <= 0 || n_cfg > 65536) return fail(XY_EINVAL, "need 1..65536 configurations");
    if (!theta || !omega) return fail(XY_EINVAL, "theta/omega must be device buffers");
    if (((uintptr_t)theta & 15) || ((uintptr_t)omega & 15)) return fail(XY_EINVAL, "theta/omega must be 16-byte aligned");
    if (!is_device_ptr(theta) || !is_device_ptr(omega)) return fail(XY_EINVAL, "theta/omega are not device memory");
    int64_t total = 0, B = 0;
    for (int c = 0; c < n_cfg; ++c) {
        const xy_config_desc& d = cfg[c];
        if (d.Lx < 4 || d.Lx % 4 != 0) return fail(XY_EINVAL, "configuration %d: Lx must be a positive multiple of 4", c);
        if (d.Ly < 1) return fail(XY_EINVAL, "configuration %d: Ly must be >= 1", c);
        if (d.n_replicas < 1 || d.n_replicas > 65535) return fail(XY_EINVAL, "configuration %d: 1..65535 replicas", c);
        if (d.init_mode < 0 || d.init_mode > 2) return fail(XY_EINVAL, "configuration %d: bad init_mode", c);
        if ((int64_t)d.Lx * d.Ly > (int64_t)1 << 30) return fail(XY_EINVAL, "configuration %d: lattice too large", c);
        if (d.cfg_id < -1 || d.cfg_id > 65535) return fail(XY_EINVAL, "configuration %d: cfg_id must be -1 or 0..65535", c);
        if (d.replica0 < 0 || (int64_t)d.replica0 + d.n_replicas > 65536)
            return fail(XY_EINVAL, "configuration %d: replica ids must stay below 65536", c);
        total += (int64_t)d.Lx * d.Ly * d.n_replicas;
        B += d.n_replicas;
    }
    if (B > ((int64_t)1 << 31) - 1) return fail(XY_EINVAL, "too many lattices");
    xy_lattice* L = new xy_lattice();
    L->n_cfg = n_cfg;
    L->B = B;
    L->total_sites = total;
    L->thA = theta;
    L->omA = omega;
    L->stream = (cudaStream_t)cuda_stream;
    L->cfg.resize(n_cfg);
    L->h_dev.resize(n_cfg);
    int64_t off = 0, b = 0;
    for (int c = 0; c < n_cfg; ++c) {
        CfgHost& h = L->cfg[c];
        h.desc = cfg[c];
        DevCfg& d = L->h_dev[c];
        std::memset(&d, 0, sizeof d);
        d.Lx = h.desc.Lx;
        d.Ly = h.desc.Ly;
        d.n_rep = h.desc.n_replicas;
        d.slot = c;
        d.noise_cfg = h.desc.cfg_id >= 0 ? h.desc.cfg_id : c;
        d.rep0 = h.desc.replica0;
        d.offset = off;
        d.N = (int64_t)h.desc.Lx * h.desc.Ly;
        d.key0 = (uint32_t)(h.desc.seed & 0xFFFFFFFFu);
        d.key1 = (uint32_t)(h.desc.seed >> 32);
        d.b_first = (int32_t)b;
        off += d.N * d.n_rep;
        b += d.n_rep;
        // the full-step omega_0 (0, or the caller's) becomes v_0 at the first step
        h.primed = false;
    }
    auto bail = [&](int code) {
        free_lattice(L);
        return code;
    };
    if (cudaMalloc(&L->thB, sizeof(float) * total) != cudaSuccess ||
        cudaMalloc(&L->omB, sizeof(float) * total) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(XY_ENOMEM, "cannot allocate the second state buffer (%lld sites)", (long long)total));
    }
    cudaError_t e;
    if ((e = cudaMalloc(&L->d_cfg, sizeof(DevCfg) * n_cfg)) != cudaSuccess ||
        (e = cudaMalloc(&L->d_call, sizeof(CallArgs))) != cudaSuccess ||
        (e = cudaMallocHost(&L->h_call, sizeof(CallArgs) * xy_lattice::kRing)) != cudaSuccess ||
        (e = cudaMalloc(&L->d_moments, sizeof(double) * 6 * n_cfg)) != cudaSuccess ||
        (e = cudaMalloc(&L->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&L->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(XY_ENOMEM, "allocation failed: %s", cudaGetErrorString(e)));
    }
    for (int i = 0; i < xy_lattice::kRing; ++i)
        if ((e = cudaEventCreateWithFlags(&L->call_ev[i], cudaEventDisableTiming)) != cudaSuccess)
            return bail(fail(XY_ECUDA, "event: %s", cudaGetErrorString(e)));
    int rc = classify(L);
    if (rc) return bail(rc);
    if ((e = cudaMalloc(&L->pa.part, sizeof(double2) * B * L->pa.max_units)) != cudaSuccess ||
        (e = cudaMalloc(&L->pa.count, sizeof(unsigned) * B)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(XY_ENOMEM, "allocation failed: %s", cudaGetErrorString(e)));
    }
    if ((e = cudaMemsetAsync(L->pa.count, 0, sizeof(unsigned) * B, L->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(L->d_moments, 0, sizeof(double) * 6 * n_cfg, L->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(L->d_err, 0, sizeof(int), L->stream)) != cudaSuccess)
        return bail(fail(XY_ECUDA, "memset: %s", cudaGetErrorString(e)));
    if ((rc = upload_cfg(L))) return bail(rc);
    for (int c = 0; c < n_cfg; ++c) {
        if ((e = launch_init(L->d_cfg, L->h_dev[c], cfg[c].init_mode, theta, omega, L->stream)) != cudaSuccess)
            return bail(fail(XY_ECUDA, "init: %s", cudaGetErrorString(e)));
        if (cfg[c].init_mode != XY_INIT_USER) ++L->launches;
    }
    *out = L;
    return XY_OK;
}

int xy_set_params(xy_lattice* L, int c, const xy_params* p)
{
    if (!L || !p) return fail(XY_EINVAL, "NULL argument");
    if (c < 0 || c >= L->n_cfg) return fail(XY_EINVAL, "configuration %d out of range", c);
    if (!(p->dt > 0.0) || !(p->eta >= 0.0) || !std::isfinite(p->J_par) || !std::isfinite(p->J_perp) ||
        !std::isfinite(p->h) || !std::isfinite(p->p) || !std::isfinite(p->q) || !std::isfinite(p->eta) ||
        !std::isfinite(p->dt))
        return fail(XY_EINVAL, "parameters must be finite with dt > 0 and eta >= 0");
    L->cfg[c].prm = *p;
    L->cfg[c].has_prm = true;
    fill_params(L->h_dev[c], *p);
    fill_e_ref(L->h_dev[c], L->cfg[c]);
    return XY_OK;
}

int xy_set_field_schedule(xy_lattice* L, int c, const int64_t* ks, const double* ss, int n_knots)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (c < 0 || c >= L->n_cfg) return fail(XY_EINVAL, "configuration %d out of range", c);
    if (n_knots < 0 || n_knots > XY_MAX_KNOTS) return fail(XY_EINVAL, "0..%d knots", XY_MAX_KNOTS);
    if (n_knots > 0 && (!ks || !ss)) return fail(XY_EINVAL, "NULL knots");
    for (int i = 0; i < n_knots; ++i) {
        if (!std::isfinite(ss[i])) return fail(XY_EINVAL, "field scales must be finite");
        if (i > 0 && ks[i] <= ks[i - 1]) return fail(XY_EINVAL, "knot steps must increase strictly");
    }
    CfgHost& h = L->cfg[c];
    h.f_n_knots = n_knots;
    for (int i = 0; i < XY_MAX_KNOTS; ++i) {
        h.f_knot_step[i] = i < n_knots ? ks[i] : 0;
        h.f_knot_s[i] = i < n_knots ? ss[i] : 0.0;
    }
    fill_field_f32(L->h_dev[c], h);
    return XY_OK;
}

int xy_set_coupling_schedule(xy_lattice* L, int c, const int64_t* ks, const double* as, const double* bs,
                             int n_knots)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (c < 0 || c >= L->n_cfg) return fail(XY_EINVAL, "configuration %d out of range", c);
    if (n_knots < 0 || n_knots > XY_MAX_KNOTS) return fail(XY_EINVAL, "0..%d knots", XY_MAX_KNOTS);
    if (n_knots > 0 && (!ks || !as || !bs)) return fail(XY_EINVAL, "NULL knots");
    for (int i = 0; i < n_knots; ++i) {
        if (!std::isfinite(as[i]) || !std::isfinite(bs[i])) return fail(XY_EINVAL, "coupling scales must be finite");
        if (i > 0 && ks[i] <= ks[i - 1]) return fail(XY_EINVAL, "knot steps must increase strictly");
    }
    CfgHost& h = L->cfg[c];
    h.c_n_knots = n_knots;
    for (int i = 0; i < XY_MAX_KNOTS; ++i) {
        h.c_knot_step[i] = i < n_knots ? ks[i] : 0;
        h.c_knot_a[i] = i < n_knots ? as[i] : 0.0;
        h.c_knot_b[i] = i < n_knots ? bs[i] : 0.0;
    }
    fill_coupling_f32(L->h_dev[c], h);
    return XY_OK;
}

int xy_set_schedule(xy_lattice* L, int c, const int64_t* ks, const double* Ts, int n_knots, int64_t n_total)
{
    if (!L || !ks || !Ts) return fail(XY_EINVAL, "NULL argument");
    if (c < 0 || c >= L->n_cfg) return fail(XY_EINVAL, "configuration %d out of range", c);
    if (n_knots < 1 || n_knots > XY_MAX_KNOTS) return fail(XY_EINVAL, "1..%d knots", XY_MAX_KNOTS);
    if (n_total < 0) return fail(XY_EINVAL, "n_steps_total must be >= 0");
    for (int i = 0; i < n_knots; ++i) {
        if (!(Ts[i] >= 0.0) || !std::isfinite(Ts[i])) return fail(XY_EINVAL, "temperatures must be finite and >= 0");
        if (i > 0 && ks[i] <= ks[i - 1]) return fail(XY_EINVAL, "knot steps must increase strictly");
    }
    CfgHost& h = L->cfg[c];
    DevCfg& d = L->h_dev[c];
    h.n_knots = n_knots;
    d.n_knots = n_knots;
    for (int i = 0; i < XY_MAX_KNOTS; ++i) {
        h.knot_step[i] = d.knot_step[i] = i < n_knots ? ks[i] : 0;
        h.knot_T[i] = d.knot_T[i] = i < n_knots ? Ts[i] : 0.0;
    }
    h.sched_kind = 0;
    h.n_total = n_total;
    d.n_total = n_total;
    fill_schedule_f32(d);
    fill_power_f32(d, h);
    h.has_sched = true;
    return XY_OK;
}

int xy_set_power_quench(xy_lattice* L, int c, double T_c, int64_t k_cross, double tau_Q, double gamma, double eps_i,
                        double eps_f, int64_t n_total)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (c < 0 || c >= L->n_cfg) return fail(XY_EINVAL, "configuration %d out of range", c);
    if (!(T_c > 0.0) || !std::isfinite(T_c)) return fail(XY_EINVAL, "T_c must be finite and > 0");
    if (!(tau_Q > 0.0) || !std::isfinite(tau_Q)) return fail(XY_EINVAL, "tau_Q must be finite and > 0");
    if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(XY_EINVAL, "gamma must be finite and > 0");
    if (!(eps_f >= -1.0) || !(eps_i >= eps_f) || !std::isfinite(eps_i))
        return fail(XY_EINVAL, "need -1 <= eps_f <= eps_i (finite)");
    if (n_total < 0) return fail(XY_EINVAL, "n_steps_total must be >= 0");
    CfgHost& h = L->cfg[c];
    DevCfg& d = L->h_dev[c];
    h.sched_kind = 1;
    const double pw[6] = {T_c, (double)k_cross, tau_Q, gamma, eps_i, eps_f};
    for (int i = 0; i < 6; ++i) h.pw[i] = pw[i];
    h.n_knots = 0;
    d.n_knots = 0;
    h.n_total = n_total;
    d.n_total = n_total;
    fill_power_f32(d, h);
    h.has_sched = true;
    return XY_OK;
}

int xy_set_path(xy_lattice* L, int path)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (path != XY_PATH_BATCHED && path != XY_PATH_PLAIN) return fail(XY_EINVAL, "unknown path %d", path);
    L->path = path;
    return XY_OK;
}

int xy_set_temporal_blocking(xy_lattice* L, int kt)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (kt < 0 || kt > 2) return fail(XY_EINVAL, "temporal blocking must be 0 (tuner), 1 or 2 steps per launch");
    L->kt_mode = kt;
    return L->tuned ? apply_kt_mode(L) : XY_OK;
}

int xy_set_adjoint_mode(xy_lattice* L, int mode)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (mode != XY_ADJOINT_AUTO && mode != XY_ADJOINT_RECOMPUTE && mode != XY_ADJOINT_BACKWARD)
        return fail(XY_EINVAL, "unknown adjoint mode %d", mode);
    L->adj_mode = mode;
    return XY_OK;
}

int xy_step_n(xy_lattice* L, int64_t n, int record_every, double* rec, int64_t t0)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (n < 0 || record_every < 0) return fail(XY_EINVAL, "n and record_every must be >= 0");
    int rc = check_ready(L);
    if (rc) return rc;
    if ((rc = prime_all(L))) return rc;
    if (n == 0) return XY_OK;
    if (record_every == 0) return advance_core(L, n, 0, nullptr, 0, false, t0);
    const int64_t R = n / record_every + 1;
    const bool dev_rec = rec && is_device_ptr(rec) && (((uintptr_t)rec & 15) == 0);
    double2* rd = nullptr;
    if (dev_rec) {
        rd = reinterpret_cast<double2*>(rec);
    } else {
        if ((rc = ensure_rec(L, (size_t)(L->B * R)))) return rc;
        rd = L->rec_buf;
    }
    if ((rc = advance_core(L, n, record_every, rd, R, true, t0))) return rc;
    if (rec && !dev_rec) {
        CK(cudaMemcpyAsync(rec, rd, sizeof(double2) * L->B * R, cudaMemcpyDeviceToHost, L->stream));
        CK(cudaStreamSynchronize(L->stream));
    }
    return XY_OK;
}

int xy_observe(xy_lattice* L, double* moments, int64_t* step_now)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    CK(cudaStreamSynchronize(L->stream));
    int err = 0;
    CK(cudaMemcpy(&err, L->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (step_now)
        for (int c = 0; c < L->n_cfg; ++c) step_now[c] = L->cfg[c].step;
    if (moments) {
        CK(cudaMemcpy(moments, L->d_moments, sizeof(double) * 6 * L->n_cfg, cudaMemcpyDeviceToHost));
        for (int i = 0; i < 6 * L->n_cfg; ++i)
            if (!std::isfinite(moments[i])) return fail(XY_ENAN, "moment %d of configuration %d is not finite", i % 6, i / 6);
    }
    if (err) return fail(err, "a device-side check failed (code %d)", err);
    return XY_OK;
}

int xy_reset_moments(xy_lattice* L)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    CK(cudaMemsetAsync(L->d_moments, 0, sizeof(double) * 6 * L->n_cfg, L->stream));
    return XY_OK;
}

int xy_omega_full(xy_lattice* L, int b_first, int b_count, float* out)
{
    if (!L || !out) return fail(XY_EINVAL, "NULL argument");
    if (b_first < 0 || b_count < 0 || b_first + (int64_t)b_count > L->B) return fail(XY_EINVAL, "lattice range out of bounds");
    if (!is_device_ptr(out) || ((uintptr_t)out & 15)) return fail(XY_EINVAL, "out must be 16-byte aligned device memory");
    int rc = check_ready(L);
    if (rc) return rc;
    if ((rc = prime_all(L))) return rc;
    set_window_idle(L);
    if ((rc = upload_cfg(L))) return rc;
    int64_t out_off = 0;
    for (int c = 0; c < L->n_cfg; ++c) {
        const DevCfg& d = L->h_dev[c];
        const int lo = std::max(b_first, d.b_first), hi = std::min(b_first + b_count, d.b_first + d.n_rep);
        if (lo >= hi) continue;
        CK(launch_omega_full(L->d_cfg, d, lo - d.b_first, hi - lo, L->thA, L->omA, out + out_off, L->stream));
        ++L->launches;
        out_off += (int64_t)(hi - lo) * d.N;
    }
    return XY_OK;
}

int xy_label_domains(xy_lattice* L, int b_first, int b_count, int32_t* labels, int64_t* hist, int64_t hist_cap,
                     int64_t* n_sizes)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    if (b_first < 0 || b_count <= 0 || b_first + (int64_t)b_count > L->B) return fail(XY_EINVAL, "lattice range out of bounds");
    if (hist && hist_cap <= 0) return fail(XY_EINVAL, "hist_cap must be > 0");
    int Lx = -1, Ly = -1;
    int64_t site0 = -1;
    for (int c = 0; c < L->n_cfg; ++c) {
        const DevCfg& d = L->h_dev[c];
        const int lo = std::max(b_first, d.b_first), hi = std::min(b_first + b_count, d.b_first + d.n_rep);
        if (lo >= hi) continue;
        if (Lx < 0) {
            Lx = d.Lx;
            Ly = d.Ly;
            site0 = d.offset + (int64_t)(lo - d.b_first) * d.N;
        } else if (Lx != d.Lx || Ly != d.Ly) {
            return fail(XY_EINVAL, "lattices of one labelling call must share Lx and Ly");
        }
    }
    const int64_t N = (int64_t)Lx * Ly;
    const bool dev_lab = labels && is_device_ptr(labels);
    const bool dev_hist = hist && is_device_ptr(hist);
    const bool dev_ns = n_sizes && is_device_ptr(n_sizes);
    const bool want = hist || n_sizes;
    // lattices per chunk: all of them unless the working memory would pass
    // 4 GB or the chunk 2^31 - 1 sites; outputs that live on the host are
    // staged behind the working memory
    const int64_t stage1 = (dev_lab ? 0 : 4 * N) + (hist && !dev_hist ? 16 * hist_cap : 0) + (want ? 8 : 0);
    const int64_t per_lat = ccl_scratch_bytes(Lx, Ly, 1, nullptr) + stage1;
    int64_t per = std::min<int64_t>(b_count, std::max<int64_t>(1, ((int64_t)4 << 30) / per_lat));
    per = std::min<int64_t>(per, std::max<int64_t>(1, INT32_MAX / N));
    while (per > 1 && ccl_scratch_bytes(Lx, Ly, (int)per, nullptr) + stage1 * per + 1024 > ((int64_t)4 << 30)) --per;
    int64_t zeroed = 0;
    const int64_t work = ccl_scratch_bytes(Lx, Ly, (int)per, &zeroed);
    const int64_t need = work + stage1 * per + 1024;
    if (need > L->ccl_bytes) {
        cudaFree(L->ccl_buf);
        L->ccl_buf = nullptr;
        L->ccl_bytes = 0;
        if (cudaMalloc(&L->ccl_buf, need) != cudaSuccess) {
            cudaGetLastError();
            L->ccl_buf = nullptr;
            return fail(XY_ENOMEM, "labelling working memory of %lld bytes", (long long)need);
        }
        L->ccl_bytes = need;
        L->ccl_clean = 0;
    }
    // the passes leave zero what they set; a larger layout than the last one,
    // or a failed call, needs the clearing done here
    if (zeroed > L->ccl_clean) CK(cudaMemsetAsync(L->ccl_buf, 0, zeroed, L->stream));
    L->ccl_clean = 0;  // until this call has ended well
    char* stage = static_cast<char*>(L->ccl_buf) + (work + 255) / 256 * 256;
    int32_t* lab = dev_lab ? nullptr : reinterpret_cast<int32_t*>(stage);
    int64_t* hs = reinterpret_cast<int64_t*>(stage + (dev_lab ? 0 : (4 * N * per + 255) / 256 * 256));
    int64_t* ns = hs + (hist && !dev_hist ? 2 * hist_cap * per : 0);
    const CclScratch scratch = ccl_scratch_carve(L->ccl_buf, Lx, Ly, (int)per);
    int rc = XY_OK;
    cudaError_t e = cudaSuccess;
    CK(cudaMemsetAsync(L->d_err, 0, sizeof(int), L->stream));
    for (int64_t b0 = 0; b0 < b_count && rc == XY_OK; b0 += per) {
        const int nl = (int)std::min<int64_t>(per, b_count - b0);
        int32_t* lab_out = dev_lab ? labels + b0 * N : lab;
        int64_t* h_out = hist ? (dev_hist ? hist + b0 * hist_cap * 2 : hs) : nullptr;
        int64_t* ns_out = n_sizes ? (dev_ns ? n_sizes + b0 : ns) : nullptr;
        cudaEvent_t span_end = nullptr;
        if ((rc = timed_begin(L, L->stream, XY_KCLASS_LABELS, &span_end))) break;
        e = launch_ccl(L->thA + site0 + b0 * N, Lx, Ly, nl, lab_out, scratch, h_out, hist ? hist_cap : 0, ns_out,
                       L->d_err, L->stream);
        if (e == cudaSuccess && span_end) e = cudaEventRecord(span_end, L->stream);
        if (e != cudaSuccess) {
            rc = fail(XY_ECUDA, "labelling: %s", cudaGetErrorString(e));
            break;
        }
        L->launches += 6;
        if (labels && !dev_lab)
            e = cudaMemcpyAsync(labels + b0 * N, lab, sizeof(int32_t) * N * nl, cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess && hist && !dev_hist)
            e = cudaMemcpyAsync(hist + b0 * hist_cap * 2, hs, sizeof(int64_t) * 2 * hist_cap * nl,
                                cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess && n_sizes && !dev_ns)
            e = cudaMemcpyAsync(n_sizes + b0, ns, sizeof(int64_t) * nl, cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess && b0 + per < b_count) e = cudaStreamSynchronize(L->stream);
        if (e != cudaSuccess) rc = fail(XY_ECUDA, "labelling: %s", cudaGetErrorString(e));
    }
    int err = 0;
    if (rc == XY_OK) {
        if (cudaMemcpyAsync(&err, L->d_err, sizeof(int), cudaMemcpyDeviceToHost, L->stream) != cudaSuccess ||
            cudaStreamSynchronize(L->stream) != cudaSuccess) {
            cudaGetLastError();
            err = XY_ECUDA;
        }
        cudaMemsetAsync(L->d_err, 0, sizeof(int), L->stream);
    }
    if (!rc && !err) L->ccl_clean = zeroed;  // else some entries were left set
    if (rc) return rc;
    if (err == XY_EINVAL) return fail(XY_EINVAL, "a lattice has more distinct domain sizes than hist_cap");
    if (err == XY_ENOMEM) return fail(XY_ENOMEM, "labelling: the list of pieces on tile edges overflowed");
    if (err) return fail(err, "labelling: a bounded union loop ran out of iterations");
    return XY_OK;
}

int xy_autocorr_time(const double* rec, int64_t n_series, int64_t R, int component, int transform, int64_t skip,
                     int64_t n, double c_window, double* out, void* cuda_stream)
{
    if (!rec || !out) return fail(XY_EINVAL, "NULL argument");
    if (n_series < 1 || n_series > INT32_MAX) return fail(XY_EINVAL, "n_series out of range");
    if (n < 2 || n > INT32_MAX / 2 || skip < 0 || R < skip + n) return fail(XY_EINVAL, "need 2 <= n and skip + n <= R");
    if (component < 0 || component > 1 || transform < 0 || transform > 3)
        return fail(XY_EINVAL, "component must be 0 or 1 and transform 0..3");
    if (!is_device_ptr(rec) || ((uintptr_t)rec & 15) != 0)
        return fail(XY_EINVAL, "rec must be a 16-byte aligned device buffer");
    if (!std::isfinite(c_window)) return fail(XY_EINVAL, "c_window must be finite");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const bool dev = is_device_ptr(out);
    double* d_out = out;
    if (!dev) {
        const cudaError_t e = cudaMalloc(&d_out, sizeof(double) * 4 * (size_t)n_series);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(XY_ENOMEM, "autocorrelation output: %s", cudaGetErrorString(e));
        }
    }
    cudaError_t e = launch_autocorr(reinterpret_cast<const double2*>(rec), n_series, R, component, transform, skip,
                                    (int)n, c_window, c_window <= 0.0 ? 1 : 0, d_out, st);
    if (e == cudaSuccess && !dev) {
        e = cudaMemcpyAsync(out, d_out, sizeof(double) * 4 * (size_t)n_series, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (!dev) cudaFree(d_out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(XY_ECUDA, "autocorrelation time: %s", cudaGetErrorString(e));
    }
    return XY_OK;
}

int xy_structure_factor(xy_lattice* L, int b_first, int b_count, int K, double rotor, double* S_par,
                        double* S_perp)
{
    if (!L || !S_par || !S_perp) return fail(XY_EINVAL, "NULL argument");
    if (b_first < 0 || b_count <= 0 || b_first + (int64_t)b_count > L->B)
        return fail(XY_EINVAL, "lattice range out of bounds");
    if (K < 1) return fail(XY_EINVAL, "K must be >= 1");
    if (!std::isfinite(rotor)) return fail(XY_EINVAL, "rotor multiplicity must be finite");
    std::vector<int64_t> off((size_t)b_count);
    std::vector<int> lx((size_t)b_count), ly((size_t)b_count);
    for (int c = 0; c < L->n_cfg; ++c) {
        const DevCfg& d = L->h_dev[c];
        const int lo = std::max(b_first, d.b_first), hi = std::min(b_first + b_count, d.b_first + d.n_rep);
        for (int b = lo; b < hi; ++b) {
            if (K > std::min(d.Lx, d.Ly)) return fail(XY_EINVAL, "K = %d exceeds min(Lx, Ly) of lattice %d", K, b);
            if (d.Lx > 8192 || d.Ly > 8192) return fail(XY_EINVAL, "structure factors need Lx, Ly <= 8192");
            off[(size_t)(b - b_first)] = d.offset + (int64_t)(b - d.b_first) * d.N;
            lx[(size_t)(b - b_first)] = d.Lx;
            ly[(size_t)(b - b_first)] = d.Ly;
        }
    }
    const bool dev = is_device_ptr(S_par) && is_device_ptr(S_perp);
    double *dp = S_par, *dq = S_perp;
    const size_t bytes = sizeof(double) * (size_t)b_count * K;
    if (!dev) {
        cudaError_t e = cudaMalloc(&dp, 2 * bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(XY_ENOMEM, "structure factor output: %s", cudaGetErrorString(e));
        }
        dq = dp + (size_t)b_count * K;
    }
    int launches = 0;
    cudaError_t e = launch_structure_factor(L->thA, off.data(), lx.data(), ly.data(), b_count, K, (float)rotor, dp, dq,
                                            &launches, L->stream);
    L->launches += launches;
    if (e == cudaSuccess && !dev) {
        e = cudaMemcpyAsync(S_par, dp, bytes, cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S_perp, dq, bytes, cudaMemcpyDeviceToHost, L->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->stream);
    }
    if (!dev) cudaFree(dp);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(XY_ECUDA, "structure factor: %s", cudaGetErrorString(e));
    }
    return XY_OK;
}

// At least `bytes` of slot i of the adjoint's working memory (reallocated
// only when it must grow; cudaFree waits for the device, so no launch still
// uses the old block).
cudaError_t adj_reserve(xy_lattice* L, int i, size_t bytes, void** out)
{
    xy_lattice::DevSlot& sl = L->adj_slot[i];
    if (bytes > sl.cap) {
        cudaFree(sl.p);
        sl.p = nullptr;
        sl.cap = 0;
        const cudaError_t e = cudaMalloc(&sl.p, bytes);
        if (e != cudaSuccess) {
            sl.p = nullptr;
            return e;
        }
        sl.cap = bytes;
    }
    *out = sl.p;
    return cudaSuccess;
}

int xy_adjoint_step_n(xy_lattice* L, int64_t n, int K, double wE, double wM, double* objective, double* grads)
{
    if (!L || !objective || !grads) return fail(XY_EINVAL, "NULL argument");
    if (n <= 0 || K <= 0) return fail(XY_EINVAL, "n and checkpoint_every must be > 0");
    int rc = check_ready(L);
    if (rc) return rc;
    const int64_t k0 = L->cfg[0].step;
    for (int c = 0; c < L->n_cfg; ++c) {
        if (L->cfg[c].step != k0) return fail(XY_EINVAL, "all configurations must be at the same step");
        if (L->cfg[c].n_total - k0 < n) return fail(XY_EINVAL, "configuration %d has fewer than n steps left", c);
    }
    if ((rc = prime_all(L))) return rc;
    const int64_t T = L->total_sites;
    const int64_t nseg = (n + K - 1) / K;
    const int64_t R_ = n + 1;
    // reverse kernel: row bands where the shape allows it (phases A and B of a
    // step in one launch), per-quad phase kernels otherwise
    struct AdjGroup {
        int Lx, Ly, H;
        uint64_t seed;
        bool wide;
        std::vector<int> cfgs;
        std::vector<BandTask> tasks;
        BandTask* d_tasks = nullptr;
        int block_base = 0;
        int64_t n_lat = 0;
    };
    std::vector<AdjGroup> adj_groups;
    std::vector<int> adj_plain;
    int n_blocks = 0;
    std::vector<int> block_base(L->n_cfg, 0);
    int sms = 148;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
    }
    for (int c = 0; c < L->n_cfg; ++c) {
        const xy_config_desc& d = L->cfg[c].desc;
        const bool wide_ok = d.Lx > 128 && d.Lx % 128 == 0 && d.Lx <= 2048 && d.Ly >= 2;
        const bool narrow_ok = d.Lx <= 128 && 32 % (d.Lx / 4) == 0 && d.Ly >= 2;
        if (!wide_ok && !narrow_ok) {
            adj_plain.push_back(c);
            continue;
        }
        AdjGroup* g = nullptr;
        for (auto& gg : adj_groups)
            if (gg.Lx == d.Lx && gg.Ly == d.Ly && gg.seed == d.seed) g = &gg;
        if (!g) {
            adj_groups.push_back(AdjGroup{d.Lx, d.Ly, 0, d.seed, wide_ok, {}, {}, nullptr, 0, 0});
            g = &adj_groups.back();
        }
        g->cfgs.push_back(c);
        g->n_lat += d.n_replicas;
    }
    // band tasks of a group for band height H: one block per band (wide), or
    // 8 warps of Lx/4-lane groups, one band per group (narrow)
    auto band_tasks = [&](const AdjGroup& g, int H, std::vector<BandTask>& out) {
        out.clear();
        const int groups = g.wide ? 1 : 32 / (g.Lx / 4);
        const int nb = g.Ly / H;
        const int per_block = g.wide ? 1 : 8 * groups;
        for (int c : g.cfgs)
            for (int r = 0; r < L->cfg[c].desc.n_replicas; ++r)
                for (int b0 = 0; b0 < nb; b0 += per_block) out.push_back(BandTask{c, r, b0, nb});
    };
    // default band height: the largest H <= 64 dividing Ly that still gives 8
    // warps per SM over the batch (each warp walks its rows serially)
    auto default_H = [&](const AdjGroup& g) {
        const int warps_per_band = g.wide ? g.Lx / 128 : 1;
        const int groups = g.wide ? 1 : 32 / (g.Lx / 4);
        int H = 1;
        for (int h : {64, 32, 16, 8, 4, 2, 1}) {
            if (g.Ly % h != 0) continue;
            H = h;
            if (g.n_lat * (g.Ly / h) * warps_per_band / groups >= (int64_t)sms * 8) break;
        }
        return H;
    };
    // states of a segment: integrated backward from the checkpoint at its end
    // inside the reverse kernel (band shapes only), or recomputed forward
    // from the checkpoint at its start and stored
    if (L->adj_mode == XY_ADJOINT_BACKWARD && (!adj_plain.empty() || adj_groups.empty()))
        return fail(XY_EINVAL, "backward integration needs shapes of the band kernels (Lx a multiple of 128 "
                               "up to 2048, or Lx <= 128 with Lx / 4 dividing 32; Ly >= 2)");
    // Undoing the damping of App. A.1 multiplies the rounding of the recovered
    // states by (1 + eta dt / 2) / (1 - eta dt / 2) per step, about
    // exp(eta dt K) over a segment of K steps.  Measured against the stored
    // recompute (64 x 64 and 256 x 64 at T_c, K = 100): the eta gradient
    // agrees to 1e-5 relative at eta dt K = 5 and only to 2e-3 at 10, so the
    // automatic choice integrates backward only up to eta dt K = 5.
    double damp = 0.0;
    for (int c = 0; c < L->n_cfg; ++c)
        damp = std::max(damp, L->h_dev[c].eta_d * L->h_dev[c].dt_d * (double)std::min<int64_t>(K, n));
    const bool back = L->adj_mode != XY_ADJOINT_RECOMPUTE && adj_plain.empty() && !adj_groups.empty() &&
                      (L->adj_mode == XY_ADJOINT_BACKWARD || damp <= kAutoBackMaxDamping);
    float *ck = nullptr, *seg = nullptr, *adjb = nullptr, *Fb = nullptr, *sbuf = nullptr;
    double2* arec = nullptr;
    double *gacc = nullptr, *mpart = nullptr;
    // the buffers are slots of the object's working memory, kept for the next call
    auto reserve = [&](int i, size_t bytes, auto** out) {
        void* p = nullptr;
        const cudaError_t e1 = adj_reserve(L, i, bytes, &p);
        *out = static_cast<std::remove_reference_t<decltype(**out)>*>(p);
        return e1;
    };
    cudaError_t e = reserve(xy_lattice::kAdjCk, sizeof(float) * 2 * T * nseg, &ck);
    // backward: two recovered states (ping-pong); recompute: the K + 1 states of a segment
    if (e == cudaSuccess && back) e = reserve(xy_lattice::kAdjSbuf, sizeof(float) * 4 * T, &sbuf);
    if (e == cudaSuccess && !back) e = reserve(xy_lattice::kAdjSeg, sizeof(float) * 2 * T * (K + 1), &seg);
    // adjoint state, double-buffered: (tb, vb) of two time levels
    if (e == cudaSuccess) e = reserve(xy_lattice::kAdjB, sizeof(float) * 4 * T, &adjb);
    if (e == cudaSuccess && !adj_plain.empty()) e = reserve(xy_lattice::kAdjFb, sizeof(float) * T, &Fb);
    if (e == cudaSuccess) e = reserve(xy_lattice::kAdjRec, sizeof(double2) * L->B * R_, &arec);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(XY_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(e));
    }
    // band height per group: tuned (timed reverse launches on zeroed buffers,
    // cached per shape and batch) or the default rule
    {
        const std::string gpu = gpu_name();
        bool zeroed = false;
        const std::vector<int> back_parts = slice_parts(adj_groups, 0, xy_lattice::kBranches + 1);
        for (auto& g : adj_groups) {
            char key[256];
            snprintf(key, sizeof key, "%s|%s|%d|%d|%lld", gpu.c_str(), back ? "adjback-sliced" : "adjband", g.Lx,
                     g.Ly, (long long)g.n_lat);
            int bh = 0, unused = 0;
            const bool big = (int64_t)g.Lx * g.Ly * g.n_lat >= ((int64_t)1 << 21);
            if (L->autotune && big && !g_tune.get(key, &bh, &unused)) {
                if (!zeroed) {
                    e = cudaMemsetAsync(back ? sbuf : seg, 0, sizeof(float) * 4 * T, L->stream);
                    if (e == cudaSuccess) e = cudaMemsetAsync(adjb, 0, sizeof(float) * 4 * T, L->stream);
                    if (e == cudaSuccess) e = cudaMemsetAsync(arec, 0, sizeof(double2) * L->B * R_, L->stream);
                    zeroed = true;
                }
                std::vector<int> cands;
                for (int h : {4, 8, 16, 32, 64})
                    if (g.Ly % h == 0) cands.push_back(h);
                std::vector<BandTask> tk;
                size_t max_tasks = 0;
                for (int h : cands) {
                    band_tasks(g, h, tk);
                    max_tasks = std::max(max_tasks, tk.size());
                }
                BandTask* d_tk = nullptr;
                double* g_tmp = nullptr;
                double* mp_tmp = nullptr;
                const int Pt = g.Ly / 4 + 1;  // partials per lattice for any candidate H >= 4
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (e == cudaSuccess) e = cudaMalloc(&d_tk, sizeof(BandTask) * max_tasks);
                if (e == cudaSuccess) e = cudaMalloc(&g_tmp, sizeof(double) * kGacc * max_tasks);
                if (e == cudaSuccess && back) e = cudaMalloc(&mp_tmp, sizeof(double) * 2 * Pt * L->B);
                if (e == cudaSuccess && back) e = cudaMemsetAsync(mp_tmp, 0, sizeof(double) * 2 * Pt * L->B, L->stream);
                // one timed reverse launch of candidate band height h on zeroed buffers
                // the backward schedule's candidates run sliced the way the
                // reverse sweep runs them
                const int n_parts = back ? back_parts[&g - adj_groups.data()] : 1;
                std::vector<int> cuts;
                auto tune_launch = [&](int h, int reps) -> cudaError_t {
                    if (back) {
                        BackArgs A{};
                        A.sched = any_sched(L, g.cfgs);
                        A.th_in = sbuf;
                        A.v_in = sbuf + T;
                        A.th_out = sbuf + 2 * T;
                        A.v_out = sbuf + 3 * T;
                        A.tb_in = adjb;
                        A.vb_in = adjb + T;
                        A.tb_out = adjb + 2 * T;
                        A.vb_out = adjb + 3 * T;
                        A.mpart = mp_tmp;
                        A.P = Pt;
                        A.rec = arec;
                        A.rec_stride = R_;
                        A.k = n >= 2 ? k0 + 1 : k0;
                        A.k0 = k0;
                        A.wE = (float)wE;
                        A.wM = (float)wM;
                        A.gacc = g_tmp;
                        return launch_sliced(L, cuts, reps, [&](cudaStream_t st, int t0, int cnt) {
                            A.block_base = t0;
                            return launch_adjoint_back(L->d_cfg, d_tk + t0, cnt, g.Lx, h, g.seed, true, A, st);
                        });
                    }
                    BandArgs R{};
                    R.theta = seg;
                    R.omega = seg + T;
                    R.tb_in = adjb;
                    R.vb_in = adjb + T;
                    R.tb_out = adjb + 2 * T;
                    R.vb_out = adjb + 3 * T;
                    R.vnext = seg + 3 * T;
                    R.rec = arec;
                    R.rec_stride = R_;
                    R.k = k0 + 1;
                    R.k0 = k0;
                    R.wE = (float)wE;
                    R.wM = (float)wM;
                    R.gacc = g_tmp;
                    cudaError_t er = cudaSuccess;
                    for (int i = 0; i < reps && er == cudaSuccess; ++i)
                        er = launch_adjoint_band(L->d_cfg, d_tk, (int)tk.size(), g.Lx, h, g.seed, R, L->stream);
                    return er;
                };
                if (e == cudaSuccess) e = cudaEventCreate(&e0);
                if (e == cudaSuccess) e = cudaEventCreate(&e1);
                float best = 1e30f;
                for (int h : cands) {
                    if (e != cudaSuccess) break;
                    band_tasks(g, h, tk);
                    cuts = cut_tasks(tk, n_parts);
                    e = cudaMemcpy(d_tk, tk.data(), sizeof(BandTask) * tk.size(), cudaMemcpyHostToDevice);
                    int reps = 2;
                    float t_best = 1e30f;
                    for (int round = 0; round < 5 && e == cudaSuccess; ++round) {
                        e = tune_launch(h, 1);
                        if (e == cudaSuccess) e = cudaEventRecord(e0, L->stream);
                        if (e == cudaSuccess) e = tune_launch(h, reps);
                        if (e == cudaSuccess) e = cudaEventRecord(e1, L->stream);
                        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                        float ms = 0.f;
                        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                        L->launches += (int64_t)(1 + reps) * (back ? (int)cuts.size() - 1 : 1);
                        t_best = std::min(t_best, ms / reps);
                        if (round == 0 && ms < 0.5f) reps = std::min(64, (int)(0.5f / std::max(ms / reps, 1e-3f)) + 1);
                    }
                    if (e == cudaSuccess && t_best < best) {
                        best = t_best;
                        bh = h;
                    }
                }
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
                cudaStreamSynchronize(L->stream);
                cudaFree(d_tk);
                cudaFree(g_tmp);
                cudaFree(mp_tmp);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return fail(XY_ECUDA, "adjoint band tuning: %s", cudaGetErrorString(e));
                }
                if (bh > 0) g_tune.put(key, bh, 0);
            }
            g.H = bh > 0 && g.Ly % bh == 0 ? bh : default_H(g);
            band_tasks(g, g.H, g.tasks);
        }
    }
    for (auto& g : adj_groups) {
        g.block_base = n_blocks;
        n_blocks += (int)g.tasks.size();
    }
    for (int c : adj_plain) {
        block_base[c] = n_blocks;
        n_blocks += adjoint_blocks(L->h_dev[c]);
    }
    {
        size_t n_tasks = 0;
        for (auto& g : adj_groups) n_tasks += g.tasks.size();
        BandTask* tasks = nullptr;
        if (e == cudaSuccess && n_tasks > 0) e = reserve(xy_lattice::kAdjTasks, sizeof(BandTask) * n_tasks, &tasks);
        for (auto& g : adj_groups) {
            if (e != cudaSuccess) break;
            g.d_tasks = tasks;
            e = cudaMemcpy(g.d_tasks, g.tasks.data(), sizeof(BandTask) * g.tasks.size(), cudaMemcpyHostToDevice);
            tasks += g.tasks.size();
        }
    }
    if (e == cudaSuccess) e = reserve(xy_lattice::kAdjGacc, sizeof(double) * kGacc * n_blocks, &gacc);
    // backward integration: per-block partial sums of M, two step slots per lattice
    int P = 1;
    for (auto& g : adj_groups) {
        const int per_block = g.wide ? 1 : 8 * (32 / (g.Lx / 4));
        P = std::max(P, (g.Ly / g.H + per_block - 1) / per_block);
    }
    if (e == cudaSuccess && back) e = reserve(xy_lattice::kAdjMpart, sizeof(double) * 2 * P * L->B, &mpart);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(XY_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(e));
    }
#define CKA(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(XY_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)
#define RCA(expr)                                                                                  \
    do {                                                                                           \
        int r_ = (expr);                                                                           \
        if (r_) return r_;                                                                         \
    } while (0)
    const size_t state_bytes = sizeof(float) * T;
    Span sp{L};
    RCA(sp.open(XY_KCLASS_ADJ_FWD));
    // ---- forward with checkpoints; observables at every step
    for (int64_t s = 0; s < nseg; ++s) {
        if (s > 0 || !back) {  // backward integration starts every segment from its end
            CKA(cudaMemcpyAsync(ck + 2 * T * s, L->thA, state_bytes, cudaMemcpyDeviceToDevice, L->stream));
            CKA(cudaMemcpyAsync(ck + 2 * T * s + T, L->omA, state_bytes, cudaMemcpyDeviceToDevice, L->stream));
        }
        const int64_t ns = std::min<int64_t>(K, n - s * K);
        RCA(advance_core(L, ns, 0, nullptr, 0, false, 0));
    }
    RCA(sp.close());
    const double inv_norm = 1.0 / ((double)L->B * (double)n);
    // ---- reverse sweep, segment by segment
    for (int c = 0; c < L->n_cfg; ++c) {
        L->h_dev[c].k_start = k0;
        L->h_dev[c].n_call = n + 1;
        L->h_dev[c].rec_first = k0;
    }
    RCA(upload_cfg(L));
    CKA(cudaMemsetAsync(adjb, 0, 4 * state_bytes, L->stream));
    CKA(cudaMemsetAsync(gacc, 0, sizeof(double) * kGacc * n_blocks, L->stream));
    int acur = 0;  // adjoint state of step k + 1 in slot acur, of step k written to slot 1 - acur
    auto tb_of = [&](int slot) { return adjb + (int64_t)slot * 2 * T; };
    auto vb_of = [&](int slot) { return adjb + (int64_t)slot * 2 * T + T; };
    if (back) {
        // ---- reverse sweep with the states integrated backward: step k0 + n
        // from the final state, then every step k from the state of k + 1 (the
        // checkpoint when k + 1 starts a segment, else the previous launch's output)
        Span sv{L};
        RCA(sv.open(XY_KCLASS_ADJ_REV));
        const float* in_th = L->thA;
        const float* in_v = L->omA;
        int sb = 0;
        // Each group's lattices run as slices on their own streams
        // (slice_groups); slice q of the whole sweep goes on stream q.
        const auto cuts = slice_groups(adj_groups, 0, xy_lattice::kBranches + 1);
        int n_slices = 0;
        for (const auto& c : cuts) n_slices += (int)c.size() - 1;
        const int n_aux = std::min(n_slices, xy_lattice::kBranches + 1) - 1;
        if (n_aux > 0) {
            const cudaError_t e0 = ensure_branch_streams(L);
            if (e0 != cudaSuccess) return fail(XY_ECUDA, "reverse streams: %s", cudaGetErrorString(e0));
        }
        if (n_aux > 0) CKA(cudaEventRecord(L->fork_ev, L->stream));
        for (int i = 0; i < n_aux; ++i) CKA(cudaStreamWaitEvent(L->aux[i], L->fork_ev, 0));
        for (int64_t k = k0 + n; k >= k0; --k) {
            const bool bk = k < k0 + n;
            const int64_t m = k + 1 - k0;
            if (bk && m < n && m % K == 0) {
                in_th = ck + 2 * T * (m / K);
                in_v = in_th + T;
            }
            float* out_th = sbuf + 2 * T * sb;
            int q = 0;  // slice of the sweep
            for (auto& g : adj_groups) {
                BackArgs A{};
                A.sched = any_sched(L, g.cfgs);
                A.th_in = in_th;
                A.v_in = in_v;
                A.th_out = bk ? out_th : nullptr;
                A.v_out = bk ? out_th + T : nullptr;
                A.tb_in = tb_of(acur);
                A.vb_in = vb_of(acur);
                A.tb_out = tb_of(1 - acur);
                A.vb_out = vb_of(1 - acur);
                A.mpart = mpart;
                A.P = P;
                A.rec = arec;
                A.rec_stride = R_;
                A.k = k;
                A.k0 = k0;
                A.wE = (float)wE;
                A.wM = (float)wM;
                A.gacc = gacc;
                const auto& c = cuts[&g - adj_groups.data()];
                for (size_t p = 0; p + 1 < c.size(); ++p, ++q) {
                    A.block_base = g.block_base + c[p];
                    CKA(launch_adjoint_back(L->d_cfg, g.d_tasks + c[p], c[p + 1] - c[p], g.Lx, g.H, g.seed, bk, A,
                                            q == 0 ? L->stream : L->aux[(q - 1) % n_aux]));
                    ++L->launches;
                }
            }
            if (bk) {
                in_th = out_th;
                in_v = out_th + T;
                sb ^= 1;
            }
            acur = 1 - acur;
        }
        for (int i = 0; i < n_aux; ++i) {
            CKA(cudaEventRecord(L->join_ev[i], L->aux[i]));
            CKA(cudaStreamWaitEvent(L->stream, L->join_ev[i], 0));
        }
        RCA(sv.close());
    }
    // reverse step k from the states at segment slot i
    auto rev_step = [&](int64_t k, int64_t i) -> int {
        const float* th = seg + 2 * T * i;
        const float* om = seg + 2 * T * i + T;
        for (auto& g : adj_groups) {
            BandArgs R{};
            R.theta = th;
            R.omega = om;
            R.tb_in = tb_of(acur);
            R.vb_in = vb_of(acur);
            R.tb_out = tb_of(1 - acur);
            R.vb_out = vb_of(1 - acur);
            // v_{k+1} is slot i + 1 of the segment for every step but k0 + n
            R.vnext = k < k0 + n ? seg + 2 * T * (i + 1) + T : nullptr;
            R.rec = arec;
            R.rec_stride = R_;
            R.k = k;
            R.k0 = k0;
            R.wE = (float)wE;
            R.wM = (float)wM;
            R.gacc = gacc;
            R.block_base = g.block_base;
            CK(launch_adjoint_band(L->d_cfg, g.d_tasks, (int)g.tasks.size(), g.Lx, g.H, g.seed, R, L->stream));
            ++L->launches;
        }
        for (int c : adj_plain) {
            // per-quad kernels update in place: carry this configuration's adjoint
            // state into the output slot first, then phase A and phase B of step k
            const DevCfg& d = L->h_dev[c];
            const size_t off = (size_t)d.offset, cnt = (size_t)d.N * d.n_rep;
            CK(cudaMemcpyAsync(tb_of(1 - acur) + off, tb_of(acur) + off, sizeof(float) * cnt,
                               cudaMemcpyDeviceToDevice, L->stream));
            CK(cudaMemcpyAsync(vb_of(1 - acur) + off, vb_of(acur) + off, sizeof(float) * cnt,
                               cudaMemcpyDeviceToDevice, L->stream));
            AdjArgs a{};
            a.theta = th;
            a.omega = om;
            a.tb = tb_of(1 - acur);
            a.vb = vb_of(1 - acur);
            a.Fb = Fb;
            a.rec = arec;
            a.rec_stride = R_;
            a.k = k;
            a.k0 = k0;
            a.k_end = k0 + n;
            a.wE = wE;
            a.wM = wM;
            a.inv_norm = inv_norm;
            a.gacc = gacc;
            CK(launch_adjoint_phase_a(L->d_cfg, d, block_base[c], a, L->stream));
            CK(launch_adjoint_phase_b(L->d_cfg, d, a, L->stream));
            L->launches += 2;
        }
        acur = 1 - acur;
        return XY_OK;
    };
    for (int64_t s = back ? -1 : nseg - 1; s >= 0; --s) {
        const int64_t ks = k0 + s * K;
        const int64_t Ks = std::min<int64_t>(K, n - s * K);
        const int64_t n_states = (s == nseg - 1) ? Ks + 1 : Ks;  // the last segment also needs k0 + n
        Span spr{L};
        RCA(spr.open(XY_KCLASS_ADJ_RECOMP));
        CKA(cudaMemcpyAsync(seg, ck + 2 * T * s, 2 * state_bytes, cudaMemcpyDeviceToDevice, L->stream));
        {
            // step ks + i runs as local step i (k = k0 + i + (ks - k0)) from slot i
            // into slot i + 1
            CallArgs ca{};
            ca.k_shift = ks - k0;
            ca.fixed_parity = 1;
            RCA(upload_call(L, ca));
        }
        // Ks steps: slots 1 .. Ks (the next checkpoint, or k0 + n) are written
        for (int64_t i = 0; i < Ks; ++i) {
            Buffers buf{seg + 2 * T * i, seg + 2 * T * i + T, seg + 2 * T * (i + 1), seg + 2 * T * (i + 1) + T};
            if (L->path == XY_PATH_PLAIN) {
                for (int c = 0; c < L->n_cfg; ++c) {
                    CKA(launch_plain_step(L->d_cfg, L->h_dev[c], i, buf, L->d_call, L->pa, 1, L->stream));
                    ++L->launches;
                }
            } else {
                for (auto& g : L->res_groups) {
                    CKA(launch_resident_step(L->d_cfg, g.d_tasks, (int)g.tasks.size(), g.Lx, g.Ly, g.threads, g.csize, g.seed, i, 1,
                                             buf, L->d_call, L->stream));
                    ++L->launches;
                }
                for (auto& g : L->strip_groups) {
                    CKA(launch_strip_step(L->d_cfg, g.d_tasks, (int)g.tasks.size(), g.H, g.variant, 0,
                                          group_sched(L, g), g.seed, i, buf, L->d_call, L->pa, L->stream));
                    ++L->launches;
                }
                for (int c : L->plain_cfgs) {
                    CKA(launch_plain_step(L->d_cfg, L->h_dev[c], i, buf, L->d_call, L->pa, 1, L->stream));
                    ++L->launches;
                }
            }
        }
        // M of the segment's states, for the signs (and values) of |M_k|
        CKA(launch_segment_m(L->d_cfg, L->n_cfg, L->B, seg, T, (int)n_states, arec, R_, ks - k0, L->stream));
        ++L->launches;
        RCA(spr.close());
        Span sv{L};
        RCA(sv.open(XY_KCLASS_ADJ_REV));
        for (int64_t i = n_states - 1; i >= 0; --i) RCA(rev_step(ks + i, i));
        RCA(sv.close());
    }
    std::vector<double2> hrec((size_t)L->B * R_);
    CKA(cudaMemcpyAsync(hrec.data(), arec, sizeof(double2) * L->B * R_, cudaMemcpyDeviceToHost, L->stream));
    std::vector<double> hg((size_t)kGacc * n_blocks);
    CKA(cudaMemcpyAsync(hg.data(), gacc, sizeof(double) * kGacc * n_blocks, cudaMemcpyDeviceToHost, L->stream));
    CKA(cudaStreamSynchronize(L->stream));
    std::vector<double> acc((size_t)kGacc * L->n_cfg, 0.0);
    for (auto& g : adj_groups)
        for (size_t t = 0; t < g.tasks.size(); ++t)
            for (int q = 0; q < kGacc; ++q)
                acc[kGacc * g.tasks[t].cfg + q] += hg[(size_t)(g.block_base + t) * kGacc + q];
    for (int c : adj_plain) {
        const int nb = adjoint_blocks(L->h_dev[c]);
        for (int bk = 0; bk < nb; ++bk)
            for (int q = 0; q < kGacc; ++q) acc[kGacc * c + q] += hg[(size_t)(block_base[c] + bk) * kGacc + q];
    }
    // objective: w_E E summed by the reverse sweep, w_M |M_k| from the forward records
    double obj = 0.0;
    for (int c = 0; c < L->n_cfg; ++c) obj += acc[kGacc * c + 6];
    for (int64_t b = 0; b < L->B; ++b)
        for (int64_t k = 1; k <= n; ++k) obj += wM * std::fabs(hrec[b * R_ + k].x);
    *objective = obj * inv_norm;
    for (int c = 0; c < L->n_cfg; ++c) {
        const xy_params& p = L->cfg[c].prm;
        const double bb = 1.0 / (1.0 + 0.5 * p.eta * p.dt);
        const double* ac = &acc[kGacc * c];
        grads[4 * c + 0] = ac[0] * inv_norm;
        grads[4 * c + 1] = ac[1] * inv_norm;
        grads[4 * c + 2] = ac[2] * inv_norm;
        grads[4 * c + 3] = (0.5 * p.dt * (ac[3] - bb * bb * ac[4]) + ac[5]) * inv_norm;
    }
    // restore the idle window
    set_window_idle(L);
    RCA(upload_cfg(L));
#undef CKA
#undef RCA
    return XY_OK;
}

// ---- snapshots
namespace {
struct SnapHeader {
    char magic[8];
    int64_t version, n_cfg, total, B;
};
struct SnapCfg {
    xy_config_desc desc;
    xy_params prm;
    int64_t has_prm, has_sched, n_knots, n_total, step, primed;
    int64_t knot_step[XY_MAX_KNOTS];
    double knot_T[XY_MAX_KNOTS];
    int64_t sched_kind;
    double pw[6];
    int64_t f_n_knots;
    int64_t f_knot_step[XY_MAX_KNOTS];
    double f_knot_s[XY_MAX_KNOTS];
    int64_t c_n_knots;
    int64_t c_knot_step[XY_MAX_KNOTS];
    double c_knot_a[XY_MAX_KNOTS];
    double c_knot_b[XY_MAX_KNOTS];
};
}  // namespace

int xy_save(xy_lattice* L, void* buf, size_t* size)
{
    if (!L || !size) return fail(XY_EINVAL, "NULL argument");
    const size_t need = sizeof(SnapHeader) + sizeof(SnapCfg) * L->n_cfg + sizeof(double) * 6 * L->n_cfg +
                        sizeof(float) * 2 * L->total_sites;
    if (!buf) {
        *size = need;
        return XY_OK;
    }
    if (*size < need) return fail(XY_EINVAL, "buffer too small: %zu < %zu", *size, need);
    int rc = check_ready(L);
    if (rc) return rc;
    if ((rc = prime_all(L))) return rc;
    char* p = (char*)buf;
    SnapHeader hd{};
    std::memcpy(hd.magic, "XYLATT1", 8);
    hd.version = 4;
    hd.n_cfg = L->n_cfg;
    hd.total = L->total_sites;
    hd.B = L->B;
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    for (int c = 0; c < L->n_cfg; ++c) {
        const CfgHost& h = L->cfg[c];
        SnapCfg s{};
        s.desc = h.desc;
        s.prm = h.prm;
        s.has_prm = h.has_prm;
        s.has_sched = h.has_sched;
        s.n_knots = h.n_knots;
        s.sched_kind = h.sched_kind;
        for (int i = 0; i < 6; ++i) s.pw[i] = h.pw[i];
        s.n_total = h.n_total;
        s.step = h.step;
        s.primed = h.primed;
        for (int i = 0; i < XY_MAX_KNOTS; ++i) {
            s.knot_step[i] = h.knot_step[i];
            s.knot_T[i] = h.knot_T[i];
            s.f_knot_step[i] = h.f_knot_step[i];
            s.f_knot_s[i] = h.f_knot_s[i];
        }
        s.f_n_knots = h.f_n_knots;
        for (int i = 0; i < XY_MAX_KNOTS; ++i) {
            s.c_knot_step[i] = h.c_knot_step[i];
            s.c_knot_a[i] = h.c_knot_a[i];
            s.c_knot_b[i] = h.c_knot_b[i];
        }
        s.c_n_knots = h.c_n_knots;
        std::memcpy(p, &s, sizeof s);
        p += sizeof s;
    }
    CK(cudaMemcpyAsync(p, L->d_moments, sizeof(double) * 6 * L->n_cfg, cudaMemcpyDeviceToHost, L->stream));
    p += sizeof(double) * 6 * L->n_cfg;
    CK(cudaMemcpyAsync(p, L->thA, sizeof(float) * L->total_sites, cudaMemcpyDeviceToHost, L->stream));
    p += sizeof(float) * L->total_sites;
    CK(cudaMemcpyAsync(p, L->omA, sizeof(float) * L->total_sites, cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    *size = need;
    return XY_OK;
}

int xy_load(xy_lattice* L, const void* buf, size_t size)
{
    if (!L || !buf) return fail(XY_EINVAL, "NULL argument");
    const size_t need = sizeof(SnapHeader) + sizeof(SnapCfg) * L->n_cfg + sizeof(double) * 6 * L->n_cfg +
                        sizeof(float) * 2 * L->total_sites;
    if (size < need) return fail(XY_EINVAL, "snapshot too small");
    const char* p = (const char*)buf;
    SnapHeader hd;
    std::memcpy(&hd, p, sizeof hd);
    p += sizeof hd;
    if (std::memcmp(hd.magic, "XYLATT1", 8) != 0 || hd.version != 4) return fail(XY_EINVAL, "not a snapshot");
    if (hd.n_cfg != L->n_cfg || hd.total != L->total_sites || hd.B != L->B)
        return fail(XY_EINVAL, "snapshot shape does not match this lattice object");
    std::vector<SnapCfg> sc(L->n_cfg);
    for (int c = 0; c < L->n_cfg; ++c) {
        std::memcpy(&sc[c], p, sizeof(SnapCfg));
        p += sizeof(SnapCfg);
        const xy_config_desc& a = sc[c].desc;
        const xy_config_desc& b = L->cfg[c].desc;
        if (a.Lx != b.Lx || a.Ly != b.Ly || a.n_replicas != b.n_replicas || a.seed != b.seed ||
            a.cfg_id != b.cfg_id || a.replica0 != b.replica0)
            return fail(XY_EINVAL, "snapshot configuration %d does not match", c);
    }
    CK(cudaStreamSynchronize(L->stream));
    for (int c = 0; c < L->n_cfg; ++c) {
        CfgHost& h = L->cfg[c];
        const SnapCfg& s = sc[c];
        h.prm = s.prm;
        h.has_prm = s.has_prm != 0;
        h.has_sched = s.has_sched != 0;
        h.n_knots = (int)s.n_knots;
        h.sched_kind = (int)s.sched_kind;
        for (int i = 0; i < 6; ++i) h.pw[i] = s.pw[i];
        h.n_total = s.n_total;
        h.step = s.step;
        h.primed = s.primed != 0;
        DevCfg& d = L->h_dev[c];
        if (h.has_prm) fill_params(d, h.prm);
        d.n_knots = h.n_knots;
        d.n_total = h.n_total;
        for (int i = 0; i < XY_MAX_KNOTS; ++i) {
            h.knot_step[i] = d.knot_step[i] = s.knot_step[i];
            h.knot_T[i] = d.knot_T[i] = s.knot_T[i];
        }
        fill_schedule_f32(d);
        fill_power_f32(d, h);
        h.f_n_knots = (int)s.f_n_knots;
        for (int i = 0; i < XY_MAX_KNOTS; ++i) {
            h.f_knot_step[i] = s.f_knot_step[i];
            h.f_knot_s[i] = s.f_knot_s[i];
        }
        h.c_n_knots = (int)s.c_n_knots;
        for (int i = 0; i < XY_MAX_KNOTS; ++i) {
            h.c_knot_step[i] = s.c_knot_step[i];
            h.c_knot_a[i] = s.c_knot_a[i];
            h.c_knot_b[i] = s.c_knot_b[i];
        }
        fill_field_f32(d, h);
        fill_coupling_f32(d, h);
    }
    CK(cudaMemcpyAsync(L->d_moments, p, sizeof(double) * 6 * L->n_cfg, cudaMemcpyHostToDevice, L->stream));
    p += sizeof(double) * 6 * L->n_cfg;
    CK(cudaMemcpyAsync(L->thA, p, sizeof(float) * L->total_sites, cudaMemcpyHostToDevice, L->stream));
    p += sizeof(float) * L->total_sites;
    CK(cudaMemcpyAsync(L->omA, p, sizeof(float) * L->total_sites, cudaMemcpyHostToDevice, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    set_window_idle(L);
    return upload_cfg(L);
}

int xy_synchronize(xy_lattice* L)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    CK(cudaStreamSynchronize(L->stream));
    return XY_OK;
}

int64_t xy_kernel_launches(xy_lattice* L) { return L ? L->launches : -1; }

int xy_set_autotune(xy_lattice* L, int on)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    L->autotune = on != 0;
    return XY_OK;
}

int xy_autotune(xy_lattice* L)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    int rc = check_ready(L);
    if (rc) return rc;
    if ((rc = prime_all(L))) return rc;
    L->tuned = false;
    const bool saved = L->autotune;
    L->autotune = true;
    rc = autotune_lattice(L);
    L->autotune = saved;
    return rc;
}

int xy_set_kernel_timing(xy_lattice* L, int on)
{
    if (!L) return fail(XY_EINVAL, "NULL lattice");
    CK(cudaStreamSynchronize(L->stream));
    L->timing = on != 0;
    L->ev_used = 0;
    return XY_OK;
}

int xy_kernel_timing(xy_lattice* L, double* ms, int64_t* launches)
{
    if (!L || !ms || !launches) return fail(XY_EINVAL, "NULL argument");
    CK(cudaStreamSynchronize(L->stream));
    for (int c = 0; c < XY_KCLASS_COUNT; ++c) {
        ms[c] = 0.0;
        launches[c] = 0;
    }
    for (size_t i = 0; i < L->ev_used; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, L->ev_pool[i].first, L->ev_pool[i].second));
        ms[L->ev_class[i]] += t;
        launches[L->ev_class[i]] += 1;
    }
    return XY_OK;
}

void xy_lattice_destroy(xy_lattice* L)
{
    if (!L) return;
    cudaStreamSynchronize(L->stream);
    free_lattice(L);
}

int xy_debug_noise(uint64_t seed, int cfg, int replica, int64_t k, int tag, int64_t n_quads, uint32_t* words,
                   float* gauss, void* stream)
{
    if (n_quads < 0 || cfg < 0 || cfg > 65535 || replica < 0 || replica > 65535 || tag < 0 || tag > 255)
        return fail(XY_EINVAL, "bad noise coordinates");
    CK(launch_debug_noise(seed, cfg, replica, k, tag, n_quads, words, gauss, (cudaStream_t)stream));
    return XY_OK;
}

int xy_debug_gauss4(const uint32_t* words, int64_t n_quads, float c, float* out, void* stream)
{
    if (n_quads < 0 || (n_quads > 0 && (!words || !out))) return fail(XY_EINVAL, "bad arguments");
    if ((((uintptr_t)words | (uintptr_t)out) & 15) != 0) return fail(XY_EINVAL, "words and out must be 16-byte aligned");
    CK(launch_debug_gauss4(words, n_quads, c, out, (cudaStream_t)stream));
    return XY_OK;
}

int xy_debug_philox(const uint32_t* counters, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out, void* stream)
{
    if (n < 0 || (n > 0 && (!counters || !out))) return fail(XY_EINVAL, "bad arguments");
    CK(launch_debug_philox(counters, k0, k1, n, out, (cudaStream_t)stream));
    return XY_OK;
}

// The slicing plan of the concurrent branches, through the same functions
// as the stepper and the reverse sweep (host only, no device call).
struct DbgTask {
    int32_t cfg, rep;
};
struct DbgGroup {
    int64_t n_lat;
    std::vector<DbgTask> tasks;
};

int xy_debug_slice_parts(const int64_t* n_lat, int n_groups, int fixed, int budget, int* parts)
{
    if (n_groups < 0 || (n_groups > 0 && (!n_lat || !parts)) || fixed < 0 || budget < 1)
        return fail(XY_EINVAL, "bad slicing arguments");
    std::vector<DbgGroup> groups(n_groups);
    for (int g = 0; g < n_groups; ++g) {
        if (n_lat[g] < 0) return fail(XY_EINVAL, "negative lattice count");
        groups[g].n_lat = n_lat[g];
    }
    const std::vector<int> p = slice_parts(groups, fixed, budget);
    for (int g = 0; g < n_groups; ++g) parts[g] = p[g];
    return XY_OK;
}

int xy_debug_slice_cuts(const int32_t* lattice_of_task, int n_tasks, int parts, int* cuts, int* n_cuts)
{
    if (n_tasks < 0 || (n_tasks > 0 && !lattice_of_task) || parts < 1 || !cuts || !n_cuts)
        return fail(XY_EINVAL, "bad slicing arguments");
    std::vector<DbgTask> tk(n_tasks);
    for (int i = 0; i < n_tasks; ++i) {
        if (i > 0 && lattice_of_task[i] < lattice_of_task[i - 1])
            return fail(XY_EINVAL, "tasks must be grouped by lattice in ascending order");
        tk[i] = DbgTask{lattice_of_task[i], 0};
    }
    const std::vector<int> c = cut_tasks(tk, parts);
    for (size_t i = 0; i < c.size(); ++i) cuts[i] = c[i];
    *n_cuts = (int)c.size();
    return XY_OK;
}

}  // extern "C"
