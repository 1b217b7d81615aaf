// Host runtime and C ABI of libsph (declared in include/sph.h).
//
// The context owns every device buffer, issues all work on one stream, and
// replays one captured step as a CUDA graph in sph_run.  Particle counts,
// the time step and the simulated time live on the device, so a captured
// step stays valid while particles enter and leave.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "sph.h"
#include "sph_internal.cuh"

using namespace sph;

namespace {

thread_local std::string g_init_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct sph_ctx {
    sph_params prm;
    std::string err;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int cap = 0, bcap = 0;
    size_t tsz = 4;              // sizeof(T)
    Grid grid{};
    PhysT<float> Pf{};
    PhysT<double> Pd{};
    Inflow inf{};
    std::vector<DevBuf> allocs;

    // device state
    Scalars *sc = nullptr;       // device scalars
    Scalars *hsc = nullptr;      // pinned host mirror
    void *raw[8] = {}, *srt[8] = {};   // pos, vel, drho, drc, mass, type, id, disp
    void *H0n = nullptr, *H1n = nullptr, *H0h = nullptr, *H1h = nullptr;
    double2 *posh = nullptr;
    void *C = nullptr, *CX = nullptr, *nhat = nullptr, *nvec = nullptr;
    void *acc = nullptr, *dr = nullptr;
    // with surface tension: pair sums of the full list walk (ax, ay, drho/dt,
    // Eq. 31 term), the normal bound G_a, and the colour range of each cell
    void *accN = nullptr, *gsum = nullptr;
    uint2 *crange = nullptr;
    void *stats = nullptr;       // sph_stats scratch: 6 FP64 sums + 3 counters
    CellSort cs{};
    NList nl{};
    uint2 *cellSE = nullptr, *cellSE_b = nullptr;
    void *bH = nullptr;
    double2 *bpos = nullptr;
    uint32_t *parent = nullptr;
    uint8_t *flag = nullptr;
    double *layer_y = nullptr;

    // host-side boundary particles (static)
    std::vector<double> bx, by, bnx, bny;

    // pinned host staging of state transfers (sized for the capacity on
    // first use, kept until the context is destroyed)
    unsigned char *pin = nullptr;
    size_t pin_bytes = 0;

    // derivative rows valid for raw[0, n_eval)
    long long n_eval = 0;
    bool csf_valid = false;

    // step graphs: [0] with a cell build, [1] reusing the last build
    cudaGraph_t graph[2] = {};
    cudaGraphExec_t gexec[2] = {};
    bool graph_dirty = true;
    unsigned long long graph_gen = 0;   // counts changes that invalidate captured steps
    // learned-surrogate step scratch: SPH accelerations and density rates at
    // the step start, residual sums, saved particle count
    void *sg_an = nullptr, *sg_drn = nullptr, *sg_sums = nullptr, *sg_t0 = nullptr;
    MpScratchHandle *sg_net = nullptr;   // the network's inference scratch
    double *sg_hsum = nullptr;           // pinned host copy of the residual sums
    bool sg_reuse = false;               // this step starts from the last evaluation
    double sg_dT = 0.0;                  // this step's span
    // the evaluation ending the last accepted surrogate step can start the
    // next one while the cell-build and step counters are those recorded
    bool sg_ready = false;
    long long sg_builds = -1, sg_step = -1;

    // tuning: lanes per particle in the pair sweeps, longest cell-build cadence
    int lanes = 4, cadence = 1;
    int start_form = SPH_START_GATED;   // how a step at cadence > 1 picks its start
    bool force_full = true;      // host: the next step must rebuild the cells
    bool hsc_fresh = false;      // hsc mirrors the device scalars (synchronised)

    // step graph whose start (rebuild / reuse) is chosen on the device
    cudaGraph_t cgraph = nullptr;
    cudaGraphExec_t cexec = nullptr;
    bool no_ticks = false;

    // autotune snapshot of the raw state
    void *snap[8] = {};
    size_t snap_n = 0;
    Scalars snap_sc{};

    // per-kernel timing: an event before each kernel group of a step
    // one event set per kind of step (0: with a cell build, 1: reusing it)
    bool prof = false, prof_pending = false, ticking = false;
    std::vector<cudaEvent_t> pev[2];
    std::vector<const char *> pname[2];
    int pidx[2] = {0, 0};
    int tick_kind = 0, last_kind = 0;
    std::map<std::string, std::pair<double, long long>> ptot;
    std::vector<std::string> report_names;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static sph_status fail(sph_ctx *c, sph_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_init_error = buf;
    return st;
}

static sph_status cuda_check(sph_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SPH_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call, what)                                              \
    do {                                                            \
        sph_status _s = cuda_check(c, (call), (what));              \
        if (_s != SPH_OK) return _s;                                \
    } while (0)

static void *dalloc(sph_ctx *c, size_t bytes, cudaError_t &e) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) {
        cudaMemset(p, 0, bytes);
        c->allocs.push_back({p, bytes});
    }
    return p;
}

// All host<->device copies go through the context's stream and wait for it,
// so they are ordered with the kernels whatever kind of stream it is.
static cudaError_t copy_sync(sph_ctx *c, void *dst, const void *src, size_t bytes,
                             cudaMemcpyKind kind) {
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, c->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

static sph_status status_from_err(sph_ctx *c, unsigned err) {
    if (err & ERR_NONFINITE) return fail(c, SPH_ERR_NONFINITE, "non-finite acceleration or density rate");
    if (err & ERR_SKIN)
        return fail(c, SPH_ERR_SKIN, "a particle moved more than skin/2 within a step; reduce dt or raise skin_over_h");
    if (err & ERR_CAPACITY) return fail(c, SPH_ERR_CAPACITY, "inflow exceeded the particle capacity");
    if (err & ERR_TIMEOUT) return fail(c, SPH_ERR_TIMEOUT, "a bounded device loop hit its iteration limit");
    if (err & ERR_NODT) return fail(c, SPH_ERR_STATE, "adaptive time step without fluid particles");
    if (err & ERR_NLIST)
        return fail(c, SPH_ERR_CAPACITY, "a particle has more neighbours than its list holds");
    if (err & ERR_BOUNDS)
        return fail(c, SPH_ERR_STATE, "a particle index out of range (bounds-check build)");
    return SPH_OK;
}

template <class T> static State<T> state_of(void *const a[8]) {
    State<T> s;
    s.pos = (double2 *)a[0];
    s.vel = (typename Vec<T>::v2 *)a[1];
    s.drho = (T *)a[2];
    s.drc = (T *)a[3];
    s.mass = (T *)a[4];
    s.type = (uint8_t *)a[5];
    s.id = (uint32_t *)a[6];
    s.disp = (typename Vec<T>::v2 *)a[7];
    return s;
}

// A cell offset as the records of precision T store it (fixed point in FP32).
template <class T> static T store_off(double off, double sc);
template <> float store_off<float>(double off, double sc) {
    int v = off_fixed(off, sc);
    float f;
    memcpy(&f, &v, sizeof f);
    return f;
}
template <> double store_off<double>(double off, double) { return off; }

template <class T> static PhysT<T> make_phys(const sph_params &p, const Grid &g, bool walls) {
    PhysT<T> P{};
    double h = p.h_over_dx * p.dx;
    double H = 2.0 * h, H2 = H * H;
    double R = 1.5 * h, R2 = R * R;
    double band = sizeof(T) == 4 ? 2e-5 : 1e-12;
    const double pi = 3.14159265358979323846;
    double kap = p.kernel == SPH_KERNEL_CUBIC ? 10.0 / (7.0 * pi) : 7.0 / (64.0 * pi);
    P.kernel = p.kernel;
    P.csf = p.sigma > 0.0;
    P.walls = walls;
    P.gamma7 = p.gamma == 7.0;
    P.summation = p.density == SPH_DENSITY_SUMMATION;
    P.h = (T)h;
    P.inv_h = (T)(1.0 / h);
    P.H2lo = (T)(H2 * (1.0 - band));
    P.H2hi = (T)(H2 * (1.0 + band));
    P.R15lo = (T)(R2 * (1.0 - band));
    P.R15hi = (T)(R2 * (1.0 + band));
    P.H2d = H2;
    P.R15d = R2;
    double RL = 2.0 * h + p.skin_over_h * h;
    P.RL2hi = (T)(RL * RL * (1.0 + band));
    P.half_skin2 = 0.25 * (p.skin_over_h * h) * (p.skin_over_h * h);
    P.half_skin = (T)(0.5 * p.skin_over_h * h);
    P.sc = (T)g.sc;
    P.wn = (T)(kap / (h * h));
    P.gn = (T)(p.kernel == SPH_KERNEL_CUBIC ? kap / (h * h * h * h) : -10.0 * kap / (h * h * h * h));
    P.W0 = (T)(p.kernel == SPH_KERNEL_CUBIC ? kap / (h * h) : 16.0 * kap / (h * h));
    P.rho0 = (T)p.rho0;
    P.inv_rho0 = (T)(1.0 / p.rho0);
    P.B = (T)(p.rho0 * p.c0 * p.c0 / p.gamma);
    P.gamma = (T)p.gamma;
    P.c0 = (T)p.c0;
    P.half_gm1 = (T)(0.5 * (p.gamma - 1.0));
    P.alpha_h = (T)(p.alpha * h);
    P.eta2 = (T)(p.eta2_over_h2 * h * h);
    P.sigma = (T)p.sigma;
    P.eps_n = (T)(p.eps_n_times_h / h);
    P.gx = (T)p.gx;
    P.gy = (T)p.gy;
    P.wall_A = (T)(p.wall_A_coef * p.c0 * p.c0 / h);
    P.wall_db = (T)(p.wall_db_over_dx * p.dx);
    P.inv_wall_db = (T)(1.0 / (p.wall_db_over_dx * p.dx));
    P.wall_h0 = (T)p.wall_h0;
    P.inv_wall_h0 = (T)(p.wall_h0 > 0.0 ? 1.0 / p.wall_h0 : 0.0);
    P.two_h = (T)(2.0 * h);
    P.c0_inv = (T)(1.0 / p.c0);
    P.ufx = (T)p.u_frame_x;
    P.ufy = (T)p.u_frame_y;
    P.ufx_d = p.u_frame_x;
    P.ufy_d = p.u_frame_y;
    // Verlet lists stay exact while every pair separation has changed by
    // less than the skin.  Measuring the displacement since the build
    // relative to any common frame keeps that bound (|d_a - d_b| <= |d_a - w|
    // + |d_b - w|), so without walls it is taken in the velocity frame, and a
    // jet translating at U does not force rebuilds.  Particles may then leave
    // their build-time cell: offsets up to two cells beyond it keep the FP32
    // pair test about 16 times inside the band where pairs are redone in
    // FP64.  Wall contacts are found by walking the build-time cells, so with
    // walls the absolute displacement counts and a particle stays within
    // skin/2 of its cell.
    double half_skin = 0.5 * p.skin_over_h * h;
    P.dfx = walls ? T(0) : (T)p.u_frame_x;
    P.dfy = walls ? T(0) : (T)p.u_frame_y;
    P.cell_lo = store_off<T>(walls ? -half_skin : -2.0 * g.sc, g.sc);
    P.cell_hi = store_off<T>(walls ? g.sc + half_skin : 3.0 * g.sc, g.sc);
    P.off_unit = (T)(g.sc / OFF_ONE);
    P.off_scale = (T)(OFF_ONE / g.sc);
    P.courant = p.courant;
    P.dt_fixed = p.dt_fixed;
    return P;
}

static void cell_of(const Grid &g, double x, double y, int &cx, int &cy) {
    cx = (int)std::floor((x - g.xmin) * g.inv_sc) + 1;
    cy = (int)std::floor((y - g.ymin) * g.inv_sc) + 1;
    cx = std::min(std::max(cx, 1), g.ncx - 2);
    cy = std::min(std::max(cy, 1), g.ncy - 2);
}

// ---------------------------------------------------------------------------
// step assembly
// ---------------------------------------------------------------------------
template <class T> struct Ops {
    static const PhysT<T> &phys(sph_ctx *c);
};
template <> const PhysT<float> &Ops<float>::phys(sph_ctx *c) { return c->Pf; }
template <> const PhysT<double> &Ops<double>::phys(sph_ctx *c) { return c->Pd; }

template <class T> static Hot<T> hot_n(sph_ctx *c) {
    return Hot<T>{(typename Vec<T>::v4 *)c->H0n, (typename Vec<T>::v4 *)c->H1n,
                  (double2 *)c->srt[0]};
}
template <class T> static Hot<T> hot_h(sph_ctx *c) {
    return Hot<T>{(typename Vec<T>::v4 *)c->H0h, (typename Vec<T>::v4 *)c->H1h, c->posh};
}
template <class T> static Csf<T> csf_of(sph_ctx *c) {
    return Csf<T>{(T *)c->C, (typename Vec<T>::v4 *)c->CX, (typename Vec<T>::v2 *)c->nhat,
                  (typename Vec<T>::v2 *)c->nvec};
}
static Boundary bd_of(sph_ctx *c) {
    Boundary b;
    b.n = (int)c->bx.size();
    b.cellSE = c->cellSE_b;
    b.bh = c->bH;
    b.pos = c->bpos;
    return b;
}

// Records a timing event before the next kernel group when profiling is on.
// Events are created up front by sph_profile (not during a capture) and are
// recorded as external event nodes when the step is captured into a graph.
static void tick(sph_ctx *c, const char *name) {
    int k = c->tick_kind;
    if (!c->prof || !c->ticking || c->no_ticks || c->pidx[k] >= (int)c->pev[k].size()) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->stream, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(c->pev[k][c->pidx[k]], c->stream, cudaEventRecordExternal);
    else
        cudaEventRecord(c->pev[k][c->pidx[k]], c->stream);
    c->pname[k][c->pidx[k]] = name;
    ++c->pidx[k];
}

// hash -> sort -> cell ranges -> gather into cell order (evaluation-n records)
template <class T> static const uint32_t *enqueue_sort(sph_ctx *c, int gate = GATE_ALWAYS) {
    const PhysT<T> &P = Ops<T>::phys(c);
    State<T> raw = state_of<T>(c->raw), srt = state_of<T>(c->srt);
    tick(c, "cell_sort");
    launch_cell_sort<T>(c->grid, raw, c->sc, c->cs, c->cap, c->stream, gate);
    tick(c, "reorder");
    launch_reorder<T>(P, c->grid, c->sc, c->cs, raw, srt, hot_n<T>(c), c->cap, c->stream, gate);
    const uint32_t *key = c->cs.key;
    return key;
}

// Neighbour list of evaluation n (the colour comes with the evaluation's
// pair sweep).
template <class T>
static void enqueue_build(sph_ctx *c, const uint32_t *key, int gate = GATE_ALWAYS) {
    const PhysT<T> &P = Ops<T>::phys(c);
    tick(c, "list");
    // the list build walks ~61 candidates of the 3x3 cells per particle; it
    // takes at least 4 lanes per particle whatever the sweeps use
    launch_build<T>(std::max(c->lanes, 4), false, P, c->grid, c->sc, c->cellSE, key,
                    hot_n<T>(c), c->nl, csf_of<T>(c), c->cap, c->stream, gate);
}

// Eq. 6 densities of the records `hot` (a no-op with Eq. 7).
// drho_out: where the state keeps the density (null at the half step).
template <class T>
static void enqueue_density(sph_ctx *c, const Hot<T> &hot, T *drho_out, int gate = GATE_ALWAYS) {
    const PhysT<T> &P = Ops<T>::phys(c);
    if (!P.summation) return;
    State<T> srt = state_of<T>(c->srt);
    tick(c, "density");
    launch_density<T>(c->lanes, P, c->sc, c->nl, hot, srt.mass, srt.type, drho_out, c->cap,
                      c->stream, gate);
}

// One evaluation of the right-hand sides on the records `hot` and the lists
// of the last build, ending in mode 0 (store), 1 (store + time-step minimum)
// or 2 (corrector, writing the next records to nH0 / nH1).  Without surface
// tension one list walk does everything; with it, one full walk (colour and
// the state-only pair sums), the normal (skip: not walked where it provably
// stays below the filter threshold) and the surface terms with the mode's end.
template <class T>
static void enqueue_eval(sph_ctx *c, const Hot<T> &hot, int mode, bool skip,
                         typename Vec<T>::v4 *nH0 = nullptr, typename Vec<T>::v4 *nH1 = nullptr) {
    const PhysT<T> &P = Ops<T>::phys(c);
    State<T> raw = state_of<T>(c->raw), srt = state_of<T>(c->srt);
    auto *acc = (typename Vec<T>::v2 *)c->acc;
    T *dr = (T *)c->dr;
    const uint32_t *key = c->cs.key;
    const char *fname = mode == 2 ? "forces_correct" : "forces";
    if (!P.csf) {
        tick(c, fname);
        launch_forces<T>(c->lanes, mode, P, c->grid, c->inf, c->sc, c->nl, key, hot,
                         csf_of<T>(c), bd_of(c), srt, raw, acc, dr, c->cap, c->stream, nH0, nH1);
        return;
    }
    auto *accN = (typename Vec<T>::v4 *)c->accN;
    T *gsum = (T *)c->gsum;
    tick(c, mode == 2 ? "pairsum_correct" : "pairsum");
    cudaMemsetAsync(c->crange, 0xFF, (size_t)c->grid.ncells * sizeof(uint2), c->stream);
    launch_pairsum<T>(c->lanes, P, c->grid, c->sc, c->nl, key, hot, csf_of<T>(c), bd_of(c),
                      srt.type, accN, gsum, c->crange, c->cap, c->stream, mode == 1);
    tick(c, "normal");
    launch_normal<T>(c->lanes, P, c->sc, c->nl, hot, csf_of<T>(c), c->cap, c->stream, key,
                     skip ? gsum : nullptr, c->crange, c->grid.ncx);
    tick(c, fname);
    launch_surface<T>(c->lanes, mode, P, c->grid, c->inf, c->sc, c->nl, hot, csf_of<T>(c), srt,
                      raw, accN, acc, dr, c->cap, c->stream, nH0, nH1);
}

// The two ways a step starts.  Rebuild: hash, sort, reorder and neighbour
// list.  Reuse: the particles keep the order, cells and lists of the last
// rebuild (exact while no particle has moved more than skin/2 since, which
// the kernels check), and the state and records of evaluation n are those
// the last corrector wrote in place, so the start is only the Eq. 6
// densities (when used).  gate: GATE_ALWAYS when the host chose the start;
// otherwise the start's kernels run only on the steps whose device flag
// selects it.
template <class T> static void enqueue_cells(sph_ctx *c, bool full, int gate = GATE_ALWAYS) {
    State<T> srt = state_of<T>(c->srt);
    Hot<T> hn = hot_n<T>(c);
    const uint32_t *key = c->cs.key;
    if (full) {
        enqueue_sort<T>(c, gate);
        enqueue_build<T>(c, key, gate);
    }
    enqueue_density<T>(c, hn, srt.drho, gate);
}

// The rest of a step (Sec. 2-8): evaluation at n, predictor, evaluation at
// n+1/2 with the corrector, inflow and time advance.
template <class T> static void enqueue_rest(sph_ctx *c) {
    const PhysT<T> &P = Ops<T>::phys(c);
    State<T> raw = state_of<T>(c->raw), srt = state_of<T>(c->srt);
    auto *acc = (typename Vec<T>::v2 *)c->acc;
    T *dr = (T *)c->dr;
    Hot<T> hn = hot_n<T>(c), hh = hot_h<T>(c);
    enqueue_eval<T>(c, hn, 1, true);
    tick(c, "predict");
    launch_predict<T>(P, c->inf, c->sc, srt, hn.H0, acc, dr, hh, c->cap, c->stream);
    enqueue_density<T>(c, hh, (T *)nullptr);
    enqueue_eval<T>(c, hh, 2, true, hn.H0, hn.H1);
    tick(c, "spawn");
    launch_spawn<T>(P, c->inf, c->sc, raw, c->layer_y, c->cap, c->cadence, c->stream);
}

template <class T> static void enqueue_step(sph_ctx *c, bool full) {
    c->tick_kind = full ? 0 : 1;
    c->last_kind = c->tick_kind;
    c->pidx[c->tick_kind] = 0;
    c->ticking = true;
    enqueue_cells<T>(c, full);
    enqueue_rest<T>(c);
    tick(c, nullptr);
    c->ticking = false;
    c->prof_pending = c->prof;
}

// sph_evaluate: a fresh cell build and one evaluation, with the normal walked
// for every particle (its CSF intermediates are returned exactly).
template <class T> static void enqueue_evaluate(sph_ctx *c) {
    State<T> srt = state_of<T>(c->srt);
    const uint32_t *key = enqueue_sort<T>(c);
    Hot<T> hn = hot_n<T>(c);
    enqueue_build<T>(c, key);
    enqueue_density<T>(c, hn, srt.drho);
    enqueue_eval<T>(c, hn, 0, false);
}

template <class T> static void enqueue_breakup(sph_ctx *c) {
    const uint32_t *key = enqueue_sort<T>(c);
    State<T> srt = state_of<T>(c->srt);
    launch_breakup<T>(Ops<T>::phys(c), c->grid, c->sc, c->cellSE, key, hot_n<T>(c), srt.type,
                      c->parent, c->flag, c->cap, c->stream);
}

static void step_any(sph_ctx *c, bool full) {
    if (c->tsz == 4) enqueue_step<float>(c, full); else enqueue_step<double>(c, full);
}

// Host-side choice of the next step's kind: rebuild when forced, when the
// device scalars are not known (not synchronised since the last step), or
// when the last step asked for it.  Forcing also sets the device flag that
// the graph's own decision reads.
static bool host_next_is_full(sph_ctx *c) {
    bool full = c->force_full || !c->hsc_fresh || c->hsc->need_full;
    if (c->force_full) {
        cudaMemsetAsync(&c->sc->need_full, 0x01, sizeof(int), c->stream);
        c->force_full = false;
    }
    c->hsc_fresh = false;
    return full;
}

static sph_status pull_scalars(sph_ctx *c) {
    CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream),
       "copy scalars");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    c->hsc_fresh = true;
    return SPH_OK;
}

static sph_status push_scalars(sph_ctx *c) {
    CK(cudaMemcpyAsync(c->sc, c->hsc, sizeof(Scalars), cudaMemcpyHostToDevice, c->stream),
       "copy scalars");
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return SPH_OK;
}

// Adds the per-kernel durations of the most recent step to the totals.
static void collect_profile(sph_ctx *c) {
    if (!c->prof_pending) return;
    c->prof_pending = false;
    int kind = c->last_kind;
    for (int k = 0; k + 1 < c->pidx[kind]; ++k) {
        if (!c->pname[kind][k]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->pev[kind][k], c->pev[kind][k + 1]) != cudaSuccess) {
            cudaGetLastError();   // do not leave the failure as the sticky last error
            continue;
        }
        auto &e = c->ptot[c->pname[kind][k]];
        e.first += ms;
        e.second += 1;
    }
}

static sph_status after_work(sph_ctx *c, const char *what) {
    CK(cudaGetLastError(), what);
    sph_status s = pull_scalars(c);
    if (s != SPH_OK) return s;
    collect_profile(c);
    return status_from_err(c, c->hsc->err);
}

// The captured step graphs (the context's own and any ensemble's) no longer
// match the context's parameters or tuning.
static void mark_graph_dirty(sph_ctx *c) {
    c->graph_dirty = true;
    ++c->graph_gen;
}

static void rebuild_phys(sph_ctx *c) {
    bool walls = !c->bx.empty();
    c->Pf = make_phys<float>(c->prm, c->grid, walls);
    c->Pd = make_phys<double>(c->prm, c->grid, walls);
    c->Pf.cap = c->Pd.cap = (int)c->cap;
    c->Pf.err = c->Pd.err = c->sc ? &c->sc->err : nullptr;
    mark_graph_dirty(c);
}

static sph_status upload_boundary(sph_ctx *c) {
    size_t nb = c->bx.size();
    std::vector<uint32_t> key(nb);
    for (size_t k = 0; k < nb; ++k) {
        int cx, cy;
        cell_of(c->grid, c->bx[k], c->by[k], cx, cy);
        key[k] = grid_key(c->grid, cx, cy);
    }
    std::vector<size_t> ord(nb);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return key[a] < key[b]; });
    std::vector<uint2> se(c->grid.ncells, make_uint2(0, 0));
    std::vector<double2> pos(nb);
    std::vector<double> hd(4 * nb);
    for (size_t r = 0; r < nb; ++r) {
        size_t k = ord[r];
        uint32_t kk = key[k];
        if (r == 0 || key[ord[r - 1]] != kk) se[kk].x = (unsigned)r;
        if (r + 1 == nb || key[ord[r + 1]] != kk) se[kk].y = (unsigned)(r + 1);
        int cx, cy;
        grid_cell(c->grid, kk, cx, cy);
        double xo = c->bx[k] - (c->grid.xmin + (double)(cx - 1) * c->grid.sc);
        double yo = c->by[k] - (c->grid.ymin + (double)(cy - 1) * c->grid.sc);
        hd[4 * r + 0] = xo;
        hd[4 * r + 1] = yo;
        hd[4 * r + 2] = c->bnx[k];
        hd[4 * r + 3] = c->bny[k];
        pos[r] = make_double2(c->bx[k], c->by[k]);
    }
    if (c->tsz == 4) {
        std::vector<float> hf(4 * nb);
        for (size_t q = 0; q < 4 * nb; ++q)
            hf[q] = q % 4 < 2 ? store_off<float>(hd[q], c->grid.sc) : (float)hd[q];
        CK(copy_sync(c, c->bH, hf.data(), 4 * nb * sizeof(float), cudaMemcpyHostToDevice), "upload boundary");
    } else {
        CK(copy_sync(c, c->bH, hd.data(), 4 * nb * sizeof(double), cudaMemcpyHostToDevice), "upload boundary");
    }
    CK(copy_sync(c, c->bpos, pos.data(), nb * sizeof(double2), cudaMemcpyHostToDevice), "upload boundary");
    CK(copy_sync(c, c->cellSE_b, se.data(), se.size() * sizeof(uint2), cudaMemcpyHostToDevice),
       "upload boundary cells");
    rebuild_phys(c);
    return SPH_OK;
}

// Runs f(lo, hi) over [0, n) in up to 8 host threads of at least `grain`
// items each (a million-particle state crosses the ABI in milliseconds); f
// must not throw.
// A chunk whose thread cannot be started runs on the calling thread.
template <class F> static void host_for(size_t n, F &&f, size_t grain = (size_t)1 << 16) {
    unsigned hw = std::thread::hardware_concurrency();
    size_t nt = std::min<size_t>(std::min<size_t>(hw ? hw : 1u, 8u), (n + grain - 1) / grain);
    if (nt <= 1) {
        f((size_t)0, n);
        return;
    }
    size_t chunk = (n + nt - 1) / nt;
    std::vector<std::thread> th;
    th.reserve(nt);
    for (size_t k = 1; k < nt; ++k) {
        size_t lo = k * chunk, hi = std::min(n, lo + chunk);
        if (lo >= hi) continue;
        try {
            th.emplace_back([&f, lo, hi] { f(lo, hi); });
        } catch (...) {
            f(lo, hi);
        }
    }
    f((size_t)0, std::min(n, chunk));
    for (auto &t : th) t.join();
}

static size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

// Bytes of pinned staging one particle needs in a state transfer: position,
// velocity, density, mass, type, id, acceleration, density rate (each array
// padded to 16 bytes).
static size_t staging_bytes(const sph_ctx *c, size_t n) {
    size_t ts = c->tsz;
    return al16(n) + al16(16 * n) + 2 * al16(2 * n * ts) + 3 * al16(n * ts) + al16(4 * n);
}

// The context's pinned staging buffer, at least `bytes` long (grown to the
// capacity's needs on first use).  Callers synchronise the stream before they
// return, so no copy from or to it is in flight when it is replaced.
static unsigned char *staging(sph_ctx *c, size_t bytes, cudaError_t &e) {
    e = cudaSuccess;
    if (bytes <= c->pin_bytes) return c->pin;
    size_t want = std::max(bytes, staging_bytes(c, (size_t)c->cap));
    if (c->pin) cudaFreeHost(c->pin);
    c->pin = nullptr;
    c->pin_bytes = 0;
    e = cudaMallocHost((void **)&c->pin, want);
    if (e != cudaSuccess) {
        c->pin = nullptr;
        return nullptr;
    }
    c->pin_bytes = want;
    return c->pin;
}

// Upload n particles into raw[at, at+n): converted into the device layout in
// the pinned staging, then one asynchronous copy per array and one wait for
// all of them (also when one fails, so that no copy from the staging is in
// flight when the call returns).
static sph_status upload_particles(sph_ctx *c, long long at, long long n, const double *x,
                                   const double *y, const double *u, const double *v,
                                   const double *rho, const double *mass,
                                   const unsigned char *type, const unsigned *id) {
    if (n == 0) return SPH_OK;
    const size_t N = (size_t)n, ts = c->tsz;
    const size_t o_pos = 0, o_vel = al16(16 * N), o_dr = o_vel + al16(2 * N * ts),
                 o_m = o_dr + al16(N * ts), o_ty = o_m + al16(N * ts), o_id = o_ty + al16(N),
                 total = o_id + al16(4 * N);
    cudaError_t e;
    unsigned char *pin = staging(c, total, e);
    CK(e, "pinned staging");
    const double ufx = c->prm.u_frame_x, ufy = c->prm.u_frame_y, rho0 = c->prm.rho0;
    double2 *pos = (double2 *)(pin + o_pos);
    host_for(N, [&](size_t lo, size_t hi) {
        for (size_t i = lo; i < hi; ++i) pos[i] = make_double2(x[i], y[i]);
        if (ts == 4) {
            float *vel = (float *)(pin + o_vel), *dr = (float *)(pin + o_dr),
                  *m = (float *)(pin + o_m);
            for (size_t i = lo; i < hi; ++i) {
                vel[2 * i] = (float)(u[i] - ufx);
                vel[2 * i + 1] = (float)(v[i] - ufy);
                dr[i] = (float)(rho[i] - rho0);
                m[i] = (float)mass[i];
            }
        } else {
            double *vel = (double *)(pin + o_vel), *dr = (double *)(pin + o_dr),
                   *m = (double *)(pin + o_m);
            for (size_t i = lo; i < hi; ++i) {
                vel[2 * i] = u[i] - ufx;
                vel[2 * i + 1] = v[i] - ufy;
                dr[i] = rho[i] - rho0;
                m[i] = mass[i];
            }
        }
        memcpy(pin + o_ty + lo, type + lo, hi - lo);
        memcpy(pin + o_id + 4 * lo, id + lo, 4 * (hi - lo));
    });
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
    cudaStream_t st = c->stream;
    cudaError_t err = cudaMemcpyAsync((double2 *)c->raw[0] + at, pin + o_pos, 16 * N, h2d, st);
    if (!err) err = cudaMemcpyAsync((char *)c->raw[1] + 2 * at * ts, pin + o_vel, 2 * N * ts, h2d, st);
    if (!err) err = cudaMemcpyAsync((char *)c->raw[2] + at * ts, pin + o_dr, N * ts, h2d, st);
    if (!err) err = cudaMemsetAsync((char *)c->raw[3] + at * ts, 0, N * ts, st);
    if (!err) err = cudaMemsetAsync((char *)c->raw[7] + 2 * at * ts, 0, 2 * N * ts, st);
    if (!err) err = cudaMemcpyAsync((char *)c->raw[4] + at * ts, pin + o_m, N * ts, h2d, st);
    if (!err) err = cudaMemcpyAsync((uint8_t *)c->raw[5] + at, pin + o_ty, N, h2d, st);
    if (!err) err = cudaMemcpyAsync((uint32_t *)c->raw[6] + at, pin + o_id, 4 * N, h2d, st);
    cudaError_t es = cudaStreamSynchronize(st);
    CK(err ? err : es, "upload");
    return SPH_OK;
}

static bool inside(const sph_ctx *c, double x, double y) {
    return x >= c->prm.xmin && x < c->prm.xmax && y >= c->prm.ymin && y < c->prm.ymax;
}

template <class T> static void to_double(const std::vector<unsigned char> &src, size_t i, size_t comp,
                                         size_t ncomp, double &out) {
    T v;
    memcpy(&v, &src[(i * ncomp + comp) * sizeof(T)], sizeof(T));
    out = (double)v;
}

static double rd(const sph_ctx *c, const std::vector<unsigned char> &b, size_t i, size_t comp, size_t ncomp) {
    double o;
    if (c->tsz == 4) to_double<float>(b, i, comp, ncomp, o); else to_double<double>(b, i, comp, ncomp, o);
    return o;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *sph_last_error(const sph_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

sph_status sph_init(const sph_params *p, sph_ctx **out) {
    if (!out) return fail(nullptr, SPH_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, SPH_ERR_ARG, "params is NULL");
    const sph_params &q = *p;
    if (q.kernel != SPH_KERNEL_CUBIC && q.kernel != SPH_KERNEL_WENDLAND)
        return fail(nullptr, SPH_ERR_ARG, "unknown kernel %d", q.kernel);
    if (q.precision != SPH_FP32 && q.precision != SPH_FP64)
        return fail(nullptr, SPH_ERR_ARG, "unknown precision %d", q.precision);
    if (!(q.dx > 0 && q.h_over_dx > 0 && q.rho0 > 0 && q.c0 > 0 && q.gamma >= 1.0))
        return fail(nullptr, SPH_ERR_ARG, "dx, h_over_dx, rho0, c0 must be > 0 and gamma >= 1");
    if (!(q.alpha >= 0 && q.eta2_over_h2 > 0 && q.sigma >= 0 && q.eps_n_times_h > 0))
        return fail(nullptr, SPH_ERR_ARG, "alpha, sigma >= 0; eta2_over_h2, eps_n_times_h > 0 required");
    if (!(q.courant > 0 && q.courant <= 1.0 && q.dt_fixed >= 0))
        return fail(nullptr, SPH_ERR_ARG, "courant in (0, 1] and dt_fixed >= 0 required");
    if (!(q.xmax > q.xmin && q.ymax > q.ymin)) return fail(nullptr, SPH_ERR_ARG, "empty domain box");
    if (q.density != SPH_DENSITY_CONTINUITY && q.density != SPH_DENSITY_SUMMATION)
        return fail(nullptr, SPH_ERR_ARG, "unknown density mode %d", q.density);
    if (!(q.skin_over_h >= 0.1 && q.skin_over_h <= 2.0))
        return fail(nullptr, SPH_ERR_ARG, "skin_over_h must lie in [0.1, 2]");
    if (!(q.capacity >= 1 && q.capacity <= (1ll << 28)))
        return fail(nullptr, SPH_ERR_ARG, "capacity must lie in [1, 2^28]");
    if (!(q.boundary_capacity >= 0 && q.boundary_capacity <= (1ll << 26)))
        return fail(nullptr, SPH_ERR_ARG, "boundary_capacity must lie in [0, 2^26]");
    if (!(std::isfinite(q.u_frame_x) && std::isfinite(q.u_frame_y)))
        return fail(nullptr, SPH_ERR_ARG, "u_frame must be finite");
    if (!(q.wall_A_coef >= 0 && q.wall_h0 >= 0 && q.wall_db_over_dx > 0))
        return fail(nullptr, SPH_ERR_ARG, "wall parameters out of range");
    double h = q.h_over_dx * q.dx, skin = q.skin_over_h * h;
    double db = q.wall_db_over_dx * q.dx;
    if (q.boundary_capacity > 0 && std::sqrt(4 * h * h + db * db) > 2 * h + 0.5 * skin)
        return fail(nullptr, SPH_ERR_ARG, "skin too small for the wall-force reach");
    double sc = 2.0 * h + skin;
    double ncx = std::floor((q.xmax - q.xmin) / sc) + 3, ncy = std::floor((q.ymax - q.ymin) / sc) + 3;
    if (ncx * ncy > 6.7e7) return fail(nullptr, SPH_ERR_ARG, "cell grid too large (%.3g cells)", ncx * ncy);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, SPH_ERR_CUDA, "no CUDA device available");
    if (q.device < 0 || q.device >= ndev) return fail(nullptr, SPH_ERR_ARG, "device %d out of range", q.device);

    sph_ctx *c = new (std::nothrow) sph_ctx();
    if (!c) return fail(nullptr, SPH_ERR_OOM, "host allocation failed");
    c->prm = q;
    c->cap = (int)q.capacity;
    c->bcap = (int)q.boundary_capacity;
    c->tsz = q.precision == SPH_FP32 ? 4 : 8;
    Grid &g = c->grid;
    g.xmin = q.xmin; g.ymin = q.ymin; g.xmax = q.xmax; g.ymax = q.ymax;
    g.sc = sc; g.inv_sc = 1.0 / sc;
    g.ncx = (int)ncx; g.ncy = (int)ncy;
    grid_finish(g);

    auto bail = [&](sph_status s) { sph_destroy(c); return s; };
    cudaError_t e = cudaSetDevice(q.device);
    if (e != cudaSuccess) { fail(nullptr, SPH_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e)); return bail(SPH_ERR_CUDA); }
    if (q.cuda_stream) {
        c->stream = (cudaStream_t)q.cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { fail(nullptr, SPH_ERR_CUDA, "stream: %s", cudaGetErrorString(e)); return bail(SPH_ERR_CUDA); }
        c->own_stream = true;
    }
    size_t N = (size_t)c->cap, ts = c->tsz, NB = (size_t)std::max(c->bcap, 1);
    size_t sizes[8] = {16, 2 * ts, ts, ts, ts, 1, 4, 2 * ts};
    for (int k = 0; k < 8; ++k) {
        c->raw[k] = dalloc(c, N * sizes[k], e); if (e) break;
        c->srt[k] = dalloc(c, N * sizes[k], e); if (e) break;
    }
    if (!e) c->H0n = dalloc(c, N * 4 * ts, e);
    if (!e) c->H1n = dalloc(c, N * 4 * ts, e);
    if (!e) c->H0h = dalloc(c, N * 4 * ts, e);
    if (!e) c->H1h = dalloc(c, N * 4 * ts, e);
    if (!e) c->posh = (double2 *)dalloc(c, N * 16, e);
    if (!e) c->C = dalloc(c, N * ts, e);
    if (!e) c->CX = dalloc(c, N * 4 * ts, e);
    if (!e) c->nhat = dalloc(c, N * 2 * ts, e);
    if (!e) c->nvec = dalloc(c, N * 2 * ts, e);
    if (!e) c->acc = dalloc(c, N * 2 * ts, e);
    if (!e) c->dr = dalloc(c, N * ts, e);
    if (!e) c->accN = dalloc(c, N * 4 * ts, e);
    if (!e) c->gsum = dalloc(c, N * ts, e);
    if (!e) c->crange = (uint2 *)dalloc(c, (size_t)g.ncells * 8, e);
    c->cs.nscan = (int)(((size_t)g.ncells + SCAN_CELLS - 1) / SCAN_CELLS);
    if (!e) c->cs.knew = (uint32_t *)dalloc(c, N * 4, e);
    if (!e) c->cs.count = (uint32_t *)dalloc(c, (size_t)g.ncells * 4, e);
    if (!e) c->cs.tmp = (uint32_t *)dalloc(c, N * 4, e);
    if (!e) c->cs.key = (uint32_t *)dalloc(c, N * 4, e);
    if (!e) c->cs.bsum = (uint32_t *)dalloc(c, (size_t)c->cs.nscan * 4, e);
    if (!e) c->cellSE = (uint2 *)dalloc(c, (size_t)g.ncells * 8, e);
    c->cs.cellSE = c->cellSE;
    if (!e) c->nl.e = (uint32_t *)dalloc(c, N * LIST_SLOTS * 4, e);
    if (!e) c->nl.cnt = (uint32_t *)dalloc(c, N * 4, e);
    if (!e) c->cellSE_b = (uint2 *)dalloc(c, (size_t)g.ncells * 8, e);
    if (!e) c->bH = dalloc(c, NB * 4 * ts, e);
    if (!e) c->bpos = (double2 *)dalloc(c, NB * 16, e);
    if (!e) c->parent = (uint32_t *)dalloc(c, N * 4, e);
    if (!e) c->flag = (uint8_t *)dalloc(c, N, e);
    if (!e) c->layer_y = (double *)dalloc(c, 1024 * sizeof(double), e);
    if (!e) c->sc = (Scalars *)dalloc(c, sizeof(Scalars), e);
    if (e) { fail(nullptr, e == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA, "device allocation: %s", cudaGetErrorString(e)); return bail(SPH_ERR_OOM); }
    e = cudaDeviceSynchronize();
    if (e) { fail(nullptr, SPH_ERR_CUDA, "device synchronize: %s", cudaGetErrorString(e)); return bail(SPH_ERR_CUDA); }
    e = cudaMallocHost(&c->hsc, sizeof(Scalars));
    if (e) { fail(nullptr, SPH_ERR_OOM, "pinned allocation: %s", cudaGetErrorString(e)); return bail(SPH_ERR_OOM); }
    memset(c->hsc, 0, sizeof(Scalars));
    for (int k = 0; k < RED_SLOTS; ++k) {
        c->hsc->dtmin_f[k] = 0x7f7f7f7fu;
        c->hsc->dtmin_d[k] = 0x7f7f7f7f7f7f7f7full;
    }
    if (push_scalars(c) != SPH_OK) { g_init_error = c->err; return bail(SPH_ERR_CUDA); }
    rebuild_phys(c);
    *out = c;
    return SPH_OK;
}

void sph_destroy(sph_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 2; ++k)
        for (auto e : c->pev[k]) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
        if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
    }
    for (auto p : c->snap) if (p) cudaFree(p);
    mpnn_scratch_free(c->sg_net);
    if (c->sg_hsum) cudaFreeHost(c->sg_hsum);
    if (c->cexec) cudaGraphExecDestroy(c->cexec);
    if (c->cgraph) cudaGraphDestroy(c->cgraph);
    for (auto &b : c->allocs) cudaFree(b.p);
    if (c->hsc) cudaFreeHost(c->hsc);
    if (c->pin) cudaFreeHost(c->pin);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

sph_status sph_add_particles(sph_ctx *c, long long n, const double *x, const double *y,
                             const double *u, const double *v, const double *rho,
                             const double *mass, const unsigned char *type, const double *nx,
                             const double *ny) {
    if (!c) return SPH_ERR_ARG;
    c->sg_ready = false;
    try {
        if (n < 0) return fail(c, SPH_ERR_ARG, "n < 0");
        if (n == 0) return SPH_OK;
        if (!x || !y || !type) return fail(c, SPH_ERR_ARG, "x, y and type are required");
        long long nf = 0, nb = 0;
        for (long long i = 0; i < n; ++i) {
            if (type[i] == SPH_BOUNDARY) ++nb;
            else if (type[i] == SPH_FLUID || type[i] == SPH_BUFFER) ++nf;
            else return fail(c, SPH_ERR_ARG, "particle %lld has unknown type %d", i, (int)type[i]);
            if (!std::isfinite(x[i]) || !std::isfinite(y[i]))
                return fail(c, SPH_ERR_ARG, "particle %lld has a non-finite position", i);
            if (!inside(c, x[i], y[i])) return fail(c, SPH_ERR_ARG, "particle %lld lies outside the domain", i);
        }
        if (nf > 0 && (!u || !v || !rho || !mass)) return fail(c, SPH_ERR_ARG, "u, v, rho and mass are required");
        if (nb > 0 && (!nx || !ny)) return fail(c, SPH_ERR_ARG, "boundary particles need nx, ny");
        for (long long i = 0; i < n; ++i) {
            if (type[i] == SPH_BOUNDARY) continue;
            if (!(rho[i] > 0) || !(mass[i] > 0) || !std::isfinite(u[i]) || !std::isfinite(v[i]))
                return fail(c, SPH_ERR_ARG, "particle %lld needs rho, mass > 0 and a finite velocity", i);
        }
        sph_status s = pull_scalars(c);
        if (s) return s;
        long long n0 = c->hsc->n;
        if (n0 + nf > c->cap) return fail(c, SPH_ERR_CAPACITY, "capacity %d exceeded", c->cap);
        if ((long long)c->bx.size() + nb > c->bcap)
            return fail(c, SPH_ERR_CAPACITY, "boundary capacity %d exceeded", c->bcap);
        if (nf > 0) {
            std::vector<double> fx, fy, fu, fv, fr, fm;
            std::vector<unsigned char> ft;
            std::vector<unsigned> fid;
            unsigned nid = c->hsc->next_id;
            for (long long i = 0; i < n; ++i) {
                if (type[i] == SPH_BOUNDARY) continue;
                fx.push_back(x[i]); fy.push_back(y[i]); fu.push_back(u[i]); fv.push_back(v[i]);
                fr.push_back(rho[i]); fm.push_back(mass[i]); ft.push_back(type[i]);
                fid.push_back(nid++);
            }
            s = upload_particles(c, n0, nf, fx.data(), fy.data(), fu.data(), fv.data(), fr.data(),
                                 fm.data(), ft.data(), fid.data());
            if (s) return s;
            c->hsc->n = (int)(n0 + nf);
            c->hsc->next_id = nid;
            c->force_full = true;
            s = push_scalars(c);
            if (s) return s;
            c->n_eval = 0;
            c->csf_valid = false;
        }
        if (nb > 0) {
            for (long long i = 0; i < n; ++i) {
                if (type[i] != SPH_BOUNDARY) continue;
                double l = std::hypot(nx[i], ny[i]);
                if (!(l > 0)) return fail(c, SPH_ERR_ARG, "boundary particle %lld has a zero normal", i);
                c->bx.push_back(x[i]); c->by.push_back(y[i]);
                c->bnx.push_back(nx[i] / l); c->bny.push_back(ny[i] / l);
            }
            s = upload_boundary(c);
            if (s) return s;
        }
        return SPH_OK;
    } catch (...) {
        return fail(c, SPH_ERR_OOM, "host allocation failed");
    }
}

sph_status sph_inflow(sph_ctx *c, double x_exit, double y0, double y1, double U, double amp,
                      double k, double phase, int layers) {
    if (!c) return SPH_ERR_ARG;
    c->sg_ready = false;
    try {
        if (c->inf.on) return fail(c, SPH_ERR_STATE, "inflow already configured");
        double dx = c->prm.dx;
        if (!(y1 > y0) || !(U > 0) || !(amp >= 0 && amp < 1) || layers < 1 || layers > 16 ||
            !std::isfinite(k) || !std::isfinite(phase))
            return fail(c, SPH_ERR_ARG, "invalid inflow parameters");
        int ny = (int)std::lround((y1 - y0) / dx);
        if (ny < 1 || ny > 1024) return fail(c, SPH_ERR_ARG, "inflow layer holds %d particles (1..1024)", ny);
        Inflow &f = c->inf;
        f.layers = layers; f.ny = ny; f.x_exit = x_exit; f.y0 = y0; f.y1 = y1; f.U = U;
        f.amp = amp; f.k = k; f.phase = phase; f.dx = dx;
        f.m_layer = c->prm.rho0 * (dx * dx);
        f.threshold = x_exit - (layers - 0.5) * dx;
        std::vector<double> ly(ny);
        for (int j = 0; j < ny; ++j) ly[j] = y0 + (j + 0.5) * dx;
        for (int j = 0; j < ny; ++j)
            if (!inside(c, f.threshold - dx, ly[j]))
                return fail(c, SPH_ERR_ARG, "inflow buffer lies outside the domain");
        sph_status s = pull_scalars(c);
        if (s) return s;
        double t = c->hsc->t;
        double u0 = U * (1.0 + amp * std::sin(k * U * t + phase));
        long long nnew = (long long)layers * ny;
        std::vector<double> xs(nnew), ys(nnew), us(nnew, u0), vs(nnew, 0.0), rs(nnew, c->prm.rho0),
            ms(nnew, f.m_layer);
        std::vector<unsigned char> ts(nnew, SPH_BUFFER);
        for (int L = 0; L < layers; ++L)
            for (int j = 0; j < ny; ++j) {
                xs[(size_t)L * ny + j] = x_exit - (L + 0.5) * dx;
                ys[(size_t)L * ny + j] = ly[j];
            }
        CK(copy_sync(c, c->layer_y, ly.data(), ny * sizeof(double), cudaMemcpyHostToDevice), "upload layer");
        s = sph_add_particles(c, nnew, xs.data(), ys.data(), us.data(), vs.data(), rs.data(),
                              ms.data(), ts.data(), nullptr, nullptr);
        if (s) return s;
        s = pull_scalars(c);
        if (s) return s;
        c->hsc->x_up = x_exit - (layers - 0.5) * dx;
        s = push_scalars(c);
        if (s) return s;
        f.on = 1;
        mark_graph_dirty(c);
        return SPH_OK;
    } catch (...) {
        return fail(c, SPH_ERR_OOM, "host allocation failed");
    }
}

static sph_status ensure_graph(sph_ctx *c);
static sph_status launch_step_graph(sph_ctx *c);

sph_status sph_step(sph_ctx *c, double *dt_used) {
    if (!c) return SPH_ERR_ARG;
    // one replay of the captured step (the same kernels as an eager launch,
    // without the per-kernel launch cost)
    sph_status gs = ensure_graph(c);
    if (gs) return gs;
    gs = launch_step_graph(c);
    if (gs) return gs;
    sph_status s = after_work(c, "step");
    if (dt_used) *dt_used = c->hsc->dt;
    c->n_eval = c->hsc->nsrt;
    c->csf_valid = false;
    return s;
}

sph_status sph_evaluate(sph_ctx *c) {
    if (!c) return SPH_ERR_ARG;
    c->force_full = true;
    c->sg_ready = false;
    if (c->tsz == 4) enqueue_evaluate<float>(c); else enqueue_evaluate<double>(c);
    sph_status s = after_work(c, "evaluate");
    c->n_eval = c->hsc->nsrt;
    c->csf_valid = true;
    return s;
}

// Appends one step of context c to graph g as a branch of its own (no
// dependencies on nodes already in g).  At cadence 1 the branch is the
// rebuilding step.  Otherwise the start (rebuild or reuse of the last build)
// is picked on the device from the flag the previous step left, in one of two
// forms with identical results:
//   gated: both starts one after the other in one straight line, each kernel
//     returning at once when its start is not the one taken (no graph node
//     beyond the kernels; every kernel of both starts is launched);
//   conditional: a one-thread kernel sets an IF node's condition, the node
//     runs the rebuild or the reuse start (only the taken start's kernels are
//     launched, but the node itself costs about 10 us per step on GB300).
// The rest of the step follows either form.
static sph_status append_step(sph_ctx *c, cudaGraph_t g) {
    c->no_ticks = true;
    struct Untick {
        sph_ctx *c;
        ~Untick() { c->no_ticks = false; }
    } untick{c};
    if (c->cadence <= 1 || c->start_form == SPH_START_GATED) {
        CK(cudaStreamBeginCaptureToGraph(c->stream, g, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal), "capture step");
        bool gated = c->cadence > 1;
        if (c->tsz == 4) {
            enqueue_cells<float>(c, true, gated ? GATE_FULL : GATE_ALWAYS);
            if (gated) enqueue_cells<float>(c, false, GATE_REUSE);
            enqueue_rest<float>(c);
        } else {
            enqueue_cells<double>(c, true, gated ? GATE_FULL : GATE_ALWAYS);
            if (gated) enqueue_cells<double>(c, false, GATE_REUSE);
            enqueue_rest<double>(c);
        }
        CK(cudaStreamEndCapture(c->stream, &g), "end capture step");
        return SPH_OK;
    }
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0u, 0u), "conditional handle");
    const Scalars *scp = c->sc;
    void *args[2] = {(void *)&h, (void *)&scp};
    cudaKernelNodeParams kp = {};
    kp.func = decide_kernel();
    kp.gridDim = dim3(1, 1, 1);
    kp.blockDim = dim3(1, 1, 1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    cudaGraphNode_t dnode;
    CK(cudaGraphAddKernelNode(&dnode, g, nullptr, 0, &kp), "decide node");
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    // without surface tension and Eq. 6 the reuse start launches nothing:
    // then the node has the rebuild body only
    bool reuse_kernels = c->prm.sigma > 0 || c->prm.density == SPH_DENSITY_SUMMATION;
    np.conditional.size = reuse_kernels ? 2 : 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, g, &dnode, nullptr, 1, &np), "conditional node");
    cudaGraph_t body[2] = {np.conditional.phGraph_out[0],
                           reuse_kernels ? np.conditional.phGraph_out[1] : nullptr};
    for (int k = 0; k < (reuse_kernels ? 2 : 1); ++k) {
        CK(cudaStreamBeginCaptureToGraph(c->stream, body[k], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal), "capture body");
        if (c->tsz == 4) enqueue_cells<float>(c, k == 0); else enqueue_cells<double>(c, k == 0);
        CK(cudaStreamEndCapture(c->stream, &body[k]), "end capture body");
    }
    CK(cudaStreamBeginCaptureToGraph(c->stream, g, &cnode, nullptr, 1,
                                     cudaStreamCaptureModeThreadLocal), "capture rest");
    if (c->tsz == 4) enqueue_rest<float>(c); else enqueue_rest<double>(c);
    CK(cudaStreamEndCapture(c->stream, &g), "end capture rest");
    return SPH_OK;
}

// The two host-chosen step graphs (rebuild / reuse; the profiling path, and
// every step at cadence 1) and the step graph whose start is chosen on the
// device.
static sph_status ensure_graph(sph_ctx *c) {
    if (!c->graph_dirty && c->gexec[0] && c->gexec[1] && c->cexec) return SPH_OK;
    for (int k = 0; k < 2; ++k) {
        if (c->gexec[k]) { cudaGraphExecDestroy(c->gexec[k]); c->gexec[k] = nullptr; }
        if (c->graph[k]) { cudaGraphDestroy(c->graph[k]); c->graph[k] = nullptr; }
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        step_any(c, k == 0);
        c->prof_pending = false;
        CK(cudaStreamEndCapture(c->stream, &c->graph[k]), "end capture");
        CK(cudaGraphInstantiate(&c->gexec[k], c->graph[k], 0), "instantiate graph");
    }
    if (c->cexec) { cudaGraphExecDestroy(c->cexec); c->cexec = nullptr; }
    if (c->cgraph) { cudaGraphDestroy(c->cgraph); c->cgraph = nullptr; }
    CK(cudaGraphCreate(&c->cgraph, 0), "graph create");
    sph_status s = append_step(c, c->cgraph);
    if (s) return s;
    CK(cudaGraphInstantiate(&c->cexec, c->cgraph, 0), "instantiate step graph");
    c->graph_dirty = false;
    return SPH_OK;
}

static sph_status launch_step_graph(sph_ctx *c) {
    c->sg_ready = false;
    if (c->prof || c->cadence <= 1) {
        // host-chosen graphs: while profiling, and for cadence 1, where every
        // step rebuilds and the gated reuse kernels would only add overhead
        bool full = c->cadence <= 1 ? true : host_next_is_full(c);
        if (c->cadence <= 1) { c->force_full = false; c->hsc_fresh = false; }
        CK(cudaGraphLaunch(c->gexec[full ? 0 : 1], c->stream), "graph launch");
        c->last_kind = full ? 0 : 1;
        c->prof_pending = c->prof;
    } else {
        if (c->force_full) {
            CK(cudaMemsetAsync(&c->sc->need_full, 0x01, sizeof(int), c->stream), "force rebuild");
            c->force_full = false;
        }
        c->hsc_fresh = false;
        CK(cudaGraphLaunch(c->cexec, c->stream), "graph launch");
    }
    return SPH_OK;
}

static sph_status breakup_now(sph_ctx *c, double D, double *L, int *broken) {
    c->force_full = true;
    if (c->tsz == 4) enqueue_breakup<float>(c); else enqueue_breakup<double>(c);
    sph_status s = after_work(c, "breakup");
    if (s) return s;
    unsigned long long k = c->hsc->xmax_key;
    if (k == 0) return fail(c, SPH_ERR_STATE, "no inflow buffer particle present");
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double xmax;
    memcpy(&xmax, &b, 8);
    *L = (xmax - c->inf.x_exit) / D;
    if (broken) *broken = c->hsc->detached > 0;
    return SPH_OK;
}

sph_status sph_breakup_length(sph_ctx *c, double D, double *L_over_D, int *broken) {
    if (!c) return SPH_ERR_ARG;
    if (!c->inf.on) return fail(c, SPH_ERR_STATE, "breakup length needs an inflow");
    if (!(D > 0) || !L_over_D) return fail(c, SPH_ERR_ARG, "D > 0 and L_over_D required");
    return breakup_now(c, D, L_over_D, broken);
}

sph_status sph_run(sph_ctx *c, long long nsteps, int breakup_every, double D, double *L_out,
                   long long *nL) {
    if (!c) return SPH_ERR_ARG;
    if (nsteps < 0) return fail(c, SPH_ERR_ARG, "nsteps < 0");
    if (breakup_every > 0) {
        if (!c->inf.on) return fail(c, SPH_ERR_STATE, "breakup sampling needs an inflow");
        if (!L_out || !nL || !(D > 0)) return fail(c, SPH_ERR_ARG, "L_out, nL and D > 0 required");
        *nL = 0;
    }
    sph_status gs = ensure_graph(c);
    if (gs) return gs;
    for (long long k = 1; k <= nsteps; ++k) {
        sph_status ls = launch_step_graph(c);
        if (ls) return ls;
        if (breakup_every > 0 && k % breakup_every == 0) {
            double L;
            sph_status s = breakup_now(c, D, &L, nullptr);
            if (s) return s;
            L_out[(*nL)++] = L;
        }
    }
    sph_status s = after_work(c, "run");
    c->n_eval = c->hsc->nsrt;
    c->csf_valid = false;
    return s;
}

}  // extern "C"

// Orders the indices in ord by ids[ord[.]] (ids unique): a scatter by id in
// O(n) when the ids are dense (they are handed out in sequence), else a
// comparison sort.
static void order_by_id(std::vector<size_t> &ord, const unsigned *ids) {
    unsigned max_id = 0;
    for (size_t i : ord) max_id = std::max(max_id, ids[i]);
    if (!ord.empty() && (size_t)max_id < 8 * ord.size() + 1024) {
        const size_t ns = (size_t)max_id + 1, n = ord.size();
        std::vector<int64_t> slot(ns);
        const size_t par = n >= ((size_t)1 << 16) ? 1 : 64;   // grain: threads only when large
        host_for(ns, [&](size_t lo, size_t hi) {
            std::fill(slot.begin() + lo, slot.begin() + hi, (int64_t)-1);
        });
        // distinct ids: the threads write distinct slots
        host_for(n, [&](size_t lo, size_t hi) {
            for (size_t r = lo; r < hi; ++r) slot[ids[ord[r]]] = (int64_t)ord[r];
        });
        // compaction in id order: count per chunk of slots, then each chunk
        // writes from its prefix
        const size_t nchunk = 64;
        std::vector<size_t> cnt(nchunk + 1, 0);
        host_for(nchunk, [&](size_t k0, size_t k1) {
            for (size_t k = k0; k < k1; ++k) {
                size_t c = 0;
                for (size_t q = ns * k / nchunk; q < ns * (k + 1) / nchunk; ++q) c += slot[q] >= 0;
                cnt[k + 1] = c;
            }
        }, par);
        for (size_t k = 0; k < nchunk; ++k) cnt[k + 1] += cnt[k];
        host_for(nchunk, [&](size_t k0, size_t k1) {
            for (size_t k = k0; k < k1; ++k) {
                size_t w = cnt[k];
                for (size_t q = ns * k / nchunk; q < ns * (k + 1) / nchunk; ++q)
                    if (slot[q] >= 0) ord[w++] = (size_t)slot[q];
            }
        }, par);
    } else {
        std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return ids[a] < ids[b]; });
    }
}

extern "C" {

sph_status sph_get_state(sph_ctx *c, long long cap, long long *n_out, double *x, double *y,
                         double *u, double *v, double *rho, double *mass, unsigned char *type,
                         unsigned *id, double *ax, double *ay, double *drho) {
    if (!c || !n_out) return SPH_ERR_ARG;
    try {
        sph_status s = pull_scalars(c);
        if (s) return s;
        if (c->n_eval < 0) c->n_eval = c->hsc->nsrt;
        const size_t n = (size_t)c->hsc->n, ts = c->tsz;
        // pinned staging: type | position | velocity | density | mass | id |
        // acceleration | density rate
        const size_t o_ty = 0, o_pos = al16(n), o_vel = o_pos + al16(16 * n),
                     o_dr = o_vel + al16(2 * n * ts), o_m = o_dr + al16(n * ts),
                     o_id = o_m + al16(n * ts), o_ac = o_id + al16(4 * n),
                     o_drt = o_ac + al16(2 * n * ts), total = o_drt + al16(n * ts);
        cudaError_t e;
        unsigned char *pin = staging(c, total, e);
        CK(e, "pinned staging");
        // the types first: a call that only asks for the count (cap too
        // small) moves one byte per particle
        if (n) CK(copy_sync(c, pin + o_ty, c->raw[5], n, cudaMemcpyDeviceToHost), "download");
        const unsigned char *ty = pin + o_ty;
        std::vector<size_t> ord;
        ord.reserve(n);
        for (size_t i = 0; i < n; ++i)
            if (ty[i] != T_DEAD) ord.push_back(i);
        *n_out = (long long)ord.size();
        if ((long long)ord.size() > cap) return fail(c, SPH_ERR_CAPACITY, "%zu particles > cap %lld", ord.size(), cap);
        if (ord.empty()) return SPH_OK;
        // one asynchronous copy per array and one wait for all of them (also
        // when one fails: no copy into the staging outlives the call)
        const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
        cudaStream_t st = c->stream;
        cudaError_t err = cudaMemcpyAsync(pin + o_pos, c->raw[0], 16 * n, d2h, st);
        if (!err) err = cudaMemcpyAsync(pin + o_vel, c->raw[1], 2 * n * ts, d2h, st);
        if (!err) err = cudaMemcpyAsync(pin + o_dr, c->raw[2], n * ts, d2h, st);
        if (!err) err = cudaMemcpyAsync(pin + o_m, c->raw[4], n * ts, d2h, st);
        if (!err) err = cudaMemcpyAsync(pin + o_id, c->raw[6], 4 * n, d2h, st);
        if (!err) err = cudaMemcpyAsync(pin + o_ac, c->acc, 2 * n * ts, d2h, st);
        if (!err) err = cudaMemcpyAsync(pin + o_drt, c->dr, n * ts, d2h, st);
        cudaError_t es = cudaStreamSynchronize(st);
        CK(err ? err : es, "download");
        const double2 *pos = (const double2 *)(pin + o_pos);
        const unsigned *ids = (const unsigned *)(pin + o_id);
        order_by_id(ord, ids);
        const double ufx = c->prm.u_frame_x, ufy = c->prm.u_frame_y, rho0 = c->prm.rho0;
        const long long n_eval = c->n_eval;
        auto convert = [&](auto tag) {
            using T = decltype(tag);
            const T *vel = (const T *)(pin + o_vel), *dr = (const T *)(pin + o_dr),
                    *m = (const T *)(pin + o_m), *ac = (const T *)(pin + o_ac),
                    *drt = (const T *)(pin + o_drt);
            host_for(ord.size(), [&](size_t lo, size_t hi) {
                for (size_t r = lo; r < hi; ++r) {
                    size_t i = ord[r];
                    bool has = (long long)i < n_eval;
                    if (x) x[r] = pos[i].x;
                    if (y) y[r] = pos[i].y;
                    if (u) u[r] = ufx + (double)vel[2 * i];
                    if (v) v[r] = ufy + (double)vel[2 * i + 1];
                    if (rho) rho[r] = rho0 + (double)dr[i];
                    if (mass) mass[r] = (double)m[i];
                    if (type) type[r] = ty[i];
                    if (id) id[r] = ids[i];
                    if (ax) ax[r] = has ? (double)ac[2 * i] : 0.0;
                    if (ay) ay[r] = has ? (double)ac[2 * i + 1] : 0.0;
                    if (drho) drho[r] = has ? (double)drt[i] : 0.0;
                }
            });
        };
        if (ts == 4) convert(0.0f); else convert(0.0);
        return SPH_OK;
    } catch (...) {
        return fail(c, SPH_ERR_OOM, "host allocation failed");
    }
}

sph_status sph_set_state(sph_ctx *c, long long n, const double *x, const double *y,
                         const double *u, const double *v, const double *rho,
                         const double *mass, const unsigned char *type, const unsigned *id) {
    if (!c) return SPH_ERR_ARG;
    try {
        if (n < 0 || n > c->cap) return fail(c, SPH_ERR_CAPACITY, "n = %lld outside [0, capacity]", n);
        if (n > 0 && (!x || !y || !u || !v || !rho || !mass || !type || !id))
            return fail(c, SPH_ERR_ARG, "all arrays are required");
        // one pass over the particles in a few threads: the largest id and,
        // per chunk, the first particle that fails a check (type, domain,
        // density and mass), reported after the duplicate-id test as before
        const size_t N = n > 0 ? (size_t)n : 0;
        const size_t nchunk = 64;
        std::vector<unsigned> cmax(nchunk, 0u);
        std::vector<long long> cbad(nchunk, -1);
        std::vector<int> cwhy(nchunk, 0);
        host_for(nchunk, [&](size_t k0, size_t k1) {
            for (size_t k = k0; k < k1; ++k) {
                size_t lo = N * k / nchunk, hi = N * (k + 1) / nchunk;
                unsigned mx = 0;
                for (size_t i = lo; i < hi; ++i) {
                    mx = std::max(mx, id[i]);
                    if (cbad[k] >= 0) continue;
                    int why = 0;
                    if (type[i] != SPH_FLUID && type[i] != SPH_BUFFER) why = 1;
                    else if (!inside(c, x[i], y[i])) why = 2;
                    else if (!(rho[i] > 0) || !(mass[i] > 0)) why = 3;
                    if (why) {
                        cbad[k] = (long long)i;
                        cwhy[k] = why;
                    }
                }
                cmax[k] = mx;
            }
        }, N >= ((size_t)1 << 16) ? 1 : nchunk);
        unsigned maxid = 0;
        for (unsigned m : cmax) maxid = std::max(maxid, m);
        // duplicate ids: a mark per id when they are dense (set in a few
        // threads with atomic exchanges; every repeated id is met by the
        // second of its marks, and the smallest one is reported), else a sort
        if (n > 0 && (size_t)maxid < 8 * (size_t)n + 1024) {
            std::vector<unsigned char> seen((size_t)maxid + 1, 0);
            std::vector<unsigned> cdup(nchunk, 0xFFFFFFFFu);
            host_for(nchunk, [&](size_t k0, size_t k1) {
                for (size_t k = k0; k < k1; ++k)
                    for (size_t i = N * k / nchunk; i < N * (k + 1) / nchunk; ++i)
                        if (__atomic_exchange_n(&seen[id[i]], (unsigned char)1, __ATOMIC_RELAXED))
                            cdup[k] = std::min(cdup[k], id[i]);
            }, N >= ((size_t)1 << 16) ? 1 : nchunk);
            unsigned dup = 0xFFFFFFFFu;
            for (unsigned d : cdup) dup = std::min(dup, d);
            if (dup != 0xFFFFFFFFu) return fail(c, SPH_ERR_ARG, "duplicate id %u", dup);
        } else if (n > 0) {
            std::vector<unsigned> sid(id, id + n);
            std::sort(sid.begin(), sid.end());
            for (long long i = 1; i < n; ++i)
                if (sid[i] == sid[i - 1]) return fail(c, SPH_ERR_ARG, "duplicate id %u", sid[i]);
        }
        for (size_t k = 0; k < nchunk; ++k) {
            long long i = cbad[k];
            if (i < 0) continue;
            if (cwhy[k] == 1)
                return fail(c, SPH_ERR_ARG, "particle %lld: set_state takes fluid or buffer particles", i);
            if (cwhy[k] == 2) return fail(c, SPH_ERR_ARG, "particle %lld lies outside the domain", i);
            return fail(c, SPH_ERR_ARG, "particle %lld needs rho, mass > 0", i);
        }
        sph_status s = pull_scalars(c);
        if (s) return s;
        s = upload_particles(c, 0, n, x, y, u, v, rho, mass, type, id);
        if (s) return s;
        c->hsc->n = (int)n;
        c->hsc->nsrt = 0;
        c->force_full = true;
        c->sg_ready = false;
        if (n > 0) c->hsc->next_id = std::max(c->hsc->next_id, maxid + 1);
        s = push_scalars(c);
        c->n_eval = 0;
        c->csf_valid = false;
        return s;
    } catch (...) {
        return fail(c, SPH_ERR_OOM, "host allocation failed");
    }
}

sph_status sph_get_csf(sph_ctx *c, long long cap, long long *n_out, unsigned *id, double *C,
                       double *nx, double *ny) {
    if (!c || !n_out) return SPH_ERR_ARG;
    if (!c->csf_valid) return fail(c, SPH_ERR_STATE, "call sph_evaluate first");
    try {
        sph_status s = pull_scalars(c);
        if (s) return s;
        size_t n = (size_t)c->hsc->nsrt, ts = c->tsz;
        *n_out = (long long)n;
        if ((long long)n > cap) return fail(c, SPH_ERR_CAPACITY, "%zu particles > cap %lld", n, cap);
        std::vector<unsigned char> cc(n * ts), nv(2 * n * ts);
        std::vector<unsigned> ids(n);
        bool on = c->prm.sigma > 0;
        if (n) {
            CK(copy_sync(c, ids.data(), c->raw[6], n * 4, cudaMemcpyDeviceToHost), "download");
            if (on) {
                CK(copy_sync(c, cc.data(), c->C, n * ts, cudaMemcpyDeviceToHost), "download");
                CK(copy_sync(c, nv.data(), c->nvec, 2 * n * ts, cudaMemcpyDeviceToHost), "download");
            }
        }
        std::vector<size_t> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        order_by_id(ord, ids.data());
        for (size_t r = 0; r < n; ++r) {
            size_t i = ord[r];
            if (id) id[r] = ids[i];
            if (C) C[r] = on ? rd(c, cc, i, 0, 1) : 0.0;
            if (nx) nx[r] = on ? rd(c, nv, i, 0, 2) : 0.0;
            if (ny) ny[r] = on ? rd(c, nv, i, 1, 2) : 0.0;
        }
        return SPH_OK;
    } catch (...) {
        return fail(c, SPH_ERR_OOM, "host allocation failed");
    }
}

sph_status sph_get_pairs(sph_ctx *c, long long cap, unsigned *id_a, unsigned *id_b,
                         long long *npairs) {
    if (!c || !npairs || cap < 0) return SPH_ERR_ARG;
    if (cap > 0 && (!id_a || !id_b)) return fail(c, SPH_ERR_ARG, "output arrays required");
    unsigned long long dcap = (unsigned long long)std::min<long long>(cap, 0x7fffffffll);
    unsigned *da = nullptr, *db = nullptr;
    c->force_full = true;
    CK(cudaMalloc(&da, std::max<size_t>(dcap, 1) * 4), "pair buffer");
    cudaError_t e = cudaMalloc(&db, std::max<size_t>(dcap, 1) * 4);
    if (e) { cudaFree(da); return cuda_check(c, e, "pair buffer"); }
    sph_status s = SPH_OK;
    if (c->tsz == 4) {
        const uint32_t *key = enqueue_sort<float>(c);
        e = launch_pairs<float>(c->Pf, c->grid, c->sc, c->cellSE, key, hot_n<float>(c),
                                (uint32_t *)c->srt[6], da, db, dcap, c->cap, c->stream);
    } else {
        const uint32_t *key = enqueue_sort<double>(c);
        e = launch_pairs<double>(c->Pd, c->grid, c->sc, c->cellSE, key, hot_n<double>(c),
                                 (uint32_t *)c->srt[6], da, db, dcap, c->cap, c->stream);
    }
    if (e != cudaSuccess) {
        cudaFree(da);
        cudaFree(db);
        return cuda_check(c, e, "pair export");
    }
    s = after_work(c, "pairs");
    if (s == SPH_OK) {
        long long np = (long long)c->hsc->pair_count;
        *npairs = np;
        if (np > cap) {
            s = fail(c, SPH_ERR_CAPACITY, "%lld pairs > cap %lld", np, cap);
        } else if (np > 0) {
            e = copy_sync(c, id_a, da, (size_t)np * 4, cudaMemcpyDeviceToHost);
            if (!e) e = copy_sync(c, id_b, db, (size_t)np * 4, cudaMemcpyDeviceToHost);
            if (e) s = cuda_check(c, e, "download pairs");
        }
    }
    cudaFree(da);
    cudaFree(db);
    return s;
}

// ---------------------------------------------------------------------------
// checkpoints: a header, then the live particles in id order as stored
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];          // "SPHCKPT1"
    int32_t tsz;            // bytes of the pair precision (4 or 8)
    int32_t reserved;
    int64_t n;              // particles
    double t;               // simulated time
    int64_t step;           // completed steps
    double x_up;            // upstream-most inflow layer position
    uint32_t next_id;       // next particle id
    uint32_t reserved2;
    int64_t deleted;        // particles deleted by the outflow
};
const char kCkptMagic[8] = {'S', 'P', 'H', 'C', 'K', 'P', 'T', '1'};
size_t ckpt_bytes(size_t n, size_t ts) { return sizeof(CkptHeader) + n * (16 + 5 * ts + 1 + 4); }
}  // namespace

// Live particles of raw in id order: their raw indices.
static sph_status live_order(sph_ctx *c, std::vector<size_t> &ord, std::vector<unsigned char> &ty,
                             std::vector<unsigned> &ids) {
    size_t n = (size_t)c->hsc->n;
    ty.resize(n);
    ids.resize(n);
    if (n) {
        CK(copy_sync(c, ty.data(), c->raw[5], n, cudaMemcpyDeviceToHost), "download");
        CK(copy_sync(c, ids.data(), c->raw[6], n * 4, cudaMemcpyDeviceToHost), "download");
    }
    ord.clear();
    for (size_t i = 0; i < n; ++i)
        if (ty[i] != T_DEAD) ord.push_back(i);
    order_by_id(ord, ids.data());
    return SPH_OK;
}

sph_status sph_checkpoint_size(sph_ctx *c, size_t *bytes) {
    if (!c || !bytes) return SPH_ERR_ARG;
    try {
        sph_status s = pull_scalars(c);
        if (s) return s;
        std::vector<size_t> ord;
        std::vector<unsigned char> ty;
        std::vector<unsigned> ids;
        s = live_order(c, ord, ty, ids);
        if (s) return s;
        *bytes = ckpt_bytes(ord.size(), c->tsz);
        return SPH_OK;
    } catch (...) {
        return fail(c, SPH_ERR_OOM, "host allocation failed");
    }
}

sph_status sph_checkpoint_save(sph_ctx *c, void *buf, size_t cap, size_t *bytes) {
    if (!c || (!buf && cap > 0)) return SPH_ERR_ARG;
    try {
        sph_status s = pull_scalars(c);
        if (s) return s;
        std::vector<size_t> ord;
        std::vector<unsigned char> ty;
        std::vector<unsigned> ids;
        s = live_order(c, ord, ty, ids);
        if (s) return s;
        const size_t n = (size_t)c->hsc->n, m = ord.size(), ts = c->tsz;
        const size_t need = ckpt_bytes(m, ts);
        if (bytes) *bytes = need;
        if (cap < need) return fail(c, SPH_ERR_CAPACITY, "checkpoint needs %zu bytes > cap %zu", need, cap);
        // raw fields: pos (16), vel (2 ts), drho (ts), drc (ts), mass (ts)
        const size_t fsz[5] = {16, 2 * ts, ts, ts, ts};
        const int fidx[5] = {0, 1, 2, 3, 4};
        CkptHeader hd{};
        memcpy(hd.magic, kCkptMagic, 8);
        hd.tsz = (int32_t)ts;
        hd.n = (int64_t)m;
        hd.t = c->hsc->t;
        hd.step = c->hsc->step;
        hd.x_up = c->hsc->x_up;
        hd.next_id = c->hsc->next_id;
        hd.deleted = c->hsc->deleted;
        unsigned char *out = (unsigned char *)buf;
        memcpy(out, &hd, sizeof hd);
        size_t off = sizeof hd;
        std::vector<unsigned char> tmp;
        for (int f = 0; f < 5; ++f) {
            tmp.resize(n * fsz[f]);
            if (n) CK(copy_sync(c, tmp.data(), c->raw[fidx[f]], n * fsz[f], cudaMemcpyDeviceToHost), "download");
            for (size_t r = 0; r < m; ++r) memcpy(out + off + r * fsz[f], &tmp[ord[r] * fsz[f]], fsz[f]);
            off += m * fsz[f];
        }
        for (size_t r = 0; r < m; ++r) out[off + r] = ty[ord[r]];
        off += m;
        for (size_t r = 0; r < m; ++r) memcpy(out + off + 4 * r, &ids[ord[r]], 4);
        return SPH_OK;
    } catch (...) {
        return fail(c, SPH_ERR_OOM, "host allocation failed");
    }
}

sph_status sph_checkpoint_load(sph_ctx *c, const void *buf, size_t bytes) {
    if (!c || !buf) return SPH_ERR_ARG;
    if (bytes < sizeof(CkptHeader)) return fail(c, SPH_ERR_ARG, "not a checkpoint (too short)");
    CkptHeader hd;
    memcpy(&hd, buf, sizeof hd);
    if (memcmp(hd.magic, kCkptMagic, 8) != 0) return fail(c, SPH_ERR_ARG, "not a checkpoint");
    const size_t ts = c->tsz;
    if (hd.tsz != (int32_t)ts) return fail(c, SPH_ERR_ARG, "checkpoint of the other pair precision");
    if (hd.n < 0 || hd.n > c->cap) return fail(c, SPH_ERR_ARG, "checkpoint of %lld particles beyond capacity %lld", (long long)hd.n, c->cap);
    const size_t m = (size_t)hd.n;
    if (bytes != ckpt_bytes(m, ts)) return fail(c, SPH_ERR_ARG, "checkpoint size does not match its header");
    const unsigned char *in = (const unsigned char *)buf + sizeof hd;
    const size_t fsz[5] = {16, 2 * ts, ts, ts, ts};
    size_t off = 0;
    const unsigned char *ty = in;
    for (int f = 0; f < 5; ++f) off += m * fsz[f];
    ty = in + off;
    for (size_t r = 0; r < m; ++r)
        if (ty[r] != SPH_FLUID && ty[r] != SPH_BUFFER) return fail(c, SPH_ERR_ARG, "checkpoint particle %zu: bad type", r);
    sph_status s = pull_scalars(c);
    if (s) return s;
    off = 0;
    for (int f = 0; f < 5; ++f) {
        if (m) CK(copy_sync(c, c->raw[f], in + off, m * fsz[f], cudaMemcpyHostToDevice), "upload");
        off += m * fsz[f];
    }
    if (m) {
        CK(copy_sync(c, c->raw[5], in + off, m, cudaMemcpyHostToDevice), "upload");
        CK(copy_sync(c, c->raw[6], in + off + m, m * 4, cudaMemcpyHostToDevice), "upload");
        CK(cudaMemsetAsync(c->raw[7], 0, m * 2 * ts, c->stream), "upload");
    }
    c->hsc->n = (int)m;
    c->hsc->nsrt = 0;
    c->hsc->t = hd.t;
    c->hsc->step = hd.step;
    c->hsc->x_up = hd.x_up;
    c->hsc->next_id = hd.next_id;
    c->hsc->deleted = hd.deleted;
    c->force_full = true;
    c->sg_ready = false;
    s = push_scalars(c);
    c->n_eval = 0;
    c->csf_valid = false;
    return s;
}

sph_status sph_stats(sph_ctx *c, sph_stats_t *out) {
    if (!c || !out) return SPH_ERR_ARG;
    if (!c->stats) {
        cudaError_t e = cudaSuccess;
        c->stats = dalloc(c, 6 * sizeof(double) + 3 * sizeof(unsigned long long), e);
        CK(e, "stats scratch");
    }
    double *acc = (double *)c->stats;
    unsigned long long *cnt = (unsigned long long *)(acc + 6);
    CK(cudaMemsetAsync(c->stats, 0, 6 * sizeof(double) + 3 * sizeof(unsigned long long), c->stream), "clear");
    const double rho0 = c->prm.rho0, B = c->prm.rho0 * c->prm.c0 * c->prm.c0 / c->prm.gamma;
    if (c->tsz == 4)
        launch_stats<float>(c->Pf, state_of<float>(c->raw), c->sc, c->prm.gx, c->prm.gy, rho0, B,
                            c->prm.gamma, acc, cnt, c->cap, c->stream);
    else
        launch_stats<double>(c->Pd, state_of<double>(c->raw), c->sc, c->prm.gx, c->prm.gy, rho0, B,
                             c->prm.gamma, acc, cnt, c->cap, c->stream);
    CK(cudaGetLastError(), "stats launch");
    double h[6];
    unsigned long long k[3];
    CK(copy_sync(c, h, acc, sizeof h, cudaMemcpyDeviceToHost), "stats");
    CK(copy_sync(c, k, cnt, sizeof k, cudaMemcpyDeviceToHost), "stats");
    sph_status s = pull_scalars(c);
    if (s) return s;
    out->n_fluid = (long long)k[0];
    out->n_buffer = (long long)k[1];
    out->n_boundary = (long long)c->bx.size();
    out->n_deleted = c->hsc->deleted;
    out->step = c->hsc->step;
    out->t = c->hsc->t;
    out->dt = c->hsc->dt;
    out->mass = h[0];
    out->momentum_x = h[1];
    out->momentum_y = h[2];
    out->kinetic = h[3];
    out->potential = h[4];
    out->elastic = h[5];
    long long bits = (long long)k[2];
    memcpy(&out->max_rel_density, &bits, sizeof bits);
    return SPH_OK;
}

sph_status sph_get_time(sph_ctx *c, double *t, long long *steps, long long *n_particles,
                        long long *n_deleted) {
    if (!c) return SPH_ERR_ARG;
    sph_status s = pull_scalars(c);
    if (s) return s;
    if (t) *t = c->hsc->t;
    if (steps) *steps = c->hsc->step;
    if (n_deleted) *n_deleted = c->hsc->deleted;
    if (n_particles) {
        // dead-marked particles are dropped at the next cell build
        long long n = c->hsc->n;
        if (n > 0) {
            std::vector<unsigned char> ty((size_t)n);
            CK(copy_sync(c, ty.data(), c->raw[5], (size_t)n, cudaMemcpyDeviceToHost), "download");
            for (auto v : ty) if (v == T_DEAD) --n;
        }
        *n_particles = n;
    }
    return SPH_OK;
}

sph_status sph_run_async(sph_ctx *c, long long nsteps) {
    if (!c) return SPH_ERR_ARG;
    if (nsteps < 0) return fail(c, SPH_ERR_ARG, "nsteps < 0");
    sph_status gs = ensure_graph(c);
    if (gs) return gs;
    for (long long k = 0; k < nsteps; ++k) {
        sph_status ls = launch_step_graph(c);
        if (ls) return ls;
    }
    if (nsteps > 0) {
        c->n_eval = -1;   // resolved at the next synchronising call
        c->csf_valid = false;
    }
    return SPH_OK;
}

sph_status sph_sync(sph_ctx *c) {
    if (!c) return SPH_ERR_ARG;
    sph_status s = after_work(c, "sync");
    if (c->n_eval < 0) c->n_eval = c->hsc->nsrt;
    return s;
}

sph_status sph_profile(sph_ctx *c, int enable) {
    if (!c) return SPH_ERR_ARG;
    for (int k = 0; k < 2; ++k)
        while (enable && c->pev[k].size() < 48) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e), "event create");
            c->pev[k].push_back(e);
            c->pname[k].push_back(nullptr);
        }
    if (c->prof != (enable != 0)) mark_graph_dirty(c);
    c->prof = enable != 0;
    c->prof_pending = false;
    c->ptot.clear();
    return SPH_OK;
}

sph_status sph_profile_report(sph_ctx *c, int cap, int *n, const char **names, double *total_ms,
                              long long *launches) {
    if (!c || !n) return SPH_ERR_ARG;
    c->report_names.clear();
    for (auto &kv : c->ptot) c->report_names.push_back(kv.first);
    *n = (int)c->report_names.size();
    if (*n > cap) return fail(c, SPH_ERR_CAPACITY, "%d kernel groups > cap %d", *n, cap);
    int k = 0;
    for (auto &kv : c->ptot) {
        if (names) names[k] = c->report_names[k].c_str();
        if (total_ms) total_ms[k] = kv.second.first;
        if (launches) launches[k] = kv.second.second;
        ++k;
    }
    return SPH_OK;
}

sph_status sph_set_tuning(sph_ctx *c, int lanes, int cadence) {
    if (!c) return SPH_ERR_ARG;
    if (!(lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8))
        return fail(c, SPH_ERR_ARG, "lanes must be 1, 2, 4 or 8");
    if (cadence < 1 || cadence > 64) return fail(c, SPH_ERR_ARG, "cadence must lie in [1, 64]");
    // both are captured into the step graphs (launch shapes; the cadence
    // is an argument of the rebuild decision)
    if (lanes != c->lanes || cadence != c->cadence) mark_graph_dirty(c);
    c->lanes = lanes;
    c->cadence = cadence;
    c->force_full = true;
    return SPH_OK;
}

sph_status sph_get_tuning(sph_ctx *c, int *lanes, int *cadence) {
    if (!c) return SPH_ERR_ARG;
    if (lanes) *lanes = c->lanes;
    if (cadence) *cadence = c->cadence;
    return SPH_OK;
}

sph_status sph_set_start_form(sph_ctx *c, int form) {
    if (!c) return SPH_ERR_ARG;
    if (form != SPH_START_GATED && form != SPH_START_CONDITIONAL)
        return fail(c, SPH_ERR_ARG, "start form must be SPH_START_GATED or SPH_START_CONDITIONAL");
    if (form != c->start_form) mark_graph_dirty(c);
    c->start_form = form;
    return SPH_OK;
}

sph_status sph_get_start_form(sph_ctx *c, int *form) {
    if (!c) return SPH_ERR_ARG;
    if (form) *form = c->start_form;
    return SPH_OK;
}

// Copies of the raw state and scalars, to run trial steps and come back.
static sph_status snapshot(sph_ctx *c, bool restore, bool scalars_current = false) {
    size_t ts = c->tsz;
    size_t sizes[8] = {16, 2 * ts, ts, ts, ts, 1, 4, 2 * ts};
    if (!restore) {
        // the copies are ordered on the context's stream; with the host
        // scalars already current (scalars_current) nothing waits here
        if (!scalars_current) {
            sph_status s = pull_scalars(c);
            if (s) return s;
        }
        size_t n = (size_t)c->hsc->n;
        if (n > c->snap_n || !c->snap[0]) {
            for (auto &p : c->snap) if (p) { cudaFree(p); p = nullptr; }
            for (int k = 0; k < 8; ++k)
                CK(cudaMalloc(&c->snap[k], std::max<size_t>(n, 1) * sizes[k]), "snapshot");
            c->snap_n = n;
        }
        for (int k = 0; k < 8; ++k)
            CK(cudaMemcpyAsync(c->snap[k], c->raw[k], n * sizes[k], cudaMemcpyDeviceToDevice,
                               c->stream), "snapshot");
        c->snap_sc = *c->hsc;
        if (!scalars_current) CK(cudaStreamSynchronize(c->stream), "snapshot");
        return SPH_OK;
    }
    size_t n = (size_t)c->snap_sc.n;
    for (int k = 0; k < 8; ++k)
        CK(cudaMemcpyAsync(c->raw[k], c->snap[k], n * sizes[k], cudaMemcpyDeviceToDevice,
                           c->stream), "restore");
    *c->hsc = c->snap_sc;
    c->force_full = true;
    c->sg_ready = false;
    return push_scalars(c);
}

sph_status sph_autotune(sph_ctx *c, int trial_steps, int *lanes, int *cadence, double *ms_per_step) {
    if (!c) return SPH_ERR_ARG;
    if (trial_steps < 1 || trial_steps > 10000) return fail(c, SPH_ERR_ARG, "trial_steps in [1, 10000]");
    sph_status s = snapshot(c, false);
    if (s) return s;
    if (c->snap_sc.err) {
        status_from_err(c, c->snap_sc.err);
        return fail(c, SPH_ERR_STATE, "autotune needs a context without a pending error (%s)",
                    c->err.c_str());
    }
    const int L[4] = {1, 2, 4, 8}, K[4] = {1, 2, 4, 8};
    int bestL = c->lanes, bestK = c->cadence, bestF = c->start_form;
    double best = 1e300;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    bool prof = c->prof;
    c->prof = false;
    // one candidate from the snapshot: a warm cycle (capture), then at least
    // two rebuild cycles timed; SPH_ERR_SKIN rejects the candidate only
    auto trial = [&](int Lv, int Kv, int Fv) -> sph_status {
        int steps = std::max(trial_steps, 2 * Kv);
        sph_status t = snapshot(c, true);
        if (!t) t = sph_set_tuning(c, Lv, Kv);
        if (!t) t = sph_set_start_form(c, Fv);
        if (!t) t = sph_run_async(c, Kv);
        if (!t) t = sph_sync(c);
        if (t) return t;
        cudaEventRecord(e0, c->stream);
        t = sph_run_async(c, steps);
        cudaEventRecord(e1, c->stream);
        if (!t) t = sph_sync(c);
        if (t) return t;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        double per = ms / steps;
        if (per < best) { best = per; bestL = Lv; bestK = Kv; bestF = Fv; }
        return SPH_OK;
    };
    // lanes x cadence up to 8, both start forms where the device picks the
    // start (cadence > 1); then longer cadences at the best lane count
    for (int a = 0; a < 4 && (!s || s == SPH_ERR_SKIN); ++a)
        for (int b = 0; b < 4 && (!s || s == SPH_ERR_SKIN); ++b)
            for (int f = 0; f < (K[b] > 1 ? 2 : 1); ++f) {
                s = trial(L[a], K[b], f == 0 ? SPH_START_GATED : SPH_START_CONDITIONAL);
                if (s) break;                             // SKIN: cadence too long here
            }
    if (best < 1e300 && (!s || s == SPH_ERR_SKIN)) {
        int L0 = bestL;
        for (int Kv = 16; Kv <= 32 && (!s || s == SPH_ERR_SKIN); Kv *= 2)
            for (int f = 0; f < 2; ++f) {
                s = trial(L0, Kv, f == 0 ? SPH_START_GATED : SPH_START_CONDITIONAL);
                if (s) break;
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof = prof;
    sph_status r = snapshot(c, true);
    if (s && s != SPH_ERR_SKIN) return s;
    if (r) return r;
    if (best >= 1e300) return fail(c, SPH_ERR_STATE, "no tuning candidate ran without error");
    r = sph_set_tuning(c, bestL, bestK);
    if (!r) r = sph_set_start_form(c, bestF);
    if (r) return r;
    if (lanes) *lanes = bestL;
    if (cadence) *cadence = bestK;
    if (ms_per_step) *ms_per_step = best;
    return SPH_OK;
}

sph_status sph_get_rebuild_stats(sph_ctx *c, long long *builds, double *disp_max,
                                 double *step_max) {
    if (!c) return SPH_ERR_ARG;
    sph_status s = pull_scalars(c);
    if (s) return s;
    if (builds) *builds = c->hsc->builds;
    if (disp_max) *disp_max = c->hsc->last_dmax;
    if (step_max) *step_max = c->hsc->last_smax;
    return SPH_OK;
}

sph_status sph_request_rebuild(sph_ctx *c) {
    if (!c) return SPH_ERR_ARG;
    c->force_full = true;
    c->sg_ready = false;
    return SPH_OK;
}

sph_status sph_kernel_counts(sph_ctx *c, int *per_full_step, int *per_reused_step,
                             int *per_breakup) {
    if (!c) return SPH_ERR_ARG;
    bool csf = c->prm.sigma > 0;
    int sort = 5;                          // hash+count, scan (2), scatter, reorder
    int full = sort + 1;                   // + neighbour list
    int reuse = 0;                         // the corrector wrote the records of step n
    int rest = 2 * (csf ? 3 : 1)           // per evaluation: pair sums, normal, surface
                                           // (or the one force sweep without CSF)
               + 1                         // predict
               + 1;                        // spawn / time advance
    if (c->prm.density == SPH_DENSITY_SUMMATION) {
        full += 1;                         // Eq. 6 sweep
        reuse += 1;                        // Eq. 6 sweep
        rest += 1;                         // Eq. 6 sweep of the half step
    }
    if (c->cadence <= 1) {
        if (per_full_step) *per_full_step = full + rest;
        if (per_reused_step) *per_reused_step = full + rest;
    } else if (c->start_form == SPH_START_GATED) {
        // every step launches the kernels of both starts; those of the start
        // not taken return at once
        if (per_full_step) *per_full_step = full + reuse + rest;
        if (per_reused_step) *per_reused_step = full + reuse + rest;
    } else {
        // the one-thread kernel that sets the IF node, then the taken start
        if (per_full_step) *per_full_step = 1 + full + rest;
        if (per_reused_step) *per_reused_step = 1 + reuse + rest;
    }
    if (per_breakup) *per_breakup = sort + 4;    // + union-find init, link, compress, reach
    return SPH_OK;
}

}  // extern "C"

void ctx_view(sph_ctx *c, CtxView *v) {
    *v = CtxView{};
    v->n = c->hsc->nsrt;
    v->cap = c->cap;
    v->fp32 = c->tsz == 4;
    v->evaluated = c->csf_valid;
    v->device = c->prm.device;
    v->stream = c->stream;
    if (!v->fp32) return;
    v->P = c->Pf;
    v->hot = hot_n<float>(c);
    v->csf = csf_of<float>(c);
    v->nl = c->nl;
    v->id = (const uint32_t *)c->srt[6];
    v->type = (const uint8_t *)c->srt[5];
    v->err = &c->sc->err;
}

extern "C" {

// ---------------------------------------------------------------------------
// Learned-surrogate step, in three stages so that a batch of contexts shares
// its host synchronisations: begin (checks, reuse decision, snapshot, and the
// start evaluation when the last one cannot be reused), enqueue (prediction,
// update, end evaluation, residual sums, copies to the host), decide (after
// the stream synchronised: accept, or restore and enqueue k plain steps).
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct SgArgs {
    sph_mpnn *net;
    int k;
    double u_ref, a_ref, threshold;
    int bf16;
};

sph_status sg_check(sph_ctx *c, const SgArgs &g) {
    if (!g.net) return fail(c, SPH_ERR_ARG, "network is NULL");
    if (c->tsz != 4) return fail(c, SPH_ERR_ARG, "the surrogate step needs an FP32 context");
    if (c->prm.density != SPH_DENSITY_CONTINUITY)
        return fail(c, SPH_ERR_ARG, "the surrogate step needs the continuity density (Eq. 7)");
    if (g.k < 1 || g.k > 64) return fail(c, SPH_ERR_ARG, "k must lie in [1, 64]");
    if (!(g.u_ref > 0) || !(g.a_ref > 0) || !(g.threshold > 0))
        return fail(c, SPH_ERR_ARG, "u_ref, a_ref and threshold must be > 0");
    return SPH_OK;
}

// The scalars copied to the host by an enqueued copy, once the stream has
// synchronised: the context's error word decides the status.
sph_status sg_scalars_arrived(sph_ctx *c, const char *what) {
    CK(cudaStreamSynchronize(c->stream), what);
    CK(cudaGetLastError(), what);
    c->hsc_fresh = true;
    collect_profile(c);
    return status_from_err(c, c->hsc->err);
}

// Stage 1.  *pull: the start evaluation was enqueued with a copy of the
// scalars, which must arrive (sg_scalars_arrived) before stage 2.
sph_status sg_begin(sph_ctx *c, const SgArgs &g, bool *pull) {
    *pull = false;
    sph_status s = sg_check(c, g);
    if (s) return s;
    // the host scalars are current after the synchronising end of an
    // accepted surrogate step that nothing has followed (sg_ready)
    s = c->sg_ready ? SPH_OK : pull_scalars(c);
    if (s) return s;
    s = status_from_err(c, c->hsc->err);
    if (s) return s;
    if (!c->sg_an) {
        cudaError_t e = cudaSuccess;
        c->sg_an = dalloc(c, (size_t)c->cap * sizeof(float2), e);
        if (!e) c->sg_drn = dalloc(c, (size_t)c->cap * sizeof(float), e);
        if (!e) c->sg_sums = dalloc(c, 12 * sizeof(double), e);
        if (!e) c->sg_t0 = dalloc(c, (size_t)c->cap, e);
        if (!e) e = cudaMallocHost(&c->sg_hsum, 8 * sizeof(double));
        CK(e, "surrogate scratch");
    }
    // the evaluation that ended the last accepted surrogate step is this
    // step's start when nothing has touched the state since (no step, cell
    // build or state change: same counters) and its time advance kept the
    // lists (device rebuild decision)
    c->sg_reuse = c->sg_ready && c->sg_builds == c->hsc->builds && c->sg_step == c->hsc->step &&
                  !c->hsc->need_full;
    c->sg_ready = false;
    s = snapshot(c, false, true);
    if (s) return s;
    if (!c->sg_reuse) {
        // SPH at the step start on fresh lists, with the time-step
        // candidates of Eqs. 30-31; the network reads every particle's
        // normal, so none is skipped
        const uint32_t *key = enqueue_sort<float>(c);
        enqueue_build<float>(c, key);
        enqueue_eval<float>(c, hot_n<float>(c), 1, false);
        CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream),
           "copy scalars");
        *pull = true;
    }
    return SPH_OK;
}

// Stage 2 (host scalars current).
sph_status sg_enqueue(sph_ctx *c, const SgArgs &g) {
    c->n_eval = c->hsc->nsrt;
    c->csf_valid = true;
    const int n = c->hsc->nsrt;
    State<float> raw = state_of<float>(c->raw), srt = state_of<float>(c->srt);
    // Eq. 32: the plain step's dt at this state; the surrogate step spans k
    double dt = c->prm.dt_fixed;
    if (!(dt > 0)) {
        float m = 3.0e38f;
        for (int q = 0; q < RED_SLOTS; ++q) {
            float v;
            std::memcpy(&v, &c->hsc->dtmin_f[q], sizeof v);
            m = std::min(m, v);
        }
        if (!(m < 1.0e37f)) {
            snapshot(c, true);
            return fail(c, SPH_ERR_STATE, "adaptive time step without fluid particles");
        }
        dt = c->prm.courant * (double)m;
    }
    const double dT = g.k * dt;
    c->sg_dT = dT;
    CK(cudaMemcpyAsync(c->sg_an, c->acc, (size_t)n * sizeof(float2), cudaMemcpyDeviceToDevice,
                       c->stream), "copy");
    CK(cudaMemcpyAsync(c->sg_drn, c->dr, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice,
                       c->stream), "copy");
    // prediction and update; the time advance lays inflow layers and decides
    // (cadence and displacements) whether the next step rebuilds the lists
    const float2 *abar = nullptr;
    sph_status s = mpnn_predict(g.net, c, g.u_ref, g.bf16 != 0, &abar, &c->sg_net);
    if (s) return fail(c, s, "surrogate: %s", sph_mpnn_last_error(g.net));
    double *ym = (double *)c->sg_sums + 8;
    CK(cudaMemsetAsync(c->sg_sums, 0, 12 * sizeof(double), c->stream), "clear");
    launch_surrogate_mean(n, srt.type, srt.mass, abar, ym, c->cap, c->stream);
    launch_surrogate_update(c->Pf, c->inf, c->grid, c->sc, srt, raw, (const float2 *)c->sg_an,
                            abar, ym, (float)g.a_ref, (const float *)c->sg_drn, dT,
                            (uint8_t *)c->sg_t0, c->cap, c->stream);
    launch_spawn<float>(c->Pf, c->inf, c->sc, raw, c->layer_y, c->cap, c->cadence, c->stream);
    // SPH at the end, on the cell order and lists of the start (exact while
    // no particle moved more than skin/2, which the refresh checks), with the
    // time-step candidates, so that it can start the next surrogate step
    launch_refresh<float>(c->Pf, c->grid, c->sc, c->cs.key, raw, srt, hot_n<float>(c), c->cap,
                          c->stream);
    enqueue_cells<float>(c, false);
    enqueue_eval<float>(c, hot_n<float>(c), 1, false);
    launch_surrogate_residual(n, (const uint8_t *)c->sg_t0, srt.type, srt.mass, abar, ym,
                              (float)g.a_ref,
                              (const float2 *)c->sg_an, (const float2 *)c->acc,
                              (const float *)c->sg_drn, (const float *)c->dr,
                              (double *)c->sg_sums, c->cap, c->stream);
    CK(cudaMemcpyAsync(c->sg_hsum, c->sg_sums, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream), "residual");
    CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream),
       "copy scalars");
    CK(cudaGetLastError(), "surrogate launch");
    return SPH_OK;
}

// Stage 3 (after sg_scalars_arrived gave s): res = (r_m, r_rho, r_a);
// *replay: the step was rejected and k plain steps are enqueued (the caller
// synchronises with sph_sync).
sph_status sg_decide(sph_ctx *c, const SgArgs &g, sph_status s, int *accepted, double res[3],
                     bool *replay) {
    *replay = false;
    *accepted = 0;
    const double *sums = c->sg_hsum;
    const double dT = c->sg_dT;
    res[0] = sums[2] > 0 ? std::sqrt(sums[0] * sums[0] + sums[1] * sums[1]) / sums[2] : 0.0;
    res[1] = sums[4] > 0 ? 0.5 * dT * std::sqrt(sums[3] / sums[4]) / c->prm.rho0 : 0.0;
    res[2] = sums[6] > 0 ? std::sqrt(sums[5] / sums[6]) : 0.0;
    if (s && s != SPH_ERR_SKIN) return s;
    if (s == SPH_ERR_SKIN || !(res[0] <= g.threshold && res[1] <= g.threshold)) {
        // moved too far for the lists, or judged off: plain steps instead
        sph_status r = snapshot(c, true);
        if (!r) r = sph_run_async(c, g.k);
        *replay = r == SPH_OK;
        return r;
    }
    // plain steps after this one rebuild first; a next surrogate step may
    // start from the evaluation just done
    c->force_full = true;
    c->sg_ready = true;
    c->sg_builds = c->hsc->builds;
    c->sg_step = c->hsc->step;
    *accepted = 1;
    return SPH_OK;
}

}  // namespace

extern "C" {

sph_status sph_surrogate_batch(sph_ctx *const *ctx, int m, sph_mpnn *net, int k, double u_ref,
                               double a_ref, double threshold, int bf16, int *accepted,
                               double *res_momentum, double *res_density, double *res_field,
                               int *bad_member) {
    if (bad_member) *bad_member = -1;
    if (m < 0 || (m > 0 && !ctx)) return SPH_ERR_ARG;
    for (int i = 0; i < m; ++i)
        if (!ctx[i]) {
            if (bad_member) *bad_member = i;
            return SPH_ERR_ARG;
        }
    const SgArgs g{net, k, u_ref, a_ref, threshold, bf16};
    auto bad = [&](int i, sph_status s) {
        if (bad_member) *bad_member = i;
        return s;
    };
    std::vector<char> pull(m, 0), replay(m, 0);
    // argument errors before any member is touched
    for (int i = 0; i < m; ++i) {
        if (accepted) accepted[i] = 0;
        sph_status s = sg_check(ctx[i], g);
        if (s) return bad(i, s);
    }
    for (int i = 0; i < m; ++i) {
        bool p = false;
        sph_status s = sg_begin(ctx[i], g, &p);
        if (s) return bad(i, s);
        pull[i] = p;
    }
    for (int i = 0; i < m; ++i) {
        if (!pull[i]) continue;
        sph_status s = sg_scalars_arrived(ctx[i], "surrogate: evaluation at the start");
        if (s) return bad(i, s);
    }
    for (int i = 0; i < m; ++i) {
        sph_status s = sg_enqueue(ctx[i], g);
        if (s) return bad(i, s);
    }
    for (int i = 0; i < m; ++i) {
        sph_status s = sg_scalars_arrived(ctx[i], "surrogate: evaluation at the end");
        int acc = 0;
        double res[3];
        bool rp = false;
        s = sg_decide(ctx[i], g, s, &acc, res, &rp);
        if (s) return bad(i, s);
        replay[i] = rp;
        if (accepted) accepted[i] = acc;
        if (res_momentum) res_momentum[i] = res[0];
        if (res_density) res_density[i] = res[1];
        if (res_field) res_field[i] = res[2];
    }
    for (int i = 0; i < m; ++i) {
        if (!replay[i]) continue;
        sph_status s = sph_sync(ctx[i]);
        if (s) return bad(i, s);
    }
    return SPH_OK;
}

sph_status sph_surrogate_step(sph_ctx *c, sph_mpnn *net, int k, double u_ref, double a_ref,
                              double threshold, int bf16, int *accepted, double *res_momentum,
                              double *res_density, double *res_field) {
    if (!c) return SPH_ERR_ARG;
    int acc = 0;
    double rm = 0.0, rd = 0.0, rf = 0.0;
    sph_status s = sph_surrogate_batch(&c, 1, net, k, u_ref, a_ref, threshold, bf16, &acc, &rm,
                                       &rd, &rf, nullptr);
    if (accepted) *accepted = acc;
    if (res_momentum) *res_momentum = rm;
    if (res_density) *res_density = rd;
    if (res_field) *res_field = rf;
    return s;
}

// ---------------------------------------------------------------------------
// Ensembles
// ---------------------------------------------------------------------------
}  // extern "C"

struct sph_ensemble {
    std::vector<sph_ctx *> m;
    std::vector<unsigned long long> gen;   // member graph generations captured
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev = nullptr;              // orders member streams and the ensemble stream
    std::string err;
};

namespace {
std::string g_ens_error;

sph_status ens_fail(sph_ensemble *e, sph_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (e) e->err = buf; else g_ens_error = buf;
    return st;
}

#define ECK(e, call, what)                                                                        \
    do {                                                                                          \
        cudaError_t ce_ = (call);                                                                 \
        if (ce_ != cudaSuccess)                                                                   \
            return ens_fail((e), ce_ == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA,   \
                            "%s: %s", (what), cudaGetErrorString(ce_));                           \
    } while (0)

// Captures one step of every member as parallel branches of one graph.
sph_status ens_ensure_graph(sph_ensemble *e) {
    bool stale = !e->exec;
    for (size_t k = 0; k < e->m.size() && !stale; ++k) stale = e->gen[k] != e->m[k]->graph_gen;
    if (!stale) return SPH_OK;
    if (e->exec) { cudaGraphExecDestroy(e->exec); e->exec = nullptr; }
    if (e->graph) { cudaGraphDestroy(e->graph); e->graph = nullptr; }
    ECK(e, cudaGraphCreate(&e->graph, 0), "ensemble graph");
    for (size_t k = 0; k < e->m.size(); ++k) {
        sph_status s = append_step(e->m[k], e->graph);
        if (s) return ens_fail(e, s, "member %zu: %s", k, e->m[k]->err.c_str());
        e->gen[k] = e->m[k]->graph_gen;
    }
    ECK(e, cudaGraphInstantiate(&e->exec, e->graph, 0), "instantiate ensemble graph");
    return SPH_OK;
}
}  // namespace

extern "C" {

sph_status sph_ensemble_create(sph_ctx *const *members, int n, void *cuda_stream,
                               sph_ensemble **out) {
    if (!out) return ens_fail(nullptr, SPH_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!members || n < 1) return ens_fail(nullptr, SPH_ERR_ARG, "need n >= 1 members");
    for (int k = 0; k < n; ++k) {
        if (!members[k]) return ens_fail(nullptr, SPH_ERR_ARG, "member %d is NULL", k);
        for (int j = 0; j < k; ++j)
            if (members[j] == members[k])
                return ens_fail(nullptr, SPH_ERR_ARG, "member %d repeats member %d", k, j);
        if (members[k]->prm.device != members[0]->prm.device)
            return ens_fail(nullptr, SPH_ERR_ARG, "members are on different devices");
    }
    sph_ensemble *e = new (std::nothrow) sph_ensemble();
    if (!e) return ens_fail(nullptr, SPH_ERR_OOM, "host allocation failed");
    e->m.assign(members, members + n);
    e->gen.assign((size_t)n, ~0ull);
    auto bail = [&](cudaError_t ce, const char *what) {
        ens_fail(nullptr, SPH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(ce));
        sph_ensemble_destroy(e);
        return SPH_ERR_CUDA;
    };
    cudaError_t ce = cudaSetDevice(members[0]->prm.device);
    if (ce != cudaSuccess) return bail(ce, "cudaSetDevice");
    if (cuda_stream) {
        e->stream = (cudaStream_t)cuda_stream;
    } else {
        ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return bail(ce, "stream");
        e->own_stream = true;
    }
    ce = cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(ce, "event");
    *out = e;
    return SPH_OK;
}

sph_status sph_ensemble_run(sph_ensemble *e, long long nsteps) {
    if (!e) return SPH_ERR_ARG;
    if (nsteps < 0) return ens_fail(e, SPH_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return SPH_OK;
    sph_status s = ens_ensure_graph(e);
    if (s) return s;
    for (sph_ctx *c : e->m) {
        ECK(e, cudaEventRecord(e->ev, c->stream), "order members");
        ECK(e, cudaStreamWaitEvent(e->stream, e->ev, 0), "order members");
    }
    for (sph_ctx *c : e->m) c->sg_ready = false;
    for (long long k = 0; k < nsteps; ++k) {
        for (sph_ctx *c : e->m) {
            if (c->force_full && c->cadence > 1)
                ECK(e, cudaMemsetAsync(&c->sc->need_full, 0x01, sizeof(int), e->stream),
                    "force rebuild");
            c->force_full = false;
        }
        ECK(e, cudaGraphLaunch(e->exec, e->stream), "ensemble graph launch");
    }
    ECK(e, cudaEventRecord(e->ev, e->stream), "order members");
    for (sph_ctx *c : e->m) {
        ECK(e, cudaStreamWaitEvent(c->stream, e->ev, 0), "order members");
        c->hsc_fresh = false;
        c->n_eval = -1;
        c->csf_valid = false;
    }
    return SPH_OK;
}

sph_status sph_ensemble_sync(sph_ensemble *e, int *bad_member) {
    if (bad_member) *bad_member = -1;
    if (!e) return SPH_ERR_ARG;
    ECK(e, cudaStreamSynchronize(e->stream), "ensemble synchronize");
    for (size_t k = 0; k < e->m.size(); ++k) {
        sph_status s = sph_sync(e->m[k]);
        if (s) {
            if (bad_member) *bad_member = (int)k;
            return ens_fail(e, s, "member %zu: %s", k, e->m[k]->err.c_str());
        }
    }
    return SPH_OK;
}

sph_status sph_ensemble_surrogate_step(sph_ensemble *e, sph_mpnn *net, int k, double u_ref,
                                       double a_ref, double threshold, int bf16, int *accepted,
                                       double *res_momentum, double *res_density,
                                       double *res_field, int *bad_member) {
    if (bad_member) *bad_member = -1;
    if (!e) return SPH_ERR_ARG;
    sph_status s = sph_ensemble_sync(e, bad_member);
    if (s) return s;
    s = sph_surrogate_batch(e->m.data(), (int)e->m.size(), net, k, u_ref, a_ref, threshold, bf16,
                            accepted, res_momentum, res_density, res_field, bad_member);
    if (s) {
        int b = bad_member ? *bad_member : -1;
        return ens_fail(e, s, "member %d: %s", b,
                        b >= 0 && b < (int)e->m.size() ? e->m[b]->err.c_str() : "");
    }
    return SPH_OK;
}

sph_status sph_ensemble_autotune(sph_ensemble *e, int trial_steps, int *lanes, int *cadence,
                                 double *ms_per_step) {
    if (!e) return SPH_ERR_ARG;
    if (trial_steps < 1 || trial_steps > 10000)
        return ens_fail(e, SPH_ERR_ARG, "trial_steps in [1, 10000]");
    sph_status s = sph_ensemble_sync(e, nullptr);
    if (s) return s;
    for (sph_ctx *c : e->m) {
        s = snapshot(c, false);
        if (s) return ens_fail(e, s, "snapshot: %s", c->err.c_str());
    }
    const int L[4] = {1, 2, 4, 8}, K[4] = {1, 2, 4, 8};
    int bestL = e->m[0]->lanes, bestK = e->m[0]->cadence, bestF = e->m[0]->start_form;
    double best = 1e300;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    ECK(e, cudaEventCreate(&t0), "event");
    ECK(e, cudaEventCreate(&t1), "event");
    auto restore_all = [&]() -> sph_status {
        for (sph_ctx *c : e->m) {
            sph_status r = snapshot(c, true);
            if (r) return r;
        }
        return SPH_OK;
    };
    // one candidate from the snapshots: a warm cycle (capture), then at least
    // two rebuild cycles timed; SPH_ERR_SKIN rejects the candidate only
    auto trial = [&](int Lv, int Kv, int Fv) -> sph_status {
        int steps = std::max(trial_steps, 2 * Kv);
        sph_status t = restore_all();
        for (size_t k = 0; k < e->m.size() && !t; ++k) {
            t = sph_set_tuning(e->m[k], Lv, Kv);
            if (!t) t = sph_set_start_form(e->m[k], Fv);
        }
        if (!t) t = sph_ensemble_run(e, Kv);
        if (!t) t = sph_ensemble_sync(e, nullptr);
        if (t) return t;
        cudaEventRecord(t0, e->stream);
        t = sph_ensemble_run(e, steps);
        cudaEventRecord(t1, e->stream);
        if (!t) t = sph_ensemble_sync(e, nullptr);
        if (t) return t;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        double per = ms / steps;
        if (per < best) { best = per; bestL = Lv; bestK = Kv; bestF = Fv; }
        return SPH_OK;
    };
    // lanes x cadence up to 8 in both start forms, then longer cadences at
    // the best lane count
    for (int a = 0; a < 4 && !s; ++a)
        for (int b = 0; b < 4 && !s; ++b)
            for (int f = 0; f < (K[b] > 1 ? 2 : 1) && !s; ++f) {
                s = trial(L[a], K[b], f == 0 ? SPH_START_GATED : SPH_START_CONDITIONAL);
                if (s == SPH_ERR_SKIN) { s = SPH_OK; break; }   // cadence too long here
            }
    if (best < 1e300 && !s) {
        int L0 = bestL;
        for (int Kv = 16; Kv <= 32 && !s; Kv *= 2)
            for (int f = 0; f < 2 && !s; ++f) {
                s = trial(L0, Kv, f == 0 ? SPH_START_GATED : SPH_START_CONDITIONAL);
                if (s == SPH_ERR_SKIN) { s = SPH_OK; break; }
            }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    sph_status r = restore_all();
    if (s) return s;
    if (r) return ens_fail(e, r, "restore failed");
    if (best >= 1e300) return ens_fail(e, SPH_ERR_STATE, "no tuning candidate ran without error");
    for (sph_ctx *c : e->m) {
        r = sph_set_tuning(c, bestL, bestK);
        if (!r) r = sph_set_start_form(c, bestF);
        if (r) return ens_fail(e, r, "%s", c->err.c_str());
    }
    if (lanes) *lanes = bestL;
    if (cadence) *cadence = bestK;
    if (ms_per_step) *ms_per_step = best;
    return SPH_OK;
}

void sph_ensemble_destroy(sph_ensemble *e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    if (e->ev) cudaEventDestroy(e->ev);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

const char *sph_ensemble_last_error(const sph_ensemble *e) {
    return e ? e->err.c_str() : g_ens_error.c_str();
}

}  // extern "C"
