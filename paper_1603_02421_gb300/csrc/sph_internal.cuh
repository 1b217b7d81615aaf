// Internal device-side declarations of libsph (not part of the C ABI).
//
// Data layout in HBM (all arrays sized for the context's capacity):
//  * "raw" particle state: the integrator's output, in the order of the
//    last cell sort, plus particles laid by the inflow appended at the end.
//  * "srt" particle state: raw gathered into cell order by the sort.
//  * hot per-evaluation records in cell order, read by the pair sweeps with
//    one vector load per candidate:
//      H0 = (x_off, y_off, u', v')  offset in the particle's cell, velocity
//                                   relative to the frame u_frame
//      H1 = (V, rho, P/rho^2, c)  volume m/rho, density, pressure term, sound speed
//    plus colour C, normal n and unit normal nhat for the CSF terms.
//  * positions are FP64 everywhere; pair arithmetic runs in T (float or double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sph.h"

namespace sph {

constexpr uint8_t T_FLUID = 0, T_BOUNDARY = 1, T_BUFFER = 2, T_DEAD = 0xFF;
enum ErrBits : unsigned {
    ERR_NONFINITE = 1u,
    ERR_SKIN = 2u,
    ERR_CAPACITY = 4u,
    ERR_TIMEOUT = 8u,
    ERR_NODT = 16u,
    ERR_NLIST = 32u,
    ERR_BOUNDS = 64u
};

struct __align__(16) f4 { float x, y, z, w; };
struct __align__(32) d4 { double x, y, z, w; };

template <class T> struct Vec;
template <> struct Vec<float> { using v2 = float2; using v4 = f4; };
template <> struct Vec<double> { using v2 = double2; using v4 = d4; };

// Uniform cell grid: cell size sc = 2h + skin; one empty padding cell on each
// side so the 3x3 block of any occupied cell stays inside the grid.  Cell keys
// run along x first: key = cy * ncx + cx.
struct Grid {
    double xmin, ymin, xmax, ymax, sc, inv_sc;
    int ncx, ncy;
    unsigned ncells, sentinel;   // sentinel key sorts after every cell
    int keybits;
    long long kxmin, kymin, kxmax, kymax;   // ordered_key of the box bounds
};

// Orders doubles as signed 64-bit integers: for non-NaN a and b, a < b
// exactly when ordered_key(a) < ordered_key(b) (-0 and +0 share the key 0).
// A NaN lies above +inf or below -inf by its sign bit, so it passes no
// two-sided bound test, as it passes no double comparison.  Bound tests on
// the keys run on the integer pipes instead of the FP64 pipe.
__host__ __device__ inline long long ordered_key(double d) {
#ifdef __CUDA_ARCH__
    long long b = __double_as_longlong(d);
#else
    long long b;
    memcpy(&b, &d, sizeof b);
#endif
    return b >= 0 ? b : -(b & 0x7FFFFFFFFFFFFFFFLL);
}

// Completes a grid whose box, cell size and cell counts are set.
inline void grid_finish(Grid &g) {
    g.kxmin = ordered_key(g.xmin);
    g.kymin = ordered_key(g.ymin);
    g.kxmax = ordered_key(g.xmax);
    g.kymax = ordered_key(g.ymax);
    g.ncells = (unsigned)(g.ncx * g.ncy);
    int bits = 1;
    while (((1ull << bits) - 1ull) < (unsigned long long)g.ncells) ++bits;
    g.keybits = bits;
    g.sentinel = (uint32_t)((1ull << bits) - 1ull);
}

__host__ __device__ __forceinline__ uint32_t grid_key(const Grid &g, int cx, int cy) {
    return (uint32_t)cy * (uint32_t)g.ncx + (uint32_t)cx;
}

__host__ __device__ __forceinline__ void grid_cell(const Grid &g, uint32_t key, int &cx, int &cy) {
    cy = (int)(key / (uint32_t)g.ncx);
    cx = (int)key - cy * g.ncx;
}

// Fixed-point cell offsets of the FP32 records (see off_diff in
// sph_device.cuh): 2^29 units per cell edge sc, held as int32 bits.
constexpr int OFF_BITS = 29;
constexpr double OFF_ONE = 536870912.0;

__host__ __device__ __forceinline__ int off_fixed(double off, double sc) {
    double u = off * (OFF_ONE / sc);
    return (int)(u >= 0.0 ? u + 0.5 : u - 0.5);   // round half away from zero
}

// Physical constants, converted once to the pair-arithmetic type T.
template <class T> struct PhysT {
    int kernel;          // 0 cubic, 1 Wendland
    int csf;             // sigma > 0
    int walls;           // boundary particles present
    int gamma7;          // gamma == 7: Eq. 26 as an exact polynomial
    int summation;       // fluid density from Eq. 6 at each evaluation
    T h, inv_h, H2lo, H2hi, R15lo, R15hi;
    T RL2hi;             // squared neighbour-list radius (2h + skin)^2, widened
    T sc;
    T wn, gn;            // kernel factors: W = wn f(q), (1/r) dW/dr = gn g(q)
    T W0;                // W(0)
    T rho0, inv_rho0, B, gamma, c0, half_gm1;
    T alpha_h, eta2, sigma, eps_n;
    T gx, gy;
    T wall_A, wall_db, inv_wall_db, wall_h0, inv_wall_h0, two_h, c0_inv;
    T ufx, ufy;          // velocity frame: stored velocities are u - u_frame
    T half_skin;         // skin / 2
    // displacement since the list build is measured relative to a frame
    // moving at (dfx, dfy): the velocity frame without walls (a common
    // translation changes no pair separation), zero with walls (their
    // contacts are found by walking the build-time cells)
    T dfx, dfy;
    T cell_lo, cell_hi;  // bounds of a particle's offset from its build-time cell,
                         // stored as the offsets are (fixed point in FP32)
    T off_unit;          // FP32: length of one fixed-point offset unit, sc / 2^29
    T off_scale;         // FP32: its inverse, 2^29 / sc
    double H2d, R15d;    // exact FP64 thresholds (2h)^2, (1.5h)^2
    double courant, dt_fixed;
    double ufx_d, ufy_d;
    double half_skin2;   // (skin/2)^2: largest displacement between list build and use
    // bounds-check build (SPH_BOUNDS_CHECK): particle indices the walks meet
    // must lie below cap; one that does not sets ERR_BOUNDS in *err and is
    // skipped
    int cap;
    unsigned *err;
};

// Inflow of the planar jet.
struct Inflow {
    int on;
    int layers, ny;
    double x_exit, y0, y1, U, amp, k, phase, dx, m_layer, threshold;
};

// Device-resident scalars of a context.
struct Scalars {
    int n;                        // raw particle count (incl. dead-marked)
    int nsrt;                     // particles in the current cell order
    unsigned next_id;
    unsigned err;                 // ErrBits, sticky
    float last_dmax;              // rebuild decision of the last step: largest
    float last_smax;              //   displacement since the build, largest move
    double dt, t, x_up;
    long long step, deleted;
    long long builds;             // cell sorts run (steps and other calls)
    unsigned long long xmax_key;  // breakup: ordered bits of max x of the jet
    unsigned detached;            // breakup: particles outside the jet
    unsigned long long pair_count;  // pairs found by the pair export (64-bit: dense
                                    // inputs can exceed 2^32 ordered pairs)
    int need_full;                // next step rebuilds the cells and lists
    int since_full;               // steps since the last rebuild
    // reductions spread over RED_SLOTS addresses (slot = block index mod
    // RED_SLOTS) so that thousands of blocks do not serialise on one atomic;
    // the next kernel folds the slots
    unsigned long long dtmin_d[32];  // double bits of min_a dt candidate (FP64 path)
    unsigned dtmin_f[32];         // float bits (FP32 path)
    unsigned max_disp2[32];       // float bits: max |displacement since the rebuild|^2
    unsigned max_step2[32];       // float bits: max |displacement in this step|^2
};
constexpr int RED_SLOTS = 32;

// Which start of a step a kernel belongs to.  A step graph holds both starts
// (rebuild: sort + list build; reuse: refresh of the last build) in one
// straight line; each start kernel reads the flag the previous step left in
// sc->need_full and returns at once when its start is not the one taken.
// Kernels launched outside such a graph run unconditionally.
enum Gate : int { GATE_ALWAYS = -1, GATE_REUSE = 0, GATE_FULL = 1 };

__device__ __forceinline__ bool gate_skips(int gate, const Scalars *sc) {
    return gate >= 0 && (sc->need_full != 0) != (gate == GATE_FULL);
}

template <class T> struct State {
    double2 *pos;
    typename Vec<T>::v2 *vel;
    T *drho, *drc;                // density offset rho - rho0 and its Kahan carry
    T *mass;
    uint8_t *type;
    uint32_t *id;
    typename Vec<T>::v2 *disp;    // displacement since the last cell build
};

template <class T> struct Hot {
    typename Vec<T>::v4 *H0, *H1;
    double2 *pos;                 // FP64 positions of this evaluation
};

template <class T> struct Csf {
    T *C;
    typename Vec<T>::v4 *CX;      // (x_off, y_off, V, C) for the normal sweep
    typename Vec<T>::v2 *nhat;    // unit normal, zero where the filter N_a = 0
    typename Vec<T>::v2 *nvec;    // normal n_a of Eq. 18
};

struct Boundary {
    int n;
    const uint2 *cellSE;          // per-cell [start, end) into the sorted boundary arrays
    const void *bh;               // Vec<T>::v4 (x_loc, y_off, nx, ny), cell order
    const double2 *pos;           // FP64 positions, cell order
};

// Counting sort of the particles by cell (Sec. 2-7 cell linked list laid out
// as contiguous cell ranges).
struct CellSort {
    uint32_t *knew;     // [cap] cell key of each raw particle (sentinel: dead)
    uint32_t *count;    // [ncells] per-cell counters, zero between sorts
    uint32_t *tmp;      // [cap] raw index at its provisional slot
    uint32_t *key;      // [cap] cell key of each sorted particle
    uint32_t *bsum;     // [nscan] cell totals of each scan block
    uint2 *cellSE;      // [ncells] [start, end) of every cell in the sorted order
    int nscan;          // scan blocks of SCAN_CELLS cells
};

// Kernel launch through cudaLaunchKernelEx (plain stream order).
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CELLS = SCAN_THREADS * SCAN_ITEMS;
constexpr int SWEEP_BLOCK = 128;    // threads per block of the pair sweeps
// lanes: threads cooperating on one particle's neighbour loop (1, 2, 4 or 8)
constexpr int LIST_SLOTS = 96;      // neighbour-list entries per particle

// Verlet neighbour list built once per step from the cell block (radius
// 2h + skin, so it still holds every pair closer than 2h at the half step).
// Entry = b | (sx + 1) << 28 | (sy + 1) << 30 with (sx, sy) = cell of the
// particle minus cell of b; the entries of particle i are contiguous at
// e[i * LIST_SLOTS + k], k < cnt[i].
struct NList {
    uint32_t *e;
    uint32_t *cnt;
};

// ---- launchers (sph_neighbour.cu) ----
// hash + count -> scan -> provisional scatter; leaves cs.cellSE final, cs.tmp
// holding raw indices grouped by cell (in arbitrary order within a cell) and
// sc->nsrt the live particle count.
template <class T>
void launch_cell_sort(const Grid &g, const State<T> &raw, Scalars *sc, CellSort &cs, int cap,
                      cudaStream_t s, int gate = GATE_ALWAYS);
// Exports every ordered pair closer than 2h; sc->pair_count receives the total
// (slots beyond cap are counted but not written).  Returns the first error of
// the enqueued memset and launch.
template <class T>
cudaError_t launch_pairs(const PhysT<T> &P, const Grid &g, Scalars *sc, const uint2 *cellSE,
                         const uint32_t *key, const Hot<T> &hot, const uint32_t *ids,
                         unsigned *out_a, unsigned *out_b, unsigned long long cap, int ncap,
                         cudaStream_t s);
template <class T>
void launch_breakup(const PhysT<T> &P, const Grid &g, Scalars *sc, const uint2 *cellSE,
                    const uint32_t *key, const Hot<T> &hot, const uint8_t *type,
                    uint32_t *parent, uint8_t *flag, int cap, cudaStream_t s);

// ---- launchers (sph_sweeps.cu) ----
// Final rank of each particle inside its cell (by raw index, so the order is
// deterministic and stable), gather raw -> cell order, records of evaluation n.
template <class T>
void launch_reorder(const PhysT<T> &P, const Grid &g, Scalars *sc, const CellSort &cs,
                    const State<T> &raw, const State<T> &srt, const Hot<T> &hot, int cap,
                    cudaStream_t s, int gate = GATE_ALWAYS);
// Neighbour list of evaluation n; with_colour also sums the colour (Eq. 14).
template <class T>
void launch_build(int lanes, bool with_colour, const PhysT<T> &P, const Grid &g, Scalars *sc,
                  const uint2 *cellSE, const uint32_t *key, const Hot<T> &hot, const NList &nl,
                  const Csf<T> &csf, int cap, cudaStream_t s, int gate = GATE_ALWAYS);
template <class T>
void launch_colour(int lanes, const PhysT<T> &P, const Scalars *sc, const NList &nl,
                   const Hot<T> &hot, const Csf<T> &csf, int cap, cudaStream_t s,
                   int gate = GATE_ALWAYS);
// Eq. 6 density of the fluid particles; rewrites their H1 records (and
// stores rho - rho0 to drho_out when given).
template <class T>
void launch_density(int lanes, const PhysT<T> &P, const Scalars *sc, const NList &nl,
                    const Hot<T> &hot, const T *mass, const uint8_t *type, T *drho_out, int cap,
                    cudaStream_t s, int gate = GATE_ALWAYS);
// Normal, filter and unit normal (Eqs. 18, 20, 21).  With gsum (the bound
// G_a of launch_pairsum) and crange (the colour range of every cell), particles
// whose normal provably stays below the filter threshold are not walked (their
// n is written as zero); with gsum null every particle is walked.
template <class T>
void launch_normal(int lanes, const PhysT<T> &P, const Scalars *sc, const NList &nl,
                   const Hot<T> &hot, const Csf<T> &csf, int cap, cudaStream_t s,
                   const uint32_t *key = nullptr, const T *gsum = nullptr,
                   const uint2 *crange = nullptr, int ncx = 0);
// With surface tension: the one full list walk of an evaluation -- colour
// (Eq. 14, to csf.C and csf.CX) and, for fluid particles, the pair sums that
// need only the state (Eqs. 7, 9, 10, 29, 31) to accN = (ax, ay, drho/dt,
// max Eq. 31 term, or 0 unless dt_term: only an evaluation whose end takes
// the time step needs it); gsum_a = sum_b V_b |grad_a W_ab|; the colour range
// of each cell to crange (min, ~max as float bits; reset to all ones before).
template <class T>
void launch_pairsum(int lanes, const PhysT<T> &P, const Grid &g, const Scalars *sc,
                    const NList &nl, const uint32_t *key, const Hot<T> &hot, const Csf<T> &csf,
                    const Boundary &bd, const uint8_t *type, typename Vec<T>::v4 *accN, T *gsum,
                    uint2 *crange, int cap, cudaStream_t s, bool dt_term);
// With surface tension: curvature (Eq. 23) of the particles with N_a = 1, CSF
// acceleration (Eq. 24), gravity, and the end of launch_forces' mode (0, 1
// or 2) from the sums of launch_pairsum.
template <class T>
void launch_surface(int lanes, int mode, const PhysT<T> &P, const Grid &g, const Inflow &inf,
                    Scalars *sc, const NList &nl, const Hot<T> &hot, const Csf<T> &csf,
                    const State<T> &srt, const State<T> &raw, const typename Vec<T>::v4 *accN,
                    typename Vec<T>::v2 *acc, T *dr, int cap, cudaStream_t s,
                    typename Vec<T>::v4 *nH0 = nullptr, typename Vec<T>::v4 *nH1 = nullptr);
// mode 0: evaluate only (store derivatives, copy srt -> raw); mode 1: first
// evaluation of a step (store derivatives, time-step minimum); mode 2:
// second evaluation + corrector (write the new state to raw, and in place to
// srt with the records of the next evaluation in nH0 / nH1, on the cells of
// the last build).
template <class T>
void launch_forces(int lanes, int mode, const PhysT<T> &P, const Grid &g, const Inflow &inf,
                   Scalars *sc, const NList &nl, const uint32_t *key, const Hot<T> &hot,
                   const Csf<T> &csf, const Boundary &bd, const State<T> &srt,
                   const State<T> &raw, typename Vec<T>::v2 *acc, T *dr, int cap,
                   cudaStream_t s, typename Vec<T>::v4 *nH0 = nullptr,
                   typename Vec<T>::v4 *nH1 = nullptr);
// raw -> srt in the same order, records of evaluation n relative to the cells
// of the last build (the learned surrogate's judge evaluation; a plain step
// that keeps the build gets these from the corrector).
template <class T>
void launch_refresh(const PhysT<T> &P, const Grid &g, Scalars *sc, const uint32_t *key,
                    const State<T> &raw, const State<T> &srt, const Hot<T> &hot, int cap,
                    cudaStream_t s, int gate = GATE_ALWAYS);
template <class T>
void launch_predict(const PhysT<T> &P, const Inflow &inf, Scalars *sc, const State<T> &srt,
                    const typename Vec<T>::v4 *H0n, const typename Vec<T>::v2 *acc, const T *dr,
                    const Hot<T> &half, int cap, cudaStream_t s);
// End of a step: lays a due inflow layer, advances time, and decides whether
// the next step rebuilds the cells (a layer was laid, `cadence` steps have
// passed, or the displacement since the last rebuild may reach skin/2 within
// the next step).
template <class T>
void launch_spawn(const PhysT<T> &P, const Inflow &inf, Scalars *sc, const State<T> &raw,
                  const double *layer_y, int cap, int cadence, cudaStream_t s);
// Run statistics of raw[0, sc->n) (see sph_stats): acc[6] FP64 sums, cnt[3]
// (fluid count, buffer count, bits of max |rho - rho0|/rho0), both zeroed
// by the caller.
template <class T>
void launch_stats(const PhysT<T> &P, const State<T> &raw, const Scalars *sc, double gx, double gy,
                  double rho0, double B, double gamma, double *acc, unsigned long long *cnt,
                  int cap, cudaStream_t s);
// Host stub of the one-thread kernel that sets a step graph's IF-node
// condition from sc->need_full (the conditional step form).
void *decide_kernel();
// Learned-surrogate step (FP32 contexts): the mass-weighted mean of the
// network output over the fluid (ym[3], zeroed by the caller), the state
// update with the predicted mean acceleration a_n + a_ref (y - ybar), and the
// residual sums against the SPH evaluations at both ends.
void launch_surrogate_mean(int n, const uint8_t *type, const float *mass, const float2 *y,
                           double *ym, int cap, cudaStream_t s);
void launch_surrogate_update(const PhysT<float> &P, const Inflow &inf, const Grid &g, Scalars *sc,
                             const State<float> &srt, const State<float> &raw, const float2 *a_n,
                             const float2 *y, const double *ym, float a_ref, const float *dr,
                             double dT, uint8_t *type0, int cap, cudaStream_t s);
// Residual sums of a surrogate step (k_surrogate_residual) over the particles
// fluid at both ends (type0: the start types the update recorded): sums[7],
// zeroed by the caller.
void launch_surrogate_residual(int n, const uint8_t *type0, const uint8_t *type, const float *mass,
                               const float2 *y, const double *ym, float a_ref,
                               const float2 *a_n, const float2 *a_k, const float *dr_n,
                               const float *dr_k, double *sums, int cap, cudaStream_t s);

// Read-only view of a context's last evaluation (for the learned surrogate):
// records, CSF fields and neighbour lists of the current state in cell
// order.  `evaluated` is false unless sph_evaluate ran on the current state.
struct CtxView {
    int n;                   // particles in cell order
    int cap;
    bool fp32;
    bool evaluated;
    int device;
    cudaStream_t stream;
    PhysT<float> P;
    Hot<float> hot;
    Csf<float> csf;
    NList nl;
    const uint32_t *id;      // particle ids in cell order
    const uint8_t *type;
    unsigned *err;           // the context's sticky device error word
};

}  // namespace sph

// Fills a view of context c (sph_api.cu).
struct sph_ctx;
struct sph_mpnn;
void ctx_view(struct sph_ctx *c, sph::CtxView *v);

// Scratch of the tensor-core inference pass owned by a context (sph_mpnn.cu;
// opaque here), made on first use at the context's capacity.
struct MpScratchHandle;
void mpnn_scratch_free(MpScratchHandle *h);

// Surrogate forward pass on an evaluated context (sph_mpnn.cu): *y receives
// the device array of the n predictions (float2, cell order).  bf16 selects
// the tensor-core pass, which runs in *scratch (allocated or grown here).
sph_status mpnn_predict(struct sph_mpnn *net, struct sph_ctx *c, double u_ref, bool bf16,
                        const float2 **y, MpScratchHandle **scratch);
