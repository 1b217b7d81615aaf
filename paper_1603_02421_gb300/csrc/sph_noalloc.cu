// Neighbour-pair search that allocates no device memory (sph_pairs_noalloc).
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool (whose allocator owns the device), a host
// application that must not grow its device footprint after start-up, or a
// plugin that only ever receives device buffers from its host.  This entry point takes the
// caller's device input and output buffers and keeps all of its scratch
// (cell counters, scan block sums, sort keys, the gathered positions) in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// It runs the same cell sort and the same exact pair test as the context
// entry points, so its pair set equals sph_get_pairs' on the same positions.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "sph.h"
#include "sph_device.cuh"

using namespace sph;

namespace {

constexpr long long NA_MAX_N = 1ll << 18;        // particles per call
constexpr unsigned NA_MAX_CELLS = 1u << 20;      // cells of the search grid
constexpr int NA_MAX_SCAN = (int)((NA_MAX_CELLS + SCAN_CELLS - 1) / SCAN_CELLS);
constexpr int NA_MAX_DEVICES = 64;

// Byte layout of the scratch array.
struct Layout {
    size_t sc, pos, type, id, spos, sid, H0, knew, count, tmp, key, bsum, cellSE, total;
};

constexpr size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr Layout make_layout() {
    Layout L{};
    size_t o = 0;
    L.sc = o;     o = align_up(o + sizeof(Scalars));
    L.pos = o;    o = align_up(o + NA_MAX_N * sizeof(double2));
    L.type = o;   o = align_up(o + NA_MAX_N);
    L.id = o;     o = align_up(o + NA_MAX_N * 4);
    L.spos = o;   o = align_up(o + NA_MAX_N * sizeof(double2));
    L.sid = o;    o = align_up(o + NA_MAX_N * 4);
    L.H0 = o;     o = align_up(o + NA_MAX_N * sizeof(f4));
    L.knew = o;   o = align_up(o + NA_MAX_N * 4);
    L.count = o;  o = align_up(o + (size_t)NA_MAX_CELLS * 4);
    L.tmp = o;    o = align_up(o + NA_MAX_N * 4);
    L.key = o;    o = align_up(o + NA_MAX_N * 4);
    L.bsum = o;   o = align_up(o + (size_t)NA_MAX_SCAN * 4);
    L.cellSE = o; o = align_up(o + (size_t)NA_MAX_CELLS * sizeof(uint2));
    L.total = o;
    return L;
}

constexpr Layout kL = make_layout();

// The scratch: about 31 MB.  Shared by every call on a device; it keeps the
// contents of the last call.
static __device__ __align__(256) unsigned char g_pairs_scratch[kL.total];

std::mutex g_mu;
unsigned char *g_base[NA_MAX_DEVICES] = {};   // device address of g_pairs_scratch per device

// Device address of the scratch on the current device (looked up once per
// device, with that device current, and kept for the life of the process: a
// cudaDeviceReset of that device invalidates it, see include/sph.h).
cudaError_t scratch_base(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pairs_scratch);
        if (e != cudaSuccess) return e;
        g_base[dev] = (unsigned char *)p;
    }
    *out = g_base[dev];
    return cudaSuccess;
}

// Copies the caller's x, y into the scratch state; particles outside the box
// (or with a NaN coordinate) are excluded and reported in sc->err, which the
// caller cleared before this launch.
__global__ void k_na_gather(const double *__restrict__ x, const double *__restrict__ y, int n,
                            Grid g, double2 *pos, uint8_t *type, uint32_t *id, Scalars *sc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) sc->n = n;
    if (i >= n) return;
    double px = x[i], py = y[i];
    bool in = px >= g.xmin && px < g.xmax && py >= g.ymin && py < g.ymax;
    pos[i] = make_double2(px, py);
    type[i] = in ? T_FLUID : T_DEAD;
    id[i] = (uint32_t)i;
    if (!in) atomicOr(&sc->err, ERR_NONFINITE);
}

// Stable in-cell rank and gather into cell order (positions, ids, offsets).
__global__ void k_na_order(Grid g, const Scalars *__restrict__ sc, CellSort cs,
                           const double2 *__restrict__ pos, const uint32_t *__restrict__ id,
                           double2 *spos, uint32_t *sid, f4 *H0) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= sc->nsrt) return;
    uint32_t j = cs.tmp[t];
    uint32_t k = cs.knew[j];
    uint2 se = cs.cellSE[k];
    uint32_t rank = 0;
    for (uint32_t u = se.x; u < se.y; ++u) rank += cs.tmp[u] < j ? 1u : 0u;
    uint32_t i = se.x + rank;
    cs.key[i] = k;
    double2 p = pos[j];
    spos[i] = p;
    sid[i] = id[j];
    float xl, yo;
    double xo, yoo;
    cell_offsets<float>(g, k, p, xl, yo, xo, yoo);
    f4 r;
    r.x = xl; r.y = yo; r.z = 0.f; r.w = 0.f;
    H0[i] = r;
}

}  // namespace

extern "C" sph_status sph_pairs_noalloc(const double *x, const double *y, long long n, double h,
                                        double xmin, double ymin, double xmax, double ymax,
                                        unsigned *pair_a, unsigned *pair_b, long long cap,
                                        long long *npairs, void *stream) {
    if (!npairs || n < 0 || cap < 0 || !(h > 0) || !(xmax > xmin) || !(ymax > ymin))
        return SPH_ERR_ARG;
    if (n > NA_MAX_N) return SPH_ERR_CAPACITY;
    if (n > 0 && (!x || !y)) return SPH_ERR_ARG;
    if (cap > 0 && (!pair_a || !pair_b)) return SPH_ERR_ARG;
    *npairs = 0;
    // the call synchronises and reads back a count, which a stream capture
    // cannot hold: refuse before anything is enqueued
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &capture) != cudaSuccess ||
        capture != cudaStreamCaptureStatusNone)
        return SPH_ERR_ARG;
    // the grid of a context with skin_over_h = 0.1
    double sc = 2.0 * h + 0.1 * h;
    double ncx = std::floor((xmax - xmin) / sc) + 3, ncy = std::floor((ymax - ymin) / sc) + 3;
    if (ncx * ncy > (double)NA_MAX_CELLS) return SPH_ERR_CAPACITY;
    if (n == 0) return SPH_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
        return SPH_ERR_CUDA;
    unsigned char *base = nullptr;
    if (scratch_base(dev, &base) != cudaSuccess) return SPH_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;

    Grid g{};
    g.xmin = xmin; g.ymin = ymin; g.xmax = xmax; g.ymax = ymax;
    g.sc = sc; g.inv_sc = 1.0 / sc;
    g.ncx = (int)ncx; g.ncy = (int)ncy;
    grid_finish(g);

    PhysT<float> P{};
    double H = 2.0 * h, H2 = H * H, band = 2e-5;
    P.h = (float)h;
    P.inv_h = (float)(1.0 / h);
    P.H2lo = (float)(H2 * (1.0 - band));
    P.H2hi = (float)(H2 * (1.0 + band));
    P.H2d = H2;
    P.sc = (float)sc;
    P.off_unit = (float)(sc / OFF_ONE);
    P.off_scale = (float)(OFF_ONE / sc);

    Scalars *scal = (Scalars *)(base + kL.sc);
    P.cap = (int)n;
    P.err = &scal->err;
    State<float> raw{};
    raw.pos = (double2 *)(base + kL.pos);
    raw.type = base + kL.type;
    raw.id = (uint32_t *)(base + kL.id);
    CellSort cs{};
    cs.knew = (uint32_t *)(base + kL.knew);
    cs.count = (uint32_t *)(base + kL.count);
    cs.tmp = (uint32_t *)(base + kL.tmp);
    cs.key = (uint32_t *)(base + kL.key);
    cs.bsum = (uint32_t *)(base + kL.bsum);
    cs.cellSE = (uint2 *)(base + kL.cellSE);
    cs.nscan = (int)((g.ncells + SCAN_CELLS - 1) / SCAN_CELLS);
    Hot<float> hot{};
    hot.H0 = (f4 *)(base + kL.H0);
    hot.pos = (double2 *)(base + kL.spos);
    uint32_t *sid = (uint32_t *)(base + kL.sid);

    int ni = (int)n;
    // the scalars (error word, counts) and the cell counters must start at
    // zero -- the scratch keeps whatever the last call left; the rest of it is
    // fully rewritten before it is read
    if (cudaMemsetAsync(scal, 0, sizeof(Scalars), s) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaMemsetAsync(cs.count, 0, (size_t)g.ncells * 4, s) != cudaSuccess) return SPH_ERR_CUDA;
    k_na_gather<<<(ni + 255) / 256, 256, 0, s>>>(x, y, ni, g, raw.pos, raw.type, raw.id, scal);
    launch_cell_sort<float>(g, raw, scal, cs, ni, s);
    k_na_order<<<(ni + 255) / 256, 256, 0, s>>>(g, scal, cs, raw.pos, raw.id, hot.pos, sid,
                                                hot.H0);
    if (launch_pairs<float>(P, g, scal, cs.cellSE, cs.key, hot, sid, pair_a, pair_b,
                            (unsigned long long)cap, ni, s) != cudaSuccess)
        return SPH_ERR_CUDA;
    // the kernels before the pair export are checked here too
    if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
    Scalars hs;
    if (cudaMemcpyAsync(&hs, scal, sizeof(Scalars), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPH_ERR_CUDA;
    *npairs = (long long)hs.pair_count;
    if (hs.err) return SPH_ERR_ARG;
    if ((long long)hs.pair_count > cap) return SPH_ERR_CAPACITY;
    return SPH_OK;
}
