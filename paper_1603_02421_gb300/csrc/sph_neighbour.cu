// Cell-linked-list neighbour build (Sec. 2-7) and the breakup-length
// connectivity (Sec. 3-2) of libsph.
//
//  k_hash_count  FP64 position -> cell key (dead -> sentinel), per-cell count
//  k_scan_*      exclusive scan of the counts -> [start, end) of every cell
//  k_scatter     provisional slot of each particle inside its cell range
//                (the deterministic in-cell order is fixed by the reorder)
//  k_pairs     neighbour pair export (exact FP64 test in the guard band)
//  k_uf_*      union-find over links shorter than 1.5 h, jet reach
#include "sph_device.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// cell hash + per-cell count
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_hash_count(Grid g, State<T> raw, const Scalars *__restrict__ sc,
                             uint32_t *__restrict__ knew, uint32_t *__restrict__ count, int gate) {
    if (gate_skips(gate, sc)) return;
    int n = sc->n;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = g.sentinel;
    if (raw.type[i] != T_DEAD) {
        double2 p = raw.pos[i];
        int cx = (int)floor((p.x - g.xmin) * g.inv_sc) + 1;
        int cy = (int)floor((p.y - g.ymin) * g.inv_sc) + 1;
        cx = min(max(cx, 1), g.ncx - 2);
        cy = min(max(cy, 1), g.ncy - 2);
        k = grid_key(g, cx, cy);
        atomicAdd(&count[k], 1u);
    }
    knew[i] = k;
}

// ---------------------------------------------------------------------------
// exclusive scan of the cell counts (two kernels)
// ---------------------------------------------------------------------------
// Block-local scan: cellSE[k] = (prefix within the block, count); bsum[b] = total.
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_local(const uint32_t *__restrict__ count, uint2 *__restrict__ cellSE,
             uint32_t *__restrict__ bsum, unsigned ncells, const Scalars *__restrict__ sc,
             int gate) {
    if (gate_skips(gate, sc)) return;
    __shared__ uint32_t wsum[SCAN_THREADS / 32];
    unsigned base = blockIdx.x * SCAN_CELLS + threadIdx.x * SCAN_ITEMS;
    uint32_t c[SCAN_ITEMS];
    uint32_t tot = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        c[j] = base + j < ncells ? count[base + j] : 0u;
        tot += c[j];
    }
    // inclusive warp scan of the per-thread totals
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t v = wsum[lane];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        wsum[lane] = x - v;          // exclusive prefix of the warp totals
        if (lane == 31) bsum[blockIdx.x] = x;
    }
    __syncthreads();
    uint32_t run = wsum[w] + inc - tot;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (base + j < ncells) cellSE[base + j] = make_uint2(run, c[j]);
        run += c[j];
    }
}

// Adds the offset of the block (sum of the earlier block totals) and turns
// (prefix, count) into [start, end); block 0 also stores the live count.
__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_add(uint2 *__restrict__ cellSE, const uint32_t *__restrict__ bsum, unsigned ncells,
           int nblocks, Scalars *__restrict__ sc, int gate) {
    if (gate_skips(gate, sc)) return;
    __shared__ uint32_t red[SCAN_THREADS / 32];
    __shared__ uint32_t off_s;
    uint32_t part = 0, all = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        uint32_t v = bsum[b];
        if (b < (int)blockIdx.x) part += v;
        all += v;
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[w] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < SCAN_THREADS / 32; ++k) t += red[k];
        off_s = t;
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        for (int o = 16; o > 0; o >>= 1) all += __shfl_xor_sync(0xffffffffu, all, o);
        __syncthreads();
        if (lane == 0) red[w] = all;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int k = 0; k < SCAN_THREADS / 32; ++k) t += red[k];
            sc->nsrt = (int)t;
            sc->builds += 1;
            // the cadence counts steps from this build, whoever asked for it
            // (the step's own decision, or a host request)
            sc->since_full = 0;
        }
    }
    uint32_t off = off_s;
    unsigned base = blockIdx.x * SCAN_CELLS + threadIdx.x * SCAN_ITEMS;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        unsigned k = base + j;
        if (k < ncells) {
            uint2 v = cellSE[k];
            uint32_t s0 = off + v.x;
            cellSE[k] = make_uint2(s0, s0 + v.y);
        }
    }
}

// Provisional slot of every live particle inside its cell's range; the
// counters return to zero.
__global__ void k_scatter(const uint32_t *__restrict__ knew, uint32_t *__restrict__ count,
                          const uint2 *__restrict__ cellSE, uint32_t *__restrict__ tmp,
                          const Scalars *__restrict__ sc, uint32_t sentinel, int gate) {
    if (gate_skips(gate, sc)) return;
    int n = sc->n;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = knew[i];
    if (k == sentinel) return;
    uint32_t slot = atomicSub(&count[k], 1u) - 1u;
    tmp[cellSE[k].x + slot] = (uint32_t)i;
}

template <class T>
void launch_cell_sort(const Grid &g, const State<T> &raw, Scalars *sc, CellSort &cs, int cap,
                      cudaStream_t s, int gate) {
    int blocks = (cap + 255) / 256;
    launch_k(k_hash_count<T>, blocks, 256, s, g, raw, (const Scalars *)sc, cs.knew, cs.count,
             gate);
    launch_k(k_scan_local, cs.nscan, SCAN_THREADS, s, (const uint32_t *)cs.count, cs.cellSE,
             cs.bsum, g.ncells, (const Scalars *)sc, gate);
    launch_k(k_scan_add, cs.nscan, SCAN_THREADS, s, cs.cellSE, (const uint32_t *)cs.bsum,
             g.ncells, cs.nscan, sc, gate);
    launch_k(k_scatter, blocks, 256, s, (const uint32_t *)cs.knew, cs.count,
             (const uint2 *)cs.cellSE, cs.tmp, (const Scalars *)sc, g.sentinel, gate);
}

// ---------------------------------------------------------------------------
// neighbour pair export
// ---------------------------------------------------------------------------
constexpr int PAIR_LANES = 4;

template <class T>
__global__ void __launch_bounds__(SWEEP_BLOCK)
k_pairs(PhysT<T> P, Grid g, Scalars *__restrict__ sc, const uint2 *__restrict__ cellSE,
        const uint32_t *__restrict__ key, Hot<T> hot, const uint32_t *__restrict__ ids,
        unsigned *out_a, unsigned *out_b, unsigned long long cap) {
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / PAIR_LANES, sub = gt % PAIR_LANES;
    if (i >= (unsigned)sc->nsrt) return;
    typename Vec<T>::v4 ha = hot.H0[i];
    unsigned ida = ids[i];
    for_neighbours<PAIR_LANES, T>(
        P, g, cellSE, hot.H0, hot.pos, i, sub, key[i], ha.x, ha.y, P.H2lo, P.H2hi, P.H2d,
        [&](unsigned b, T, T, T, const typename Vec<T>::v4 &) {
            unsigned long long slot = atomicAdd(&sc->pair_count, 1ull);
            if (slot < cap) {
                out_a[slot] = ida;
                out_b[slot] = ids[b];
            }
        });
}

template <class T>
cudaError_t launch_pairs(const PhysT<T> &P, const Grid &g, Scalars *sc, const uint2 *cellSE,
                         const uint32_t *key, const Hot<T> &hot, const uint32_t *ids,
                         unsigned *out_a, unsigned *out_b, unsigned long long cap, int ncap,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&sc->pair_count, 0, sizeof(sc->pair_count), s);
    if (e != cudaSuccess) return e;
    int blocks = (int)(((long long)ncap * PAIR_LANES + SWEEP_BLOCK - 1) / SWEEP_BLOCK);
    k_pairs<T><<<blocks, SWEEP_BLOCK, 0, s>>>(P, g, sc, cellSE, key, hot, ids, out_a, out_b, cap);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// breakup: union-find over links shorter than 1.5 h (Sec. 3-2)
// ---------------------------------------------------------------------------
constexpr int UF_MAX_ITERS = 1 << 22;

__device__ __forceinline__ uint32_t uf_find(uint32_t *parent, uint32_t x, unsigned *err) {
    for (int it = 0; it < UF_MAX_ITERS; ++it) {
        uint32_t px = __ldcg(&parent[x]);
        if (px == x) return x;
        uint32_t ppx = __ldcg(&parent[px]);
        if (ppx != px) atomicMin(&parent[x], ppx);   // path halving (parents only decrease)
        x = px;
    }
    atomicOr(err, ERR_TIMEOUT);
    return x;
}

__device__ __forceinline__ void uf_union(uint32_t *parent, uint32_t a, uint32_t b,
                                         unsigned *err) {
    for (int it = 0; it < UF_MAX_ITERS; ++it) {
        uint32_t ra = uf_find(parent, a, err), rb = uf_find(parent, b, err);
        if (ra == rb) return;
        if (ra < rb) { uint32_t t = ra; ra = rb; rb = t; }
        // hook the larger root under the smaller one: roots end up minimal
        uint32_t old = atomicCAS(&parent[ra], ra, rb);
        if (old == ra) return;
        a = old;
        b = rb;
    }
    atomicOr(err, ERR_TIMEOUT);
}

__global__ void k_uf_init(const Scalars *__restrict__ sc, uint32_t *parent) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < sc->nsrt) parent[i] = (uint32_t)i;
}

template <class T>
__global__ void k_uf_link(PhysT<T> P, Grid g, Scalars *__restrict__ sc,
                          const uint2 *__restrict__ cellSE, const uint32_t *__restrict__ key,
                          Hot<T> hot, uint32_t *parent) {
    unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (unsigned)sc->nsrt) return;
    typename Vec<T>::v4 ha = hot.H0[i];
    for_neighbours<1, T>(P, g, cellSE, hot.H0, hot.pos, i, 0u, key[i], ha.x, ha.y, P.R15lo,
                         P.R15hi, P.R15d, [&](unsigned b, T, T, T, const typename Vec<T>::v4 &) {
                             if (b < i) uf_union(parent, i, b, &sc->err);
                         });
}

__global__ void k_uf_compress(Scalars *__restrict__ sc, uint32_t *parent,
                              const uint8_t *__restrict__ type, uint8_t *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc->nsrt) return;
    uint32_t r = uf_find(parent, (uint32_t)i, &sc->err);
    if (type[i] == T_BUFFER) flag[r] = 1;
}

__device__ __forceinline__ unsigned long long ordered_bits(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <class T>
__global__ void k_uf_reach(Scalars *__restrict__ sc, uint32_t *parent, const double2 *pos,
                           const uint8_t *__restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc->nsrt) return;
    uint32_t r = uf_find(parent, (uint32_t)i, &sc->err);
    if (flag[r])
        atomicMax(&sc->xmax_key, ordered_bits(pos[i].x));
    else
        atomicAdd(&sc->detached, 1u);
}

template <class T>
void launch_breakup(const PhysT<T> &P, const Grid &g, Scalars *sc, const uint2 *cellSE,
                    const uint32_t *key, const Hot<T> &hot, const uint8_t *type,
                    uint32_t *parent, uint8_t *flag, int cap, cudaStream_t s) {
    int blocks = (cap + 255) / 256;
    cudaMemsetAsync(flag, 0, (size_t)cap, s);
    cudaMemsetAsync(&sc->xmax_key, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(&sc->detached, 0, sizeof(unsigned), s);
    k_uf_init<<<blocks, 256, 0, s>>>(sc, parent);
    k_uf_link<T><<<(cap + 127) / 128, 128, 0, s>>>(P, g, sc, cellSE, key, hot, parent);
    k_uf_compress<<<blocks, 256, 0, s>>>(sc, parent, type, flag);
    k_uf_reach<T><<<blocks, 256, 0, s>>>(sc, parent, hot.pos, flag);
}

template void launch_cell_sort<float>(const Grid &, const State<float> &, Scalars *, CellSort &,
                                       int, cudaStream_t, int);
template void launch_cell_sort<double>(const Grid &, const State<double> &, Scalars *,
                                        CellSort &, int, cudaStream_t, int);
template cudaError_t launch_pairs<float>(const PhysT<float> &, const Grid &, Scalars *,
                                         const uint2 *, const uint32_t *, const Hot<float> &,
                                         const uint32_t *, unsigned *, unsigned *,
                                         unsigned long long, int, cudaStream_t);
template cudaError_t launch_pairs<double>(const PhysT<double> &, const Grid &, Scalars *,
                                          const uint2 *, const uint32_t *, const Hot<double> &,
                                          const uint32_t *, unsigned *, unsigned *,
                                          unsigned long long, int, cudaStream_t);
template void launch_breakup<float>(const PhysT<float> &, const Grid &, Scalars *,
                                    const uint2 *, const uint32_t *, const Hot<float> &,
                                    const uint8_t *, uint32_t *, uint8_t *, int, cudaStream_t);
template void launch_breakup<double>(const PhysT<double> &, const Grid &, Scalars *,
                                     const uint2 *, const uint32_t *, const Hot<double> &,
                                     const uint8_t *, uint32_t *, uint8_t *, int,
                                     cudaStream_t);

}  // namespace sph
