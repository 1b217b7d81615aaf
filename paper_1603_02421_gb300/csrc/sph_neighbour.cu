// Cell-linked-list neighbour build (Sec. 2-7) and the breakup-length
// connectivity (Sec. 3-2) of libsph.
//
//  k_hash      FP64 position -> cell key (dead particles -> sentinel key)
//  k_rs_*      stable LSD radix sort of (key, index), 8-bit digits
//  k_cells     [start, end) of every occupied cell, live particle count
//  k_pairs     neighbour pair export (exact FP64 test in the guard band)
//  k_uf_*      union-find over links shorter than 1.5 h, jet reach
#include "sph_device.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// cell hash
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_hash(Grid g, State<T> raw, const Scalars *__restrict__ sc,
                       uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
    int n = sc->n;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = g.sentinel;
    if (raw.type[i] != T_DEAD) {
        double2 p = raw.pos[i];
        int cx = (int)floor((p.x - g.xmin) / g.sc) + 1;
        int cy = (int)floor((p.y - g.ymin) / g.sc) + 1;
        cx = min(max(cx, 1), g.ncx - 2);
        cy = min(max(cy, 1), g.ncy - 2);
        k = (uint32_t)cy * (uint32_t)g.ncx + (uint32_t)cx;
    }
    key[i] = k;
    val[i] = (uint32_t)i;
}

template <class T>
void launch_hash(const Grid &g, const State<T> &raw, Scalars *sc, uint32_t *key, uint32_t *val,
                 int cap, cudaStream_t s) {
    int blocks = (cap + 255) / 256;
    k_hash<T><<<blocks, 256, 0, s>>>(g, raw, sc, key, val);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, one 8-bit digit per pass
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RS_THREADS)
k_rs_hist(const uint32_t *__restrict__ keys, const Scalars *__restrict__ sc, int shift,
          uint32_t *__restrict__ tileHist, int ntiles) {
    __shared__ uint32_t h[RS_BINS];
    for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x) h[d] = 0;
    __syncthreads();
    int n = sc->n;
    int base = blockIdx.x * RS_TILE;
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        int idx = base + k * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x)
        tileHist[d * ntiles + blockIdx.x] = h[d];
}

// Exclusive scan of the digit-major tile histogram (one block).
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ a, int M) {
    __shared__ uint32_t part[1024];
    int t = threadIdx.x;
    int chunk = (M + 1023) / 1024;
    int lo = min(t * chunk, M), hi = min(lo + chunk, M);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the 1024 partial sums
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;
    for (int i = lo; i < hi; ++i) {
        uint32_t x = a[i];
        a[i] = run;
        run += x;
    }
}

// Scatter of one tile.  Warp w owns tile items [w*256, w*256+256) in eight
// rounds of 32; ranks among equal digits follow tile order, so the sort is
// stable.
__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
             uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
             const Scalars *__restrict__ sc, int shift, const uint32_t *__restrict__ tileOff,
             int ntiles) {
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t cnt[NW][RS_BINS];
    __shared__ uint32_t gbase[RS_BINS];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x) {
        gbase[d] = tileOff[d * ntiles + blockIdx.x];
#pragma unroll
        for (int j = 0; j < NW; ++j) cnt[j][d] = 0;
    }
    __syncthreads();
    int n = sc->n;
    int base = blockIdx.x * RS_TILE + w * (RS_ITEMS * 32);
    uint32_t kk[RS_ITEMS], vv[RS_ITEMS], rk[RS_ITEMS];
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        int idx = base + r * 32 + lane;
        bool valid = idx < n;
        uint32_t key = valid ? kin[idx] : 0u;
        uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned pos = __popc(peers & lt);
        uint32_t b = valid ? cnt[w][d] : 0u;
        __syncwarp();
        if (valid && pos == 0) cnt[w][d] = b + __popc(peers);
        __syncwarp();
        kk[r] = key;
        vv[r] = valid ? vin[idx] : 0u;
        rk[r] = valid ? (b + pos) : 0xffffffffu;
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x) {
        uint32_t run = 0;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            uint32_t c = cnt[j][d];
            cnt[j][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        if (rk[r] == 0xffffffffu) continue;
        uint32_t d = (kk[r] >> shift) & 255u;
        uint32_t dst = gbase[d] + cnt[w][d] + rk[r];
        kout[dst] = kk[r];
        vout[dst] = vv[r];
    }
}

int launch_radix_sort(SortBufs &sb, const Grid &g, Scalars *sc, int cap, cudaStream_t s) {
    int passes = (g.keybits + 7) / 8;
    int ntiles = sb.ntiles;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<ntiles, RS_THREADS, 0, s>>>(sb.key[cur], sc, shift, sb.tileHist, ntiles);
        k_rs_scan<<<1, 1024, 0, s>>>(sb.tileHist, RS_BINS * ntiles);
        k_rs_scatter<<<ntiles, RS_THREADS, 0, s>>>(sb.key[cur], sb.val[cur], sb.key[cur ^ 1],
                                                   sb.val[cur ^ 1], sc, shift, sb.tileHist,
                                                   ntiles);
        cur ^= 1;
    }
    (void)cap;
    return cur;
}

// ---------------------------------------------------------------------------
// cell ranges
// ---------------------------------------------------------------------------
__global__ void k_cells(const uint32_t *__restrict__ key, Scalars *__restrict__ sc,
                        uint2 *__restrict__ cellSE, uint32_t sentinel) {
    int n = sc->n;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 0) {
        if (i == 0) sc->nsrt = 0;
        return;
    }
    if (i >= n) return;
    uint32_t k = key[i];
    if (k == sentinel) {
        if (i == 0) sc->nsrt = 0;
        return;
    }
    uint32_t kn = (i + 1 < n) ? key[i + 1] : sentinel;
    if (kn == sentinel) sc->nsrt = i + 1;
    uint32_t kp = i > 0 ? key[i - 1] : 0xffffffffu;
    unsigned *se = reinterpret_cast<unsigned *>(cellSE);
    if (kp != k) se[2 * (size_t)k] = (unsigned)i;
    if (kn != k) se[2 * (size_t)k + 1] = (unsigned)(i + 1);
}

void launch_cells(const Grid &g, const uint32_t *key, Scalars *sc, uint2 *cellSE, int cap,
                  cudaStream_t s) {
    cudaMemsetAsync(cellSE, 0, sizeof(uint2) * (size_t)g.ncells, s);
    int blocks = (cap + 255) / 256;
    k_cells<<<blocks, 256, 0, s>>>(key, sc, cellSE, g.sentinel);
}

// ---------------------------------------------------------------------------
// neighbour pair export
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_pairs(PhysT<T> P, Grid g, Scalars *__restrict__ sc,
                        const uint2 *__restrict__ cellSE, const uint32_t *__restrict__ key,
                        Hot<T> hot, const uint32_t *__restrict__ ids, unsigned *out_a,
                        unsigned *out_b, unsigned cap) {
    unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (unsigned)sc->nsrt) return;
    typename Vec<T>::v4 ha = hot.H0[i];
    unsigned ida = ids[i];
    for_neighbours<T>(P, g, cellSE, hot.H0, hot.pos, i, key[i], ha.x, ha.y, P.H2lo, P.H2hi,
                      P.H2d, [&](unsigned b, T, T, T, const typename Vec<T>::v4 &) {
                          unsigned slot = atomicAdd(&sc->pair_count, 1u);
                          if (slot < cap) {
                              out_a[slot] = ida;
                              out_b[slot] = ids[b];
                          }
                      });
}

template <class T>
void launch_pairs(const PhysT<T> &P, const Grid &g, const Scalars *, Scalars *sc,
                  const uint2 *cellSE, const uint32_t *key, const Hot<T> &hot,
                  const uint32_t *ids, unsigned *out_a, unsigned *out_b, unsigned cap, int ncap,
                  cudaStream_t s) {
    cudaMemsetAsync(&sc->pair_count, 0, sizeof(unsigned), s);
    int blocks = (ncap + 127) / 128;
    k_pairs<T><<<blocks, 128, 0, s>>>(P, g, sc, cellSE, key, hot, ids, out_a, out_b, cap);
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
    for_neighbours<T>(P, g, cellSE, hot.H0, hot.pos, i, key[i], ha.x, ha.y, P.R15lo, P.R15hi,
                      P.R15d, [&](unsigned b, T, T, T, const typename Vec<T>::v4 &) {
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

template void launch_hash<float>(const Grid &, const State<float> &, Scalars *, uint32_t *,
                                 uint32_t *, int, cudaStream_t);
template void launch_hash<double>(const Grid &, const State<double> &, Scalars *, uint32_t *,
                                  uint32_t *, int, cudaStream_t);
template void launch_pairs<float>(const PhysT<float> &, const Grid &, const Scalars *,
                                  Scalars *, const uint2 *, const uint32_t *,
                                  const Hot<float> &, const uint32_t *, unsigned *, unsigned *,
                                  unsigned, int, cudaStream_t);
template void launch_pairs<double>(const PhysT<double> &, const Grid &, const Scalars *,
                                   Scalars *, const uint2 *, const uint32_t *,
                                   const Hot<double> &, const uint32_t *, unsigned *,
                                   unsigned *, unsigned, int, cudaStream_t);
template void launch_breakup<float>(const PhysT<float> &, const Grid &, Scalars *,
                                    const uint2 *, const uint32_t *, const Hot<float> &,
                                    const uint8_t *, uint32_t *, uint8_t *, int, cudaStream_t);
template void launch_breakup<double>(const PhysT<double> &, const Grid &, Scalars *,
                                     const uint2 *, const uint32_t *, const Hot<double> &,
                                     const uint8_t *, uint32_t *, uint8_t *, int,
                                     cudaStream_t);

}  // namespace sph
