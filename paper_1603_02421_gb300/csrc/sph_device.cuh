// Device helpers shared by the libsph kernels: kernel functions (Sec. 2-5),
// Tait EOS (Eq. 26) and the cell-list neighbour walk (Sec. 2-7).
#pragma once

#include "sph_internal.cuh"

namespace sph {

__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float log1p_t(float x) { return log1pf(x); }
__device__ __forceinline__ double log1p_t(double x) { return log1p(x); }
__device__ __forceinline__ float expm1_t(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_t(double x) { return expm1(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return cospi(x); }
__device__ __forceinline__ float abs_t(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_t(double x) { return fabs(x); }

// Eq. 27 (K = 0, cubic spline) / Eq. 28 (K = 1, Wendland C2): W(q) with the
// 2D normalisation kappa / h^2 folded into P.wn.  Callers pass q < 2 (up to
// rounding; t is clamped at 0).
template <class T, int K> __device__ __forceinline__ T kernel_W(const PhysT<T> &P, T q) {
    T t = T(2) - q;
    t = t > T(0) ? t : T(0);
    if (K == 1) {
        T t2 = t * t;
        return P.wn * (T(1) + T(2) * q) * (t2 * t2);
    }
    if (q <= T(1)) return P.wn * (T(1) + q * q * (T(-1.5) + T(0.75) * q));
    return P.wn * T(0.25) * t * t * t;
}

// (1/r) dW/dr, finite at r = 0; grad_a W_ab = F * (r_a - r_b).
//   Wendland: -10 kappa/h^4 (2-q)^3
//   cubic:    kappa/h^4 (-3 + 9q/4) for q <= 1, -(3 kappa/4h^4)(2-q)^2 / q above
// inv_q = 1/q (used by the cubic outer branch only).
template <class T, int K> __device__ __forceinline__ T kernel_F(const PhysT<T> &P, T q, T inv_q) {
    T t = T(2) - q;
    t = t > T(0) ? t : T(0);
    if (K == 1) return P.gn * t * t * t;
    if (q <= T(1)) return P.gn * (T(-3) + T(2.25) * q);
    return P.gn * T(-0.75) * t * t * inv_q;
}

// Eq. 26 with rho = rho0 + drho, x = drho / rho0:
//   P = B ((1 + x)^gamma - 1),  c = c0 (1 + x)^((gamma - 1)/2).
// For gamma = 7 the binomial expansion x (7 + 21x + 35x^2 + 35x^3 + 21x^4 +
// 7x^5 + x^6) and c0 (1 + x)^3 are exact and keep full relative precision for
// small x; otherwise B expm1(gamma log1p(x)).
template <class T>
__device__ __forceinline__ void eos(const PhysT<T> &P, T drho, T &rho, T &P_over_rho2, T &c) {
    rho = P.rho0 + drho;
    T x = drho * P.inv_rho0;
    T p;
    if (P.gamma7) {
        T poly = T(7) + x * (T(21) + x * (T(35) + x * (T(35) + x * (T(21) + x * (T(7) + x)))));
        p = P.B * x * poly;
        T s = T(1) + x;
        c = P.c0 * s * s * s;
    } else {
        T lg = log1p_t(x);
        p = P.B * expm1_t(P.gamma * lg);
        c = P.c0 * exp_t(P.half_gm1 * lg);
    }
    P_over_rho2 = p / (rho * rho);
}

// Exact FP64 distance test, written out so that it matches a plain
// (dx*dx + dy*dy < r2max) evaluation without fused multiply-add.
__device__ __forceinline__ bool exact_within(double2 pa, double2 pb, double r2max) {
    double dx = __dsub_rn(pa.x, pb.x);
    double dy = __dsub_rn(pa.y, pb.y);
    double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return d2 < r2max;
}

// Cell coordinates from a key.
__device__ __forceinline__ void key_cell(const Grid &g, uint32_t key, int &cx, int &cy) {
    grid_cell(g, key, cx, cy);
}

// ---------------------------------------------------------------------------
// Cell offsets.  A particle's position enters the pair sweeps as its offset
// from the origin of its cell of the last build.  FP64 records hold that
// offset.  FP32 records hold it in fixed point -- OFF_ONE = 2^29 units per
// cell edge sc, stored as the bits of an int32 in the record's float slot --
// so that the difference of two offsets plus the cell shift between them is
// exact integer arithmetic and the separation is rounded to FP32 once,
// relative to its own length; a float offset would be rounded relative to
// the cell edge, which made the FP32 pair geometry the largest error of the
// surface-tension terms.  Offsets span [-2 sc, 3 sc) (drift between builds
// in the velocity frame), inside int32; differences are taken modulo 2^32
// and are exact because separations stay below one cell edge.
// ---------------------------------------------------------------------------
// The stored offset of a length `off` (from the cell origin).
template <class T> __device__ __forceinline__ T off_make(double off, double sc) {
    return (T)off;
}
template <> __device__ __forceinline__ float off_make<float>(double off, double sc) {
    return __int_as_float(off_fixed(off, sc));
}

// Separation (a - b) + cells * sc of two stored offsets whose cells differ by
// `cells` (cell of a minus cell of b along the axis), in length units.
template <class T>
__device__ __forceinline__ T off_diff(const PhysT<T> &P, T a, T b, int cells) {
    return (a - b) + T(cells) * P.sc;
}
template <>
__device__ __forceinline__ float off_diff<float>(const PhysT<float> &P, float a, float b,
                                                 int cells) {
    unsigned d = (unsigned)__float_as_int(a) - (unsigned)__float_as_int(b) +
                 ((unsigned)cells << OFF_BITS);
    return __int2float_rn((int)d) * P.off_unit;
}

// FP32 separation from a1 = (own offset bits) - 2^29 and a neighbour's stored
// offset b, with shift = (cell code of the list entry) << 29, the code being
// the cell difference + 1: the same exact difference as off_diff.
__device__ __forceinline__ float off_sep_code(const PhysT<float> &P, unsigned a1, float b,
                                              unsigned shift) {
    unsigned d = a1 - (unsigned)__float_as_int(b) + shift;
    return __int2float_rn((int)d) * P.off_unit;
}

// A stored offset moved by the displacement `disp` (length units).
template <class T> __device__ __forceinline__ T off_add(const PhysT<T> &P, T a, T disp) {
    return a + disp;
}
template <>
__device__ __forceinline__ float off_add<float>(const PhysT<float> &P, float a, float disp) {
    return __int_as_float(__float_as_int(a) + __float2int_rn(disp * P.off_scale));
}

// Whether a stored offset lies in [P.cell_lo, P.cell_hi) (stored the same way).
template <class T> __device__ __forceinline__ bool off_in(const PhysT<T> &P, T a) {
    return a >= P.cell_lo && a < P.cell_hi;
}
template <> __device__ __forceinline__ bool off_in<float>(const PhysT<float> &P, float a) {
    int v = __float_as_int(a);
    return v >= __float_as_int(P.cell_lo) && v < __float_as_int(P.cell_hi);
}

// Stored offsets of position p in the cell of key.
template <class T>
__device__ __forceinline__ void cell_offsets(const Grid &g, uint32_t key, double2 p, T &xoff,
                                             T &yoff, double &xo, double &yo) {
    int cx, cy;
    key_cell(g, key, cx, cy);
    xo = p.x - (g.xmin + (double)(cx - 1) * g.sc);
    yo = p.y - (g.ymin + (double)(cy - 1) * g.sc);
    xoff = off_make<T>(xo, g.sc);
    yoff = off_make<T>(yo, g.sc);
}

// Particle range of the three cells (cx-1, cx, cx+1) of one row, centred on
// cell key c.  Cells of a row are contiguous in the sorted order, so the
// range is [lo, hi) with the cell cx-1 part below b1 and the cell cx+1 part
// from b2 on.
struct RowRange {
    unsigned lo, b1, b2, hi;
};

__device__ __forceinline__ RowRange row_range(const uint2 *__restrict__ cellSE, int c) {
    uint2 s0 = __ldg(&cellSE[c - 1]);
    uint2 s1 = __ldg(&cellSE[c]);
    uint2 s2 = __ldg(&cellSE[c + 1]);
    bool e0 = s0.y > s0.x, e1 = s1.y > s1.x, e2 = s2.y > s2.x;
    RowRange r;
    r.lo = e0 ? s0.x : (e1 ? s1.x : (e2 ? s2.x : 0u));
    r.hi = e2 ? s2.y : (e1 ? s1.y : (e0 ? s0.y : 0u));
    r.b1 = e0 ? s0.y : r.lo;
    r.b2 = e2 ? s2.x : r.hi;
    return r;
}

// x-cell difference cx_a - cx_b (+1, 0 or -1) of candidate b of a row range.
__device__ __forceinline__ int row_step(const RowRange &rr, unsigned b) {
    return b < rr.b1 ? 1 : (b < rr.b2 ? 0 : -1);
}


// q = r/h, 1/q and 1/r from the squared distance (r2 > 0 except for
// coincident particles, where q = 0 and 1/q, 1/r are returned as 0).
__device__ __forceinline__ void q_of(float r2, float h, float inv_h, float &q, float &inv_q,
                                     float &ri) {
    ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
    q = r2 * ri * inv_h;
    inv_q = h * ri;
}
__device__ __forceinline__ void q_of(double r2, double h, double inv_h, double &q, double &inv_q,
                                     double &ri) {
    double r = sqrt(r2);
    q = r * inv_h;
    ri = r > 0.0 ? 1.0 / r : 0.0;
    inv_q = h * ri;
}
__device__ __forceinline__ void q_of(float r2, float h, float inv_h, float &q, float &inv_q) {
    float ri;
    q_of(r2, h, inv_h, q, inv_q, ri);
}
__device__ __forceinline__ void q_of(double r2, double h, double inv_h, double &q, double &inv_q) {
    double ri;
    q_of(r2, h, inv_h, q, inv_q, ri);
}
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

// Bounds-check build (SPH_BOUNDS_CHECK): true, with ERR_BOUNDS recorded in
// the context's error word, when particle index k is not below the capacity
// of the particle arrays; the walks then skip the entry.  Without the macro
// the test is the constant false and costs nothing.
template <class T> __device__ __forceinline__ bool index_bad(const PhysT<T> &P, unsigned k) {
#ifdef SPH_BOUNDS_CHECK
    if (k < (unsigned)P.cap) return false;
    if (P.err) atomicOr(P.err, (unsigned)ERR_BOUNDS);
    return true;
#else
    (void)P;
    (void)k;
    return false;
#endif
}

// Visit every particle b != i of the 3x3 cell block of particle i whose FP64
// distance is below the threshold.  Squared distances in T inside [lo, hi)
// are re-tested exactly in FP64 on the stored positions, so the visited set
// is exactly {b : |r_a - r_b|^2 < r2exact} of the FP64 positions.  G threads
// share one particle: thread `sub` takes every G-th candidate of each row, so
// the G threads of a particle load G consecutive records.
// body(b, rx, ry, r2, H0[b]) with (rx, ry) = r_a - r_b.
template <int G, class T, class Body>
__device__ __forceinline__ void for_neighbours(const PhysT<T> &P, const Grid &g,
                                               const uint2 *__restrict__ cellSE,
                                               const typename Vec<T>::v4 *__restrict__ H0,
                                               const double2 *__restrict__ pos, unsigned i,
                                               unsigned sub, uint32_t key, T xa, T ya, T r2lo,
                                               T r2hi, double r2exact, Body &&body) {
    double2 pa = make_double2(0.0, 0.0);
    bool have_pa = false;
#pragma unroll 1
    for (int dy = -1; dy <= 1; ++dy) {
        RowRange rr = row_range(cellSE, (int)key + dy * g.ncx);
#pragma unroll 2
        for (unsigned b = rr.lo + sub; b < rr.hi; b += G) {
            if (index_bad(P, b)) break;
            typename Vec<T>::v4 hb = H0[b];
            T rx = off_diff<T>(P, xa, hb.x, row_step(rr, b));
            T ry = off_diff<T>(P, ya, hb.y, -dy);
            T r2 = rx * rx + ry * ry;
            if (r2 >= r2hi || b == i) continue;
            if (r2 >= r2lo) {
                if (!have_pa) { pa = pos[i]; have_pa = true; }
                if (!exact_within(pa, pos[b], r2exact)) continue;
            }
            body(b, rx, ry, r2, hb);
        }
    }
}

// Cell difference (code - 1) of a list entry's 2-bit cell-offset code.
__device__ __forceinline__ int code_cells(uint32_t code) { return (int)code - 1; }

// Loads CH consecutive list entries with one vector load (the address is a
// multiple of CH entries from a row start, and rows start 384-byte aligned).
template <int CH> __device__ __forceinline__ void load_entries(const uint32_t *p, uint32_t *ent) {
    if constexpr (CH == 4) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        ent[0] = v.x; ent[1] = v.y; ent[2] = v.z; ent[3] = v.w;
    } else if constexpr (CH == 2) {
        uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        ent[0] = v.x; ent[1] = v.y;
    } else {
        ent[0] = __ldg(p);
    }
}

// Walk lane `sub`'s part of the neighbour list of particle i: the G lanes of a
// particle take chunks of CH consecutive entries in turn (lane sub: entries
// [c*G*CH + sub*CH, +CH) of round c).  A chunk is read with one vector load,
// and every gather of the chunk -- gather(b), the sweep's record of b with
// its cell offsets in .x -- is issued before any of them is used, so a lane
// keeps CH independent gathers in flight instead of a chain of index ->
// record loads; the next chunk's entries are loaded while this one is
// processed.  Entries whose squared distance in T is below H2lo are
// taken; those below H2hi are re-tested exactly in FP64 below (2h)^2.  Slots
// past the list end (inside the 96-slot row, so the vector load stays in
// bounds) are masked and gather particle i's own record instead of an index
// they do not hold.  body(b, rx, ry, r2, record) with (rx, ry) = r_a - r_b.
template <int G, int CH, class T, class Gather, class Body>
__device__ __forceinline__ void for_list(const PhysT<T> &P, const NList &nl,
                                         const double2 *__restrict__ pos, unsigned i,
                                         unsigned sub, T xa, T ya, Gather &&gather, Body &&body) {
    static_assert(CH == 1 || CH == 2 || CH == 4, "chunk of 1, 2 or 4 entries");
    static_assert(LIST_SLOTS % CH == 0, "rows hold whole chunks");
    using Rec = decltype(gather(0u));
    unsigned cnt = nl.cnt[i];
    const uint32_t *__restrict__ e = nl.e + (size_t)i * LIST_SLOTS;
    double2 pa = make_double2(0.0, 0.0);
    bool have_pa = false;
    uint32_t ent[CH], nxt[CH];
    // FP32: the own fixed-point offsets less one cell edge, so that an
    // entry's 2-bit cell code (cell difference + 1), moved to the offset's
    // cell bit, completes the exact separation in one three-input add
    static_assert(OFF_BITS == 29, "cell codes are moved to bits 29-30");
    unsigned xa1 = 0u, ya1 = 0u;
    if constexpr (sizeof(T) == 4) {
        xa1 = (unsigned)__float_as_int(xa) - (1u << OFF_BITS);
        ya1 = (unsigned)__float_as_int(ya) - (1u << OFF_BITS);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) nxt[u] = 0u;
    if (sub * CH < cnt) load_entries<CH>(e + sub * CH, ent);
#pragma unroll 1
    for (unsigned base = sub * CH; base < cnt; base += G * CH) {
        // the next chunk's entries load while this chunk is processed
        if (base + G * CH < cnt) load_entries<CH>(e + base + G * CH, nxt);
        Rec rec[CH];
        unsigned bb[CH], skip = 0u;
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            bb[u] = base + u < cnt ? (ent[u] & 0x0FFFFFFFu) : i;
            if (index_bad(P, bb[u])) {
                bb[u] = i;
                skip |= 1u << u;
            }
            rec[u] = gather(bb[u]);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            if (base + u >= cnt || ((skip >> u) & 1u)) continue;
            T rx, ry;
            if constexpr (sizeof(T) == 4) {
                rx = off_sep_code(P, xa1, rec[u].x.x, (ent[u] << 1) & 0x60000000u);
                ry = off_sep_code(P, ya1, rec[u].x.y, (ent[u] >> 1) & 0x60000000u);
            } else {
                rx = off_diff<T>(P, xa, rec[u].x.x, code_cells((ent[u] >> 28) & 3u));
                ry = off_diff<T>(P, ya, rec[u].x.y, code_cells(ent[u] >> 30));
            }
            T r2 = rx * rx + ry * ry;
            if (r2 >= P.H2lo) {   // one compare for the pairs well inside 2h
                if (r2 >= P.H2hi) continue;
                if (!have_pa) { pa = pos[i]; have_pa = true; }
                if (!exact_within(pa, pos[bb[u]], P.H2d)) continue;
            }
            body(bb[u], rx, ry, r2, rec[u]);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) ent[u] = nxt[u];
    }
}

// (double)f, exactly, for a normal or zero float by moving its bits into the
// FP64 layout (exponent rebiased by 1023 - 127, mantissa shifted up by 29)
// on the integer pipes; subnormals, infinities and NaN take the hardware
// conversion.  FP64 conversions run on the FP64 pipe, which on this GPU has a
// small fraction of the FP32 rate.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e - 1u < 254u) {
        const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
}

// p lies in the box [xmin, xmax) x [ymin, ymax) (false for NaN), decided on
// the ordered integer keys of the coordinates.
__device__ __forceinline__ bool in_box(const Grid &g, double2 p) {
    const long long kx = ordered_key(p.x), ky = ordered_key(p.y);
    return kx >= g.kxmin && kx < g.kxmax && ky >= g.kymin && ky < g.kymax;
}

template <int G, class T> __device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G, class T> __device__ __forceinline__ T group_max(T v) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

}  // namespace sph
