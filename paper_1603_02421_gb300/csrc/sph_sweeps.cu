// Pair sweeps and integrator of libsph (Secs. 2-2 to 2-8 of the paper).
//
//  k_reorder   gather raw -> cell order; EOS and hot records of evaluation n
//  k_build     neighbour list of the step from the 3x3 cell block, fused
//              with the colour of evaluation n                       (Eq. 14)
//  k_colour    C_a = sum_b V_b W_ab, self included (evaluation n+1/2) (Eq. 14)
//  k_normal    n_a = sum_b V_b (C_b - C_a) grad W; filter N_a; nhat (Eqs. 18, 20, 21)
//  k_forces    continuity (Eq. 7), momentum with pressure, viscosity,
//              curvature + CSF, gravity, repulsive walls (Eqs. 9, 10, 23-25,
//              29); time-step terms (Eqs. 30-31); fused corrector
//  k_predict   dt (Eq. 32), predictor half step, hot records of evaluation n+1/2
//  k_spawn     inflow layer laying, time advance
//
// G consecutive threads share one particle (G = 1, 2, 4 or 8, chosen at run
// time): in the list build each takes every G-th candidate of the 3x3 cell
// block and the finds are compacted with a G-lane ballot; later sweeps split
// each particle's list G ways; partial sums are combined with warp shuffles.  Consecutive particles are spatially
// adjacent, so their neighbours' records are served from L1.
#include <algorithm>
#include <type_traits>

#include "sph_device.cuh"

namespace sph {

// List entries a lane takes per chunk in each pair sweep (1, 2 or 4).
#ifndef SPH_CH_COLOUR
#define SPH_CH_COLOUR 4
#endif
#ifndef SPH_CH_NORMAL
#define SPH_CH_NORMAL 4
#endif
#ifndef SPH_CH_FORCES
#define SPH_CH_FORCES 1
#endif

// List entries per chunk of the full list walk (colour + state-only forces);
// two, with the register budget of 8 blocks per SM (1M-particle jet, same
// box: 95.5 -> 93.9 us per sweep at 2 lanes, 135 -> 101 us at 1 lane).
#ifndef SPH_CH_PAIRSUM
#define SPH_CH_PAIRSUM 2
#endif

// Blocks per SM the pair sweeps are compiled for (register budget).
#ifndef SPH_SWEEP_MINB
#define SPH_SWEEP_MINB 10
#endif
#ifndef SPH_PAIRSUM_MINB
#define SPH_PAIRSUM_MINB 9
#endif
// k_surface (mostly streaming: one lane per particle, walks only where N_a = 1)
#ifndef SPH_SURFACE_MINB
#define SPH_SURFACE_MINB 10
#endif


template <class T> using V2 = typename Vec<T>::v2;
template <class T> using V4 = typename Vec<T>::v4;

// Neighbour records the pair sweeps gather ahead of use.  .x holds the cell
// offsets (x, y).
template <class T> struct ColourRec {     // offsets and volume
    V4<T> x;
};
template <class T> struct NormalRec {     // offsets, volume, colour
    V4<T> x;
};
template <class T> struct ForceRec {      // offsets and velocity; volume, density,
    V4<T> x;                              // pressure term, sound speed; unit normal
    V4<T> h1;                             // (zero unless particle a has one)
    V2<T> nb;
};

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

template <class T> __device__ __forceinline__ V4<T> mk4(T a, T b, T c, T d) {
    V4<T> r;
    r.x = a; r.y = b; r.z = c; r.w = d;
    return r;
}

__device__ __forceinline__ double inflow_u(const Inflow &f, double t) {
    return f.U * (1.0 + f.amp * sin(f.k * f.U * t + f.phase));
}

template <class T>
__device__ __forceinline__ V4<T> hot1(const PhysT<T> &P, T drho, T mass) {
    T rho, pr2, c;
    eos(P, drho, rho, pr2, c);
    return mk4<T>(mass / rho, rho, pr2, c);
}

// ---------------------------------------------------------------------------
// Fixes each particle's place inside its cell by its id (ids are unique), so
// the cell order depends only on the positions and ids -- not on where the
// particles stood in raw -- which makes a rebuild from a restored checkpoint
// reproduce the running context's order exactly.  Gathers raw -> cell order
// and writes the records of evaluation n.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_reorder(PhysT<T> P, Grid g, const Scalars *__restrict__ sc, CellSort cs,
                          State<T> raw, State<T> srt, Hot<T> hot, int gate) {
    if (gate_skips(gate, sc)) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= sc->nsrt) return;
    uint32_t j = cs.tmp[t];
    uint32_t k = cs.knew[j];
    uint2 se = cs.cellSE[k];
    const uint32_t idj = raw.id[j];
    uint32_t rank = 0;
    for (uint32_t u = se.x; u < se.y; ++u) rank += raw.id[cs.tmp[u]] < idj ? 1u : 0u;
    uint32_t i = se.x + rank;
    cs.key[i] = k;
    double2 p = raw.pos[j];
    V2<T> v = raw.vel[j];
    T dr = raw.drho[j];
    T m = raw.mass[j];
    srt.pos[i] = p;
    srt.vel[i] = v;
    srt.drho[i] = dr;
    srt.drc[i] = raw.drc[j];
    srt.mass[i] = m;
    srt.type[i] = raw.type[j];
    srt.id[i] = raw.id[j];
    srt.disp[i] = mk2(T(0), T(0));
    T xl, yo;
    double xo, yoo;
    cell_offsets<T>(g, k, p, xl, yo, xo, yoo);
    hot.H0[i] = mk4<T>(xl, yo, v.x, v.y);
    hot.H1[i] = hot1<T>(P, dr, m);
}

// ---------------------------------------------------------------------------
// Step without a cell build: the particles keep their order and cells; the
// records of evaluation n are recomputed from the integrated state.  Particles
// deleted since the build keep their slot with zero volume and mass, so they
// drop out of every sum.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_refresh(PhysT<T> P, Grid g, Scalars *__restrict__ sc,
                          const uint32_t *__restrict__ key, State<T> raw, State<T> srt,
                          Hot<T> hot, int gate) {
    if (gate_skips(gate, sc)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc->nsrt) return;
    double2 p = raw.pos[i];
    V2<T> v = raw.vel[i];
    T dr = raw.drho[i];
    T m = raw.mass[i];
    uint8_t typ = raw.type[i];
    V2<T> ds = raw.disp[i];
    srt.pos[i] = p;
    srt.vel[i] = v;
    srt.drho[i] = dr;
    srt.drc[i] = raw.drc[i];
    srt.mass[i] = m;
    srt.type[i] = typ;
    srt.id[i] = raw.id[i];
    srt.disp[i] = ds;
    T xl, yo;
    double xo, yoo;
    cell_offsets<T>(g, key[i], p, xl, yo, xo, yoo);
    hot.H0[i] = mk4<T>(xl, yo, v.x, v.y);
    if (typ == T_DEAD) {
        hot.H1[i] = mk4<T>(T(0), P.rho0, T(0), P.c0);
        return;
    }
    hot.H1[i] = hot1<T>(P, dr, m);
    // the lists and cell walks of the last build stay exact while no particle
    // has moved more than skin/2 (relative to the frame of P.dfx, P.dfy) and
    // its offset from the build-time cell stays within bounds
    if (!(off_in<T>(P, xl) && off_in<T>(P, yo)) ||
        !(ds.x * ds.x + ds.y * ds.y <= P.half_skin * P.half_skin))
        atomicOr(&sc->err, ERR_SKIN);
}

template <class T>
void launch_refresh(const PhysT<T> &P, const Grid &g, Scalars *sc, const uint32_t *key,
                    const State<T> &raw, const State<T> &srt, const Hot<T> &hot, int cap,
                    cudaStream_t s, int gate) {
    launch_k(k_refresh<T>, (cap + 255) / 256, 256, s, P, g, sc, key, raw, srt, hot, gate);
}

template <class T>
void launch_reorder(const PhysT<T> &P, const Grid &g, Scalars *sc, const CellSort &cs,
                    const State<T> &raw, const State<T> &srt, const Hot<T> &hot, int cap,
                    cudaStream_t s, int gate) {
    launch_k(k_reorder<T>, (cap + 255) / 256, 256, s, P, g, (const Scalars *)sc, cs, raw, srt,
             hot, gate);
}

// ---------------------------------------------------------------------------
// Neighbour list (Sec. 2-7) + colour of evaluation n (Eq. 14)
// ---------------------------------------------------------------------------
template <class T, int K, bool COLOUR, int G>
__global__ void __launch_bounds__(SWEEP_BLOCK, SPH_SWEEP_MINB)
k_build(PhysT<T> P, Grid g, Scalars *__restrict__ sc, const uint2 *__restrict__ cellSE,
        const uint32_t *__restrict__ key, Hot<T> hot, NList nl, Csf<T> csf, int gate) {
    if (gate_skips(gate, sc)) return;
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / G, sub = gt % G;
    unsigned lane = threadIdx.x & 31u;
    unsigned gbase = lane & ~(unsigned)(G - 1);
    unsigned gmask = ((1u << G) - 1u) << gbase;
    bool active = i < (unsigned)sc->nsrt;
    const V4<T> *__restrict__ H0 = hot.H0;
    const V4<T> *__restrict__ H1 = hot.H1;
    T sum = T(0);
    V4<T> ha = mk4<T>(T(0), T(0), T(0), T(0));
    if (active) {
        ha = H0[i];
        T xa = ha.x, ya = ha.y;
        const int ka = (int)key[i];
        unsigned cnt = 0;
        uint32_t *__restrict__ e = nl.e + (size_t)i * LIST_SLOTS;
        double2 pa = make_double2(0.0, 0.0);
        bool have_pa = false;
#pragma unroll 1
        for (int dy = -1; dy <= 1; ++dy) {
            RowRange rr = row_range(cellSE, ka + dy * g.ncx);
            // the lanes of a particle run the same number of iterations, so
            // they can compact their finds with a group ballot
            unsigned nit = rr.hi > rr.lo ? (rr.hi - rr.lo + G - 1) / G : 0u;
            for (unsigned it = 0; it < nit; ++it) {
                unsigned b = rr.lo + it * G + sub;
                bool keep = false;
                uint32_t ent = 0;
                if (b < rr.hi) {
                    V4<T> hb = H0[b];
                    // cell differences c_a - c_b along x and y
                    int sx = row_step(rr, b);
                    int sy = -dy;
                    T rx = off_diff<T>(P, xa, hb.x, sx);
                    T ry = off_diff<T>(P, ya, hb.y, sy);
                    T r2 = rx * rx + ry * ry;
                    if (r2 < P.RL2hi && b != i) {
                        keep = true;
                        ent = b | ((uint32_t)(sx + 1) << 28) | ((uint32_t)(sy + 1) << 30);
                        if (COLOUR && r2 < P.H2hi) {
                            bool in = true;
                            if (r2 >= P.H2lo) {
                                if (!have_pa) { pa = hot.pos[i]; have_pa = true; }
                                in = exact_within(pa, hot.pos[b], P.H2d);
                            }
                            if (in) {
                                T q, iq;
                                q_of(r2, P.h, P.inv_h, q, iq);
                                sum += H1[b].x * kernel_W<T, K>(P, q);
                            }
                        }
                    }
                }
                unsigned m = __ballot_sync(gmask, keep) & gmask;
                unsigned slot = cnt + __popc(m & ((1u << lane) - 1u));
                if (keep && slot < LIST_SLOTS) e[slot] = ent;
                cnt += __popc(m);
            }
        }
        if (sub == 0) {
            if (cnt > LIST_SLOTS) atomicOr(&sc->err, ERR_NLIST);
            nl.cnt[i] = cnt < LIST_SLOTS ? cnt : LIST_SLOTS;
        }
    }
    if (COLOUR) {
        sum = group_sum<G>(sum);
        if (active && sub == 0) {
            T Va = H1[i].x;
            T C = sum + Va * P.W0;
            csf.C[i] = C;
            csf.CX[i] = mk4<T>(ha.x, ha.y, Va, C);
        }
    }
}

// ---------------------------------------------------------------------------
// Eq. 6: summation density of the fluid particles (over the list), in place of
// the integrated Eq. 7.  Rewrites the particle's record H1 = (V, rho, P/rho^2,
// c) and, when drho_out is given, stores rho - rho0.  Neighbour masses come
// from the mass array (zero for particles deleted since the build), so no
// record that this kernel rewrites is read.
// ---------------------------------------------------------------------------
template <class T> struct DensityRec {    // offsets and mass
    V4<T> x;
};

template <class T, int K, int G>
__global__ void __launch_bounds__(SWEEP_BLOCK, SPH_SWEEP_MINB)
k_density(PhysT<T> P, const Scalars *__restrict__ sc, NList nl, Hot<T> hot,
          const T *__restrict__ mass, const uint8_t *__restrict__ type, T *__restrict__ drho_out,
          int gate) {
    if (gate_skips(gate, sc)) return;
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / G, sub = gt % G;
    bool fluid = i < (unsigned)sc->nsrt && type[i] == T_FLUID;
    const V4<T> *__restrict__ H0 = hot.H0;
    T sum = T(0);
    if (fluid) {
        V4<T> ha = H0[i];
        for_list<G, SPH_CH_COLOUR, T>(
            P, nl, hot.pos, i, sub, ha.x, ha.y,
            [&](unsigned b) {
                DensityRec<T> r;
                V4<T> h0 = H0[b];
                r.x = mk4<T>(h0.x, h0.y, type[b] == T_DEAD ? T(0) : mass[b], T(0));
                return r;
            },
            [&](unsigned, T, T, T r2, const DensityRec<T> &r) {
                T q, iq;
                q_of(r2, P.h, P.inv_h, q, iq);
                sum += r.x.z * kernel_W<T, K>(P, q);
            });
    }
    sum = group_sum<G>(sum);
    if (fluid && sub == 0) {
        T m = mass[i];
        T dr = (sum + m * P.W0) - P.rho0;
        hot.H1[i] = hot1<T>(P, dr, m);
        if (drho_out) drho_out[i] = dr;
    }
}

// ---------------------------------------------------------------------------
// Eq. 14: colour at the half step (over the list)
// ---------------------------------------------------------------------------
template <class T, int K, int G>
__global__ void __launch_bounds__(SWEEP_BLOCK, SPH_SWEEP_MINB)
k_colour(PhysT<T> P, const Scalars *__restrict__ sc, NList nl, Hot<T> hot, Csf<T> csf,
         int gate) {
    if (gate_skips(gate, sc)) return;
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / G, sub = gt % G;
    bool active = i < (unsigned)sc->nsrt;
    const V4<T> *__restrict__ H0 = hot.H0;
    const V4<T> *__restrict__ H1 = hot.H1;
    T sum = T(0);
    V4<T> ha = mk4<T>(T(0), T(0), T(0), T(0));
    if (active) {
        ha = H0[i];
        for_list<G, SPH_CH_COLOUR, T>(
            P, nl, hot.pos, i, sub, ha.x, ha.y,
            [&](unsigned b) {
                ColourRec<T> r;
                V4<T> h0 = H0[b];
                r.x = mk4<T>(h0.x, h0.y, H1[b].x, T(0));
                return r;
            },
            [&](unsigned, T, T, T r2, const ColourRec<T> &r) {
                T q, iq;
                q_of(r2, P.h, P.inv_h, q, iq);
                sum += r.x.z * kernel_W<T, K>(P, q);
            });
    }
    sum = group_sum<G>(sum);
    if (active && sub == 0) {
        T Va = H1[i].x;
        T C = sum + Va * P.W0;
        csf.C[i] = C;
        csf.CX[i] = mk4<T>(ha.x, ha.y, Va, C);
    }
}

// ---------------------------------------------------------------------------
// Eqs. 18, 20, 21: normal, filter, unit normal.  With SKIP (the steps), a
// particle whose normal provably stays below the filter threshold is not
// walked: |n_a| <= sum_b V_b |C_b - C_a| |grad_a W_ab| <= D_a G_a, with G_a =
// sum_b V_b |grad_a W_ab| from k_pairsum and D_a the largest |C_b - C_a| over
// the colour ranges of the 3x3 cells of the last build around a (every list
// neighbour of a lies in them).  When D_a G_a is at most half the threshold,
// N_a = 0 and nhat_a = 0 exactly as the walk would give; n_a (used only
// where N_a = 1) is then written as zero.  Without SKIP (sph_evaluate) every
// particle is walked and n_a is exact everywhere.
// ---------------------------------------------------------------------------
template <class T, int K, int G, bool SKIP>
__global__ void __launch_bounds__(SWEEP_BLOCK, SPH_SWEEP_MINB)
k_normal(PhysT<T> P, const Scalars *__restrict__ sc, NList nl, Hot<T> hot, Csf<T> csf,
         const uint32_t *__restrict__ key, const T *__restrict__ gsum,
         const uint2 *__restrict__ crange, int ncx) {
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / G, sub = gt % G;
    bool active = i < (unsigned)sc->nsrt;
    const V4<T> *__restrict__ CX = csf.CX;
    T nx = T(0), ny = T(0);
    if (active) {
        V4<T> xa = CX[i];
        T Ca = xa.w;
        bool walk = true;
        if (SKIP) {
            const int k = (int)key[i];
            float lo = 3.0e38f, hi = 0.0f;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    uint2 r = __ldg(&crange[k + dy * ncx + dx]);
                    lo = fminf(lo, __uint_as_float(r.x));
                    hi = fmaxf(hi, __uint_as_float(~r.y));
                }
            }
            T D = (T)hi - Ca;
            D = Ca - (T)lo > D ? Ca - (T)lo : D;
            walk = !(D * gsum[i] <= T(0.5) * P.eps_n);
        }
        if (walk)
            for_list<G, SPH_CH_NORMAL, T>(
                P, nl, hot.pos, i, sub, xa.x, xa.y,
                [&](unsigned b) {
                    NormalRec<T> r;
                    r.x = CX[b];
                    return r;
                },
                [&](unsigned, T rx, T ry, T r2, const NormalRec<T> &r) {
                    T q, iq;
                    q_of(r2, P.h, P.inv_h, q, iq);
                    T wgt = r.x.z * (r.x.w - Ca) * kernel_F<T, K>(P, q, iq);
                    nx += wgt * rx;
                    ny += wgt * ry;
                });
    }
    nx = group_sum<G>(nx);
    ny = group_sum<G>(ny);
    if (active && sub == 0) {
        T mag = sqrt_t(nx * nx + ny * ny);
        V2<T> nh = mk2(T(0), T(0));
        if (mag > P.eps_n) nh = mk2(nx / mag, ny / mag);
        csf.nhat[i] = nh;
        csf.nvec[i] = mk2(nx, ny);
    }
}

// ---------------------------------------------------------------------------
// Eq. 29: repulsive wall force per unit mass from the boundary particles in
// the 3x3 cell block (R(psi) P(xi) eps(z, u_perp) along the wall normal).
// ---------------------------------------------------------------------------
template <class T, int G>
__device__ __forceinline__ void wall_forces(const PhysT<T> &P, const Grid &g, const Boundary &bd,
                                            uint32_t key, unsigned sub, T xa, T ya, T ua, T va,
                                            T y_abs, T &ax, T &ay) {
    const V4<T> *__restrict__ BH = (const V4<T> *)bd.bh;
    T ez = T(1);
    if (P.wall_h0 > T(0)) {
        T z = y_abs - P.wall_h0;
        if (z >= T(0)) ez = T(0.02);
        else if (z > -P.wall_h0) ez = abs_t(z * P.inv_wall_h0) + T(0.02);
    }
    for (int dy = -1; dy <= 1; ++dy) {
        RowRange rr = row_range(bd.cellSE, (int)key + dy * g.ncx);
        for (unsigned k = rr.lo + sub; k < rr.hi; k += G) {
            V4<T> bk = BH[k];
            T rx = off_diff<T>(P, xa, bk.x, row_step(rr, k));
            T ry = off_diff<T>(P, ya, bk.y, -dy);
            T psi = rx * bk.z + ry * bk.w;
            T xi = -rx * bk.w + ry * bk.z;
            if (!(psi > T(0) && psi < P.two_h && abs_t(xi) < P.wall_db)) continue;
            T q = psi / P.two_h;
            T R = P.wall_A * (T(1) - q) / sqrt_t(q);
            T Pf = T(0.5) * (T(1) + cospi_t(xi * P.inv_wall_db));
            T up = (ua + P.ufx) * bk.z + (va + P.ufy) * bk.w;
            T eu = T(0);
            if (up < T(0)) {
                eu = abs_t(T(20) * up) * P.c0_inv;
                eu = eu > T(1) ? T(1) : eu;
            }
            T mag = R * Pf * (ez + eu);
            ax += mag * bk.z;
            ay += mag * bk.w;
        }
    }
}

// ---------------------------------------------------------------------------
// Pair terms of the momentum and continuity equations for fluid particle a
// with neighbour b (Eqs. 7, 9, 10) and, when DT (an evaluation whose end
// takes the time step), the Eq. 31 term.
// ---------------------------------------------------------------------------
template <class T, bool DT>
__device__ __forceinline__ void pair_forces(const PhysT<T> &P, T rx, T ry, T r2, T ri, T F,
                                            T ua, T va, T rhoa, T PAa, T ca, const V4<T> &hb,
                                            const V4<T> &h1b, T &ax, T &ay, T &drho, T &vmax) {
    T du = ua - hb.z, dv = va - hb.w;
    T udotr = du * rx + dv * ry;
    T mb = h1b.x * h1b.y;
    drho += mb * udotr * F;                       // Eq. 7
    // Eq. 10 (approaching pairs only), evaluated without a branch
    T cbar = T(0.5) * (ca + h1b.w);
    T rbar = T(0.5) * (rhoa + h1b.y);
    T Pi = -P.alpha_h * cbar * udotr * fast_div(T(1), rbar * (r2 + P.eta2));
    Pi = udotr < T(0) ? Pi : T(0);
    T coef = mb * (PAa + h1b.z + Pi) * F;         // Eq. 9 / 25
    ax -= coef * rx;
    ay -= coef * ry;
    if constexpr (DT) {                           // only the time step uses it
        T cv = abs_t(P.h * udotr) * (ri * ri);    // Eq. 31 (0 if r = 0)
        vmax = cv > vmax ? cv : vmax;
    }
}

// ---------------------------------------------------------------------------
// End of a force evaluation for particle i, once the pair sums of its G
// lanes are combined (ax, ay, drho, vmax; the curvature sums num, den of
// Eq. 23 when the filter N_a is set): CSF acceleration (Eq. 24), gravity
// (Eq. 25), the non-finite check, the time-step candidate (Eqs. 30-31) and,
// by mode, 0: store the derivatives and copy srt -> raw; 1: store them and
// fold the time-step minimum; 2: corrector.  Every thread of the block calls
// it (mode 1 has a block barrier).
// ---------------------------------------------------------------------------
template <class T, int MODE>
__device__ __forceinline__ void forces_finish(const PhysT<T> &P, const Grid &g, const Inflow &inf,
                                              Scalars *__restrict__ sc, const Hot<T> &hot,
                                              const Csf<T> &csf, const State<T> &srt,
                                              const State<T> &raw, V2<T> *__restrict__ acc,
                                              T *__restrict__ drout, V4<T> *__restrict__ nH0,
                                              V4<T> *__restrict__ nH1, unsigned i, unsigned sub,
                                              int nsrt, bool active, uint8_t typ, bool Na,
                                              const V4<T> &h1a, T ax, T ay, T drho, T vmax,
                                              T num, T den) {
    const bool fluid = typ == T_FLUID;
    T dtc = T(3.0e38);   // per-particle time-step candidate (fluid only)
    if (fluid) {
        if (Na) {                                              // Eq. 24
            den += h1a.x * P.W0;
            T kappa = num / den;
            V2<T> na = csf.nvec[i];
            T s = P.sigma / h1a.y * kappa;
            ax -= s * na.x;
            ay -= s * na.y;
        }
        ax += P.gx;
        ay += P.gy;
        if (sub == 0 && !(isfinite(ax) && isfinite(ay) && isfinite(drho)))
            atomicOr(&sc->err, ERR_NONFINITE);
        if (MODE == 1 && sub == 0) {                           // Eqs. 30-31
            T fa = sqrt_t(ax * ax + ay * ay);
            T dtf = fa > T(0) ? sqrt_t(P.h / fa) : T(3.0e38);
            T dtcv = P.h / (h1a.w + vmax);
            dtc = dtf < dtcv ? dtf : dtcv;
        }
    }

    if (MODE == 0 || MODE == 1) {
        if (active && sub == 0) {
            acc[i] = mk2(ax, ay);
            drout[i] = drho;
            if (MODE == 0) {
                if (i == 0) sc->n = nsrt;
                raw.pos[i] = srt.pos[i];
                raw.vel[i] = srt.vel[i];
                raw.drho[i] = srt.drho[i];
                raw.drc[i] = srt.drc[i];
                raw.mass[i] = srt.mass[i];
                raw.type[i] = srt.type[i];
                raw.id[i] = srt.id[i];
                raw.disp[i] = srt.disp[i];
            }
        }
        if (MODE == 1) {
            // block minimum of the time-step candidates, then one atomic
            T v = dtc;
            for (int o = 16; o > 0; o >>= 1) {
                T w = __shfl_xor_sync(0xffffffffu, v, o);
                v = w < v ? w : v;
            }
            __shared__ T wmin[SWEEP_BLOCK / 32];
            if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                T m = wmin[0];
                for (int k = 1; k < SWEEP_BLOCK / 32; ++k) m = wmin[k] < m ? wmin[k] : m;
                if (m < T(3.0e38)) {
                    int slot = blockIdx.x & (RED_SLOTS - 1);
                    if (sizeof(T) == 4)
                        atomicMin(&sc->dtmin_f[slot], __float_as_uint((float)m));
                    else
                        atomicMin(&sc->dtmin_d[slot],
                                  (unsigned long long)__double_as_longlong((double)m));
                }
            }
        }
        return;
    }

    // MODE 2: corrector X^{n+1} = X^n + dt Xdot^{n+1/2}, positions with
    // u* = u^n + dt/2 a^{n+1/2}; buffer particles follow the inflow velocity.
    const double dt = sc->dt, t = sc->t;
    // the step's factors in T: in FP32 lane 0 rounds them and the warp
    // shares them (FP64 runs at a small fraction of the FP32 rate; every
    // lane of the warp is here)
    T th, tdt;
    if constexpr (sizeof(T) == 4) {
        float a = 0.0f, b = 0.0f;
        if ((threadIdx.x & 31u) == 0u) {
            a = (float)(0.5 * dt);
            b = (float)dt;
        }
        th = __shfl_sync(0xffffffffu, a, 0);
        tdt = __shfl_sync(0xffffffffu, b, 0);
    } else {
        th = 0.5 * dt;
        tdt = dt;
    }
    if (!active || sub != 0) return;
    // every load of the particle's state first: the stores below go to
    // arrays the compiler cannot prove distinct from these
    const double2 p0 = srt.pos[i];
    const V2<T> v0 = srt.vel[i];
    const T d0 = srt.drho[i], c0 = srt.drc[i];
    const T mass = srt.mass[i];
    const uint32_t pid = srt.id[i];
    const V4<T> h0n = nH0[i];
    const T rho_half = P.summation ? hot.H1[i].y : T(0);
    V2<T> ds = srt.disp[i];
    double2 p1 = p0;
    V2<T> v1 = v0;
    T d1 = d0, c1 = c0;
    T stx = T(0), sty = T(0);           // this step's displacement (cell offsets)
    T srx = T(0), sry = T(0);           // the same relative to (dfx, dfy) (rebuild decision)
    if (typ == T_DEAD) {
        // deleted since the last cell build: kept as is until it is dropped
    } else if (typ == T_FLUID) {
        T usx = v0.x + th * ax, usy = v0.y + th * ay;
        stx = tdt * (P.ufx + usx);
        sty = tdt * (P.ufy + usy);
        if constexpr (sizeof(T) == 4) {
            // the FP32 step added to the FP64 position (its rounding, ~6e-8
            // of a step's move, is far below the FP32 pair sums'; the cell
            // offsets take the same increment)
            p1 = make_double2(p0.x + f2d_exact(stx), p0.y + f2d_exact(sty));
        } else {
            p1 = make_double2(p0.x + dt * (P.ufx_d + (double)usx), p0.y + dt * (P.ufy_d + (double)usy));
        }
        v1 = mk2(v0.x + tdt * ax, v0.y + tdt * ay);
        if (P.summation) {              // Eq. 6: the density of the half-step evaluation
            d1 = rho_half - P.rho0;
            c1 = T(0);
        } else {
            T y = tdt * drho - c0;      // compensated density update
            T s = d0 + y;
            c1 = (s - d0) - y;
            d1 = s;
        }
        srx = tdt * (P.ufx - P.dfx + usx);
        sry = tdt * (P.ufy - P.dfy + usy);
    } else {
        const double half = 0.5 * dt;
        double uh = inf.on ? inflow_u(inf, t + half) : P.ufx_d + (double)v0.x;
        p1 = make_double2(p0.x + dt * uh, p0.y);
        v1 = inf.on ? mk2((T)(inflow_u(inf, t + dt) - P.ufx_d), (T)(-P.ufy_d)) : v0;
        if (inf.on && p1.x >= inf.x_exit) typ = T_FLUID;
        stx = (T)(dt * uh);
        srx = (T)(dt * (uh - (double)P.dfx));
    }
    ds = mk2(ds.x + srx, ds.y + sry);
    if (typ == T_FLUID && !in_box(g, p1)) {
        typ = T_DEAD;
        atomicAdd((unsigned long long *)&sc->deleted, 1ull);
    }
    raw.pos[i] = p1;
    raw.vel[i] = v1;
    raw.drho[i] = d1;
    raw.drc[i] = c1;
    raw.mass[i] = mass;
    raw.type[i] = typ;
    raw.id[i] = pid;
    raw.disp[i] = ds;
    // the same state in place in the cell order of the last build, with the
    // records of evaluation n+1 on its cells: a next step that keeps the
    // build starts from them (one that rebuilds sorts raw instead).  No
    // thread of this sweep reads another particle's srt entries (neighbours
    // come from the half-step records).
    srt.pos[i] = p1;
    srt.vel[i] = v1;
    srt.drho[i] = d1;
    srt.drc[i] = c1;
    srt.type[i] = typ;
    srt.disp[i] = ds;
    // offsets from the cell: those of evaluation n plus this step's
    // displacement (in T, as the displacement since the build; a few ulps
    // from the offsets of the FP64 position over the steps between builds,
    // far inside the band where pair tests are redone in FP64)
    T xl = off_add<T>(P, h0n.x, stx), yo = off_add<T>(P, h0n.y, sty);
    nH0[i] = mk4<T>(xl, yo, v1.x, v1.y);
    nH1[i] = typ == T_DEAD ? mk4<T>(T(0), P.rho0, T(0), P.c0) : hot1<T>(P, d1, mass);
    // largest displacements (squared, as float bits: monotone for >= 0)
    if (typ != T_DEAD) {
        float d2 = (float)(ds.x * ds.x + ds.y * ds.y);
        float s2 = (float)(srx * srx + sry * sry);
        // the cell walks and FP32 offsets of the build stay exact while every
        // particle's offset from its build-time cell stays within bounds; a
        // particle outside reports twice skin/2, so that the time advance
        // rebuilds before the next step
        if (!(off_in<T>(P, xl) && off_in<T>(P, yo)))
            d2 = fmaxf(d2, 4.0f * (float)(P.half_skin * P.half_skin));
        unsigned m = __activemask();
        unsigned a = __reduce_max_sync(m, __float_as_uint(d2));
        unsigned b2 = __reduce_max_sync(m, __float_as_uint(s2));
        if ((threadIdx.x & 31u) == (unsigned)(__ffs(m) - 1)) {
            int slot = (blockIdx.x * (SWEEP_BLOCK / 32) + (threadIdx.x >> 5)) & (RED_SLOTS - 1);
            atomicMax(&sc->max_disp2[slot], a);
            atomicMax(&sc->max_step2[slot], b2);
        }
    }
}

// ---------------------------------------------------------------------------
// Eqs. 7, 9, 10, 23-25, 29-31 in one list walk (+ corrector in mode 2): the
// form used without surface tension, where no colour, normal or curvature
// precedes the forces.
// ---------------------------------------------------------------------------
template <class T, int K, int MODE, int G>
__global__ void __launch_bounds__(SWEEP_BLOCK, SPH_SWEEP_MINB)
k_forces(PhysT<T> P, Grid g, Inflow inf, Scalars *__restrict__ sc, NList nl,
         const uint32_t *__restrict__ key, Hot<T> hot, Csf<T> csf, Boundary bd, State<T> srt,
         State<T> raw, V2<T> *__restrict__ acc, T *__restrict__ drout, V4<T> *__restrict__ nH0,
         V4<T> *__restrict__ nH1) {
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / G, sub = gt % G;
    int nsrt = sc->nsrt;
    bool active = i < (unsigned)nsrt;
    uint8_t typ = active ? srt.type[i] : T_DEAD;
    bool fluid = typ == T_FLUID;
    T ax = T(0), ay = T(0), drho = T(0), vmax = T(0), num = T(0), den = T(0);
    V4<T> ha = mk4<T>(T(0), T(0), T(0), T(0)), h1a = ha;
    V2<T> nha = mk2(T(0), T(0));
    bool Na = false;
    if (fluid) {
        ha = hot.H0[i];
        h1a = hot.H1[i];
        T rhoa = h1a.y, PAa = h1a.z, ca = h1a.w;
        T ua = ha.z, va = ha.w;
        if (P.csf) {
            nha = csf.nhat[i];
            Na = (nha.x != T(0)) || (nha.y != T(0));
        }
        const V4<T> *__restrict__ H0 = hot.H0;
        const V4<T> *__restrict__ H1 = hot.H1;
        const V2<T> *__restrict__ NH = csf.nhat;
        for_list<G, SPH_CH_FORCES, T>(
            P, nl, hot.pos, i, sub, ha.x, ha.y,
            [&](unsigned b) {
                ForceRec<T> r;
                r.x = H0[b];
                r.h1 = H1[b];
                r.nb = Na ? NH[b] : mk2(T(0), T(0));
                return r;
            },
            [&](unsigned, T rx, T ry, T r2, const ForceRec<T> &r) {
                T q, iq, ri;
                q_of(r2, P.h, P.inv_h, q, iq, ri);
                T F = kernel_F<T, K>(P, q, iq);
                pair_forces<T, MODE == 1>(P, rx, ry, r2, ri, F, ua, va, rhoa, PAa, ca, r.x, r.h1,
                                          ax, ay, drho, vmax);
                if (Na) {                                      // Eq. 23
                    V2<T> nb = r.nb;
                    if (nb.x != T(0) || nb.y != T(0)) {
                        num += r.h1.x * ((nb.x - nha.x) * rx + (nb.y - nha.y) * ry) * F;
                        den += r.h1.x * kernel_W<T, K>(P, q);
                    }
                }
            });
        if (P.walls) {
            double2 pa = hot.pos[i];
            wall_forces<T, G>(P, g, bd, key[i], sub, ha.x, ha.y, ua, va, (T)pa.y, ax, ay);
        }
    }
    ax = group_sum<G>(ax);
    ay = group_sum<G>(ay);
    drho = group_sum<G>(drho);
    num = group_sum<G>(num);
    den = group_sum<G>(den);
    vmax = group_max<G>(vmax);
    forces_finish<T, MODE>(P, g, inf, sc, hot, csf, srt, raw, acc, drout, nH0, nH1, i, sub, nsrt,
                           active, typ, Na, h1a, ax, ay, drho, vmax, num, den);
}

// ---------------------------------------------------------------------------
// With surface tension an evaluation is three sweeps, of which only the
// first walks every particle's list:
//   k_pairsum  colour (Eq. 14) of every particle together with the pair sums
//              of the fluid particles that need only the state -- continuity
//              (Eq. 7), pressure and viscosity (Eqs. 9, 10), the Eq. 31 term,
//              the walls (Eq. 29) -- and, per particle, the bound
//              G_a = sum_b V_b |grad_a W_ab| and the colour range of its cell;
//   k_normal   Eqs. 18, 20, 21; in a step it skips (n_a = 0, N_a = 0) every
//              particle whose normal provably stays below the filter
//              threshold: |n_a| <= max_b |C_b - C_a| G_a, with the colour
//              range taken over the 3x3 cells around it;
//   k_surface  curvature (Eq. 23) for the particles with N_a = 1, then CSF,
//              gravity, time-step candidate and integrator (forces_finish).
// The sums are those of k_forces, term for term and in the same order.
// ---------------------------------------------------------------------------
template <class T> struct PairRec {       // offsets and velocity; volume, density,
    V4<T> x;                              // pressure term, sound speed
    V4<T> h1;
};

// Colour range of a cell: (min C, ~max C) as float bits (C >= 0, so the bit
// patterns order as the values), both reduced with atomicMin from the
// all-ones reset; FP64 colours are rounded outward.
__device__ __forceinline__ void colour_bits(float c, unsigned &lo, unsigned &nhi) {
    lo = __float_as_uint(c);
    nhi = ~__float_as_uint(c);
}
__device__ __forceinline__ void colour_bits(double c, unsigned &lo, unsigned &nhi) {
    lo = __float_as_uint(__double2float_rd(c));
    nhi = ~__float_as_uint(__double2float_ru(c));
}

template <class T, int K, int G, bool DT>
__global__ void __launch_bounds__(SWEEP_BLOCK, SPH_PAIRSUM_MINB)
k_pairsum(PhysT<T> P, Grid g, const Scalars *__restrict__ sc, NList nl,
          const uint32_t *__restrict__ key, Hot<T> hot, Csf<T> csf, Boundary bd,
          const uint8_t *__restrict__ type, V4<T> *__restrict__ accN, T *__restrict__ gsum,
          uint2 *__restrict__ crange) {
    // FP32 Wendland: the kernel's constant factors are taken once per particle
    constexpr bool WSCALED = K == 1 && sizeof(T) == 4;
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / G, sub = gt % G;
    bool active = i < (unsigned)sc->nsrt;
    uint8_t typ = active ? type[i] : T_DEAD;
    bool fluid = typ == T_FLUID;
    T csum = T(0), gs = T(0), ax = T(0), ay = T(0), drho = T(0), vmax = T(0);
    V4<T> ha = mk4<T>(T(0), T(0), T(0), T(0)), h1a = ha;
    if (active) {
        ha = hot.H0[i];
        h1a = hot.H1[i];
        T rhoa = h1a.y, PAa = h1a.z, ca = h1a.w;
        T ua = ha.z, va = ha.w;
        const V4<T> *__restrict__ H0 = hot.H0;
        const V4<T> *__restrict__ H1 = hot.H1;
        for_list<G, SPH_CH_PAIRSUM, T>(
            P, nl, hot.pos, i, sub, ha.x, ha.y,
            [&](unsigned b) {
                PairRec<T> r;
                r.x = H0[b];
                r.h1 = H1[b];
                return r;
            },
            [&](unsigned, T rx, T ry, T r2, const PairRec<T> &r) {
                T q, iq, ri;
                q_of(r2, P.h, P.inv_h, q, iq, ri);
                if constexpr (WSCALED) {
                    // Wendland (Eq. 28) without its constant factors, which
                    // the sums take once below: W / wn = (1 + 2q) t^4 and
                    // F / gn = t^3, t = 2 - q
                    T t = T(2) - q;
                    t = t > T(0) ? t : T(0);
                    T t2 = t * t, t3 = t2 * t;
                    csum += r.h1.x * ((T(1) + T(2) * q) * (t2 * t2));  // Eq. 14
                    gs += r.h1.x * t3 * (r2 * ri);
                    if (fluid)
                        pair_forces<T, DT>(P, rx, ry, r2, ri, t3, ua, va, rhoa, PAa, ca, r.x,
                                           r.h1, ax, ay, drho, vmax);
                } else {
                    T F = kernel_F<T, K>(P, q, iq);
                    csum += r.h1.x * kernel_W<T, K>(P, q);             // Eq. 14
                    gs += r.h1.x * abs_t(F) * (r2 * ri);
                    if (fluid)
                        pair_forces<T, DT>(P, rx, ry, r2, ri, F, ua, va, rhoa, PAa, ca, r.x,
                                           r.h1, ax, ay, drho, vmax);
                }
            });
        if constexpr (WSCALED) {
            csum *= P.wn;
            gs *= -P.gn;          // gn < 0 for the Wendland kernel: |F| = -gn t^3
            ax *= P.gn;
            ay *= P.gn;
            drho *= P.gn;
        }
        if (fluid && P.walls) {
            double2 pa = hot.pos[i];
            wall_forces<T, G>(P, g, bd, key[i], sub, ha.x, ha.y, ua, va, (T)pa.y, ax, ay);
        }
    }
    csum = group_sum<G>(csum);
    gs = group_sum<G>(gs);
    ax = group_sum<G>(ax);
    ay = group_sum<G>(ay);
    drho = group_sum<G>(drho);
    vmax = group_max<G>(vmax);
    T Va = h1a.x;
    T C = csum + Va * P.W0;
    if (active && sub == 0) {
        csf.C[i] = C;
        csf.CX[i] = mk4<T>(ha.x, ha.y, Va, C);
        accN[i] = mk4<T>(ax, ay, drho, vmax);
        gsum[i] = gs;
    }
    // colour range of each cell of the last build, over the particles with
    // a volume (those deleted since the build have none and enter no sum);
    // the lanes of a warp holding the same cell combine first
    bool rep = active && sub == 0 && Va > T(0);
    unsigned m = __ballot_sync(0xffffffffu, rep);
    if (rep) {
        unsigned k = key[i];
        unsigned peers = __match_any_sync(m, k);
        unsigned lo, nhi;
        colour_bits(C, lo, nhi);
        lo = __reduce_min_sync(peers, lo);
        nhi = __reduce_min_sync(peers, nhi);
        if ((threadIdx.x & 31u) == (unsigned)(__ffs(peers) - 1)) {
            atomicMin(&crange[k].x, lo);
            atomicMin(&crange[k].y, nhi);
        }
    }
}

template <class T, int K, int MODE, int G>
__global__ void __launch_bounds__(SWEEP_BLOCK, SPH_SURFACE_MINB)
k_surface(PhysT<T> P, Grid g, Inflow inf, Scalars *__restrict__ sc, NList nl, Hot<T> hot,
          Csf<T> csf, State<T> srt, State<T> raw, const V4<T> *__restrict__ accN,
          V2<T> *__restrict__ acc, T *__restrict__ drout, V4<T> *__restrict__ nH0,
          V4<T> *__restrict__ nH1) {
    unsigned gt = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned i = gt / G, sub = gt % G;
    int nsrt = sc->nsrt;
    bool active = i < (unsigned)nsrt;
    uint8_t typ = active ? srt.type[i] : T_DEAD;
    bool fluid = typ == T_FLUID;
    T num = T(0), den = T(0);
    V4<T> an = mk4<T>(T(0), T(0), T(0), T(0)), h1a = an;
    bool Na = false;
    if (fluid) {
        an = accN[i];
        h1a = hot.H1[i];
        V2<T> nha = csf.nhat[i];
        Na = (nha.x != T(0)) || (nha.y != T(0));
        if (Na) {                                              // Eq. 23
            const V4<T> *__restrict__ H0 = hot.H0;
            const V4<T> *__restrict__ H1 = hot.H1;
            const V2<T> *__restrict__ NH = csf.nhat;
            V4<T> ha = H0[i];
            for_list<G, SPH_CH_FORCES, T>(
                P, nl, hot.pos, i, sub, ha.x, ha.y,
                [&](unsigned b) {
                    ForceRec<T> r;
                    r.x = H0[b];
                    r.h1 = mk4<T>(H1[b].x, T(0), T(0), T(0));
                    r.nb = NH[b];
                    return r;
                },
                [&](unsigned, T rx, T ry, T r2, const ForceRec<T> &r) {
                    V2<T> nb = r.nb;
                    if (nb.x != T(0) || nb.y != T(0)) {
                        T q, iq;
                        q_of(r2, P.h, P.inv_h, q, iq);
                        T F = kernel_F<T, K>(P, q, iq);
                        num += r.h1.x * ((nb.x - nha.x) * rx + (nb.y - nha.y) * ry) * F;
                        den += r.h1.x * kernel_W<T, K>(P, q);
                    }
                });
        }
    }
    num = group_sum<G>(num);
    den = group_sum<G>(den);
    forces_finish<T, MODE>(P, g, inf, sc, hot, csf, srt, raw, acc, drout, nH0, nH1, i, sub, nsrt,
                           active, typ, Na, h1a, an.x, an.y, an.z, an.w, num, den);
}

// ---------------------------------------------------------------------------
// Eq. 32 + predictor: X^{n+1/2} = X^n + dt/2 Xdot^n; hot records at n+1/2
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_predict(PhysT<T> P, Inflow inf, Scalars *__restrict__ sc, State<T> srt,
                          const V4<T> *__restrict__ H0n, const V2<T> *__restrict__ acc,
                          const T *__restrict__ dr, Hot<T> half, int cap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    // the particle's data first (in bounds for any i < cap; used only for
    // i < nsrt), so that these loads overlap the fold of the dt slots
    const int j = i < cap ? i : 0;
    const int nsrt = sc->nsrt;
    const V4<T> h0 = H0n[j];            // offsets and velocity at n
    const T d = srt.drho[j];
    const uint8_t typ = srt.type[j];
    const double2 p = srt.pos[j];
    const V2<T> a = acc[j];
    const T dri = dr[j];
    const T mass = srt.mass[j];
    const V2<T> ds = srt.disp[j];
    // dt, and the half step th in T; every warp folds the 32 minimum slots
    // itself (cached loads), so no warp waits for another at a block barrier
    const int lane = threadIdx.x & 31;
    double dt;
    T th;
    if constexpr (sizeof(T) == 4) {
        // FP32: the slots' minimum in FP32 (exact); the Courant product and
        // the half step's rounding on lane 0 only (FP64 runs at a small
        // fraction of the FP32 rate), broadcast to the warp.  dt_fixed >= 0
        // (checked at init), so its sign test is an integer one.
        double d0 = 0.0;
        float t0 = 0.0f;
        if (__double_as_longlong(P.dt_fixed) > 0) {
            if (lane == 0) d0 = P.dt_fixed;
        } else {
            float mf = __uint_as_float(sc->dtmin_f[lane]);
            for (int o = 16; o > 0; o >>= 1) mf = fminf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
            if (lane == 0) d0 = mf < 1.0e37f ? P.courant * (double)mf : 0.0;
            if (!(mf < 1.0e37f) && i == 0) atomicOr(&sc->err, ERR_NODT);
        }
        if (lane == 0) t0 = (float)(0.5 * d0);
        dt = __shfl_sync(0xffffffffu, d0, 0);
        th = __shfl_sync(0xffffffffu, t0, 0);
    } else {
        if (P.dt_fixed > 0.0) {
            dt = P.dt_fixed;
        } else {
            double m = __longlong_as_double((long long)sc->dtmin_d[lane]);
            for (int o = 16; o > 0; o >>= 1) {
                double w = __shfl_xor_sync(0xffffffffu, m, o);
                m = w < m ? w : m;
            }
            dt = m < 1.0e37 ? P.courant * m : 0.0;
            if (!(m < 1.0e37) && i == 0) atomicOr(&sc->err, ERR_NODT);
        }
        th = 0.5 * dt;
    }
    if (i == 0) sc->dt = dt;
    if (i >= nsrt) return;
    V2<T> v = mk2(h0.z, h0.w);
    // displacement over the half step (absolute velocity = frame + stored)
    T ddx = th * (P.ufx + v.x), ddy = th * (P.ufy + v.y);
    double2 ph;
    if constexpr (sizeof(T) == 4) {
        // the FP32 increment added to the FP64 position (its rounding,
        // ~6e-8 of a half-step move, is far below the FP32 pair sums')
        ph = make_double2(p.x + f2d_exact(ddx), p.y + f2d_exact(ddy));
    } else {
        const double hdt = 0.5 * dt;
        ph = make_double2(p.x + hdt * (P.ufx_d + (double)v.x), p.y + hdt * (P.ufy_d + (double)v.y));
    }
    V2<T> vh = v;
    T dh = d;
    if (typ == T_FLUID) {
        vh = mk2(v.x + th * a.x, v.y + th * a.y);
        dh = d + th * dri;
    } else if (typ == T_BUFFER && inf.on) {
        vh = mk2((T)(inflow_u(inf, sc->t + 0.5 * dt) - P.ufx_d), (T)(-P.ufy_d));
    }
    T xo = off_add<T>(P, h0.x, ddx), yo = off_add<T>(P, h0.y, ddy);
    half.pos[i] = ph;
    half.H0[i] = mk4<T>(xo, yo, vh.x, vh.y);
    if (typ == T_DEAD) {
        half.H1[i] = mk4<T>(T(0), P.rho0, T(0), P.c0);
        return;
    }
    half.H1[i] = hot1<T>(P, dh, mass);
    // the neighbour list stays exact while no particle has moved more than
    // skin/2 since it was built (relative to the frame of P.dfx, P.dfy), and
    // the cell walks and FP32 offsets while every offset from the build-time
    // cell stays within bounds
    T tx = ds.x + th * (P.ufx - P.dfx + v.x), ty = ds.y + th * (P.ufy - P.dfy + v.y);
    if (!(off_in<T>(P, xo) && off_in<T>(P, yo)) ||
        !(tx * tx + ty * ty <= P.half_skin * P.half_skin))
        atomicOr(&sc->err, ERR_SKIN);
}

// ---------------------------------------------------------------------------
// inflow layers + time advance (one block)
// ---------------------------------------------------------------------------
static_assert(RED_SLOTS == 32, "one reduction slot per lane of a warp");

template <class T>
__global__ void k_spawn(Inflow inf, double ufx, double ufy, float half_skin,
                        Scalars *__restrict__ sc, State<T> raw,
                        const double *__restrict__ layer_y, int cap, int cadence) {
    __shared__ int do_spawn, base;
    __shared__ unsigned idbase;
    __shared__ double xnew, unew;
    if (threadIdx.x < 32) {
        // warp 0: each lane folds and resets one reduction slot, lanes 0 and
        // 1 evaluate the two inflow velocities; lane 0 takes the decisions
        const unsigned lane = threadIdx.x;
        // every scalar this kernel reads, loaded at once
        const unsigned d2l = sc->max_disp2[lane], s2l = sc->max_step2[lane];
        const double dt = sc->dt, t = sc->t, x_up = sc->x_up;
        const int nsrt = sc->nsrt, since_full = sc->since_full;
        const unsigned next_id = sc->next_id;
        double half = 0.5 * dt;
        unsigned d2 = __reduce_max_sync(0xffffffffu, d2l);
        unsigned s2 = __reduce_max_sync(0xffffffffu, s2l);
        sc->max_disp2[lane] = 0u;
        sc->max_step2[lane] = 0u;
        sc->dtmin_f[lane] = 0x7f7f7f7fu;
        sc->dtmin_d[lane] = 0x7f7f7f7f7f7f7f7full;
        double uq = (inf.on && lane < 2) ? inflow_u(inf, lane == 0 ? t + half : t + dt) : 0.0;
        double uh = __shfl_sync(0xffffffffu, uq, 0);
        double ue = __shfl_sync(0xffffffffu, uq, 1);
        if (lane == 0) {
            int n = nsrt;
            do_spawn = 0;
            if (inf.on) {
                double xs = __dadd_rn(x_up, __dmul_rn(half, uh));
                double xu = __dsub_rn(__dmul_rn(2.0, xs), x_up);
                sc->x_up = xu;
                if (xu >= inf.threshold) {
                    if (n + inf.ny <= cap) {
                        do_spawn = 1;
                        base = n;
                        idbase = next_id;
                        xnew = __dsub_rn(xu, inf.dx);
                        unew = ue;
                        sc->x_up = xnew;
                        sc->next_id = next_id + (unsigned)inf.ny;
                        n += inf.ny;
                    } else {
                        atomicOr(&sc->err, ERR_CAPACITY);
                    }
                }
            }
            sc->n = n;
            sc->t = __dadd_rn(t, dt);
            sc->step += 1;
            // rebuild next step if particles were appended, the cadence is
            // reached, or one more step (twice this one's largest move) could
            // carry a particle past skin/2 from where the lists were built
            float dmax = sqrtf(__uint_as_float(d2));
            float smax = sqrtf(__uint_as_float(s2));
            sc->last_dmax = dmax;
            sc->last_smax = smax;
            int need = do_spawn || since_full + 1 >= cadence || dmax + 2.0f * smax > half_skin;
            sc->need_full = need;
            sc->since_full = need ? 0 : since_full + 1;
        }
    }
    __syncthreads();
    if (!do_spawn) return;
    for (int j = threadIdx.x; j < inf.ny; j += blockDim.x) {
        int k = base + j;
        raw.pos[k] = make_double2(xnew, layer_y[j]);
        raw.vel[k] = mk2((T)(unew - ufx), (T)(-ufy));
        raw.drho[k] = T(0);
        raw.drc[k] = T(0);
        raw.mass[k] = (T)inf.m_layer;
        raw.type[k] = T_BUFFER;
        raw.id[k] = idbase + (unsigned)j;
        raw.disp[k] = mk2(T(0), T(0));
    }
}

// ---------------------------------------------------------------------------
static int sweep_blocks(int cap, int lanes) {
    return (int)(((long long)cap * lanes + SWEEP_BLOCK - 1) / SWEEP_BLOCK);
}

// Calls f.template operator()<G>() for the run-time lane count.
template <class F> static void with_lanes(int lanes, F &&f) {
    switch (lanes) {
        case 1: f(std::integral_constant<int, 1>()); break;
        case 2: f(std::integral_constant<int, 2>()); break;
        case 8: f(std::integral_constant<int, 8>()); break;
        default: f(std::integral_constant<int, 4>()); break;
    }
}

template <class T>
void launch_build(int lanes, bool with_colour, const PhysT<T> &P, const Grid &g, Scalars *sc,
                  const uint2 *cellSE, const uint32_t *key, const Hot<T> &hot, const NList &nl,
                  const Csf<T> &csf, int cap, cudaStream_t s, int gate) {
    with_lanes(lanes, [&](auto Gc) {
        constexpr int G = decltype(Gc)::value;
        int b = sweep_blocks(cap, G);
        if (P.kernel == 1) {
            if (with_colour) launch_k(k_build<T, 1, true, G>, b, SWEEP_BLOCK, s, P, g, sc, cellSE, key, hot, nl, csf, gate);
            else launch_k(k_build<T, 1, false, G>, b, SWEEP_BLOCK, s, P, g, sc, cellSE, key, hot, nl, csf, gate);
        } else {
            if (with_colour) launch_k(k_build<T, 0, true, G>, b, SWEEP_BLOCK, s, P, g, sc, cellSE, key, hot, nl, csf, gate);
            else launch_k(k_build<T, 0, false, G>, b, SWEEP_BLOCK, s, P, g, sc, cellSE, key, hot, nl, csf, gate);
        }
    });
}

template <class T>
void launch_colour(int lanes, const PhysT<T> &P, const Scalars *sc, const NList &nl,
                   const Hot<T> &hot, const Csf<T> &csf, int cap, cudaStream_t s, int gate) {
    with_lanes(lanes, [&](auto Gc) {
        constexpr int G = decltype(Gc)::value;
        int b = sweep_blocks(cap, G);
        if (P.kernel == 1)
            launch_k(k_colour<T, 1, G>, b, SWEEP_BLOCK, s, P, sc, nl, hot, csf, gate);
        else
            launch_k(k_colour<T, 0, G>, b, SWEEP_BLOCK, s, P, sc, nl, hot, csf, gate);
    });
}

template <class T>
void launch_density(int lanes, const PhysT<T> &P, const Scalars *sc, const NList &nl,
                    const Hot<T> &hot, const T *mass, const uint8_t *type, T *drho_out, int cap,
                    cudaStream_t s, int gate) {
    with_lanes(lanes, [&](auto Gc) {
        constexpr int G = decltype(Gc)::value;
        int b = sweep_blocks(cap, G);
        if (P.kernel == 1)
            launch_k(k_density<T, 1, G>, b, SWEEP_BLOCK, s, P, sc, nl, hot, mass, type, drho_out,
                     gate);
        else
            launch_k(k_density<T, 0, G>, b, SWEEP_BLOCK, s, P, sc, nl, hot, mass, type, drho_out,
                     gate);
    });
}

// In a step (skip) one lane per particle: every lane repeats the particle's
// skip test, and only the particles near the surface walk (1M-particle jet,
// same box: 57.5 us per sweep at 2 lanes, 45.6 at 1).
template <class T>
void launch_normal(int lanes, const PhysT<T> &P, const Scalars *sc, const NList &nl,
                   const Hot<T> &hot, const Csf<T> &csf, int cap, cudaStream_t s,
                   const uint32_t *key, const T *gsum, const uint2 *crange, int ncx) {
    const bool skip = gsum != nullptr;
    if (skip) lanes = 1;
    with_lanes(lanes, [&](auto Gc) {
        constexpr int G = decltype(Gc)::value;
        int b = sweep_blocks(cap, G);
        if (P.kernel == 1) {
            if (skip) launch_k(k_normal<T, 1, G, true>, b, SWEEP_BLOCK, s, P, sc, nl, hot, csf, key, gsum, crange, ncx);
            else launch_k(k_normal<T, 1, G, false>, b, SWEEP_BLOCK, s, P, sc, nl, hot, csf, key, gsum, crange, ncx);
        } else {
            if (skip) launch_k(k_normal<T, 0, G, true>, b, SWEEP_BLOCK, s, P, sc, nl, hot, csf, key, gsum, crange, ncx);
            else launch_k(k_normal<T, 0, G, false>, b, SWEEP_BLOCK, s, P, sc, nl, hot, csf, key, gsum, crange, ncx);
        }
    });
}

template <class T>
void launch_pairsum(int lanes, const PhysT<T> &P, const Grid &g, const Scalars *sc,
                    const NList &nl, const uint32_t *key, const Hot<T> &hot, const Csf<T> &csf,
                    const Boundary &bd, const uint8_t *type, V4<T> *accN, T *gsum, uint2 *crange,
                    int cap, cudaStream_t s, bool dt_term) {
    with_lanes(lanes, [&](auto Gc) {
        constexpr int G = decltype(Gc)::value;
        int b = sweep_blocks(cap, G);
        auto go = [&](auto kern) {
            launch_k(kern, b, SWEEP_BLOCK, s, P, g, sc, nl, key, hot, csf, bd, type, accN, gsum,
                     crange);
        };
        if (P.kernel == 1) {
            if (dt_term) go(k_pairsum<T, 1, G, true>); else go(k_pairsum<T, 1, G, false>);
        } else {
            if (dt_term) go(k_pairsum<T, 0, G, true>); else go(k_pairsum<T, 0, G, false>);
        }
    });
}

template <class T, int K, int G>
static void launch_surface_k(int mode, const PhysT<T> &P, const Grid &g, const Inflow &inf,
                             Scalars *sc, const NList &nl, const Hot<T> &hot, const Csf<T> &csf,
                             const State<T> &srt, const State<T> &raw, const V4<T> *accN,
                             V2<T> *acc, T *dr, V4<T> *nH0, V4<T> *nH1, int cap, cudaStream_t s) {
    int b = sweep_blocks(cap, G);
    if (mode == 0)
        launch_k(k_surface<T, K, 0, G>, b, SWEEP_BLOCK, s, P, g, inf, sc, nl, hot, csf, srt, raw, accN, acc, dr, nH0, nH1);
    else if (mode == 1)
        launch_k(k_surface<T, K, 1, G>, b, SWEEP_BLOCK, s, P, g, inf, sc, nl, hot, csf, srt, raw, accN, acc, dr, nH0, nH1);
    else
        launch_k(k_surface<T, K, 2, G>, b, SWEEP_BLOCK, s, P, g, inf, sc, nl, hot, csf, srt, raw, accN, acc, dr, nH0, nH1);
}

// One lane per particle whatever the sweeps use: most particles only stream
// through the epilogue (the curvature walk is for N_a = 1 alone), which a
// particle's other lanes would sit out.
template <class T>
void launch_surface(int, int mode, const PhysT<T> &P, const Grid &g, const Inflow &inf,
                    Scalars *sc, const NList &nl, const Hot<T> &hot, const Csf<T> &csf,
                    const State<T> &srt, const State<T> &raw, const V4<T> *accN, V2<T> *acc,
                    T *dr, int cap, cudaStream_t s, V4<T> *nH0, V4<T> *nH1) {
    if (P.kernel == 1)
        launch_surface_k<T, 1, 1>(mode, P, g, inf, sc, nl, hot, csf, srt, raw, accN, acc, dr, nH0, nH1, cap, s);
    else
        launch_surface_k<T, 0, 1>(mode, P, g, inf, sc, nl, hot, csf, srt, raw, accN, acc, dr, nH0, nH1, cap, s);
}

template <class T, int K, int G>
static void launch_forces_k(int mode, const PhysT<T> &P, const Grid &g, const Inflow &inf,
                            Scalars *sc, const NList &nl, const uint32_t *key, const Hot<T> &hot,
                            const Csf<T> &csf, const Boundary &bd, const State<T> &srt,
                            const State<T> &raw, V2<T> *acc, T *dr, V4<T> *nH0, V4<T> *nH1,
                            int cap, cudaStream_t s) {
    int b = sweep_blocks(cap, G);
    if (mode == 0)
        launch_k(k_forces<T, K, 0, G>, b, SWEEP_BLOCK, s, P, g, inf, sc, nl, key, hot, csf, bd, srt, raw, acc, dr, nH0, nH1);
    else if (mode == 1)
        launch_k(k_forces<T, K, 1, G>, b, SWEEP_BLOCK, s, P, g, inf, sc, nl, key, hot, csf, bd, srt, raw, acc, dr, nH0, nH1);
    else
        launch_k(k_forces<T, K, 2, G>, b, SWEEP_BLOCK, s, P, g, inf, sc, nl, key, hot, csf, bd, srt, raw, acc, dr, nH0, nH1);
}

template <class T>
void launch_forces(int lanes, int mode, const PhysT<T> &P, const Grid &g, const Inflow &inf,
                   Scalars *sc, const NList &nl, const uint32_t *key, const Hot<T> &hot,
                   const Csf<T> &csf, const Boundary &bd, const State<T> &srt,
                   const State<T> &raw, V2<T> *acc, T *dr, int cap, cudaStream_t s,
                   V4<T> *nH0, V4<T> *nH1) {
    with_lanes(lanes, [&](auto Gc) {
        constexpr int G = decltype(Gc)::value;
        if (P.kernel == 1)
            launch_forces_k<T, 1, G>(mode, P, g, inf, sc, nl, key, hot, csf, bd, srt, raw, acc, dr, nH0, nH1, cap, s);
        else
            launch_forces_k<T, 0, G>(mode, P, g, inf, sc, nl, key, hot, csf, bd, srt, raw, acc, dr, nH0, nH1, cap, s);
    });
}

template <class T>
void launch_predict(const PhysT<T> &P, const Inflow &inf, Scalars *sc, const State<T> &srt,
                    const V4<T> *H0n, const V2<T> *acc, const T *dr, const Hot<T> &half, int cap,
                    cudaStream_t s) {
    launch_k(k_predict<T>, (cap + 255) / 256, 256, s, P, inf, sc, srt, H0n, acc, dr, half, cap);
}

template <class T>
void launch_spawn(const PhysT<T> &P, const Inflow &inf, Scalars *sc, const State<T> &raw,
                  const double *layer_y, int cap, int cadence, cudaStream_t s) {
    launch_k(k_spawn<T>, 1, 256, s, inf, P.ufx_d, P.ufy_d, (float)P.half_skin, sc, raw,
             layer_y, cap, cadence);
}

// ---------------------------------------------------------------------------
// Surrogate step (learned surrogate): one step of length dT = k dt with the
// mean acceleration abar = a_n + a_ref y (a_n: the SPH acceleration at the
// step start; y: the network's correction, cell order) in place of the SPH
// accelerations.  Fluid: u' = u + dT abar, r' = r + dT (u + u')/2,
// rho' = rho + dT (drho/dt)_n (the SPH continuity rate of the evaluation at
// n); inflow buffer, buffer -> fluid conversion and outflow as in the
// corrector.  Writes raw in the cell order of the evaluation and sets the
// step length for the time advance that follows.
// ---------------------------------------------------------------------------
// Adds the block's sums of v[0..NV) to out[0..NV): FP32 within a warp (a few
// terms per thread and 32 threads: rounding far below what the sums are
// compared with), FP64 across the warps of the block and across blocks (one
// atomic per value and block; blockDim.x a multiple of 32, <= 1024).  FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU, so none
// of it is per particle.
template <int NV>
__device__ __forceinline__ void block_sum_atomic(float (&v)[NV], double *__restrict__ out) {
    __shared__ double part[32][NV];
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) part[w][k] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)NV) {
        double t = 0.0;
        for (unsigned q = 0; q < nw; ++q) t += part[q][threadIdx.x];
        atomicAdd(&out[threadIdx.x], t);
    }
}

// Blocks of a grid-stride reduction over n items: few enough that the
// per-block atomics on the same addresses stay cheap.
inline int reduce_blocks(int n) { return std::max(1, std::min((n + 511) / 512, 128)); }

// Mass-weighted sums of the network's output over the fluid particles of the
// step start: ym[0..1] = sum m y, ym[2] = sum m (FP64).  The correction
// a_ref (y - ybar), ybar = ym[0..1] / ym[2], then changes the fluid's
// momentum by nothing: the pair forces that make up most of the k-step
// correction cancel in the sum (Eqs. 9, 10 are antisymmetric in a, b).
__global__ void k_surrogate_mean(int n, const uint8_t *__restrict__ type,
                                 const float *__restrict__ mass, const float2 *__restrict__ y,
                                 double *__restrict__ ym) {
    float v[3] = {0.f, 0.f, 0.f};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (type[i] != T_FLUID) continue;
        const float m = mass[i];
        const float2 yi = y[i];
        v[0] += m * yi.x;
        v[1] += m * yi.y;
        v[2] += m;
    }
    block_sum_atomic<3>(v, ym);
}

void launch_surrogate_mean(int n, const uint8_t *type, const float *mass, const float2 *y,
                           double *ym, int cap, cudaStream_t s) {
    (void)cap;
    launch_k(k_surrogate_mean, reduce_blocks(n), 512, s, n, type, mass, y, ym);
}

__device__ __forceinline__ float2 mean_of(const double *__restrict__ ym) {
    double w = ym[2];
    return w > 0.0 ? make_float2((float)(ym[0] / w), (float)(ym[1] / w)) : make_float2(0.f, 0.f);
}

// The update of particle i; d2o, s2o receive its squared displacement since
// the build and in this step (0 when it left the domain).
__device__ __forceinline__ void surrogate_update_one(
    const PhysT<float> &P, const Inflow &inf, const Grid &g, Scalars *__restrict__ sc,
    const State<float> &srt, const State<float> &raw, const float2 *__restrict__ a_n,
    const float2 *__restrict__ y, const float2 yb, float a_ref, const float *__restrict__ dr,
    double dT, int i, float &d2o, float &s2o, uint8_t *__restrict__ type0) {
    double t = sc->t, half = 0.5 * dT;
    double2 p0 = srt.pos[i];
    float2 v0 = srt.vel[i];
    float d0 = srt.drho[i], c0 = srt.drc[i];
    uint8_t typ = srt.type[i];
    type0[i] = typ;
    double2 p1 = p0;
    float2 v1 = v0;
    float d1 = d0, c1 = c0;
    float2 ds = srt.disp[i];
    float2 st = make_float2(0.f, 0.f);   // this step's move relative to the frame
    if (typ == T_FLUID) {
        float tdt = (float)dT;
        float ax = a_n[i].x + a_ref * (y[i].x - yb.x), ay = a_n[i].y + a_ref * (y[i].y - yb.y);
        float uhx = v0.x + 0.5f * tdt * ax, uhy = v0.y + 0.5f * tdt * ay;
        p1 = make_double2(p0.x + dT * (P.ufx_d + (double)uhx), p0.y + dT * (P.ufy_d + (double)uhy));
        v1 = make_float2(v0.x + tdt * ax, v0.y + tdt * ay);
        float y = tdt * dr[i] - c0;     // compensated density update
        float s = d0 + y;
        c1 = (s - d0) - y;
        d1 = s;
        st = make_float2(tdt * (P.ufx - P.dfx + uhx), tdt * (P.ufy - P.dfy + uhy));
        ds = make_float2(ds.x + st.x, ds.y + st.y);
    } else if (typ == T_BUFFER) {
        double uh = inf.on ? inflow_u(inf, t + half) : P.ufx_d + (double)v0.x;
        p1 = make_double2(p0.x + dT * uh, p0.y);
        v1 = inf.on ? make_float2((float)(inflow_u(inf, t + dT) - P.ufx_d), (float)(-P.ufy_d)) : v0;
        if (inf.on && p1.x >= inf.x_exit) typ = T_FLUID;
        st = make_float2((float)(dT * (uh - (double)P.dfx)), (float)(-dT * (double)P.dfy));
        ds = make_float2(ds.x + st.x, ds.y);
    }
    if (typ == T_FLUID && !in_box(g, p1)) {
        typ = T_DEAD;
        atomicAdd((unsigned long long *)&sc->deleted, 1ull);
    }
    raw.pos[i] = p1;
    raw.vel[i] = v1;
    raw.drho[i] = d1;
    raw.drc[i] = c1;
    raw.mass[i] = srt.mass[i];
    raw.type[i] = typ;
    raw.id[i] = srt.id[i];
    raw.disp[i] = ds;
    // largest displacement since the build and in this step, for the time
    // advance's rebuild decision (the step's move relative to the frame)
    if (typ != T_DEAD) {
        d2o = ds.x * ds.x + ds.y * ds.y;
        s2o = st.x * st.x + st.y * st.y;
    }
}

__global__ void k_surrogate_update(PhysT<float> P, Inflow inf, Grid g, Scalars *__restrict__ sc,
                                   State<float> srt, State<float> raw,
                                   const float2 *__restrict__ a_n, const float2 *__restrict__ y,
                                   const double *__restrict__ ym, float a_ref,
                                   const float *__restrict__ dr, double dT,
                                   uint8_t *__restrict__ type0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) sc->dt = dT;
    __shared__ float2 s_yb;
    if (threadIdx.x == 0) s_yb = mean_of(ym);
    __syncthreads();
    float d2 = 0.f, s2 = 0.f;
    if (i < sc->nsrt)
        surrogate_update_one(P, inf, g, sc, srt, raw, a_n, y, s_yb, a_ref, dr, dT, i, d2, s2, type0);
    // block maxima (non-negative floats order as their bits), then one atomic
    // per block and value
    __shared__ unsigned bm[2];
    if (threadIdx.x == 0) bm[0] = bm[1] = 0u;
    __syncthreads();
    const unsigned a = __reduce_max_sync(0xffffffffu, __float_as_uint(d2));
    const unsigned b2 = __reduce_max_sync(0xffffffffu, __float_as_uint(s2));
    if ((threadIdx.x & 31u) == 0) {
        atomicMax(&bm[0], a);
        atomicMax(&bm[1], b2);
    }
    __syncthreads();
    if (threadIdx.x == 0 && (bm[0] | bm[1])) {
        const int slot = blockIdx.x & (RED_SLOTS - 1);
        atomicMax(&sc->max_disp2[slot], bm[0]);
        atomicMax(&sc->max_step2[slot], bm[1]);
    }
}

void launch_surrogate_update(const PhysT<float> &P, const Inflow &inf, const Grid &g, Scalars *sc,
                             const State<float> &srt, const State<float> &raw, const float2 *a_n,
                             const float2 *y, const double *ym, float a_ref, const float *dr,
                             double dT, uint8_t *type0, int cap, cudaStream_t s) {
    launch_k(k_surrogate_update, (cap + 255) / 256, 256, s, P, inf, g, sc, srt, raw, a_n, y, ym,
             a_ref, dr, dT, type0);
}

// Residual sums of a surrogate step over the particles that are fluid at
// both ends (cell order; type0 from the start, type from the end of the
// step: inflow particles that became fluid during the step and outflow
// deletions are left out), accumulated in FP64 across blocks:
//   sums[0..1] = sum m (abar - (a_n + a_k)/2)      (momentum balance)
//   sums[2]    = sum m |(a_n + a_k)/2|
//   sums[3]    = sum (drho/dt_k - drho/dt_n)^2     (density)
//   sums[4]    = fluid count
//   sums[5]    = sum |abar - (a_n + a_k)/2|^2      (acceleration field)
//   sums[6]    = sum |(a_n + a_k)/2|^2
// with abar = a_n + a_ref (y - ybar) (k_surrogate_mean).
__global__ void k_surrogate_residual(int n, const uint8_t *__restrict__ type0,
                                     const uint8_t *__restrict__ type,
                                     const float *__restrict__ mass,
                                     const float2 *__restrict__ y, const double *__restrict__ ym,
                                     float a_ref,
                                     const float2 *__restrict__ a_n, const float2 *__restrict__ a_k,
                                     const float *__restrict__ dr_n, const float *__restrict__ dr_k,
                                     double *__restrict__ sums) {
    float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    __shared__ float2 s_yb;
    if (threadIdx.x == 0) s_yb = mean_of(ym);
    __syncthreads();
    const float2 yb = s_yb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (type0[i] != T_FLUID || type[i] != T_FLUID) continue;
        // per particle in FP32 (the rounding of a term is far below the
        // threshold)
        const float m = mass[i];
        const float2 an = a_n[i], ak = a_k[i], yi = y[i];
        const float mx = 0.5f * (an.x + ak.x), my = 0.5f * (an.y + ak.y);
        const float ex = an.x + a_ref * (yi.x - yb.x) - mx;
        const float ey = an.y + a_ref * (yi.y - yb.y) - my;
        const float dd = dr_k[i] - dr_n[i];
        const float t2 = mx * mx + my * my;
        v[0] += m * ex;
        v[1] += m * ey;
        v[2] += m * sqrtf(t2);
        v[3] += dd * dd;
        v[4] += 1.f;
        v[5] += ex * ex + ey * ey;
        v[6] += t2;
    }
    block_sum_atomic<7>(v, sums);
}

void launch_surrogate_residual(int n, const uint8_t *type0, const uint8_t *type, const float *mass,
                               const float2 *abar, const double *ym, float a_ref,
                               const float2 *a_n, const float2 *a_k, const float *dr_n,
                               const float *dr_k, double *sums, int cap, cudaStream_t s) {
    (void)cap;
    launch_k(k_surrogate_residual, reduce_blocks(n), 512, s, n, type0, type, mass, abar, ym, a_ref,
             a_n, a_k, dr_n, dr_k, sums);
}

// ---------------------------------------------------------------------------
// Run statistics over raw[0, n): per fluid particle m, m u, m |u|^2 / 2,
// -m g . r, m e(rho) (Tait elastic energy) accumulated in FP64; counts of
// fluid and buffer particles; max |rho - rho0| / rho0 as ordered bits.
// acc[0..5] = mass, px, py, kinetic, potential, elastic; cnt[0..1] = fluid,
// buffer; cnt[2] = bits of the maximum.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_stats(State<T> raw, const Scalars *__restrict__ sc, double ufx, double ufy,
                        double gx, double gy, double rho0, double B, double gamma,
                        double *__restrict__ acc, unsigned long long *__restrict__ cnt) {
    const int n = sc->n;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long nf = 0, nb = 0, mx = 0;
    if (i < n) {
        uint8_t typ = raw.type[i];
        if (typ == T_FLUID) {
            double m = (double)raw.mass[i];
            double ux = ufx + (double)raw.vel[i].x, uy = ufy + (double)raw.vel[i].y;
            double2 p = raw.pos[i];
            // the compensated offset: drho - carry
            double d = ((double)raw.drho[i] - (double)raw.drc[i]) / rho0;
            double e = B / rho0 * (expm1((gamma - 1.0) * log1p(d)) / (gamma - 1.0) - d / (1.0 + d));
            v[0] = m;
            v[1] = m * ux;
            v[2] = m * uy;
            v[3] = 0.5 * m * (ux * ux + uy * uy);
            v[4] = -m * (gx * p.x + gy * p.y);
            v[5] = m * e;
            nf = 1;
            mx = (unsigned long long)__double_as_longlong(fabs(d));
        } else if (typ == T_BUFFER) {
            nb = 1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
        unsigned long long w = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = w > mx ? w : mx;
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) atomicAdd(&acc[k], v[k]);
        atomicAdd(&cnt[0], nf);
        atomicAdd(&cnt[1], nb);
        atomicMax(&cnt[2], mx);
    }
}

template <class T>
void launch_stats(const PhysT<T> &P, const State<T> &raw, const Scalars *sc, double gx, double gy,
                  double rho0, double B, double gamma, double *acc, unsigned long long *cnt,
                  int cap, cudaStream_t s) {
    launch_k(k_stats<T>, (cap + 255) / 256, 256, s, raw, sc, P.ufx_d, P.ufy_d, gx, gy, rho0, B,
             gamma, acc, cnt);
}

__global__ void k_decide(cudaGraphConditionalHandle h, const Scalars *__restrict__ sc) {
    cudaGraphSetConditional(h, sc->need_full ? 1u : 0u);
}

void *decide_kernel() { return (void *)k_decide; }

#define SPH_INST(T)                                                                              \
    template void launch_reorder<T>(const PhysT<T> &, const Grid &, Scalars *, const CellSort &,  \
                                    const State<T> &, const State<T> &, const Hot<T> &, int,      \
                                    cudaStream_t, int);                                           \
    template void launch_refresh<T>(const PhysT<T> &, const Grid &, Scalars *, const uint32_t *,  \
                                    const State<T> &, const State<T> &, const Hot<T> &, int,      \
                                    cudaStream_t, int);                                           \
    template void launch_build<T>(int, bool, const PhysT<T> &, const Grid &, Scalars *,          \
                                  const uint2 *, const uint32_t *, const Hot<T> &,                \
                                  const NList &, const Csf<T> &, int, cudaStream_t, int);         \
    template void launch_colour<T>(int, const PhysT<T> &, const Scalars *, const NList &,         \
                                   const Hot<T> &, const Csf<T> &, int, cudaStream_t, int);       \
    template void launch_density<T>(int, const PhysT<T> &, const Scalars *, const NList &,        \
                                    const Hot<T> &, const T *, const uint8_t *, T *, int,         \
                                    cudaStream_t, int);                                           \
    template void launch_normal<T>(int, const PhysT<T> &, const Scalars *, const NList &,         \
                                   const Hot<T> &, const Csf<T> &, int, cudaStream_t,             \
                                   const uint32_t *, const T *, const uint2 *, int);              \
    template void launch_pairsum<T>(int, const PhysT<T> &, const Grid &, const Scalars *,         \
                                    const NList &, const uint32_t *, const Hot<T> &,              \
                                    const Csf<T> &, const Boundary &, const uint8_t *, V4<T> *,   \
                                    T *, uint2 *, int, cudaStream_t, bool);                       \
    template void launch_surface<T>(int, int, const PhysT<T> &, const Grid &, const Inflow &,    \
                                    Scalars *, const NList &, const Hot<T> &, const Csf<T> &,     \
                                    const State<T> &, const State<T> &, const V4<T> *, V2<T> *,   \
                                    T *, int, cudaStream_t, V4<T> *, V4<T> *);                    \
    template void launch_forces<T>(int, int, const PhysT<T> &, const Grid &, const Inflow &,     \
                                   Scalars *, const NList &, const uint32_t *, const Hot<T> &,    \
                                   const Csf<T> &, const Boundary &, const State<T> &,            \
                                   const State<T> &, V2<T> *, T *, int, cudaStream_t, V4<T> *,    \
                                   V4<T> *);                                                      \
    template void launch_predict<T>(const PhysT<T> &, const Inflow &, Scalars *,                 \
                                    const State<T> &, const V4<T> *, const V2<T> *, const T *,    \
                                    const Hot<T> &, int, cudaStream_t);                           \
    template void launch_spawn<T>(const PhysT<T> &, const Inflow &, Scalars *, const State<T> &, \
                                  const double *, int, int, cudaStream_t);                        \
    template void launch_stats<T>(const PhysT<T> &, const State<T> &, const Scalars *, double,   \
                                  double, double, double, double, double *,                       \
                                  unsigned long long *, int, cudaStream_t);

SPH_INST(float)
SPH_INST(double)

}  // namespace sph
