/*
 * FP64 CPU oracle for the 2D WCSPH jet-breakup method of arXiv 1603.02421.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests/, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  See the header
 * for the contract.  Built with -ffp-contract=off so that no multiply-add is
 * fused and the arithmetic is the same on every host.
 *
 * Each function cites the section / equation of the paper it restates.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Sec. 2-5: kernel functions, W(r,h) = kappa / h^nu * f(q), q = r/h, nu = 2 */
/* ------------------------------------------------------------------------ */

/* 2D normalisation constants.  Eq. 27 prints 10/(7 pi) for the cubic spline,
 * which integrates to one.  Eq. 28 prints 7/(8 pi) for the Wendland form
 * (1+2q)(2-q)^4, which integrates to 8 in 2D; the unit-integral value for
 * that polynomial is 7/(64 pi).  The oracle uses the unit-integral value,
 * since Sec. 2-2 states that the kernels integrate to one. */
double orc_kernel_norm(int kernel)
{
    if (kernel == ORC_CUBIC) return 10.0 / (7.0 * ORC_PI);
    return 7.0 / (64.0 * ORC_PI);
}

/* Eq. 27 (cubic spline) and Eq. 28 (Wendland C2). */
double orc_W(int kernel, double r, double h)
{
    double q = r / h;
    double k = orc_kernel_norm(kernel) / (h * h);
    if (q >= 2.0) return 0.0;
    if (kernel == ORC_CUBIC) {
        if (q <= 1.0) return k * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
        double t = 2.0 - q;
        return k * 0.25 * t * t * t;
    }
    double t = 2.0 - q;
    return k * (1.0 + 2.0 * q) * t * t * t * t;
}

/* dW/dr of Eq. 27 / Eq. 28, differentiated by hand:
 *   cubic:    q <= 1:  (kappa/h^3)(-3q + 9q^2/4);  1 < q < 2: -(3 kappa/(4h^3))(2-q)^2
 *   Wendland: -(10 kappa/h^3) q (2-q)^3 */
double orc_dWdr(int kernel, double r, double h)
{
    double q = r / h;
    double k = orc_kernel_norm(kernel) / (h * h * h);
    if (q >= 2.0) return 0.0;
    if (kernel == ORC_CUBIC) {
        if (q <= 1.0) return k * (-3.0 * q + 2.25 * q * q);
        double t = 2.0 - q;
        return -0.75 * k * t * t;
    }
    double t = 2.0 - q;
    return -10.0 * k * q * t * t * t;
}

/* (1/r) dW/dr, written so that it is finite at r = 0.  The kernel gradient
 * is grad_a W_ab = (1/r dW/dr) * (r_a - r_b). */
static double grad_factor(int kernel, double r, double h)
{
    double q = r / h;
    double k = orc_kernel_norm(kernel) / (h * h * h * h);
    if (q >= 2.0) return 0.0;
    if (kernel == ORC_CUBIC) {
        if (q <= 1.0) return k * (-3.0 + 2.25 * q);
        double t = 2.0 - q;
        return -0.75 * k * t * t / q;
    }
    double t = 2.0 - q;
    return -10.0 * k * t * t * t;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2-4, Eq. 26: Tait equation of state, B = rho0 c0^2 / gamma.          */
/* ------------------------------------------------------------------------ */
double orc_pressure(double rho, double rho0, double c0, double gamma)
{
    double B = rho0 * c0 * c0 / gamma;
    return B * (pow(rho / rho0, gamma) - 1.0);
}

/* The paper uses c_a in Eq. 10 and Eq. 31 without defining it; the reading
 * taken is the local sound speed of Eq. 26, c = sqrt(dP/drho)
 * = c0 (rho/rho0)^((gamma-1)/2). */
double orc_sound_speed(double rho, double rho0, double c0, double gamma)
{
    return c0 * pow(rho / rho0, 0.5 * (gamma - 1.0));
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Sec. 2-7: neighbour search.  The brute-force mode tests every pair; the   */
/* cell mode bins particles into square cells slightly larger than the       */
/* search radius and tests the 3x3 block of cells around each particle.      */
/* Both produce the same lists, ascending in b.                              */
/* ------------------------------------------------------------------------ */
static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static int is_pair(const double *x, const double *y, long long a, long long b, double r2max)
{
    double dx = x[a] - x[b];
    double dy = y[a] - y[b];
    double r2 = dx * dx + dy * dy;
    return r2 < r2max;
}

/* Threads of the particle loops (OpenMP, when the oracle is built with it).
 * Every particle's sums keep their fixed ascending-neighbour order whatever
 * the thread count, so results do not depend on it. */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Candidates of particle a: every b of the 3x3 cell block (cell mode) or
 * every particle (brute force).  Pass 1 counts the pairs of each particle,
 * pass 2 writes them at the offsets of the counts; both visit candidates in
 * the same order, and each particle's list is then sorted ascending. */
typedef struct {
    long long n, ncx, ncy;
    const double *x, *y;
    const unsigned char *active;
    double r2max;
    int use_cells;
    const long long *head, *next, *cid;
} nb_grid;

static long long visit(const nb_grid *G, long long a, int *out)
{
    long long k = 0;
    if (G->active && !G->active[a]) return 0;
    if (!G->use_cells) {
        for (long long b = 0; b < G->n; ++b) {
            if (b == a || (G->active && !G->active[b])) continue;
            if (!is_pair(G->x, G->y, a, b, G->r2max)) continue;
            if (out) out[k] = (int)b;
            ++k;
        }
        return k;
    }
    if (G->cid[a] < 0) return 0;
    long long cx = G->cid[a] % G->ncx, cy = G->cid[a] / G->ncx;
    for (long long jy = cy - 1; jy <= cy + 1; ++jy) {
        if (jy < 0 || jy >= G->ncy) continue;
        for (long long jx = cx - 1; jx <= cx + 1; ++jx) {
            if (jx < 0 || jx >= G->ncx) continue;
            for (long long b = G->head[jy * G->ncx + jx]; b >= 0; b = G->next[b]) {
                if (b == a || !is_pair(G->x, G->y, a, b, G->r2max)) continue;
                if (out) out[k] = (int)b;
                ++k;
            }
        }
    }
    return k;
}

long long orc_neighbours(long long n, const double *x, const double *y,
                         const unsigned char *active, double radius,
                         int use_cells, long long **start_out, int **list_out)
{
    nb_grid G;
    memset(&G, 0, sizeof(G));
    G.n = n; G.x = x; G.y = y; G.active = active;
    G.r2max = radius * radius;
    G.use_cells = use_cells;
    G.ncx = G.ncy = 1;
    long long *start = (long long *)calloc((size_t)n + 1, sizeof(long long));
    long long *head = NULL, *next = NULL, *cid = NULL;
    if (!start) return -1;

    if (use_cells) {
        /* cell list: square cells slightly larger than the search radius */
        double cell = radius * 1.01;
        double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
        for (long long a = 0; a < n; ++a) {
            if (active && !active[a]) continue;
            if (x[a] < x0) x0 = x[a];
            if (y[a] < y0) y0 = y[a];
            if (x[a] > x1) x1 = x[a];
            if (y[a] > y1) y1 = y[a];
        }
        if (x1 >= x0) {
            G.ncx = (long long)floor((x1 - x0) / cell) + 1;
            G.ncy = (long long)floor((y1 - y0) / cell) + 1;
        }
        long long ncell = G.ncx * G.ncy;
        head = (long long *)malloc((size_t)ncell * sizeof(long long));
        next = (long long *)malloc(((size_t)n + 1) * sizeof(long long));
        cid = (long long *)malloc(((size_t)n + 1) * sizeof(long long));
        if (!head || !next || !cid) {
            free(head); free(next); free(cid); free(start);
            return -1;
        }
        for (long long c = 0; c < ncell; ++c) head[c] = -1;
        /* push in descending index so that each cell's chain is ascending */
        for (long long a = n - 1; a >= 0; --a) {
            cid[a] = -1;
            if (active && !active[a]) continue;
            long long cx = (long long)floor((x[a] - x0) / cell);
            long long cy = (long long)floor((y[a] - y0) / cell);
            if (cx >= G.ncx) cx = G.ncx - 1;
            if (cy >= G.ncy) cy = G.ncy - 1;
            cid[a] = cy * G.ncx + cx;
            next[a] = head[cid[a]];
            head[cid[a]] = a;
        }
        G.head = head; G.next = next; G.cid = cid;
    }

    /* pass 1: counts; prefix sum into start */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
    for (long long a = 0; a < n; ++a) start[a + 1] = visit(&G, a, NULL);
    for (long long a = 0; a < n; ++a) start[a + 1] += start[a];
    long long total = start[n];
    int *list = (int *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int));
    if (!list) {
        free(head); free(next); free(cid); free(start);
        return -1;
    }
    /* pass 2: fill, each list ascending in b */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
    for (long long a = 0; a < n; ++a) {
        long long k = visit(&G, a, list + start[a]);
        (void)k;
        qsort(list + start[a], (size_t)(start[a + 1] - start[a]), sizeof(int), cmp_int);
    }
    free(head); free(next); free(cid);
    *start_out = start;
    *list_out = list;
    return total;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2-6, Eq. 29: repulsive boundary force per unit mass on fluid a from  */
/* boundary particle k, f = n R(psi) P(xi) eps(z, u_perp).                   */
/* The paper prints only this product; the factors are the Monaghan-Kos /    */
/* Rogers et al. forms it cites:                                             */
/*   R(psi) = A (1 - q)/sqrt(q), q = psi/(2h), for 0 < psi < 2h              */
/*   P(xi)  = (1 + cos(pi xi / db))/2 for |xi| < db (sums to one along a     */
/*            straight wall of spacing db, so the force does not vary as a   */
/*            particle slides between two boundary particles)                */
/*   eps    = eps(z) + eps(u_perp), z = y_a - h0:                            */
/*            eps(z) = 0.02 (z >= 0), |z/h0| + 0.02 (-h0 < z < 0), 1 else    */
/*            eps(u) = 0 (u >= 0), min(|20 u| / c0, 1) (u < 0)              */
/* ------------------------------------------------------------------------ */
static void wall_force(const orc_params *p, double xa, double ya, double ua, double va,
                       double bx, double by, double bnx, double bny, double *fx, double *fy)
{
    double h = p->h;
    double dx = xa - bx, dy = ya - by;
    double psi = dx * bnx + dy * bny;
    double xi = -dx * bny + dy * bnx;
    if (!(psi > 0.0 && psi < 2.0 * h && fabs(xi) < p->wall_db)) return;
    double q = psi / (2.0 * h);
    double R = p->wall_A * (1.0 - q) / sqrt(q);
    double P = 0.5 * (1.0 + cos(ORC_PI * xi / p->wall_db));
    double ez;
    if (p->wall_h0 > 0.0) {
        double z = ya - p->wall_h0;
        if (z >= 0.0) ez = 0.02;
        else if (z > -p->wall_h0) ez = fabs(z / p->wall_h0) + 0.02;
        else ez = 1.0;
    } else {
        ez = 1.0;
    }
    double uperp = ua * bnx + va * bny;
    double eu;
    if (uperp >= 0.0) eu = 0.0;
    else {
        eu = fabs(20.0 * uperp) / p->c0;
        if (eu > 1.0) eu = 1.0;
    }
    double mag = R * P * (ez + eu);
    *fx += mag * bnx;
    *fy += mag * bny;
}

/* ------------------------------------------------------------------------ */
/* One evaluation of the semi-discrete equations at a given state.           */
/* ------------------------------------------------------------------------ */
int orc_evaluate(const orc_params *p, const orc_state *s, orc_out *o)
{
    long long n = s->n;
    int K = p->kernel;
    double h = p->h;
    long long *start = NULL;
    int *nb = NULL;

    /* Sec. 2-7: neighbours of every fluid/buffer particle within 2h. */
    if (orc_neighbours(n, s->x, s->y, NULL, 2.0 * h, p->use_cells, &start, &nb) < 0)
        return -1;

    double *P = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *c = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *V = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *nhx = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *nhy = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!P || !c || !V || !nhx || !nhy) {
        free(P); free(c); free(V); free(nhx); free(nhy); free(start); free(nb);
        return -1;
    }

    /* Eq. 26 and the sound-speed reading; V_b = m_b / rho_b (Eq. 4). */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
    for (long long a = 0; a < n; ++a) {
        P[a] = orc_pressure(s->rho[a], p->rho0, p->c0, p->gamma);
        c[a] = orc_sound_speed(s->rho[a], p->rho0, p->c0, p->gamma);
        V[a] = s->m[a] / s->rho[a];
    }

    /* Sec. 2-3: CSF surface tension (Morris). */
    for (long long a = 0; a < n; ++a) {
        o->C[a] = 0.0; o->nx[a] = 0.0; o->ny[a] = 0.0; o->kappa[a] = 0.0; o->Nflag[a] = 0;
    }
    if (p->sigma > 0.0) {
        double W0 = orc_W(K, 0.0, h);
        /* Eq. 14: colour C_a = sum_b V_b W_ab, the particle itself included. */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
        for (long long a = 0; a < n; ++a) {
            double sum = V[a] * W0;
            for (long long k = start[a]; k < start[a + 1]; ++k) {
                int b = nb[k];
                double dx = s->x[a] - s->x[b], dy = s->y[a] - s->y[b];
                double r = sqrt(dx * dx + dy * dy);
                sum += V[b] * orc_W(K, r, h);
            }
            o->C[a] = sum;
        }
        /* Eq. 18: n_a = sum_b V_b (C_b - C_a) grad_a W_ab;
         * Eq. 20: N_a = 1 if |n_a| > eps; Eq. 21: unit normal or zero. */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
        for (long long a = 0; a < n; ++a) {
            double sx = 0.0, sy = 0.0;
            for (long long k = start[a]; k < start[a + 1]; ++k) {
                int b = nb[k];
                double dx = s->x[a] - s->x[b], dy = s->y[a] - s->y[b];
                double r = sqrt(dx * dx + dy * dy);
                double F = grad_factor(K, r, h);
                double w = V[b] * (o->C[b] - o->C[a]) * F;
                sx += w * dx;
                sy += w * dy;
            }
            o->nx[a] = sx;
            o->ny[a] = sy;
            double mag = sqrt(sx * sx + sy * sy);
            if (mag > p->eps_n) {
                o->Nflag[a] = 1;
                nhx[a] = sx / mag;
                nhy[a] = sy / mag;
            }
        }
        /* Eq. 23: normalised curvature
         *   kappa_a = sum_b min(N_a,N_b) V_b (nhat_b - nhat_a).grad_a W_ab
         *           / sum_b min(N_a,N_b) V_b W_ab,
         * the denominator including the particle itself; kappa = 0 when the
         * denominator vanishes (N_a = 0). */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
        for (long long a = 0; a < n; ++a) {
            if (!o->Nflag[a]) continue;
            double num = 0.0, den = V[a] * W0;
            for (long long k = start[a]; k < start[a + 1]; ++k) {
                int b = nb[k];
                if (!o->Nflag[b]) continue;
                double dx = s->x[a] - s->x[b], dy = s->y[a] - s->y[b];
                double r = sqrt(dx * dx + dy * dy);
                double F = grad_factor(K, r, h);
                num += V[b] * ((nhx[b] - nhx[a]) * dx + (nhy[b] - nhy[a]) * dy) * F;
                den += V[b] * orc_W(K, r, h);
            }
            o->kappa[a] = den > 0.0 ? num / den : 0.0;
        }
    }

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
    for (long long a = 0; a < n; ++a) {
        o->ax[a] = 0.0; o->ay[a] = 0.0; o->drho[a] = 0.0;
        o->dt_f[a] = INFINITY; o->dt_cv[a] = INFINITY;
        if (s->type[a] != ORC_FLUID) continue;   /* buffer motion is prescribed */

        double Pa = P[a] / (s->rho[a] * s->rho[a]);
        double drho = 0.0, ax = 0.0, ay = 0.0, vmax = 0.0;
        for (long long k = start[a]; k < start[a + 1]; ++k) {
            int b = nb[k];
            double dx = s->x[a] - s->x[b], dy = s->y[a] - s->y[b];
            double r2 = dx * dx + dy * dy;
            double r = sqrt(r2);
            double F = grad_factor(K, r, h);
            double gx = F * dx, gy = F * dy;             /* grad_a W_ab */
            double du = s->u[a] - s->u[b], dv = s->v[a] - s->v[b];
            double udotr = du * dx + dv * dy;
            /* Eq. 7: continuity. */
            drho += s->m[b] * (du * gx + dv * gy);
            /* Eq. 10: Monaghan artificial viscosity, approaching pairs only. */
            double Pi = 0.0;
            if (udotr < 0.0) {
                double cbar = 0.5 * (c[a] + c[b]);
                double rbar = 0.5 * (s->rho[a] + s->rho[b]);
                Pi = -p->alpha * h * cbar * udotr / (rbar * (r2 + p->eta2));
            }
            /* Eq. 9 / Eq. 25: pressure gradient plus viscosity. */
            double t = Pa + P[b] / (s->rho[b] * s->rho[b]) + Pi;
            ax -= s->m[b] * t * gx;
            ay -= s->m[b] * t * gy;
            /* Eq. 31: max_b |h u_ab . r_ab / r_ab^2| */
            if (r2 > 0.0) {
                double cv = fabs(h * udotr / r2);
                if (cv > vmax) vmax = cv;
            }
        }
        /* Eq. 24: (a_s)_a = -(sigma/rho_a) kappa_a n_a, sigma uniform. */
        if (p->sigma > 0.0) {
            ax -= p->sigma / s->rho[a] * o->kappa[a] * o->nx[a];
            ay -= p->sigma / s->rho[a] * o->kappa[a] * o->ny[a];
        }
        /* Eq. 25: body force. */
        ax += p->gx;
        ay += p->gy;
        /* Eq. 29: repulsive walls. */
        for (long long k = 0; k < s->nb; ++k)
            wall_force(p, s->x[a], s->y[a], s->u[a], s->v[a],
                       s->bx[k], s->by[k], s->bnx[k], s->bny[k], &ax, &ay);

        o->ax[a] = ax;
        o->ay[a] = ay;
        o->drho[a] = drho;
        /* Eq. 30 and Eq. 31 per-particle terms; Eq. 32 takes their minimum. */
        double fa = sqrt(ax * ax + ay * ay);
        o->dt_f[a] = fa > 0.0 ? sqrt(h / fa) : INFINITY;
        o->dt_cv[a] = h / (c[a] + vmax);
    }

    free(P); free(c); free(V); free(nhx); free(nhy); free(start); free(nb);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3-2: breakup criterion.  Two particles are joined when closer than   */
/* the radius (1.5 h); the jet is broken where no chain of such links        */
/* remains.  Plain breadth-first search over the neighbour lists.            */
/* ------------------------------------------------------------------------ */
long long orc_components(long long n, const double *x, const double *y,
                         double radius, int use_cells, long long *label)
{
    long long *start = NULL;
    int *nb = NULL;
    if (orc_neighbours(n, x, y, NULL, radius, use_cells, &start, &nb) < 0) return -1;
    long long *queue = (long long *)malloc((size_t)(n > 0 ? n : 1) * sizeof(long long));
    if (!queue) { free(start); free(nb); return -1; }
    for (long long a = 0; a < n; ++a) label[a] = -1;
    long long ncomp = 0;
    for (long long a = 0; a < n; ++a) {
        if (label[a] >= 0) continue;
        ++ncomp;
        long long head = 0, tail = 0;
        queue[tail++] = a;
        label[a] = a;
        while (head < tail) {
            long long i = queue[head++];
            for (long long k = start[i]; k < start[i + 1]; ++k) {
                int b = nb[k];
                if (label[b] < 0) {
                    label[b] = a;
                    queue[tail++] = b;
                }
            }
        }
    }
    free(queue); free(start); free(nb);
    return ncomp;
}

int orc_summation_density(const orc_params *p, const orc_state *s, double *rho)
{
    long long n = s->n;
    int K = p->kernel;
    double h = p->h;
    long long *start = NULL;
    int *nb = NULL;
    if (orc_neighbours(n, s->x, s->y, NULL, 2.0 * h, p->use_cells, &start, &nb) < 0)
        return -1;
    double W0 = orc_W(K, 0.0, h);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
    for (long long a = 0; a < n; ++a) {
        double sum = s->m[a] * W0;
        for (long long k = start[a]; k < start[a + 1]; ++k) {
            int b = nb[k];
            double dx = s->x[a] - s->x[b], dy = s->y[a] - s->y[b];
            sum += s->m[b] * orc_W(K, sqrt(dx * dx + dy * dy), h);
        }
        rho[a] = sum;
    }
    free(start);
    free(nb);
    return 0;
}
