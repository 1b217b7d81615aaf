/*
 * Memory and undefined-behaviour check of the FP64 oracle (TEST
 * INFRASTRUCTURE ONLY): built with -fsanitize=address,undefined by
 * tests/test_oracle_sanitized.py, it drives every entry point of
 * sph_oracle.c over the edge cases of the method -- no particles, one
 * particle, coincident particles (r = 0 in Eqs. 7, 9-10, 18, 23, 31),
 * particles exactly 2h apart and on cell edges, a lattice patch with
 * surface tension and walls (Eq. 29), buffer particles -- and exits 0 when
 * no check fires.  The sanitizers abort on the first error.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sph_oracle.h"

static unsigned long long lcg = 88172645463325252ull;
static double uniform(void)
{
    lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg >> 11) / 9007199254740992.0;
}

typedef struct {
    long long n, nb;
    double *x, *y, *u, *v, *rho, *m, *bx, *by, *bnx, *bny;
    unsigned char *type;
} case_t;

static case_t make_case(long long n, long long nb)
{
    case_t c;
    c.n = n;
    c.nb = nb;
    size_t k = (size_t)(n > 0 ? n : 1), kb = (size_t)(nb > 0 ? nb : 1);
    c.x = calloc(k, sizeof(double)); c.y = calloc(k, sizeof(double));
    c.u = calloc(k, sizeof(double)); c.v = calloc(k, sizeof(double));
    c.rho = calloc(k, sizeof(double)); c.m = calloc(k, sizeof(double));
    c.type = calloc(k, 1);
    c.bx = calloc(kb, sizeof(double)); c.by = calloc(kb, sizeof(double));
    c.bnx = calloc(kb, sizeof(double)); c.bny = calloc(kb, sizeof(double));
    for (long long i = 0; i < n; ++i) { c.rho[i] = 1000.0; c.m[i] = 0.4; }
    return c;
}

static void free_case(case_t *c)
{
    free(c->x); free(c->y); free(c->u); free(c->v); free(c->rho); free(c->m); free(c->type);
    free(c->bx); free(c->by); free(c->bnx); free(c->bny);
}

static int run_all(const case_t *c, double h, int kernel, double sigma)
{
    orc_params p;
    memset(&p, 0, sizeof p);
    p.kernel = kernel;
    p.h = h;
    p.rho0 = 1000.0; p.c0 = 10.0; p.gamma = 7.0;
    p.alpha = 0.3; p.eta2 = 0.01 * h * h;
    p.sigma = sigma; p.eps_n = 0.01 / h;
    p.gy = -9.81;
    p.wall_A = 0.01 * 100.0 / h; p.wall_db = 0.5 * h / 1.3; p.wall_h0 = 0.3;
    orc_state s = {c->n, c->x, c->y, c->u, c->v, c->rho, c->m, c->type,
                   c->nb, c->bx, c->by, c->bnx, c->bny};
    size_t k = (size_t)(c->n > 0 ? c->n : 1);
    double *buf = calloc(9 * k, sizeof(double));
    unsigned char *N = calloc(k, 1);
    orc_out o = {buf, buf + k, buf + 2 * k, buf + 3 * k, buf + 4 * k, buf + 5 * k, buf + 6 * k,
                 N, buf + 7 * k, buf + 8 * k};
    int bad = 0;
    for (int cells = 0; cells <= 1; ++cells) {
        p.use_cells = cells;
        if (orc_evaluate(&p, &s, &o) != 0) bad = 1;
        for (long long i = 0; i < c->n; ++i)
            if (c->type[i] == ORC_FLUID && !(isfinite(o.ax[i]) && isfinite(o.ay[i])))
                bad = 1;
        double *rs = calloc(k, sizeof(double));
        if (orc_summation_density(&p, &s, rs) != 0) bad = 1;
        free(rs);
        long long *lab = calloc(k, sizeof(long long));
        if (orc_components(c->n, c->x, c->y, 1.5 * h, cells, lab) < 0) bad = 1;
        free(lab);
        long long *start = NULL;
        int *list = NULL;
        if (orc_neighbours(c->n, c->x, c->y, c->type, 2.0 * h, cells, &start, &list) < 0) bad = 1;
        orc_free(start);
        orc_free(list);
    }
    free(buf);
    free(N);
    return bad;
}

int main(void)
{
    int bad = 0;
    double h = 0.026;
    for (int kernel = 0; kernel <= 1; ++kernel) {
        /* no particles, one particle */
        case_t c0 = make_case(0, 0);
        bad |= run_all(&c0, h, kernel, 1.0);
        free_case(&c0);
        case_t c1 = make_case(1, 0);
        bad |= run_all(&c1, h, kernel, 1.0);
        free_case(&c1);
        /* coincident pair, a pair exactly 2h apart on a cell edge, a buffer particle */
        case_t c2 = make_case(5, 0);
        c2.x[1] = 0.0; c2.x[2] = 0.5; c2.x[3] = 0.5 + 2.0 * h; c2.x[4] = 0.25;
        c2.u[0] = 0.1; c2.u[1] = -0.1;
        c2.type[4] = ORC_BUFFER;
        bad |= run_all(&c2, h, kernel, 1.0);
        free_case(&c2);
        /* jittered lattice patch with a wall below it and surface tension */
        long long nx = 30, ny = 20, nb = 120;
        case_t c3 = make_case(nx * ny, nb);
        double dx = h / 1.3;
        for (long long j = 0; j < ny; ++j)
            for (long long i = 0; i < nx; ++i) {
                long long a = j * nx + i;
                c3.x[a] = (i + 0.5) * dx + 0.05 * dx * (uniform() - 0.5);
                c3.y[a] = (j + 0.5) * dx + 0.05 * dx * (uniform() - 0.5);
                c3.u[a] = 0.1 * (uniform() - 0.5);
                c3.v[a] = 0.1 * (uniform() - 0.5);
                c3.rho[a] = 1000.0 * (1.0 + 0.01 * (uniform() - 0.5));
                c3.type[a] = i == 0 ? ORC_BUFFER : ORC_FLUID;
            }
        for (long long b = 0; b < nb; ++b) {
            c3.bx[b] = (b - 10) * 0.5 * dx;
            c3.by[b] = 0.0;
            c3.bnx[b] = 0.0;
            c3.bny[b] = 1.0;
        }
        bad |= run_all(&c3, h, kernel, 1.0);
        bad |= run_all(&c3, h, kernel, 0.0);
        free_case(&c3);
    }
    if (bad) {
        fprintf(stderr, "oracle returned an error or a non-finite value\n");
        return 1;
    }
    printf("oracle sanitized run ok\n");
    return 0;
}
