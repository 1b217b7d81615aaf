/*
 * FP64 CPU oracle for the 2D weakly-compressible SPH method of Pourabdian,
 * Omidvar & Morad, "Numerical simulation of liquid jet breakup using SPH"
 * (arXiv 1603.02421).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.  It
 * may be built, loaded and called only by the test suite, by the package's
 * smoke check and by the benchmark's CPU-baseline leg.  The product path
 * never links it and shares no code, header, table or helper with it.
 *
 * Everything is plain double precision, evaluated in the order the paper
 * states the method, with neighbour sums taken in ascending particle-index
 * order (particles are stored in id order).
 *
 * Parity is pinned for every function by the tests under tests/ (closed
 * forms, invariants, brute force).  The repulsive wall force (Sec. 2-6,
 * Eq. 29) prints only the product structure of the force; its factor
 * functions follow a literature reading, and their magnitudes are "parity
 * unpinned" against the paper; pinned are only the properties the paper
 * states: the force acts along the wall normal, stays constant along a
 * straight wall, repels with a strength that decreases with the normal
 * distance (zero from 2h on), and grows with the local depth of the fluid and
 * with the speed at which a particle approaches the wall.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CUBIC = 0, ORC_WENDLAND = 1 };
enum { ORC_FLUID = 0, ORC_BOUNDARY = 1, ORC_BUFFER = 2 };

typedef struct {
    int kernel;        /* ORC_CUBIC (Eq. 27) or ORC_WENDLAND (Eq. 28)          */
    int use_cells;     /* 0: O(N^2) neighbour search, 1: cell linked list     */
    double h;          /* smoothing length, h = 1.3 dx (Sec. 2-2)             */
    double rho0, c0, gamma;           /* Tait EOS, Eq. 26                      */
    double alpha, eta2;               /* artificial viscosity, Eq. 10          */
    double sigma, eps_n;              /* CSF, Eqs. 20-24 (sigma = 0: off)      */
    double gx, gy;                    /* body force g, Eq. 2                   */
    double wall_A, wall_db, wall_h0;  /* repulsive wall force, Eq. 29         */
} orc_params;

typedef struct {
    long long n;                                    /* fluid + buffer       */
    const double *x, *y, *u, *v, *rho, *m;
    const unsigned char *type;                      /* ORC_FLUID/ORC_BUFFER */
    long long nb;                                   /* boundary particles   */
    const double *bx, *by, *bnx, *bny;              /* positions, normals   */
} orc_state;

typedef struct {
    double *ax, *ay, *drho;         /* du/dt (Eq. 25), drho/dt (Eq. 7)       */
    double *C, *nx, *ny, *kappa;    /* colour, normal, curvature (CSF)       */
    unsigned char *Nflag;           /* filter N_a, Eq. 20                    */
    double *dt_f, *dt_cv;           /* per-particle Eq. 30 and Eq. 31 terms  */
} orc_out;

/* Kernel functions (Sec. 2-5). */
double orc_kernel_norm(int kernel);
double orc_W(int kernel, double r, double h);
double orc_dWdr(int kernel, double r, double h);

/* Tait equation of state (Eq. 26) and the sound speed c = sqrt(dP/drho). */
double orc_pressure(double rho, double rho0, double c0, double gamma);
double orc_sound_speed(double rho, double rho0, double c0, double gamma);

/* Neighbour lists: all ordered pairs (a, b), a != b, with
 * (x_a-x_b)^2 + (y_a-y_b)^2 < radius^2, each list ascending in b.
 * Only particles with active[a] != 0 take part.  Returns total pair count,
 * or -1 on allocation failure.  *start has n+1 entries, *list the pairs;
 * free both with orc_free. */
long long orc_neighbours(long long n, const double *x, const double *y,
                         const unsigned char *active, double radius,
                         int use_cells, long long **start, int **list);
void orc_free(void *p);

/* Threads of the particle loops when built with OpenMP (default 1).  Each
 * particle's sums keep their order, so results do not depend on it.
 * orc_max_threads() is the host's OpenMP thread count (1 without OpenMP). */
void orc_set_threads(int n);
int orc_max_threads(void);

/* One evaluation of the right-hand sides at a given state (Sec. 2-2 to 2-8).
 * Returns 0 on success, -1 on allocation failure. */
int orc_evaluate(const orc_params *p, const orc_state *s, orc_out *o);

/* Summation density (Eq. 6): rho_a = sum_b m_b W_ab over the fluid and buffer
 * particles within 2h, the particle itself included.  Returns 0 on success,
 * -1 on allocation failure. */
int orc_summation_density(const orc_params *p, const orc_state *s, double *rho);

/* Connected components of the graph with edges r_ab < radius among the
 * n particles (Sec. 3-2 breakup criterion).  label[a] = smallest index in
 * a's component.  Returns the number of components or -1. */
long long orc_components(long long n, const double *x, const double *y,
                         double radius, int use_cells, long long *label);

#ifdef __cplusplus
}
#endif
#endif
