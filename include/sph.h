/*
 * sph.h -- C ABI of libsph, a GB300 (sm_103a) implementation of the per-step
 * particle-interaction sweep of the 2D weakly-compressible SPH method for
 * liquid-jet breakup of Pourabdian, Omidvar & Morad (arXiv 1603.02421).
 *
 * One step (Sec. 2-8) is: cell-linked-list neighbour build (Sec. 2-7), two
 * evaluations of the semi-discrete equations -- colour (Eq. 14), surface
 * normal (Eqs. 18, 20, 21), curvature (Eq. 23), continuity (Eq. 7), momentum
 * with Tait pressure, artificial viscosity and CSF surface tension (Eqs. 9,
 * 10, 24, 25, 26) and repulsive walls (Eq. 29) -- with the predictor-corrector
 * update in between, the adaptive time step of Eqs. 30-32, and inflow /
 * outflow of the planar jet.  The breakup length follows the criterion of
 * Sec. 3-2.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an sph_status; nothing throws across the ABI.
 *  - Pointer arguments are HOST pointers.  Inputs are copied by the library
 *    (the caller keeps ownership); outputs are caller-allocated host buffers
 *    of the stated length.
 *  - The context owns all device memory it allocates (sph_init) and frees it
 *    in sph_destroy.  Work is issued on params.cuda_stream (a cudaStream_t,
 *    or NULL for a stream the library creates).  Calls that return host data
 *    synchronise that stream.
 *  - Particle ids: fluid and buffer particles get consecutive ids in the
 *    order they are added; particles laid by the inflow get the next ids.
 *    Boundary particles carry no id.  State queries return particles sorted
 *    by id.
 *  - On error the function returns a negative status and sph_last_error()
 *    describes it.  A failed call leaves the particle state as it was,
 *    except SPH_ERR_NONFINITE / SPH_ERR_SKIN / SPH_ERR_CAPACITY raised during
 *    a step, after which the state is that of the completed step and should
 *    be treated as suspect.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef SPH_H
#define SPH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_ERR_ARG = -1,        /* invalid argument or parameter                */
    SPH_ERR_OOM = -2,        /* device allocation failed                     */
    SPH_ERR_CAPACITY = -3,   /* particle capacity, neighbour-list capacity or
                                output buffer too small                      */
    SPH_ERR_CUDA = -4,       /* CUDA runtime / launch error                  */
    SPH_ERR_NONFINITE = -5,  /* NaN / Inf in an acceleration or density rate */
    SPH_ERR_TIMEOUT = -6,    /* a bounded device loop hit its limit          */
    SPH_ERR_STATE = -7,      /* call not valid in the current state; in the
                                bounds-check build (SPH_BOUNDS_CHECK) also a
                                particle index out of range                  */
    SPH_ERR_SKIN = -8        /* a particle moved more than skin/2 between the
                                cell build and an evaluation (reduce dt or
                                raise skin_over_h)                           */
} sph_status;

typedef enum { SPH_KERNEL_CUBIC = 0, SPH_KERNEL_WENDLAND = 1 } sph_kernel;
typedef enum { SPH_FP32 = 0, SPH_FP64 = 1 } sph_precision;
/* Density of the fluid particles: integrated continuity equation (Eq. 7, the
 * paper's choice) or the summation of Eq. 6 at each evaluation. */
typedef enum { SPH_DENSITY_CONTINUITY = 0, SPH_DENSITY_SUMMATION = 1 } sph_density;
enum { SPH_FLUID = 0, SPH_BOUNDARY = 1, SPH_BUFFER = 2 };

/* Run parameters (all SI or consistently nondimensional). */
typedef struct {
    int kernel;            /* sph_kernel: cubic spline Eq. 27, Wendland C2 Eq. 28
                              (2D unit-integral normalisation 10/(7 pi), 7/(64 pi)) */
    int precision;         /* sph_precision of the pair sums; positions and time are
                              always FP64                                           */
    double dx;             /* initial particle spacing                              */
    double h_over_dx;      /* h = h_over_dx * dx (the paper uses 1.3, Sec. 2-2)      */
    double rho0, c0, gamma;/* Tait EOS Eq. 26, B = rho0 c0^2 / gamma                */
    double alpha;          /* artificial viscosity coefficient, Eq. 10              */
    double eta2_over_h2;   /* eta^2 / h^2 in Eq. 10 (0.01)                          */
    double sigma;          /* surface tension coefficient, Eq. 24 (0: CSF off)      */
    double eps_n_times_h;  /* normal filter eps * h in Eq. 20 (0.01)                */
    double gx, gy;         /* gravity, Eq. 25                                       */
    double courant;        /* Cr of Eq. 32 (0.2)                                    */
    double dt_fixed;       /* > 0: fixed step; 0: adaptive Eqs. 30-32               */
    double xmin, ymin, xmax, ymax;  /* domain box; fluid leaving it is deleted      */
    double skin_over_h;    /* cell size = 2h + skin, skin = skin_over_h * h (>= 0.1) */
    double wall_A_coef;    /* wall force strength A = wall_A_coef * c0^2 / h, Eq. 29 */
    double wall_h0;        /* still-water depth of the eps(z) factor (0: eps(z) = 1) */
    double wall_db_over_dx;/* boundary particle spacing db = wall_db_over_dx * dx   */
    double u_frame_x, u_frame_y; /* reference velocity: velocities are stored as
                              u - u_frame (the equations are Galilean invariant, so
                              any value gives the same results to rounding; the
                              stream velocity of a jet keeps its small velocity
                              differences accurate in FP32)                      */
    long long capacity;    /* maximum fluid + buffer particles held at once (<= 2^28) */
    long long boundary_capacity; /* maximum boundary particles                      */
    void *cuda_stream;     /* cudaStream_t to issue work on, or NULL                */
    int device;            /* CUDA device ordinal                                   */
    int density;           /* sph_density.  With SPH_DENSITY_SUMMATION each
                              evaluation takes the fluid density from Eq. 6 at its
                              positions (buffer particles keep theirs); the state's
                              density is that of the step's last evaluation (the
                              half step), and sph_evaluate stores the density it
                              used.  FP32 and FP64 contexts; not with
                              sph_surrogate_step.                               */
} sph_params;

/* Create a context: validates *params, selects the device, allocates all
 * device buffers for params->capacity particles.  *out receives the
 * context, or NULL on failure (then sph_last_error(NULL) has the reason). */
sph_status sph_init(const sph_params *params, sph_ctx **out);

/* Release every device buffer and the library-created stream. NULL is ignored. */
void sph_destroy(sph_ctx *ctx);

/* Last error message of ctx (or of the last failed sph_init when ctx is NULL). */
const char *sph_last_error(const sph_ctx *ctx);

/* Append n particles (Sec. 2-2: each carries m, rho, u, r).  Arrays of length
 * n: x, y (positions), u, v (velocity), rho (density), mass, type (SPH_FLUID,
 * SPH_BOUNDARY or SPH_BUFFER).  nx, ny are the unit wall normals of boundary
 * particles (pointing into the fluid, Eq. 29) and may be NULL when no
 * boundary particle is added.  Fluid and buffer particles must lie inside the
 * domain box.  Returns SPH_ERR_CAPACITY if a capacity would be exceeded. */
sph_status sph_add_particles(sph_ctx *ctx, long long n, const double *x, const double *y,
                             const double *u, const double *v, const double *rho,
                             const double *mass, const unsigned char *type,
                             const double *nx, const double *ny);

/* Configure the planar-jet inflow (the paper's tank/nozzle is replaced by an
 * inflow buffer, Sec. 3-2): `layers` layers of buffer particles at spacing dx
 * across [y0, y1], laid at x_exit - (j + 0.5) dx (j = 0..layers-1), moving with
 * u_in(t) = U (1 + amp sin(k U t + phase)), rho = rho0, mass rho0 dx^2.  A
 * buffer particle becomes fluid when x >= x_exit; a new layer is laid one
 * spacing upstream whenever the upstream-most layer passes its initial slot.
 * At most 1024 particles per layer.  May be called once per context. */
sph_status sph_inflow(sph_ctx *ctx, double x_exit, double y0, double y1, double U,
                      double amp, double k, double phase, int layers);

/* Advance one time step (Sec. 2-8).  *dt_used (nullable) receives the step
 * size.  Synchronises the stream. */
sph_status sph_step(sph_ctx *ctx, double *dt_used);

/* Advance nsteps steps by replaying a CUDA graph of one step.  When
 * breakup_every > 0, after every breakup_every steps the breakup length
 * (L/D, see sph_breakup_length) is appended to L_out (capacity
 * nsteps / breakup_every entries) and *nL receives the count; L_out and nL
 * may be NULL when breakup_every <= 0. */
sph_status sph_run(sph_ctx *ctx, long long nsteps, int breakup_every, double D,
                   double *L_out, long long *nL);

/* Breakup length of the jet (Sec. 3-2): particles closer than 1.5 h are
 * linked; the jet is the union of connected components holding an inflow
 * buffer particle; *L_over_D = (max x over the jet - x_exit) / D.  *broken
 * (nullable) is set to 1 if some fluid particle lies outside the jet.
 * Requires sph_inflow. */
sph_status sph_breakup_length(sph_ctx *ctx, double D, double *L_over_D, int *broken);

/* One evaluation of the right-hand sides at the current state, without
 * advancing it (for inspection and tests).  Afterwards sph_get_state's ax,
 * ay, drho and sph_get_csf return this evaluation. */
sph_status sph_evaluate(sph_ctx *ctx);

/* Copy out the fluid + buffer state, sorted by id.  cap = length of every
 * output array; *n receives the particle count (SPH_ERR_CAPACITY if > cap;
 * such a call, e.g. cap = 0 to ask for the count, downloads only the
 * particle types).  rho is the density; ax, ay, drho the derivatives du/dt
 * (Eq. 25) and drho/dt (Eq. 7) of the last evaluation at the start of a step
 * (or of sph_evaluate), zero for particles laid since.  Any output pointer
 * except n may be NULL.  State transfers (this call, sph_set_state,
 * sph_add_particles) go through a pinned host buffer of the context, about
 * 49 (FP32) or 77 (FP64) bytes per particle of capacity, allocated on first
 * use and freed by sph_destroy. */
sph_status sph_get_state(sph_ctx *ctx, long long cap, long long *n, double *x, double *y,
                         double *u, double *v, double *rho, double *mass,
                         unsigned char *type, unsigned *id, double *ax, double *ay,
                         double *drho);

/* Replace the fluid + buffer state by n particles with the given ids (e.g.
 * a checkpoint taken with sph_get_state).  Boundary particles, inflow, time
 * and step count are kept. */
sph_status sph_set_state(sph_ctx *ctx, long long n, const double *x, const double *y,
                         const double *u, const double *v, const double *rho,
                         const double *mass, const unsigned char *type,
                         const unsigned *id);

/* CSF intermediates of the last sph_evaluate, sorted by id: colour C (Eq. 14)
 * and normal n (Eq. 18).  Zero when sigma = 0. */
sph_status sph_get_csf(sph_ctx *ctx, long long cap, long long *n, unsigned *id,
                       double *C, double *nx, double *ny);

/* All ordered neighbour pairs (id_a, id_b), a != b, at distance < 2h
 * (Sec. 2-7), from the cell build at the current state; order unspecified.
 * *npairs receives the count (SPH_ERR_CAPACITY if > cap). */
sph_status sph_get_pairs(sph_ctx *ctx, long long cap, unsigned *id_a, unsigned *id_b,
                         long long *npairs);

/* Checkpoint and resume (no counterpart in the paper; SPHysics writes
 * output frames).  A checkpoint holds what a later run needs to continue
 * bit for bit: the live fluid and buffer particles in id order exactly as
 * the context stores them (FP64 positions; velocities, density offsets
 * rho - rho0 with their compensation carries and masses in the pair
 * precision), the simulated time, step count, inflow layer position, next
 * particle id and deleted count.  sph_checkpoint_size: the bytes a save
 * writes now.  sph_checkpoint_save: writes them to the host buffer buf of
 * cap bytes (*bytes, nullable, receives the count; SPH_ERR_CAPACITY if cap
 * is short).  sph_checkpoint_load: replaces the particles and clocks of ctx
 * -- a context made with the same parameters, boundary and inflow, which
 * keeps them -- by those of the checkpoint (SPH_ERR_ARG for a buffer that
 * is not one, of the other pair precision, or beyond the capacity).  The
 * next step of the loaded context rebuilds its cells and lists; its state
 * after k steps is bit for bit that of the saved context after k steps of
 * its own when that context also rebuilds at the first of them
 * (sph_request_rebuild), with the same tuning: the cell order after a
 * rebuild depends only on the positions and ids. */
sph_status sph_checkpoint_size(sph_ctx *ctx, size_t *bytes);
sph_status sph_checkpoint_save(sph_ctx *ctx, void *buf, size_t cap, size_t *bytes);
sph_status sph_checkpoint_load(sph_ctx *ctx, const void *buf, size_t bytes);

/* Run statistics of the current state (no counterpart in the paper): over
 * the fluid particles, their mass, momentum sum m u, kinetic energy
 * sum m |u|^2 / 2, potential energy -sum m g . r, the elastic energy of the
 * Tait equation of state (Eq. 26), sum m e(rho) with
 * e = (B/rho0) ((x^(gamma-1) - 1)/(gamma - 1) + 1/x - 1), x = rho/rho0 (the
 * work P/rho^2 d rho stored from rho0 to rho), and max |rho - rho0|/rho0;
 * counts of fluid, buffer and boundary particles; time, step, last step size
 * and deleted count.  Sums in FP64 on the device. */
typedef struct {
    long long n_fluid, n_buffer, n_boundary, n_deleted, step;
    double t, dt;
    double mass, momentum_x, momentum_y;
    double kinetic, potential, elastic;
    double max_rel_density;
} sph_stats_t;
sph_status sph_stats(sph_ctx *ctx, sph_stats_t *out);

/* Simulated time, completed steps, live fluid + buffer particles, and
 * particles deleted by the outflow so far. */
sph_status sph_get_time(sph_ctx *ctx, double *t, long long *steps, long long *n_particles,
                        long long *n_deleted);

/* Enqueue nsteps steps (CUDA-graph replay) on the context's stream and return
 * without waiting.  Device-side errors surface at the next synchronising call
 * (sph_sync, sph_step, sph_get_*). */
sph_status sph_run_async(sph_ctx *ctx, long long nsteps);

/* Wait for all work enqueued on the context's stream and report device-side
 * errors of the steps it ran. */
sph_status sph_sync(sph_ctx *ctx);

/* Per-kernel timing.  enable = 1 records a CUDA event before each kernel
 * group of every later step (the step graph is re-captured with the events);
 * each synchronising call then adds the durations of the most recent step to
 * running totals, which enable (0 or 1) resets. */
sph_status sph_profile(sph_ctx *ctx, int enable);

/* Totals per kernel group: names[k] (library-owned strings, valid until the
 * next sph_profile_report), total_ms[k], launches[k]; *n receives the number
 * of groups (SPH_ERR_CAPACITY if > cap).  Output arrays may be NULL. */
sph_status sph_profile_report(sph_ctx *ctx, int cap, int *n, const char **names,
                              double *total_ms, long long *launches);

/* Tuning of the step.  lanes (1, 2, 4 or 8): threads that share one particle's
 * neighbour loop in the pair sweeps (the neighbour-list build uses at least
 * 4).  cadence (1..64): the cells and neighbour lists are rebuilt at least
 * every `cadence` steps, and earlier when the step before spawned an inflow
 * layer or when one more step could move a particle more than skin/2 from
 * where the lists were built (decided on the device); also after the
 * particles were added, replaced or reordered by another call.  Without
 * walls the displacement is taken relative to the velocity frame
 * (u_frame_x, u_frame_y): a common translation changes no pair separation,
 * so a jet moving at the frame velocity keeps its lists; particles may then
 * move up to two cells from their build-time cell.  With walls it is the
 * absolute displacement (wall contacts are found by walking the build-time
 * cells).  The steps in between keep the last build, which stays exact
 * (checked: SPH_ERR_SKIN otherwise).  Defaults: lanes 4, cadence 1 (every
 * step). */
sph_status sph_set_tuning(sph_ctx *ctx, int lanes, int cadence);
sph_status sph_get_tuning(sph_ctx *ctx, int *lanes, int *cadence);

/* How a step at cadence > 1 picks its start -- rebuild the cells and lists,
 * or refresh the records on the last build -- on the device, from the flag
 * the step before left, with nothing returned to the host in between.  Both
 * forms launch the same kernels on the same data, so results are identical:
 *   SPH_START_GATED        the step graph holds both starts in one line; each
 *                          start kernel returns at once when its start is not
 *                          the one taken (every kernel of both starts is
 *                          launched, each skipped one costing about 1 us and
 *                          a pass over its blocks);
 *   SPH_START_CONDITIONAL  a one-thread kernel sets a CUDA-graph IF node that
 *                          runs only the taken start (about 10 us per step for
 *                          the node, whatever the particle count).
 * The gated form is faster for one context of up to a few 1e5 particles, the
 * conditional one for large contexts and many-member ensembles, whose graphs
 * are bound by the number of launches; sph_autotune and
 * sph_ensemble_autotune time both.  Default: SPH_START_GATED. */
typedef enum { SPH_START_GATED = 0, SPH_START_CONDITIONAL = 1 } sph_start_form;
sph_status sph_set_start_form(sph_ctx *ctx, int form);
sph_status sph_get_start_form(sph_ctx *ctx, int *form);

/* Autotuner: from a copy of the current state, times each lanes in {1, 2, 4,
 * 8} with cadence in {1, 2, 4, 8}, then cadence 16 and 32 at the best lanes
 * (at cadence > 1 in both start forms), each over max(trial_steps,
 * 2 x cadence) steps after a warm cycle, rejecting settings that trip
 * SPH_ERR_SKIN; restores the state and keeps the fastest setting.  Outputs
 * (nullable): the chosen lanes, cadence and its ms per step;
 * sph_get_start_form gives the form. */
sph_status sph_autotune(sph_ctx *ctx, int trial_steps, int *lanes, int *cadence,
                        double *ms_per_step);

/* Cell builds so far (cell sorts run by steps and by the calls that sort:
 * evaluate, pairs, breakup length), and the rebuild decision taken at the end
 * of the last step: the largest displacement of a particle since the last
 * build and the largest move in that step (both in length units, FP32;
 * relative to the velocity frame when there are no walls, see
 * sph_set_tuning).  Any pointer may be NULL. */
sph_status sph_get_rebuild_stats(sph_ctx *ctx, long long *builds, double *disp_max,
                                 double *step_max);

/* The next step rebuilds the cells and neighbour lists (Sec. 2-7) whatever
 * the cadence and the device's displacement test decide; the steps after it
 * follow them again.  Results do not change (every build is exact); this
 * only places a rebuild, e.g. at the start of a timed window. */
sph_status sph_request_rebuild(sph_ctx *ctx);

/* Number of device kernels (memsets excluded) launched at the current
 * settings by a step that rebuilds the cells and lists, by a step that reuses
 * the last build, and by one breakup-length evaluation.  At cadence 1 every
 * step rebuilds.  At cadence > 1 in the gated start form every step launches
 * the kernels of both starts (those of the start not taken return at once),
 * so the two step counts are equal; in the conditional form each step also
 * runs the one-thread kernel that sets the IF node.  Any pointer may be
 * NULL. */
sph_status sph_kernel_counts(sph_ctx *ctx, int *per_full_step, int *per_reused_step,
                             int *per_breakup);

/* Neighbour pairs without any device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc --
 * code running inside another framework's memory pool (whose allocator owns
 * the device memory), an application that must not grow its device footprint
 * after start-up, or a plugin that only receives device buffers from its
 * host.
 *
 * x, y: DEVICE arrays of n FP64 positions, all inside the box
 * [xmin, xmax) x [ymin, ymax).  Finds every ordered pair (a, b), a != b, with
 * |r_a - r_b| < 2h (Sec. 2-7), exactly as sph_get_pairs does, and writes the
 * input indices a, b to the DEVICE arrays pair_a, pair_b (cap entries each,
 * order unspecified); *npairs (host) receives the total count (a 64-bit
 * count, whatever the density of the input).  Work runs on `stream` (a
 * cudaStream_t, NULL = legacy default stream) of the current device; the call
 * waits for it and copies the count to the host, so it cannot be part of a
 * stream capture: on a stream being captured it returns SPH_ERR_ARG before
 * enqueuing anything.
 *
 * Errors decided on the device still report the pairs found: particles
 * outside the box or with a NaN coordinate are left out of the search and
 * the call returns SPH_ERR_ARG with the pairs of the others written and
 * counted; a count above cap returns SPH_ERR_CAPACITY with the first cap
 * pairs written and *npairs the full count.
 *
 * Limits: n <= 262144 particles and a search grid of at most 1048576 cells of
 * size 2.1 h over the box (SPH_ERR_CAPACITY beyond).  The scratch is one
 * static device array of about 31 MB that every GPU loading the library holds
 * until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress), so make the first call on each
 * device before any stream capture.  The address is kept for the life of the
 * process, so a device reset (cudaDeviceReset) leaves it stale: do not call
 * this entry point on a device after resetting it.  All calls share the
 * array: calls whose work overlaps on the GPU (other host threads, other
 * streams) race and must be serialised by the caller. */
sph_status sph_pairs_noalloc(const double *x, const double *y, long long n, double h,
                             double xmin, double ymin, double xmax, double ymax,
                             unsigned *pair_a, unsigned *pair_b, long long cap,
                             long long *npairs, void *stream);

/* Arithmetic peak of `device` (no counterpart in the paper): the fused
 * multiply-add rate of the SIMT pipes in `precision` (SPH_FP32 or SPH_FP64),
 * the bound of the pair sweeps, which are FP32 (or FP64) arithmetic on
 * irregular neighbour sets rather than dense contractions.  Every SM is
 * filled with threads running 8 independent FMA chains each; *tflops
 * receives 2 x FMAs / time of the best of 5 launches timed with CUDA events,
 * *ms that launch's duration (both nullable).  Runs at whatever clocks the
 * device is at; changes no device setting.  Allocates a small output buffer. */
sph_status sph_fma_peak(int device, int precision, double *tflops, double *ms);

/* ------------------------------------------------------------------------
 * Ensembles: several independent simulations (e.g. jets on a grid of Re and
 * We, Table 1, with different dx and particle counts) advanced together.
 * One ensemble step is one step of every member, each with its own time
 * step; the members' steps are the branches of one CUDA graph, so one graph
 * launch runs all of them and the GPU overlaps the kernels of different
 * members.  Each member computes exactly what sph_run computes for it alone.
 * ------------------------------------------------------------------------ */
typedef struct sph_ensemble sph_ensemble;

/* Groups n >= 1 distinct contexts of one device.  The ensemble keeps the
 * pointers (the contexts stay owned by the caller and must outlive it) and
 * works on cuda_stream (a cudaStream_t; NULL creates a stream of its own).
 * Work enqueued on the members' streams before an ensemble run completes
 * before it, and later work on them waits for it.  On error *out is NULL and
 * sph_ensemble_last_error(NULL) describes it. */
sph_status sph_ensemble_create(sph_ctx *const *members, int n, void *cuda_stream,
                               sph_ensemble **out);

/* Enqueue nsteps ensemble steps and return without waiting.  The graph is
 * re-captured when a member's parameters or tuning changed since the last
 * run. */
sph_status sph_ensemble_run(sph_ensemble *e, long long nsteps);

/* Wait for the enqueued steps and report the first member whose steps
 * raised a device-side error (*bad_member = its index, else -1; nullable);
 * the member's own sph_last_error holds the description. */
sph_status sph_ensemble_sync(sph_ensemble *e, int *bad_member);

/* Autotuner over one (lanes, cadence, start form) for all members, with the
 * candidates and trial lengths of sph_autotune, timed as ensemble steps from
 * copies of the members' states (rejecting settings that trip
 * SPH_ERR_SKIN); restores the states and keeps the fastest setting.  Outputs
 * nullable. */
sph_status sph_ensemble_autotune(sph_ensemble *e, int trial_steps, int *lanes, int *cadence,
                                 double *ms_per_step);

/* Waits for the ensemble's work and frees it (not the members). */
void sph_ensemble_destroy(sph_ensemble *e);

/* Description of the last error of an ensemble call (e = NULL: of the last
 * failed sph_ensemble_create). */
const char *sph_ensemble_last_error(const sph_ensemble *e);

/* ------------------------------------------------------------------------
 * Learned surrogate (no counterpart in the paper): a message-passing network
 * on the SPH neighbour graph that predicts each particle's mean acceleration
 * over the next k substeps.  Definition (all sums over ordered pairs a != b
 * with r_ab < 2h of the context's last evaluation, Sec. 2-7):
 *   node inputs  x_a = [100 (rho_a/rho0 - 1), N_a (Eq. 20), C_a (Eq. 14),
 *                       h |n_a| (Eq. 18)]
 *   edge weights V_b = m_b/rho_b, W and F = (1/r) dW/dr of Eqs. 27-28:
 *                w0 = V_b W_ab, w1 = V_b F_ab (x_a - x_b) h,
 *                w2 = V_b F_ab (y_a - y_b) h,
 *                w3 = V_b F_ab ((u_a - u_b).(r_a - r_b)) h / u_ref
 *   layers       h0 = relu(x W_in + b_in); for l = 0, 1, 2: z = h Pi_l
 *                (128 -> 32), g_a[32k + j] = sum_b w_k,ab z_b[j],
 *                h = h + relu([h, g] U_l + c_l) (256 -> 128); y = h D + d.
 *   loss         L = (1/N) sum_a |y_a - t_a|^2.
 * Parameters are packed float32 in the order W_in (4x128), b_in (128), then
 * per layer Pi_l (128x32), U_l (256x128), c_l (128), then D (128x2), d (2);
 * matrices row-major (fan-in x fan-out).  Every call works on a context that
 * sph_evaluate left on its current state (SPH_ERR_STATE otherwise), FP32
 * contexts only, on the context's stream; particles are in the context's
 * cell order, reported with their ids.
 * ------------------------------------------------------------------------ */
typedef struct sph_mpnn sph_mpnn;

/* Number of packed parameters. */
long long sph_mpnn_param_count(void);

/* A network for up to `capacity` particles on `device` (parameters zero;
 * set them with sph_mpnn_set_params).  On error *out is NULL and
 * sph_mpnn_last_error(NULL) describes it. */
sph_status sph_mpnn_create(int device, long long capacity, sph_mpnn **out);
void sph_mpnn_destroy(sph_mpnn *net);
const char *sph_mpnn_last_error(const sph_mpnn *net);

/* Host copies of the packed parameters / of the gradients of the last
 * sph_mpnn_backward (n must equal sph_mpnn_param_count()).  Setting the
 * parameters resets the optimiser state. */
sph_status sph_mpnn_set_params(sph_mpnn *net, const float *host, long long n);
sph_status sph_mpnn_get_params(sph_mpnn *net, float *host, long long n);
sph_status sph_mpnn_get_grads(sph_mpnn *net, float *host, long long n);

/* The network's inputs for inspection: *n particles (ids to id[], x to
 * x[4n]) and *ne ordered pairs (cell-order indices ea, eb; weights w[4 ne]);
 * SPH_ERR_CAPACITY if cap or ecap is too small (the counts are still set). */
sph_status sph_mpnn_features(sph_mpnn *net, sph_ctx *ctx, double u_ref, long long cap,
                             long long *n, unsigned *id, float *x, long long ecap,
                             long long *ne, int *ea, int *eb, float *w);

/* Forward pass: y[2n] for the *n particles (ids to id[]).  bf16 != 0 runs
 * the tensor-core inference pass: tcgen05.mma with BF16 operands and FP32
 * accumulation for the dense layers, BF16 hidden state and messages, FP16
 * edge weights, FP32 message sums; otherwise everything is FP32.  A bounded
 * wait of the tensor-core pass that ran out returns SPH_ERR_TIMEOUT. */
sph_status sph_mpnn_forward(sph_mpnn *net, sph_ctx *ctx, double u_ref, int bf16, long long cap,
                            long long *n, unsigned *id, float *y);

/* FP32 forward and backward pass against host targets t[2n] (cell order, as
 * reported by sph_mpnn_forward): the loss to *loss (nullable) and the
 * gradients kept for sph_mpnn_get_grads / sph_mpnn_adam. */
sph_status sph_mpnn_backward(sph_mpnn *net, sph_ctx *ctx, double u_ref, const float *target,
                             long long n, double *loss);

/* One Adam update (beta 0.9 / 0.999, eps 1e-8) from the last gradients. */
sph_status sph_mpnn_adam(sph_mpnn *net, double lr);

/* Test hook for the bounded waits of the tensor-core inference pass: with
 * on != 0 the following passes issue no operand loads, so every mbarrier
 * wait of the layer kernels runs out (after about a second each), the
 * kernels record ERR_TIMEOUT in the context's error word, free their tensor
 * memory and return; sph_mpnn_forward and sph_surrogate_step then report
 * SPH_ERR_TIMEOUT (the context keeps the error: make a new one).  No GPU
 * fault or hang is involved.  on = 0 restores normal passes. */
sph_status sph_mpnn_inject_stall(sph_mpnn *net, int on);

/* One surrogate step of length dT = k dt (dt from Eq. 32 at the current
 * state, or dt_fixed), with plain SPH as judge and fallback:
 *   1. evaluate SPH at the current state (a_n, drho/dt_n) -- or take the
 *      evaluation that ended the previous accepted surrogate step, when no
 *      call has changed the state since and its time advance kept the lists;
 *   2. predict the mean acceleration over the k substeps as abar = a_n +
 *      a_ref (y - ybar), y the network's output (bf16 != 0: tensor cores)
 *      and ybar its mass-weighted mean over the fluid: the correction moves
 *      momentum between particles but adds none (the pair forces that make
 *      up most of it cancel in the sum, Eqs. 9-10);
 *   3. fluid: u' = u + dT abar, r' = r + dT (u + u')/2, rho' = rho + dT
 *      drho/dt_n; inflow buffer, buffer -> fluid and outflow as in a plain
 *      step; inflow layers, time advance for dT and the device's rebuild
 *      decision (cadence counted in surrogate steps, displacements);
 *   4. evaluate SPH at the new state (same cell order and lists) and form,
 *      over the particles fluid at both ends, the momentum balance residual
 *      r_m = |sum m (abar - (a_n + a_k)/2)| / sum m |(a_n + a_k)/2| (the
 *      step's momentum change against the trapezoidal impulse of the SPH
 *      forces at its ends), the density residual
 *      r_rho = (dT/2) rms(drho/dt_k - drho/dt_n) / rho0, and, reported only,
 *      the acceleration-field residual r_a = |abar - (a_n + a_k)/2| /
 *      |(a_n + a_k)/2| (L2), which the step-to-step acoustic noise of the
 *      accelerations keeps near 0.1 even for plain SPH's exact k-step mean;
 *   5. accept when r_m and r_rho are <= threshold; otherwise restore the
 *      state and run k plain steps instead (also when a particle moved more
 *      than skin/2, so the lists of the start no longer hold).
 * *accepted (nullable) says which; the residuals go to res_momentum,
 * res_density and res_field (nullable).  FP32 contexts only. */
sph_status sph_surrogate_step(sph_ctx *ctx, sph_mpnn *net, int k, double u_ref, double a_ref,
                              double threshold, int bf16, int *accepted, double *res_momentum,
                              double *res_density, double *res_field);

/* sph_surrogate_step on m contexts at once (an ensemble of jets): every
 * context's work is enqueued on its own stream before the host waits, so the
 * batch pays one round of host synchronisations (two when some context
 * cannot reuse its last evaluation), not m.  accepted, res_momentum,
 * res_density and res_field are arrays of m (each nullable); the contexts
 * may share a stream; all use the one network (read-only here).  On an
 * error *bad_member (nullable) names the context that failed.  Argument
 * errors (a NULL network, an FP64 context, summation density, k or the
 * scalars out of range) are found before any context is touched; after a
 * later error the contexts' steps may be incomplete: call sph_sync on each
 * before using them. */
sph_status sph_surrogate_batch(sph_ctx *const *ctx, int m, sph_mpnn *net, int k, double u_ref,
                               double a_ref, double threshold, int bf16, int *accepted,
                               double *res_momentum, double *res_density, double *res_field,
                               int *bad_member);

/* One surrogate step of every member (the ensemble's batched surrogate
 * form): waits for the enqueued ensemble steps, then sph_surrogate_batch over
 * the members in order (arrays of the member count, nullable); plain
 * ensemble steps after it rebuild the members' lists first.  Errors as
 * sph_surrogate_batch, *bad_member naming the member. */
sph_status sph_ensemble_surrogate_step(sph_ensemble *e, sph_mpnn *net, int k, double u_ref,
                                       double a_ref, double threshold, int bf16, int *accepted,
                                       double *res_momentum, double *res_density,
                                       double *res_field, int *bad_member);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
