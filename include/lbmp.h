/*
 * lbmp — GB300-native time step of the generalized lattice Boltzmann model
 * for flow through tight porous media with Klinkenberg's effect
 * (Chen, Fang, Kang, Hyman, Viswanathan, Tao, arXiv:1411.7051).
 *
 * C ABI.  Plain pointers and sizes; no C++ or framework types cross it.
 * Every entry point returns an lbmp_status; no exception escapes.  On an
 * error the thread-local message of lbmp_last_error() says what failed.
 *
 * Model (Section III): D2Q9 (Eq. 13), BGK evolution (Eq. 12) with the
 * porosity-weighted equilibrium (Eq. 14), Guo's forcing term (Eq. 15, last
 * term taken over eps so that sum_i F_i = 0), density and velocity from
 * Eq. 16-17 (the quadratic form when the Forchheimer drag of Eq. 2 is kept),
 * total force Eq. 2 / Eq. 8, and the apparent permeability k_a = k_i f_c(Kn)
 * of Eq. 3 with the Beskok-Karniadakis-Civan factor of Eq. 6-7 (b = -1).
 * Lattice units: dt = dx = 1, c = 1, c_s^2 = 1/3, nu_e = (tau - 1/2)/3,
 * nu = nu_e / J.
 *
 * Array conventions: node fields are row-major [ny][nx] (x fastest) float64;
 * populations are plane-major [9][ny][nx] float64 in the order of Eq. 13:
 * e_0 = (0,0), e_1..e_4 = (1,0), (0,1), (-1,0), (0,-1),
 * e_5..e_8 = (1,1), (-1,1), (-1,-1), (1,-1).
 * The caller owns every pointer it passes; the library copies what it needs
 * and owns every device buffer it allocates.  `where` says whether a caller
 * pointer is host (LBMP_HOST) or device (LBMP_DEVICE) memory of the
 * context's GPU.
 */
#ifndef LBMP_H
#define LBMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lbmp_status;
#define LBMP_OK 0
#define LBMP_EINVAL 1   /* invalid argument or field value */
#define LBMP_ENOMEM 2   /* device or host allocation failed */
#define LBMP_ECUDA 3    /* a CUDA call failed (no device, launch error ...) */
#define LBMP_ESTATE 4   /* call out of order (e.g. step before set_fields) */
#define LBMP_ENAN 5     /* a reduction met a non-finite velocity or density */
#define LBMP_ETIMEOUT 6 /* a bounded device wait gave up (staged kernel); the
                           state of the context is then undefined */

/* boundary kinds */
#define LBMP_BCX_PERIODIC 0
#define LBMP_BCX_PRESSURE 1 /* density imposed at x = 0 and x = nx-1 */
#define LBMP_BCY_PERIODIC 0
#define LBMP_BCY_WALLS 1 /* rows 0 and ny-1 are solid plates */

/* population storage in device memory (arithmetic is FP32 in both) */
#define LBMP_STORE_FP32 0 /* f_i - w_i rho0 as float */
#define LBMP_STORE_FP16 1 /* (f_i - w_i rho0) * S as IEEE half, S = 2^s.  With
                             stochastic rounding (default) the random offsets
                             are a hash of (seed, time level, node), so runs
                             and checkpoint restarts are reproducible. */

/* rounding of FP16 stores */
#define LBMP_ROUND_STOCHASTIC 0 /* unbiased in expectation (default) */
#define LBMP_ROUND_NEAREST 1    /* round to nearest even */

/* step kernel */
#define LBMP_KERNEL_AUTO 0   /* the faster one measured on GB300: direct for FP32
                                storage, staged for FP16 */
#define LBMP_KERNEL_STAGED 1 /* bulk copies into a shared-memory ring (persistent) */
#define LBMP_KERNEL_DIRECT 2 /* one-pass loads from global memory */
#define LBMP_KERNEL_WIDE 3   /* FP16 storage only: four consecutive nodes per thread,
                                8-byte loads and stores per plane */

#define LBMP_HOST 0
#define LBMP_DEVICE 1

/* correction factor f_c of Eq. 3 */
#define LBMP_KN_BKC 0         /* Beskok-Karniadakis-Civan, Eq. 6-7 (b = -1): the paper's */
#define LBMP_KN_FIRST_ORDER 1 /* Klinkenberg's first-order Eq. 4-5: f_c = 1 + 4 Kn (c = 1) */

typedef struct lbmp_params {
  int32_t nx, ny;       /* lattice size; nx, ny >= 1 */
  double tau;           /* relaxation time of Eq. 12, > 0.5 */
  double J;             /* viscosity ratio nu_e / nu of Eq. 1b (paper: 1); 0 means 1 */
  double Gx, Gy;        /* external body force G of Eq. 2 */
  int32_t bc_x;         /* LBMP_BCX_*; PRESSURE needs nx >= 3 */
  int32_t bc_y;         /* LBMP_BCY_*; WALLS needs ny >= 3 */
  double rho0;          /* initial density; also the storage shift; 0 means 1 */
  double rho_in;        /* density imposed at x = 0 (PRESSURE only) */
  double rho_out;       /* density imposed at x = nx-1 (PRESSURE only) */
  int32_t forchheimer;  /* 1: Eq. 2 with F_eps = 1.75/sqrt(150 eps^3); 0: Eq. 8 */
  int32_t storage;      /* LBMP_STORE_* */
  int32_t fp16_log2_scale; /* s of S = 2^s for FP16 storage; 0 = automatic */
  int32_t fp16_rounding;   /* LBMP_ROUND_*: how FP16 stores round */
  int32_t kernel;          /* LBMP_KERNEL_*: implementation of the step */
  int32_t kn_model;        /* LBMP_KN_*: the correlation f_c(Kn) */
  uint64_t seed;           /* stream of the stochastic rounding (any value) */
  void *stream;         /* cudaStream_t for all work; NULL = a private stream */
  double kn_beta;       /* dynamic Knudsen number ("dynamic apparent permeability",
                           Section IV.B and V): 0 keeps the Kn given to
                           lbmp_set_fields.  Otherwise that Kn belongs to the
                           pressure p0 of density rho0, a node's pressure is
                           p = p0 (1 + kn_beta (rho - rho0)) with rho its density
                           at the time level, its Kn = Kn(p0) p0 / p (the mean
                           free path of Eq. 10 is inversely proportional to p)
                           and k_a = k_i f_c(Kn) is formed at every step.
                           FP32 storage needs the direct kernel, FP16 runs the
                           staged one (AUTO) or the direct one; 1 + kn_beta
                           (rho - rho0) must stay > 0 (checked for rho_in and
                           rho_out), else velocities turn non-finite (ENAN).
                           Not available to lbmp_batch_* and the adjoint. */
} lbmp_params;

typedef struct lbmp_info {
  int32_t nx, ny;
  int32_t pitch;          /* padded row length (elements) of device planes */
  int32_t storage;
  int64_t fluid_nodes;    /* lattice updates per time step */
  int64_t steps;          /* time level of the current state */
  double bytes_per_update;/* algorithmic HBM bytes per lattice update */
  double fp16_scale;      /* S (1 for FP32 storage) */
  double eps_mean;        /* mean porosity of the fluid nodes */
  int64_t device_bytes;   /* device memory held by the context */
  int64_t launches;       /* kernels launched by this context so far */
} lbmp_info;

typedef struct lbmp_ctx lbmp_ctx;

/* Message of the last error raised on the calling thread ("" if none). */
const char *lbmp_last_error(void);

/* Create a context on the current CUDA device: validates p, allocates the
 * two population buffers, the per-node medium and the reduction scratch.
 * Every later call on the context (and on a batch, created the same way)
 * runs on that device and gives the caller's current device back before it
 * returns; device pointers passed to it must be memory of that device.
 * Errors: EINVAL (bad parameters; nothing allocated), ENOMEM, ECUDA.
 * Section III (Eq. 12-17) defines the state the context holds. */
lbmp_status lbmp_create(const lbmp_params *p, lbmp_ctx **out);

/* Free every resource of ctx.  NULL is accepted. */
lbmp_status lbmp_destroy(lbmp_ctx *ctx);

/* Set the medium and restart from rest.  eps: porosity in [0, 1] (0 =
 * impermeable node, Section III); k_i: intrinsic permeability > 0 or +inf
 * (open pore); kn: Knudsen number >= 0, finite.  All [ny][nx] float64.
 * Stores per node eps and 1 / k_a with k_a = k_i f_c(Kn) (Eq. 3, 6-7), and
 * sets every population to w_i rho0.  Values of wall rows are ignored.
 * 1 / k_a is formed in FP32-pair arithmetic (~44 significant bits; Kn^-0.4348
 * from the hardware base-2 logarithm and power) and rounded to FP32: within
 * ~1 FP32 ulp of Eq. 3.  Host arrays in pinned, device-mapped memory are read
 * in place; other host memory is copied first.
 * Errors: EINVAL (a value out of range, or k_a < 1e-15; the context then
 * holds no valid medium until the next successful call), ECUDA. */
lbmp_status lbmp_set_fields(lbmp_ctx *ctx, const double *eps, const double *k_i,
                            const double *kn, int32_t where);

/* Advance n >= 0 time steps of Eq. 12 (collide and stream, walls, periodic
 * edges and pressure columns fused).  Asynchronous on the context stream.
 * Errors: EINVAL (n < 0), ESTATE (no fields set), ECUDA. */
lbmp_status lbmp_step(lbmp_ctx *ctx, int64_t n);

/* Wait for all work queued on the context stream. */
lbmp_status lbmp_synchronize(lbmp_ctx *ctx);

/* Density (Eq. 16a) and velocity (Eq. 17, or its quadratic form) of the
 * current time level, [ny][nx] float64 each; wall rows read 0.  Any output
 * pointer may be NULL.  Synchronous. */
lbmp_status lbmp_macroscopic(lbmp_ctx *ctx, double *rho, double *ux, double *uy,
                             int32_t where);

/* Apparent permeability k_a = k_i f_c(Kn) (Eq. 3 with Eq. 6-7, or Eq. 4-5)
 * of every node as the step uses it: the reciprocal of the FP32 1/k_a that
 * lbmp_set_fields stored, [ny][nx] float64; +inf
 * for an open pore, whatever the porosity of the node.  With a dynamic Kn,
 * k_a at the reference pressure p0 (the step's FP32 f_c of the Kn given).
 * Plate rows read 0.  Synchronous.  Errors: EINVAL, ESTATE (no fields
 * set), ECUDA. */
lbmp_status lbmp_apparent_permeability(lbmp_ctx *ctx, double *ka, int32_t where);

/* Post-stream populations f_i(x, t) of the current time level,
 * [9][ny][nx] float64; wall rows read 0.  Synchronous. */
lbmp_status lbmp_populations(lbmp_ctx *ctx, double *f, int32_t where);

/* Replace the current post-stream populations by f ([9][ny][nx] float64;
 * wall rows ignored).  With LBMP_BCX_PRESSURE columns 0 and nx-1 are then
 * re-extrapolated from their neighbours, as at every time level.  FP16
 * storage rounds the values.  Synchronous. */
lbmp_status lbmp_set_populations(lbmp_ctx *ctx, const double *f, int32_t where);

/* Global permeability by Darcy's law over the whole domain (Section IV.A,
 * discussion of Fig. 3): k_g = nu <u_x> / G_eff, <u_x> the mean velocity of
 * all fluid nodes, G_eff = G_x + c_s^2 (rho_in - rho_out) / (eps_mean rho0
 * (nx - 1)) (the pressure term only with LBMP_BCX_PRESSURE; eps p = c_s^2
 * rho, Eq. 1b).  FP64 reduction, deterministic order.  Synchronous.
 * Errors: ENAN (a non-finite velocity), ECUDA. */
lbmp_status lbmp_permeability(lbmp_ctx *ctx, double *k_g, double *u_mean);

/* Normalised velocity magnitude (Section IV.B, Fig. 6): u0 = |u| / max |u|
 * over every node of the fluid rows (impermeable nodes count with u = 0),
 * counted in nbins equal ranges of [0, 1]: counts[k] (host, nbins int64)
 * holds the nodes with min(floor(u0 nbins), nbins - 1) = k, so u0 = 1 falls
 * in the last range; max |u| = 0 puts every node in counts[0].  |u| =
 * sqrt(ux^2 + uy^2) in FP64 from the FP32 velocity lbmp_macroscopic
 * reports, each operation rounded separately (no fused multiply-add), and
 * u0 nbins likewise.  *umax (host, may be NULL) receives max |u|.
 * 1 <= nbins <= 64.  Synchronous.  Errors: EINVAL, ESTATE, ENAN (a
 * non-finite velocity), ECUDA. */
lbmp_status lbmp_velocity_histogram(lbmp_ctx *ctx, int32_t nbins, double *umax,
                                    int64_t *counts);

/* Relative velocity residual ||u - u_prev||_2 / ||u||_2 over fluid nodes,
 * u_prev being the velocity at the previous lbmp_residual call (zero after
 * set_fields); then stores u as the new u_prev.  FP64.  Synchronous. */
lbmp_status lbmp_residual(lbmp_ctx *ctx, double *r);

/* Total mass sum(rho) over fluid nodes, FP64.  Synchronous. */
lbmp_status lbmp_mass(lbmp_ctx *ctx, double *m);

/* Eq. 6-7 correction factor f_c(Kn), b = -1, f_c(0) = 1.  Host function;
 * returns NaN for Kn < 0 or NaN. */
double lbmp_fc(double kn);
/* f_c(Kn) of the correlation kn_model (LBMP_KN_*).  Host; NaN for Kn < 0,
 * NaN, or an unknown model. */
double lbmp_fc_model(int32_t kn_model, double kn);

/* ---------------------------------------------------------------------
 * Physical inputs of the Knudsen number (Section II, Eq. 9-11).  Host
 * functions, SI units.
 * --------------------------------------------------------------------- */
/* Eq. 9, Kozeny-Carman: intrinsic permeability [m^2] of packed spheres of
 * diameter d [m], k_d = (d^2 / 180) eps^3 / (1 - eps)^2.  NaN outside
 * 0 <= eps < 1 or for d < 0. */
double lbmp_kozeny_carman(double eps, double d);
/* Eq. 10: mean free path [m] of a gas of viscosity mu [Pa s] at pressure
 * p [Pa], temperature T [K] and molar mass M [kg/mol],
 * lambda = (mu / p) sqrt(pi R T / (2 M)).  NaN for non-positive inputs. */
double lbmp_mean_free_path(double mu, double p, double T, double M);
/* Eq. 11 (Herd et al.): characteristic pore radius [m] from k_d [m^2],
 * r [um] = 8.886e-2 sqrt(k_d [mD] / eps), 1 mD = 9.869e-16 m^2.  NaN for
 * k_d < 0 or eps <= 0. */
double lbmp_pore_radius(double k_d, double eps);
/* Lattice medium from physical data, for lbmp_set_fields: per node i of n,
 * k_d = Eq. 9 (eps[i], d[i]), k_i[i] = k_d / dx^2 (lattice units, dx [m]
 * the node spacing) and kn[i] = lambda / r with r = Eq. 11 (k_d, eps[i]) and
 * lambda [m] the mean free path (Eq. 10).  Impermeable nodes (eps = 0) get
 * k_i = 1, kn = 0 (unused); open pores (eps = 1) k_i = +inf, kn = 0.  Host
 * arrays.  Errors: EINVAL (NULL pointer, eps outside [0, 1], d <= 0 at a
 * porous node, lambda < 0, dx <= 0). */
lbmp_status lbmp_physical_medium(int64_t n, const double *eps, const double *d, double lambda,
                                 double dx, double *k_i, double *kn);

/* Checkpoint: bytes of a state blob (header + raw population buffer). */
lbmp_status lbmp_state_size(lbmp_ctx *ctx, size_t *bytes);
/* Copy the current state into buf (bytes >= lbmp_state_size).  Synchronous. */
lbmp_status lbmp_get_state(lbmp_ctx *ctx, void *buf, size_t bytes, int32_t where);
/* Restore a state written by lbmp_get_state of a context with the same
 * nx, ny and storage.  Errors: EINVAL (size or header mismatch). */
lbmp_status lbmp_set_state(lbmp_ctx *ctx, const void *buf, size_t bytes, int32_t where);

/* Sizes, storage and counters of ctx. */
lbmp_status lbmp_get_info(lbmp_ctx *ctx, lbmp_info *out);

/* Gradient of the global permeability with respect to the medium, by the
 * discrete adjoint of the time loop.  The objective is
 *   J(ln k_i, eps) = k_g after nsteps time steps from rest,
 * k_g as lbmp_permeability defines it (Darcy's law over the whole domain,
 * Section IV.A) and each step the collide-stream update of Section III
 * (Eq. 12, equilibrium Eq. 14, forcing Eq. 15, velocity Eq. 16-17 with the
 * drag of Eq. 2), the plates, periodic edges and pressure columns of this
 * context.  On return:
 *   k_g      (host, may be NULL) J, equal to what lbmp_permeability reports
 *            after lbmp_set_fields + lbmp_step(ctx, nsteps);
 *   d_logk   [ny][nx] float64, dJ/d ln k_i of every node (k_a = k_i f_c(Kn)
 *            with Kn held fixed, so also dJ/d ln k_a);
 *   d_eps    [ny][nx] float64, dJ/d eps of every node, including the
 *            mean-porosity term of the pressure drop in G_eff;
 *   where    LBMP_HOST or LBMP_DEVICE for d_logk and d_eps.
 * Plate rows read 0.  At impermeable (eps = 0) and open (k_a infinite)
 * nodes the derivatives of the flow part are the one-sided ones of the
 * branch the step takes there (0 for d_logk).  The forward states are
 * recomputed from checkpoints taken every `every` steps (0: ceil(sqrt(
 * nsteps))), of which the reverse steps need only the moments (rho, m):
 * the device holds ceil(nsteps / every) + 4 population buffers (FP32, like
 * the adjoint populations) and the moments of `every` levels (a third of a
 * population buffer each); each reverse step's
 * parameter derivatives are summed in FP32 over at most 32 steps, then in
 * FP64.  The context is left at time level nsteps of a run from rest (its
 * previous state is replaced).  Needs FP32 storage.  Synchronous.
 * Errors: EINVAL (NULL pointer, nsteps < 1, every < 0, FP16 storage, a
 * dynamic Kn), ESTATE (no fields set), ENOMEM, ENAN, ETIMEOUT, ECUDA. */
lbmp_status lbmp_permeability_gradient(lbmp_ctx *ctx, int64_t nsteps, int64_t every,
                                       double *k_g, double *d_logk, double *d_eps,
                                       int32_t where);

/* ---------------------------------------------------------------------
 * Batched sweeps.  `count` lattices of their own sizes (e.g. media
 * realizations x Knudsen numbers) share the physics parameters of p (tau, J,
 * G, boundary kinds, densities, Forchheimer, storage, rounding, seed; p->nx,
 * p->ny and p->kernel are ignored) and advance together: one launch per time
 * step covers a work list of row segments of all instances (one block per
 * segment, or a persistent grid walking it), or the tiles of all instances
 * in the staged bulk-copy kernel (CUDA graphs of 32 steps).  Each instance has its own populations, medium
 * and FP16 scale; the arithmetic per node is that of lbmp_step (Section III,
 * Eq. 12-17).  The launch shape (threads per block x nodes per thread x
 * grid mode) is chosen by lbmp_batch_tune.
 * --------------------------------------------------------------------- */
typedef struct lbmp_batch lbmp_batch;

typedef struct lbmp_batch_info {
  int32_t count;
  int32_t shape_threads;          /* launch shape in use */
  int32_t shape_nodes_per_thread;
  int32_t persistent;             /* 0: one block per work item, 1: persistent grid,
                                     2: staged kernel (bulk copies of tiles of W
                                     nodes into shared memory; threads = consumer
                                     threads, nodes per thread per tile) */
  int64_t total_nodes;            /* lattice updates per time step */
  int64_t steps;
  int64_t launches;
  int64_t device_bytes;
  double bytes_per_update;        /* algorithmic HBM bytes per lattice update */
} lbmp_batch_info;

/* Validate every (nx[i], ny[i]) with p under the rules of lbmp_create and
 * allocate all instances.  Errors: EINVAL, ENOMEM, ECUDA. */
lbmp_status lbmp_batch_create(const lbmp_params *p, int32_t count, const int32_t *nx,
                              const int32_t *ny, lbmp_batch **out);
/* Wait for the batch's queued work and free every resource it holds.  NULL
 * is accepted.  Always LBMP_OK. */
lbmp_status lbmp_batch_destroy(lbmp_batch *b);
/* Medium of instance i ([ny_i][nx_i] float64, as lbmp_set_fields), restart
 * it from rest. */
lbmp_status lbmp_batch_set_fields(lbmp_batch *b, int32_t i, const double *eps, const double *k_i,
                                  const double *kn, int32_t where);
/* n time steps of every instance; ESTATE until every instance has fields. */
lbmp_status lbmp_batch_step(lbmp_batch *b, int64_t n);
/* Wait for the queued steps; ETIMEOUT if a bounded wait of the staged
 * kernel gave up (the instances' state is then undefined). */
lbmp_status lbmp_batch_synchronize(lbmp_batch *b);
/* Global permeability and <u_x> of every instance (host arrays of count
 * doubles; either may be NULL), FP64 segmented reductions.  Synchronous. */
lbmp_status lbmp_batch_permeability(lbmp_batch *b, double *k_g, double *u_mean);
/* Post-stream populations of instance i, [9][ny_i][nx_i] float64. */
lbmp_status lbmp_batch_populations(lbmp_batch *b, int32_t i, double *f, int32_t where);
/* Autotuner: time `steps` steps of every candidate launch shape on this
 * batch, keep the fastest, restore the populations and time level.  Returns
 * the chosen candidate index and its time per step (either may be NULL). */
lbmp_status lbmp_batch_tune(lbmp_batch *b, int32_t steps, int32_t *chosen, double *ms_per_step);
/* Autotuner with a cache.  The shape tuned for a batch is reused, without
 * timing, by every later batch of the same class (lbmp_batch_class): from
 * this process's cache, else from the file named by the environment
 * variable LBMP_TUNE_CACHE (lines "key shape ms_per_step", the last line of a
 * key wins).  On a miss it runs lbmp_batch_tune and stores the choice (and
 * appends it to that file).  *from_cache = 1 when nothing was timed; any of
 * the outputs may be NULL.  Cache file errors are ignored.  Errors: those of
 * lbmp_batch_tune on a miss. */
lbmp_status lbmp_batch_tune_cached(lbmp_batch *b, int32_t steps, int32_t *chosen,
                                   double *ms_per_step, int32_t *from_cache);
/* Empty this process's shape cache (the file is left as it is). */
lbmp_status lbmp_batch_tune_cache_clear(void);
/* Class of a batch, as the cache keys it: storage and FP16 rounding,
 * boundary kinds, Forchheimer, the node-weighted median of ceil(log2 nx)
 * over the instances, floor(log2 of all nx*ny nodes), and nsm (the SM count
 * of the device).  Writes a NUL-terminated key of at most 64 bytes into
 * key[0..cap).  Host only, touches no device.  Errors: EINVAL for NULL
 * pointers, count < 1, nsm < 1, a size < 1 or cap too small. */
lbmp_status lbmp_batch_class(const lbmp_params *p, int32_t count, const int32_t *nx,
                             const int32_t *ny, int32_t nsm, char *key, int32_t cap);
/* Use launch candidate `shape` (0 <= shape < the number of candidates, as
 * lbmp_batch_tune reports them; the last one is the staged bulk-copy
 * kernel).  Errors: EINVAL. */
lbmp_status lbmp_batch_set_shape(lbmp_batch *b, int32_t shape);
/* Fill *out (host) with the batch's instance count, launch shape, lattice
 * updates per step, steps and launches so far, device bytes held and
 * algorithmic bytes per update.  Host-side values; no synchronisation.
 * Errors: EINVAL (NULL argument). */
lbmp_status lbmp_batch_get_info(lbmp_batch *b, lbmp_batch_info *out);

/* Global permeability of a lattice state held entirely in caller memory,
 * allocating nothing.  The paper has no counterpart: this serves callers
 * that cannot call cudaMalloc -- processes whose device memory is owned by
 * another framework's pool (an allocation behind the pool's back can fail or
 * take memory the pool has budgeted), and latency-bound loops that may not
 * pay for an allocation or for the device-wide synchronisation of cudaFree.
 * It computes what lbmp_permeability computes (Darcy's
 * law over the whole domain with eps p = c_s^2 rho for the pressure drop),
 * in FP64, from:
 *   p            lattice size, tau, J, G, boundary kinds, rho0, rho_in,
 *                rho_out, forchheimer, kn_model, kn_beta (other fields
 *                ignored; a dynamic Kn takes each node's density from f);
 *   f            device, [9][ny][nx] float64 post-stream populations, as
 *                lbmp_populations(..., LBMP_DEVICE) returns them;
 *   eps,k_i,kn   device, [ny][nx] float64 medium as for lbmp_set_fields;
 *   out          device, 3 doubles: k_g, <u_x>, number of fluid nodes whose
 *                velocity is not finite;
 *   stream       cudaStream_t (NULL: the legacy default stream); the call
 *                is asynchronous on it.
 * Scratch: the per-block partial sums live in a fixed 2 MiB array inside
 * the library (held by every GPU that loads it until exit), so the lattice
 * may need at most 65536 reduction blocks: ceil(nx / 256) * ny <= 65536
 * (e.g. 4096 x 4096); larger lattices get LBMP_EINVAL.  Every call uses the
 * same array: calls that overlap on the GPU (other streams, other threads)
 * race.  The first call on each device looks up the array's device address
 * (once, under a lock).
 * The sizes of the caller's arrays cannot be checked here: they must hold
 * what nx and ny imply.
 * Errors: EINVAL (NULL pointer, a parameter lbmp_create would reject among
 * those read here, a lattice beyond the scratch), ECUDA. */
lbmp_status lbmp_permeability_noalloc(const lbmp_params *p, const double *f, const double *eps,
                                      const double *k_i, const double *kn, double *out,
                                      void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBMP_H */
