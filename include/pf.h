/*
 * libpf -- GB300 (sm_103a) implementation of the time-stepping hot path of the
 * consistent and conservative lattice Boltzmann method for the gas-liquid-solid
 * diffuse-interface model of Zhan, Liu, Chai & Shi, "A thermodynamically
 * consistent and conservative diffuse-interface model for gas-liquid-solid
 * multiphase flows" (arXiv 2311.05097).
 *
 * One time step advances two lattices in one fused kernel (Sec. 3.3, steps 2-6):
 *   - the order-parameter lattice of Sec. 3.1 (conservative Cahn-Hilliard
 *     equation, Eq. 2, with the chemical potential of Eq. 9),
 *   - the flow lattice of Sec. 3.2 (consistent Navier-Stokes equations, Eq. 16,
 *     forced by surface tension, the solid penalty rho f and wetting),
 *   - both collided with the Hermite-moment MRT operator of Eqs. (37)-(38) and
 *     streamed by pulling.
 * Free rigid particles add a force/torque reduction (Eq. 27) and an explicit
 * Newton-Euler update (Eqs. 26, 28) on the device (Sec. 3.3, steps 7-10).
 *
 * Lattice units throughout: dx = dt = c = 1, cs^2 = d0.  2D uses D2Q9 for both
 * lattices; 3D uses D3Q19 (flow) and D3Q7 (order parameter).  Boundaries are
 * periodic, except optional no-flux walls at the two ends of y
 * (pf_grid.periodic[1] = 0: halfway bounce-back, mirrored stencil rows);
 * solids, and walls inside a periodic box, are marked by the smooth indicator
 * phi0 (Sec. 2.1).
 *
 * Conventions for every call:
 *   - Return value: PF_OK (0) or a negative PF_E* code.  The message of the last
 *     error of the calling thread is available from pf_last_error().
 *   - Field arrays are double, x-fastest: index (z*ny + y)*nx + x, N = nx*ny*nz.
 *     Vector fields are component-major: u[a*N + index], a = 0..dim-1.
 *   - `where` is PF_HOST (caller's host memory) or PF_DEVICE (device memory on
 *     the handle's GPU).  The caller owns every array it passes; the library
 *     copies what it needs and keeps no pointer to caller memory.
 *   - The library owns all device state of a handle and frees it in
 *     pf_destroy / pf_batch_destroy.
 *   - Work is issued on the handle's stream (pf_params.stream, or a stream the
 *     library creates when that is NULL).  pf_step is asynchronous; errors of
 *     asynchronous work are sticky and are returned by the next call on the
 *     handle or by pf_sync.
 */
#ifndef PF_H
#define PF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define PF_OK 0
#define PF_EINVAL (-1)   /* invalid argument or parameter */
#define PF_ENOMEM (-2)   /* device or host allocation failed */
#define PF_ECUDA (-3)    /* a CUDA runtime call failed */
#define PF_ENUMERIC (-4) /* a non-finite phi or u appeared, or a 16-bit order-parameter
                            population was saturated (see pf_diag.nan_flag) */
#define PF_ETIMEOUT (-5) /* a bounded device wait gave up (sticky: the handle's state is lost);
                           the environment variable PF_WAIT_POLLS, read at create, sets the
                           polls of one wait (fault injection: a tiny value makes the staged
                           kernel 2 give up at once) */
#define PF_ESTATE (-6)   /* call out of order (e.g. step before init) */

/* ---- precision policies ---- */
#define PF_P64 0        /* FP64 storage and arithmetic */
#define PF_P32 1        /* FP32 storage and arithmetic */
#define PF_PMIX_FP16 2  /* FP16 moving populations (scaled by 2^k), exact
                           fixed-point rest population of the order-parameter
                           lattice, FP32 arithmetic and auxiliary fields */
#define PF_PMIX_BF16 3  /* as PF_PMIX_FP16 with BF16 moving populations */

/* ---- memory location of caller arrays ---- */
#define PF_HOST 0
#define PF_DEVICE 1

/* Grid: dim = 2 or 3; nz is ignored (1) in 2D.  periodic[a] = 1: periodic
 * along axis a.  periodic[1] = 0 (2D or 3D) puts no-flux walls at y = -1/2
 * and y = ny - 1/2 (the paper's box walls): halfway bounce-back of both
 * lattices at resting walls, and the finite-difference stencils see mirror
 * images of the rows inside (zero normal gradient of phi, mu and phi0).  In
 * 2D walls run the one-cell-per-thread step (kernel 0), the strip step
 * (kernel 4) or, with particles, the split step (kernel 3).  Solid walls of
 * any shape can also be given through the smooth indicator phi0. */
typedef struct pf_grid {
    int dim;
    int nx, ny, nz;
    int periodic[3];
} pf_grid;

/* Model parameters, lattice units (Secs. 2-3). */
typedef struct pf_params {
    double sigma;      /* sigma_12, surface tension (Eq. 1); >= 0 */
    double D;          /* interface width (Eq. 1); > 0 */
    double M;          /* mobility (Eq. 2); > 0 */
    double eta;        /* eta of Eq. (30); <= 0 selects 2M/cs^2, i.e. s_1phi = 1 */
    double rho1, rho2; /* densities of phases 1 and 2 (Eq. 17); > 0 */
    double mu1, mu2;   /* dynamic viscosities (Eq. 18); > 0 */
    double d0;         /* cs^2 / c^2 (Sec. 3.2), in (0, 1/2) */
    double s0, s1, s2, s3, s4; /* relaxation rates of S_H (Eq. 38), in (0, 2);
                                  s2 is the second-order rate of the
                                  order-parameter lattice; s_2a, s_2b of the flow
                                  lattice follow from the viscosity (Eq. 35) */
    double theta_deg;  /* contact angle of phase 1 on solids (Young's law, Eq. 8) */
    double Fb[3];      /* body force density on the fluid (Eq. 16b) */
    double g[3];       /* gravity acting on particles (Eq. 26a) */
    double solid_eps;  /* lower bound of 1 - phi0 in mu/(1 - phi0) (Eq. 35);
                          in (0, 1), typically 1e-3 */
    double rep_xi;     /* particle-particle repulsion (Sec. 4.5): range xi >= 0 */
    double rep_eps;    /* and stiffness eps; 0 switches it off.  Force on k from j:
                          (x_k - x_j)/eps (R_k + R_j + xi - d)^2 for
                          R_k + R_j <= d <= R_k + R_j + xi, (x_k - x_j)/eps
                          (R_k + R_j - d) for d < R_k + R_j (as printed), zero
                          beyond; added to Eq. 26a, not to pf_particle.F.
                          With eps > 0 each particle is also pushed off the
                          nearest wall: the same form with 2 R_k for R_k + R_j,
                          eps/2 for eps and the mirror image of the particle
                          across that wall for x_j (the box walls of pf_grid,
                          and the circle wall_circle) */
    double wall_circle[3]; /* 2D: a circular wall (centre x, y; radius) seen only
                              by the particle-wall repulsion (the fluid sees
                              walls through phi0); radius 0: none */
    int phase_model;   /* 0 (default): the Cahn-Hilliard order parameter of
                          Eq. 2 on the lattice of Eq. 30.  1 (2D kernels 0 and 1,
                          and 3D): a conservative Allen-Cahn order
                          parameter, d_t phi + div(phi u) =
                          div(M (grad phi - theta n)), theta = (2/D)(1 - phi^2),
                          n = grad phi/|grad phi|, on the same lattice
                          (equilibrium with eta mu replaced by phi, s_1phi =
                          1/(M/cs^2 + 1/2), cs^2 theta n in the source) and the
                          mass flux S = M (rho1 - rho2)/2 (grad phi - theta n);
                          eta is unused; mu_phi of Eq. 9 still drives the
                          surface force.  The paper prints no such scheme */
    int precision;     /* PF_P64, PF_P32, PF_PMIX_FP16, PF_PMIX_BF16 */
    int store_log2_scale[2]; /* PMIX: stored value = population * 2^k for the
                                order-parameter [0] and flow [1] lattices;
                                0 selects a default from sigma, D and M */
    void *stream;      /* cudaStream_t to issue work on, or NULL */
} pf_params;

/* A free rigid particle (Sec. 2.4), FP64.  Disc (2D, per unit depth) or
 * sphere (3D) of radius R and density rho_p; its wettability is its own
 * theta_deg, or the handle's when that is NaN.  F and T are the hydrodynamic
 * force and torque of Eq. (27) of the last step (read only). */
typedef struct pf_particle {
    double x[3], u[3], w[3];
    double R, rho_p;
    double theta_deg;  /* own contact angle (Sec. 4.5; 2D and 3D), or NaN for the
                          handle's theta_deg.  The wetting terms of Eqs. 8, 9, 19
                          are then summed per solid, each with its own angle;
                          all solids without an own angle form one solid. */
    double F[3], T[3];
    int prescribed;    /* held motion, bit flags (0: Newton-Euler, Eqs. 26, 28):
                          1 keeps all of the u and w it was given (prescribed
                          motion, e.g. a rotating cylinder); 2, 4, 8 keep the
                          translation along x, y, z; 16 keeps the rotation (the
                          two-particle balance of Sec. 4.4 holds 2 | 16).  x
                          advances by u; F and T are still reported.  Values
                          outside 0..31: PF_EINVAL */
} pf_particle;

/* FP64 diagnostics at the current time: mass = sum phi, E_F of Eq. (8),
 * E_K = sum rho |u|^2 / 2, E_total = E_F + E_K (Sec. 2.3).  nan_flag is 0 when
 * every step stayed in range; bit 0 (value 1) is set if a step produced a
 * non-finite phi or u, bit 1 (value 2) if a 16-bit order-parameter population
 * reached the storage range (|value| * 2^store_log2_scale[0] >= 8) and was
 * saturated there: the order parameter stays exactly conserved, but the
 * populations no longer follow Eq. (21) at that cell. */
typedef struct pf_diag {
    double mass, E_F, E_K, E_total;
    int nan_flag;
} pf_diag;

typedef struct pf_handle pf_handle;
typedef struct pf_batch pf_batch;

/* Fill *p with the paper's defaults (d0 = 0.4, all s = 1, D = 4, Sec. 4.1),
 * sigma = 0.01, M = 0.02, rho1 = rho2 = 1, mu1 = mu2 = 0.1, theta = 90 deg,
 * solid_eps = 1e-3, no particle repulsion, PF_P64, NULL stream. */
int pf_params_default(pf_params *p);

/* Create a single-domain simulation.  Validates g and p (PF_EINVAL), allocates
 * the device state (PF_ENOMEM / PF_ECUDA).  *out is set on success only. */
int pf_create(const pf_grid *g, const pf_params *p, pf_handle **out);

/* Step 1 of Sec. 3.3: set the fields and initialise both lattices with their
 * equilibria (Eqs. 30, 32).  phi0 (fixed solids, values in [0, 1]) and phi are
 * required; u (dim*N) and P (N) may be NULL (zero).  phi should vanish inside
 * solids and particles (e.g. (1 - phi0) tanh(...) as in Eq. 39).  Particles set
 * before this call are included in the indicator.  Synchronous. */
int pf_init_fields(pf_handle *h, const double *phi0, const double *phi, const double *u,
                   const double *P, int where);

/* Advance n >= 0 time steps (Sec. 3.3 steps 2-10).  Asynchronous; replays a
 * CUDA graph of the step sequence.  PF_ESTATE before pf_init_fields.  A
 * single simulation runs kernel 0 (32x8 tiles in 2D) unless pf_set_config
 * or pf_autotune has chosen otherwise. */
int pf_step(pf_handle *h, int64_t n);

/* Choose the launch configuration of a single simulation by timing the
 * candidates of the batch autotuner (kernel, tile shape, CTAs per SM) on its
 * live state, or take the configuration cached for this kind of launch (see
 * pf_batch_create).  The timed candidate steps are real time steps of the
 * simulation (every configuration computes the same update, to rounding
 * order); their count, an even number plus one if the simulation stood at an
 * odd step, is returned in *steps_taken (may be NULL).  No counterpart in the
 * paper.  Synchronous.  PF_ESTATE before pf_init_fields. */
int pf_autotune(pf_handle *h, int64_t *steps_taken);

/* Macroscopic fields at the current time recomputed from the populations
 * (Eqs. 31, 17, 36): phi (N), rho (N), u (dim*N), P (N), mu = mu_phi of Eq. (9)
 * (N).  NULL outputs are skipped.  Synchronous. */
int pf_get_macros(pf_handle *h, double *phi, double *rho, double *u, double *P, double *mu,
                  int where);

/* Interface normal n = grad phi / |grad phi| at the current time (dim*N,
 * component-major like u), from phi of Eq. (31) with the central isotropic
 * stencil of Sec. 3.2 (mirror rows at walls); 0 where |grad phi|^2 <= 1e-24.
 * The unit normal of the fluid-fluid interface that the contact angle of
 * Eq. (8) is measured against, and the direction of the Allen-Cahn flux.
 * n is caller-owned; where = PF_HOST or PF_DEVICE.  Synchronous. */
int pf_get_normal(pf_handle *h, double *n, int where);

/* Checkpoint and resume (the paper has no counterpart; the step has no
 * randomness, so a resumed run is bit-identical to an uninterrupted one).
 * pf_state_size: bytes of the state of h (current populations, PMIX rest
 * populations, lagged fields, fixed indicator, particles, time).
 * pf_save_state: writes it into the caller's host buffer buf of `bytes`
 * (>= pf_state_size); synchronous; PF_ESTATE before pf_init_fields.
 * pf_load_state: replaces the state of h by one saved from a handle with the
 * same grid, walls, precision and particle count (set the particles first;
 * their saved positions and velocities replace them); the parameters are the
 * handle's own.  PF_EINVAL on a mismatch or a short buffer. */
int pf_state_size(pf_handle *h, int64_t *bytes);
int pf_save_state(pf_handle *h, void *buf, int64_t bytes);
int pf_load_state(pf_handle *h, const void *buf, int64_t bytes);

/* Particles: set = 1 adds (k == count) or overwrites (k < count) particle k
 * from *inout (its F, T are ignored); set = 0 copies particle k into *inout.
 * At most PF_MAX_PARTICLES.  Synchronous. */
#define PF_MAX_PARTICLES 64
int pf_particle_state(pf_handle *h, int k, pf_particle *inout, int set);
int pf_num_particles(pf_handle *h);

/* Deterministic FP64 diagnostics (fixed-order reductions).  Synchronous. */
int pf_diagnostics(pf_handle *h, pf_diag *out);

/* Wait for the handle's stream; PF_ENUMERIC if a non-finite value appeared or a
 * 16-bit population was saturated (pf_diag.nan_flag tells which). */
int pf_sync(pf_handle *h);

/* Number of time steps taken since pf_init_fields. */
int64_t pf_time(pf_handle *h);

void pf_destroy(pf_handle *h);

/* Thread-local message of the last error (never NULL). */
const char *pf_last_error(void);

/* ---- batched independent domains (2D or 3D, one dim per batch) ----
 * nd domains of uneven size, each with its own grid g[i] and parameters p[i]
 * (all of one precision; stream taken from p[0]).  pf_batch_step advances all
 * domains with one persistent launch per step captured in a CUDA graph; the
 * kernel, tile shape and CTAs per SM are chosen by an autotuner (which times
 * the candidates on the live state) in the first step call of at least 256
 * steps, and cached per (dim, precision, size mix, domain count and the
 * features that decide which kernels can run it: walls, the Allen-Cahn
 * lattice, own contact angles, strip eligibility, unit relaxation rates); a
 * later batch of the same kind takes the cached configuration in its first
 * step call of any length.  Before that, steps run kernel 0.  Step calls
 * shorter than a 16-step chunk replay one-step graphs. */
int pf_batch_create(int nd, const pf_grid *g, const pf_params *p, pf_batch **out);
int pf_batch_init(pf_batch *b, int i, const double *phi0, const double *phi, const double *u,
                  const double *P, int where);
int pf_batch_step(pf_batch *b, int64_t n);
int pf_batch_get_macros(pf_batch *b, int i, double *phi, double *rho, double *u, double *P,
                        double *mu, int where);
/* Every domain of a batch in one call (no counterpart in the paper): the
 * same work as pf_batch_init / pf_batch_get_macros for i = 0 .. nd - 1 (the
 * same results, bit for bit), with one wait at the end instead of one per
 * domain.  Host copies run on a stream of the library's own, so that the
 * copies of one domain overlap the kernels of others.  pf_batch_init_all
 * stages host inputs in a device ring of 2^25 doubles (256 MiB, or the
 * environment variable PF_INIT_RING read at create; at least one domain's
 * inputs), allocated for the call and freed before it returns, reads device
 * inputs in place, and runs the init kernels of consecutive domains on the
 * batch's stream and up to seven more streams of its own in turn (as many as
 * keep their scratch, 32 bytes per cell of the largest domain each, within
 * 512 MiB; the batch's stream waits for them before the call returns).
 * pf_batch_get_macros_all runs the macroscopic passes in domain order on the
 * batch's stream, rotating over up to four macro buffers (the extra ones,
 * as many as fit in 256 MiB, are allocated at its first call and kept with
 * the batch).  Each argument is an array of nd pointers, one per domain,
 * with the layout of the single-domain call; phi0 and phi (and their
 * entries) are required; u, P (init) and any output array may be NULL (the
 * field is not given / not read), and so may single entries.  where applies
 * to every pointer.  Synchronous: the caller's arrays may be reused when
 * the call returns.  Errors as for the single-domain calls; on an error the
 * domains before the failing one may already be done. */
int pf_batch_init_all(pf_batch *b, const double *const *phi0, const double *const *phi,
                      const double *const *u, const double *const *P, int where);
int pf_batch_get_macros_all(pf_batch *b, double *const *phi, double *const *rho, double *const *u,
                            double *const *P, double *const *mu, int where);
int pf_batch_diagnostics(pf_batch *b, int i, pf_diag *out);
int pf_batch_sync(pf_batch *b);
/* Total lattice cells of the batch and the chosen launch configuration
 * (tile_x, tile_y in cells, ctas_per_sm, kernel) after the first step; -1
 * before.  Null out-pointers are skipped. */
int64_t pf_batch_cells(pf_batch *b);
int pf_batch_config(pf_batch *b, int *tile_x, int *tile_y, int *ctas_per_sm, int *kernel);

/* Fix the launch configuration instead of letting the autotuner choose it
 * (for benchmarks and tests of one configuration; no counterpart in the
 * paper).  tile_x x tile_y cells per tile; ctas_per_sm 0 = as many as fit,
 * else a cap.  kernel:
 *   0  one cell per thread (all policies, particles, walls, either
 *      order-parameter lattice; 2D tiles 32x8, 64x4, 32x16; 3D the tile
 *      of its policy);
 *   1  2D, two vertically adjacent cells per thread in packed FP32
 *      arithmetic (P32 and PMIX, fixed solids, no walls, either lattice;
 *      tiles 32x16, 64x8, 32x32);
 *   2  as 1, with each tile's inputs copied into shared memory by
 *      asynchronous bulk copies one tile ahead (tile 32x16; every nx a
 *      multiple of 8 for 16-bit storage, of 4 for FP32; the Cahn-Hilliard
 *      lattice only);
 *   3  2D with free particles: the tiles out of every particle's reach run
 *      kernel 1 (with walls at the ends of y: kernel 0 without the particle
 *      terms), with the fixed solids' mu_phi0 grad phi0 of Eq. 19, the
 *      others kernel 0 with them, chosen on the device each step (one
 *      domain, P32 or PMIX, tile 32x16, the Cahn-Hilliard lattice; particles
 *      may have their own contact angles);
 *   4  2D, two horizontally adjacent cells per thread in packed FP32
 *      arithmetic on strips of 64 columns marched in y, every input staged
 *      in shared memory by tensor copies one band of rows ahead, periodic
 *      wrap in x through ghost columns (P32 and PMIX, fixed solids, walls
 *      at the ends of y or not, either lattice, every nx even and >= 8;
 *      tile_x = 64, the strip width; tile_y = the rows of one work item,
 *      any value >= 1).
 * Adding a particle later falls back to kernel 0.  PF_EINVAL for a
 * configuration that is not built or not allowed; a pending odd time step is
 * issued first.  Call after init (pf_set_config) or at any time between steps
 * (pf_batch_set_config). */
int pf_batch_set_config(pf_batch *b, int tile_x, int tile_y, int kernel, int ctas_per_sm);
int pf_set_config(pf_handle *h, int tile_x, int tile_y, int kernel, int ctas_per_sm);
/* The launch configuration of a single simulation, as pf_batch_config: -1
 * until pf_autotune has chosen it, pf_set_config has fixed it, or a step has
 * run with the default (kernel 0). */
int pf_get_config(pf_handle *h, int *tile_x, int *tile_y, int *ctas_per_sm, int *kernel);
void pf_batch_destroy(pf_batch *b);

/* ---- diagnostics without device allocation ----
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory: work recorded by CUDA stream capture (where
 * cudaMalloc/cudaFree are illegal), real-time or fixed-budget loops, and hosts
 * whose device memory is owned by another allocator.
 *
 * Computes the same FP64 quantities as pf_diagnostics -- out4 = {sum phi,
 * E_F of Eq. (8), E_K = sum rho |u|^2 / 2, E_F + E_K} -- from caller-owned
 * device arrays (x-fastest, N = nx*ny*nz; u component-major, dim*N), e.g. the
 * PF_DEVICE output of pf_get_macros, with phi0 the total solid indicator.
 * Only g->dim, nx, ny, nz, periodic and p->sigma, D, theta_deg are read.  The
 * boundaries follow pf_create: periodic, or walls at the ends of y
 * (periodic[1] = 0), whose stencils read the mirror image of the rows inside
 * as pf_diagnostics does; anything else returns PF_EINVAL.  The wetting
 * energy uses the one angle p->theta_deg for the whole of phi0: for a handle
 * whose particles carry their own contact angles (Sec. 4.5), where
 * pf_diagnostics sums the wetting energy per solid, E_F differs -- use
 * pf_diagnostics there.  out4 is
 * host (where = PF_HOST; the call then waits for the result) or device memory
 * (PF_DEVICE; asynchronous).  Work runs on `stream` (NULL = default stream).
 *
 * Nothing is allocated: the reduction's per-block partial sums live in one
 * fixed array in device global memory, sized for at most
 * PF_NOALLOC_MAX_CELLS cells (PF_NOALLOC_MAX_BLOCKS blocks of 4096 cells,
 * about 192 KiB); larger grids return PF_EINVAL.  Every GPU that loads the
 * library holds that array until the process exits.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress), so make
 * that first call before any stream capture; the address is kept per device
 * and per driver context, and a call made in a new context of the device
 * (after cudaDeviceReset, for example) looks it up again, so make the first
 * call after such a change before any capture too.  All calls share the array: each
 * call overwrites every partial it reads, so nothing carries over, but calls
 * whose kernels overlap on the GPU (different streams, no ordering) race on
 * it and must be serialised by the caller. */
#define PF_NOALLOC_MAX_BLOCKS 8192
#define PF_NOALLOC_MAX_CELLS (8192LL * 4096LL)
int pf_diagnostics_noalloc(const pf_grid *g, const pf_params *p, const double *phi,
                           const double *rho, const double *u, const double *phi0, double *out4,
                           int where, void *stream);

/* Number of kernel launches issued by the library since load (all handles). */
int64_t pf_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
