/*
 * lbm_imb.h -- C ABI of the GB300 LB-IMB-DEM library (liblbm_imb.so).
 *
 * The library advances a gas-solid suspension with the method of Xiong et al.,
 * "Large-Scale DNS of Gas-Solid Flow on Mole-8.5" (arXiv:1011.2613):
 *   - LBGK on D2Q9 or D3Q19 (section "Numerical scheme"),
 *   - the Noble-Torczynski immersed moving boundary term, Eq. (1), with the
 *     weighting beta(eps, tau) of Eq. (2) and the solid collision term
 *     Omega^S printed after Eq. (2),
 *   - the solid fraction eps of each lattice cell = covered area/volume (text
 *     after the Omega^S equation), computed exactly for disks and spheres,
 *   - the hydrodynamic force and torque on each particle, Eq. (3),
 *   - frictionless linear spring-dashpot DEM contacts, Eqs. (4)-(5), and a
 *     symplectic Euler particle update.
 * Every step runs in hand-written sm_103a CUDA kernels on the caller's stream.
 *
 * Conventions (all calls):
 *   - Every call returns an int status (LBM_IMB_OK = 0 or a negative code);
 *     output parameters are written only on success.
 *   - Lattice units: spacing h = 1, time step 1.  Node (i,j,k) sits at
 *     (i,j,k); the domain spans [-1/2, n-1/2) along each axis.
 *   - Population direction order (the interface order, used by
 *     lbm_imb_get/set_populations):
 *       D2Q9 : (0,0) (1,0) (-1,0) (0,1) (0,-1) (1,1) (-1,-1) (1,-1) (-1,1)
 *       D3Q19: (0,0,0) (+-1,0,0) (0,+-1,0) (0,0,+-1) (1,1,0) (-1,-1,0)
 *              (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
 *              (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *     i.e. the rest direction, then opposite pairs.
 *   - Field and population arrays are dense, x fastest:
 *       f[q][z][y][x], rho[z][y][x], u[d][z][y][x] (d < dim), eps[z][y][x].
 *     Particle arrays are [n][3] (z and the x/y spin components are zero
 *     in 2D).
 *   - Pointers documented as "host" must be host memory; "device" pointers
 *     must be device memory of the device current at lbm_imb_init.
 *   - A handle is not thread-safe; calls on one handle must be serialised.
 *
 * Readings of the paper used where it is silent or garbled:
 *   - state between steps = post-collision populations; one step =
 *     rasterise eps -> pull-stream -> collide (Eq. 1) -> force/torque (Eq. 3)
 *     -> DEM.
 *   - several particles covering one cell: eps = min(1, sum_p e_p), solid
 *     velocity = e-weighted mean of the particles' velocities, node force
 *     split in proportion e_p.  At most LBM_IMB_MAX_OWNERS particles may
 *     cover one cell (else LBM_IMB_EOWNERS).
 *   - solid velocity includes rotation, V = v_p + omega_p x (x_n - x_p).
 *   - body force F_i = 3 w_i rho (c_i . g_f) at every node.
 *   - force on a particle = - sum_n beta_n sum_i Omega_i^S c_i (momentum the
 *     solid term gives the fluid is taken from the particle); torque likewise
 *     with (x_n - x_p) x.
 *   - walls (wall_y = 1): halfway bounce-back at y = -1/2 and ny - 1/2.
 *   - DEM: overlap xi = R_i + R_j - |r_i - r_j|; force on i =
 *     k_n xi n_ij - eta v_n,ij, n_ij = (r_i - r_j)/|r_i - r_j|,
 *     eta = -2 ln(e) sqrt(m* k_n / (pi^2 + ln^2 e)), m* = m_i m_j/(m_i+m_j)
 *     (m* = m_i against a wall).  v += (F_f + F_c + m g_s)/m dt, x += v dt,
 *     omega += T_f / I dt over dem_substeps sub-steps of dt = 1/dem_substeps.
 *   - masses: 2D m = rho_s pi R^2 (per unit depth), I = m R^2/2;
 *             3D m = rho_s 4/3 pi R^3, I = 2/5 m R^2.
 */
#ifndef LBM_IMB_H
#define LBM_IMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_IMB_MAX_OWNERS 4

/* status codes */
enum {
  LBM_IMB_OK = 0,
  LBM_IMB_EINVAL = -1,      /* invalid argument or configuration */
  LBM_IMB_ENOMEM = -2,      /* caller buffer smaller than lbm_imb_required_bytes */
  LBM_IMB_ECUDA = -3,       /* a CUDA runtime call failed */
  LBM_IMB_ETIMEOUT = -4,    /* a bounded device wait gave up */
  LBM_IMB_ENONFINITE = -5,  /* NaN/Inf found by a health check */
  LBM_IMB_EUNSUPPORTED = -6,/* configuration outside the implemented limits */
  LBM_IMB_EOWNERS = -7,     /* a lattice cell was covered by too many particles */
  LBM_IMB_EBIN = -8         /* a DEM cell-list bin overflowed */
};

/* population storage (the arithmetic follows the storage) */
enum {
  LBM_IMB_STORE_F64 = 0,    /* FP64 populations, FP64 arithmetic */
  LBM_IMB_STORE_F32DEV = 1, /* FP32 storage of f_i - w_i rho0, FP32 arithmetic */
  LBM_IMB_STORE_F16DEV = 2, /* FP16 storage of (f_i - w_i rho0)/w_i, FP32 arithmetic */
  LBM_IMB_STORE_DFDEV = 3   /* f_i - w_i rho0 as an unevaluated pair of FP32 numbers (8 bytes,
                               48-bit significand: finer than FP64 on f_i); pair arithmetic
                               for plain nodes, FP64 for covered nodes */
};

/* Problem statement: lattice, relaxation time, body force, particles with
 * radii and densities (the quantities of the paper's Table 2). */
typedef struct lbm_imb_config {
  uint32_t struct_size;    /* = sizeof(lbm_imb_config) */
  int32_t dim;             /* 2 (D2Q9) or 3 (D3Q19) */
  int32_t nx, ny, nz;      /* lattice nodes; nz = 1 for dim = 2 */
  int32_t wall_y;          /* 0: periodic in y; 1: bounce-back walls in y */
  int32_t storage;         /* LBM_IMB_STORE_* */
  double tau;              /* BGK relaxation time, > 0.5 */
  double body_force[3];    /* gas acceleration g_f (F_i built from it) */
  double gravity[3];       /* particle acceleration g_s */
  double rho_fluid;        /* initial gas density rho0 (fluid starts at rest) */
  double k_n;              /* DEM normal stiffness, >= 0 */
  double restitution;      /* DEM restitution coefficient e in (0, 1] */
  int32_t dem_substeps;    /* DEM sub-steps per lattice step, >= 1 */
  int32_t eps_method;      /* covered fractions: 0 exact closed forms; 1 the table
                            * lookup of Eq. 6: exact fractions on a grid over the
                            * cell's offset from the centre (2D 256 radii x 128
                            * slopes, 3D 96 x 64 x 48), FP32 interpolation;
                            * needs all radii equal and > 1, else
                            * LBM_IMB_EUNSUPPORTED */
  int64_t n_particles;     /* >= 0 */
  const double* pos;       /* host, [n][3], copied at init */
  const double* vel;       /* host, [n][3], copied at init */
  const double* omega;     /* host, [n][3], copied at init */
  const double* radius;    /* host, [n], copied at init; > 0 and at most 8
                            * (3D with exact fractions) or 29 (2D, and 3D
                            * with eps_method = 1), else LBM_IMB_EUNSUPPORTED */
  const double* density;   /* host, [n], solid density in lattice units */
  double dem_skin;         /* 0: DEM contacts from a cell list rebuilt every
                            * (sub)step; > 0: from Verlet neighbour lists of the
                            * pairs closer than R_i + R_j + dem_skin, rebuilt on
                            * the device when a particle has moved more than
                            * dem_skin/2 since the last build (the same contact
                            * forces, summed in the same order); not for batch
                            * members (LBM_IMB_EUNSUPPORTED) */
} lbm_imb_config;

typedef struct lbm_imb lbm_imb_t; /* opaque, library-owned host state */

/* Device bytes the caller must provide to lbm_imb_init for this config
 * (populations, solid-fraction slots, particle state, DEM bins), or 0 if the
 * config is invalid. */
size_t lbm_imb_required_bytes(const lbm_imb_config* cfg);

/* The problem of the paper's section "Numerical scheme" and Table 2: a
 * D2Q9/D3Q19 lattice with relaxation time tau, a body force on the gas, and
 * particles with radii and densities (masses as in Table 2's reduced
 * units), initially in a gas at rest.  Lay out the caller's device block
 * (dev_buf, >= required bytes, 256-byte aligned, owned by the caller and
 * never freed by the library), upload the particles, set the populations to
 * the rest equilibrium w_i rho0 and rasterise eps (covered fraction of each
 * cell, text after the Omega^S equation).  Particles must be finite, inside
 * the walls (y in [-1/2, ny - 1/2] when wall_y = 1) and in [-1/2, n) along
 * periodic axes, else EINVAL.  cuda_stream (a cudaStream_t, may be NULL for the legacy
 * stream) is the stream every later call of this handle uses.  On success
 * *out receives the handle.  The device current at this call is used.
 * A rejected config returns its status (EINVAL, EUNSUPPORTED) before the
 * buffer is looked at, so a call with dev_buf = NULL reports why
 * lbm_imb_required_bytes returned 0. */
int lbm_imb_init(const lbm_imb_config* cfg, void* dev_buf, size_t bytes,
                 void* cuda_stream, lbm_imb_t** out);

/* Queue n >= 0 time steps on the handle's stream (asynchronous; replays a
 * captured CUDA graph).  One step is the paper's time step ("Numerical
 * scheme"): eps from the particle positions, pull streaming and the LBGK
 * collision with the immersed-boundary term of Eq. (1) (beta of Eq. (2),
 * Omega^S), the hydrodynamic force and torque of Eq. (3), and the DEM
 * contacts of Eqs. (4)-(5) with the particle update.  Every
 * lbm_imb_set_health_check steps (default 100) a health check scans the
 * stored rest-direction populations and the particle state; a NaN/Inf (or a
 * particle centre beyond 2^30 lattice units), like the other device-side
 * errors (EOWNERS, EBIN), is reported by the next synchronising call
 * (LBM_IMB_ENONFINITE).  The kernels skip a particle whose centre is not
 * finite instead of indexing the lattice with it. */
int lbm_imb_step(lbm_imb_t* h, int64_t n);

/* Steps between health checks of lbm_imb_step (0 turns them off). */
int lbm_imb_set_health_check(lbm_imb_t* h, int64_t every);

/* Run the health check now on the handle's stream and synchronise:
 * LBM_IMB_ENONFINITE if a stored rest-direction population, a particle
 * velocity or spin is NaN/Inf or a particle centre is NaN/Inf or beyond
 * 2^30 lattice units; any other pending device error likewise.  A NaN in
 * any population reaches the rest direction of some node within one step,
 * so a check one step after it appeared finds it. */
int lbm_imb_check_health(lbm_imb_t* h);

/* Kernel families of one time step, in launch order (indices into the
 * timing array of lbm_imb_step_profiled). */
enum {
  LBM_IMB_K_EPS_CLEAR = 0, /* clear the previous eps footprint, zero Eq. 3 sums */
  LBM_IMB_K_EPS_RASTER = 1,/* exact eps of every covered cell */
  LBM_IMB_K_COLLIDE = 2,   /* pull-stream + Eq. 1 collision + Eq. 3 sums */
  LBM_IMB_K_DEM = 3,       /* cell list, Eqs. 4-5 contacts, integration */
  LBM_IMB_NUM_KERNELS = 4
};

/* Run n (1..4096) time steps like lbm_imb_step but launched directly (no
 * graph) with CUDA events between the kernel families, then synchronise.
 * kernel_ms[LBM_IMB_NUM_KERNELS] receives the summed device time of each
 * family over the n steps, *total_ms the device time from the first launch
 * to the end of the last step.  Same results as lbm_imb_step. */
int lbm_imb_step_profiled(lbm_imb_t* h, int64_t n, double* kernel_ms, double* total_ms);

/* Number of Verlet-list builds so far (0 with dem_skin = 0); synchronises. */
int lbm_imb_dem_rebuilds(lbm_imb_t* h, int64_t* builds);

/* Number of kernel launches one time step issues (for launch accounting). */
int lbm_imb_launches_per_step(lbm_imb_t* h, int* launches);

/* Kernel form of the collision step (results are the same; the speed
 * depends on lattice, storage and GPU; the autotuner times them):
 *   0 persistent CTAs walking row tiles, each warp queueing its covered
 *   nodes in shared memory for the immersed-boundary update, with a
 *   register budget for 4 CTAs per SM (default),
 *   1 the same with a register budget for 8 CTAs per SM, 2 a form that
 *   bulk-copies (TMA) the next row tile's source rows into shared memory
 *   while colliding the current one (reduced-precision storages only; FP64
 *   falls back to 0), 3 as 0 with a register budget for 6 CTAs per SM,
 *   4 as 0 with the next row tile's populations pulled into registers
 *   before the current one is collided, 5 the same with a budget for 3
 *   CTAs per SM, 6 one CTA per row tile that packs its covered nodes into
 *   full warps through shared memory (register budget for 8 CTAs per SM),
 *   7 the same with a budget for 5 CTAs per SM, 8 two adjacent nodes per
 *   thread with paired FP32 arithmetic and aligned pair loads/stores
 *   (reduced-precision storages only; FP64 falls back to 0; 6 CTAs per SM),
 *   9 the same with 5 CTAs per SM.
 * The pair storage (LBM_IMB_STORE_DFDEV) has its own set: 0, 3 and 1 the
 * persistent queue form with budgets for 4, 3 and 2 CTAs per SM, 5 and 4
 * the pulled-ahead form with 3 and 2, 2 the TMA form, 6 and 7 the split
 * forms (plain nodes in one launch, then the covered nodes listed by the
 * rasteriser in a second: in FP64 for 6, in pair arithmetic for 7, and
 * for 8 as 7 with the plain part two adjacent nodes per thread in paired
 * FP32 instructions; 9 as 7 with the covered nodes' pulled populations and
 * moments handed from the plain launch to the covered one through a
 * compact buffer instead of the rasteriser's list).
 * Returns EINVAL outside 0..9.  Not for batch members or batches. */
int lbm_imb_set_collide_variant(lbm_imb_t* h, int variant);

/* Wait for the handle's stream and report device-side errors. */
int lbm_imb_sync(lbm_imb_t* h);

/* Copy particle state into caller-owned host arrays ([n][3] each, any may be
 * NULL): positions, velocities, spins, and the hydrodynamic force and torque
 * of the last step (Eq. 3).  cap = capacity in particles (>= n).
 * Synchronises the stream. */
int lbm_imb_particles(lbm_imb_t* h, double* pos, double* vel, double* omega,
                      double* force, double* torque, int64_t cap);

/* Replace particle positions/velocities/spins (host, [n][3], any may be
 * NULL to keep the current value); n must equal the configured count.
 * The values are checked on the host first: every given value finite,
 * positions inside the walls (y in [-1/2, ny - 1/2] when wall_y = 1) and
 * in [-1/2, n) along periodic axes; EINVAL (nothing copied) otherwise.  Copied on the stream, which is then synchronised. */
int lbm_imb_set_particles(lbm_imb_t* h, const double* pos, const double* vel,
                          const double* omega, int64_t n);

/* Macroscopic fields of the populations the next collision sees (the
 * moments the LBGK collision of Eq. (1) is built on): rho = sum_i f_i,
 * u = sum_i f_i c_i / rho + g_f/2 (dim components; the half-force shift of
 * the reported velocity is a reading, the paper is silent) and
 * eps = min(1, sum of covered fractions), the solid fraction of the text
 * after the Omega^S equation, at the current particle positions.  cap = capacity in
 * nodes (>= nx*ny*nz).  on_device = 1: the pointers are device memory, the
 * call is enqueued on the stream; 0: host memory, the call synchronises.
 * Any pointer may be NULL. */
int lbm_imb_fields(lbm_imb_t* h, double* rho, double* u, double* eps,
                   int64_t cap, int on_device);

/* Read / overwrite the stored post-collision populations as FP64
 * f[q][z][y][x] (reduced storages convert).  cap = capacity in values
 * (>= Q*nx*ny*nz).  on_device as for lbm_imb_fields. */
int lbm_imb_get_populations(lbm_imb_t* h, double* f, int64_t cap, int on_device);
int lbm_imb_set_populations(lbm_imb_t* h, const double* f, int64_t cap, int on_device);

/* Global sums (synchronises): total fluid mass sum f, fluid momentum
 * sum f c [3], particle momentum sum m v [3].  Any pointer may be NULL. */
int lbm_imb_totals(lbm_imb_t* h, double* fluid_mass, double* fluid_momentum,
                   double* particle_momentum);

/* Steps taken since init. */
int lbm_imb_steps_done(lbm_imb_t* h, int64_t* steps);

/* Checkpoint / resume.  The paper's suspensions run for millions of steps
 * (section "Simulation results"), which a run survives only by restarting
 * from saved state.  lbm_imb_save synchronises the stream, reports any
 * pending device error instead of saving, and writes to the file at `path`
 * (created or truncated): a header (format version, a hash of the
 * configuration given to lbm_imb_init, lattice sizes, storage, particle
 * count, steps taken), the stored post-collision populations in their raw
 * storage format, and the particle positions, velocities, spins and the
 * last step's hydrodynamic force and torque.  lbm_imb_load reads such a file
 * into a handle made from the same configuration (same hash; EINVAL for any
 * other file or an unreadable one, with the handle unchanged if the header
 * is rejected) and restores the step count; eps and the DEM neighbour data
 * are rebuilt by the next step from the loaded positions, so a run that is
 * saved and resumed continues as it would have (up to the order of the
 * FP64 force atomics).  Single simulations only: EUNSUPPORTED for batches,
 * slab decompositions and their members.  Both synchronise. */
int lbm_imb_save(lbm_imb_t* h, const char* path);
int lbm_imb_load(lbm_imb_t* h, const char* path);

/* ---- batches of independent suspensions ----
 * A batch advances n independent suspensions (same dim and storage; any
 * lattice sizes, particle counts, densities; dem_substeps = 1) by one
 * cooperative persistent kernel launch per time step, replayed from a CUDA
 * graph.  Inside the launch the CTAs walk shared work lists (particles for
 * eps and DEM, collision tiles of tile_x x 128/tile_x nodes) and meet at
 * grid barriers between the phases of the step; each member evolves exactly
 * as it would alone (up to the order of the FP64 force atomics).  A barrier
 * wait that does not complete within its poll limit makes the launch end and
 * the next synchronising call return LBM_IMB_ETIMEOUT.  Not in the paper: a
 * throughput form for many small suspensions that would underfill the GPU
 * one at a time. */

/* Device bytes for the batch (0 if a config is invalid). */
size_t lbm_imb_batch_required_bytes(const lbm_imb_config* cfgs, int n);

/* Initialise a batch of n (1..256) configs in the caller's device block.
 * tile_x: 32, 64 or 128 (0 = 128); blocks_per_sm: CTAs per SM of the
 * persistent grid (0 = as many as fit).  The batch handle steps with
 * lbm_imb_step / lbm_imb_step_profiled (whose time goes to the
 * LBM_IMB_K_COLLIDE slot) and is released with lbm_imb_destroy.  Members
 * need dem_substeps = 1 and dem_skin = 0 (LBM_IMB_EUNSUPPORTED otherwise);
 * a rejected config set returns its status before the buffer is looked at. */
int lbm_imb_batch_init(const lbm_imb_config* cfgs, int n, int tile_x, int blocks_per_sm,
                       void* dev_buf, size_t bytes, void* cuda_stream, lbm_imb_t** out);

/* Handle of member i for the accessors (lbm_imb_particles, _fields,
 * _get/_set_populations, _totals, _set_particles).  It shares the batch's
 * memory and stream, cannot be stepped or destroyed on its own, and lives as
 * long as the batch. */
int lbm_imb_batch_member(lbm_imb_t* batch, int i, lbm_imb_t** member);

/* Number of members (1 for a single suspension). */
int lbm_imb_batch_size(lbm_imb_t* h, int* n);

/* Change / read the launch shape of a batch (tile width, CTAs per SM;
 * the grid actually used is returned in *grid). */
int lbm_imb_batch_set_launch(lbm_imb_t* batch, int tile_x, int blocks_per_sm);
int lbm_imb_batch_get_launch(lbm_imb_t* batch, int* tile_x, int* grid);


/* ---- standalone DEM contact forces (Eqs. 4-5) ----
 * The cell-list contact kernel of the time step, callable on its own: for n
 * particles (device arrays pos[n][3], vel[n][3], radius[n], mass[n]) in a
 * lattice of extent[3] nodes (extent[2] = 1 in 2D; periodic except along y
 * when wall_y = 1, where the walls at y = -1/2 and extent[1] - 1/2 also
 * push), write the frictionless spring-dashpot contact force on every
 * particle to fc[n][3] (device).  Pairs are summed in ascending partner id,
 * then the wall terms.  rmax bounds every radius (it sizes the bins; a
 * larger radius is reported as LBM_IMB_EBIN).  Needs a caller-owned device
 * workspace of lbm_imb_dem_workspace_bytes bytes (256-byte aligned; the DEM
 * bins).  The call is enqueued on `stream` (a cudaStream_t) and then
 * synchronises it to report LBM_IMB_EBIN (a bin or contact list overflowed,
 * or a radius above rmax). */
size_t lbm_imb_dem_workspace_bytes(int32_t dim, const int32_t* extent, int32_t wall_y,
                                   int64_t n, double rmax);
int lbm_imb_dem_forces(int32_t dim, const int32_t* extent, int32_t wall_y, int64_t n,
                       double rmax, const double* pos, const double* vel,
                       const double* radius, const double* mass, double k_n,
                       double restitution, double* fc, void* workspace,
                       size_t workspace_bytes, void* stream);

/* lbm_imb_dem_forces without a workspace argument, for callers that cannot
 * allocate device memory: code running with the device memory already
 * handed out to another allocator, or hosts that forbid allocation after
 * start-up (no cudaMalloc, cudaFree or allocating library call happens here).
 * There is no counterpart in the paper; this only changes where the scratch
 * lives.  The cell-list bins are taken from a fixed 8 MiB array compiled into
 * the library (every device that loads the library keeps it until the process
 * exits); a problem whose bins need more (error word + 4 B per particle +
 * 68 B per bin, each rounded up to 256 B) is rejected with
 * LBM_IMB_EUNSUPPORTED.  The first call on a device looks up the array's
 * device address for that device, so make that first call before any stream
 * capture.  All calls share the one array: calls that overlap on the GPU (on
 * different streams or threads) race and give wrong forces.  Same arguments,
 * results and errors as lbm_imb_dem_forces otherwise. */
int lbm_imb_dem_forces_static(int32_t dim, const int32_t* extent, int32_t wall_y,
                              int64_t n, double rmax, const double* pos,
                              const double* vel, const double* radius,
                              const double* mass, double k_n, double restitution,
                              double* fc, void* stream);

/* ---- learned drag closure ----
 * Not in the paper.  The paper compares the drag it resolves with Wen-Yu and
 * EMMS closures (section "Simulation results"); here the resolved forces of
 * the method are used to train a small network that predicts a particle's
 * drag from its surroundings, and the resolved solve measures its error.
 *
 * Drag samples: for every particle of a simulation, features
 *   [0] mean solid fraction eps over the nodes at distance (R, R + shell]
 *       from the centre (minimum image),
 *   [1..3] slip velocity u_shell - v_p, where u_shell is the (1 - eps)
 *       weighted mean fluid velocity over the same nodes,
 *   [4] particle Reynolds number |slip| 2R / nu, nu = (tau - 1/2)/3,
 *   [5] density ratio rho_s / rho_fluid,
 * and target F_f / (6 pi rho_fluid nu R) (3D) or F_f / (4 pi rho_fluid nu)
 * (2D), with F_f the hydrodynamic force of the last step (Eq. 3).  u_dev and
 * eps_dev are device arrays from lbm_imb_fields(..., on_device = 1): u
 * [dim][N], eps [N].  feats [n][6], target [n][3]: device FP32, caller-owned,
 * cap >= n particles.  Enqueued on the handle's stream. */
int lbm_imb_drag_samples(lbm_imb_t* h, const double* u_dev, const double* eps_dev, double shell,
                         float* feats, float* target, int64_t cap);

/* The network: 6 -> 128 -> 128 -> 128 -> 128 -> 3, ReLU, BF16 tensor-core
 * products with FP32 accumulation, FP32 master weights trained by Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error of normalised
 * targets.  Inputs and outputs are normalised inside with the statistics set
 * by lbm_imb_mlp_set_normalization (identity until then).  Parameters
 * (FP32, flat): for each layer l = 1..5, W_l [out][in] then b_l [out]. */
typedef struct lbm_imb_mlp lbm_imb_mlp_t;

/* Device bytes for a network that trains on minibatches of up to max_batch. */
size_t lbm_imb_mlp_required_bytes(int64_t max_batch);
/* Lay out the network in the caller's device block (256-byte aligned), He
 * initial weights from seed.  Calls run on cuda_stream. */
int lbm_imb_mlp_init(void* dev_buf, size_t bytes, int64_t max_batch, uint64_t seed,
                     void* cuda_stream, lbm_imb_mlp_t** out);
int lbm_imb_mlp_num_params(int* n);
int lbm_imb_mlp_set_params(lbm_imb_mlp_t* m, const float* host_params);
int lbm_imb_mlp_get_params(lbm_imb_mlp_t* m, float* host_params);
int lbm_imb_mlp_set_normalization(lbm_imb_mlp_t* m, const float* x_mean, const float* x_std,
                                  const float* y_mean, const float* y_std);
/* y [n][3] (device) = network(x [n][6] device), denormalised.  Synchronises. */
int lbm_imb_mlp_predict(lbm_imb_mlp_t* m, const float* x, float* y, int64_t n);
/* Gradients of the minibatch loss w.r.t. the parameters (host, flat order)
 * and the loss, without changing the parameters. */
int lbm_imb_mlp_gradients(lbm_imb_mlp_t* m, const float* x, const float* t, int64_t batch,
                          float* host_grads, float* host_loss);
/* steps Adam steps on consecutive minibatches of the device dataset x [n][6],
 * t [n][3] (wrapping at the end); *last_loss = loss of the last minibatch. */
int lbm_imb_mlp_train_steps(lbm_imb_mlp_t* m, const float* x, const float* t, int64_t n,
                            int64_t batch, int64_t steps, float lr, float* last_loss);
int lbm_imb_mlp_destroy(lbm_imb_mlp_t* m);



/* One lattice decomposed along y into nslabs (2..16) slabs on this device,
 * exchanging halo rows after every collision: the multi-GPU design of the
 * paper (a subdomain per GPU, boundary populations passed to the
 * neighbours; "Numerical scheme", Fig. 2) emulated in one block.
 * Slab s computes ny_s rows (ny split as evenly as possible, the first
 * ny % nslabs slabs one row more; ny_s >= 2), stored between two halo rows.
 * Particles are shared by the slabs (each rasterises them into its rows and
 * adds its Eq. 3 sums), and the DEM runs once per step.  The handle steps
 * with lbm_imb_step and answers lbm_imb_particles / set_particles /
 * sync / steps_done; per-slab populations and fields come from the member
 * handles (lbm_imb_slab_member; local lattice of ny_s + 2 rows, row 0 and
 * row ny_s + 1 the halos; a halo row is current only in the directions that
 * cross into the slab, c_y = +1 below and c_y = -1 above).  2 <= nslabs
 * <= 16.  The collision uses form 0 for every slab.
 * dem_skin must be 0 (LBM_IMB_EUNSUPPORTED).  Device bytes from
 * lbm_imb_slabs_required_bytes (0 if the config is rejected; lbm_imb_slabs_init
 * with dev_buf = NULL then reports why). */
size_t lbm_imb_slabs_required_bytes(const lbm_imb_config* cfg, int nslabs);
int lbm_imb_slabs_init(const lbm_imb_config* cfg, int nslabs, void* dev_buf, size_t bytes,
                       void* cuda_stream, lbm_imb_t** out);
int lbm_imb_slab_member(lbm_imb_t* h, int i, lbm_imb_t** member);

/* ==================================================================
 * Test hooks.  Not part of the simulation interface: they expose one
 * internal piece each (a barrier's timeout path, the tensor-core operand
 * layout, the arctangent and the FP64 <-> pair conversions of the exact
 * covered fractions) so that tests can check it against a reference, and
 * one measures the FP64 pipe the FP64 collision is bound by.
 * ================================================================== */

/* Test hook for the barrier timeout path: poll limit of every barrier wait
 * (default 2^25 polls of ~64 ns) and a number of arrivals the barriers wait
 * for beyond the grid (0 in normal use; > 0 makes every wait run out). */
int lbm_imb_batch_set_barrier_test(lbm_imb_t* batch, int64_t spin_limit, int phantom_arrivals);

/* Test hook for the tensor-core operand layout: D [128][N] = A [128][K] *
 * B [N][K]^T with BF16 host inputs (raw bits, row-major) and FP32 host
 * output, through one tcgen05 product; dev_scratch >= 128 KB + 256,
 * 256-byte aligned; N, K in {16, 32, ..., 128}. */
int lbm_imb_mlp_probe_gemm(const uint16_t* a_host, const uint16_t* b_host, int N, int K,
                           float* d_host, void* dev_scratch, size_t scratch_bytes, void* stream);

/* Test hook for the first-quadrant arctangent of the exact-volume formulas
 * (FP64 rasterisation): for device arrays y, x [n] (y, x >= 0, not both
 * zero) writes the library's atan2 to fast [n] and CUDA's atan2 to ref [n]
 * (device arrays, caller-owned), then synchronises the stream.  n > 2^31
 * elements is not supported.  EINVAL on null pointers or n < 0. */
int lbm_imb_probe_atan2q1(const double* y, const double* x, double* fast, double* ref, int64_t n, void* stream);

/* Test hook for the FP64 <-> FP32-pair conversions of the pair storage
 * (LBM_IMB_STORE_DFDEV, covered nodes): for device arrays of n elements writes
 * to_double[i] = the FP64 value of the pair (h[i], l[i]) (|l| at most half
 * an FP32 ulp of h) and roundtrip[i] = d[i] split into a pair and converted
 * back, then synchronises the stream.  EINVAL on null pointers or n < 0. */
int lbm_imb_probe_df(const float* h, const float* l, const double* d, double* to_double, double* roundtrip,
                     int64_t n, void* stream);

/* Test hook for the FP64 pipe's throughput, the peak the FP64 collision is
 * measured against: one wave of resident 256-thread blocks on every SM (at
 * most sink_len threads; sink_len a multiple of 256; dev_sink holds one
 * double per thread, device, caller-owned), each thread running 16
 * independent chains of 16 * trips FP64 instructions of one kind (0 fused
 * multiply-add, 1 add, 2 multiply; the constant operands in the constant
 * bank, so that register-file bandwidth does not cap the rate); one
 * warm-up launch, then one launch
 * timed with CUDA events on `stream`.  *gops = instructions per second /
 * 1e9 (over all threads), *ms_out (may be NULL) the timed launch's
 * duration.  Synchronises the stream.  EINVAL on bad sizes, kind or
 * pointers. */
int lbm_imb_probe_fp64_rate(double* dev_sink, int64_t sink_len, int64_t trips, int kind, double* gops,
                            double* ms_out, void* stream);

/* Release the handle (its CUDA graphs and host state).  The caller's device
 * block is not touched. */
int lbm_imb_destroy(lbm_imb_t* h);

/* Static description of a status code. */
const char* lbm_imb_strerror(int status);

/* Library version string. */
const char* lbm_imb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_IMB_H */
