/*
 * lbe.h — C ABI of the GB300 (sm_103a) lattice Boltzmann library.
 *
 * The library runs the time step of §2 of Günther, Janoschek, Frijters,
 * Harting, "Lattice Boltzmann simulations of anisotropic particles at liquid
 * interfaces" (arXiv:1109.3277): a two-component Shan–Chen D3Q19 BGK fluid
 * (Eq. 1–3) coupled to rigid ellipsoids by moving bounce-back (Eq. 4) with
 * momentum exchange (Eq. 5), anisotropic Hertz and lubrication pair forces
 * (Eq. 6–9), outer-shell density fill and particle colour (Eq. 10 and the
 * colour rule after it), all on one GPU.
 *
 * Conventions
 *  - Lattice units: spacing and time step 1, c_s^2 = 1/3.  Node (x,y,z) sits
 *    at position (x,y,z); node index n = x + nx*(y + ny*z).
 *  - Component 0 is "red", component 1 is "blue".
 *  - A particle's symmetry axis is its body x axis; quaternions are
 *    (w, x, y, z) and rotate body vectors into the lab frame.
 *  - Ownership: the caller owns every host pointer; the library copies
 *    inputs and writes outputs into caller buffers.  Each lbe_ctx owns all
 *    device memory it allocates and frees it in lbe_destroy.
 *  - Errors: every call returns an lbe_status; nothing aborts and no C++
 *    exception crosses the ABI.  An invalid argument leaves the context
 *    unchanged.  lbe_last_error() gives a one-line message.
 *  - Streams: work is enqueued on the descriptor's cuda_stream (a
 *    cudaStream_t; NULL makes the library create its own stream).
 *    lbe_step returns once the work is enqueued; lbe_read_*, lbe_mass and
 *    lbe_get_populations synchronise that stream and report any deferred
 *    device error.
 */
#ifndef LBE_H
#define LBE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LBE_API __attribute__((visibility("default")))
#else
#define LBE_API
#endif

typedef struct lbe_ctx lbe_ctx;

typedef enum {
    LBE_OK = 0,
    LBE_EINVAL = -1,   /* invalid argument; nothing changed */
    LBE_ENOMEM = -2,   /* device or host allocation failed */
    LBE_ECUDA = -3,    /* a CUDA call failed; see lbe_last_error */
    LBE_ENUMERIC = -4, /* non-finite or negative density detected */
    LBE_EOVERLAP = -5, /* reserved */
    LBE_ETIMEOUT = -6, /* a bounded wait ran out */
    LBE_EBUSY = -7     /* the request cannot be taken now (serving) */
} lbe_status;

/* Population storage.  Arithmetic is FP32 in every mode; the 16-bit modes
 * store δf = f - w_i rho_ref^c and halve the population bytes. */
typedef enum {
    LBE_STORE_F32 = 0,
    LBE_STORE_BF16_OFS = 1,
    LBE_STORE_F16_OFS = 2
} lbe_storage;

/* Particle motion. */
typedef enum {
    LBE_PARTICLES_FREE = 0,       /* Newton–Euler under fluid + pair forces */
    LBE_PARTICLES_STATIC = 1,     /* geometry fixed; V, ω still enter Eq. 4 */
    LBE_PARTICLES_PRESCRIBED = 2  /* V and lab-frame ω held constant, geometry moves */
} lbe_particle_mode;

typedef struct {
    int32_t nx, ny, nz;      /* lattice extent, each >= 1, ny and nz <= 65535, nx*ny*nz < 2^31
                                (nz >= 3 with walls) */
    int32_t walls_z;         /* 0: periodic in z; 1: one-node walls at z=0 and z=nz-1
                                (the impenetrable walls of the §4 adsorption box) */
    double  tau[2];          /* BGK relaxation time per component, > 1/2 (Eq. 2) */
    double  g_br;            /* Shan–Chen coupling of Eq. 3; > 0 demixes (§4: 0.1, 0.08) */
    double  body_force[3];   /* extra force per unit density on every fluid node */
    double  rho_ref[2];      /* 16-bit offset base per component; also the density given
                                to a node uncovered with no fluid neighbour */
    int32_t storage;         /* lbe_storage */
    int32_t particle_mode;   /* lbe_particle_mode */
    double  k_hertz;         /* K_H of the Hertz potential (§2: 100) */
    double  lub_cut;         /* Δc of the lubrication correction (§2: 2/3); 0 disables it */
    double  lub_rho;         /* density in μ = ν ρ of the lubrication correction */
    void   *cuda_stream;     /* cudaStream_t to enqueue on (of the chosen device), or NULL */
    int32_t device;          /* CUDA device ordinal; -1 = the library's current device */
    int32_t flags;           /* 0, or LBE_FLAG_TWO_PASS | LBE_FLAG_WIDE_OFFSETS */
    double  rho_particle;    /* particle mass density (mass ρ_p times the ellipsoid's volume,
                                solid-ellipsoid inertia); the paper gives none; 0 means 1 */
} lbe_lattice_desc;

/* Run the fluid update as two passes (densities and ψ of every node to
 * memory, then collide+stream) instead of the fused single pass.  Same
 * results up to FP32 rounding; kept as the comparison point of the fused
 * kernel. */
#define LBE_FLAG_TWO_PASS 1

/* The fused kernel addresses its stores with 32-bit offsets from the node's
 * component where they fit (19 x the slot stride + 2 N < 2^32, lattices up
 * to about 214 M nodes) and with 64-bit offsets otherwise.  This flag takes
 * the 64-bit form on any lattice: same results, bit for bit (for tests). */
#define LBE_FLAG_WIDE_OFFSETS 2

/* Create a lattice on the current CUDA device with populations at the rest
 * equilibrium f_i^c = w_i rho0^c (Eq. 2 at u = 0).
 *  rho0: host, double [2][nz][ny][nx], caller-owned, copied; values on wall
 *        nodes are ignored.
 * Returns LBE_EINVAL for a bad descriptor, LBE_ENOMEM if device memory runs
 * out (nothing is kept), LBE_ECUDA for other CUDA failures. */
LBE_API lbe_status lbe_init_lattice(const lbe_lattice_desc *d, const double *rho0, lbe_ctx **out);

/* Add n rigid ellipsoids (§2: radius r_par along the symmetry axis, r_perp
 * across it; colour delta_rho, the surface-density parameter of the
 * wettability rule).  Host arrays, caller-owned, copied:
 *  pos [n][3] (inside the lattice), quat [n][4] (normalised on entry),
 *  vel [n][3] and omega [n][3] (lab frame; NULL = zero),
 *  r_par [n], r_perp [n] (> 0), delta_rho [n].
 * Non-wall nodes inside a particle become solid (a node inside several
 * particles belongs to the lowest index); their fluid is discarded. */
LBE_API lbe_status lbe_add_particles(lbe_ctx *c, int32_t n, const double *pos, const double *quat,
                             const double *vel, const double *omega, const double *r_par,
                             const double *r_perp, const double *delta_rho);

/* Advance nsteps time steps (Eq. 1 per step, with every coupling above),
 * asynchronously on the context's stream. */
LBE_API lbe_status lbe_step(lbe_ctx *c, int32_t nsteps);

/* Read the current fields (synchronises).  Host outputs, any may be NULL:
 *  rho  double [2][N]: ρ^c on fluid nodes, 0 on solid nodes;
 *  vel  double [3][N]: (Σ_c j^c + ½ Σ_c F^c) / Σ_c ρ^c on fluid nodes, 0 on solid;
 *  node_type uint8 [N]: 0 fluid, 1 wall, 2 particle. */
LBE_API lbe_status lbe_read_fields(lbe_ctx *c, double *rho, double *vel, uint8_t *node_type);

/* Read the particle state (synchronises).  Host outputs, each n*k doubles or
 * NULL: pos, quat (w,x,y,z), vel, omega (lab), force and torque = the total
 * of the last update (momentum exchange + pair forces + fill/empty). */
LBE_API lbe_status lbe_read_particles(lbe_ctx *c, double *pos, double *quat, double *vel, double *omega,
                              double *force, double *torque);

/* Per-component fluid mass Σ_x Σ_i f_i^c over fluid nodes (synchronises).
 * Each node's 19 FP32 populations are summed error-free (TwoSum) and the
 * node sums are added in FP64 in a fixed order. */
LBE_API lbe_status lbe_mass(lbe_ctx *c, double out[2]);

/* Raw populations f[2][19][N] as doubles (synchronises / uploads).  Solid
 * nodes hold unspecified values. */
LBE_API lbe_status lbe_get_populations(lbe_ctx *c, double *f);
LBE_API lbe_status lbe_set_populations(lbe_ctx *c, const double *f);

/* Per-kernel timing with CUDA events on the context's stream.  When enabled,
 * every launch of the dominant fluid kernel is bracketed by events;
 * lbe_profile_read returns the summed milliseconds and the launch count
 * since the last enable, and synchronises. */
LBE_API lbe_status lbe_profile_enable(lbe_ctx *c, int32_t enable);
LBE_API lbe_status lbe_profile_read(lbe_ctx *c, double *ms_total, int64_t *launches);

/* Number of kernels one lbe_step(c, 1) enqueues (for launch accounting). */
LBE_API int32_t lbe_kernels_per_step(const lbe_ctx *c);

/* Device bytes held by the context. */
LBE_API size_t lbe_device_bytes(const lbe_ctx *c);

/* Allocation-free FP64 mass sums.  The paper has no counterpart: this entry
 * point exists for callers that keep their populations in memory they manage
 * themselves and cannot call cudaMalloc (a fixed device-memory budget, a
 * memory pool owned by another framework, or a place in their program where
 * an allocation's implicit synchronisation is not allowed).  It computes the
 * same per-component sums as lbe_mass, but on caller-owned buffers, and it
 * allocates nothing: its per-block partial sums live in a fixed 16 KiB array
 * (2 x 1024 doubles) that the library keeps on every GPU that loads it until
 * the process exits.
 *  f:         device pointer, the library's population layout: the two
 *             components of direction i at node n side by side, component c
 *             at element 2 * (i * slot_stride + n) + c (elements of the
 *             storage type; the 16-bit modes hold f - w_i rho_ref[c]);
 *  node_type: device pointer, [nodes] bytes, 0 = fluid (summed), others skipped;
 *  rho_ref:   host pointer to 2 doubles (ignored for LBE_STORE_F32);
 *  out:       device pointer to 2 doubles, written in stream order;
 *  device:    CUDA device ordinal, or -1 for the caller's current device;
 *             the caller's current device is the same on return;
 *  cuda_stream: the cudaStream_t to enqueue on (NULL = legacy default).
 * Returns LBE_EINVAL for a null pointer, nodes < 1 or nodes >
 * LBE_NOALLOC_MAX_NODES, slot_stride < nodes, device < -1 or an unknown
 * storage mode; LBE_ECUDA if a CUDA call fails.  The first call on a device
 * looks up the device address of the fixed array (cudaGetSymbolAddress):
 * make that first call before any stream capture.  The address stays cached
 * for the life of the process and does not survive a cudaDeviceReset of
 * that device.  All calls share the one array, so calls that overlap on the
 * GPU (other streams, other threads) race and must be ordered by the
 * caller. */
#define LBE_NOALLOC_MAX_NODES 2147483647LL
LBE_API lbe_status lbe_mass_noalloc(const void *f, int32_t storage, const uint8_t *node_type,
                                    int64_t nodes, int64_t slot_stride, const double rho_ref[2],
                                    int32_t device, void *cuda_stream, double *out);

/* Pick the fused kernel's tile height and z-chunk length for this lattice
 * by timing the candidates (heights 8 and, where built, 4, times chunks
 * 4, 8, 16, ... and the full height) with CUDA events on the current state
 * (which is not changed); later steps use the fastest.  *chosen_zc (may be
 * NULL) receives the chunk; lbe_get_tile gives both. */
LBE_API lbe_status lbe_autotune(lbe_ctx *c, int32_t *chosen_zc);

/* Set the fused kernel's z-chunk length (planes per CTA; 0 restores the
 * default, sized for about 16 waves of CTAs).  A chunk longer than the
 * lattice is clipped.  Only the order in which tiles run depends on it,
 * never a result.  Synchronises first (and returns a pending error of
 * earlier steps).  LBE_EINVAL for a negative length. */
LBE_API lbe_status lbe_set_zchunk(lbe_ctx *c, int32_t zc);

/* The fused kernel's tile: 32 nodes wide and rows = 4 or 8 rows high (4 is
 * built for τ = 1 lattices with TMA copies; others take 8), walking a z
 * chunk of zc planes (0: the default for the lattice).  lbe_autotune picks
 * both; lbe_set_tile fixes them (synchronises first, LBE_EINVAL for other
 * heights or a negative chunk) and lbe_get_tile reads the ones in use
 * (0, 0 with LBE_FLAG_TWO_PASS).  Only the order in which nodes are
 * visited depends on them, never a result. */
LBE_API lbe_status lbe_set_tile(lbe_ctx *c, int32_t rows, int32_t zc);
LBE_API lbe_status lbe_get_tile(const lbe_ctx *c, int32_t *rows, int32_t *zc);

/* Failure detection of the fused kernel's copies: every wait for a plane's
 * box copy gives up after a bounded number of tries (a non-blocking look,
 * then about 2^22 tries by default, each of which may suspend the thread
 * for a while).  The CTA then stops, waits with the default bound for its
 * copies in flight, and sets the lattice's status word; the next
 * synchronising call returns LBE_ETIMEOUT.  lbe_set_wait_limit sets the
 * number of tries (0 restores the default); with unreachable != 0 every
 * wait is for a barrier phase that no copy completes, so that tests can
 * make the wait run out without any fault.  A run that timed out has left
 * the populations of the step partly written.  Synchronises first;
 * LBE_EINVAL for a negative count. */
LBE_API lbe_status lbe_set_wait_limit(lbe_ctx *c, int32_t tries, int32_t unreachable);

/* Failure detection of allocations (for tests): the next `after` device
 * allocations of the library succeed and every later one fails as if the
 * device were out of memory, until lbe_fail_allocations(-1).  A call that
 * meets the failure returns LBE_ENOMEM and frees what it had allocated
 * (lbe_init_lattice keeps nothing; lbe_add_particles keeps the context as
 * it was); a server request whose lattice cannot be created fails with
 * LBE_ENOMEM and releases its share of the server's budget.  Process-wide. */
LBE_API void lbe_fail_allocations(int32_t after);

/* Batches: several lattices stepped together, every kernel of the step
 * covering all of them in one launch (the fused fluid kernel as a persistent
 * kernel taking tiles of all boxes from one queue), replayed as a captured
 * CUDA graph on a stream of the batch's own, ordered by events after the
 * members' earlier work and before their later work.  Members must share
 * device and storage mode, must not
 * use LBE_FLAG_TWO_PASS, and must not change (add particles) while the
 * batch exists; the batch does not own them.  After lbe_batch_step the
 * members are read with the usual calls.  Every member's populations and
 * particles are bit-identical to those of stepping it alone with lbe_step,
 * whatever else is in the batch.  The pair forces run one thread per
 * particle over the member's particles, so members are limited to
 * LBE_BATCH_MAX_PARTICLES particles each (LBE_EINVAL beyond). */
#define LBE_BATCH_MAX_PARTICLES 4096
typedef struct lbe_batch lbe_batch;
LBE_API lbe_status lbe_batch_create(lbe_ctx *const *members, int32_t n, lbe_batch **out);
LBE_API lbe_status lbe_batch_step(lbe_batch *b, int32_t nsteps);
/* Pick the persistent CTAs per SM of the batched fused kernel by timing. */
LBE_API lbe_status lbe_batch_autotune(lbe_batch *b, int32_t *chosen_ctas_per_sm);
/* Kernels of this library one batched step launches (0 if b is NULL). */
LBE_API int32_t lbe_batch_kernels_per_step(const lbe_batch *b);
LBE_API void lbe_batch_destroy(lbe_batch *b);

/* Device bytes a context with descriptor d and nparticles particles holds
 * at most (populations, fields, maps, particle state, and the transient
 * buffer of the initial densities); 0 for an invalid descriptor.  Used for
 * admission by HBM footprint. */
LBE_API size_t lbe_footprint(const lbe_lattice_desc *d, int32_t nparticles);

/* Orientation (w, x, y, z) of the first particle of every member, in the
 * order the members were given to lbe_batch_create (zeros for members
 * without particles): one gather kernel and one copy; synchronises the
 * batch's stream.  quat_out holds 4 doubles per member. */
LBE_API lbe_status lbe_batch_first_quat(lbe_batch *b, double *quat_out);

/* ---- Serving: single-particle adsorption requests (§4 of the paper: an
 * ellipsoid released at a flat interface, run until its tilt settles) with
 * continuous batching.
 *
 * A server owns one worker thread on the device current at creation.  Its
 * loop admits queued requests in arrival order while fewer than max_slots
 * run and the sum of their lbe_footprint stays within hbm_budget_bytes
 * (setting up new lattices while the running ones step on the GPU), steps
 * all running boxes as one batch in chunks of 100 steps, and after each
 * chunk retires every box whose first particle's tilt (angle of its body x
 * axis to z, radians) changed by less than tilt_tol over the chunk, or
 * that reached max_steps (rounded up to a multiple of 100).  A request's
 * result is bit-identical to running it alone.  The server's storage mode
 * replaces the descriptor's; the descriptor's stream, device and flags are
 * ignored.
 *
 * particle_blob: per particle LBE_PARTICLE_IN doubles,
 *   pos[3], quat[4] (w,x,y,z), vel[3], omega[3], r_par, r_perp, delta_rho.
 * particle_out:  per particle LBE_PARTICLE_OUT doubles,
 *   pos[3], quat[4], vel[3], omega[3], force[3], torque[3]
 *   (the state after the last step, as lbe_read_particles gives it).
 * Host buffers are the caller's; submit copies its inputs.
 * lbe_server_submit: LBE_ENOMEM if the request alone exceeds the budget.
 * lbe_server_poll: *done = 1 once the request finished; a failed request
 *   returns its error status (LBE_ENUMERIC if its particle state is not
 *   finite at the end: the run diverged).  LBE_EINVAL for an unknown id.
 * lbe_server_wait: block until the request finished or timeout_ms passed
 *   (LBE_ETIMEOUT).
 * lbe_server_timing: seconds from submission to admission and to the end
 *   (LBE_EBUSY while it runs).
 * lbe_server_stats: out = {completed requests, lattice node updates done,
 *   most boxes run at once, chunks run}.
 * lbe_server_destroy: stops after the chunk in flight; unfinished requests
 *   are dropped. */
#define LBE_PARTICLE_IN 16
#define LBE_PARTICLE_OUT 19
typedef struct lbe_server lbe_server;
LBE_API lbe_status lbe_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t storage, lbe_server **out);
LBE_API lbe_status lbe_server_submit(lbe_server *s, const lbe_lattice_desc *d, const double *rho0, int32_t nparticles,
                                     const double *particle_blob, int32_t max_steps, double tilt_tol,
                                     uint64_t *req_id);
LBE_API lbe_status lbe_server_poll(lbe_server *s, uint64_t req_id, int32_t *done, int32_t *steps_run,
                                   double *particle_out);
LBE_API lbe_status lbe_server_wait(lbe_server *s, uint64_t req_id, int32_t timeout_ms);
LBE_API lbe_status lbe_server_timing(lbe_server *s, uint64_t req_id, double *queued_s, double *latency_s);
LBE_API lbe_status lbe_server_stats(lbe_server *s, int64_t out[4]);
LBE_API void lbe_server_destroy(lbe_server *s);

LBE_API const char *lbe_last_error(const lbe_ctx *c);
LBE_API void lbe_destroy(lbe_ctx *c);

#ifdef __cplusplus
}
#endif
#endif
