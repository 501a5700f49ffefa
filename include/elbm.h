/*
 * elbm.h -- C ABI of the GB300 (sm_103a) entropic lattice Boltzmann library.
 *
 * The library advances a periodic lattice by the ELBM update, Eq. (1) of
 * Zhao & Yong, "Relaxation-rate formula for the entropic lattice Boltzmann
 * method":
 *     f_i(x + c_i, t + 1) = f_i(x, t) + alpha beta (f^eq_i(x, t) - f_i(x, t)),
 * with beta = c_s^2 / (2 nu + c_s^2) (Eq. (2), dt = 1, c_s^2 = 1/3), f^eq the
 * minimiser of H(f) = sum_i f_i ln(f_i / W_i) (Eq. (3)) under the mass and
 * momentum constraints, and alpha chosen per node by
 *   ELBM_ALPHA_FORMULA: alpha_* = min(2, alpha_max) (Eq. (8)) when
 *                       H(f*(alpha_*)) <= H(f), else Eq. (9);
 *   ELBM_ALPHA_ROOT:    the bisection root of H(f + alpha (f^eq - f)) = H(f)
 *                       (Eq. (4)) on [1, alpha_max], stopped when
 *                       -1e-13 <= H(f*(alpha)) - H(f) <= 0 (the comparison
 *                       method of the paper's double-shear-layer experiment);
 *   ELBM_ALPHA_SECANT:  the modified secant iteration of the paper's
 *                       conclusion, whose first iterate is Eq. (9).
 *
 * Conventions
 *   - Lattice units: dt = 1, c_s^2 = 1/3.  Periodic boundaries on all axes.
 *   - Velocity ordering (index: velocity), rest first, then +/- pairs:
 *       D2Q9:  0 (0,0)  1 (1,0)  2 (-1,0)  3 (0,1)  4 (0,-1)
 *              5 (1,1)  6 (-1,-1) 7 (1,-1) 8 (-1,1)
 *       D3Q27: 0 (0,0,0); faces 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0)
 *              5 (0,0,1) 6 (0,0,-1); edges 7 (1,1,0) 8 (-1,-1,0)
 *              9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1)
 *              14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1);
 *              corners 19 (1,1,1) 20 (-1,-1,-1) 21 (1,1,-1) 22 (-1,-1,1)
 *              23 (1,-1,1) 24 (-1,1,-1) 25 (-1,1,1) 26 (1,-1,-1)
 *     Weights are products of the D1Q3 weights {2/3, 1/6, 1/6}.
 *   - Field layouts (all x fastest): scalar fields [nz][ny][nx]; velocity
 *     [d][nz][ny][nx] with d = 2 (D2Q9) or 3 (D3Q27); populations
 *     [Q][nz][ny][nx].  2D lattices use nz = 1.
 *   - "Step n" state is the pre-collision f^n (left-hand side of Eq. (1) at
 *     t = n).  Readouts (moments, populations) return f^n.
 *   - Every host pointer argument is a caller-owned HOST buffer unless the
 *     name ends in _device; the library copies from/to it and keeps no
 *     reference.  Device buffers are owned by the handle.
 *   - Every call returns an elbm_status; no exception or abort crosses the
 *     ABI.  elbm_step is asynchronous on the handle's stream; the calls that
 *     return data synchronise that stream and report errors the kernels
 *     flagged (ELBM_ENEGATIVE for a population <= 0, ELBM_ENONFINITE for a
 *     NaN/Inf or |u| >= 1); after such an error the state is undefined until
 *     the next elbm_init_fields / elbm_set_populations.
 *   - Threading: a handle is used by one host thread at a time.
 */
#ifndef ELBM_H
#define ELBM_H

#include <stddef.h>

#if defined(__GNUC__)
#define ELBM_API __attribute__((visibility("default")))
#else
#define ELBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elbm_handle elbm_handle;

/* Velocity sets: D2Q9 and D3Q27 are tensor products of D1Q3 (velocities
 * {0, +1, -1}, weights {2/3, 1/6, 1/6}); D1Q3 itself serves one-dimensional
 * problems such as the shock tube of Fig. 2 (nx nodes, ny = nz = 1, FP64
 * storage only; the batched and static entry points take D2Q9 and D3Q27). */
typedef enum { ELBM_D2Q9 = 0, ELBM_D3Q27 = 1, ELBM_D1Q3 = 2 } elbm_lattice;

/* Storage (and arithmetic) of the populations.
 *   ELBM_FP64          f_i in FP64, FP64 arithmetic throughout.
 *   ELBM_FP32          f_i in FP32.
 *   ELBM_FP32_SHIFTED  delta_i = f_i - W_i rho0 in FP32 (rho0 a per-handle
 *                      constant, the FP32-rounded mean initial density).
 *   ELBM_FP16_SHIFTED  delta_i 2^k_i in IEEE binary16, k_i = round(log2(1/W_i))
 *                      (D2Q9: 1, 3, 5; D3Q27: 2, 4, 6, 8 for 0..3 nonzero
 *                      velocity components); the shift W_i rho0 stays a
 *                      per-handle constant.  Each stored value is rounded
 *                      to nearest once per step (relative 2^-11), so mass
 *                      and momentum are conserved to that rounding only.
 * FP32 and FP16 storages compute FORMULA in FP32 with a certified error bound
 * on the entropy differences (see elbm_step) applied to the values as
 * loaded; ROOT and SECANT, and nodes far from equilibrium, are computed in
 * FP64 from the stored values. */
typedef enum {
  ELBM_FP64 = 0,
  ELBM_FP32 = 1,
  ELBM_FP32_SHIFTED = 2,
  ELBM_FP16_SHIFTED = 3
} elbm_dtype;

typedef enum {
  ELBM_ALPHA_FORMULA = 0,
  ELBM_ALPHA_ROOT = 1,
  ELBM_ALPHA_SECANT = 2
} elbm_alpha_mode;

/* How FP32 / FP16 FORMULA steps decide a node whose FP32 entropy test is
 * not certified (the sign of Delta H(2) or Delta H(1) within the FP32 error
 * bound).
 *   ELBM_DECISION_EXACT (default): a second stage recomputes f^eq - f in
 *     double-float arithmetic and retakes the acceptance test after Eq. (8)
 *     and Eq. (9) with that error bound (then with the leading terms of
 *     Delta H(2) in double-float as well, and FP64 for the rare node still
 *     undecided), so every node takes the branch the exact arithmetic
 *     takes and an Eq. (9) alpha lies within 2^-16 of the chord of the
 *     stored state: alpha and the Fig. 5 counter are the paper's.  Costs
 *     about 10 % per step on developed 3D flows, more where most nodes are
 *     within FP32 noise of equilibrium (the first step after
 *     elbm_init_fields; thin shear layers).
 *   ELBM_DECISION_CERTIFIED: such a node keeps the certified alpha -- the
 *     Eq. (9) chord on the upper bounds, rounded down, or 1 when no chord
 *     is certified -- which also satisfies H(f*(alpha)) <= H(f) but may
 *     take the other branch than the exact arithmetic; faster (no second
 *     stage).
 * FP64 storage and the ROOT / SECANT modes are unaffected. */
typedef enum {
  ELBM_DECISION_EXACT = 0,
  ELBM_DECISION_CERTIFIED = 1
} elbm_decision;

typedef enum {
  ELBM_OK = 0,
  ELBM_EINVAL = 1,      /* invalid argument                                */
  ELBM_ENOMEM = 2,      /* device allocation failed                        */
  ELBM_ECUDA = 3,       /* CUDA runtime error (message in elbm_last_error) */
  ELBM_ENONFINITE = 4,  /* a node had NaN/Inf moments or |u_a| >= 1        */
  ELBM_ENEGATIVE = 5,   /* a node had a population <= 0                    */
  ELBM_EROOT_CAP = 6,   /* ROOT bisection stopped at its iteration cap at
                           one or more nodes of the reported step (returned
                           by elbm_entropy_stats after filling *out)       */
  ELBM_ESTATE = 7       /* call not valid in the handle's state            */
} elbm_status;

/* Diagnostics of one step (the step that maps f^n to f^{n+1}): moments and
 * entropy of f^n and counters of the collisions performed. */
typedef struct {
  long long step;           /* n                                          */
  long long n_nodes;
  double mass;              /* sum_x rho                                  */
  double momentum[3];       /* sum_x rho u                                */
  double kinetic_energy;    /* 1/2 sum_x rho |u|^2                        */
  double alpha_min, alpha_max, alpha_sum;
  long long n_accept_two;   /* alpha_* = 2 accepted (Fig. 5 counter)      */
  long long n_accept_star;  /* alpha_* accepted (any alpha_*)             */
  long long n_formula;      /* Eq. (9) / secant / root alpha used         */
  long long n_band;         /* FP32 FORMULA: FP32 decision not certified,
                               decided by the double-float second stage   */
  long long n_far;          /* FP32 FORMULA: node solved in FP64 (far from
                               equilibrium, invalid, or undecided by the
                               second stage and its double-float series
                               pass)                                      */
  long long n_degenerate;   /* f^eq == f: alpha = 2                       */
  long long n_root_iters;   /* ROOT/SECANT iterations                     */
  long long n_root_cap;     /* ROOT stopped at the iteration cap          */
  long long n_no_root;      /* ROOT: Delta H(alpha_max) <= 0, alpha_max   */
  int checked;              /* 1: the FP64 check below was evaluated      */
  int reserved;
  double h_total;           /* sum_x H(f^n(x)), Eq. (3), FP64             */
  long long n_violations;   /* nodes with Delta H(alpha) above its FP64
                               rounding bound (Eq. (7) violated)          */
  long long n_decision_mismatch; /* FP32 accept/formula decision differs
                               from the FP64 one (nodes where f = f^eq at
                               the evaluation's precision -- the update
                               is the identity for every alpha -- are
                               not compared)                              */
  double alpha_dev_max;     /* max |alpha - alpha_FORMULA in FP64|        */
} elbm_entropy_stats_t;

/* Create a handle for a periodic nx x ny x nz lattice (nz = 1 for D2Q9,
 * ny = nz = 1 for D1Q3) of viscosity nu > 0 (beta from Eq. (2)).  A D1Q3
 * handle with another storage than ELBM_FP64 is ELBM_EINVAL.  No device
 * memory is touched until elbm_init_fields / elbm_set_populations.  *out is
 * NULL on failure. */
ELBM_API elbm_status elbm_create(elbm_handle **out, elbm_lattice lattice, int nx,
                        int ny, int nz, double nu, elbm_dtype dtype);

/* Destroy a handle and free its device buffers (synchronises its stream). */
ELBM_API void elbm_destroy(elbm_handle *h);

/* Message of the last failed call on h (or of the last failed elbm_create
 * when h is NULL).  Valid until the next call on h. */
ELBM_API const char *elbm_last_error(const elbm_handle *h);

/* Run the handle's work on the given cudaStream_t (NULL: legacy default
 * stream).  The caller keeps ownership of the stream. */
ELBM_API elbm_status elbm_set_stream(elbm_handle *h, void *cuda_stream);

/* Device memory callbacks used for every buffer the handle allocates
 * (NULL alloc: cudaMalloc/cudaFree).  Valid only before the first
 * allocation (ELBM_ESTATE otherwise). */
ELBM_API elbm_status elbm_set_allocator(elbm_handle *h,
                               void *(*alloc)(size_t bytes, void *ctx),
                               void (*free_fn)(void *ptr, void *ctx),
                               void *ctx);

/* Diagnostics schedule: fused statistics on steps n with n % diag_every == 0
 * (0: never), the FP64 entropy/violation check on steps with
 * n % check_every == 0 (0: never), alpha map written on steps with
 * n % alpha_map_every == 0 (0: never), and the iteration count of
 * ELBM_ALPHA_SECANT (>= 1).  Defaults: 1, 0, 0, 4. */
ELBM_API elbm_status elbm_set_diagnostics(elbm_handle *h, int diag_every,
                                 int check_every, int alpha_map_every,
                                 int secant_iters);

/* Decision mode of the FP32 / FP16 FORMULA steps (elbm_decision above).
 * Takes effect from the next elbm_step. */
ELBM_API elbm_status elbm_set_decision(elbm_handle *h, elbm_decision decision);

/* f^0 = f^eq(rho, u) at every node.  rho: [nz][ny][nx] > 0,
 * u: [d][nz][ny][nx] with |u_a| < 1, FP64 host buffers.  Resets the step
 * counter to 0 and sets rho0 to the FP32-rounded mean of rho.
 * Page-locked host buffers (cudaHostAlloc, cudaHostRegister, pinned
 * framework tensors) are read by the init kernels directly over the host
 * link; pageable ones go through a device staging buffer of (1 + d) x n
 * doubles, allocated by the first such call of elbm_init_fields,
 * elbm_moments or elbm_enstrophy and kept (and reused) until
 * elbm_destroy.  Synchronises. */
ELBM_API elbm_status elbm_init_fields(elbm_handle *h, const double *rho,
                             const double *u);
/* Same with device pointers (on the handle's device, FP64). */
ELBM_API elbm_status elbm_init_fields_device(elbm_handle *h, const double *rho_device,
                                    const double *u_device);

/* Set the pre-collision state f^n from FP64 populations [Q][nz][ny][nx]
 * (host), rounded to the storage type.  Resets the step counter to 0. */
ELBM_API elbm_status elbm_set_populations(elbm_handle *h, const double *f);

/* Advance nsteps >= 0 steps of Eq. (1) with the given alpha mode.
 * Asynchronous on the handle's stream.
 * FP32 FORMULA: Delta H(2) and Delta H(1) are evaluated in FP32 from the
 * moments sum_i f_i x_i^k (k = 2..4, or 2..8 when max|x_i| > 1/100) with a
 * bound E on their error.  alpha = 2 is accepted when Delta H(2) + E <= 0
 * (the acceptance test after Eq. (8)); the Eq. (9) chord, evaluated on the
 * upper bounds and rounded down, is taken when Delta H(2) - E > 0 and
 * Delta H(1) + E < 0.  A node where either sign lies within E is
 * recomputed in double-float arithmetic (f^eq - f to about 1e-12 of f) and
 * decided again with that smaller error; the rare node still undecided is
 * solved in FP64.  So each node takes the branch of the exact arithmetic
 * and H(f*(alpha)) <= H(f) holds for the stored state.  Nodes with
 * max|x_i| > 1/8, |u_a| >= 1/4 or invalid populations are solved in FP64.
 * FP32 and FP16 storages take fewer than 2^31 nodes. */
ELBM_API elbm_status elbm_step(elbm_handle *h, long long nsteps, elbm_alpha_mode mode);

/* Block until the handle's queued work is done; reports flagged errors. */
ELBM_API elbm_status elbm_sync(elbm_handle *h);

/* Density [nz][ny][nx] and velocity [d][nz][ny][nx] of f^n (host, FP64):
 * rho = sum_i f_i and rho u = sum_i c_i f_i, the mass and momentum moments
 * that the equilibrium of Eq. (3) conserves (the constraints stated after
 * Eq. (3)).  Either pointer may be NULL.  When both are page-locked host
 * buffers the kernel writes them directly; otherwise through the staging
 * buffer (elbm_init_fields).  Synchronises. */
ELBM_API elbm_status elbm_moments(elbm_handle *h, double *rho_out, double *u_out);

/* Populations f^n as FP64 [Q][nz][ny][nx] (host).  Synchronises. */
ELBM_API elbm_status elbm_get_populations(elbm_handle *h, double *f_out);

/* Populations f^n of `count` nodes (flat indices (z ny + y) nx + x), written
 * as f_out[k * Q + i] (host).  Synchronises. */
ELBM_API elbm_status elbm_get_populations_nodes(elbm_handle *h, const long long *nodes,
                                       int count, double *f_out);

/* Per-node alpha [nz][ny][nx] (FP32, host) of the last step that wrote the
 * alpha map (ELBM_ESTATE if none did): the relaxation parameter of Eq. (1)
 * chosen by the step's alpha mode, the field the paper shows for the
 * double shear layer in Fig. 4.  Synchronises. */
ELBM_API elbm_status elbm_alpha_map(elbm_handle *h, float *alpha_out);

/* Diagnostics of the last step that computed them (ELBM_ESTATE if none):
 * mass, momentum and kinetic energy of f^n; the total entropy of Eq. (3)
 * and the count of nodes whose collision raised H beyond rounding (the
 * local H-theorem of Eq. (7), whose sum over the lattice is Eq. (6)); the
 * count of nodes accepting alpha = 2 (the proportion plotted in Fig. 5);
 * and the alpha-selection counters.  Synchronises.  Returns
 * ELBM_EROOT_CAP, with *out filled, when ROOT bisection stopped at its
 * iteration cap at one or more nodes of that step. */
ELBM_API elbm_status elbm_entropy_stats(elbm_handle *h, elbm_entropy_stats_t *out);

/* Enstrophy 1/2 <|omega|^2> of f^n: omega = curl u by second-order central
 * differences on the periodic lattice (2D: omega_z), averaged over nodes;
 * 0 for D1Q3, whose velocity field has no curl.  Synchronises. */
ELBM_API elbm_status elbm_enstrophy(elbm_handle *h, double *out);

/* Steps taken since the last initialisation. */
ELBM_API long long elbm_step_count(const elbm_handle *h);

/* Bytes of device memory held by the handle. */
ELBM_API size_t elbm_device_bytes(const elbm_handle *h);

/* Number of CUDA kernel launches issued by the library in this process
 * (all handles).  Used to account the work of a timed region. */
ELBM_API long long elbm_launch_count(void);

/* Record CUDA events (on the handle's stream) around every stream-collide
 * kernel launch while enable != 0. */
ELBM_API elbm_status elbm_set_profiling(elbm_handle *h, int enable);

/* Total device time (ms) and number of the stream-collide launches recorded
 * since the last call; resets the record.  Synchronises. */
ELBM_API elbm_status elbm_profile(elbm_handle *h, double *stream_collide_ms,
                                  long long *launches);

/* One FP32-shifted FORMULA step that allocates no device memory.
 *
 * The paper has no counterpart: this is a deployment variant of elbm_step
 * for callers that cannot call cudaMalloc -- an application that reserves
 * its whole device-memory budget in its own pool at start-up and passes the
 * library only buffers from that pool, or a latency-critical loop that must
 * not pay for the allocator's implicit device synchronisation.
 *
 * f_in_device / f_out_device: caller-owned device buffers of Q * nx*ny*nz
 * floats (distinct), in the library's FP32-shifted pull layout: population i
 * of node x is stored at [i][x - c_i] as f~_i - W_i rho0 (the post-collision
 * value of the previous step; the same layout elbm_step keeps internally).
 * The step reads f_in and writes f_out.  alpha_out_device (nullable,
 * nx*ny*nz floats) receives the per-node alpha.  rho0 is the shift's
 * reference density (rounded to FP32).  cuda_stream: the stream to run on.
 * stats_out (nullable, host): when given, the call computes the fused
 * diagnostics of the step, synchronises the stream, fills *stats_out (step
 * 0, FP64 check not evaluated) and reports flagged invalid states
 * (ELBM_ENEGATIVE / ELBM_ENONFINITE); without it the call returns right
 * after queueing the kernels.
 *
 * Limits and sharing: the kernels' scratch (deferred-node queue, diagnostic
 * rows, statistics, counters) is one fixed ~9.1 MB __device__ array inside
 * the library, held by every GPU that loads it until the process exits;
 * lattices above 2,097,152 nodes are rejected with ELBM_EINVAL.  Every call
 * uses the same array and clears its counters first, so calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  Errors: ELBM_EINVAL for invalid arguments or
 * sizes (checked before anything is queued), ELBM_ECUDA for CUDA errors and,
 * when stats_out is given, for a kernel whose bounded wait ran out (the
 * opt-in bulk-copy variant selected by ELBM_SC32_VARIANT=tma); the message
 * is elbm_last_error(NULL).
 * No cudaMalloc, cudaFree or allocating library call is made. */
ELBM_API elbm_status elbm_step_static(elbm_lattice lattice, int nx, int ny,
                                      int nz, double nu, double rho0,
                                      const float *f_in_device,
                                      float *f_out_device,
                                      float *alpha_out_device,
                                      void *cuda_stream,
                                      elbm_entropy_stats_t *stats_out);

/* ------------------------------------------------------------------------
 * Batched stepping of many independent lattices: up to 256 periodic
 * lattices of mixed type, size and viscosity advanced together.  Every member uses FP32-shifted storage and
 * FORMULA alpha; one persistent launch per step covers the tiles of all
 * members (the same per-node arithmetic as elbm_step), and bursts of steps
 * are replayed from a captured CUDA graph.  Block size and blocks per SM are
 * chosen by an autotuner (timed dry steps, cached per membership signature;
 * ELBM_AUTOTUNE_CACHE names an optional JSON-lines cache file).
 * ------------------------------------------------------------------------ */
typedef struct elbm_batch elbm_batch;

typedef struct {
  elbm_lattice lattice; /* ELBM_D2Q9 or ELBM_D3Q27 (D1Q3: ELBM_EINVAL) */
  int nx, ny, nz;      /* nz = 1 for D2Q9 */
  double nu;           /* > 0; beta from Eq. (2) */
} elbm_member_spec;

/* Empty batch of at most max_members (1..256) members. */
ELBM_API elbm_status elbm_batch_create(elbm_batch **out, int max_members);
ELBM_API void elbm_batch_destroy(elbm_batch *b);
ELBM_API const char *elbm_batch_last_error(const elbm_batch *b);
ELBM_API elbm_status elbm_batch_set_stream(elbm_batch *b, void *cuda_stream);
/* Device memory callbacks for every buffer of the batch (before the first
 * member is added). */
ELBM_API elbm_status elbm_batch_set_allocator(
    elbm_batch *b, void *(*alloc)(size_t bytes, void *ctx),
    void (*free_fn)(void *ptr, void *ctx), void *ctx);
/* diag_every: fused statistics on each member's last step of every
 * diag_every-th burst (0: never); burst: steps per burst (1..4096, graph
 * length); use_graphs / autotune: 0 or 1.  Defaults 0, 16, 1, 1. */
ELBM_API elbm_status elbm_batch_set_options(elbm_batch *b, int diag_every,
                                            int burst, int use_graphs,
                                            int autotune);
/* Add a member initialised to f^eq(rho, u) (host FP64 fields, layouts as
 * elbm_init_fields).  Allocates its two population buffers.  *id_out is the
 * member's id (slot), valid until elbm_batch_remove. */
ELBM_API elbm_status elbm_batch_add(elbm_batch *b, const elbm_member_spec *spec,
                                    const double *rho, const double *u,
                                    int *id_out);
/* Remove a member and free its buffers (synchronises the stream). */
ELBM_API elbm_status elbm_batch_remove(elbm_batch *b, int id);
/* Limit a member to `remaining` more steps (default: unlimited); a member
 * with none left is frozen (not stepped) by later elbm_batch_step calls. */
ELBM_API elbm_status elbm_batch_set_steps(elbm_batch *b, int id,
                                          long long remaining);
ELBM_API elbm_status elbm_batch_member_info(elbm_batch *b, int id,
                                            long long *steps_done,
                                            long long *remaining);
/* Record the per-node alpha of the member's steps (0 / 1). */
ELBM_API elbm_status elbm_batch_record_alpha(elbm_batch *b, int id, int enable);
/* Advance every member with steps left by up to nsteps steps (each member
 * stops when its remaining count reaches zero).  Asynchronous except on
 * statistics bursts. */
ELBM_API elbm_status elbm_batch_step(elbm_batch *b, long long nsteps);
/* Synchronise; report flagged invalid states. */
ELBM_API elbm_status elbm_batch_sync(elbm_batch *b);
/* Readouts of one member (host buffers, layouts as the single-lattice
 * calls).  Synchronise. */
ELBM_API elbm_status elbm_batch_moments(elbm_batch *b, int id, double *rho_out,
                                        double *u_out);
ELBM_API elbm_status elbm_batch_get_populations(elbm_batch *b, int id,
                                                double *f_out);
ELBM_API elbm_status elbm_batch_alpha_map(elbm_batch *b, int id,
                                          float *alpha_out);
/* Statistics of the member's last statistics step (FP64 check fields are
 * not evaluated in batches). */
ELBM_API elbm_status elbm_batch_entropy_stats(elbm_batch *b, int id,
                                              elbm_entropy_stats_t *out);
/* Decision of the FP32 entropy tests the first stage leaves undecided, as
 * elbm_set_decision (default ELBM_DECISION_EXACT). */
ELBM_API elbm_status elbm_batch_set_decision(elbm_batch *b,
                                             elbm_decision decision);
/* Launch configuration in use (after the first step: the tuned one). */
ELBM_API elbm_status elbm_batch_tuning(const elbm_batch *b, int *threads,
                                       int *blocks_per_sm, int *burst);
ELBM_API size_t elbm_batch_device_bytes(const elbm_batch *b);

/* Reference density rho0 of the shifted storage (meaningful after init). */
ELBM_API double elbm_rho0(const elbm_handle *h);

/* The beta of Eq. (2) the handle's steps use, c_s^2 / (2 nu + c_s^2) with
 * dt = 1 and c_s^2 = 1/3 (NaN for a NULL handle).  Needs no device. */
ELBM_API double elbm_beta(const elbm_handle *h);


#ifdef __cplusplus
}
#endif
#endif /* ELBM_H */
