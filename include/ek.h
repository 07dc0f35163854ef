/*
 * ek.h -- C ABI of the GB300 lattice electrokinetics library (libek.so).
 *
 * The library advances the moving-boundary lattice electrokinetics method of
 * Kuron et al., "Moving Charged Particles in Lattice Boltzmann-Based
 * Electrokinetics" (arXiv 1607.04572), on one GPU.  One call of ek_step(ctx, n)
 * runs n time steps, each made of
 *
 *   S1  charge assembly and periodic FFT Poisson solve           (Sec. III.C, Eq. 3;
 *                                                                  particle charge Eq. 21)
 *   S2  Capuani link fluxes (diffusion + migration, partial       (Eqs. 13, 20, 16)
 *       volumes) and their force on the fluid, fused with the
 *       D3Q19 TRT/BGK collision (Guo force term) and push stream  (Sec. III.A, Eqs. 5-9)
 *       with velocity bounce-back and momentum exchange           (Eq. 12, Eqs. 10-11)
 *   S3  species update: flux divergence + volume-of-fluid         (Eq. 15, Sec. III.C)
 *       advection
 *   S4  particle force (momentum exchange, electrostatic, fluid   (Sec. III.B)
 *       create/destroy) and symplectic Euler integration
 *   S5  re-flagging, octree partial volumes Psi, fluid            (Sec. III.B, III.D,
 *       create/destroy, solute expulsion and refill                Eqs. 17-18)
 *
 * Units: lattice units, grid spacing a = 1, time step tau = 1, k_B T = 1,
 * elementary charge e = 1 (the paper's energy unit is k_B T, Table I).
 *
 * Layout of every field exchanged through this ABI: structure of arrays, FP64,
 * node index  x + nx*(y + ny*z)  (x fastest).  A vector or multi-component field
 * is component-major: component c of node i at [c*N + i], N = nx*ny*nz.
 *
 * Ownership: the context owns all of its device memory (allocated in ek_create,
 * freed in ek_destroy).  Every pointer passed in is owned by the caller and only
 * read or written during the call; host pointers must stay valid for the call,
 * device pointers must be device memory of the context's GPU.
 *
 * Errors: every entry point returns an ek_status and never throws, aborts or
 * exits.  On failure ek_last_error(ctx) gives a human-readable reason.  A
 * device-side condition (non-finite value, overlapping particles, nowhere to
 * expel solute) is recorded in a device status word and returned by the next
 * ek_step / ek_sync / ek_get_* call; the context is then unusable except for
 * ek_get_* and ek_destroy.
 *
 * Threading: a context is not thread-safe; use one context per host thread.
 * All work is enqueued on the context's stream (the legacy default stream
 * unless ek_set_stream was called).
 */
#ifndef EK_H
#define EK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EK_MAX_SPECIES 4

typedef struct ek_ctx ek_ctx;

typedef enum {
  EK_OK = 0,
  EK_ERR_ARG = -1,       /* invalid argument (null pointer, size, range)          */
  EK_ERR_NOMEM = -2,     /* device or host allocation failed                      */
  EK_ERR_CUDA = -3,      /* a CUDA runtime call failed                            */
  EK_ERR_UNSTABLE = -4,  /* a non-finite density or velocity was produced         */
  EK_ERR_OVERLAP = -5,   /* a node lies inside two particles                      */
  EK_ERR_EXPEL = -6,     /* a newly covered node has no fluid neighbour           */
  EK_ERR_TIMEOUT = -7,   /* a bounded device wait gave up (batch grid barrier)    */
  EK_ERR_STATE = -8      /* call not valid in the context's state, or a capacity  */
} ek_status;

/* ek_params.flags */
enum {
  EK_PV = 1,             /* partial-volume flux, Eq. 20, and Psi-smeared particle
                            charge, Eq. 21 (the paper's enhanced scheme); without
                            it: Eq. 13 fluxes and charge spread evenly over the
                            particle's boundary nodes (the simple scheme)          */
  EK_VACATE_ZERO = 2,    /* vacated nodes are left empty instead of refilled by
                            Eqs. 17-18 (allowed with EK_PV, Sec. III.D.2)          */
  EK_CHARGE_NORM_VP = 4, /* Eq. 21 literally: divide by the continuous volume V_p;
                            default divides by sum Psi_p so the charge is exactly Z */
  EK_NEUTRALIZE = 8,     /* at fill time add counter-ions of the first species of
                            opposite valence so the box is neutral                 */
  EK_FP32 = 16           /* FP32-storage form: populations stored as f_i - w_i rho0
                            in float, species as int32 multiples of a per-species
                            unit 2^-e (e = ceil(20 - log2 rho_k), rho_k the larger
                            of bulk_k and the initial density after
                            neutralisation: at least 2^20 units per initial
                            density), Phi, Psi, u, charges and the
                            FFT in float, arithmetic in float; particle forces,
                            torques and the integrator stay FP64.  Every species
                            transfer moves whole units between nodes, so the
                            species totals are conserved exactly.  Fields are
                            still exchanged as FP64 (converted on set/get).      */
};

typedef struct {
  int nx, ny, nz;        /* periodic box, each in [8, 1024]                        */
  double nu;             /* kinematic viscosity; tau_e = 3 nu + 1/2 (Sec. III.A)   */
  double rho0;           /* fluid rest density                                     */
  double bjerrum;        /* Bjerrum length l_B (Eq. 4)                             */
  double magic;          /* TRT magic product Lambda (the paper's 3/16); <= 0 or
                            NaN selects BGK, lambda_o = lambda_e                   */
  int nspecies;          /* K in [0, EK_MAX_SPECIES]; 0 runs the fluid alone        */
  int valence[EK_MAX_SPECIES];   /* z_k                                            */
  double D[EK_MAX_SPECIES];      /* diffusion coefficients, each in (0, 0.39]      */
  double bulk[EK_MAX_SPECIES];   /* initial density on fluid nodes                 */
  unsigned flags;        /* EK_PV | EK_VACATE_ZERO | EK_CHARGE_NORM_VP | EK_NEUTRALIZE
                            | EK_FP32                                              */
} ek_params;

typedef enum {
  /* readable and writable */
  EK_FIELD_SPECIES = 0,     /* density rho_k of species `component`, N values         */
  EK_FIELD_POPULATIONS = 1, /* f_i, 19*N values, direction-major (see ek_lattice_dirs) */
  EK_FIELD_VELOCITY = 2,    /* set: f = f^eq(current rho, u) on fluid nodes; get: the
                               fluid velocity u = (sum f c + f_ext/2)/rho of the last
                               collision; 3*N values                                 */
  EK_FIELD_E_EXT = 3,       /* uniform external field E, 3 values                      */
  EK_FIELD_BODY_FORCE = 4,  /* uniform body force density on the fluid, 3 values      */
  EK_FIELD_WALL = 5,        /* static boundary mask, N values (nonzero = wall); set
                               re-flags and refills like ek_add_particle             */
  EK_FIELD_WALL_CHARGE = 6, /* static boundary charge density rho_b, N values          */
  /* read only */
  EK_FIELD_DENSITY = 7,     /* fluid density sum_i f_i, N values                       */
  EK_FIELD_PHI = 8,         /* electrostatic potential of the last solve, N values     */
  EK_FIELD_PSI = 9,         /* overlap fraction Psi = min(1, sum_p Psi_p), N values    */
  EK_FIELD_OWNER = 10,      /* node class as doubles: -1 fluid, -2 wall, p >= 0 inside
                               particle p; N values                                  */
  EK_FIELD_CHARGE = 11      /* charge density q of the last Poisson solve, N values    */
} ek_field;

typedef struct {
  double pos[3], vel[3], omega[3];
  double force[3], torque[3];  /* total force/torque of the last integration        */
  double radius, charge, rho_p;
  int fixed;
} ek_particle;

/* Create a context.  Copies *p; allocates all device state on the current CUDA
 * device; fills populations with the rest equilibrium f^eq(rho0, 0) and species
 * with their bulk densities.  Returns EK_ERR_ARG for invalid parameters. */
ek_status ek_create(const ek_params* p, ek_ctx** out);
ek_status ek_destroy(ek_ctx* ctx);

/* Add a sphere of radius R and charge Z (units of e) at pos (wrapped into the
 * box) with velocity vel and angular velocity omega (Sec. III.B).  Mass
 * rho_p (4/3) pi R^3, moment of inertia (2/5) m R^2.  fixed != 0: the particle
 * is a stationary boundary moving with vel (the co-moving frame of Sec. IV.A).
 * Requires 2R + 6 <= min(nx, ny, nz).  Re-flags the lattice and refills it:
 * species back to bulk on fluid nodes (plus counter-ions with EK_NEUTRALIZE),
 * populations to rest equilibrium.  *out_id (may be NULL) receives the index. */
ek_status ek_add_particle(ek_ctx* ctx, const double pos[3], const double vel[3],
                          const double omega[3], double radius, double charge,
                          double rho_p, int fixed, int* out_id);

/* Write a field (see ek_field).  count must equal the field's size; src is a
 * host pointer, or a device pointer when src_on_device != 0. */
ek_status ek_set_field(ek_ctx* ctx, ek_field which, int component, const double* src,
                       size_t count, int src_on_device);

/* Read a field into dst (host, or device when dst_on_device != 0); synchronises
 * the context's stream. */
ek_status ek_get_fields(ek_ctx* ctx, ek_field which, int component, double* dst,
                        size_t count, int dst_on_device);

/* Enqueue nsteps full time steps (S1-S5) on the context's stream, then wait for
 * them and check the device status word. */
ek_status ek_step(ek_ctx* ctx, int nsteps);

/* Enqueue nsteps full time steps without waiting (no status check). */
ek_status ek_step_async(ek_ctx* ctx, int nsteps);

/* Run one stage of a time step on the current state (1..5 = S1..S5; S2 includes
 * the buffer swap of populations and species that closes S2/S3).  For
 * stage-by-stage comparisons; ek_step runs S1..S5 in order. */
ek_status ek_run_stage(ek_ctx* ctx, int stage);

/* Copy up to count particle records to host memory dst (synchronises). */
ek_status ek_get_particles(ek_ctx* ctx, ek_particle* dst, int count);

/* The same records, enqueued on the context's stream without waiting (for a
 * caller that reads every step's particle state while the next steps run):
 * the first min(count, P) records are packed on the device and copied to dst,
 * which must be page-locked host memory (cudaHostAlloc, or a pinned torch
 * tensor) or device memory; they are valid once the stream has passed this
 * call (an event recorded after it, or ek_sync).  The device status word is not
 * read (ek_sync reads it).  Errors: EK_ERR_ARG, EK_ERR_CUDA. */
ek_status ek_get_particles_async(ek_ctx* ctx, ek_particle* dst, int count);
int ek_num_particles(const ek_ctx* ctx);

/* Checkpoint and resume (the paper has no counterpart; the state is what a
 * time step of Sec. III reads).  ek_get_state: with buf == NULL, *bytes
 * receives the size of a checkpoint; otherwise buf (host memory of *bytes
 * bytes, caller owned) receives the checkpoint and *bytes its size.  The
 * checkpoint holds a header (shape, species, storage form, flags, particle
 * count and box size, species units, E, body force) and, as stored on the
 * device, both population buffers, the species, Psi, particle
 * and wall charge, Phi, u, node owners, the wall mask and the particles'
 * records and Psi_p boxes.  Waits for the context's work.  Errors: EK_ERR_ARG
 * (null bytes; buffer smaller than the checkpoint, *bytes then holds the size
 * needed), EK_ERR_CUDA, and the device status of ek_sync. */
ek_status ek_get_state(ek_ctx* ctx, void* buf, size_t* bytes);
/* Restore a checkpoint into a context created with the same parameters and
 * particles (any number of steps later, or a fresh context): the steps that
 * follow give bit for bit what the checkpointed context's next steps give.
 * buf is host memory of `bytes` bytes, read only during the call.  Errors:
 * EK_ERR_ARG (null, too short, not a checkpoint of this library version),
 * EK_ERR_STATE (a checkpoint of a different system: shape, species, storage
 * form, flags, particle count or box size, species units), EK_ERR_CUDA. */
ek_status ek_set_state(ek_ctx* ctx, const void* buf, size_t bytes);

/* Run nsteps steps like ek_step, recording CUDA events on the context's stream
 * between the stages, and add the device time of each to stage_ms (caller
 * owned, 6 doubles): [0] S1 Poisson, [1] S2 fused flux/LB kernel, [2] S3
 * advection, [3] S4, [4] S5, [5] the whole nsteps steps.  Waits for the work. */
ek_status ek_step_timed(ek_ctx* ctx, int nsteps, double stage_ms[6]);

/* Number of kernels the step and stage calls (ek_step, ek_step_async,
 * ek_run_stage, ek_step_timed and batch steps) have enqueued on this context
 * since it was created; device memsets and set-up work are not counted. */
long long ek_kernel_launches(const ek_ctx* ctx);

/* Use the CUDA stream `stream` (a cudaStream_t) for all later work; waits for
 * the work already enqueued on the previous stream first.  On a stream other
 * than the legacy default one, ek_step / ek_step_async capture one step as a
 * CUDA graph (one per parity of the double-buffered populations) and replay
 * it; the graphs are rebuilt after a change of set-up, E, body force or
 * stream.  Results are the same as with separate launches. */
ek_status ek_set_stream(ek_ctx* ctx, void* stream);
/* Wait for all enqueued work and check the device status word. */
ek_status ek_sync(ek_ctx* ctx);
/* Reason of the last failure, or "" (the string is owned by the context). */
const char* ek_last_error(const ek_ctx* ctx);

/* The D3Q19 velocity set used for EK_FIELD_POPULATIONS: c[3*i + a], i = 0..18. */
void ek_lattice_dirs(int c[57]);

/* Standalone periodic Poisson solve of Eq. 3 on the device (S1 without the
 * charge assembly): phi = solution of lap_7 phi = -4 pi l_B (q - mean q) with
 * the 7-point Laplacian, mean(phi) = 0.  q and phi are device arrays of
 * nx*ny*nz doubles (may alias); spectrum is caller-allocated device scratch of
 * at least ek_poisson_scratch_bytes(nx, ny, nz) bytes; stream is a
 * cudaStream_t or NULL.  Supported edges: 2^a 3^b, 8 <= n <= 1024. */
size_t ek_poisson_scratch_bytes(int nx, int ny, int nz);
ek_status ek_poisson_solve(const double* q, double* phi, int nx, int ny, int nz,
                           double bjerrum, void* spectrum, void* stream);

/* The same periodic problem of Eq. 3 solved iteratively (the paper names
 * iterative solvers as the alternative to the FFT, Sec. III.C): geometric
 * multigrid V-cycles (two red-black Gauss-Seidel sweeps before and after,
 * full-weighting restriction, trilinear prolongation) on the box and its
 * coarsenings by 2 (while every coarse edge stays even and >= 8, n_x / 2
 * even, and the level holds more than 4096 nodes), the coarsest level solved
 * exactly by the FFT; cycles until max|r| <= tol * max|b|, b = 4 pi l_B
 * (q - mean q), r = b - (6 phi - sum of the 6 neighbours), at most max_cycles.
 * A box that cannot be coarsened is solved by the FFT in one cycle.  phi is
 * returned with mean 0.  q, phi: device arrays of nx*ny*nz doubles (may
 * alias); scratch: caller-allocated device memory of at least
 * ek_poisson_mg_scratch_bytes(nx, ny, nz) bytes; stream: a cudaStream_t or
 * NULL; *cycles and *residual (max|r| / max|b|), when not NULL, receive the
 * V-cycles run and the final relative residual.  Waits for the work.
 * Supported edges as for ek_poisson_solve.  Errors: EK_ERR_ARG (null
 * pointer, unsupported edges, tol <= 0, max_cycles < 1), EK_ERR_CUDA.
 * ek_poisson_mg_scratch_bytes returns 0 for unsupported edges. */
size_t ek_poisson_mg_scratch_bytes(int nx, int ny, int nz);
ek_status ek_poisson_solve_mg(const double* q, double* phi, int nx, int ny, int nz,
                              double bjerrum, double tol, int max_cycles, void* scratch,
                              void* stream, int* cycles, double* residual);

/* Poisson solve with an inhomogeneous permittivity and fixed-potential nodes:
 * the problem the paper leaves to iterative solvers such as Krylov subspace
 * methods, which also handle inhomogeneous dielectric coefficients (Sec.
 * III.C, the paragraph after Eq. 16).  Solves div(eps grad Phi) = -4 pi l_B q
 * on the periodic nx x ny x nz box, eps the permittivity relative to the
 * solvent whose Bjerrum length is l_B: the 7-point operator of
 * ek_poisson_solve with face permittivities, the harmonic mean
 * 2 eps_i eps_j / (eps_i + eps_j) of the face's two nodes; a free node
 * satisfies sum_f eps_f (Phi_i - Phi_j) = 4 pi l_B q_i over its six faces, a
 * node with fixed[i] != 0 holds Phi = phi_fixed[i] (walls, electrodes).
 * Without fixed nodes the mean charge is removed and phi is returned with
 * mean 0 (then with eps = 1 the result is ek_poisson_solve's).  Method:
 * preconditioned conjugate gradients in FP64 from Phi = 0 on the free nodes,
 * until ||r||_2 <= tol ||b||_2 over the free nodes or max_iter iterations.
 * The preconditioner is one multigrid V-cycle of the same operator (levels
 * halved while every edge is even and stays >= 4, coarse face permittivity
 * the halved sum of the 4 fine faces it covers, damped Jacobi smoothing,
 * the coarsest level of at most 8192 nodes by 40 sweeps) when the box has
 * at least two levels, else the diagonal (Jacobi); the residual is checked
 * every 2 (multigrid) or 10 (Jacobi) iterations.  Every inner product is a
 * fixed-order sum, so a solve is bit-reproducible.
 *
 * All arrays are device arrays of nx*ny*nz values, index x + nx*(y + ny*z):
 * q, phi (double; may alias), eps (double, positive and finite; NULL: 1
 * everywhere), fixed (unsigned char; NULL: none), phi_fixed (double; NULL:
 * 0; may alias phi).  scratch: caller-allocated device memory of at least
 * ek_poisson_cg_scratch_bytes(nx, ny, nz) bytes.  stream: a cudaStream_t or
 * NULL.  *iters and *residual (||r|| / ||b||), when not NULL, receive the
 * iterations run and the final relative residual (a residual above tol means
 * max_iter ran out).  Waits for the work.  Any edge >= 1 (nx*ny*nz < 2^31).
 * Errors: EK_ERR_ARG (null q, phi or scratch, bad sizes, tol <= 0,
 * max_iter < 1, a permittivity that is not positive and finite), EK_ERR_CUDA.
 * ek_poisson_cg_scratch_bytes returns 0 for bad sizes. */
size_t ek_poisson_cg_scratch_bytes(int nx, int ny, int nz);
ek_status ek_poisson_solve_cg(const double* q, const double* eps, const unsigned char* fixed,
                              const double* phi_fixed, double* phi, int nx, int ny, int nz,
                              double bjerrum, double tol, int max_iter, void* scratch, void* stream,
                              int* iters, double* residual);

/* The same Poisson solve for callers that cannot allocate device memory:
 * code whose device memory is entirely reserved up front by another runtime's
 * pool (so a raw cudaMalloc would fail), latency-critical loops that must not
 * let cudaMalloc/cudaFree synchronise the device, and code under a policy that
 * forbids allocation after initialisation.  The paper has no counterpart; it
 * is a service of this library.
 *
 * Allocates nothing: the spectrum scratch (at most EK_POISSON_STATIC_MAX
 * complex doubles, 8 MiB) and the FFT tables live in fixed file-scope device
 * arrays that every GPU which loads the library holds until the process exits.
 * The caller passes q and phi (device arrays of nx*ny*nz doubles, may alias).
 * Returns EK_ERR_ARG when (nx/2 + 1)*ny*nz exceeds EK_POISSON_STATIC_MAX or an
 * edge is not 2^a 3^b in [8, 1024] (nx even).  The first call on a device
 * resolves the arrays' device addresses (cudaGetSymbolAddress), so make the
 * first call on each device before any stream capture.  A call with a box
 * shape other than the previous call's reloads the tables by copies queued on
 * `stream`, after the work already queued there: calls issued in order on one
 * stream may change shape freely.  All calls share the arrays, which keep the
 * last call's contents (nothing in them needs to start at zero: the first FFT
 * pass writes the whole spectrum); calls that overlap on the GPU (on different
 * streams with no ordering between them) race and give wrong results. */
#define EK_POISSON_STATIC_MAX (1u << 19)
ek_status ek_poisson_solve_static(const double* q, double* phi, int nx, int ny, int nz,
                                  double bjerrum, void* stream);

/* ---------------------------------------------------------------------------
 * Batched ensemble: many independent systems (box sizes, salts, fields and
 * particles of their own, e.g. a mobility sweep) advanced together.  The
 * paper runs one system at a time; batching is a service of this library.
 *
 * The systems are ordinary contexts, created and set up by the caller
 * (ek_create, ek_add_particle, ek_set_field); the batch borrows them (they
 * must outlive it and are not destroyed by it).  One batch step advances
 * every system by one time step, exactly as ek_step would, in one CUDA graph
 * launch, in one of two forms:
 *  - fused (when every system has the FP32 storage form, the same number of
 *    species and the same partial-volume choice; the default then): each
 *    kernel of the step runs once for the whole batch over a list of
 *    (system, block) ranges -- a system's CTAs find its arguments in a device
 *    table -- so a step is about twenty launches whatever the number of
 *    systems.  S1 of the systems whose edges are all 32, 48 or 64 shares
 *    launches by FFT kernel variant; other systems' S1 runs per system.
 *    A variant of it (form 2) runs the particle kernels between two
 *    stream-ordered points as phases of one persistent cooperative launch
 *    whose CTAs meet at a grid barrier between phases; every wait there is
 *    bounded (EK_ERR_TIMEOUT, ek_batch_wait_test).
 *  - branches: each system's own step is an independent branch of the graph,
 *    so the systems' kernels run side by side on the GPU.
 * The graph is captured on the first step (one per ping-pong parity) and
 * again whenever a system's set-up, field E / body force or tuning changes.
 *
 * Work of a batch step is ordered on the batch stream only: call
 * ek_batch_sync before reading a system (ek_get_fields, ek_get_particles) or
 * stepping it alone, and do not step a system alone while batch steps are in
 * flight. */
typedef struct ek_batch ek_batch;

/* Batch over systems[0..nsys-1] (distinct contexts on the same GPU, each set
 * up; copies the pointer list).  Waits for the systems' pending work.  Errors:
 * EK_ERR_ARG (null, repeated or cross-device contexts), EK_ERR_STATE (a
 * context in an error state), EK_ERR_CUDA. */
ek_status ek_batch_create(ek_ctx* const* systems, int nsys, ek_batch** out);
/* Waits for the batch stream and frees the batch (not its systems). */
ek_status ek_batch_destroy(ek_batch* b);
/* Launch later batch steps on `stream` (a cudaStream_t other than the legacy
 * default stream); waits for the batch's earlier work. */
ek_status ek_batch_set_stream(ek_batch* b, void* stream);
/* Enqueue nsteps batch steps; returns without waiting. */
ek_status ek_batch_step_async(ek_batch* b, int nsteps);
/* ek_batch_step_async, then ek_batch_sync. */
ek_status ek_batch_step(ek_batch* b, int nsteps);
/* Wait for the batch stream and read every system's device status word; the
 * first failing system's status is returned (ek_batch_last_error names it). */
ek_status ek_batch_sync(ek_batch* b);
/* Autotuner: times every candidate configuration -- the fused forms (where
 * the batch allows them) or branches with 8, 16, 32, 64 or one branch stream
 * per system (at most 64), FP32 S2 segment length (2, 4 or 8 planes per
 * block), and whether the particle chain runs beside the advection or in line
 * -- over 2 + trial_steps real batch steps each (the systems advance by those
 * steps), keeps the fastest and stores its time per batch step in *best_ms
 * (may be null).  Results do not depend on the choice except for the
 * summation order of the lattice-block force sums. */
ek_status ek_batch_tune(ek_batch* b, int trial_steps, double* best_ms);
/* Current configuration: cfg[0] branch streams, cfg[1] planes per S2 block,
 * cfg[2] particle chain beside the advection (1) or in line (0), cfg[3] the
 * form: 0 branches, 1 fused, 2 fused with the particle kernels other than the
 * forces as three persistent launches whose phases meet at grid barriers. */
ek_status ek_batch_config(const ek_batch* b, int cfg[4]);
/* Set the configuration (cfg as ek_batch_config gives it: branch streams 1 ..
 * min(nsys, 64), planes per S2 block 1 .. 64, overlap 0 or 1, form 0, 1 or 2);
 * waits for the batch's earlier work.  EK_ERR_ARG for a value out of range or
 * a fused form on a batch that does not allow it. */
ek_status ek_batch_set_config(ek_batch* b, const int cfg[4]);
/* Failure-detection test hook: the n-th device allocation of a field that
 * ek_create makes from now on (counting across calls) fails as if the device
 * were out of memory, so that ek_create frees what it allocated and returns
 * EK_ERR_NOMEM; n <= 0 clears the hook.  Process-wide; for tests. */
void ek_debug_fail_alloc(int n);
/* Failure-detection test hook for form 2: in the steps captured from now on,
 * CTA leave_cta of each persistent particle-chain launch returns before the
 * first grid barrier (-1: none), and a wait at a barrier gives up after
 * limit_ms (default 1000; at most 60000).  A wait that gives up makes every
 * CTA of the launch return; ek_batch_sync then returns EK_ERR_TIMEOUT and
 * puts every system of the batch into the error state (their step stopped
 * part way).  Waits for the batch's earlier work.  Errors: EK_ERR_ARG. */
ek_status ek_batch_wait_test(ek_batch* b, int leave_cta, double limit_ms);
/* Number of systems; 0 for a null batch. */
int ek_batch_size(const ek_batch* b);
/* Reason for the last failure of a batch call. */
const char* ek_batch_last_error(const ek_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* EK_H */
