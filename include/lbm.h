/*
 * liblbm: GB300 (sm_103a) hot path of the thermal pseudopotential MRT lattice
 * Boltzmann method for 3D liquid-vapor phase change of Huang, Wang, He & Huang,
 * "An efficient thermal lattice Boltzmann method for simulating
 * three-dimensional liquid-vapor phase change" (arXiv 2206.00946).
 *
 * One time step updates every lattice cell:
 *   (a) Peng-Robinson p_EOS(rho, T) (Sec. 4, Eq. 37) and the pseudopotential
 *       psi = sqrt(2 (p_EOS - rho c_s^2) / G) (Sec. 2.1, Eq. 7);
 *   (b) the 18-neighbour interaction force F = -G psi(x) sum w(|c|^2) psi(x+c) c (Eq. 6);
 *   (c) the D3Q19 non-orthogonal MRT collision with the exact-difference forcing
 *       (Eqs. 2-5, 8-10, appendix matrix M-hat), streaming, bounce-back walls
 *       (Sec. 3.1) and the constant-pressure open boundary (Sec. 3.3);
 *   (d) the D3Q7 MRT temperature collision with the source -w_i Fbar,
 *       Fbar = rho c_v u.grad T + T (dp/dT)_rho div u (Eqs. 13-15, 27-29), the
 *       relaxed streaming of Eq. 13 and the non-equilibrium extrapolation at
 *       Dirichlet faces (Sec. 3.1).
 *
 * Conventions
 *  - Lattice units, dx = dt = 1.  Cell index c = x + nx*(y + ny*z), x fastest.
 *  - Population layout (state exchanged by lbm_set_state / lbm_get_state):
 *    structure of arrays, f[i*N + c] for i = 0..18 and g[i*N + c] for i = 0..6,
 *    N = nx*ny*nz, float32.  Velocity order: 0 rest, 1/2 +-x, 3/4 +-y, 5/6 +-z,
 *    7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
 *    13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1),
 *    read off rows 1-3 of the appendix matrix; D3Q7: 0 rest, 1/2 +-x, 3/4 +-y, 5/6 +-z.
 *  - Faces are numbered 0..5 = -x, +x, -y, +y, -z, +z.
 *  - Every function returns an lbm_status; the library never aborts.  Work is
 *    enqueued asynchronously on the stream given to lbm_init; device-side
 *    error flags are read (and the stream synchronised) by lbm_sync,
 *    lbm_reduce, lbm_macros and lbm_get_state.
 *  - Pointer arguments marked "mem" are device pointers when mem ==
 *    LBM_MEM_DEVICE and host pointers when mem == LBM_MEM_HOST; the caller owns
 *    them.  The library owns the population and scratch buffers it allocates
 *    in lbm_init and frees in lbm_destroy.
 *
 * Environment (tuning and comparison only; results do not depend on them
 * beyond rounding):
 *   LBM_SLAB_PLANES, LBM_SLAB_STREAMS, LBM_GRAPH_STEPS  planes per slab, streams
 *       and steps per CUDA graph of the pipelined slab schedule (read by lbm_init);
 *   LBM_STAGE19, LBM_STAGE7  tiles of 256 cells per CTA of the FP32 force + D3Q19 and D3Q7
 *       kernels that stage their populations in shared memory (default 4; 0 turns staging
 *       off; read by lbm_init; lattices whose planes do not divide into 256-cell tiles, or
 *       of fewer than 622,592 cells, never stage);
 *   LBM_ADJ_EAGER, LBM_ADJ_NOPDL  launch every adjoint step on its own instead of
 *       replaying K-step segments from graphs / without programmatic dependent
 *       launches (read by each lbm_adjoint_step).
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,        /* invalid argument or unsupported parameter combination */
  LBM_ERR_CUDA = -2,       /* a CUDA runtime call failed (allocation, launch, copy) */
  LBM_ERR_NONFINITE = -3,  /* a population became NaN/Inf */
  LBM_ERR_PSI_DOMAIN = -4, /* 2 (p_EOS - rho/3) / G < 0 somewhere: psi of Eq. 7 undefined */
  LBM_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up */
  LBM_ERR_STATE = -6       /* call out of order (e.g. step before any state was set) */
} lbm_status;

typedef enum { LBM_FACE_PERIODIC = 0, LBM_FACE_WALL = 1, LBM_FACE_OPEN = 2 } lbm_face_kind;
typedef enum {
  LBM_STORE_F32 = 0,
  LBM_STORE_F16_SHIFTED = 1,  /* IEEE half of f_i - w_i rho_ref, g_i - w_i T_ref (one global shift) */
  LBM_STORE_BF16_SHIFTED = 2, /* bfloat16, the same shift */
  LBM_STORE_F16_LOCAL = 3     /* IEEE half with per-cell references: rho_ref and T_ref of a stored
                                 population are the density and temperature its cell had before the
                                 step that wrote it (8 bytes per cell, twice, kept by the library) */
} lbm_storage;
typedef enum { LBM_MEM_DEVICE = 0, LBM_MEM_HOST = 1 } lbm_mem;
typedef enum { LBM_SCHED_FUSED = 0, LBM_SCHED_PHASES = 1, LBM_SCHED_SLABS = 2 } lbm_schedule;

/* Problem statement.  Physical parameters follow the paper's notation. */
typedef struct lbm_params {
  int nx, ny, nz;                /* lattice size; >= 3 along an axis with non-periodic faces */
  double a, b, R, omega;         /* Peng-Robinson EOS, Sec. 4 Eqs. 37-38 (T_c follows from a, b, R) */
  double G;                      /* interaction strength of Eq. 6 (the paper uses -1) */
  double s_e, s_v, s_q, s_pi;    /* D3Q19 relaxation rates of Lambda-hat, Eq. 10 */
  double cv;                     /* specific heat at constant volume, Eq. 12 */
  double wbar;                   /* D3Q7 weight parameter of Eq. 14, 0 < wbar < 1, c_s^2 = wbar/3 */
  double lambda_l, lambda_v;     /* thermal conductivity of liquid / vapor; lambda is interpolated
                                    linearly in the liquid fraction (rho-rho_v)/(rho_l-rho_v), and
                                    varsigma_{1,2,3} = 1 / (lambda / c_s^2 + 1/2) (Sec. 2.2) */
  double rho_l, rho_v;           /* coexistence densities used by that interpolation */
  int vartheta;                  /* correction switch of Eq. 13: 0 (the paper's choice) or 1, the
                                    S_i of Eq. 16 with d^2T/dt^2 the backward second difference of
                                    the per-cell T of the two previous steps (kept by the library,
                                    8 bytes per cell; a state set by lbm_init or lbm_set_state is
                                    taken to be at rest before, and checkpoints carry the history);
                                    lbm_record and batching need 0 */
  int meq_printed;               /* 0: m^eq = M-hat f^eq; 1: rows 16-18 exactly as printed in Eq. 9 */
  int wall_ueq_zero;             /* at bounce-back wall nodes the real velocity u is 0 (Sec. 3.1: the
                                    wall-node velocity is specified by the no-slip condition) in the
                                    outputs, in div u and in Fbar; the collision's u^eq there is 0
                                    when 1 (the node's momentum leaves the collision as F), or the
                                    node's own j / rho when 0 */
  int eos_kind;                  /* 0: Peng-Robinson; 1: ideal gas p = eos_c0 * rho (verification) */
  double eos_c0;
  int face_kind[6];              /* lbm_face_kind per face; periodic faces come in pairs; a wall face
                                    may not share an edge with an open face */
  double face_T[6];              /* Dirichlet temperature of every non-periodic face (Sec. 3.1) */
  double face_rho[6];            /* prescribed density of an open face (Sec. 3.3) */
  double face_theta_deg[6];      /* contact angle of a wall face, Eq. 36 */
  int storage;                   /* lbm_storage: FP32 populations, or 16-bit IEEE half / bfloat16
                                    holding f_i - w_i rho_ref and g_i - w_i T_ref (all arithmetic in FP32;
                                    the FUSED schedule supports FP32 only) */
  double store_rho_ref;          /* global shift rho_ref of the 16-bit storage (e.g. rho_v) */
  double store_T_ref;            /* global shift T_ref of the 16-bit storage (e.g. the mean temperature) */
  int schedule;                  /* lbm_schedule: one persistent launch per step (FUSED), one launch
                                    per phase (PHASES), or per phase and z-slab on several streams,
                                    replayed from a CUDA graph (SLABS) */
  int face_T_fixed[6];           /* 1: the node layer of face f holds the Dirichlet temperature
                                    face_T[f] (non-equilibrium extrapolation, Sec. 3.1) even where
                                    the face is periodic for the flow -- the droplet of Sec. 4.2
                                    (periodic velocity field, temperature fixed at the boundaries);
                                    non-periodic faces hold theirs regardless.  A periodic axis with
                                    a held layer needs >= 3 cells; lbm_record needs 0 everywhere */
} lbm_params;

/* Creates a context on the current CUDA device and, if rho0 and T0 are not
 * NULL, initialises f = f^eq(rho0, u = 0) and g_i = w_i T0 (Sec. 4.2).
 * rho0, T0: N floats each (mem).  stream: a cudaStream_t (NULL = legacy default).
 * On error *out is NULL. */
int lbm_init(lbm_ctx** out, const lbm_params* p, const float* rho0, const float* T0, int mem, void* stream);

/* Replaces the populations: f 19*N floats, g 7*N floats, SoA layout above (mem). */
int lbm_set_state(lbm_ctx* ctx, const float* f, const float* g, int mem);

/* Copies the current populations out (mem); synchronises the stream. */
int lbm_get_state(lbm_ctx* ctx, float* f, float* g, int mem);

/* Checkpoint / restore of the time-stepping state (the populations in the
 * context's storage format), e.g. for recomputation between checkpoints.
 * The image is a 256-byte header (magic, lattice size, storage mode and
 * shifts) followed by f and g (then the T history for vartheta = 1 and the
 * per-cell references of LBM_STORE_F16_LOCAL); lbm_checkpoint_bytes gives its size.
 * lbm_checkpoint writes the image to dst (mem), synchronises the stream and
 * returns the error flags like lbm_get_state.  lbm_restore reads an image
 * written by a context with the same lattice size, storage mode and shifts
 * (else LBM_ERR_ARG) and makes it the current state; device images are
 * copied asynchronously, host images before it returns.  The caller owns
 * the image buffer. */
long long lbm_checkpoint_bytes(const lbm_ctx* ctx);
int lbm_checkpoint(lbm_ctx* ctx, void* dst, int mem);
int lbm_restore(lbm_ctx* ctx, const void* src, int mem);

/* Discrete adjoint of the time step (no counterpart in the paper, which solves
 * forward problems only).  The gradients are those of the FP32 step exactly
 * as the library computes it, accumulated in FP64 over the steps.
 *
 * lbm_record advances n steps from the current state like lbm_step and keeps
 * a checkpoint of the populations every K steps (device memory: n/K + 1
 * checkpoints of 104 bytes per cell, and one or, when it fits, two segment
 * buffers of min(K, n) + 1 slots of 168 bytes per cell: a step's state and the
 * forward scratch computed from it).
 * Requirements: FP32 storage, vartheta = 0, wall faces at 90 degrees
 * (LBM_ERR_ARG otherwise); a state must be set (LBM_ERR_STATE).
 *
 * lbm_adjoint_step runs the adjoint backwards through the n recorded steps (n
 * must equal the recorded count, else LBM_ERR_STATE), recomputing each
 * K-step segment from its checkpoint.  Inputs (device, N floats, NULL = 0):
 * dL_drho and dL_dT, the gradient of the loss with respect to the final
 * rho = sum f and T = sum g.  Outputs (device, NULL to skip): dL_dTface, the
 * gradient with respect to the per-node face temperatures of lbm_set_face_T,
 * the arrays of the non-periodic faces concatenated in face order (periodic
 * faces contribute none), FP64; dL_dT0, N doubles, the gradient with respect
 * to an initial temperature field T0 entering as g_i = w_i T0 (Sec. 4.2).
 * On return the current state is the recorded final state.
 *
 * lbm_adjoint_state copies the adjoint of the recorded initial populations
 * (d L / d f, 19 N floats; d L / d g, 7 N floats; mem) after lbm_adjoint_step. */
int lbm_record(lbm_ctx* ctx, int n, int K);
int lbm_adjoint_step(lbm_ctx* ctx, int n, const float* dL_drho, const float* dL_dT, double* dL_dTface,
                     double* dL_dT0);
int lbm_adjoint_state(lbm_ctx* ctx, float* f_bar, float* g_bar, int mem);

/* Batched stepping of many independent lattices (no counterpart in the
 * paper): one persistent cooperative launch per time step runs phases A,
 * force + D3Q19, D3Q7 and D over a tile list spanning every domain, with a
 * bounded grid-wide barrier between phases (a barrier that waits ~2 s without
 * progress aborts the launch: LBM_ERR_TIMEOUT from lbm_batch_sync), or, when
 * the autotuner finds it faster, one launch per phase over the same tile
 * list; runs of eight steps are replayed from a CUDA graph.
 *
 * lbm_batch_create takes n contexts made by lbm_init with FP32 storage, a
 * state, and the same stream (else LBM_ERR_ARG / LBM_ERR_STATE).  The contexts
 * keep their buffers and stay usable (lbm_get_state, lbm_macros, lbm_reduce);
 * they must outlive the batch.  lbm_batch_step advances every domain n steps
 * (asynchronous); lbm_batch_sync waits and returns the first error.
 * lbm_batch_tune times the candidate launch shapes on the domains' own
 * states, restores the states and their error flags and keeps the fastest:
 * the persistent launch (threads per CTA 128/256, CTAs per SM 1-4, cells per
 * tile 1024-8192) or one launch per phase over the same tile list (reported
 * as ctas_per_sm = 0).  Outputs may be NULL.
 * lbm_batch_cells returns the total number of cells.
 * After LBM_ERR_TIMEOUT from lbm_batch_sync the domains hold partial states
 * (some phases of the last step ran, others did not): set them again
 * (lbm_set_state) before stepping; lbm_batch_sync has already reset the
 * barrier and the abort flag, so the batch then steps like a new one.
 * lbm_batch_inject_stall (failure-detection tests) makes the next persistent
 * launch's first grid barrier unable to complete, so that its bounded waits
 * give up; LBM_ERR_ARG when the batch runs one launch per phase (no barrier). */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_batch** out, lbm_ctx* const* ctxs, int n);
int lbm_batch_tune(lbm_batch* batch, int* threads, int* ctas_per_sm, int* tile_cells);
int lbm_batch_step(lbm_batch* batch, int n);
int lbm_batch_sync(lbm_batch* batch);
long long lbm_batch_cells(const lbm_batch* batch);
int lbm_batch_inject_stall(lbm_batch* batch);
void lbm_batch_destroy(lbm_batch* batch);

/* Per-node Dirichlet temperature of non-periodic face `face` (Sec. 3.1): an
 * array over the face's two tangential coordinates, lower axis fastest
 * (z faces: nx*ny, x faces: ny*nz, y faces: nx*nz floats) (mem).  Edge and
 * corner nodes take the mean of the faces they lie on. */
int lbm_set_face_T(lbm_ctx* ctx, int face, const float* T_face, int mem);

/* Advances n >= 0 time steps; asynchronous on the context stream. */
int lbm_step(lbm_ctx* ctx, int n);

/* Failure detection test support (host-side injection; no GPU fault).
 * LBM_SCHED_FUSED: makes the next lbm_step wait on plane-completion counters that
 * nothing will advance (they are cleared while the step count is kept), so that its
 * bounded device-side waits give up after about 2 s; the launch then aborts.
 * LBM_SCHED_PHASES / LBM_SCHED_SLABS with staged kernels (FP32 lattices of at least
 * 622,592 cells whose planes divide into 256-cell tiles): the first CTA 0 of the next
 * staged launch expects 16 bytes more than its first tile's bulk copies bring, so that
 * its bounded mbarrier waits give up after about 1 s; it waits (bounded) for the copies
 * it issued, which all complete, and leaves its tiles unstepped.
 * Either way lbm_sync then returns LBM_ERR_TIMEOUT and the state is not to be used; the
 * context stays usable: lbm_set_state or lbm_restore clears the condition.
 * LBM_ERR_ARG for a context with neither; LBM_ERR_STATE for a fused context before its
 * first step. */
int lbm_inject_stall(lbm_ctx* ctx);

/* Macroscopic fields of the current state: rho = sum f (Eq. 3), the real
 * velocity u = (sum c f + F/2) / rho (Eq. 5; 0 at wall nodes) and T = sum g.
 * Each output N floats (mem) or NULL to skip.  Synchronises the stream. */
int lbm_macros(lbm_ctx* ctx, float* rho, float* ux, float* uy, float* uz, float* T, int mem);

/* FP64 reductions of the current state, host output:
 * out[0] = sum rho (mass), out[1] = sum rho c_v T, out[2] = droplet volume
 * sum clamp((rho - rho_v)/(rho_l - rho_v), 0, 1) (Sec. 4.2 d^2 law),
 * out[3] = number of cells whose populations are not finite.  Synchronises. */
int lbm_reduce(lbm_ctx* ctx, double out[4]);

/* Synchronises the stream and returns the first error any kernel flagged. */
int lbm_sync(lbm_ctx* ctx);

/* Integer maps used by the kernels, host outputs (any may be NULL):
 * map19[i*N + c] = destination slot i'*N + c' of population i leaving c
 * (bounce-back gives the opposite direction at c), -1 if it leaves through an
 * open face; map7 likewise for D3Q7 (-1 beyond any non-periodic face);
 * node_class[c] has bit f set when c lies on non-periodic face f.
 * Computed on the device by the same index code the step kernels use. */
int lbm_stream_map(lbm_ctx* ctx, int32_t* map19, int32_t* map7, uint8_t* node_class);

/* Frees everything the context owns; NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Static description of a status code. */
const char* lbm_status_string(int status);

/* Host helpers of Sec. 4 (Eq. 38 and the Maxwell construction); no device work. */
double lbm_Tc(const lbm_params* p);
int lbm_maxwell(const lbm_params* p, double T, double* rho_v, double* rho_l, double* p_sat);

/* Kernel timing.  While enabled, every kernel that lbm_step launches is
 * bracketed by CUDA events on the context stream.  lbm_profile(ctx, 1) clears
 * the counters and starts recording; lbm_profile(ctx, 0) stops.
 * lbm_profile_read synchronises on the recorded events and writes, for the
 * first nkinds kernel kinds, the number of launches and their total device
 * time in milliseconds since the last clear (host arrays, may be NULL).
 * Kinds: 0 phase A (macro/psi), 1 phase B (force/velocity), 2 phase C
 * (D3Q19 collide + stream), 3 phase D (boundary), 4 fused step, 5 phase C of
 * the D3Q7 lattice. */
int lbm_profile(lbm_ctx* ctx, int enable);
int lbm_profile_read(lbm_ctx* ctx, long long* launches, double* ms, int nkinds);

/* The reductions of lbm_reduce for caller-owned population buffers, with no
 * device allocation.  The paper has no counterpart: this exists for callers
 * that cannot call cudaMalloc when they need the diagnostics -- an application
 * that serves all device memory from its own pool and forbids allocations
 * after start-up, or a plug-in that receives device pointers from its host and
 * owns no lbm_ctx.
 *   f, g     device pointers to 19*n_cells and 7*n_cells floats (SoA layout above);
 *   cv, rho_v, rho_l   as in lbm_params;
 *   out      device pointer to 4 doubles, written as by lbm_reduce (mass,
 *            sum rho c_v T, droplet volume, count of non-finite cells);
 *   stream   cudaStream_t the two kernels are enqueued on (asynchronous).
 * Scratch: a fixed device array of 4096 x 4 doubles (128 KiB) inside the
 * library, held by every GPU that loads the library until the process exits.
 * n_cells may be at most 4096 * 8192 = 33,554,432; larger sizes return
 * LBM_ERR_ARG before any device work.  Every call looks up the array's device
 * address on the current device (cudaGetSymbolAddress, which enqueues no work)
 * and passes it to the kernels; make the first call on a device before any
 * stream capture, since that lookup may initialise the module on the device.
 * All calls share the one array, which keeps the last call's partial sums, so
 * calls that overlap on the GPU (other streams, other threads) race: serialise
 * them.  Every partial sum a call reads is written by that call first. */
int lbm_reduce_static(const float* f, const float* g, long long n_cells, double cv, double rho_v, double rho_l,
                      double* out, void* stream);

/* Kernel launches per time step within a long run.  When the face nodes are whole
 * z planes (x and y faces periodic without held temperature layers) and the
 * storage has no per-cell references, the slab schedule leaves the face rules
 * (phase D) of every step but the last of a call to the next step's phase A, so
 * a call adds its phase D launches once per sequence; lbm_step_launches counts
 * them: the exact number of kernel launches of lbm_step(ctx, n), -1 for a bad
 * argument. */
int lbm_launches_per_step(const lbm_ctx* ctx);
long long lbm_step_launches(const lbm_ctx* ctx, int n);

#ifdef __cplusplus
}
#endif
#endif
