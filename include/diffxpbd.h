/*
 * diffxpbd.h -- C ABI of the GB300 (sm_103a) differentiable XPBD library.
 *
 * The library runs the XPBD time step of DiffXPBD (Stuyck & Chen) and its exact discrete
 * adjoint on one GPU:
 *   forward  (Sec. 3.1, Eq. xpbdUpdateRule): inertial prediction
 *            p = x_n + dt v_n + dt^2 M^-1 f_ext, then `iters` Gauss-Seidel iterations
 *            that visit the constraint colors in order (Sec. 3.1, graph coloring), each
 *            constraint j taking the single-constraint XPBD update of Eq. xpbd
 *              dlambda = (-C_j - alpha~_j lambda_j) / (sum_i w_i |grad_i C_j|^2 + alpha~_j),
 *              alpha~_j = alpha_j / dt^2,   x_i += w_i grad_i C_j dlambda,
 *            then one collision pass (Sec. 4.6) over the contacts detected at p, and the
 *            velocity update v_{n+1} = (x_{n+1} - x_n) / dt.
 *   adjoint  (Sec. 4.2, Eq. rawAdjoint and Eq. gradientRule, in discrete form): the
 *            reverse-time sweep of the linearised constraint updates, replaying each step
 *            from its checkpoint, giving dL/d(compliance), dL/dx0, dL/dv0 (Sec. 5.5),
 *            dL/d(per-step global force) and dL/d(per-vertex force) (Sec. 5.6), and
 *            dL/d(plane height, sphere centre, sphere radius) (Sec. 4.6).
 *
 * Conventions (all entry points):
 *   - Every call returns an xpbd_status and never aborts.  On failure the thread-local
 *     message of xpbd_last_error() says why.  Errors found by kernels (non-finite state)
 *     are latched in a device word and reported by xpbd_sync_status().
 *   - "HOST" pointers are read during the call only.  "DEVICE" pointers are CUDA device
 *     memory owned by the caller; they must stay valid until the work queued on `stream`
 *     has finished.  `stream` is a cudaStream_t (NULL = legacy default stream); all GPU
 *     work of a call is queued on it and the call returns without synchronising unless
 *     stated otherwise.
 *   - A handle is not reentrant: calls on one handle must not overlap in time or run on
 *     two streams at once.  Distinct handles are independent.
 *   - Layouts: vertex arrays are [V][3] float32 row-major.  Constraint ids are global:
 *       [0, n_dist) distance, [n_dist, +n_bend) bending, then n_tet hydrostatic and
 *       n_tet deviatoric tet constraints.
 *   - Checkpoints (caller-owned DEVICE buffer of xpbd_checkpoint_bytes()): for each step
 *     n = 0..steps, V float4 positions (x, y, z, inverse mass) followed by V float4
 *     velocities (vx, vy, vz, 0).
 */
#ifndef DIFFXPBD_H
#define DIFFXPBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  XPBD_OK = 0,
  XPBD_ERR_INVALID = 1,    /* bad argument, index out of range, non-finite rest data   */
  XPBD_ERR_COLORING = 2,   /* a color has two constraints sharing a vertex, or the
                              coloring misses / repeats a constraint                    */
  XPBD_ERR_OOM = 3,        /* device allocation failed                                  */
  XPBD_ERR_CUDA = 4,       /* a CUDA runtime call failed                                */
  XPBD_ERR_NONFINITE = 5,  /* a kernel produced a NaN/Inf state (latched device word)   */
  XPBD_ERR_TIMEOUT = 6,    /* a bounded device wait gave up                             */
  XPBD_ERR_BOUNDS = 7      /* a size exceeds a fixed limit of the entry point           */
} xpbd_status;

enum { XPBD_COLLIDE_PLANE = 1, XPBD_COLLIDE_SPHERE = 2 };

typedef struct xpbd_solver* xpbd_handle;

/* Mesh, constraints and coloring.  All HOST pointers, copied by xpbd_create. */
typedef struct {
  int32_t n_vertices;
  const float* rest_x;          /* [V*3] rest positions: define spring rest lengths, hinge
                                   rest angles, tet reference shapes Dm^-1 and volumes    */
  const float* inv_mass;        /* [V] w = 1/m; 0 pins the vertex (infinite mass, Sec. 4.2.1) */
  int32_t n_dist;
  const int32_t* dist_idx;      /* [n_dist*2]   C = |x_a - x_b| - L                      */
  int32_t n_bend;
  const int32_t* bend_idx;      /* [n_bend*4] hinge edge v0-v1, wing v2 (side A), wing v3
                                   (side B); C = theta - theta0, theta the signed dihedral
                                   angle between nA = e x (x2-x0) and nB = (x3-x0) x e
                                   about e = x1 - x0 (Sec. 5.1 discrete bending)           */
  int32_t n_tet;
  const int32_t* tet_idx;       /* [n_tet*4] positively oriented; F = Ds Dm^-1,
                                   C_H = det F - gamma, C_D = sqrt(tr F^T F) (Sec. 5.2)   */
  const float* tet_gamma;       /* [n_tet] hydrostatic rest offset, or NULL for 1          */
  int32_t n_colors;
  const int32_t* color_offsets; /* [n_colors+1]; color c = color_order[offsets[c]..offsets[c+1]) */
  const int32_t* color_order;   /* [offsets[n_colors]] every colored constraint id exactly
                                   once: all m ids, or with tet_coupled all but the C_D ids */
  int32_t exec_mode;            /* How the colored sweep is launched; all modes give the same
                                   colored Gauss-Seidel results.  Phase plan: runs of
                                   consecutive colors whose constraints split into small
                                   vertex-disjoint components as one launch per run
                                   (vertices staged in shared memory).
                                   0: the phase plan when it needs at most a quarter of the
                                      launches of one launch per color (below that, one
                                      launch per color measured faster), else per color;
                                   1: one launch per color;
                                   2: the phase plan whenever it needs fewer launches.     */
  int32_t tet_coupled;          /* 0: each constraint is colored and updated on its own.
                                   1: each tet's C_H and C_D are updated together by one
                                   2x2 solve (S dlambda = -C - A~ lambda, S = G W G^T + A~;
                                   the neo-Hookean constraint pair of Sec. 3.2 follows
                                   Macklin and Mueller 2021, who update it this way);
                                   color_order then lists every id but the C_D ids
                                   n_dist + n_bend + n_tet + t, and the C_H id of tet t
                                   stands for the pair.  Multipliers, compliances and their
                                   gradients keep one entry per constraint (m).  Such
                                   models run one launch per color whatever exec_mode
                                   says; the serving entry points refuse them.  Other
                                   values fail with XPBD_ERR_INVALID.                       */
  int32_t n_memb;               /* orthotropic StVK membrane triangles (Sec. "Cloth Material
                                   Parameter Estimation"), coloring ids m + t.  Triangle t:
                                   C = (E_uu, E_vv, 2 E_uv) of the Green strain
                                   E = (F^T F - I)/2, F = [x1-x0, x2-x0] Dm^-1, Dm from the
                                   warp/weft rest coordinates; compliance block (A K)^-1
                                   with A the rest area and K = [C00 C01 0; C01 C11 0;
                                   0 0 C22] (xpbd_params.memb_stiffness); its three
                                   multipliers are solved together.  The serving entry
                                   points refuse models with membranes.                     */
  const int32_t* memb_idx;      /* [n_memb*3] vertices of each triangle                     */
  const float* memb_uv;         /* [n_memb*6] (u, v) rest coordinates of each triangle's
                                   three vertices (u warp, v weft); a triangle whose rest
                                   area is 0 fails with XPBD_ERR_INVALID                   */
} xpbd_model;

/* Per-call parameters.  The float fields are HOST values; the pointers are DEVICE. */
typedef struct {
  float dt;
  float gravity[3];             /* acceleration applied to free vertices                  */
  const float* compliance;      /* DEVICE [m] alpha_j for distance and bending constraints;
                                   for tet constraints the inverse modulus alpha_hat_j with
                                   alpha_j = alpha_hat_j / V_e (V_e the rest volume)      */
  const float* f_global;        /* DEVICE [steps*3] force added to every vertex at step n,
                                   or NULL                                                 */
  const float* f_vertex;        /* DEVICE [V*3] time-constant per-vertex force, or NULL   */
  int32_t collider_flags;       /* XPBD_COLLIDE_PLANE | XPBD_COLLIDE_SPHERE               */
  float plane_h;                /* plane y = plane_h, normal +y:  C = y - h - thickness    */
  float sphere[4];              /* centre cx, cy, cz and radius r:  C = |x - c| - r - thickness */
  float contact_compliance;     /* compliance of every contact spring                     */
  float thickness;              /* separation kept from the colliders                     */
  const float* f_vertex_steps;  /* DEVICE [steps*V*3] force on vertex i at step n, or NULL:
                                   the keyframe example's control variables (Sec. "Keyframe
                                   Simulation").  Not accepted by the serving API.         */
  const float* memb_stiffness;  /* DEVICE [n_memb*4] (C00, C11, C01, C22) per membrane
                                   triangle (NULL when n_memb = 0).  K must be finite and
                                   positive definite (C22 > 0); otherwise xpbd_sync_status
                                   reports XPBD_ERR_NONFINITE, as for a bad compliance.    */
} xpbd_params;

/* Gradient outputs.  DEVICE float64 buffers owned by the caller; each non-NULL buffer is
   overwritten (not accumulated into).  NULL skips that gradient. */
typedef struct {
  double* d_compliance;         /* [m] dL/d compliance (the xpbd_params.compliance entries) */
  double* d_x0;                 /* [V*3] dL/dx_0                                          */
  double* d_v0;                 /* [V*3] dL/dv_0                                          */
  double* d_f_global;           /* [steps*3] dL/dG_n                                      */
  double* d_f_vertex;           /* [V*3] dL/dW_i                                          */
  double* d_collider;           /* [5] dL/d(plane_h, cx, cy, cz, r)                        */
  double* d_f_vertex_steps;     /* [steps*V*3] dL/dF_{n,i} (force per vertex per step)    */
  double* d_memb_stiffness;     /* [n_memb*4] dL/d(C00, C11, C01, C22) per membrane         */
} xpbd_grads;

/* Build a solver.  Validates indices (XPBD_ERR_INVALID), the coloring
   (XPBD_ERR_COLORING: every constraint once; no vertex twice within a color) and the rest
   data; computes rest lengths, hinge angles, Dm^-1 and rest volumes from rest_x; sorts
   each color's constraints by type and first vertex and uploads them.  The order inside
   a color does not change results (its constraints are vertex-disjoint).  Synchronous. */
xpbd_status xpbd_create(const xpbd_model* model, xpbd_handle* out);

/* Release every device buffer the handle owns.  Synchronises the device first. */
xpbd_status xpbd_destroy(xpbd_handle h);

/* Sizes: number of vertices / constraints / colors of a handle. */
xpbd_status xpbd_sizes(xpbd_handle h, int32_t* n_vertices, int32_t* n_constraints, int32_t* n_colors);

/* Bytes of the checkpoint buffer for `steps` steps: (steps+1) * V * 32. */
size_t xpbd_checkpoint_bytes(xpbd_handle h, int32_t steps);

/* Device bytes the handle allocates for a forward or adjoint call with `iters`
   iterations (working state, multiplier and position tapes, gradient scratch); the
   library allocates them on first use and keeps them until xpbd_destroy or
   xpbd_release_workspace. */
size_t xpbd_workspace_bytes(xpbd_handle h, int32_t iters);

/* Free the handle's workspace (synchronises the device first); the next call that needs it
   allocates it again.  For a process that keeps many handles and runs them one at a time.
   The constraint records and the execution plan stay. */
xpbd_status xpbd_release_workspace(xpbd_handle h);

/* Forward simulation of `steps` steps (Sec. 3.1).  x0, v0: DEVICE [V*3].  Writes
   checkpoints 0..steps (checkpoint 0 = x0, v0).  Pinned vertices should start with
   v0 = 0. */
xpbd_status xpbd_forward(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                         const float* x0, const float* v0, float* checkpoints, void* stream);

/* Copy positions and velocities of checkpoint `step` into DEVICE [V*3] buffers (either
   may be NULL). */
xpbd_status xpbd_read_state(xpbd_handle h, const float* checkpoints, int32_t step, float* x_out,
                            float* v_out, void* stream);

/* Goal function of Sec. 4.1 with W = I, beta = 0 over keyframes:
     L = 1/2 sum_k |x_{n_k} - x*_k|^2
   key_steps HOST [n_keys]; targets DEVICE [n_keys*V*3].  Writes L (float64, reduced in a
   fixed order) to DEVICE loss_out[0] and dL/dx_{n_k} = x_{n_k} - x*_k (float32) to
   DEVICE seeds_out [n_keys*V*3] (either output may be NULL). */
xpbd_status xpbd_loss(xpbd_handle h, const float* checkpoints, int32_t n_keys,
                      const int32_t* key_steps, const float* targets, double* loss_out,
                      float* seeds_out, void* stream);

/* Reverse sweep (discrete adjoint).  checkpoints: as written by xpbd_forward with the same
   params/steps/iters.  Seeds dL/dx_n for n = seed_steps[s] (HOST [n_seeds], each in
   0..steps) in seed_dx (DEVICE [n_seeds*V*3]); seed_dv_T DEVICE [V*3] dL/dv_steps or NULL.
   Recomputes each step's in-step positions and multipliers from its checkpoint; keeps
   positions, multipliers and adjoint states in float32 and reduces parameter gradients
   across constraints and steps in float64 in a fixed order (deterministic). */
xpbd_status xpbd_adjoint(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                         const float* checkpoints, int32_t n_seeds, const int32_t* seed_steps,
                         const float* seed_dx, const float* seed_dv_T, const xpbd_grads* out,
                         void* stream);

/* ---- Sparse checkpoints (recompute instead of storing every step) ----------------------
   The paper stores every step's state for the adjoint pass and names the resulting memory
   growth as a limitation (section "Discussion, Limitations, and Future Work").  These
   calls store the state (x, v) only at every `stride`-th step and at the last step; the
   reverse sweep recomputes the states inside
   each stride from the stored one with the same forward kernels (one extra forward pass)
   and then reverses them exactly as xpbd_adjoint does, so its gradients are bit-identical
   to xpbd_adjoint's.  Checkpoint memory falls from (steps+1) to about steps/stride + 2
   states, plus stride-1 recomputed states (32 B per vertex each). */

/* Number of stored states for `steps` steps: steps/stride + 1, plus 1 when stride does not
   divide steps (the last state).  -1 for steps < 0 or stride < 1.  Host only. */
int32_t xpbd_sparse_slots(int32_t steps, int32_t stride);

/* Slot of step `step` in a sparse checkpoint buffer, or -1 if that step is not stored.
   Host only.  xpbd_read_state and xpbd_loss read a sparse buffer when given slot indices. */
int32_t xpbd_sparse_slot(int32_t steps, int32_t stride, int32_t step);

/* Forward simulation like xpbd_forward, writing only the stored states to `checkpoints`
   (DEVICE [xpbd_sparse_slots(steps, stride) * V * 8], same per-state layout).  The states
   in between pass through a two-state buffer the handle allocates on first use
   (64 B per vertex).  XPBD_ERR_INVALID for stride < 1. */
xpbd_status xpbd_forward_sparse(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                const float* x0, const float* v0, int32_t stride, float* checkpoints,
                                void* stream);

/* Reverse sweep from a sparse checkpoint buffer written by xpbd_forward_sparse with the same
   params/steps/iters/stride.  Seeds, outputs and determinism as xpbd_adjoint (seeds may sit
   at any step).  The handle allocates (stride-1) recomputed states on first use. */
xpbd_status xpbd_adjoint_sparse(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                const float* checkpoints, int32_t stride, int32_t n_seeds,
                                const int32_t* seed_steps, const float* seed_dx, const float* seed_dv_T,
                                const xpbd_grads* out, void* stream);

/* ---- The paper's implicit adjoint (Sec. "Adjoint State Computation", Eq. adjointXPBD) ----
   Instead of reversing the iterations, each step is differentiated as if solved exactly:
   with x_{n+1} and the multipliers lambda the step ended with,
     A = M + sum_j B_j,  B_j = grad C_j^T grad C_j / alpha~_j - lambda_j hess C_j
   over the constraints and the step's active contacts, each block projected to positive
   semi-definite in the constraint's relative coordinates when pd_project
   (Sec. "Positive Definite Projection"); A y = xbar_{n+1} + vbar_{n+1}/dt is solved on the
   free vertices by preconditioned conjugate gradients, pinned vertices filtered out
   (Sec. "Linear System Filtering"), the preconditioner a 3x3 block Jacobi or, for a grid
   model, a geometric multigrid V-cycle (below); then pbar = M y (free), pbar = b - A y
   (pinned), alphabar~_j += -(lambda_j / alpha~_j) grad C_j . y, and the prediction adjoint
   as in xpbd_adjoint.  A membrane is one block, G^T alpha~^-1 G - sum_k lambda_k hess C_k
   over its three rows, with alphabar~ += -(alpha~^-1 G y) lambda^T (then dL/dK in
   d_memb_stiffness).  The gradient differs from xpbd_adjoint's by design: XPBD's
   iterations leave the primal residual M (x - p) - grad C^T lambda nonzero, so this is the
   derivative of the exactly solved step at XPBD's end state. */
typedef struct {
  double cg_tol;                /* stop when |r| <= cg_tol |b| (free vertices, float64)   */
  int32_t cg_max_iters;         /* per step                                                */
  int32_t pd_project;           /* 1: project every block (the paper); 0: raw blocks       */
  int32_t* cg_iters_out;        /* HOST [steps] iterations used per step, or NULL          */
  /* Multigrid preconditioner (mg_nx = 0: block Jacobi).  With mg_nx, mg_ny > 0 the V
     vertices must form an mg_nx x mg_ny grid, vertex (i, j) = j * mg_nx + i, V = mg_nx *
     mg_ny, and every constraint must couple only vertices at most two cells apart in each
     grid direction; otherwise the call returns XPBD_ERR_INVALID.  Levels: 5x5 stencils of
     3x3 float64 blocks, Galerkin coarse operators with bilinear prolongation down to at
     most 4x4 vertices (inverted densely), symmetric Gauss-Seidel smoothing.  The V-cycle is
     symmetric positive definite when A is (pd_project = 1 guarantees it).  Each call
     captures its V-cycle once into a CUDA graph on a private stream and replays it on
     `stream` (launched directly if capture fails).  Workspace:
     about 2.6 KB of device memory per vertex (+108 B with line smoothing).             */
  int32_t mg_nx, mg_ny;
  int32_t mg_lines;             /* level-0 smoother: 0 point Gauss-Seidel (9 colours);
                                   +1 / -1 exact solves along the grid diagonals
                                   x - y = c / x + y = c (5 colours), for a cloth
                                   triangulated along that diagonal with hinges only on
                                   its axis-aligned edges (such a sheet folds freely along
                                   the diagonals)                                          */
  int32_t mg_sweeps;            /* smoothing sweeps before and after each coarse
                                   correction (0 means 1)                                  */
} xpbd_implicit_opts;

/* Implicit-adjoint gradients from dense checkpoints (as xpbd_adjoint: seeds, outputs,
   determinism).  Every compliance must be > 0.  d_collider must be NULL (no collider
   gradient is formed).  Synchronises `stream` a few times per step (convergence checks).
   Works on the per-color records whatever exec_mode the handle has. */
xpbd_status xpbd_adjoint_implicit(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                  const float* checkpoints, int32_t n_seeds, const int32_t* seed_steps,
                                  const float* seed_dx, const float* seed_dv_T, const xpbd_grads* out,
                                  const xpbd_implicit_opts* opts, void* stream);

/* ---- Tet materials (Sec. "Volumetric Material Parameter Estimation") -------------------
   An object of several materials: material k has Lame parameters mu_k = a_k^2 and
   lambda_k = b_k^2 (optimising over a, b keeps them positive).  A tet of material k then
   has the inverse moduli alpha_hat_D = 1/a_k^2 (deviatoric) and alpha_hat_H = 1/b_k^2
   (hydrostatic), the tet entries of xpbd_params.compliance. */

/* Writes the tet entries of `compliance` (DEVICE [m], caller order: hydrostatic constraints
   at n_dist+n_bend+t, deviatoric at n_dist+n_bend+n_tet+t) from tet_material (DEVICE
   [n_tet], 0..n_materials-1), a and b (DEVICE [n_materials]); other entries untouched.
   A material id out of range latches XPBD_ERR_INVALID for xpbd_sync_status. */
xpbd_status xpbd_material_compliance(xpbd_handle h, int32_t n_materials, const int32_t* tet_material,
                                     const float* a, const float* b, float* compliance, void* stream);

/* Chain rule to the material parameters: from d_compliance (DEVICE [m] float64, as written
   by an adjoint call) writes dL/da and dL/db (DEVICE [n_materials] float64; either may be
   NULL), each a fixed-order sum over the material's tets (deterministic). */
xpbd_status xpbd_material_gradient(xpbd_handle h, int32_t n_materials, const int32_t* tet_material, const float* a,
                                   const float* b, const double* d_compliance, double* d_a, double* d_b,
                                   void* stream);

/* Synchronise `stream` and report (then clear) the device error word of the handle:
   XPBD_ERR_TIMEOUT if, since the last check, a bounded wait of a phase kernel gave up (the
   message says whether that kernel also gave up waiting for its own copies in flight before
   returning, after which the CUDA context may be unusable); XPBD_ERR_NONFINITE if a call was given a negative or non-finite compliance or a step
   produced a non-finite state. */
xpbd_status xpbd_sync_status(xpbd_handle h, void* stream);

/* Self-test of failure detection in the phase kernels.  Every wait of a phase kernel (for a
   staged copy, or for the consumers to release a stage) gives up after a bounded time,
   latches bit 4 of the device error word and lets the kernel return, so the context stays
   usable.  This call launches one CTA of the handle's first phase kernel whose producer
   issues no copies and whose waits give up after ~2 ms: every consumer wait runs out.
   Queued on `stream`; the caller then expects XPBD_ERR_TIMEOUT from xpbd_sync_status.
   It writes no simulation state.  XPBD_ERR_INVALID if the handle runs no phase kernels.
   The paper has no counterpart. */
xpbd_status xpbd_selftest_wait_timeout(xpbd_handle h, void* stream);

/* Allocation-free forward simulation.  The paper has no counterpart: this entry point
   exists for callers that cannot allocate device memory when they simulate, for example
   because another allocator owns the device memory under a fixed budget, or because the
   call sits in a latency-critical loop where cudaMalloc/cudaFree would synchronise the
   device.  Such a caller creates the handle during start-up (xpbd_create allocates the
   handle's constraint records) and afterwards calls this instead of xpbd_forward, which
   allocates its working state on first use.

   Same arguments, steps and results as xpbd_forward (it always runs one launch per color;
   with a handle in the multi-color phase mode the results agree with xpbd_forward's to
   float32 rounding).  The working state (predicted positions, multipliers, contact state)
   lives in one fixed device array inside the library, sized for at most
   XPBD_STATIC_MAX_VERTICES vertices and XPBD_STATIC_MAX_CONSTRAINTS multiplier slots (one
   per constraint, four per membrane; about 3.1 MiB, held by every GPU that loads the
   library until the process exits); larger models get XPBD_ERR_BOUNDS before any GPU work.
   The call allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Set-up
   happens in xpbd_create: with the handle's device current, it looks up the array's device
   address (cudaGetSymbolAddress, which under CUDA's lazy module loading is also when the
   array's memory is taken) and stores it in the handle.  Each device has one copy of the
   array, shared by every call on that device and keeping what the last call left in it
   (nothing in it needs clearing: each step overwrites the positions and contact flags, and
   each step's first iteration reads no multiplier); calls whose GPU work overlaps in time
   on one device (different streams, or different handles) race on it and give wrong
   results, so serialise them. */
#define XPBD_STATIC_MAX_VERTICES 65536
#define XPBD_STATIC_MAX_CONSTRAINTS 393216
xpbd_status xpbd_forward_static(xpbd_handle h, const xpbd_params* p, int32_t steps, int32_t iters,
                                const float* x0, const float* v0, float* checkpoints, void* stream);

/* ---------------------------------------------------------------- serving
   Continuous batching of forward + gradient requests (one GPU).  A request is one solve:
   `steps` steps of `iters` iterations from (x0, v0), the loss L = 1/2 |x_steps - target|^2
   (Sec. 4.1 with one keyframe at the last step), and the full reverse sweep.  The server
   keeps every admitted request's state, checkpoints and tapes resident and advances all
   of them together: each tick runs the next pass (a color of a forward or reverse
   iteration, a contact pass, a prediction, ...) of every resident request, reading a
   concatenated table of those passes; one cooperative launch of the dispatch kernel runs
   a batch of ticks, its blocks meeting at a grid-wide barrier between ticks (every wait
   bounded: one that runs out is reported as XPBD_ERR_TIMEOUT by a later
   xpbd_server_run, and that batch's results are invalid).  Requests submitted while others
   run are admitted at the next xpbd_server_run call, in submission order, as soon as a
   slot is free and their workspace fits in the memory budget; their passes then share the
   GPU with the requests already running.  Every request computes exactly the values it
   would compute alone on the server: its passes run the same per-element code in the same
   order, whatever else shares the launch.

   Ownership: the request's handle (one handle per in-flight request: the server writes the
   handle's per-call parameters into its records), params pointers, x0, v0, target and the
   output buffers belong to the caller and must stay valid until xpbd_server_poll reports
   the request done.  The server allocates each request's workspace (stream-ordered, on the
   server's stream) at admission and frees it when the request completes. */
typedef struct xpbd_server_t* xpbd_server;

typedef struct {
  xpbd_handle handle;       /* model of the request                                       */
  xpbd_params params;       /* as for xpbd_forward (device pointers stay caller-owned)     */
  int32_t steps, iters;
  const float* x0;          /* DEVICE [V*3]                                                */
  const float* v0;          /* DEVICE [V*3]                                                */
  const float* target;      /* DEVICE [V*3] target positions at the last step              */
  double* loss_out;         /* DEVICE [1] L (float64), or NULL                             */
  xpbd_grads grads;         /* DEVICE outputs as for xpbd_adjoint (NULL entries skipped)   */
} xpbd_request;

typedef struct {
  int64_t submitted, admitted, completed;
  int32_t pending, active;  /* waiting for admission / resident on the GPU                 */
  size_t bytes_in_use, budget;
  int64_t ticks;            /* ticks dispatched so far (one cooperative launch per batch)  */
  int64_t items;            /* passes executed by them                                     */
  int64_t batches;          /* cooperative launches so far                                 */
  double host_wait_s;       /* host time xpbd_server_run spent waiting for the GPU (a batch
                               table still in use)                                         */
  double host_build_s;      /* host time spent building batch tables and launching         */
} xpbd_server_stats;

/* Device bytes a request allocates at admission (checkpoints, tapes, gradient state). */
size_t xpbd_request_bytes(xpbd_handle h, int32_t steps, int32_t iters, int32_t collider_flags);

/* Create a server on `stream` (cudaStream_t) that keeps at most `max_slots` requests
   resident and at most `hbm_budget` bytes of request workspace (0: 90% of the device
   memory free now).  Allocates its dispatch tables (device and pinned host memory). */
xpbd_status xpbd_server_create(size_t hbm_budget, int32_t max_slots, void* stream, xpbd_server* out);

/* Wait for the server's work, free everything it owns (requests not yet polled are
   dropped). */
xpbd_status xpbd_server_destroy(xpbd_server s);

/* Queue a request (HOST struct, copied).  XPBD_ERR_OOM if its workspace alone exceeds the
   budget; XPBD_ERR_INVALID for bad arguments.  Returns a ticket. */
xpbd_status xpbd_server_submit(xpbd_server s, const xpbd_request* r, uint64_t* ticket);

/* Retire finished requests, admit queued ones that fit, and queue a batch of up to
   `max_ticks` ticks (at most 256; fewer if every resident request finishes) as one
   cooperative launch on the server's stream.  Returns without waiting for the GPU; at most
   two batches are in flight.  XPBD_ERR_TIMEOUT if a grid barrier of an earlier batch gave
   up.  *active_out (may be NULL) receives the number of resident requests afterwards. */
xpbd_status xpbd_server_run(xpbd_server s, int32_t max_ticks, int32_t* active_out);

/* *done = 1 once every pass of the request has finished on the GPU (its outputs are then
   valid and its workspace freed), else 0.  Non-blocking.  Polling a completed ticket
   again returns XPBD_ERR_INVALID. */
xpbd_status xpbd_server_poll(xpbd_server s, uint64_t ticket, int32_t* done);

xpbd_status xpbd_server_get_stats(xpbd_server s, xpbd_server_stats* out);

/* Kernel launch statistics.  Every kernel launch of a handle is counted per class; while
   profiling is enabled each launch is also bracketed by two CUDA events recorded on the
   stream it is launched on, so `ms` is the summed device time of that class.  `units` is
   the number of constraints (projection and reverse classes) or vertices (per-vertex
   classes) the launches processed. */
enum {
  XPBD_K_FWD_DIST = 0, XPBD_K_FWD_BEND, XPBD_K_FWD_TETH, XPBD_K_FWD_TETD, XPBD_K_FWD_CONTACT,
  XPBD_K_REPLAY_DIST, XPBD_K_REPLAY_BEND, XPBD_K_REPLAY_TETH, XPBD_K_REPLAY_TETD, XPBD_K_REPLAY_CONTACT,
  XPBD_K_VJP_DIST, XPBD_K_VJP_BEND, XPBD_K_VJP_TETH, XPBD_K_VJP_TETD, XPBD_K_VJP_CONTACT,
  XPBD_K_PREDICT, XPBD_K_VELOCITY, XPBD_K_ADJ_OTHER, XPBD_K_OTHER,
  XPBD_K_FWD_PHASE, XPBD_K_REPLAY_PHASE, XPBD_K_VJP_PHASE,
  XPBD_K_FWD_MEMB, XPBD_K_REPLAY_MEMB, XPBD_K_VJP_MEMB,
  XPBD_KERNEL_CLASSES
};

typedef struct {
  int64_t launches;        /* launches counted since the last xpbd_profile() call          */
  int64_t units;           /* constraints or vertices processed by them                    */
  double ms;               /* summed event time of the timed launches                      */
  int64_t timed_launches;  /* launches bracketed by events (0 while profiling is off)      */
  double alg_bytes;        /* algorithmic bytes the launches must move: records, multipliers,
                              tapes and vertex state at one read and one write per vertex
                              per launch (0 for classes without a byte model)              */
} xpbd_kernel_stat;

/* Execution plan of a handle: *uses_phases = 1 when the forward and reverse sweeps run
   multi-color launches, with *n_phases launches per iteration (else one per color). */
xpbd_status xpbd_exec_info(xpbd_handle h, int32_t* uses_phases, int32_t* n_phases);

/* Synchronise the device, reset the counters and turn event timing on (enable != 0) or
   off.  Timing adds two event records per launch on the launching stream. */
xpbd_status xpbd_profile(xpbd_handle h, int32_t enable);

/* Synchronise the device and fill out[XPBD_KERNEL_CLASSES]. */
xpbd_status xpbd_profile_read(xpbd_handle h, xpbd_kernel_stat* out);

/* Name of a kernel class ("fwd_dist", "vjp_bend", ...), or "" if out of range. */
const char* xpbd_kernel_class_name(int32_t cls);

/* Thread-local description of the last failure (empty string if none). */
const char* xpbd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DIFFXPBD_H */
