/*
 * kamino.h -- C ABI of the GB300 (sm_103a) constrained forward-dynamics step.
 *
 * The library advances many independent "worlds" of rigid bodies in maximal coordinates by one
 * time step each (Kamino, arXiv 2603.16536):
 *   - body kinematics and the block-diagonal mass matrix             (Sec. 3, Eq. 1)
 *   - joint constraints f(q) = 0, incl. loop closures, and frictional contacts with a Baumgarte
 *     bias v*, assembled into the constraint Jacobian J              (Sec. 3, Eq. 2)
 *   - the Delassus matrix D = J M^-1 J^T and free velocity v_f       (Sec. 4, Eq. 4)
 *   - Jacobi preconditioning, a regularised factorisation of D + (eta + rho) I computed once per
 *     step, and the Proximal-ADMM iteration with De Saxce correction, friction-cone projection
 *     and Nesterov acceleration with adaptive restart                (Sec. 4, Alg. 1, Sec. 4.1)
 *   - semi-implicit Euler with the SO(3) exponential map             (Sec. 3)
 * Every stage runs in this library's own CUDA kernels.  There is no CPU fallback: every entry
 * point that needs the GPU returns KAMINO_E_CUDA when no usable device is present.
 *
 * Conventions shared by every buffer:
 *   - gravity is a model parameter; the ground plane is z = 0 with normal +z;
 *   - a body's frame is its centre of mass and principal frame (diagonal inertia);
 *   - pose q = (r[3], quat[4] stored x,y,z,w); twist u = (v[3], omega[3]), omega in the world frame;
 *   - a joint frame is (pos[3], quat[4]) in its body's frame.  Revolute: hinge about the frame's
 *     e3.  Prismatic: slide along e3.  Universal: free about e1 of the parent frame and e2 of the
 *     child frame.  Spherical: point.  Fixed: weld.  joint_parent = -1 attaches to the world;
 *   - constraint rows of a world: the joints' rows in joint order (revolute 5, prismatic 5,
 *     universal 4, spherical 3, fixed 6), then one (t1, t2, n) triple per active contact in
 *     candidate order.  A contact candidate is active when its signed distance is below
 *     params.margin.
 *
 * Ownership: all host pointers passed in are read during the call only; the caller keeps them.
 * Device memory of a model is allocated by the library (cudaMalloc) and freed by
 * kamino_model_destroy.  State memory is either a caller-provided device buffer (e.g. from the
 * PyTorch caching allocator) that must outlive the state, or allocated by the library when the
 * buffer pointer is NULL.  Calls that take a stream are asynchronous on that stream (NULL = the
 * legacy default stream); host-detectable errors are returned before anything is enqueued.
 * Errors never cross the ABI as exceptions; kamino_last_error() gives a message for the calling
 * thread's last failed call.
 */
#ifndef KAMINO_H
#define KAMINO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KAMINO_OK = 0,
    KAMINO_E_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, a bad parameter       */
    KAMINO_E_TOPOLOGY = 2,      /* inconsistent world description (indices, offsets, masses)   */
    KAMINO_E_NOMEM = 3,         /* device allocation failed or caller buffer too small        */
    KAMINO_E_CUDA = 4,          /* a CUDA runtime call failed (also: no device present)       */
    KAMINO_E_NONFINITE = 5,     /* not returned: per-world failures are status bits (kamino_residual) */
    KAMINO_E_TIMEOUT = 6,       /* not returned: a device wait that expires sets KAMINO_WORLD_TIMEOUT */
    KAMINO_E_UNSUPPORTED = 7    /* a size this build does not support (e.g. too many rows)     */
} kamino_status;

enum { KAMINO_JOINT_REVOLUTE = 0, KAMINO_JOINT_PRISMATIC = 1, KAMINO_JOINT_UNIVERSAL = 2,
       KAMINO_JOINT_SPHERICAL = 3, KAMINO_JOINT_FIXED = 4 };
enum { KAMINO_TERRAIN_NONE = 0, KAMINO_TERRAIN_PLANE = 1, KAMINO_TERRAIN_HEIGHTFIELD = 2 };
/* Arithmetic of a model.  KAMINO_FP32: FP32 storage and arithmetic, the swept FP32 inverse applied
 * with FP32 FMA.  KAMINO_MIXED: FP32 storage; the factorisation's rank-16 updates are TF32 tensor-
 * core products with FP32 accumulation (tcgen05 into the matrix held in tensor memory for worlds of
 * up to 256 padded rows run by a whole CTA, mma.sync otherwise); the inverse is applied in FP32
 * from tensor memory, or, for larger worlds and sub-CTA groups, as BF16 tiles on tensor cores
 * (FP32 accumulation); every iteration refines against the FP32 matrix-free residual.
 * KAMINO_FP64: FP64 throughout.  In every mode the reduced-precision inverse only preconditions
 * that refinement step. */
enum { KAMINO_FP32 = 0, KAMINO_FP64 = 1, KAMINO_MIXED = 2 };
/* warm start of Alg. 1 (Sec. 4.1): zero, the impulses cached by the previous step, or impulses
 * supplied by the caller through KAMINO_BUF_WARM (e.g. a learned predictor). */
enum { KAMINO_WARM_COLD = 0, KAMINO_WARM_CACHED = 1, KAMINO_WARM_EXTERNAL = 2 };

/* per-world status bits in kamino_residual.status.  NONFINITE: the step produced a non-finite
 * velocity; the world's state and impulse cache are left as they were before the step.  TIMEOUT: a
 * bounded device wait (the tensor cores' completion signal in the mixed-precision factorisation)
 * expired twice; the world is abandoned for this step, its state left as it was. */
enum { KAMINO_WORLD_NOT_CONVERGED = 1, KAMINO_WORLD_NONFINITE = 2, KAMINO_WORLD_TIMEOUT = 4,
       KAMINO_WORLD_STALLED = 8 };

typedef struct {
    double eta;        /* proximal regularisation, Alg. 1 (scaled units), >= 0              */
    double rho;        /* augmented-Lagrangian penalty, Alg. 1 (scaled units), > 0          */
    double beta;       /* Baumgarte factor of the bias v* (Sec. 3), in [0, 1]               */
    double margin;     /* contact activation distance in metres, >= 0                       */
    int32_t nesterov;  /* 1: Nesterov acceleration with adaptive restart (Sec. 4.1)         */
    int32_t precond;   /* 1: Jacobi preconditioning P = diag(D)^-1/2 (Sec. 4.1)              */
    int32_t warm_mode; /* KAMINO_WARM_*                                                       */
    int32_t refine64;  /* 1: when tol < KAMINO_REFINE64_BELOW, once r_p and r_d fall below that
                        * level the PADMM iteration finishes in FP64 refinement: the right-hand
                        * side (from the FP64 free velocity), the refinement residual b + A x and
                        * the iterates x, y, z are FP64, the correction still comes from the
                        * reduced-precision inverse (FP32 and MIXED precision; FP64 worlds always
                        * are FP64).  0: FP32 throughout.                                         */
    int32_t integrator; /* KAMINO_INTEGRATOR_*: time stepping of Sec. 3                            */
    int32_t cr_iters;  /* 0: dense formulation (the Delassus matrix assembled and factorised once
                        * per step, Sec. 5.1).  k >= 1: sparse formulation (Sec. 5.1): D applied
                        * matrix-free from the rows, each PADMM x-step k Conjugate Residual
                        * iterations warm-started at the previous x (the paper uses 9)         */
    int32_t ncp_stop;  /* 0: a world has converged when Sec. 4.1's residuals r_p, r_d, r_c are below
                        * tol (the paper's test).  1: in addition, the natural-map NCP residual of
                        * the iterate's (lambda, u+) on the contact and joint-limit blocks
                        * (kamino_residual.r_ncp) must be below tol; it is evaluated only in the
                        * iterations whose residuals pass, and the world iterates on otherwise. */
    int32_t stall_window; /* 0: off.  W > 0 (dense formulation, with ncp_stop): every W iterations, a
                        * world whose r_p and r_c are below tol but whose r_d is not also stops when
                        * the natural-map residual is below tol and u+ moved by less than tol
                        * (relative to max(|u+|inf, |g| dt)) over the last W iterations: the dual
                        * residual's floor of redundant rows, which no iteration removes and which
                        * leaves u+ (nearly) fixed.  Reported as KAMINO_WORLD_STALLED. */
    int32_t schedule;  /* KAMINO_SCHEDULE_*: order in which the one-CTA-per-world launch takes the
                        * worlds (results do not depend on it; every world is independent) */
    int32_t residual_every; /* dense formulation: every PADMM x-step is one refinement step
                        * x^i = x^{i-1} - A^-1 c with the swept (reduced-precision) inverse.
                        * 0 or 1: c = b^i + A x^{i-1}, the residual evaluated matrix-free from the
                        * rows in every iteration.  K >= 2: evaluated in iterations 1, K+1, 2K+1, ...
                        * and in every iteration of the FP64 end game; the others take
                        * c = b^i - b^{i-1}, which equals the residual when the previous x-step was
                        * solved exactly.  What the reduced-precision inverse leaves is corrected
                        * at the next evaluated iteration, so the fixed point is the same; the
                        * skipped iterations save the per-body gather, the residual rows and one
                        * barrier.  K is capped at 4 where the inverse is held as BF16 tiles (mixed
                        * precision beyond tensor memory).  Ignored by the sparse formulation. */
} kamino_solver_params;

/* IN_ORDER: world w in CTA w.  LONGEST_FIRST: before each step a one-CTA kernel orders the worlds by
 * the PADMM iterations of their previous step (counting sort, most first), so that the worlds that
 * will run longest start first and do not extend the end of the launch (the SMs take CTAs in launch
 * order).  On a state's first step (no previous report) the order is arbitrary. */
enum { KAMINO_SCHEDULE_IN_ORDER = 0, KAMINO_SCHEDULE_LONGEST_FIRST = 1 };

/* Time stepping (Sec. 3).  EULER: semi-implicit Euler, everything evaluated at the start-of-step
 * pose q-, then q+ = q- (+) dt u+.  MIDPOINT: Moreau-Jean, kinematics, rows, contacts and biases
 * evaluated at the half-step pose q_m = q- (+) (dt/2) u-, then q+ = q_m (+) (dt/2) u+.  (+) moves
 * positions along v and orientations by the exponential map of the world-frame angular velocity. */
enum { KAMINO_INTEGRATOR_EULER = 0, KAMINO_INTEGRATOR_MIDPOINT = 1 };
#define KAMINO_MAX_CR_ITERS 64

/* Scaled-unit residual level below which refine64 switches the refinement residual to FP64: the
 * FP32 residual's own rounding (~1e-6 on the closed-loop bipeds) is then no longer small beside it. */
#define KAMINO_REFINE64_BELOW 1e-5

/* World description, sum-allocated over worlds: world w owns bodies
 * [world_body_offset[w], world_body_offset[w+1]) and likewise joints and contact candidates.
 * Body indices inside joint_parent / joint_child / contact_body are LOCAL to the world. */
typedef struct {
    int32_t num_worlds;
    int32_t precision;                  /* KAMINO_FP32, KAMINO_MIXED or KAMINO_FP64            */
    const int32_t *world_body_offset;   /* [W+1] */
    const int32_t *world_joint_offset;  /* [W+1] */
    const int32_t *world_contact_offset;/* [W+1] */
    const int32_t *world_num_actuators; /* [W]   length of the world's actuation vector        */
    const double  *world_mu;            /* [W]   Coulomb friction coefficient, >= 0            */
    const double  *body_mass;           /* [B]   kg, > 0                                       */
    const double  *body_inertia;        /* [B*3] principal moments, kg m^2, > 0                */
    const int32_t *joint_type;          /* [J]   KAMINO_JOINT_*                                */
    const int32_t *joint_parent;        /* [J]   local body index or -1 (world)                */
    const int32_t *joint_child;         /* [J]   local body index                              */
    const int32_t *joint_actuator;      /* [J]   slot in the actuation vector or -1            */
    const double  *joint_frame_parent;  /* [J*7] pos(3) + quat xyzw(4) in the parent frame    */
    const double  *joint_frame_child;   /* [J*7] pos(3) + quat xyzw(4) in the child frame      */
    const int32_t *contact_body;        /* [C]   local body index                              */
    const double  *contact_point;       /* [C*3] point in the body frame                       */
    double gravity[3];
    int32_t terrain_kind;               /* KAMINO_TERRAIN_*                                     */
    int32_t hf_nx, hf_ny;               /* heightfield vertex counts (>= 2 each)                */
    double hf_origin[2];                /* world (x, y) of vertex (0, 0)                        */
    double hf_cell;                     /* vertex spacing, > 0                                  */
    const double *hf_heights;           /* [ny*nx] heights, vertex (i, j) at [j*nx + i]         */
    const double *body_q0;              /* [B*7] initial poses (NULL: origin, identity)         */
    const double *body_u0;              /* [B*6] initial twists (NULL: zero)                    */
    kamino_solver_params params;
    /* Joint-space dynamics on the joint coordinate d of revolute and prismatic joints (Sec. 3; Eq. 2's
     * R and v*, Eq. 4's D = J M^-1 J^T + R).  NULL: none.
     * joint_drive[j*5] = (mode, Kp, Kd, armature, damping), all >= 0 and finite.  mode
     * KAMINO_DRIVE_PD: the joint's actuation value is the position target of an implicit PD
     * controller (zero velocity target) and is not applied as a torque; KAMINO_DRIVE_TORQUE: the
     * actuation stays a torque/force and the row carries armature and damping only.  A joint with a
     * nonzero drive gets one regularised row after the joint rows, whose impulse over the step is
     * lambda = I_a (d'- - d'+) + dt Kp (target - d - dt d'+) - dt (Kd + b) d'+, i.e. R = 1/C and
     * v* = -(I_a d'- + dt Kp (target - d)) / C with C = I_a + dt^2 Kp + dt (Kd + b).
     * joint_limit[j*2] = (lower, upper) on d, +-INFINITY for none: every finite bound is a unilateral
     * row 0 <= lambda ⟂ g >= 0 (g = d - lower, upper - d), active when g < params.margin, with the
     * contact normal's bias (g/dt while g > 0, beta g/dt once violated).  Constraint rows of a world
     * are then: joint rows, drive rows (joint order), active limit rows (joint order, lower before
     * upper), contact triples; the impulse cache holds the joint and drive rows, one impulse per
     * finite bound, then 3 per contact candidate. */
    const double *joint_drive;          /* [J*5] or NULL                                        */
    const double *joint_limit;          /* [J*2] or NULL                                        */
} kamino_model_desc;

enum { KAMINO_DRIVE_TORQUE = 0, KAMINO_DRIVE_PD = 1 };

typedef struct {
    int32_t num_worlds;
    int32_t num_bodies;        /* B, all worlds                                              */
    int32_t max_bodies;        /* max bodies of one world                                    */
    int32_t max_rows;          /* max constraint rows of one world (all candidates active)   */
    int32_t n_act_max;         /* row length of the actuation input [W][n_act_max]           */
    int32_t cache_len;         /* length of the impulse cache / external warm-start buffer  */
    int32_t precision;
    int32_t threads_per_world; /* CTA size of the step kernel                                */
    int64_t smem_bytes;        /* dynamic shared memory of one world's CTA                   */
} kamino_model_info;

/* Per-world solver report (8 words), written by kamino_step (Sec. 4.1, convergence budget). */
typedef struct {
    int32_t iterations;        /* PADMM iterations run                                       */
    int32_t status;            /* KAMINO_WORLD_* bits, 0 = converged and finite              */
    int32_t num_rows;          /* constraint rows this step                                  */
    int32_t num_contacts;      /* active contacts this step                                  */
    float r_primal;            /* ||x - y||_inf   (scaled units)                              */
    float r_dual;              /* ||eta (x - x_prev) + rho (y - y_hat_prev)||_inf             */
    float r_compl;             /* max over contacts |y_k . z_k|                               */
    float r_ncp;               /* natural-map NCP residual of the returned (lambda, u+) on the
                                  contact blocks (Eq. 3), scaled units: with v~ = P (J u+ + v*)
                                  and lambda~ = P^-1 lambda, max over contacts k of
                                  || lambda~_k - Pi_K(lambda~_k - (v~_k + Gamma(v~_k))) ||_inf
                                  (0 without contacts)                                          */
} kamino_residual;

/* Buffers of a state, for zero-copy access (kamino_state_get). Element type is float for
 * KAMINO_FP32 models and double for KAMINO_FP64 models, except RESIDUAL (kamino_residual). */
typedef enum {
    KAMINO_BUF_BODY_Q = 0,     /* [B*7]  poses                                               */
    KAMINO_BUF_BODY_U = 1,     /* [B*6]  twists                                              */
    KAMINO_BUF_CACHE = 2,      /* [cache_len] impulses lambda* of the last step, physical units:
                                  world w's joint and drive rows, one per joint-limit bound, then
                                  3 per contact CANDIDATE (zero for limits and candidates that
                                  were not active)                                           */
    KAMINO_BUF_WARM = 3,       /* [cache_len] caller-supplied initial impulses (warm_mode 2)  */
    KAMINO_BUF_RESIDUAL = 4,   /* [W] kamino_residual                                         */
    KAMINO_BUF_TAU = 5         /* [W*n_act_max] actuation staging buffer: fill it (upload or
                                  zero-copy) and pass its device pointer to kamino_step        */
} kamino_buffer;

typedef struct kamino_model_s *kamino_model_t;
typedef struct kamino_state_s *kamino_state_t;

/* Validate a world description and copy it to the device.  Host-side checks (offsets monotone,
 * indices in range, parent != child, positive masses and inertias, unit-normalisable frame and
 * initial-pose quaternions, finite frames, contact points, gravity and initial state, supported
 * sizes, valid parameters) run first and return KAMINO_E_TOPOLOGY, KAMINO_E_INVALID_ARG or
 * KAMINO_E_UNSUPPORTED without touching the GPU. */
kamino_status kamino_model_create(const kamino_model_desc *desc, kamino_model_t *out);
kamino_status kamino_model_destroy(kamino_model_t model);
kamino_status kamino_model_get_info(kamino_model_t model, kamino_model_info *out);
/* Replace the solver parameters of a model (host-side only, takes effect at the next step). */
kamino_status kamino_model_set_params(kamino_model_t model, const kamino_solver_params *params);

/* Bytes of device memory a state of this model needs (256-byte aligned sub-buffers). */
kamino_status kamino_state_bytes(kamino_model_t model, size_t *bytes);
/* Create a state over `device_buffer` (>= kamino_state_bytes bytes, 256-byte aligned, owned by the
 * caller) or, when `device_buffer` is NULL, over memory the library allocates and later frees.
 * The state starts at the description's initial poses and twists with zero impulse caches
 * (synchronous: the state is ready when the call returns). */
kamino_status kamino_state_alloc(kamino_model_t model, void *device_buffer, size_t bytes,
                                 kamino_state_t *out);
kamino_status kamino_state_free(kamino_state_t state);
/* Device pointer and element count of one buffer of the state (zero-copy view). */
kamino_status kamino_state_get(kamino_state_t state, kamino_buffer which, void **dev_ptr,
                               int64_t *count);
/* Copy `count` elements (the state's element type, or kamino_residual) from / to host memory;
 * asynchronous on `stream` (pinned host memory makes it truly asynchronous). */
kamino_status kamino_state_upload(kamino_state_t state, kamino_buffer which, const void *host,
                                  int64_t count, void *stream);
kamino_status kamino_state_download(kamino_state_t state, kamino_buffer which, void *host,
                                    int64_t count, void *stream);

/* One time step of every world of the state (the whole hot path: one kernel launch, or one per
 * size bucket in the persistent plan).
 *   dt      time step in seconds, > 0
 *   iters   N_max of Alg. 1, >= 1
 *   tol     epsilon of the convergence test of Alg. 1 / Sec. 4.1, >= 0 (0 = run N_max)
 *   tau_dev device pointer to the actuation [W][n_act_max] (torques about revolute hinges, forces
 *           along prismatic axes, the state's element type) or NULL for none
 *   stream  cudaStream_t to launch on (NULL = legacy default stream)
 * Per-world failures (not converged within iters, non-finite result) are reported in the
 * RESIDUAL buffer; the return value covers argument and launch errors only. */
kamino_status kamino_step(kamino_state_t state, double dt, int32_t iters, double tol,
                          const void *tau_dev, void *stream);

/* Copy the per-world reports into `out_dev` (device memory, [W] kamino_residual) on `stream`. */
kamino_status kamino_residuals(kamino_state_t state, kamino_residual *out_dev, void *stream);

/* ---- Heterogeneous worlds (Sec. 5.2: worlds with different body and constraint counts in one
 * batch).  The model groups its worlds into size buckets by padded row count.  Two launch plans
 * (both keep the swept inverse of worlds of up to 256 padded rows in tensor memory when one
 * 256-thread CTA runs one world at a time and fills the SM's shared memory):
 *   KAMINO_LAUNCH_SINGLE      one CTA of 256 threads per world, shared memory sized for the
 *                             largest world (default; best for homogeneous batches)
 *   KAMINO_LAUNCH_PERSISTENT  one persistent launch per bucket (grid = SMs x resident CTAs); each
 *                             CTA is split into groups of 32/64/128/256 threads, one world per
 *                             group, each group pulling worlds from an atomic counter; buckets run
 *                             concurrently on forked streams.  Group size and panel width per
 *                             bucket come from kamino_autotune or from a size heuristic. */
enum { KAMINO_LAUNCH_SINGLE = 0, KAMINO_LAUNCH_PERSISTENT = 1 };

typedef struct {
    int32_t rows_pad;          /* padded row bound of the bucket (multiple of 32)             */
    int32_t num_worlds;        /* worlds in the bucket                                         */
    int32_t group_threads;     /* threads per world (32, 64, 128, 256)                         */
    int32_t panel;             /* sweep panel width (8 or 16)                                  */
    int32_t grid;              /* persistent CTAs launched for the bucket                      */
    int32_t worlds_per_cta;    /* concurrent worlds per CTA (= 256 / group_threads)           */
    float tuned_ms;            /* autotuner time of the chosen configuration (0 = heuristic)  */
    float reserved;
} kamino_bucket_info;

/* Current plan: up to `capacity` bucket records, their count and the launch mode. */
kamino_status kamino_plan_get(kamino_model_t model, kamino_bucket_info *out, int32_t capacity,
                              int32_t *count, int32_t *mode);
/* Select KAMINO_LAUNCH_SINGLE or KAMINO_LAUNCH_PERSISTENT for subsequent steps and graphs. */
kamino_status kamino_plan_set_mode(kamino_model_t model, int32_t mode);
/* Autotuner: for every bucket, time each feasible (group size, panel width) on the state's own
 * worlds and keep the fastest; then time one whole step with the tuned persistent plan and with
 * KAMINO_LAUNCH_SINGLE and switch the model to the faster.  The state is snapshotted and restored
 * around every trial, so it is left unchanged.  Synchronous. */
kamino_status kamino_autotune(kamino_state_t state, double dt, int32_t iters, double tol,
                              const void *tau_dev, void *stream);

/* ---- CUDA graph of one step (Sec. 5.2: the solver loop captured and replayed each step).  The
 * graph bakes in dt, iters, tol, the actuation pointer and the current plan; refill the actuation
 * buffer between launches.  Launch it on any stream; destroy before the state. */
typedef struct kamino_graph_s *kamino_graph_t;
kamino_status kamino_graph_create(kamino_state_t state, double dt, int32_t iters, double tol,
                                  const void *tau_dev, void *stream, kamino_graph_t *out);
kamino_status kamino_graph_launch(kamino_graph_t graph, void *stream);
kamino_status kamino_graph_destroy(kamino_graph_t graph);

/* ---- Learned warm start (one MLP per world type): features of a world (per body the position
 * relative to the first body, quaternion and twist; the first body's height; the actuation; per
 * contact candidate the signed distance and terrain normal; the state's impulse cache, i.e. the
 * previous step's solution) -> initial impulses in the impulse-cache layout.  L = 3 hidden layers
 * of width `hidden`, GELU, BF16 weights and activations, FP32 accumulation on tensor cores
 * (mma.sync m16n8k16), FP32 master weights and Adam.  Features and
 * targets are normalised per column (kamino_mlp_fit_normalization).  The network only supplies
 * the starting point of Alg. 1 (KAMINO_WARM_EXTERNAL); the solver's convergence test decides. */
typedef struct kamino_mlp_s *kamino_mlp_t;
typedef struct {
    int32_t num_worlds;        /* worlds the network serves                                   */
    int32_t d_in, d_hidden, hidden_layers, d_out;
    int32_t max_batch;         /* largest training / prediction batch                         */
    int64_t num_params;        /* [W0 (h x d_in), b0, W1, b1, ..., W_L (d_out x h), b_L]      */
} kamino_mlp_info;

/* `worlds` (host, `count` entries) lists worlds of one type: identical body, joint, candidate and
 * actuator counts (KAMINO_E_TOPOLOGY otherwise).  Weights: N(0, 2 / fan_in) from `seed`, bias 0. */
kamino_status kamino_mlp_create(kamino_model_t model, const int32_t *worlds, int32_t count, int32_t hidden,
                                int32_t max_batch, uint64_t seed, kamino_mlp_t *out);
kamino_status kamino_mlp_destroy(kamino_mlp_t mlp);
kamino_status kamino_mlp_get_info(kamino_mlp_t mlp, kamino_mlp_info *out);
/* Raw features [count][d_in] (FP32, device) of the state's worlds for actuation `tau_dev`. */
kamino_status kamino_mlp_features(kamino_mlp_t mlp, kamino_state_t state, const void *tau_dev, float *out_dev,
                                  void *stream);
/* Converged impulses of the last step (the state's cache) as raw targets [count][d_out]. */
kamino_status kamino_mlp_targets(kamino_mlp_t mlp, kamino_state_t state, float *out_dev, void *stream);
/* Column means and standard deviations of `rows` raw feature / target rows (device). */
kamino_status kamino_mlp_fit_normalization(kamino_mlp_t mlp, const float *x_dev, const float *y_dev, int64_t rows,
                                           void *stream);
/* One Adam step on the mean squared error of the normalised targets over the rows `rows_dev`
 * ([batch] indices into x_dev / y_dev; NULL = the first `batch` rows).  `loss_dev` (nullable)
 * receives the batch loss before the update. */
kamino_status kamino_mlp_train_step(kamino_mlp_t mlp, const float *x_dev, const float *y_dev,
                                    const int32_t *rows_dev, int32_t batch, float lr, float *loss_dev,
                                    void *stream);
/* Gradients of that loss with respect to every parameter (FP32 [num_params], device), no update. */
kamino_status kamino_mlp_gradients(kamino_mlp_t mlp, const float *x_dev, const float *y_dev,
                                   const int32_t *rows_dev, int32_t batch, float *grad_dev, float *loss_dev,
                                   void *stream);
/* Raw impulses [batch][d_out] predicted for raw features [batch][d_in]. */
kamino_status kamino_mlp_predict(kamino_mlp_t mlp, const float *x_dev, int32_t batch, float *y_dev, void *stream);
/* Features of the state -> prediction -> the state's KAMINO_BUF_WARM (use with warm_mode 2). */
kamino_status kamino_mlp_warm_start(kamino_mlp_t mlp, kamino_state_t state, const void *tau_dev, void *stream);
/* FP32 master parameters and the normalisation [x_mean(d_in), x_inv_std(d_in), y_mean(d_out),
 * y_inv_std(d_out)] to / from host memory (synchronous). */
kamino_status kamino_mlp_get_params(kamino_mlp_t mlp, float *host, int64_t count);
kamino_status kamino_mlp_set_params(kamino_mlp_t mlp, const float *host, int64_t count);
kamino_status kamino_mlp_get_normalization(kamino_mlp_t mlp, float *host);
kamino_status kamino_mlp_set_normalization(kamino_mlp_t mlp, const float *host);

/* ---- Forward kinematics for resets (Sec. 6.3: the Gauss-Newton solver that resets mechanisms with
 * kinematic loops to poses consistent with given joint coordinates).  For every world, from the poses
 * in KAMINO_BUF_BODY_Q, Gauss-Newton on F(q) = [f(q); d_j(q) - target_j over the selected joints]:
 * f are the errors of the joint rows (the rows the step uses, whose J is the rate of f) and d_j the
 * joint coordinate of the drives (hinge angle, slide; revolute differences wrapped into (-pi, pi]).
 * Each iteration takes the minimum-norm least-squares step over the twists of the bodies that are
 * not held, delta = -J^T P (P J J^T P + 1e-10 I)^-1 P F with P scaling the rows to unit norm
 * (factorised in FP64 on chip), and moves the poses along it (r += delta_v, q = exp(delta_w) q).
 * It stops when max|F| < tol or after max_iters iterations.
 *   joint_target_dev  [J] double, device: target coordinate of every joint (read where selected)
 *   joint_select_dev  [J] int32, device: nonzero = the joint's coordinate is prescribed (revolute and
 *                     prismatic joints; others are ignored).  NULL = the actuated joints
 *   body_fixed_dev    [B] int32, device: nonzero = the body keeps its pose.  NULL = none
 * Writes the poses (in the state's precision; twists are not changed) and, per world, into
 * KAMINO_BUF_RESIDUAL: iterations, status (KAMINO_WORLD_NOT_CONVERGED when max|F| >= tol, e.g. a
 * target the mechanism cannot reach), num_rows = rows of F, r_primal = max|F| (m, rad) at the
 * returned poses; the other fields 0.  Asynchronous on `stream`; the arrays must stay valid until
 * the work completes.  KAMINO_E_INVALID_ARG: NULL state or targets, max_iters < 1, tol < 0 or not
 * finite.  KAMINO_E_UNSUPPORTED: a world's FP64 system does not fit in one SM's shared memory
 * (about 216 rows of F). */
kamino_status kamino_fk(kamino_state_t state, const double *joint_target_dev, const int32_t *joint_select_dev,
                        const int32_t *body_fixed_dev, int32_t max_iters, double tol, void *stream);

/* ---- Allocation-free inference of the warm-start network (the paper has no counterpart).
 * kamino_mlp_predict with its activations in a file-scope device array of
 * KAMINO_MLP_STATIC_SCRATCH_BYTES instead of the network's own workspace: for callers that cannot
 * let memory be allocated for them (another framework owns the allocator, or a real-time loop
 * cannot afford the synchronisation of cudaMalloc).  Every GPU that loads the library holds the
 * array until exit.  The first call on a device looks up the array's device address (make it
 * before any stream capture); the address is kept for the life of the process, so do not call this
 * on a device after a cudaDeviceReset of it.  The calling thread's current device must be the one
 * the network was created on (KAMINO_E_INVALID_ARG otherwise).  All calls share the array: calls
 * that overlap on the GPU race, so serialise them.  A batch whose activations exceed the array
 * returns KAMINO_E_UNSUPPORTED, whose message names the largest batch that fits; this call
 * allocates nothing. */
#define KAMINO_MLP_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
kamino_status kamino_mlp_predict_static(kamino_mlp_t mlp, const float *x_dev, int32_t batch, float *y_dev,
                                        void *stream);

/* Message of the calling thread's last failed call ("" if none). */
const char *kamino_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KAMINO_H */
