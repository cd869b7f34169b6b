/* C ABI of the GB300 CR-Solver hot path (libcrsolver.so).
 *
 * The library evaluates and optimises tendon-driven piecewise-constant-curvature (PCC) continuum
 * robots in large batches on one GPU (sm_103a). Every entry point below is `extern "C"`, takes
 * plain pointers and sizes, and returns a cr_status. No torch or CUDA C++ types appear here; the
 * stream argument is a cudaStream_t passed as an opaque pointer (NULL = the legacy default stream).
 *
 * Conventions shared by all entry points
 *  - Model (Sec. III): segment i (0-based, i < n) has arc length L_i, m = 3 tendons at radius r_c,i
 *    and angles alpha_j = 2 pi j / 3. Its state is the tendon displacement triple
 *    u_i = (u_i0, u_i1, u_i2), u_ij = l_ij - L_i (Eq. 4 read per segment). The bending of the
 *    segment follows from the exact inverse of Eq. 4: theta_i cos(phi_i) = -(2 / (3 r_c,i)) sum_j
 *    u_ij cos(alpha_j) and theta_i sin(phi_i) = -(2 / (3 r_c,i)) sum_j u_ij sin(alpha_j). The segment
 *    transform is Eq. 1-3, and the chain T_0^n = T_0^1 ... T_{n-1}^n is the tip pose.
 *  - States are structure-of-arrays: u[q][B], q = 3 i + j over d = 3 n components, batch fastest.
 *  - Pose outputs T[12][B]: the rotation R row-major (9 rows), then the position p (3 rows).
 *  - Device pointers: every array argument is a caller-owned DEVICE pointer unless it is marked
 *    "host". The library never allocates device memory. Where an entry point needs scratch space,
 *    the caller passes a `workspace` of at least the size its *_workspace_size function returns
 *    (256-byte aligned). Structs (cr_robot, cr_task, ...) are host pointers. Their contents are
 *    copied into kernel parameters at the call, so they may be freed when the call returns.
 *  - Asynchrony: work is enqueued on `stream` and the call returns at once. Outputs are valid
 *    after the stream is synchronised.
 *  - Errors: invalid arguments (null pointers where required, n outside 1..CR_MAX_SEG, m != 3,
 *    negative sizes, misaligned pointers, too-small workspace) return CR_EINVAL before anything
 *    is launched. A failed launch returns CR_ECUDA. cr_last_error_string() describes the last
 *    failure on the calling thread. Conditions found on the device never trap: they are written
 *    to per-problem flags and to the status word at the start of the workspace, read by
 *    cr_poll_status.
 */
#ifndef CR_H_
#define CR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CR_API __attribute__((visibility("default")))
#else
#define CR_API
#endif

typedef void* cr_stream; /* cudaStream_t */

typedef enum {
  CR_OK = 0,
  CR_EINVAL = 1,     /* invalid argument; nothing was launched */
  CR_ECUDA = 2,      /* a CUDA launch or runtime call failed */
  CR_ENONFINITE = 3, /* a non-finite input or iterate was met (device status bit) */
  CR_ETIMEOUT = 4,   /* a bounded device wait gave up (device status bit) */
} cr_status;

/* Arithmetic of the bulk evaluation. CR_F32: FP32 kinematics, Jacobian, cost and adjoint;
 * the LM Cholesky and the final acceptance stay FP64. CR_F64: everything FP64. */
typedef enum { CR_F32 = 0, CR_F64 = 1 } cr_dtype;

#define CR_MAX_SEG 6
#define CR_MAX_SPHERES 256 /* obstacles (spheres + primitives) per scene or problem */
#define CR_MAX_NB 64
#define CR_MAX_SEEDS 256

/* argmin of Algorithm 1 (the last step of cr_solve_ik and of every solver built on it): refined
 * candidates whose final FP64 cost is at most CR_ARGMIN_TIE (about 8 um of tip position, or the
 * rotation equivalent, under the default pose weights) are equally good solutions, whose cost
 * differences are rounding: the first of them in SelectTop order is kept. Above it, the lowest cost
 * wins (ties to the earlier candidate). */
#define CR_ARGMIN_TIE 1e-8

/* Decision variables of a segment (cr_robot.model). Three per segment in both models.
 * CR_MODEL_TENDON: the tendon displacements u_ij = l_ij - L_i of Eq. 4; the exact inverse of Eq. 4
 *   gives the bend (theta_i, phi_i), L_i is the robot's; bounds |u_ij| <= u_max_i, sum_j u_ij = 0.
 * CR_MODEL_ARC: the paper's own segment configuration q_i = (theta_i, phi_i, L_i) of Sec. IV-A in
 *   Cartesian form (theta cos phi, theta sin phi, L): the same configurations, smooth at theta = 0
 *   where phi is undefined. L_i is free within [l_min_i, l_max_i] (extendable segments; equal bounds
 *   pin it); bounds theta_i <= theta_max_i. Entry points that take the arc model: cr_fk,
 *   cr_fk_jac, cr_cost_grad, cr_seeds, cr_lm_step, cr_pg_steps, cr_solve_ik (and its two stages)
 *   for 1..4 segments; the others return CR_EINVAL for it. */
/* CR_MODEL_COUPLED: coupled tendon routing (Eq. l_eq read literally: tendon j of segment s runs through
 *   segments 1..s, its length the sum of the per-segment lengths of Eq. 4). The state holds the
 *   actuator displacements q_sj = sum_{i <= s} u_ij; the kinematics take the per-segment displacements
 *   u_s = q_s - q_{s-1}, and gradients and Jacobian columns leave through the transpose of that map
 *   (d/dq_s = d/du_s - d/du_{s+1}). Bounds |q_sj| <= u_max_s and sum_j q_sj = 0 act on the actuators
 *   (sum_j q_sj = 0 for every s exactly when every segment's displacements sum to zero), so seeds and
 *   the stage-one projection are those of the tendon model. Taken by cr_fk, cr_fk_jac, cr_cost_grad,
 *   cr_cost_vjp, cr_seeds, cr_lm_step, cr_pg_steps, cr_solve_ik (and its stages, and the static
 *   variant), 1..CR_MAX_SEG segments; the others return CR_EINVAL for it. */
typedef enum { CR_MODEL_TENDON = 0, CR_MODEL_ARC = 1, CR_MODEL_COUPLED = 2 } cr_model;
#define CR_MAX_SEG_ARC 4

/* Robot geometry (Sec. III, Fig. 2). Host struct. */
typedef struct {
  int32_t n;       /* segments, 1..CR_MAX_SEG */
  int32_t m;       /* tendons per segment; must be 3 */
  int32_t n_b;     /* backbone samples per segment for clearance (1..CR_MAX_NB); sample k of
                      segment i is the end of the sub-arc of fraction k / n_b, k = 1..n_b */
  int32_t model;   /* cr_model */
  double L[CR_MAX_SEG];         /* arc lengths (m); CR_MODEL_ARC: unused (the state holds them) */
  double r_c[CR_MAX_SEG];       /* tendon routing radii (m) */
  double u_max[CR_MAX_SEG];     /* bound |u_ij| <= u_max_i (m), Eq. ik_limits */
  double theta_max[CR_MAX_SEG]; /* bending-angle limit (rad), Eq. ik_limits */
  double r_body;                /* backbone radius added to every obstacle radius (m) */
  double l_min[CR_MAX_SEG];     /* CR_MODEL_ARC: length bounds l_min_i <= L_i <= l_max_i (m) */
  double l_max[CR_MAX_SEG];
} cr_robot;

/* Penalty and objective weights of Eq. penalized_form, as a least-squares sum 1/2 sum r^2. */
typedef struct {
  double w_p, w_R;                    /* pose rows: w_p (p - p_t) and w_R Log(R_t^T R) */
  double rho_b, rho_eq, rho_k, rho_c; /* squared-hinge / equality weights: bounds, sum-zero,
                                         curvature, clearance */
  double w_s, w_len, rho_v, rho_a;    /* path smoothness, trajectory length, tendon speed and
                                         acceleration hinges */
  double dt, v_max, a_max;            /* time step (s), tendon speed (m/s) and acceleration
                                         (m/s^2) limits */
  double delta;                       /* clearance margin of Eq. ik_coll (m) */
  double rho_s;                       /* self-contact rows of Eq. ik_coll over the robot itself:
                                         sqrt(rho_s) max(0, 2 r_body + delta - |p_a - p_b|) for
                                         backbone samples a, b of segments two or more apart;
                                         0 leaves them out. Taken by cr_cost_grad, cr_cost_vjp,
                                         cr_pg_steps, cr_lm_step, cr_solve_ik (and its stages),
                                         cr_traj_cost and cr_solve_traj, whose acceptance then
                                         also requires those samples 2 r_body apart; the path,
                                         batch, PRM and plain solvers return CR_EINVAL for
                                         rho_s > 0. */
} cr_weights;

/* Obstacle primitives beyond spheres: the convex pieces into which Sec. IV-C decomposes a
 * non-convex obstacle (a shelf or a cabinet of Sec. V-C is a set of boxes). A primitive is a record
 * of CR_PRIM_DOUBLES doubles: [0] kind, [1] radius r >= 0, then
 *   CR_PRIM_CAPSULE: [2..4] end point a, [5..7] end point b;
 *   CR_PRIM_BOX:     [2..4] centre c, [5..7] half extents h >= 0, [8..11] orientation quaternion
 *                    (w, x, y, z), box frame to world (normalised when read);
 * the rest unused. Its clearance rows are those of a sphere with the centre distance replaced by
 * the signed distance sd(x) from the backbone sample x to the primitive's core set (the segment
 * [a, b]; the solid box, sd < 0 inside it): sqrt(rho_c) max(0, r + r_body + delta - sd(x)). A box
 * with r > 0 has rounded edges. A record of any other kind is read as a sphere of radius r centred at
 * [2..4]. */
#define CR_PRIM_DOUBLES 16
#define CR_PRIM_SPHERE 0
#define CR_PRIM_CAPSULE 1
#define CR_PRIM_BOX 2

/* Obstacles: spheres and primitives for the clearance rows of Eq. ik_coll. Host struct; `spheres`
 * is a device array [n_o][4] = (centre x, y, z, radius), FP64, shared by all problems; with
 * per_problem = 1 it is [P][n_o][4] and problem p uses its own n_o spheres (trajectory and path
 * workloads place obstacles around each problem). `prims` is a device array [n_p][CR_PRIM_DOUBLES]
 * (FP64), [P][n_p][CR_PRIM_DOUBLES] with per_problem = 1. n_o + n_p <= CR_MAX_SPHERES. Primitives are
 * taken by cr_cost_grad, cr_cost_vjp, cr_pg_steps, cr_lm_step, cr_seeds, cr_solve_ik (and its stages
 * and cr_solve_ik_static), cr_solve_ik_plain, cr_traj_cost, cr_solve_traj and cr_solve_path; the
 * batch and PRM entry points return CR_EINVAL for n_p > 0. */
typedef struct {
  const double* spheres;
  int32_t n_o;         /* 0..CR_MAX_SPHERES */
  int32_t per_problem; /* 0: one obstacle set for all problems; 1: one set per problem */
  const double* prims; /* device [n_p][CR_PRIM_DOUBLES] (or per problem); NULL when n_p = 0 */
  int32_t n_p;         /* 0..CR_MAX_SPHERES - n_o */
} cr_scene;

typedef enum {
  CR_TASK_IK6 = 0, /* full pose: r = [w_p (p - p_t); w_R Log(R_t^T R)] (Eq. ik_opt, split) */
  CR_TASK_IK5 = 1, /* position + tip axis: r = [w_p (p - p_t); w_R (z - z_t)] */
} cr_task_kind;

/* An IK-type task over a batch of states. Host struct. State b aims at target b / S.
 * `targets` is a device array [7][n_targets] (FP64, component-major): p_x, p_y, p_z, then the
 * unit quaternion (w, x, y, z) for CR_TASK_IK6, or the tip axis (z_x, z_y, z_z, unused) for
 * CR_TASK_IK5. */
typedef struct {
  int32_t kind;
  int32_t seeds_per_target; /* S >= 1 */
  const double* targets;
  int64_t n_targets;
  cr_weights w;
} cr_task;

/* Settings of Algorithm 1 (beam-search IK). Host struct. */
typedef struct {
  int32_t S;        /* seeds per target, 1..CR_MAX_SEEDS (one CTA per target) */
  int32_t n_final;  /* candidates kept by SelectTop, 1..min(S, 32) */
  int32_t k_init;   /* stage-one projected-gradient steps (0 = single-stage: SelectTop only) */
  int32_t k_final;  /* stage-two LM iterations */
  double lambda0;   /* initial LM damping */
  double alpha0;    /* first stage-one step length (m of tendon displacement) */
  double dedup_eps; /* SelectTop skips candidates within this max-norm distance of a kept one */
  double lim_tol;   /* acceptance: |u| <= u_max + lim_tol and |sum_j u_ij| <= lim_tol */
  double pos_tol;   /* acceptance: position error (m) */
  double rot_tol;   /* acceptance: rotation error (rad) */
  uint64_t seed;    /* counter-based seed generator key */
  int64_t p0;       /* global index of the first target (seed counter offset) */
  int32_t precision;/* cr_dtype of the bulk evaluation */
  int32_t reserved;
} cr_ik_params;

/* ---------------------------------------------------------------------------------------------
 * Kinematics (Sec. III, Eq. 1-4)
 * ------------------------------------------------------------------------------------------- */

/* Forward kinematics of B states. u: [3n][B] in `dtype`; T_out: [12][B] in `dtype`;
 * backbone_out (nullable): [n * n_b][3][B] in `dtype`, the backbone samples (Fig. 2; the paper
 * samples 10 points per segment, Sec. V-B). */
CR_API cr_status cr_fk(const cr_robot* robot, const void* u, int64_t B, void* T_out, void* backbone_out,
                int32_t dtype, cr_stream stream);

/* Tip Jacobian of B states: J_out [6][3n][B] in `dtype`. Rows 0-2: d p / d u. Rows 3-5: the world
 * angular velocity w with dR = [w]x R per unit du. Needed by the LM step of Sec. IV-C. */
CR_API cr_status cr_fk_jac(const cr_robot* robot, const void* u, int64_t B, void* J_out, int32_t dtype,
                    cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Penalised cost and its adjoint (Sec. IV-A, Eq. ik_opt, ik_limits, ik_coll, penalized_form)
 * ------------------------------------------------------------------------------------------- */

/* Per-state cost F_b = 1/2 sum r^2 of an IK task, with rows
 *   pose (6), bounds sqrt(rho_b) max(0, +-u - u_max) (2 per tendon), sum-zero sqrt(rho_eq) sum_j u_ij
 *   (1 per segment), curvature sqrt(rho_k) max(0, theta_i - theta_max_i) (1 per segment) and
 *   clearance sqrt(rho_c) max(0, r_s + r_body + delta - |x_k - c_s|) per (sample, sphere) pair and
 *   sqrt(rho_c) max(0, r + r_body + delta - sd(x_k)) per (sample, primitive) pair.
 * cost_out [B] (required), coll_out [B] (nullable: the clearance part of F_b), grad_u_out [3n][B]
 * (nullable: dF_b / du), grad_param_out [2n][B] (nullable: dF_b / dL_i for i < n, then dF_b / dr_c,i),
 * all in `dtype`. The gradients come from a hand-written reverse sweep over the segments. */
CR_API cr_status cr_cost_grad(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                       const void* u, int64_t B, void* cost_out, void* coll_out, void* grad_u_out,
                       void* grad_param_out, int32_t dtype, cr_stream stream);

/* Deterministic row sums: out[r] = sum_b x[r][b] for r < rows (x [rows][B] in `dtype`, out FP64).
 * One block per row, fixed summation order (used to reduce per-state parameter gradients). */
CR_API cr_status cr_reduce_rows(const void* x, int64_t rows, int64_t B, double* out, int32_t dtype,
                         cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Solver steps (Sec. IV-C; Algorithm 1)
 * ------------------------------------------------------------------------------------------- */

/* `n_iter` Levenberg-Marquardt iterations on each of B states of an IK task, all in registers:
 * A = J^T J + lambda D (D = diag(max(diag(J^T J), 1e-12))), Cholesky in FP64, delta = -A^-1 J^T r,
 * accept iff F(u + delta) < F(u), then lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2; otherwise
 * lambda *= nu, nu *= 2. A non-positive pivot rejects the iteration the same way.
 * u_inout [3n][B] (`dtype`), lambda_inout / nu_inout [B] (FP64, caller-initialised),
 * F_out [B] (FP64, cost at the returned state, nullable), accepted_out [B] (nullable; the
 * number of accepted iterations). */
CR_API cr_status cr_lm_step(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                     void* u_inout, double* lambda_inout, double* nu_inout, double* F_out,
                     int32_t* accepted_out, int64_t B, int32_t n_iter, int32_t dtype,
                     cr_stream stream);

/* `steps` stage-one projected-gradient steps on each of B states: trial u' = Pi(u - alpha g/|g|),
 * accept iff F(u') < F(u) (then alpha *= 1.25) else alpha *= 0.5; Pi is the Euclidean projection
 * of each segment onto {|u_ij| <= u_max_i, sum_j u_ij = 0}. u_inout [3n][B], alpha_inout [B],
 * F_out [B], all in `dtype`. */
CR_API cr_status cr_pg_steps(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                      void* u_inout, void* alpha_inout, void* F_out, int64_t B, int32_t steps,
                      int32_t dtype, cr_stream stream);

/* SampleSeeds of Algorithm 1: S seeds for each of P problems (global index p0 + p), uniform on
 * each segment's feasible hexagon, from the counter-based SplitMix64 generator keyed by `seed`.
 * With obstacles, a seed whose backbone comes closer than r + r_body + delta to an obstacle's core
 * (a sphere's centre, a primitive's core set) is redrawn, at most 8 draws. u_out [3n][P * S] in `dtype` (seed s of problem p at p * S + s). */
CR_API cr_status cr_seeds(const cr_robot* robot, const cr_scene* scene, const cr_weights* w,
                   uint64_t seed, int64_t p0, int64_t P, int32_t S, void* u_out, int32_t dtype,
                   cr_stream stream);

/* SelectTop of Algorithm 1 for P problems of S candidates each: rank by (cost, coll, index)
 * ascending (non-finite costs last), skip candidates within `dedup_eps` (max-norm over u) of a
 * kept one, fill up with the best skipped ones. cost/coll [P * S] FP32, u [3n][P * S] in
 * `dtype`, idx_out [P][k] (int32, -1 where fewer than k candidates). k <= 32, S <= CR_MAX_SEEDS. */
CR_API cr_status cr_topk(const float* cost, const float* coll, const void* u, int32_t d, int64_t P,
                  int32_t S, int32_t k, double dedup_eps, int32_t* idx_out, int32_t dtype,
                  cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Solvers
 * ------------------------------------------------------------------------------------------- */

/* Scratch bytes cr_solve_ik needs for P targets. The workspace starts with the status word
 * (int32, read by cr_poll_status); at byte offset 8 a uint64 counts the projected-gradient steps
 * that stage one accepted, over all seeds (both are cleared by cr_solve_ik and cr_ik_stage1). It
 * also holds every seed's end state after stage one (P * S states), which SelectTop reads back:
 * about P * S * (3n + 2) * 4 bytes in FP32 (46 MB for 4096 targets of 256 seeds, 3 segments). */
CR_API size_t cr_ik_workspace_size(const cr_robot* robot, int64_t P, const cr_ik_params* prm);

/* Algorithm 1 (beam-search IK) for the P targets of `task` (task->seeds_per_target is ignored):
 * SampleSeeds(S) -> k_init projected-gradient steps per seed (registers) -> SelectTop(n_final)
 * (one warp per target, in a kernel of its own) -> k_final LM iterations per candidate -> FP64
 * re-evaluation and argmin.
 * Outputs (device, FP64 unless noted): u_out [3n][P], cost_out [P], pos_err [P] (m),
 * rot_err [P] (rad), success [P] (uint8: pos_err <= pos_tol, rot_err <= rot_tol, within limits,
 * collision-free). */
CR_API cr_status cr_solve_ik(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                      const cr_ik_params* prm, double* u_out, double* cost_out, double* pos_err,
                      double* rot_err, uint8_t* success, void* workspace, size_t ws_bytes,
                      cr_stream stream);

/* The two stages of cr_solve_ik as separate calls (same arguments, same workspace): stage 1 runs
 * SampleSeeds, the k_init projected-gradient steps and SelectTop and leaves the n_final candidates
 * of every target in the workspace; stage 2 refines them (k_final LM iterations), re-evaluates
 * them in FP64 and writes the argmin outputs. cr_solve_ik = stage 1 followed by stage 2 on one
 * stream; the status word is cleared by stage 1. */
CR_API cr_status cr_ik_stage1(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                              const cr_ik_params* prm, void* workspace, size_t ws_bytes, cr_stream stream);
CR_API cr_status cr_ik_stage2(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                              const cr_ik_params* prm, double* u_out, double* cost_out, double* pos_err,
                              double* rot_err, uint8_t* success, void* workspace, size_t ws_bytes,
                              cr_stream stream);

/* The straightforward comparator of cr_solve_ik: the same algorithm in FP64, one launch per
 * target, states kept in global memory as an array of structures. Same outputs; its workspace
 * is cr_ik_workspace_size with precision CR_F64. */
CR_API cr_status cr_solve_ik_plain(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                            const cr_ik_params* prm, double* u_out, double* cost_out,
                            double* pos_err, double* rot_err, uint8_t* success, void* workspace,
                            size_t ws_bytes, cr_stream stream);

/* Allocation-free variant of cr_solve_ik (the paper has no counterpart: it is a service to
 * callers that must not allocate device memory, such as a real-time control loop that reserves
 * everything at start-up or a host program that gives out device memory from its own pool).
 * Same arguments and outputs as cr_solve_ik, without the workspace: the scratch is a file-scope
 * device array of CR_STATIC_WS_BYTES bytes that every GPU loading the library holds until exit.
 * Sizes whose scratch (cr_ik_workspace_size) exceeds it return CR_EINVAL. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device current,
 * so make the first call before any stream capture. All calls share the array and overwrite it
 * (the status word at its start is cleared by each call; cr_poll_status cannot read it, the
 * per-target outputs carry the result): calls that overlap on the GPU race and must be serialised
 * by the caller. Allocates nothing. */
#define CR_STATIC_WS_BYTES ((size_t)8 << 20)
CR_API cr_status cr_solve_ik_static(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                                    const cr_ik_params* prm, double* u_out, double* cost_out, double* pos_err,
                                    double* rot_err, uint8_t* success, cr_stream stream);
/* Capacity of that array in bytes (CR_STATIC_WS_BYTES). */
CR_API size_t cr_static_workspace_capacity(void);

/* ---------------------------------------------------------------------------------------------
 * Trajectory planning (Sec. IV-A, Eq. mp_length_only and the tendon speed / acceleration limits
 * by finite differences; Alg. 2 refinement after the linear initialiser of Sec. V-C)
 * ------------------------------------------------------------------------------------------- */

/* P trajectories of T states u_0..u_{T-1}; u_0 = u_start is fixed. Host struct; device arrays:
 * u_start [3n][P] and goal [7][P] (full pose: position + quaternion w, x, y, z), FP64. The cost of
 * one trajectory is 1/2 sum r^2 over, for t = 1..T-1: path length rows sqrt(w_len)(p_t - p_{t-1}),
 * tendon speed hinges sqrt(rho_v) max(0, +-(u_t - u_{t-1})/dt - v_max), the state rows of u_t
 * (bounds, sum-zero, curvature, clearance); for t >= 2 the acceleration hinges sqrt(rho_a)
 * max(0, +-(u_t - 2 u_{t-1} + u_{t-2})/dt^2 - a_max); and the goal pose rows of u_{T-1}. */
typedef struct {
  const double* u_start;
  const double* goal;
  int64_t P;
  int32_t T; /* 2..256 */
  int32_t reserved;
  cr_weights w;
} cr_traj_task;

/* Trajectory cost per problem (cost_out [P]) of the free states x [3n][P * (T-1)] (state t >= 1 of
 * problem p at column p * (T-1) + t - 1), and optionally its gradient grad_out [3n][P * (T-1)] by
 * the hand-written adjoint; with upstream [P] (nullable) the gradient of problem p is scaled by
 * upstream[p] (a vector-Jacobian product). The adjoint recomputes the kinematics instead of storing
 * them. All arrays in `dtype`. */
CR_API cr_status cr_traj_cost(const cr_robot* robot, const cr_scene* scene, const cr_traj_task* task,
                              const void* x, void* cost_out, void* grad_out, const void* upstream, int32_t dtype,
                              cr_stream stream);

/* Scratch bytes of cr_solve_traj. */
CR_API size_t cr_traj_workspace_size(const cr_robot* robot, int64_t P, const cr_ik_params* goal_ik);

/* Trajectory planning: IK to every goal pose (Algorithm 1 with goal_ik), linear interpolation
 * u_t = u_start + t/(T-1) (u_goal - u_start), then k_traj projected-gradient steps of all free
 * states (step rule of stage one, norm over the whole trajectory). Outputs (device, FP64): X_out
 * [3n][P * T] (all states), cost_out [P], goal_pos / goal_rot [P] (m, rad), speed / accel [P]
 * (largest |du|/dt / v_max and |d2u|/dt^2 / a_max), lim_ok / col_ok [P] (uint8: every state within
 * limits / collision-free). goal_ik->precision selects the bulk precision of the whole solve. */
CR_API cr_status cr_solve_traj(const cr_robot* robot, const cr_scene* scene, const cr_traj_task* task,
                               const cr_ik_params* goal_ik, int32_t k_traj, double alpha0, double* X_out,
                               double* cost_out, double* goal_pos, double* goal_rot, double* speed, double* accel,
                               uint8_t* lim_ok, uint8_t* col_ok, void* workspace, size_t ws_bytes, cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * PRM exploration of Algorithm 2 (Sec. IV-B, "Trajectory Planning"): ParallelSample and
 * ParallelConnect build a roadmap per scene once; every query attaches its start and goal states
 * (ConnectToRoadmap), takes the shortest path (the distances of Dijkstra's algorithm, computed by
 * synchronous relaxation rounds) and resamples it at equal arc length (ResampleLinear) into the
 * initial states of the trajectory refinement.
 *
 * Readings of the paper (it gives no further detail): node i of roadmap r is the first of
 * `attempts` draws of the SampleSeeds generator (problem r, seed i, attempt a) whose backbone is
 * collision-free (invalid if none is); the edge {i, j} exists when either node is among the k
 * nearest valid nodes of the other (squared Euclidean distance in u, ties to the lower index) and
 * the segment, interpolated from the lower index to the higher, is collision-free at its n_check
 * interior states c / (n_check + 1), c = 1..n_check; its weight is the Euclidean distance. The
 * start (goal) is linked to those of its k nearest valid nodes whose segment from the state is
 * free at the same interior states; there is no direct start-goal edge. The path is read back
 * from the goal through the lowest-index neighbour u with d(u) < d(v) and d(u) + w(u, v) == d(v).
 * The resampled state t (t = 0..T-1) lies at arc length t / (T-1) of the path (state 0 the start,
 * T-1 the goal); with no path it is u_start + t/(T-1) (u_goal - u_start). Collision: any backbone
 * sample of the state closer than r + r_body + delta to a sphere centre, decided in FP64.
 * ------------------------------------------------------------------------------------------- */
#define CR_PRM_MAX_N 1024
#define CR_PRM_MAX_K 32
#define CR_PRM_MAX_CHECK 64
#define CR_PRM_MAX_ATTEMPTS 8

/* Roadmap settings. Host struct. */
typedef struct {
  int32_t N;        /* nodes per roadmap, 2..CR_PRM_MAX_N */
  int32_t k;        /* nearest neighbours, 1..min(CR_PRM_MAX_K, N - 1) */
  int32_t n_check;  /* interior states tested per edge, 1..CR_PRM_MAX_CHECK */
  int32_t attempts; /* draws per node, 1..CR_PRM_MAX_ATTEMPTS */
  uint64_t seed;    /* key of the node draws */
} cr_prm_params;

/* R roadmaps of N nodes (host struct of caller-owned device arrays). Roadmap r is built in the
 * scene's sphere set r (scene->per_problem = 1: R sets) or in the shared set.
 *   nodes   [3n][R * N]  FP64 node states (node i of roadmap r at column r * N + i; an invalid
 *                        node holds its last draw)
 *   node_ok [R * N]      uint8, 1 = valid
 *   nbr     [R * N][k]   int32 k nearest valid nodes (roadmap-local index), -1 past the last
 *   row     [R][N + 1]   int32 CSR offsets of each roadmap's graph (local to the roadmap's rows)
 *   col     [R][2 N k]   int32 neighbours, ascending within a row
 *   wt      [R][2 N k]   FP64 edge weights (Euclidean distance in u) */
typedef struct {
  int64_t R;
  double* nodes;
  uint8_t* node_ok;
  int32_t* nbr;
  int32_t* row;
  int32_t* col;
  double* wt;
} cr_roadmap;

/* Scratch bytes of cr_prm_build. */
CR_API size_t cr_prm_workspace_size(const cr_robot* robot, int64_t R, const cr_prm_params* prm);

/* Builds the roadmaps (the offline stage of Algorithm 2). Only w->delta of the weights is used.
 * Tendon model; map->R in 1..65535; scene->per_problem = 1 requires map->R sphere sets.
 * Asynchronous on `stream`. */
CR_API cr_status cr_prm_build(const cr_robot* robot, const cr_scene* scene, const cr_weights* w,
                              const cr_prm_params* prm, const cr_roadmap* map, void* workspace, size_t ws_bytes,
                              cr_stream stream);

/* Queries (the online stage up to ResampleLinear): P start / goal state pairs u_start, u_goal
 * [3n][P] (device, FP64); query p uses roadmap 0 when map->R == 1, else roadmap p (map->R == P),
 * and sphere set p of a per-problem scene. Outputs (device): X [3n][P * T] FP64 (state t of query
 * p at column p * T + t), length [P] FP64 (path length, +inf with no path), hops [P] int32 (path
 * edges, 0 with no path). T in 2..256. */
CR_API cr_status cr_prm_query(const cr_robot* robot, const cr_scene* scene, const cr_weights* w,
                              const cr_prm_params* prm, const cr_roadmap* map, const double* u_start,
                              const double* u_goal, int64_t P, int32_t T, double* X, double* length, int32_t* hops,
                              cr_stream stream);

/* Scratch bytes of cr_solve_traj_prm. */
CR_API size_t cr_traj_prm_workspace_size(const cr_robot* robot, int64_t P, int32_t T, const cr_ik_params* goal_ik);

/* Trajectory planning with the PRM initialiser (Algorithm 2): IK to every goal pose as in
 * cr_solve_traj, cr_prm_query from u_start to the IK state on the prebuilt roadmaps, then the
 * k_traj projected-gradient steps of cr_solve_traj from the resampled states. Outputs as
 * cr_solve_traj, plus length [P] and hops [P] of the roadmap path (device, nullable). */
CR_API cr_status cr_solve_traj_prm(const cr_robot* robot, const cr_scene* scene, const cr_traj_task* task,
                                   const cr_ik_params* goal_ik, const cr_prm_params* prm, const cr_roadmap* map,
                                   int32_t k_traj, double alpha0, double* X_out, double* cost_out, double* goal_pos,
                                   double* goal_rot, double* speed, double* accel, uint8_t* lim_ok, uint8_t* col_ok,
                                   double* length, int32_t* hops, void* workspace, size_t ws_bytes,
                                   cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Path following (Sec. IV-A, Eq. constrained_mp; Sec. IV-B, "Path Following")
 * ------------------------------------------------------------------------------------------- */

/* P reference paths of H full-pose waypoints. Host struct; waypoints is a device array [7][P * H]
 * (FP64; waypoint t of path p at column p * H + t: position, then quaternion w, x, y, z). */
typedef struct {
  const double* waypoints;
  int64_t P;
  int32_t H; /* 2..128 */
  int32_t reserved;
  cr_weights w;
} cr_path_task;

/* Scratch bytes of cr_solve_path. */
CR_API size_t cr_path_workspace_size(const cr_robot* robot, int64_t P, int32_t H, const cr_ik_params* first_ik);

/* Path following:
 *  1. exploration: IK at waypoint 0 (Algorithm 1 with first_ik), then for t = 1..H-1 k_warm LM
 *     iterations of waypoint t's IK residual starting from the solution at t-1 (bulk precision);
 *  2. refinement: k_joint LM iterations over all waypoints jointly, residual = every waypoint's IK
 *     rows plus the smoothness rows sqrt(w_s)(u_t - u_{t-1}); the normal matrix is block tridiagonal
 *     and is factorised by a block Cholesky in FP64 (lambda0 and the LM rule of cr_lm_step).
 * Outputs (device, FP64): X_out [3n][P * H], cost_out [P] (joint cost), pos_err / rot_err [P * H],
 * lim_ok / col_ok [P] (uint8: every waypoint within limits / collision-free). first_ik->precision
 * selects the bulk precision of the whole solve. */
CR_API cr_status cr_solve_path(const cr_robot* robot, const cr_scene* scene, const cr_path_task* task,
                               const cr_ik_params* first_ik, int32_t k_warm, int32_t k_joint, double* X_out,
                               double* cost_out, double* pos_err, double* rot_err, uint8_t* lim_ok, uint8_t* col_ok,
                               void* workspace, size_t ws_bytes, cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Kinematic calibration and vector-Jacobian products (differentiation w.r.t. the robot)
 * ------------------------------------------------------------------------------------------- */

/* Bytes of device workspace cr_calibrate needs for K poses (0 on invalid arguments). */
CR_API size_t cr_calibrate_workspace_size(const cr_robot* robot, int64_t K);

/* LM calibration of theta = (L_1..n, r_c,1..n) from K known displacements U [3n][K] (`dtype`) and
 * measured tip positions P_meas [3][K] (FP64): residual p(u_k; theta) - p_k. theta (device, FP64,
 * [2n]) holds the initial guess and receives the estimate; F_out (device, [1]) the final cost;
 * hist (device, nullable, [iters][2n]) the iterates. Same LM rule as cr_lm_step; J^T J and J^T r
 * reduced in FP64 in a fixed order (per block of 128 poses, then over the blocks in order),
 * Cholesky in FP64. Per iteration one many-block launch forms the partial sums and one single-block
 * launch solves, evaluates the trial cost and applies the rule. `workspace` (device, 8-byte
 * aligned, at least cr_calibrate_workspace_size bytes, caller-owned) holds the damping state and
 * the partial sums; it is overwritten. */
CR_API cr_status cr_calibrate(const cr_robot* robot, const void* U, const double* P_meas, int64_t K, double* theta,
                              int32_t iters, double lambda0, double* F_out, double* hist, int32_t dtype,
                              void* workspace, size_t ws_bytes, cr_stream stream);

/* Sharded calibration: the pieces of one cr_calibrate iteration, for processes (one GPU each) that
 * each hold a share of the K poses. Per iteration every process runs
 *   cr_calib_sums (its share) -> all-reduce (sum) of `sums` -> cr_calib_trial ->
 *   cr_calib_cost (its share, at theta_trial) -> all-reduce (sum) of F_trial -> cr_calib_accept,
 * and so keeps the same theta and damping state as the others. One process with all the poses
 * reproduces cr_calibrate exactly (same partial sums in the same order, same factorisation, same
 * rule). Arrays are device FP64: theta, theta_trial [2n]; sums [cr_calib_nv(n)] = packed J^T J (lower
 * triangle by rows), J^T r, F = 1/2 |r|^2; state [4] = lambda, nu, ok, pred, initialised by the
 * caller to (lambda0, 2, 0, 0). cr_calib_sums needs cr_calibrate_workspace_size(robot, K) bytes of
 * workspace; U and P_meas as in cr_calibrate. cr_calib_nv returns 0 for n out of range. */
CR_API int32_t cr_calib_nv(int32_t n);
CR_API cr_status cr_calib_sums(const cr_robot* robot, const void* U, const double* P_meas, int64_t K,
                               const double* theta, double* sums, int32_t dtype, void* workspace, size_t ws_bytes,
                               cr_stream stream);
CR_API cr_status cr_calib_trial(const cr_robot* robot, const double* sums, const double* theta, double* state,
                                double* theta_trial, cr_stream stream);
CR_API cr_status cr_calib_cost(const cr_robot* robot, const void* U, const double* P_meas, int64_t K,
                               const double* theta_trial, double* F_trial, int32_t dtype, cr_stream stream);
CR_API cr_status cr_calib_accept(const cr_robot* robot, const double* sums, const double* F_trial,
                                 const double* theta_trial, double* theta, double* state, cr_stream stream);

/* Vector-Jacobian product of the IK cost: grad_u_out[:, b] = upstream[b] dF_b/du_b and
 * grad_param_out [2n] (FP64) = sum_b upstream[b] dF_b/d(L, r_c). workspace: [2n][B] in `dtype`.
 * upstream [B], grad_u_out [3n][B] in `dtype`. The adjoint recomputes the forward sweep. */
CR_API cr_status cr_cost_vjp(const cr_robot* robot, const cr_scene* scene, const cr_task* task, const void* u,
                             int64_t B, const void* upstream, void* grad_u_out, double* grad_param_out, void* workspace,
                             int32_t dtype, cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Status and diagnostics
 * ------------------------------------------------------------------------------------------- */

/* Copies the device status word at the start of `workspace` to *host_status (a bit set of
 * 1 << CR_ENONFINITE and 1 << CR_ETIMEOUT) after synchronising `stream`. */
CR_API cr_status cr_poll_status(const void* workspace, int32_t* host_status, cr_stream stream);

/* Description of the last error on the calling thread (static storage; never NULL). */
CR_API const char* cr_last_error_string(void);

/* Peak-calibration kernels (FP32 FMA chains, special-function chains, FP64 FMA chains and a
 * streaming copy), timed by the caller with events around the launch. kind: 0 FFMA, 1 MUFU
 * (sin/cos approximations), 2 DFMA, 3 copy, 4 DFMA with one active lane per warp (how the FP64
 * pipe charges partly active warps), 5 paired FFMA (two FP32 FMAs per lane per instruction).
 * `buf` is a device buffer of `bytes` bytes (copy reads the first half and writes the second).
 * *ops_out (host) receives the operations one launch performs (flops for 0, 2, 4 and 5,
 * special-function results for 1, bytes moved for 3). */
CR_API cr_status cr_peak_launch(int32_t kind, void* buf, size_t bytes, int32_t iters, double* ops_out,
                         cr_stream stream);

/* ---------------------------------------------------------------------------------------------
 * Ragged batch (serving-shaped): IK and path-following problems of mixed segment count, waypoint
 * count, seed count and obstacle count in one CUDA-graph launch of persistent kernels over a work
 * queue. The paper runs each problem on its own (Algorithm 1, Sec. IV); the batching is the GPU
 * form of running many of them at once.
 *
 * Item i (caller's order) uses the first n_i segments of `family`, waypoints
 * targets[:, w_i .. w_i + H_i - 1] (w_i = sum_{j<i} H_j, targets a device [7][W] FP64 array as in
 * cr_path_task, W = sum H) and spheres[o_i .. o_i + n_o_i - 1] (o_i = sum_{j<i} n_o_j, a device
 * [*][4] FP64 array). An IK item (H = 1) is Algorithm 1 on its target with S_i seeds; a path item is
 * the path pipeline of cr_solve_path (first-waypoint IK with S_i seeds, exploration sweep of k_warm
 * LM iterations per waypoint, k_joint joint LM iterations). Outputs (device): u_out item-packed,
 * item i's block [3 n_i][H_i] (component-major) starting at sum_{j<i} 3 n_j H_j; cost_out [N];
 * pos_err, rot_err [W] (FP64 acceptance per waypoint); flags_out [N]: bit 0 success (every waypoint
 * within pos_tol / rot_tol, limits and clearance), bit 1 limits met, bit 2 collision-free;
 * t_done_ns [N]: completion time of the item after the batch start (%globaltimer, ns).
 * ------------------------------------------------------------------------------------------- */
#define CR_ITEM_IK 0
#define CR_ITEM_PATH 1
#define CR_BATCH_MAX_SPHERES 64
#define CR_BATCH_MAX_H 128

typedef struct {
  int32_t kind; /* CR_ITEM_IK (H must be 1) or CR_ITEM_PATH */
  int32_t n;    /* segments, 1..CR_MAX_SEG */
  int32_t H;    /* waypoints, 1..CR_BATCH_MAX_H */
  int32_t S;    /* seeds of the (first-waypoint) IK, 1..CR_MAX_SEEDS */
  int32_t n_o;  /* spheres, 0..CR_BATCH_MAX_SPHERES */
  int32_t reserved;
} cr_batch_item;

typedef struct {
  cr_ik_params ik;        /* n_final, k_init, k_final, lambda0, alpha0, dedup_eps, lim_tol, pos_tol,
                             rot_tol, seed, p0 (item i draws seeds as problem p0 + i); S and
                             precision are ignored (per item; FP32 bulk, FP64 solves) */
  int32_t k_warm, k_joint;
  int32_t seeds_per_unit; /* seeds one warp takes per work unit: 32, 64, 128 or 256; 0: chosen by
                             timing the candidates in cr_batch_plan_create */
  int32_t seed_regs;      /* register budget of the seeds phase: 1 wide (168 registers per thread
                             for n <= 4, 255 above), 2 tight (128, 168: more resident warps, with
                             spills where a state does not fit); 0: chosen by timing together with
                             seeds_per_unit in cr_batch_plan_create (wide in cr_solve_batch) */
} cr_batch_params;

typedef struct cr_batch_plan cr_batch_plan;

/* Workspace bytes for the batch (also covers every seeds_per_unit and seed_regs candidate); 0 on bad
 * input. */
CR_API size_t cr_batch_workspace_size(const cr_robot* family, const cr_batch_item* items, int64_t N,
                                      const cr_batch_params* prm);

/* Validates the batch, builds the work queue (longest estimated item first) in `workspace`
 * (caller-owned device memory, >= cr_batch_workspace_size bytes, 256-byte aligned), captures the
 * CUDA graph (start node; per segment count present one branch of four persistent phase kernels in
 * order: seeds and projected gradient, SelectTop + refinement + argmin, exploration sweep, joint LM;
 * the branches in parallel)
 * and returns the plan (host object). With seeds_per_unit = 0 or seed_regs = 0 every open
 * combination of the two is run and timed on `stream` (the outputs then hold a valid result). Synchronises `stream`. All pointers stay bound
 * to the plan: cr_batch_plan_run re-solves the batch from the current contents of targets and
 * spheres. CR_EINVAL for a bad item (kind, n, H, S, n_o out of range, IK with H != 1), NULL or
 * misaligned pointers, or a short workspace; CR_EINVAL for seed_regs outside 0..2. */
CR_API cr_status cr_batch_plan_create(const cr_robot* family, const cr_weights* w, const cr_batch_item* items,
                                      int64_t N, const cr_batch_params* prm, const double* targets,
                                      const double* spheres, double* u_out, double* cost_out, double* pos_err,
                                      double* rot_err, uint8_t* flags_out, uint64_t* t_done_ns, void* workspace,
                                      size_t ws_bytes, cr_stream stream, cr_batch_plan** plan);
/* One graph launch on `stream` (asynchronous). Two runs of one plan must not overlap. */
CR_API cr_status cr_batch_plan_run(cr_batch_plan* plan, cr_stream stream);
/* The plan's seeds per unit, number of work units, resident worker warps of the seeds phase and
 * register budget of that phase (1 wide, 2 tight) (host pointers, each may be NULL). */
CR_API cr_status cr_batch_plan_info(const cr_batch_plan* plan, int32_t* seeds_per_unit, int64_t* units,
                                    int64_t* workers, int32_t* seed_regs);
/* Frees the plan (graph, streams, events); the caller makes sure no run is in flight. */
CR_API cr_status cr_batch_plan_destroy(cr_batch_plan* plan);
/* Plan, run, synchronise and free in one call (seeds_per_unit 0 takes 64, without timing). */
CR_API cr_status cr_solve_batch(const cr_robot* family, const cr_weights* w, const cr_batch_item* items, int64_t N,
                                const cr_batch_params* prm, const double* targets, const double* spheres,
                                double* u_out, double* cost_out, double* pos_err, double* rot_err,
                                uint8_t* flags_out, uint64_t* t_done_ns, void* workspace, size_t ws_bytes,
                                cr_stream stream);

/* Contiguous partition of a ragged batch over `parts` processes (one GPU each) by estimated cost:
 * the planner's relative time of each item (the one cr_batch_plan_create orders its queue by). On
 * return bounds[0] = 0 <= bounds[1] <= ... <= bounds[parts] = N and process r takes the items
 * [bounds[r], bounds[r + 1]), in the caller's order; bounds[r] is the first item whose prefix
 * cost (through that item) exceeds r / parts of the total, so a part exceeds the mean by at most
 * one item's cost. The items are independent (no data crosses processes); with
 * prm->ik.p0 + bounds[r] as a process's p0 its seeds equal those of the unpartitioned batch.
 * Host only (no GPU work); bounds: host array of parts + 1 values. CR_EINVAL for N < 0, parts < 1,
 * NULL pointers or a bad item. */
CR_API cr_status cr_batch_partition(const cr_batch_item* items, int64_t N, const cr_batch_params* prm, int32_t parts,
                                    int64_t* bounds);

/* The plain form of the same batch, for comparison: one cr_solve_ik / cr_solve_path call per item
 * (P = 1) in the caller's order on `stream`, each followed by a completion stamp. Same outputs,
 * except that flags_out bits 1 and 2 are set for path items only. Workspace: */
CR_API size_t cr_batch_plain_workspace_size(const cr_robot* family, const cr_batch_item* items, int64_t N,
                                            const cr_batch_params* prm);
CR_API cr_status cr_solve_batch_plain(const cr_robot* family, const cr_weights* w, const cr_batch_item* items,
                                      int64_t N, const cr_batch_params* prm, const double* targets,
                                      const double* spheres, double* u_out, double* cost_out, double* pos_err,
                                      double* rot_err, uint8_t* flags_out, uint64_t* t_done_ns, void* workspace,
                                      size_t ws_bytes, cr_stream stream);

/* Elementwise run of a device helper the solvers rely on, for checking it against CUDA's own
 * operations (the paper has no counterpart; this is numerics verification). which:
 * CR_CHECK_RECIP: out[i] = FP64 reciprocal of in[i] as the block solves of cr_solve_path compute it
 * (Newton-Raphson from the single-precision approximation; within a few ulp of 1/in[i]).
 * CR_CHECK_SIN, CR_CHECK_COS: out[i] = sin(in[i]), cos(in[i]) as the FP64 kinematics compute them.
 * in, out: device arrays of n doubles (8-byte aligned). Asynchronous on `stream`; CR_EINVAL for a
 * NULL or misaligned pointer, n < 0 or an unknown helper. */
#define CR_CHECK_RECIP 0
#define CR_CHECK_SIN 1
#define CR_CHECK_COS 2
CR_API cr_status cr_device_check(int32_t which, const double* in, double* out, int64_t n, cr_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* CR_H_ */
