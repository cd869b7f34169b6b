// C ABI of trajectory planning and calibration: cr_traj_cost, cr_traj_workspace_size, cr_solve_traj,
// cr_traj_prm_workspace_size, cr_solve_traj_prm, cr_calibrate and the pieces of the sharded calibration.
#include "cr_traj_impl.cuh"

namespace crk {
CR_TRAJ_INSTANTIATE(extern, float)
CR_TRAJ_INSTANTIATE(extern, double)
}

using namespace crh;

namespace {

cr_status check_traj_task(const cr_traj_task* t) {
  if (!t) return fail(CR_EINVAL, "traj task is NULL");
  if (t->P < 0) return fail(CR_EINVAL, "traj task: P < 0");
  if (t->T < 2 || t->T > 256) return fail(CR_EINVAL, "traj task: T = %d outside 2..256", t->T);
  if (!(t->w.dt > 0) || !(t->w.v_max > 0) || !(t->w.a_max > 0)) return fail(CR_EINVAL, "traj task: dt, v_max, a_max must be > 0");
  cr_status st;
  if ((st = check_ptr(t->u_start, 8, "u_start", t->P > 0)) || (st = check_ptr(t->goal, 8, "goal", t->P > 0))) return st;
  return CR_OK;
}

// Workspace of cr_solve_traj; with T > 0 (the PRM initialiser) also the initial states [3n][P*T] and
// the path length / hop count when the caller passes none.
struct TrajWs {
  size_t ik, ug, cost, pos, rot, succ, x0, len, hops, total;
};

TrajWs traj_ws(const cr_robot& r, int64_t P, const cr_ik_params& g, int T = 0) {
  TrajWs w;
  size_t off = 0;
  w.ik = off; off = align256(off + cr_ik_workspace_size(&r, P, &g));
  w.ug = off; off = align256(off + (size_t)3 * r.n * P * 8);
  w.cost = off; off = align256(off + (size_t)P * 8);
  w.pos = off; off = align256(off + (size_t)P * 8);
  w.rot = off; off = align256(off + (size_t)P * 8);
  w.succ = off; off = align256(off + (size_t)P);
  w.x0 = w.len = w.hops = off;
  if (T > 0) {
    w.x0 = off; off = align256(off + (size_t)3 * r.n * P * T * 8);
    w.len = off; off = align256(off + (size_t)P * 8);
    w.hops = off; off = align256(off + (size_t)P * 4);
  }
  w.total = off;
  return w;
}

// Trajectory planning: goal IK, then the linear initialiser (prm == nullptr) or the PRM query on the
// roadmaps, then the projected-gradient refinement.
cr_status solve_traj(const cr_robot* robot, const cr_scene* scene, const cr_traj_task* task,
                     const cr_ik_params* goal_ik, const cr_prm_params* prm, const cr_roadmap* map, int32_t k_traj,
                     double alpha0, double* X_out, double* cost_out, double* goal_pos, double* goal_rot, double* speed,
                     double* accel, uint8_t* lim_ok, uint8_t* col_ok, double* length, int32_t* hops, void* workspace,
                     size_t ws_bytes, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "trajectory entry points")) ||
      (st = check_scene(scene)) || (st = check_traj_task(task)))
    return st;
  if (!goal_ik) return fail(CR_EINVAL, "goal_ik is NULL");
  if (k_traj < 0 || !(alpha0 >= 0)) return fail(CR_EINVAL, "k_traj < 0 or alpha0 < 0");
  const int64_t P = task->P;
  if (P == 0) return CR_OK;
  if ((st = check_ptr(X_out, 8, "X_out", true)) || (st = check_ptr(cost_out, 8, "cost_out", true)) ||
      (st = check_ptr(goal_pos, 8, "goal_pos", true)) || (st = check_ptr(goal_rot, 8, "goal_rot", true)) ||
      (st = check_ptr(speed, 8, "speed", true)) || (st = check_ptr(accel, 8, "accel", true)) ||
      (st = check_ptr(lim_ok, 1, "lim_ok", true)) || (st = check_ptr(col_ok, 1, "col_ok", true)) ||
      (st = check_ptr(length, 8, "length", false)) || (st = check_ptr(hops, 4, "hops", false)) ||
      (st = check_ptr(workspace, 256, "workspace", true)))
    return st;
  TrajWs lay = traj_ws(*robot, P, *goal_ik, prm ? task->T : 0);
  if (ws_bytes < lay.total) return fail(CR_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, lay.total);
  unsigned char* ws = (unsigned char*)workspace;
  // 1. IK to the goal poses (per-problem spheres when the scene has them)
  cr_task it{};
  it.kind = CR_TASK_IK6;
  it.seeds_per_target = 1;
  it.targets = task->goal;
  it.n_targets = P;
  it.w = task->w;
  double* ug = (double*)(ws + lay.ug);
  if ((st = cr_solve_ik(robot, scene, &it, goal_ik, ug, (double*)(ws + lay.cost), (double*)(ws + lay.pos),
                        (double*)(ws + lay.rot), ws + lay.succ, ws + lay.ik, lay.ug - lay.ik, stream)))
    return st;
  // 2. initial states: the PRM query (Algorithm 2) or, without a roadmap, the linear interpolation
  double* x0 = nullptr;
  if (prm) {
    x0 = (double*)(ws + lay.x0);
    double* len = length ? length : (double*)(ws + lay.len);
    int32_t* hp = hops ? hops : (int32_t*)(ws + lay.hops);
    if ((st = cr_prm_query(robot, scene, &task->w, prm, map, task->u_start, ug, P, task->T, x0, len, hp, stream)))
      return st;
  }
  // 3. projected-gradient refinement
  crk::TrajLaunch l{};
  l.robot = *robot;
  if (scene) l.scene = *scene;
  l.task = *task;
  l.u_goal = ug;
  l.x_init = x0;
  l.k_traj = k_traj;
  l.alpha0 = alpha0;
  l.lim_tol = goal_ik->lim_tol;
  l.X_out = X_out;
  l.F_out = cost_out;
  l.goal_pos = goal_pos;
  l.goal_rot = goal_rot;
  l.speed = speed;
  l.accel = accel;
  l.lim_ok = lim_ok;
  l.col_ok = col_ok;
  l.stream = stream_of(stream);
  return goal_ik->precision == CR_F64 ? crk::launch_traj_solve<double>(l) : crk::launch_traj_solve<float>(l);
}

}  // namespace

extern "C" {

cr_status cr_traj_cost(const cr_robot* robot, const cr_scene* scene, const cr_traj_task* task, const void* x,
                       void* cost_out, void* grad_out, const void* upstream, int32_t dtype, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "trajectory entry points")) ||
      (st = check_scene(scene)) || (st = check_traj_task(task)) ||
      (st = check_dtype(dtype)))
    return st;
  if (task->P == 0) return CR_OK;
  size_t es = dsize(dtype);
  if ((st = check_ptr(x, es, "x", true)) || (st = check_ptr(cost_out, es, "cost_out", true)) ||
      (st = check_ptr(grad_out, es, "grad_out", false)) || (st = check_ptr(upstream, es, "upstream", false)))
    return st;
  crk::TrajLaunch l{};
  l.robot = *robot;
  if (scene) l.scene = *scene;
  l.task = *task;
  l.x = x;
  l.cost = cost_out;
  l.grad = grad_out;
  l.upstream = upstream;
  l.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_traj_cost<double>(l) : crk::launch_traj_cost<float>(l);
}

size_t cr_traj_workspace_size(const cr_robot* robot, int64_t P, const cr_ik_params* goal_ik) {
  if (!robot || !goal_ik || P < 0) return 0;
  return traj_ws(*robot, P, *goal_ik).total;
}

cr_status cr_solve_traj(const cr_robot* robot, const cr_scene* scene, const cr_traj_task* task,
                        const cr_ik_params* goal_ik, int32_t k_traj, double alpha0, double* X_out, double* cost_out,
                        double* goal_pos, double* goal_rot, double* speed, double* accel, uint8_t* lim_ok,
                        uint8_t* col_ok, void* workspace, size_t ws_bytes, cr_stream stream) {
  return solve_traj(robot, scene, task, goal_ik, nullptr, nullptr, k_traj, alpha0, X_out, cost_out, goal_pos, goal_rot,
                    speed, accel, lim_ok, col_ok, nullptr, nullptr, workspace, ws_bytes, stream);
}

size_t cr_traj_prm_workspace_size(const cr_robot* robot, int64_t P, int32_t T, const cr_ik_params* goal_ik) {
  if (!robot || !goal_ik || P < 0 || T < 2) return 0;
  return traj_ws(*robot, P, *goal_ik, T).total;
}

cr_status cr_solve_traj_prm(const cr_robot* robot, const cr_scene* scene, const cr_traj_task* task,
                            const cr_ik_params* goal_ik, const cr_prm_params* prm, const cr_roadmap* map,
                            int32_t k_traj, double alpha0, double* X_out, double* cost_out, double* goal_pos,
                            double* goal_rot, double* speed, double* accel, uint8_t* lim_ok, uint8_t* col_ok,
                            double* length, int32_t* hops, void* workspace, size_t ws_bytes, cr_stream stream) {
  if (!prm || !map) return fail(CR_EINVAL, "cr_solve_traj_prm: prm and map are required");
  if (task && check_self_rows(task->w, false, "cr_solve_traj_prm")) return CR_EINVAL;
  cr_status st = check_scene_spheres_only(scene, "cr_solve_traj_prm");
  if (st) return st;
  return solve_traj(robot, scene, task, goal_ik, prm, map, k_traj, alpha0, X_out, cost_out, goal_pos, goal_rot, speed,
                    accel, lim_ok, col_ok, length, hops, workspace, ws_bytes, stream);
}

size_t cr_calibrate_workspace_size(const cr_robot* robot, int64_t K) {
  if (!robot || robot->n < 1 || robot->n > CR_MAX_SEG || K < 1) return 0;
  return crk::calibrate_ws_bytes(robot->n, K);
}

cr_status cr_calibrate(const cr_robot* robot, const void* U, const double* P_meas, int64_t K, double* theta,
                       int32_t iters, double lambda0, double* F_out, double* hist, int32_t dtype, void* workspace,
                       size_t ws_bytes, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "cr_calibrate")) || (st = check_dtype(dtype)))
    return st;
  if (K < 1 || iters < 0 || !(lambda0 > 0)) return fail(CR_EINVAL, "cr_calibrate: K >= 1, iters >= 0, lambda0 > 0");
  if ((st = check_ptr(U, dsize(dtype), "U", true)) || (st = check_ptr(P_meas, 8, "P_meas", true)) ||
      (st = check_ptr(theta, 8, "theta", true)) || (st = check_ptr(F_out, 8, "F_out", true)) ||
      (st = check_ptr(hist, 8, "hist", false)) || (st = check_ptr(workspace, 8, "workspace", true)))
    return st;
  if (ws_bytes < crk::calibrate_ws_bytes(robot->n, K))
    return fail(CR_EINVAL, "cr_calibrate: workspace of %zu bytes, %zu needed", ws_bytes,
                crk::calibrate_ws_bytes(robot->n, K));
  crk::TrajLaunch l{};
  l.robot = *robot;
  l.U = U;
  l.Pm = P_meas;
  l.K = K;
  l.iters = iters;
  l.lambda0 = lambda0;
  l.theta_dev = theta;
  l.F_dev = F_out;
  l.hist_dev = hist;
  l.calib_ws = workspace;
  l.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_calibrate<double>(l) : crk::launch_calibrate<float>(l);
}

int32_t cr_calib_nv(int32_t n) {
  if (n < 1 || n > CR_MAX_SEG) return 0;
  return 2 * n * (2 * n + 1) / 2 + 2 * n + 1;
}

// Shared checks and launch of one piece of the sharded calibration.
static cr_status calib_piece(const char* who, int piece, const cr_robot* robot, const void* U, const double* P_meas,
                             int64_t K, double* theta, double* sums, double* state, double* theta_trial,
                             const double* F_trial, double* F_out, int32_t dtype, void* workspace, size_t ws_bytes,
                             cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, who)) || (st = check_dtype(dtype))) return st;
  const bool data = piece == 0 || piece == 2;
  if (data && K < 1) return fail(CR_EINVAL, "%s: K >= 1", who);
  if ((st = check_ptr(U, dsize(dtype), "U", data)) || (st = check_ptr(P_meas, 8, "P_meas", data)) ||
      (st = check_ptr(theta, 8, "theta", true)) || (st = check_ptr(sums, 8, "sums", piece != 2)) ||
      (st = check_ptr(state, 8, "state", piece == 1 || piece == 3)) ||
      (st = check_ptr(theta_trial, 8, "theta_trial", piece == 1 || piece == 3)) ||
      (st = check_ptr(F_trial, 8, "F_trial", piece == 3)) || (st = check_ptr(F_out, 8, "F_out", piece == 2)) ||
      (st = check_ptr(workspace, 8, "workspace", piece == 0)))
    return st;
  if (piece == 0 && ws_bytes < crk::calibrate_ws_bytes(robot->n, K))
    return fail(CR_EINVAL, "%s: workspace of %zu bytes, %zu needed", who, ws_bytes, crk::calibrate_ws_bytes(robot->n, K));
  crk::TrajLaunch l{};
  l.robot = *robot;
  l.U = U;
  l.Pm = P_meas;
  l.K = K;
  l.theta_dev = theta;
  l.F_dev = F_out;
  l.calib_ws = workspace;
  l.calib_piece = piece;
  l.sums = sums;
  l.state = state;
  l.theta_trial = theta_trial;
  l.F_trial = F_trial;
  l.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_calib_piece<double>(l) : crk::launch_calib_piece<float>(l);
}

cr_status cr_calib_sums(const cr_robot* robot, const void* U, const double* P_meas, int64_t K, const double* theta,
                        double* sums, int32_t dtype, void* workspace, size_t ws_bytes, cr_stream stream) {
  return calib_piece("cr_calib_sums", 0, robot, U, P_meas, K, const_cast<double*>(theta), sums, nullptr, nullptr,
                     nullptr, nullptr, dtype, workspace, ws_bytes, stream);
}

cr_status cr_calib_trial(const cr_robot* robot, const double* sums, const double* theta, double* state,
                         double* theta_trial, cr_stream stream) {
  return calib_piece("cr_calib_trial", 1, robot, nullptr, nullptr, 0, const_cast<double*>(theta),
                     const_cast<double*>(sums), state, theta_trial, nullptr, nullptr, CR_F64, nullptr, 0, stream);
}

cr_status cr_calib_cost(const cr_robot* robot, const void* U, const double* P_meas, int64_t K,
                        const double* theta_trial, double* F_out, int32_t dtype, cr_stream stream) {
  return calib_piece("cr_calib_cost", 2, robot, U, P_meas, K, const_cast<double*>(theta_trial), nullptr, nullptr,
                     nullptr, nullptr, F_out, dtype, nullptr, 0, stream);
}

cr_status cr_calib_accept(const cr_robot* robot, const double* sums, const double* F_trial, const double* theta_trial,
                          double* theta, double* state, cr_stream stream) {
  return calib_piece("cr_calib_accept", 3, robot, nullptr, nullptr, 0, theta, const_cast<double*>(sums), state,
                     const_cast<double*>(theta_trial), F_trial, nullptr, CR_F64, nullptr, 0, stream);
}

}  // extern "C"
