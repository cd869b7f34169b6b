// C ABI of the solver entry points: cr_solve_ik, cr_lm_step, cr_pg_steps, cr_seeds, cr_topk.
#include "cr_solve_impl.cuh"

namespace crk {
CR_SOLVE_INSTANTIATE(extern, float)
CR_SOLVE_INSTANTIATE(extern, double)
}

using namespace crh;

namespace {

cr_status check_ik_params(const cr_ik_params* p) {
  if (!p) return fail(CR_EINVAL, "ik params is NULL");
  if (p->S < 1 || p->S > CR_MAX_SEEDS) return fail(CR_EINVAL, "S = %d outside 1..%d", p->S, CR_MAX_SEEDS);
  if (p->n_final < 1 || p->n_final > 32 || p->n_final > p->S)
    return fail(CR_EINVAL, "n_final = %d outside 1..min(S, 32)", p->n_final);
  if (p->k_init < 0 || p->k_final < 0) return fail(CR_EINVAL, "negative iteration count");
  if (!(p->lambda0 > 0) || !(p->alpha0 >= 0) || !(p->dedup_eps >= 0))
    return fail(CR_EINVAL, "lambda0 must be > 0, alpha0 and dedup_eps >= 0");
  return check_dtype(p->precision);
}

}  // namespace

extern "C" {

static cr_status solve_ik_common(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                                 const cr_ik_params* prm, double* u_out, double* cost_out, double* pos_err,
                                 double* rot_err, uint8_t* success, void* workspace, size_t ws_bytes,
                                 cr_stream stream, int which) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_scene(scene)) || (st = check_ik_params(prm))) return st;
  if (!task) return fail(CR_EINVAL, "task is NULL");
  cr_task t = *task;
  t.seeds_per_target = 1;
  if ((st = check_task(&t, t.n_targets))) return st;
  const int64_t P = t.n_targets;
  if (P == 0) return CR_OK;
  if (P > 2147483647LL) return fail(CR_EINVAL, "too many targets");
  if (which & 2) {
    if ((st = check_ptr(u_out, 8, "u_out", true)) || (st = check_ptr(cost_out, 8, "cost_out", true)) ||
        (st = check_ptr(pos_err, 8, "pos_err", true)) || (st = check_ptr(rot_err, 8, "rot_err", true)) ||
        (st = check_ptr(success, 1, "success", true)))
      return st;
  }
  if ((st = check_ptr(workspace, 256, "workspace", true))) return st;
  IkLayout lay = ik_layout(*robot, P, *prm);
  if (ws_bytes < lay.total)
    return fail(CR_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, lay.total);
  crk::SolveArgs a{};
  a.robot = *robot;
  if (scene) a.scene = *scene;
  a.task = t;
  a.prm = *prm;
  a.ws = workspace;
  a.lay = lay;
  a.u_out = u_out;
  a.cost_out = cost_out;
  a.pos = pos_err;
  a.rot = rot_err;
  a.success = success;
  a.stream = stream_of(stream);
  if (which & 1) {
    // the status word and, at offset 8, the count of accepted stage-one steps
    cudaError_t e = cudaMemsetAsync((unsigned char*)workspace + lay.status, 0, 16, a.stream);
    if (e != cudaSuccess) return fail(CR_ECUDA, "cr_solve_ik: %s", cudaGetErrorString(e));
  }
  return prm->precision == CR_F64 ? crk::launch_solve_ik<double>(a, which) : crk::launch_solve_ik<float>(a, which);
}

cr_status cr_solve_ik(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                      const cr_ik_params* prm, double* u_out, double* cost_out, double* pos_err,
                      double* rot_err, uint8_t* success, void* workspace, size_t ws_bytes,
                      cr_stream stream) {
  return solve_ik_common(robot, scene, task, prm, u_out, cost_out, pos_err, rot_err, success, workspace,
                         ws_bytes, stream, 3);
}

cr_status cr_ik_stage1(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                       const cr_ik_params* prm, void* workspace, size_t ws_bytes, cr_stream stream) {
  return solve_ik_common(robot, scene, task, prm, nullptr, nullptr, nullptr, nullptr, nullptr, workspace,
                         ws_bytes, stream, 1);
}

cr_status cr_ik_stage2(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                       const cr_ik_params* prm, double* u_out, double* cost_out, double* pos_err,
                       double* rot_err, uint8_t* success, void* workspace, size_t ws_bytes,
                       cr_stream stream) {
  return solve_ik_common(robot, scene, task, prm, u_out, cost_out, pos_err, rot_err, success, workspace,
                         ws_bytes, stream, 2);
}

cr_status cr_lm_step(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                     void* u_inout, double* lambda_inout, double* nu_inout, double* F_out,
                     int32_t* accepted_out, int64_t B, int32_t n_iter, int32_t dtype,
                     cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_scene_shared(scene)) || (st = check_task(task, B)) ||
      (st = check_dtype(dtype)))
    return st;
  if (B < 0 || n_iter < 0) return fail(CR_EINVAL, "cr_lm_step: negative size");
  if (B == 0) return CR_OK;
  if ((st = check_ptr(u_inout, dsize(dtype), "u_inout", true)) ||
      (st = check_ptr(lambda_inout, 8, "lambda_inout", true)) ||
      (st = check_ptr(nu_inout, 8, "nu_inout", true)) || (st = check_ptr(F_out, 8, "F_out", false)) ||
      (st = check_ptr(accepted_out, 4, "accepted_out", false)))
    return st;
  crk::SolveArgs a{};
  a.robot = *robot;
  if (scene) a.scene = *scene;
  a.task = *task;
  a.u = u_inout;
  a.B = B;
  a.iters = n_iter;
  a.lam = lambda_inout;
  a.nu = nu_inout;
  a.F64 = F_out;
  a.acc = accepted_out;
  a.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_lm_steps<double>(a) : crk::launch_lm_steps<float>(a);
}

cr_status cr_pg_steps(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                      void* u_inout, void* alpha_inout, void* F_out, int64_t B, int32_t steps,
                      int32_t dtype, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_scene_shared(scene)) || (st = check_task(task, B)) ||
      (st = check_dtype(dtype)))
    return st;
  if (B < 0 || steps < 0) return fail(CR_EINVAL, "cr_pg_steps: negative size");
  if (B == 0) return CR_OK;
  size_t es = dsize(dtype);
  if ((st = check_ptr(u_inout, es, "u_inout", true)) || (st = check_ptr(alpha_inout, es, "alpha_inout", true)) ||
      (st = check_ptr(F_out, es, "F_out", true)))
    return st;
  crk::SolveArgs a{};
  a.robot = *robot;
  if (scene) a.scene = *scene;
  a.task = *task;
  a.u = u_inout;
  a.B = B;
  a.iters = steps;
  a.alpha = alpha_inout;
  a.F = F_out;
  a.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_pg_steps<double>(a) : crk::launch_pg_steps<float>(a);
}

cr_status cr_seeds(const cr_robot* robot, const cr_scene* scene, const cr_weights* w, uint64_t seed,
                   int64_t p0, int64_t P, int32_t S, void* u_out, int32_t dtype, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_scene(scene)) || (st = check_dtype(dtype))) return st;
  if (P < 0 || S < 1 || S > 65536 || p0 < 0) return fail(CR_EINVAL, "cr_seeds: bad P / S / p0");
  if (scene && scene->n_o > 0 && !w) return fail(CR_EINVAL, "cr_seeds: weights (delta) needed with spheres");
  if (P == 0) return CR_OK;
  if ((st = check_ptr(u_out, dsize(dtype), "u_out", true))) return st;
  crk::SolveArgs a{};
  a.robot = *robot;
  if (scene) a.scene = *scene;
  if (w) a.task.w = *w;
  a.key = seed;
  a.p0 = p0;
  a.P = P;
  a.S = S;
  a.u = u_out;
  a.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_seeds<double>(a) : crk::launch_seeds<float>(a);
}

cr_status cr_topk(const float* cost, const float* coll, const void* u, int32_t d, int64_t P, int32_t S,
                  int32_t k, double dedup_eps, int32_t* idx_out, int32_t dtype, cr_stream stream) {
  cr_status st;
  if ((st = check_dtype(dtype))) return st;
  if (P < 0 || S < 1 || S > CR_MAX_SEEDS || k < 1 || k > 32 || d < 1 || d > 3 * CR_MAX_SEG || !(dedup_eps >= 0))
    return fail(CR_EINVAL, "cr_topk: bad sizes");
  if (P == 0) return CR_OK;
  if ((st = check_ptr(cost, 4, "cost", true)) || (st = check_ptr(coll, 4, "coll", true)) ||
      (st = check_ptr(u, dsize(dtype), "u", true)) || (st = check_ptr(idx_out, 4, "idx_out", true)))
    return st;
  crk::SolveArgs a{};
  a.tk_cost = cost;
  a.tk_coll = coll;
  a.u = (void*)u;
  a.D = d;
  a.P = P;
  a.S = S;
  a.K = k;
  a.eps = dedup_eps;
  a.tk_idx = idx_out;
  a.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_topk<double>(a) : crk::launch_topk<float>(a);
}

}  // extern "C"
