// C ABI of the kinematics and cost entry points: cr_fk, cr_fk_jac, cr_cost_grad, cr_reduce_rows.
#include "cr_eval_impl.cuh"

namespace crk {
CR_EVAL_INSTANTIATE(extern, float)
CR_EVAL_INSTANTIATE(extern, double)
}

using namespace crh;

extern "C" {

cr_status cr_fk(const cr_robot* robot, const void* u, int64_t B, void* T_out, void* backbone_out,
                int32_t dtype, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_dtype(dtype))) return st;
  if (B < 0) return fail(CR_EINVAL, "cr_fk: B < 0");
  if (B == 0) return CR_OK;
  size_t es = dsize(dtype);
  if ((st = check_ptr(u, es, "u", true)) || (st = check_ptr(T_out, es, "T_out", true)) ||
      (st = check_ptr(backbone_out, es, "backbone_out", false)))
    return st;
  crk::EvalArgs a{};
  a.robot = *robot;
  a.u = u;
  a.B = B;
  a.Tout = T_out;
  a.bb = backbone_out;
  a.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_fk<double>(a) : crk::launch_fk<float>(a);
}

cr_status cr_fk_jac(const cr_robot* robot, const void* u, int64_t B, void* J_out, int32_t dtype,
                    cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_dtype(dtype))) return st;
  if (B < 0) return fail(CR_EINVAL, "cr_fk_jac: B < 0");
  if (B == 0) return CR_OK;
  size_t es = dsize(dtype);
  if ((st = check_ptr(u, es, "u", true)) || (st = check_ptr(J_out, es, "J_out", true))) return st;
  crk::EvalArgs a{};
  a.robot = *robot;
  a.u = u;
  a.B = B;
  a.J = J_out;
  a.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_fk_jac<double>(a) : crk::launch_fk_jac<float>(a);
}

cr_status cr_cost_grad(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                       const void* u, int64_t B, void* cost_out, void* coll_out, void* grad_u_out,
                       void* grad_param_out, int32_t dtype, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_scene_shared(scene)) || (st = check_task(task, B)) ||
      (st = check_dtype(dtype)))
    return st;
  if (B < 0) return fail(CR_EINVAL, "cr_cost_grad: B < 0");
  if (B == 0) return CR_OK;
  size_t es = dsize(dtype);
  if ((st = check_ptr(u, es, "u", true)) || (st = check_ptr(cost_out, es, "cost_out", true)) ||
      (st = check_ptr(coll_out, es, "coll_out", false)) ||
      (st = check_ptr(grad_u_out, es, "grad_u_out", false)) ||
      (st = check_ptr(grad_param_out, es, "grad_param_out", false)))
    return st;
  if (grad_param_out && !grad_u_out)
    return fail(CR_EINVAL, "cr_cost_grad: grad_param_out needs grad_u_out");
  crk::EvalArgs a{};
  a.robot = *robot;
  if (scene) a.scene = *scene;
  a.task = *task;
  a.u = u;
  a.B = B;
  a.cost = cost_out;
  a.coll = coll_out;
  a.gu = grad_u_out;
  a.gp = grad_param_out;
  a.stream = stream_of(stream);
  return dtype == CR_F64 ? crk::launch_cost_grad<double>(a) : crk::launch_cost_grad<float>(a);
}

cr_status cr_cost_vjp(const cr_robot* robot, const cr_scene* scene, const cr_task* task, const void* u, int64_t B,
                      const void* upstream, void* grad_u_out, double* grad_param_out, void* workspace, int32_t dtype,
                      cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "cr_cost_vjp")) ||
      (st = check_scene_shared(scene)) || (st = check_task(task, B)) || (st = check_dtype(dtype)))
    return st;
  if (B < 0) return fail(CR_EINVAL, "cr_cost_vjp: B < 0");
  if (B == 0) return CR_OK;
  size_t es = dsize(dtype);
  if ((st = check_ptr(u, es, "u", true)) || (st = check_ptr(upstream, es, "upstream", true)) ||
      (st = check_ptr(grad_u_out, es, "grad_u_out", true)) ||
      (st = check_ptr(grad_param_out, 8, "grad_param_out", false)) ||
      (st = check_ptr(workspace, es, "workspace", grad_param_out != nullptr)))
    return st;
  crk::EvalArgs a{};
  a.robot = *robot;
  if (scene) a.scene = *scene;
  a.task = *task;
  a.u = u;
  a.B = B;
  a.gu = grad_u_out;
  a.gp = grad_param_out ? workspace : nullptr;
  a.upstream = upstream;
  a.stream = stream_of(stream);
  st = dtype == CR_F64 ? crk::launch_cost_grad<double>(a) : crk::launch_cost_grad<float>(a);
  if (st || !grad_param_out) return st;
  return dtype == CR_F64 ? crk::launch_reduce_rows<double>(workspace, 2 * robot->n, B, grad_param_out, a.stream)
                         : crk::launch_reduce_rows<float>(workspace, 2 * robot->n, B, grad_param_out, a.stream);
}

cr_status cr_reduce_rows(const void* x, int64_t rows, int64_t B, double* out, int32_t dtype,
                         cr_stream stream) {
  cr_status st;
  if ((st = check_dtype(dtype))) return st;
  if (rows < 0 || B < 0) return fail(CR_EINVAL, "cr_reduce_rows: negative size");
  if (rows == 0) return CR_OK;
  if ((st = check_ptr(x, dsize(dtype), "x", B > 0)) || (st = check_ptr(out, 8, "out", true))) return st;
  if (rows > 2147483647LL) return fail(CR_EINVAL, "cr_reduce_rows: too many rows");
  return dtype == CR_F64 ? crk::launch_reduce_rows<double>(x, rows, B, out, stream_of(stream))
                         : crk::launch_reduce_rows<float>(x, rows, B, out, stream_of(stream));
}

}  // extern "C"
