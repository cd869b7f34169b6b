// C ABI of path following: cr_path_workspace_size, cr_solve_path.
#include "cr_path_impl.cuh"

namespace crk {
CR_PATH_INSTANTIATE(extern, float)
CR_PATH_INSTANTIATE(extern, double)

// Waypoint 0 of every path as a [7][P] target array.
__global__ void k_first_waypoints(const double* wp, int64_t P, int H, double* out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  for (int c = 0; c < 7; ++c) out[c * P + p] = wp[c * P * H + p * H];
}
}  // namespace crk

using namespace crh;

namespace {

struct PathWs {
  size_t ik, tg0, u0, cost, pos, rot, succ, X, Z, total;
};

PathWs path_ws(const cr_robot& r, int64_t P, int H, const cr_ik_params& g) {
  PathWs w;
  const size_t D = 3 * (size_t)r.n, tb = g.precision == CR_F64 ? 8 : 4;
  size_t off = 0;
  w.ik = off; off = align256(off + cr_ik_workspace_size(&r, P, &g));
  w.tg0 = off; off = align256(off + (size_t)7 * P * 8);
  w.u0 = off; off = align256(off + D * P * 8);
  w.cost = off; off = align256(off + (size_t)P * 8);
  w.pos = off; off = align256(off + (size_t)P * 8);
  w.rot = off; off = align256(off + (size_t)P * 8);
  w.succ = off; off = align256(off + (size_t)P);
  w.X = off; off = align256(off + D * P * H * tb);
  w.Z = off; off = align256(off + (size_t)P * H * crk::path_z_stride((int)D) * 8);
  w.total = off;
  return w;
}

}  // namespace

extern "C" {

size_t cr_path_workspace_size(const cr_robot* robot, int64_t P, int32_t H, const cr_ik_params* first_ik) {
  if (!robot || !first_ik || P < 0 || H < 1) return 0;
  return path_ws(*robot, P, H, *first_ik).total;
}

cr_status cr_solve_path(const cr_robot* robot, const cr_scene* scene, const cr_path_task* task,
                        const cr_ik_params* first_ik, int32_t k_warm, int32_t k_joint, double* X_out, double* cost_out,
                        double* pos_err, double* rot_err, uint8_t* lim_ok, uint8_t* col_ok, void* workspace,
                        size_t ws_bytes, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "cr_solve_path")) || (st = check_scene(scene)))
    return st;
  if (!task || !first_ik) return fail(CR_EINVAL, "cr_solve_path: NULL task or params");
  if ((st = check_self_rows(task->w, false, "cr_solve_path"))) return st;
  if (task->P < 0 || task->H < 2 || task->H > 128) return fail(CR_EINVAL, "cr_solve_path: P >= 0, H in 2..128");
  if (k_warm < 0 || k_joint < 0) return fail(CR_EINVAL, "cr_solve_path: negative iteration count");
  if (task->P == 0) return CR_OK;
  if (task->P > 2147483647LL) return fail(CR_EINVAL, "cr_solve_path: too many paths");
  if ((st = check_ptr(task->waypoints, 8, "waypoints", true)) || (st = check_ptr(X_out, 8, "X_out", true)) ||
      (st = check_ptr(cost_out, 8, "cost_out", true)) || (st = check_ptr(pos_err, 8, "pos_err", true)) ||
      (st = check_ptr(rot_err, 8, "rot_err", true)) || (st = check_ptr(lim_ok, 1, "lim_ok", true)) ||
      (st = check_ptr(col_ok, 1, "col_ok", true)) || (st = check_ptr(workspace, 256, "workspace", true)))
    return st;
  if ((st = check_dtype(first_ik->precision))) return st;
  const int64_t P = task->P;
  const int H = task->H;
  PathWs lay = path_ws(*robot, P, H, *first_ik);
  if (ws_bytes < lay.total) return fail(CR_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, lay.total);
  unsigned char* ws = (unsigned char*)workspace;
  cudaStream_t s = stream_of(stream);
  double* tg0 = (double*)(ws + lay.tg0);
  crk::k_first_waypoints<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(task->waypoints, P, H, tg0);
  if ((st = check_launch("cr_solve_path first waypoints"))) return st;
  cr_task it{};
  it.kind = CR_TASK_IK6;
  it.seeds_per_target = 1;
  it.targets = tg0;
  it.n_targets = P;
  it.w = task->w;
  double* u0 = (double*)(ws + lay.u0);
  if ((st = cr_solve_ik(robot, scene, &it, first_ik, u0, (double*)(ws + lay.cost), (double*)(ws + lay.pos),
                        (double*)(ws + lay.rot), ws + lay.succ, ws + lay.ik, lay.tg0 - lay.ik, stream)))
    return st;
  crk::PathLaunch l{};
  l.robot = *robot;
  if (scene) l.scene = *scene;
  l.wp = task->waypoints;
  l.P = P;
  l.H = H;
  l.w = task->w;
  l.k_warm = k_warm;
  l.k_joint = k_joint;
  l.lambda0 = first_ik->lambda0;
  l.lim_tol = first_ik->lim_tol;
  l.u0 = u0;
  l.X = ws + lay.X;
  l.Z = (double*)(ws + lay.Z);
  l.X_out = X_out;
  l.F_out = cost_out;
  l.pos = pos_err;
  l.rot = rot_err;
  l.lim_ok = lim_ok;
  l.col_ok = col_ok;
  l.stream = s;
  return first_ik->precision == CR_F64 ? crk::launch_path<double>(l) : crk::launch_path<float>(l);
}

}  // extern "C"
