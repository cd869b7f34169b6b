// C ABI plumbing: thread-local error string, argument validation, workspace layout, status poll.
#include <string.h>

#include "cr_host.h"

namespace crh {

static thread_local char g_err[512] = "no error";

cr_status fail(cr_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

cr_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return CR_OK;
}

cr_status check_dtype(int32_t dtype) {
  if (dtype != CR_F32 && dtype != CR_F64) return fail(CR_EINVAL, "dtype %d is not CR_F32/CR_F64", dtype);
  return CR_OK;
}

cr_status check_ptr(const void* p, size_t align, const char* name, bool required) {
  if (!p) return required ? fail(CR_EINVAL, "%s is NULL", name) : CR_OK;
  if (!aligned(p, align)) return fail(CR_EINVAL, "%s is not %zu-byte aligned", name, align);
  return CR_OK;
}

cr_status check_robot(const cr_robot* r) {
  if (!r) return fail(CR_EINVAL, "robot is NULL");
  if (r->n < 1 || r->n > CR_MAX_SEG) return fail(CR_EINVAL, "robot.n = %d outside 1..%d", r->n, CR_MAX_SEG);
  if (r->m != 3) return fail(CR_EINVAL, "robot.m = %d: only 3 tendons per segment are supported", r->m);
  if (r->n_b < 1 || r->n_b > CR_MAX_NB) return fail(CR_EINVAL, "robot.n_b = %d outside 1..%d", r->n_b, CR_MAX_NB);
  for (int i = 0; i < r->n; ++i) {
    if (!(r->L[i] > 0) || !(r->r_c[i] > 0) || !(r->u_max[i] > 0) || !(r->theta_max[i] > 0))
      return fail(CR_EINVAL, "segment %d: L, r_c, u_max and theta_max must be positive", i);
  }
  if (!(r->r_body >= 0)) return fail(CR_EINVAL, "robot.r_body must be >= 0");
  if (r->model != CR_MODEL_TENDON && r->model != CR_MODEL_ARC && r->model != CR_MODEL_COUPLED)
    return fail(CR_EINVAL, "robot.model = %d is not a cr_model", r->model);
  if (r->model == CR_MODEL_ARC) {
    if (r->n > CR_MAX_SEG_ARC) return fail(CR_EINVAL, "arc model: robot.n = %d above %d", r->n, CR_MAX_SEG_ARC);
    for (int i = 0; i < r->n; ++i)
      if (!(r->l_min[i] > 0) || !(r->l_max[i] >= r->l_min[i]))
        return fail(CR_EINVAL, "arc model, segment %d: need 0 < l_min <= l_max", i);
  }
  return CR_OK;
}

cr_status check_tendon_model(const cr_robot* r, const char* what) {
  if (r && r->model != CR_MODEL_TENDON) return fail(CR_EINVAL, "%s takes the tendon model only", what);
  return CR_OK;
}

cr_status check_scene(const cr_scene* s) {
  if (!s) return CR_OK;  // no scene = no obstacles
  if (s->n_o < 0 || s->n_o > CR_MAX_SPHERES)
    return fail(CR_EINVAL, "scene.n_o = %d outside 0..%d", s->n_o, CR_MAX_SPHERES);
  if (s->n_p < 0 || s->n_p > CR_MAX_SPHERES - s->n_o)
    return fail(CR_EINVAL, "scene.n_p = %d: n_o + n_p must lie in 0..%d", s->n_p, CR_MAX_SPHERES);
  if (s->per_problem != 0 && s->per_problem != 1) return fail(CR_EINVAL, "scene.per_problem must be 0 or 1");
  cr_status st = CR_OK;
  if (s->n_o > 0 && (st = check_ptr(s->spheres, 8, "scene.spheres", true))) return st;
  if (s->n_p > 0 && (st = check_ptr(s->prims, 8, "scene.prims", true))) return st;
  return CR_OK;
}

cr_status check_scene_shared(const cr_scene* s) {
  cr_status st = check_scene(s);
  if (st) return st;
  if (s && s->per_problem && s->n_o + s->n_p > 0)
    return fail(CR_EINVAL, "this entry point takes one obstacle set for the whole batch (per_problem = 0)");
  return CR_OK;
}

cr_status check_scene_spheres_only(const cr_scene* s, const char* who) {
  cr_status st = check_scene(s);
  if (st) return st;
  if (s && s->n_p > 0) return fail(CR_EINVAL, "%s takes sphere obstacles only (scene.n_p = %d)", who, s->n_p);
  return CR_OK;
}

cr_status check_self_rows(const cr_weights& w, bool supported, const char* who) {
  if (!(w.rho_s >= 0.0)) return fail(CR_EINVAL, "%s: weights.rho_s must be >= 0", who);
  if (w.rho_s > 0.0 && !supported)
    return fail(CR_EINVAL, "%s: self-contact rows (weights.rho_s > 0) are not built for this solver", who);
  return CR_OK;
}

cr_status check_task(const cr_task* t, int64_t B) {
  if (!t) return fail(CR_EINVAL, "task is NULL");
  if (!(t->w.rho_s >= 0.0)) return fail(CR_EINVAL, "task.w.rho_s must be >= 0");
  if (t->kind != CR_TASK_IK6 && t->kind != CR_TASK_IK5) return fail(CR_EINVAL, "task.kind = %d invalid", t->kind);
  if (t->seeds_per_target < 1) return fail(CR_EINVAL, "task.seeds_per_target must be >= 1");
  if (t->n_targets < 0) return fail(CR_EINVAL, "task.n_targets < 0");
  if (B > 0 && (B + t->seeds_per_target - 1) / t->seeds_per_target > t->n_targets)
    return fail(CR_EINVAL, "task has %lld targets, batch of %lld states needs %lld", (long long)t->n_targets,
                (long long)B, (long long)((B + t->seeds_per_target - 1) / t->seeds_per_target));
  return check_ptr(t->targets, 8, "task.targets", B > 0);
}

IkLayout ik_layout(const cr_robot& r, int64_t P, const cr_ik_params& prm) {
  IkLayout L;
  const size_t D = 3 * (size_t)r.n;
  const size_t PK = (size_t)P * (size_t)prm.n_final;
  const size_t tb = prm.precision == CR_F64 ? 8 : 4;
  size_t off = 0;
  L.status = off; off = align256(off + 4);
  L.cand_u = off; off = align256(off + D * PK * tb);
  L.cand_u64 = off; off = align256(off + D * PK * 8);
  L.cand_F = off; off = align256(off + PK * 8);
  L.cand_pos = off; off = align256(off + PK * 8);
  L.cand_rot = off; off = align256(off + PK * 8);
  L.cand_flag = off; off = align256(off + PK);
  L.plain_u = off; off = align256(off + (size_t)prm.S * D * 8);
  L.plain_g = off; off = align256(off + (size_t)prm.S * D * 8);
  L.plain_F = off; off = align256(off + (size_t)prm.S * 8 * 3 + 32 * 4 + (size_t)prm.S * 5);
  const size_t PS = (size_t)P * (size_t)(prm.S > 0 ? prm.S : 0);
  L.stage_F = off; off = align256(off + PS * 4);
  L.stage_C = off; off = align256(off + PS * 4);
  L.stage_u = off; off = align256(off + D * PS * tb);
  L.total = off;
  return L;
}

}  // namespace crh

extern "C" {

const char* cr_last_error_string(void) { return crh::g_err; }

size_t cr_ik_workspace_size(const cr_robot* robot, int64_t P, const cr_ik_params* prm) {
  if (!robot || !prm || P < 0) return 0;
  return crh::ik_layout(*robot, P, *prm).total;
}

cr_status cr_poll_status(const void* workspace, int32_t* host_status, cr_stream stream) {
  if (!workspace || !host_status) return crh::fail(CR_EINVAL, "cr_poll_status: NULL argument");
  cudaStream_t s = crh::stream_of(stream);
  cudaError_t e = cudaMemcpyAsync(host_status, workspace, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return crh::fail(CR_ECUDA, "cr_poll_status: %s", cudaGetErrorString(e));
  return CR_OK;
}

}  // extern "C"
