// Host-side helpers of the C ABI: argument validation, the thread-local error string, conversion
// of the public structs to kernel parameters, and the workspace layout.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "cr.h"
#include "cr_device.cuh"

namespace crh {

cr_status fail(cr_status st, const char* fmt, ...);
cr_status check_launch(const char* what);

inline cudaStream_t stream_of(cr_stream s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline size_t dsize(int32_t dtype) { return dtype == CR_F64 ? 8 : 4; }

cr_status check_robot(const cr_robot* r);
cr_status check_tendon_model(const cr_robot* r, const char* what);  // CR_EINVAL for the arc model
cr_status check_scene(const cr_scene* s);
cr_status check_scene_shared(const cr_scene* s);
cr_status check_scene_spheres_only(const cr_scene* s, const char* who);
cr_status check_task(const cr_task* t, int64_t B);
cr_status check_dtype(int32_t dtype);
cr_status check_ptr(const void* p, size_t align, const char* name, bool required);

template <typename T> crk::RobotK<T> robot_k(const cr_robot& r) {
  crk::RobotK<T> k;
  k.n = r.n;
  k.nb = r.n_b;
  for (int i = 0; i < crk::NMAX; ++i) {
    bool on = i < r.n;
    k.L[i] = T(on ? r.L[i] : 0.0);
    k.K[i] = T(on ? -2.0 / (3.0 * r.r_c[i]) : 0.0);
    k.umax[i] = T(on ? r.u_max[i] : 0.0);
    k.thmax[i] = T(on ? r.theta_max[i] : 0.0);
    k.rc[i] = T(on ? r.r_c[i] : 1.0);
  }
  k.rbody = T(r.r_body);
  for (int i = 0; i < crk::NMAX; ++i) {
    bool on = i < r.n && r.model == CR_MODEL_ARC;
    k.lmin[i] = T(on ? r.l_min[i] : 0.0);
    k.lmax[i] = T(on ? r.l_max[i] : 0.0);
  }
  return k;
}

template <typename T> crk::WeightsK<T> weights_k(const cr_weights& w) {
  crk::WeightsK<T> k;
  k.wp = T(w.w_p);
  k.wR = T(w.w_R);
  k.wp2 = T(w.w_p * w.w_p);
  k.wR2 = T(w.w_R * w.w_R);
  k.rho_b = T(w.rho_b);
  k.rho_eq = T(w.rho_eq);
  k.rho_k = T(w.rho_k);
  k.rho_c = T(w.rho_c);
  k.sb = T(sqrt(w.rho_b));
  k.se = T(sqrt(w.rho_eq));
  k.sk = T(sqrt(w.rho_k));
  k.sc = T(sqrt(w.rho_c));
  k.delta = T(w.delta);
  k.rho_s = T(w.rho_s);
  k.ss = T(sqrt(w.rho_s));
  return k;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace of cr_solve_ik (and its plain comparator):
//   status word | candidate states (bulk precision) [D][P*K] | candidate FP64 states [D][P*K] |
//   candidate FP64 cost, pos, rot [P*K] each | candidate flags [P*K] | plain-form scratch (states,
//   gradients, costs) |
//   stage-one end states: cost, clearance part (FP32) [P*S] each, states (bulk precision) [D][P*S]
struct IkLayout {
  size_t status, cand_u, cand_u64, cand_F, cand_pos, cand_rot, cand_flag, plain_u, plain_g, plain_F, stage_F,
      stage_C, stage_u, total;
};
// weights.rho_s must be >= 0; with supported = false it must be 0 (the solver has no self-contact rows)
cr_status check_self_rows(const cr_weights& w, bool supported, const char* who);
IkLayout ik_layout(const cr_robot& r, int64_t P, const cr_ik_params& prm);

// Launch helper: the number of segments is a template parameter of every kernel.
#define CR_DISPATCH_NT(n, FN, T, ...)             \
  switch (n) {                                    \
    case 1: FN<T, 1>(__VA_ARGS__); break;         \
    case 2: FN<T, 2>(__VA_ARGS__); break;         \
    case 3: FN<T, 3>(__VA_ARGS__); break;         \
    case 4: FN<T, 4>(__VA_ARGS__); break;         \
    case 5: FN<T, 5>(__VA_ARGS__); break;         \
    default: FN<T, 6>(__VA_ARGS__); break;        \
  }

}  // namespace crh
