// Kernels of the kinematics and cost entry points (cr_fk, cr_fk_jac, cr_cost_grad,
// cr_reduce_rows). One thread per state; states are structure-of-arrays [q][B] so that the
// per-component loads and stores of a warp are coalesced.
#pragma once

#include "cr_host.h"

namespace crk {

template <typename T, int N, int MODEL = CR_MODEL_TENDON>
__global__ void __launch_bounds__(128) k_fk(RobotK<T> rb, const T* __restrict__ u, int64_t B,
                                             T* __restrict__ Tout, T* __restrict__ bb) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  T uu[3 * N];
#pragma unroll
  for (int q = 0; q < 3 * N; ++q) uu[q] = u[q * B + b];
  Chain<T, N> ch;
  chain_forward<T, N, MODEL>(rb, uu, ch);
#pragma unroll
  for (int a = 0; a < 9; ++a) Tout[a * B + b] = ch.R[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) Tout[(9 + a) * B + b] = ch.p[a];
  if (bb) {
    const T inb = T(1) / T(rb.nb);
#pragma unroll
    for (int i = 0; i < N; ++i)
      for (int k = 1; k <= rb.nb; ++k) {
        T q[3], w[3], s, c;
        backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], T(k) * inb, q, w, s, c);
        int64_t row = (int64_t)(i * rb.nb + (k - 1)) * 3;
        bb[(row + 0) * B + b] = w[0];
        bb[(row + 1) * B + b] = w[1];
        bb[(row + 2) * B + b] = w[2];
      }
  }
}

template <typename T, int N, int MODEL = CR_MODEL_TENDON>
__global__ void __launch_bounds__(128) k_fk_jac(RobotK<T> rb, const T* __restrict__ u, int64_t B,
                                                 T* __restrict__ J) {
  constexpr int D = 3 * N;
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  T uu[D];
#pragma unroll
  for (int q = 0; q < D; ++q) uu[q] = u[q * B + b];
  Chain<T, N> ch;
  chain_forward<T, N, MODEL>(rb, uu, ch);
  T Jp[3][D], Jw[3][D];
  tip_jacobian<T, N, MODEL>(rb, ch, Jp, Jw);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int q = 0; q < D; ++q) {
      J[((int64_t)a * D + q) * B + b] = Jp[a][q];
      J[((int64_t)(3 + a) * D + q) * B + b] = Jw[a][q];
    }
}

// MODE 0: cost only; 1: cost + dF/du; 2: cost + dF/du + dF/d(L, r_c)
template <typename T, int N, bool OBST, int MODE, int MODEL = CR_MODEL_TENDON>
__global__ void __launch_bounds__(128) k_cost_grad(RobotK<T> rb, WeightsK<T> w, int kind,
                                                    const double* __restrict__ targets, int64_t P,
                                                    int S, const double* __restrict__ spheres, int no,
                                                    const double* __restrict__ prims, int np,
                                                    const T* __restrict__ u, int64_t B, T* cost,
                                                    T* coll, T* gu, T* gp, const T* __restrict__ upstream) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ObsK<T> ob(nullptr);
  if (OBST) {
    ob = stage_obstacles(spheres, no, prims, np, rb, w.delta, smem_raw);
    __syncthreads();
  }
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  T uu[D];
#pragma unroll
  for (int q = 0; q < D; ++q) uu[q] = u[q * B + b];
  TargetK<T> tg = load_target<T>(targets, P, b / S, kind);
  T g[D], gL[N], grc[N], cl;
  T F = eval_ik<T, N, OBST, (MODE >= 1), (MODE >= 2), true, MODEL>(rb, w, kind, tg, ob, no + np, uu, g, gL, grc,
                                                                    &cl);
  if (cost) cost[b] = F;
  if (coll) coll[b] = cl;
  const T up = upstream ? upstream[b] : T(1);  // vector-Jacobian product weight
  if (MODE >= 1) {
#pragma unroll
    for (int q = 0; q < D; ++q) gu[q * B + b] = up * g[q];
  }
  if (MODE >= 2) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      gp[(int64_t)i * B + b] = up * gL[i];
      gp[(int64_t)(N + i) * B + b] = up * grc[i];
    }
  }
}

// Deterministic row sums: one block per row, fixed per-thread strides and a fixed tree order.
template <typename T>
__global__ void __launch_bounds__(256) k_reduce_rows(const T* __restrict__ x, int64_t B, double* out) {
  __shared__ double part[256];
  const T* row = x + (int64_t)blockIdx.x * B;
  double s = 0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) s += double(row[b]);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = part[0];
}

// ------------------------------------------------------------------------------------------------
// Host launchers (instantiated for float and double in separate translation units)
// ------------------------------------------------------------------------------------------------
struct EvalArgs {
  cr_robot robot;
  cr_scene scene;
  cr_task task;
  const void* u;
  int64_t B;
  void *cost, *coll, *gu, *gp, *Tout, *bb, *J;
  const void* upstream;
  cudaStream_t stream;
};

template <typename T> cr_status launch_fk(const EvalArgs& a);
template <typename T> cr_status launch_fk_jac(const EvalArgs& a);
template <typename T> cr_status launch_cost_grad(const EvalArgs& a);
template <typename T> cr_status launch_reduce_rows(const void* x, int64_t rows, int64_t B, double* out,
                                                   cudaStream_t s);

inline unsigned grid_of(int64_t B, int bs) { return (unsigned)((B + bs - 1) / bs); }

template <typename T, int N, int MODEL = CR_MODEL_TENDON> void fk_n(const EvalArgs& a) {
  RobotK<T> rb = crh::robot_k<T>(a.robot);
  k_fk<T, N, MODEL><<<grid_of(a.B, 128), 128, 0, a.stream>>>(rb, (const T*)a.u, a.B, (T*)a.Tout, (T*)a.bb);
}
template <typename T, int N, int MODEL = CR_MODEL_TENDON> void fk_jac_n(const EvalArgs& a) {
  RobotK<T> rb = crh::robot_k<T>(a.robot);
  k_fk_jac<T, N, MODEL><<<grid_of(a.B, 128), 128, 0, a.stream>>>(rb, (const T*)a.u, a.B, (T*)a.J);
}
template <typename T, int N, int MODEL = CR_MODEL_TENDON> void cost_grad_n(const EvalArgs& a) {
  RobotK<T> rb = crh::robot_k<T>(a.robot);
  WeightsK<T> w = crh::weights_k<T>(a.task.w);
  int no = a.scene.n_o, np = a.scene.n_p;
  int mode = a.gp ? 2 : (a.gu ? 1 : 0);
  size_t sm = obstacles_smem<T>(no, np);
  unsigned g = grid_of(a.B, 128);
#define CR_CG(OB, MO)                                                                              \
  k_cost_grad<T, N, OB, MO, MODEL><<<g, 128, sm, a.stream>>>(rb, w, a.task.kind, a.task.targets,   \
                                                       a.task.n_targets, a.task.seeds_per_target,  \
                                                       a.scene.spheres, no, a.scene.prims, np,     \
                                                       (const T*)a.u, a.B,                         \
                                                       (T*)a.cost, (T*)a.coll, (T*)a.gu, (T*)a.gp, \
                                                       (const T*)a.upstream)
  if (no + np > 0 || a.task.w.rho_s > 0) {  // collision rows: obstacles and / or self-contact
    if (mode == 0) CR_CG(true, 0); else if (mode == 1) CR_CG(true, 1); else CR_CG(true, 2);
  } else {
    if (mode == 0) CR_CG(false, 0); else if (mode == 1) CR_CG(false, 1); else CR_CG(false, 2);
  }
#undef CR_CG
}

// The arc model's launchers (1..CR_MAX_SEG_ARC segments) live in their own translation units.
#define CR_EVAL_ARC(FN, T, a)                  \
  switch ((a).robot.n) {                       \
    case 1: FN<T, 1, CR_MODEL_ARC>(a); break;  \
    case 2: FN<T, 2, CR_MODEL_ARC>(a); break;  \
    case 3: FN<T, 3, CR_MODEL_ARC>(a); break;  \
    default: FN<T, 4, CR_MODEL_ARC>(a); break; \
  }
template <typename T> void launch_eval_arc(const EvalArgs& a, int what) {
  if (what == 0) { CR_EVAL_ARC(fk_n, T, a) }
  else if (what == 1) { CR_EVAL_ARC(fk_jac_n, T, a) }
  else { CR_EVAL_ARC(cost_grad_n, T, a) }
}

// Coupled routing (model B), 1..CR_MAX_SEG segments, in its own translation units.
#define CR_EVAL_COUPLED(FN, T, a)                  \
  switch ((a).robot.n) {                           \
    case 1: FN<T, 1, CR_MODEL_COUPLED>(a); break;  \
    case 2: FN<T, 2, CR_MODEL_COUPLED>(a); break;  \
    case 3: FN<T, 3, CR_MODEL_COUPLED>(a); break;  \
    case 4: FN<T, 4, CR_MODEL_COUPLED>(a); break;  \
    case 5: FN<T, 5, CR_MODEL_COUPLED>(a); break;  \
    default: FN<T, 6, CR_MODEL_COUPLED>(a); break; \
  }
template <typename T> void launch_eval_coupled(const EvalArgs& a, int what) {
  if (what == 0) { CR_EVAL_COUPLED(fk_n, T, a) }
  else if (what == 1) { CR_EVAL_COUPLED(fk_jac_n, T, a) }
  else { CR_EVAL_COUPLED(cost_grad_n, T, a) }
}

template <typename T> cr_status launch_fk(const EvalArgs& a) {
  if (a.robot.model == CR_MODEL_ARC) launch_eval_arc<T>(a, 0);
  else if (a.robot.model == CR_MODEL_COUPLED) launch_eval_coupled<T>(a, 0);
  else CR_DISPATCH_NT(a.robot.n, fk_n, T, a);
  return crh::check_launch("cr_fk");
}
template <typename T> cr_status launch_fk_jac(const EvalArgs& a) {
  if (a.robot.model == CR_MODEL_ARC) launch_eval_arc<T>(a, 1);
  else if (a.robot.model == CR_MODEL_COUPLED) launch_eval_coupled<T>(a, 1);
  else CR_DISPATCH_NT(a.robot.n, fk_jac_n, T, a);
  return crh::check_launch("cr_fk_jac");
}
template <typename T> cr_status launch_cost_grad(const EvalArgs& a) {
  if (a.robot.model == CR_MODEL_ARC) launch_eval_arc<T>(a, 2);
  else if (a.robot.model == CR_MODEL_COUPLED) launch_eval_coupled<T>(a, 2);
  else CR_DISPATCH_NT(a.robot.n, cost_grad_n, T, a);
  return crh::check_launch("cr_cost_grad");
}

#define CR_EVAL_ARC_INSTANTIATE(EXT, T) EXT template void launch_eval_arc<T>(const EvalArgs&, int);
#define CR_EVAL_COUPLED_INSTANTIATE(EXT, T) EXT template void launch_eval_coupled<T>(const EvalArgs&, int);
template <typename T>
cr_status launch_reduce_rows(const void* x, int64_t rows, int64_t B, double* out, cudaStream_t s) {
  k_reduce_rows<T><<<(unsigned)rows, 256, 0, s>>>((const T*)x, B, out);
  return crh::check_launch("cr_reduce_rows");
}

#define CR_EVAL_INSTANTIATE(EXT, T)                                                              \
  EXT template cr_status launch_fk<T>(const EvalArgs&);                                          \
  EXT template cr_status launch_fk_jac<T>(const EvalArgs&);                                      \
  EXT template cr_status launch_cost_grad<T>(const EvalArgs&);                                   \
  EXT template cr_status launch_reduce_rows<T>(const void*, int64_t, int64_t, double*, cudaStream_t);

}  // namespace crk
