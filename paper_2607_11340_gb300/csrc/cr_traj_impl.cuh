// Trajectory planning (Sec. IV-A, Eq. mp_length_only with the tendon speed / acceleration limits by
// finite differences) and kinematic calibration.
//
// One CTA per trajectory, one thread per timestep t. Each thread runs the forward phase of its own
// state (chain, clearance, penalty rows), shares its tip position and tendon state through shared
// memory, evaluates the coupling rows it owns (length, speed, acceleration between t and its
// predecessors), shares their derivatives, and runs the reverse phase of its state with the tip
// force of the length rows (and of the goal pose at the last state). Sums over the trajectory are
// deterministic block reductions.
#pragma once

#include "cr_solve_impl.cuh"

namespace crk {

template <typename T> struct TrajW {
  T dt, vmax, amax, w_len, rho_v, rho_a;
};

// Deterministic block sum: butterfly inside each warp, then every thread adds the warp totals in
// warp order. red[] holds 32 values; blockDim.x is a multiple of 32.
template <typename T> __device__ T block_sum(T v, T* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
  for (int k = 0; k < nw; ++k) s += red[k];
  return s;
}
template <typename T> __device__ T block_max(T v, T* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = c_max(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = red[0];
  for (int k = 1; k < nw; ++k) s = c_max(s, red[k]);
  return s;
}

// Shared buffers of one trajectory: tip positions [Tn][3], states [Tn][D], speed and acceleration
// row derivatives [Tn][D] each, reduction scratch [32]; for the split evaluation (two threads per
// state, see traj_state_eval) the second thread's clearance aggregates [Tn][8 N] and the gradient
// handed back to it [Tn][D].
template <typename T> struct TrajSmem {
  T* p;
  T* u;
  T* sv;
  T* sa;
  T* red;
  T* xag;
  T* xg;
  __host__ __device__ static size_t bytes(int Tn, int D) {
    return sizeof(T) * ((size_t)Tn * (3 + 3 * D) + 32 + (size_t)Tn * (8 * (D / 3) + D));
  }
  __device__ void carve(unsigned char* base, int Tn, int D) {
    T* q = reinterpret_cast<T*>(base);
    p = q;
    u = p + (size_t)Tn * 3;
    sv = u + (size_t)Tn * D;
    sa = sv + (size_t)Tn * D;
    red = sa + (size_t)Tn * D;
    xag = red + 32;
    xg = xag + (size_t)Tn * 8 * (D / 3);
  }
};

// Thread t's share of the trajectory cost; with GRAD, gu = dF/du_t (zero for t = 0 and t >= Tn).
// Every thread of the block must call it (it synchronises). Split evaluation (split = true): two
// threads per state, each with its own part of the spheres (sph, no); the helper (aux = true) adds
// only the clearance rows of its spheres to F and passes their force / moment aggregates to the
// owner through shared memory, the owner runs everything else and hands the gradient back.
template <typename T, int N, bool OBST, bool GRAD>
__device__ T traj_state_eval(const RobotK<T>& rb, const WeightsK<T>& w, const TrajW<T>& tw, int t, int Tn,
                             const T (&u)[3 * N], const TargetK<T>& goal, ObsK<T> sph, int no,
                             TrajSmem<T>& sm, T (&gu)[3 * N], bool split = false, bool aux = false) {
  constexpr int D = 3 * N;
  const bool active = t < Tn;
  Chain<T, N> ch;
  StateAgg<T, N> ag;
  T F = T(0);
  T Ftip[3] = {T(0), T(0), T(0)}, Rtip[3] = {T(0), T(0), T(0)};
  if (aux) {
    if (active && t >= 1) {
      T coll = T(0);
      state_forward<T, N, OBST, GRAD, false>(rb, w, sph, no, u, ch, ag, &coll, false);  // the owner has the self rows
      F = coll;
      if (GRAD) {
        T* x = sm.xag + (size_t)t * 8 * N;
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
          for (int a = 0; a < 3; ++a) { x[6 * i + a] = ag.G[i][a]; x[6 * i + 3 + a] = ag.M[i][a]; }
          x[6 * N + 2 * i] = ag.Dx[i];
          x[6 * N + 2 * i + 1] = ag.Dy[i];
        }
      }
    }
    __syncthreads();
    if (!GRAD) return F;
    __syncthreads();
    __syncthreads();
#pragma unroll
    for (int q = 0; q < D; ++q) gu[q] = (active && t >= 1) ? sm.xg[(size_t)t * D + q] : T(0);
    return F;
  }
  if (active) {
    if (t == 0) {
      chain_forward(rb, u, ch);  // the start state is fixed: only its tip enters the length rows
    } else {
      F = state_forward<T, N, OBST, GRAD, false>(rb, w, sph, no, u, ch, ag, nullptr);
    }
    if (t == Tn - 1) {
      T r[6], e[3], ang, sn, cs;
      pose_rows(CR_TASK_IK6, w, goal, ch.R, ch.p, r, e, ang, sn, cs);
      F += T(0.5) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
      if (GRAD) pose_tip_force(CR_TASK_IK6, w, goal, ch.R, r, e, Ftip, Rtip);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) sm.p[t * 3 + a] = ch.p[a];
#pragma unroll
    for (int q = 0; q < D; ++q) sm.u[t * D + q] = u[q];
  }
  __syncthreads();
  T sv[D], sa[D];
#pragma unroll
  for (int q = 0; q < D; ++q) { sv[q] = T(0); sa[q] = T(0); }
  if (active && t >= 1) {
    T dp0 = ch.p[0] - sm.p[(t - 1) * 3], dp1 = ch.p[1] - sm.p[(t - 1) * 3 + 1], dp2 = ch.p[2] - sm.p[(t - 1) * 3 + 2];
    F += T(0.5) * tw.w_len * (dp0 * dp0 + dp1 * dp1 + dp2 * dp2);
    const T idt = T(1) / tw.dt, idt2 = idt * idt;
#pragma unroll
    for (int q = 0; q < D; ++q) {
      T v = (u[q] - sm.u[(t - 1) * D + q]) * idt;
      T hu = v - tw.vmax, hl = -tw.vmax - v;
      hu = hu > T(0) ? hu : T(0);
      hl = hl > T(0) ? hl : T(0);
      F += T(0.5) * tw.rho_v * (hu * hu + hl * hl);
      sv[q] = tw.rho_v * (hu - hl) * idt;
      if (t >= 2) {
        T acc = (u[q] - T(2) * sm.u[(t - 1) * D + q] + sm.u[(t - 2) * D + q]) * idt2;
        T au = acc - tw.amax, al = -tw.amax - acc;
        au = au > T(0) ? au : T(0);
        al = al > T(0) ? al : T(0);
        F += T(0.5) * tw.rho_a * (au * au + al * al);
        sa[q] = tw.rho_a * (au - al) * idt2;
      }
    }
  }
  if (!GRAD) return F;
  if (active) {
#pragma unroll
    for (int q = 0; q < D; ++q) { sm.sv[t * D + q] = sv[q]; sm.sa[t * D + q] = sa[q]; }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < D; ++q) gu[q] = T(0);
  if (split && active && t >= 1) {  // add the helper's clearance aggregates
    const T* x = sm.xag + (size_t)t * 8 * N;
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int a = 0; a < 3; ++a) { ag.G[i][a] += x[6 * i + a]; ag.M[i][a] += x[6 * i + 3 + a]; }
      ag.Dx[i] += x[6 * N + 2 * i];
      ag.Dy[i] += x[6 * N + 2 * i + 1];
    }
  }
  if (active && t >= 1) {
    // length rows (t-1, t) and (t, t+1) act on the tip of state t
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T f = tw.w_len * (ch.p[a] - sm.p[(t - 1) * 3 + a]);
      if (t + 1 < Tn) f -= tw.w_len * (sm.p[(t + 1) * 3 + a] - ch.p[a]);
      Ftip[a] += f;
    }
    state_reverse<T, N, false>(rb, w, u, ch, ag, Ftip, Rtip, gu, nullptr, nullptr);
    // speed rows of t and t+1, acceleration rows of t, t+1 and t+2 act on u_t directly
#pragma unroll
    for (int q = 0; q < D; ++q) {
      T g = sv[q] + sa[q];
      if (t + 1 < Tn) g += -sm.sv[(t + 1) * D + q] - T(2) * sm.sa[(t + 1) * D + q];
      if (t + 2 < Tn) g += sm.sa[(t + 2) * D + q];
      gu[q] += g;
    }
  }
  if (split) {  // hand the gradient to the helper thread of the same state
    if (active) {
#pragma unroll
      for (int q = 0; q < D; ++q) sm.xg[(size_t)t * D + q] = gu[q];
    }
    __syncthreads();
  }
  return F;
}

template <typename T> struct TrajArgs {
  const double* u_start;  // [D][P]
  const double* goal;     // [7][P]
  int64_t P;
  int Tn;
  const double* spheres;
  int no;
  const double* prims;
  int np;
  int sph_pp;
  // cost / gradient
  const T* x;             // [D][P*(Tn-1)]
  T* cost;
  T* grad;
  const T* upstream;
  // solve
  const double* u_goal;   // [D][P]
  const double* x_init;   // [D][P*Tn] initial states (nullable: linear interpolation to u_goal)
  int k_traj;
  T alpha0;
  double lim_tol;
  double dt_d, vmax_d, amax_d;
  double* X_out;          // [D][P*Tn]
  double* F_out;
  double* goal_pos;
  double* goal_rot;
  double* speed;
  double* accel;
  unsigned char* lim_ok;
  unsigned char* col_ok;
};

// Stage problem p's obstacle set (the shared one without per-problem scenes) at base (PRIMS:
// stage_obstacles_as).
template <bool PRIMS = true, typename T, typename A>
__device__ ObsK<T> stage_traj_obstacles(const A& a, int64_t p, const RobotK<T>& rb, T delta, unsigned char* base) {
  const int64_t q = a.sph_pp ? p : 0;
  return stage_obstacles_as<PRIMS>(a.spheres + q * a.no * 4, a.no,
                                   a.np > 0 ? a.prims + q * a.np * CR_PRIM_DOUBLES : nullptr, a.np, rb, delta, base);
}

template <typename T, int N, bool OBST, bool GRAD>
__global__ void __launch_bounds__(256) k_traj_cost(RobotK<T> rb, WeightsK<T> w, TrajW<T> tw, TrajArgs<T> a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t p = blockIdx.x;
  const int t = threadIdx.x, Tn = a.Tn;
  size_t off = (obstacles_smem<T>(a.no, a.np) + 15) & ~size_t(15);
  TrajSmem<T> sm;
  sm.carve(smem_raw + off, Tn, D);
  ObsK<T> sph(nullptr);
  if (OBST) {
    sph = stage_traj_obstacles(a, p, rb, w.delta, smem_raw);
    __syncthreads();
  }
  const int64_t ld = a.P * (Tn - 1);
  T u[D];
#pragma unroll
  for (int q = 0; q < D; ++q) {
    if (t == 0) u[q] = T(a.u_start[q * a.P + p]);
    else if (t < Tn) u[q] = a.x[q * ld + p * (Tn - 1) + (t - 1)];
    else u[q] = T(0);
  }
  TargetK<T> goal = load_target<T>(a.goal, a.P, p, CR_TASK_IK6);
  T gu[D];
  T F = traj_state_eval<T, N, OBST, GRAD>(rb, w, tw, t, Tn, u, goal, sph, a.no + a.np, sm, gu);
  T Ft = block_sum(F, sm.red);
  if (t == 0) a.cost[p] = Ft;
  if (GRAD && t >= 1 && t < Tn) {
    T s = a.upstream ? a.upstream[p] : T(1);
#pragma unroll
    for (int q = 0; q < D; ++q) a.grad[q * ld + p * (Tn - 1) + (t - 1)] = s * gu[q];
  }
}

// Trajectory planning after the goal IK: linear initialisation (or the given initial states x_init), k_traj
// projected-gradient steps of all free states, FP64 metrics of the result.
template <typename T, int N, bool OBST, bool PRIMS = true>
__global__ void __launch_bounds__(256, 1) k_traj_solve(RobotK<T> rb, WeightsK<T> w, TrajW<T> tw, RobotK<double> rbd,
                                                     WeightsK<double> wd, TrajArgs<T> a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t p = blockIdx.x;
  const int Tn = a.Tn, Wt = ((Tn + 31) / 32) * 32;
  // split evaluation (blockDim = 2 Wt): thread t and t + Wt share state t, each with half the obstacles
  const bool split = (int)blockDim.x == 2 * Wt;
  const bool aux = split && (int)threadIdx.x >= Wt;
  const int t = aux ? (int)threadIdx.x - Wt : (int)threadIdx.x;
  const int nob = a.no + a.np;
  const size_t offd = (obstacles_smem<T>(a.no, a.np) + 15) & ~size_t(15);
  size_t off = offd + ((obstacles_smem<double>(a.no, a.np) + 15) & ~size_t(15));
  TrajSmem<T> sm;
  sm.carve(smem_raw + off, Tn, D);
  ObsK<T> sph(nullptr);
  ObsK<double> sphd(nullptr);
  if (OBST) {
    sph = stage_traj_obstacles<PRIMS>(a, p, rb, w.delta, smem_raw);
    sphd = stage_traj_obstacles<PRIMS>(a, p, rbd, wd.delta, smem_raw + offd);
    __syncthreads();
  }
  const bool active = t < Tn;
  const int nh = split ? (nob + 1) / 2 : nob;
  const ObsK<T> sph_m = aux ? sph.from(nh) : sph;
  const int no_m = aux ? nob - nh : nh;
  T u[D];
#pragma unroll
  for (int q = 0; q < D; ++q) {
    if (a.x_init) {
      u[q] = active ? T(a.x_init[q * a.P * Tn + p * Tn + t]) : T(0);
      continue;
    }
    double u0 = a.u_start[q * a.P + p], ug = a.u_goal[q * a.P + p];
    u[q] = active ? T(u0 + (double)t / (Tn - 1) * (ug - u0)) : T(0);
  }
  TargetK<T> goal = load_target<T>(a.goal, a.P, p, CR_TASK_IK6);
  T g[D];
  T F = block_sum(traj_state_eval<T, N, OBST, true>(rb, w, tw, t, Tn, u, goal, sph_m, no_m, sm, g, split, aux),
                  sm.red);
  T alpha = a.alpha0;
  const bool free_state = active && t >= 1;
  for (int it = 0; it < a.k_traj; ++it) {
    T gn2l = T(0);
#pragma unroll
    for (int q = 0; q < D; ++q) gn2l += aux ? T(0) : g[q] * g[q];  // the helper holds a copy
    T gn2 = block_sum(gn2l, sm.red);
    T scale = gn2 > T(0) ? alpha * c_rsqrt(gn2) : T(0);
    T u1[D];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (free_state)
        project3(u[3 * i] - scale * g[3 * i], u[3 * i + 1] - scale * g[3 * i + 1], u[3 * i + 2] - scale * g[3 * i + 2],
                 rb.umax[i], u1[3 * i], u1[3 * i + 1], u1[3 * i + 2]);
      else {
        u1[3 * i] = u[3 * i]; u1[3 * i + 1] = u[3 * i + 1]; u1[3 * i + 2] = u[3 * i + 2];
      }
    }
    T g1[D];
    T F1 = block_sum(traj_state_eval<T, N, OBST, true>(rb, w, tw, t, Tn, u1, goal, sph_m, no_m, sm, g1, split, aux),
                     sm.red);
    if (F1 < F) {
#pragma unroll
      for (int q = 0; q < D; ++q) { u[q] = u1[q]; g[q] = g1[q]; }
      F = F1;
      alpha *= T(1.25);
    } else {
      alpha *= T(0.5);
    }
  }
  // outputs and FP64 metrics
  double ud[D];
#pragma unroll
  for (int q = 0; q < D; ++q) ud[q] = double(u[q]);
  const bool owner = active && !aux;  // outputs and FP64 metrics from one thread per state
  if (owner) {
#pragma unroll
    for (int q = 0; q < D; ++q) a.X_out[q * (a.P * Tn) + p * Tn + t] = ud[q];
  }
  double pos = 0, rot = 0;
  unsigned char flags = 3;
  if (owner) {
    TargetK<double> gd = load_target<double>(a.goal, a.P, p, CR_TASK_IK6);
    accept_fp64<N, OBST>(rbd, wd, CR_TASK_IK6, gd, sphd, nob, ud, a.lim_tol, pos, rot, flags);
  }
  // speed / acceleration ratios in FP64 over the states shared in a double buffer
  double* sd = reinterpret_cast<double*>(smem_raw + off + ((TrajSmem<T>::bytes(Tn, D) + 15) & ~size_t(15)));
  double* redd = sd + (size_t)Tn * D;
  if (owner)
#pragma unroll
    for (int q = 0; q < D; ++q) sd[t * D + q] = ud[q];
  __syncthreads();
  double vmax_r = 0, amax_r = 0;
  if (owner && t >= 1) {
#pragma unroll
    for (int q = 0; q < D; ++q) {
      vmax_r = fmax(vmax_r, fabs(ud[q] - sd[(t - 1) * D + q]) / a.dt_d / a.vmax_d);
      if (t >= 2)
        amax_r = fmax(amax_r, fabs(ud[q] - 2.0 * sd[(t - 1) * D + q] + sd[(t - 2) * D + q]) / (a.dt_d * a.dt_d) / a.amax_d);
    }
  }
  double vr = block_max(vmax_r, redd);
  double ar = block_max(amax_r, redd);
  double lim = block_max(double((flags & 1) ? 0 : 1), redd);
  double col = block_max(double((flags & 2) ? 0 : 1), redd);
  if (!aux && t == Tn - 1) {
    a.goal_pos[p] = pos;
    a.goal_rot[p] = rot;
  }
  if (!aux && t == 0) {
    a.F_out[p] = double(F);
    a.speed[p] = vr;
    a.accel[p] = ar;
    a.lim_ok[p] = lim == 0.0;
    a.col_ok[p] = col == 0.0;
  }
}

// ------------------------------------------------------------------------------------------------
// Calibration: theta = (L_1..n, r_c,1..n); residual p(u_k; theta) - p_k.
// ------------------------------------------------------------------------------------------------
// dp/dL_i = Rb_i d_i / L_i (everything after segment i translates); dp/dr_c,i = -(ax dp/dax +
// ay dp/day) / r_c with dp/da_k = v + w x p from the segment twists.
template <typename T, int N>
__device__ void calib_rows(const RobotK<T>& rb, const T (&u)[3 * N], const double* pm, T (&r)[3], T (&J)[3][2 * N]) {
  Chain<T, N> ch;
  chain_forward(rb, u, ch);
  T tv[N][2][3], tw[N][2][3];
  segment_twists(rb, ch, tv, tw);
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = ch.p[a] - T(pm[a]);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T di[3], Rd[3];
    di[0] = rb.L[i] * ch.c[i] * ch.ax[i];
    di[1] = rb.L[i] * ch.c[i] * ch.ay[i];
    di[2] = rb.L[i] * ch.s[i];
    matvec(ch.Rb[i], di, Rd);
    T wp0[3], wp1[3];
    cross(tw[i][0], ch.p, wp0);
    cross(tw[i][1], ch.p, wp1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      J[a][i] = Rd[a] / rb.L[i];
      T dpx = tv[i][0][a] + wp0[a], dpy = tv[i][1][a] + wp1[a];
      J[a][N + i] = -(ch.ax[i] * dpx + ch.ay[i] * dpy) / rb.rc[i];
    }
  }
}

// Multi-block form. Per LM iteration, k_calib_accum (one thread per pose, 128 poses per block) adds
// each block's contributions to J^T J (packed), J^T r and F = 1/2 sum r^2 in FP64 (warp butterflies,
// then the four warps in order) into part[block][.]; k_calib_step (one block) adds the partials in
// block order, factors the damped system in FP64, evaluates the trial cost over all poses and applies
// the LM rule to theta (in place), lambda and nu (workspace). All sums have a fixed order.
constexpr int kCalibThreads = 128;
template <int N> constexpr int calib_nv() { return (2 * N) * (2 * N + 1) / 2 + 2 * N + 1; }

template <typename T, int N> __device__ RobotK<T> calib_robot(RobotK<T> rb, const double* theta) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    rb.L[i] = T(theta[i]);
    rb.rc[i] = T(theta[N + i]);
    rb.K[i] = T(-2.0 / (3.0 * theta[N + i]));
  }
  return rb;
}

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <typename T, int N>
__global__ void __launch_bounds__(kCalibThreads) k_calib_accum(RobotK<T> rb0, const T* __restrict__ U,
                                                              const double* __restrict__ Pm, int64_t K,
                                                              const double* theta, double* part) {
  constexpr int D = 3 * N, NP = 2 * N, NV = calib_nv<N>();
  __shared__ double red[kCalibThreads / 32][NV];
  __shared__ double th[NP];
  if (threadIdx.x < NP) th[threadIdx.x] = theta[threadIdx.x];
  __syncthreads();
  const RobotK<T> rb = calib_robot<T, N>(rb0, th);
  const int64_t k = (int64_t)blockIdx.x * kCalibThreads + threadIdx.x;
  T r[3] = {T(0), T(0), T(0)}, J[3][NP];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int x = 0; x < NP; ++x) J[a][x] = T(0);
  if (k < K) {
    T u[D];
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = U[q * K + k];
    const double pm[3] = {Pm[k], Pm[K + k], Pm[2 * K + k]};
    calib_rows<T, N>(rb, u, pm, r, J);
  }
  double Jd[3][NP], rd[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    rd[a] = double(r[a]);
#pragma unroll
    for (int x = 0; x < NP; ++x) Jd[a][x] = double(J[a][x]);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int v = 0;
#pragma unroll
  for (int x = 0; x < NP; ++x)
#pragma unroll
    for (int y = 0; y <= x; ++y, ++v) {
      const double c = warp_sum_d(fma(Jd[2][x], Jd[2][y], fma(Jd[1][x], Jd[1][y], Jd[0][x] * Jd[0][y])));
      if (lane == 0) red[wid][v] = c;
    }
#pragma unroll
  for (int x = 0; x < NP; ++x, ++v) {
    const double c = warp_sum_d(fma(Jd[2][x], rd[2], fma(Jd[1][x], rd[1], Jd[0][x] * rd[0])));
    if (lane == 0) red[wid][v] = c;
  }
  {
    const double c = warp_sum_d(0.5 * fma(rd[2], rd[2], fma(rd[1], rd[1], rd[0] * rd[0])));
    if (lane == 0) red[wid][v] = c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NV; e += kCalibThreads) {
    double s = red[0][e];
    for (int w = 1; w < kCalibThreads / 32; ++w) s += red[w][e];
    part[(int64_t)blockIdx.x * NV + e] = s;
  }
}

// Cost 1/2 sum |p(u_k; theta) - p_k|^2 (FP32 kinematics, FP64 sum) over all poses by one block.
template <typename T, int N>
__device__ double calib_cost_block(const RobotK<T>& rb, const T* __restrict__ U, const double* __restrict__ Pm,
                                   int64_t K, double* red) {
  constexpr int D = 3 * N;
  double lF = 0.0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
    T u[D];
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = U[q * K + k];
    Chain<T, N> ch;
    chain_forward(rb, u, ch);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double ra = double(ch.p[a] - T(Pm[a * K + k]));
      lF += 0.5 * ra * ra;
    }
  }
  return block_sum(lF, red);
}

// state: [0] lambda, [1] nu; part: [nblk][NV]
template <typename T, int N>
__global__ void __launch_bounds__(256) k_calib_step(RobotK<T> rb0, const T* __restrict__ U, const double* __restrict__ Pm,
                                                     int64_t K, int nblk, int it, double lambda0, double* theta,
                                                     double* state, const double* part, double* hist) {
  constexpr int NP = 2 * N, NA = NP * (NP + 1) / 2, NV = calib_nv<N>();
  __shared__ double tot[NV], thn[NP], red[32];
  __shared__ int ok;
  for (int e = threadIdx.x; e < NV; e += blockDim.x) {
    double s = part[e];
    for (int b = 1; b < nblk; ++b) s += part[(int64_t)b * NV + e];
    tot[e] = s;
  }
  __syncthreads();
  double lam = it == 0 ? lambda0 : state[0], nu = it == 0 ? 2.0 : state[1];
  double dl[NP], Dg[NP];
  if (threadIdx.x == 0) {
    double Ad[NA], iv[NP];
#pragma unroll
    for (int a = 0; a < NA; ++a) Ad[a] = tot[a];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      Dg[q] = fmax(Ad[tri(q, q)], 1e-12);
      Ad[tri(q, q)] += lam * Dg[q];
    }
    ok = cholesky_packed<NP>(Ad, iv) ? 1 : 0;
#pragma unroll
    for (int q = 0; q < NP; ++q) dl[q] = -tot[NA + q];
    if (ok) {
      cholesky_solve<NP>(Ad, iv, dl);
#pragma unroll
      for (int q = 0; q < NP; ++q) thn[q] = theta[q] + dl[q];
    }
  }
  __syncthreads();
  double Fn = 0.0;
  if (ok) Fn = calib_cost_block<T, N>(calib_robot<T, N>(rb0, thn), U, Pm, K, red);
  if (threadIdx.x == 0) {
    const double F = tot[NV - 1];
    if (ok && Fn < F) {
      double pred = 0.0;
#pragma unroll
      for (int q = 0; q < NP; ++q) pred += dl[q] * (lam * Dg[q] * dl[q] - tot[NA + q]);
      pred *= 0.5;
      const double rho = (F - Fn) / pred, tt = 2.0 * rho - 1.0;
      lam *= fmax(1.0 / 3.0, 1.0 - tt * tt * tt);
      nu = 2.0;
#pragma unroll
      for (int q = 0; q < NP; ++q) theta[q] = thn[q];
    } else {
      lam *= nu;
      nu *= 2.0;
    }
    state[0] = lam;
    state[1] = nu;
  }
  __syncthreads();
  if (hist && threadIdx.x < NP) hist[(int64_t)it * NP + threadIdx.x] = theta[threadIdx.x];
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_calib_final(RobotK<T> rb0, const T* __restrict__ U, const double* __restrict__ Pm,
                                                      int64_t K, const double* theta, double* F_out) {
  constexpr int NP = 2 * N;
  __shared__ double th[NP], red[32];
  if (threadIdx.x < NP) th[threadIdx.x] = theta[threadIdx.x];
  __syncthreads();
  const double F = calib_cost_block<T, N>(calib_robot<T, N>(rb0, th), U, Pm, K, red);
  if (threadIdx.x == 0) *F_out = F;
}

// Sharded calibration: the pieces of k_calib_step as separate launches, so that processes holding
// shares of the poses can add their partial sums (an all-reduce) in between. Each piece repeats the
// arithmetic of k_calib_step in the same order, so one process running them equals cr_calibrate.
// sums [NV]: the share's packed J^T J, J^T r and F; state [4]: lambda, nu, ok, pred.
template <int N>
__global__ void __launch_bounds__(256) k_calib_sum_parts(int nblk, const double* part, double* sums) {
  constexpr int NV = calib_nv<N>();
  for (int e = threadIdx.x; e < NV; e += blockDim.x) {
    double s = part[e];
    for (int b = 1; b < nblk; ++b) s += part[(int64_t)b * NV + e];
    sums[e] = s;
  }
}

template <int N>
__global__ void k_calib_trial(const double* sums, const double* theta, double* state, double* theta_trial) {
  constexpr int NP = 2 * N, NA = NP * (NP + 1) / 2;
  if (threadIdx.x != 0) return;
  const double lam = state[0];
  double Ad[NA], iv[NP], Dg[NP], dl[NP];
#pragma unroll
  for (int a = 0; a < NA; ++a) Ad[a] = sums[a];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    Dg[q] = fmax(Ad[tri(q, q)], 1e-12);
    Ad[tri(q, q)] += lam * Dg[q];
  }
  const bool ok = cholesky_packed<NP>(Ad, iv);
#pragma unroll
  for (int q = 0; q < NP; ++q) dl[q] = -sums[NA + q];
  double pred = 0.0;
  if (ok) {
    cholesky_solve<NP>(Ad, iv, dl);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      theta_trial[q] = theta[q] + dl[q];
      pred += dl[q] * (lam * Dg[q] * dl[q] - sums[NA + q]);
    }
    pred *= 0.5;
  } else {
#pragma unroll
    for (int q = 0; q < NP; ++q) theta_trial[q] = theta[q];
  }
  state[2] = ok ? 1.0 : 0.0;
  state[3] = pred;
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_calib_cost(RobotK<T> rb0, const T* __restrict__ U, const double* __restrict__ Pm,
                                                     int64_t K, const double* theta, double* F_out) {
  constexpr int NP = 2 * N;
  __shared__ double th[NP], red[32];
  if (threadIdx.x < NP) th[threadIdx.x] = theta[threadIdx.x];
  __syncthreads();
  const double F = calib_cost_block<T, N>(calib_robot<T, N>(rb0, th), U, Pm, K, red);
  if (threadIdx.x == 0) *F_out = F;
}

template <int N>
__global__ void k_calib_accept(const double* sums, const double* F_trial, const double* theta_trial, double* theta,
                               double* state) {
  constexpr int NP = 2 * N, NV = calib_nv<N>();
  if (threadIdx.x != 0) return;
  double lam = state[0], nu = state[1];
  const double F = sums[NV - 1], Fn = *F_trial;
  if (state[2] != 0.0 && Fn < F) {
    const double rho = (F - Fn) / state[3], tt = 2.0 * rho - 1.0;
    lam *= fmax(1.0 / 3.0, 1.0 - tt * tt * tt);
    nu = 2.0;
#pragma unroll
    for (int q = 0; q < NP; ++q) theta[q] = theta_trial[q];
  } else {
    lam *= nu;
    nu *= 2.0;
  }
  state[0] = lam;
  state[1] = nu;
}

// ------------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------------
struct TrajLaunch {
  cr_robot robot;
  cr_scene scene;
  cr_traj_task task;
  const void* x;
  void *cost, *grad;
  const void* upstream;
  // solve
  const double* u_goal;
  const double* x_init;  // nullable
  int k_traj;
  double alpha0, lim_tol;
  double *X_out, *F_out, *goal_pos, *goal_rot, *speed, *accel;
  unsigned char *lim_ok, *col_ok;
  // calibration
  const void* U;
  const double* Pm;
  int64_t K;
  int iters;
  double lambda0;
  double *theta_dev, *F_dev, *hist_dev;
  void* calib_ws;
  // sharded calibration: which piece (0 sums, 1 trial, 2 cost, 3 accept) and its arrays
  int calib_piece;
  double *sums, *state, *theta_trial;
  const double* F_trial;
  cudaStream_t stream;
};

template <typename T> cr_status launch_traj_cost(const TrajLaunch& l);
template <typename T> cr_status launch_traj_solve(const TrajLaunch& l);
template <typename T> cr_status launch_calibrate(const TrajLaunch& l);
template <typename T> cr_status launch_calib_piece(const TrajLaunch& l);

template <typename T> TrajW<T> traj_w(const cr_weights& w) {
  TrajW<T> t;
  t.dt = T(w.dt);
  t.vmax = T(w.v_max);
  t.amax = T(w.a_max);
  t.w_len = T(w.w_len);
  t.rho_v = T(w.rho_v);
  t.rho_a = T(w.rho_a);
  return t;
}

template <typename T> TrajArgs<T> traj_args(const TrajLaunch& l) {
  TrajArgs<T> a{};
  a.u_start = l.task.u_start;
  a.goal = l.task.goal;
  a.P = l.task.P;
  a.Tn = l.task.T;
  a.spheres = l.scene.spheres;
  a.no = l.scene.n_o;
  a.prims = l.scene.prims;
  a.np = l.scene.n_p;
  a.sph_pp = (l.scene.per_problem && l.scene.n_o + l.scene.n_p > 0) ? 1 : 0;
  a.x = (const T*)l.x;
  a.cost = (T*)l.cost;
  a.grad = (T*)l.grad;
  a.upstream = (const T*)l.upstream;
  a.u_goal = l.u_goal;
  a.x_init = l.x_init;
  a.k_traj = l.k_traj;
  a.alpha0 = T(l.alpha0);
  a.lim_tol = l.lim_tol;
  a.dt_d = l.task.w.dt;
  a.vmax_d = l.task.w.v_max;
  a.amax_d = l.task.w.a_max;
  a.X_out = l.X_out;
  a.F_out = l.F_out;
  a.goal_pos = l.goal_pos;
  a.goal_rot = l.goal_rot;
  a.speed = l.speed;
  a.accel = l.accel;
  a.lim_ok = l.lim_ok;
  a.col_ok = l.col_ok;
  return a;
}

template <typename T, int N> cr_status traj_cost_n(const TrajLaunch& l) {
  constexpr int D = 3 * N;
  RobotK<T> rb = crh::robot_k<T>(l.robot);
  WeightsK<T> w = crh::weights_k<T>(l.task.w);
  TrajW<T> tw = traj_w<T>(l.task.w);
  TrajArgs<T> a = traj_args<T>(l);
  const int threads = ((a.Tn + 31) / 32) * 32;
  size_t sm = ((obstacles_smem<T>(a.no, a.np) + 15) & ~size_t(15)) + TrajSmem<T>::bytes(a.Tn, D);
  cr_status st;
  if (a.no + a.np > 0 || w.rho_s > T(0)) {  // collision rows: obstacles and / or self-contact
    if (l.grad) { if ((st = set_smem(k_traj_cost<T, N, true, true>, sm))) return st;
      k_traj_cost<T, N, true, true><<<(unsigned)a.P, threads, sm, l.stream>>>(rb, w, tw, a); }
    else { if ((st = set_smem(k_traj_cost<T, N, true, false>, sm))) return st;
      k_traj_cost<T, N, true, false><<<(unsigned)a.P, threads, sm, l.stream>>>(rb, w, tw, a); }
  } else {
    if (l.grad) { if ((st = set_smem(k_traj_cost<T, N, false, true>, sm))) return st;
      k_traj_cost<T, N, false, true><<<(unsigned)a.P, threads, sm, l.stream>>>(rb, w, tw, a); }
    else { if ((st = set_smem(k_traj_cost<T, N, false, false>, sm))) return st;
      k_traj_cost<T, N, false, false><<<(unsigned)a.P, threads, sm, l.stream>>>(rb, w, tw, a); }
  }
  return crh::check_launch("cr_traj_cost");
}

template <typename T, int N> cr_status traj_solve_n(const TrajLaunch& l) {
  constexpr int D = 3 * N;
  RobotK<T> rb = crh::robot_k<T>(l.robot);
  WeightsK<T> w = crh::weights_k<T>(l.task.w);
  RobotK<double> rbd = crh::robot_k<double>(l.robot);
  WeightsK<double> wd = crh::weights_k<double>(l.task.w);
  TrajW<T> tw = traj_w<T>(l.task.w);
  TrajArgs<T> a = traj_args<T>(l);
  // FP32 with obstacles: two threads per state share the clearance rows (the FP64 form keeps one, its
  // sums in the oracle's order)
  const int Wt = ((a.Tn + 31) / 32) * 32;
  const int threads = (sizeof(T) == 4 && a.no + a.np >= 2 && 2 * Wt <= 256) ? 2 * Wt : Wt;
  size_t sm = ((obstacles_smem<T>(a.no, a.np) + 15) & ~size_t(15)) +
              ((obstacles_smem<double>(a.no, a.np) + 15) & ~size_t(15)) +
              ((TrajSmem<T>::bytes(a.Tn, D) + 15) & ~size_t(15)) + ((size_t)a.Tn * D + 32) * sizeof(double);
  cr_status st;
  if (a.np > 0) {
    if ((st = set_smem(k_traj_solve<T, N, true>, sm))) return st;
    k_traj_solve<T, N, true><<<(unsigned)a.P, threads, sm, l.stream>>>(rb, w, tw, rbd, wd, a);
  } else if (a.no > 0 || w.rho_s > T(0)) {  // spheres and / or self-contact: the form without primitive code
    if ((st = set_smem(k_traj_solve<T, N, true, false>, sm))) return st;
    k_traj_solve<T, N, true, false><<<(unsigned)a.P, threads, sm, l.stream>>>(rb, w, tw, rbd, wd, a);
  } else {
    if ((st = set_smem(k_traj_solve<T, N, false>, sm))) return st;
    k_traj_solve<T, N, false><<<(unsigned)a.P, threads, sm, l.stream>>>(rb, w, tw, rbd, wd, a);
  }
  return crh::check_launch("cr_solve_traj");
}

template <typename T, int N> cr_status calibrate_n(const TrajLaunch& l) {
  RobotK<T> rb = crh::robot_k<T>(l.robot);
  const int nblk = (int)((l.K + kCalibThreads - 1) / kCalibThreads);
  double* state = (double*)l.calib_ws;
  double* part = state + 2;
  const T* U = (const T*)l.U;
  for (int it = 0; it < l.iters; ++it) {
    k_calib_accum<T, N><<<nblk, kCalibThreads, 0, l.stream>>>(rb, U, l.Pm, l.K, l.theta_dev, part);
    k_calib_step<T, N><<<1, 256, 0, l.stream>>>(rb, U, l.Pm, l.K, nblk, it, l.lambda0, l.theta_dev, state, part,
                                                 l.hist_dev);
  }
  k_calib_final<T, N><<<1, 256, 0, l.stream>>>(rb, U, l.Pm, l.K, l.theta_dev, l.F_dev);
  return crh::check_launch("cr_calibrate");
}

template <typename T, int N> cr_status calib_piece_n(const TrajLaunch& l) {
  RobotK<T> rb = crh::robot_k<T>(l.robot);
  const T* U = (const T*)l.U;
  switch (l.calib_piece) {
    case 0: {  // partial sums of this share: per-block partials, then their sum in block order
      const int nblk = (int)((l.K + kCalibThreads - 1) / kCalibThreads);
      double* part = (double*)l.calib_ws + 2;
      k_calib_accum<T, N><<<nblk, kCalibThreads, 0, l.stream>>>(rb, U, l.Pm, l.K, l.theta_dev, part);
      k_calib_sum_parts<N><<<1, 256, 0, l.stream>>>(nblk, part, l.sums);
      break;
    }
    case 1: k_calib_trial<N><<<1, 32, 0, l.stream>>>(l.sums, l.theta_dev, l.state, l.theta_trial); break;
    case 2: k_calib_cost<T, N><<<1, 256, 0, l.stream>>>(rb, U, l.Pm, l.K, l.theta_dev, l.F_dev); break;
    default: k_calib_accept<N><<<1, 32, 0, l.stream>>>(l.sums, l.F_trial, l.theta_trial, l.theta_dev, l.state);
  }
  return crh::check_launch("sharded calibration");
}

// Workspace of cr_calibrate: lambda, nu, then the per-block partial sums.
inline size_t calibrate_ws_bytes(int n, int64_t K) {
  const int NP = 2 * n;
  const int64_t nblk = (K + kCalibThreads - 1) / kCalibThreads;
  return (size_t)(2 + nblk * (NP * (NP + 1) / 2 + NP + 1)) * sizeof(double);
}

#define CR_TRAJ_DISPATCH(FN, T, l)         \
  switch ((l).robot.n) {                   \
    case 1: return FN<T, 1>(l);            \
    case 2: return FN<T, 2>(l);            \
    case 3: return FN<T, 3>(l);            \
    case 4: return FN<T, 4>(l);            \
    case 5: return FN<T, 5>(l);            \
    default: return FN<T, 6>(l);           \
  }

template <typename T> cr_status launch_traj_cost(const TrajLaunch& l) { CR_TRAJ_DISPATCH(traj_cost_n, T, l) }
template <typename T> cr_status launch_traj_solve(const TrajLaunch& l) { CR_TRAJ_DISPATCH(traj_solve_n, T, l) }
template <typename T> cr_status launch_calibrate(const TrajLaunch& l) { CR_TRAJ_DISPATCH(calibrate_n, T, l) }
template <typename T> cr_status launch_calib_piece(const TrajLaunch& l) { CR_TRAJ_DISPATCH(calib_piece_n, T, l) }

#define CR_TRAJ_INSTANTIATE(EXT, T)                                  \
  EXT template cr_status launch_traj_cost<T>(const TrajLaunch&);     \
  EXT template cr_status launch_traj_solve<T>(const TrajLaunch&);    \
  EXT template cr_status launch_calibrate<T>(const TrajLaunch&);    \
  EXT template cr_status launch_calib_piece<T>(const TrajLaunch&);

}  // namespace crk
