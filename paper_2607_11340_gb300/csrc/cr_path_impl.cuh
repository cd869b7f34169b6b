// Path following (Sec. IV-A, Eq. constrained_mp; Sec. IV-B): IK at the first waypoint, then the
// exploration sweep (waypoint t starts from the solution of t-1 and runs k_warm LM iterations on
// its own IK residual), then the refinement: joint LM over all H waypoints with the successive-
// state smoothness rows sqrt(w_s)(u_t - u_{t-1}), whose normal matrix is block tridiagonal.
//
//  k_path_warm  : one warp per path. Every lane holds the path's state; residual rows are formed
//                 column-wise (lane q: entry q), J^T J accumulates in packed slots spread over the
//                 lanes, the damped system is solved by a warp sweep (bulk precision: this is
//                 exploration); backbone samples are split over the lanes for the clearance rows.
//  k_path_joint : one CTA per path. Thread t evaluates waypoint t's rows and its block of J^T J;
//                 one warp runs the FP64 block elimination over t (S_t = M_t - w_s^2 S_{t-1}^-1,
//                 forward and back substitution), each block inverted by a symmetric sweep whose
//                 packed entries are spread over the 32 lanes, so a block step needs no CTA barrier.
#pragma once

#include "cr_traj_impl.cuh"
#include "cr_warp.cuh"

namespace crk {

template <typename T> struct PathArgs {
  const double* wp;       // [7][P*H]
  int64_t P;
  int H;
  const double* spheres;  // [P][no][4] when sph_pp, else [no][4]
  int no;
  const double* prims;    // [P][np][CR_PRIM_DOUBLES] when sph_pp, else [np][CR_PRIM_DOUBLES]
  int np;
  int sph_pp;
  int k_warm, k_joint;
  double lambda0, lim_tol;
  T w_s;
  const double* u0;       // [D][P]   first waypoint (IK result)
  T* X;                   // [D][P*H] working states (bulk precision)
  double* Z;              // [P][H][path_z_stride(D)] swept blocks -S_t^-1 of the joint solve
  double* X_out;          // [D][P*H]
  double* F_out;          // [P]
  double* pos;            // [P*H]
  double* rot;            // [P*H]
  unsigned char* lim_ok;  // [P]
  unsigned char* col_ok;  // [P]
};

// ------------------------------------------------------------------------------------------------
// Exploration: warp-cooperative LM on one waypoint's IK residual
// ------------------------------------------------------------------------------------------------
// Per-warp shared scratch: obstacles (no spheres, np primitives) | col, colr, sx, sdg [32 each]
template <typename T> __host__ __device__ inline size_t warm_warp_bytes(int no, int np) {
  return ((obstacles_smem<T>(no, np) + 15) / 16 * 16) + 4 * 32 * sizeof(T);
}

template <typename T, int N, bool OBST>
__device__ void warm_sweep_warp(const RobotK<T>& rb, const WeightsK<T>& w, const double* wp, int64_t PH, int64_t base,
                                int H, int k_warm, T lam0, ObsK<T> sph, int no, T (&u)[3 * N], T* scratch,
                                T* Xout, int64_t xstride) {
  constexpr int D = 3 * N;
  const int lane = threadIdx.x & 31;
  const AugSlots<D> sl = aug_slots<D>(lane);
  T* col = scratch;
  T* colr = col + 32;
  T* sx = colr + 32;
  T* sdg = sx + 32;
  for (int t = 1; t < H; ++t) {
    TargetK<T> tg = load_target<T>(wp, PH, base + t, CR_TASK_IK6);
    T lam = lam0, nu = T(2);
    for (int it = 0; it < k_warm; ++it) warp_lm_step<T, N, OBST>(rb, w, tg, sph, no, u, sl, lam, nu, col, colr, sx, sdg);
#pragma unroll
    for (int q = 0; q < D; ++q)
      if (q == lane) Xout[q * xstride + t] = u[q];
  }
}

template <typename T, int N, bool OBST, bool PRIMS = true>
// 128 threads; the register cap is explicit (the default heuristic settles below what the exploration
// step needs and spills). PRIMS = false: the form for scenes without primitives.
__global__ void __maxnreg__(255) k_path_warm(RobotK<T> rb, WeightsK<T> w, PathArgs<T> a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * 4 + wid;
  unsigned char* mine = smem_raw + (size_t)wid * warm_warp_bytes<T>(a.no, a.np);
  T* scratch = reinterpret_cast<T*>(mine + (obstacles_smem<T>(a.no, a.np) + 15) / 16 * 16);
  const bool live = p < a.P;
  ObsK<T> sph(nullptr);
  if (OBST && live) {
    const int64_t q = a.sph_pp ? p : 0;
    sph = stage_obstacles_as<PRIMS>(a.spheres + q * a.no * 4, a.no,
                                    a.np > 0 ? a.prims + q * a.np * CR_PRIM_DOUBLES : nullptr, a.np, rb, w.delta, mine,
                                    lane, 32);
  }
  __syncwarp();
  if (!live) return;
  const int H = a.H;
  const int64_t PH = a.P * H;
  T u[D];
#pragma unroll
  for (int q = 0; q < D; ++q) u[q] = T(a.u0[q * a.P + p]);
  if (lane < D) a.X[lane * PH + p * H] = T(a.u0[lane * a.P + p]);
  warm_sweep_warp<T, N, OBST>(rb, w, a.wp, PH, p * H, H, a.k_warm, T(a.lambda0), sph, a.no + a.np, u, scratch,
                              a.X + p * H, PH);
}

// ------------------------------------------------------------------------------------------------
// Refinement: joint LM over the path, FP64 block-tridiagonal elimination
// ------------------------------------------------------------------------------------------------
// The joint LM system is block tridiagonal: diagonal blocks M_t = J_t^T J_t + w_s nb_t I + lambda D_t
// (nb_t = number of neighbours of waypoint t), off-diagonal blocks -w_s I, right-hand side r = -g.
// Block elimination: S_0 = M_0, S_t = M_t - w_s^2 S_{t-1}^-1; z_t = S_t^-1 (r_t + w_s z_{t-1});
// x_{H-1} = z_{H-1}, x_t = z_t + w_s S_t^-1 x_{t+1}. One warp runs it in FP64: the sweep of the
// augmented [S_t, r_t + w_s z_{t-1}] gives -S_t^-1 (kept in registers for the next Schur update and
// stored to Zg for the back substitution) and z_t together.
//   Af [H][DD] J^T J blocks (bulk precision), g [H][D], z [H][D] (z_t, then x_t in place)
template <typename TA, int D>
__device__ bool joint_solve_warp(const TA* Af, const double* g, double* z, double* Zg, double* col, double* colr,
                                 double* Zs, int H, double ws, double lam) {
  constexpr int SL = AugSlots<D>::SL, DD = D * (D + 1) / 2, ZS = aug_stride<D>();
  const int lane = threadIdx.x & 31;
  const AugSlots<D> sl = aug_slots<D>(lane);
  const double ws2 = ws * ws;
  double v[SL];
  bool ok = true;
  for (int t = 0; t < H; ++t) {
    const double nb = double((t > 0) + (t + 1 < H));
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      if (!sl.on[s]) continue;
      const int i = sl.r[s], j = sl.c[s];
      double a;
      if (i < D) {
        a = double(Af[(size_t)t * DD + tri(i, j)]);
        if (i == j) {
          a += ws * nb;
          a += lam * fmax(a, 1e-12);
        }
        if (t > 0) a = fma(ws2, v[s], a);  // v = -S_{t-1}^-1
      } else {
        a = j < D ? -g[t * D + j] + (t > 0 ? ws * z[(t - 1) * D + j] : 0.0) : 0.0;
      }
      v[s] = a;
    }
    ok = sweep_aug<double, D>(v, sl, col, colr) && ok;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      Zg[(size_t)t * ZS + s * 32 + lane] = v[s];
      if (sl.on[s] && sl.r[s] == D && sl.c[s] < D) z[t * D + sl.c[s]] = v[s];
    }
    __syncwarp();
  }
  // back substitution: x_t = z_t - w_s V_t x_{t+1}, V_t = -S_t^-1 as stored
  double nxt[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) nxt[s] = H >= 2 ? Zg[(size_t)(H - 2) * ZS + s * 32 + lane] : 0.0;
  for (int t = H - 2; t >= 0; --t) {
#pragma unroll
    for (int s = 0; s < SL; ++s)
      if (sl.on[s] && sl.r[s] < D) Zs[tri(sl.r[s], sl.c[s])] = nxt[s];
    if (t > 0) {
#pragma unroll
      for (int s = 0; s < SL; ++s) nxt[s] = Zg[(size_t)(t - 1) * ZS + s * 32 + lane];
    }
    __syncwarp();
    if (lane < D) {
      double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
      for (int j = 0; j < D; j += 2) {
        acc0 = fma(Zs[lane >= j ? tri(lane, j) : tri(j, lane)], z[(t + 1) * D + j], acc0);
        if (j + 1 < D) acc1 = fma(Zs[lane >= j + 1 ? tri(lane, j + 1) : tri(j + 1, lane)], z[(t + 1) * D + j + 1], acc1);
      }
      z[t * D + lane] = fma(-ws, acc0 + acc1, z[t * D + lane]);
    }
    __syncwarp();
  }
  return ok;
}

// Packs slot values v (this lane's slots of a swept block, the D x D part) into Zs [DD] (packed
// lower triangle) for the block-times-vector products of the back substitution.
template <int D>
__device__ inline void unpack_block(const AugSlots<D>& sl, const double (&v)[AugSlots<D>::SL], double* Zs) {
#pragma unroll
  for (int s = 0; s < AugSlots<D>::SL; ++s)
    if (sl.on[s] && sl.r[s] < D) Zs[tri(sl.r[s], sl.c[s])] = v[s];
}

// The same block-tridiagonal system as joint_solve_warp, eliminated from both ends at once (a
// twisted factorisation) by two warps: warp 0 eliminates t = 0 .. m-1 forward (S_t = M_t - w_s^2
// S_{t-1}^-1, z_t = S_t^-1 (r_t + w_s z_{t-1})), warp 1 eliminates t = H-1 .. m+1 backward (T_t = M_t -
// w_s^2 T_{t+1}^-1, y_t = T_t^-1 (r_t + w_s y_{t+1})); warp 0 then solves the middle block,
// (M_m - w_s^2 S_{m-1}^-1 - w_s^2 T_{m+1}^-1) x_m = r_m + w_s z_{m-1} + w_s y_{m+1}, and the two warps
// substitute back towards their ends (x_t = z_t + w_s S_t^-1 x_{t+1} below m, x_t = y_t + w_s
// T_t^-1 x_{t-1} above). The two sequential chains are half as long. Every thread of the block
// calls it (it synchronises the block); warps 0 and 1 work, col / colr / Zs hold one scratch per
// working warp ([2][32], [2][32], [2][DD]). Returns whether every pivot was positive.
template <typename TA, int D>
__device__ bool joint_solve_twisted(const TA* Af, const double* g, double* z, double* Zg, double* col, double* colr,
                                    double* Zs, int* okf, int H, double ws, double lam) {
  constexpr int SL = AugSlots<D>::SL, DD = D * (D + 1) / 2, ZS = aug_stride<D>();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = H / 2;
  const double ws2 = ws * ws;
  const AugSlots<D> sl = aug_slots<D>(lane);
  double* mycol = col + 32 * wid;
  double* mycolr = colr + 32 * wid;
  double* myZs = Zs + DD * wid;
  if (threadIdx.x == 0) *okf = 1;
  __syncthreads();
  // diagonal block of waypoint t with its damping, plus ws^2 times the slots of prev / prev2 (the
  // neighbours' -S^-1), and the right-hand side -g_t + ws (the neighbours' z, rows zn1 / zn2)
  auto build = [&](int t, const double* prev, const double* prev2, int zn1, int zn2, double (&v)[SL]) {
    const double nb = double((t > 0) + (t + 1 < H));
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      if (!sl.on[s]) continue;
      const int i = sl.r[s], j = sl.c[s];
      double a;
      if (i < D) {
        a = double(Af[(size_t)t * DD + tri(i, j)]);
        if (i == j) {
          a += ws * nb;
          a += lam * fmax(a, 1e-12);
        }
        if (prev) a = fma(ws2, prev[s], a);
        if (prev2) a = fma(ws2, prev2[s], a);
      } else {
        a = 0.0;
        if (j < D) {
          a = -g[t * D + j];
          if (zn1 >= 0) a += ws * z[zn1 * D + j];
          if (zn2 >= 0) a += ws * z[zn2 * D + j];
        }
      }
      v[s] = a;
    }
  };
  double v[SL];
  bool ok = true;
  if (wid < 2) {
    const int dir = wid == 0 ? 1 : -1;
    const int t0 = wid == 0 ? 0 : H - 1, t1 = wid == 0 ? m : m;  // exclusive end
    for (int t = t0; t != t1; t += dir) {
      double prevs[SL];
      const bool has_prev = t != t0;
#pragma unroll
      for (int s = 0; s < SL; ++s) prevs[s] = v[s];
      build(t, has_prev ? prevs : nullptr, nullptr, has_prev ? t - dir : -1, -1, v);
      ok = sweep_aug<double, D>(v, sl, mycol, mycolr) && ok;
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        Zg[(size_t)t * ZS + s * 32 + lane] = v[s];
        if (sl.on[s] && sl.r[s] == D && sl.c[s] < D) z[t * D + sl.c[s]] = v[s];
      }
      __syncwarp();
    }
    if (!ok && lane == 0) atomicAnd(okf, 0);
  }
  __syncthreads();
  // middle block (warp 0)
  if (wid == 0) {
    double pl[SL], pr[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      pl[s] = m > 0 ? Zg[(size_t)(m - 1) * ZS + s * 32 + lane] : 0.0;
      pr[s] = m + 1 < H ? Zg[(size_t)(m + 1) * ZS + s * 32 + lane] : 0.0;
    }
    build(m, m > 0 ? pl : nullptr, m + 1 < H ? pr : nullptr, m > 0 ? m - 1 : -1, m + 1 < H ? m + 1 : -1, v);
    const bool okm = sweep_aug<double, D>(v, sl, mycol, mycolr);
#pragma unroll
    for (int s = 0; s < SL; ++s)
      if (sl.on[s] && sl.r[s] == D && sl.c[s] < D) z[m * D + sl.c[s]] = v[s];
    if (!okm && lane == 0) atomicAnd(okf, 0);
  }
  __syncthreads();
  // back substitution towards the ends: x_t = z_t - ws V_t x_n, V_t = -S_t^-1 (or -T_t^-1) as
  // stored, n the neighbour on the middle's side
  if (wid < 2) {
    const int dir = wid == 0 ? -1 : 1;
    const int t0 = wid == 0 ? m - 1 : m + 1, t1 = wid == 0 ? -1 : H;
    for (int t = t0; t != t1; t += dir) {
      double vb[SL];
#pragma unroll
      for (int s = 0; s < SL; ++s) vb[s] = Zg[(size_t)t * ZS + s * 32 + lane];
      unpack_block<D>(sl, vb, myZs);
      __syncwarp();
      const int n = t - dir;
      if (lane < D) {
        double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
        for (int j = 0; j < D; j += 2) {
          acc0 = fma(myZs[lane >= j ? tri(lane, j) : tri(j, lane)], z[n * D + j], acc0);
          if (j + 1 < D) acc1 = fma(myZs[lane >= j + 1 ? tri(lane, j + 1) : tri(j + 1, lane)], z[n * D + j + 1], acc1);
        }
        z[t * D + lane] = fma(-ws, acc0 + acc1, z[t * D + lane]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  return *okf != 0;
}

// One CTA per path, one thread per waypoint (blockDim = H rounded up to a warp). Per iteration:
// every thread forms its waypoint's J^T J block and gradient (bulk precision) plus the smoothness
// terms; warp 0 solves the block system in FP64; all threads evaluate the trial path.
template <typename T, int N, bool OBST, bool PRIMS = true>
__global__ void __launch_bounds__(128) k_path_joint(RobotK<T> rb, WeightsK<T> w, RobotK<double> rbd,
                                                     WeightsK<double> wd, PathArgs<T> a) {
  constexpr int D = 3 * N, DD = D * (D + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t p = blockIdx.x;
  const int tid = threadIdx.x, H = a.H;
  const int64_t PH = a.P * H;
  // shared layout: obstacles (T, double) | g [H][D] | z [H][D] | col, colr [32] | Zs [DD] | red [32] |
  // misc [8] | col2, colr2 [2][32], Zs2 [2][DD] | Af [H][DD] (T) | ush [H][D] (T)
  const int nob = a.no + a.np;
  const size_t offd = (obstacles_smem<T>(a.no, a.np) + 15) & ~size_t(15);
  size_t off = offd + ((obstacles_smem<double>(a.no, a.np) + 15) & ~size_t(15));
  double* g = reinterpret_cast<double*>(smem_raw + off);
  double* z = g + (size_t)H * D;
  double* col = z + (size_t)H * D;
  double* colr = col + 32;
  double* Zs = colr + 32;
  double* red = Zs + DD;
  double* misc = red + 32;  // [8]: ok flag
  double* col2 = misc + 8;  // the twisted solve's scratch: col, colr [2][32], Zs [2][DD]
  double* colr2 = col2 + 64;
  double* Zs2 = colr2 + 64;
  T* Af = reinterpret_cast<T*>(Zs2 + 2 * DD);
  T* ush = Af + (size_t)H * DD;
  double* Zg = a.Z + (size_t)p * H * aug_stride<D>();
  ObsK<T> sph(nullptr);
  ObsK<double> sphd(nullptr);
  if (OBST) {
    const int64_t q = a.sph_pp ? p : 0;
    const double* sp = a.spheres + q * a.no * 4;
    const double* pr = a.np > 0 ? a.prims + q * a.np * CR_PRIM_DOUBLES : nullptr;
    sph = stage_obstacles_as<PRIMS>(sp, a.no, pr, a.np, rb, w.delta, smem_raw);
    sphd = stage_obstacles_as<PRIMS>(sp, a.no, pr, a.np, rbd, wd.delta, smem_raw + offd);
  }
  const bool wthr = tid < H;
  T u[D];
#pragma unroll
  for (int q = 0; q < D; ++q) u[q] = wthr ? a.X[q * PH + p * H + tid] : T(0);
  TargetK<T> tg = load_target<T>(a.wp, PH, p * H + (wthr ? tid : 0), CR_TASK_IK6);
  __syncthreads();
  const double ws = double(a.w_s);
  double lam = a.lambda0, nu = 2.0;

  // cost of the path at states `uu` (thread t: waypoint t), with the smoothness rows
  auto path_cost = [&](const T (&uu)[D]) -> double {
    double Fl = 0.0;
    if (wthr) {
      T dummy[D];
      Fl = double(eval_ik<T, N, OBST, false, false>(rb, w, CR_TASK_IK6, tg, sph, nob, uu, dummy, nullptr, nullptr, nullptr));
#pragma unroll
      for (int q = 0; q < D; ++q) ush[tid * D + q] = uu[q];
    }
    __syncthreads();
    if (wthr && tid >= 1) {
#pragma unroll
      for (int q = 0; q < D; ++q) {
        double dq = double(uu[q]) - double(ush[(tid - 1) * D + q]);
        Fl += 0.5 * ws * dq * dq;
      }
    }
    double F = block_sum(Fl, red);
    __syncthreads();
    return F;
  };

  for (int it = 0; it < a.k_joint; ++it) {
    // 1. J^T J block and J^T r of every waypoint, plus the smoothness rows' gradient
    double Fl = 0.0;
    if (wthr) {
      T At[DD], gt[D];
      Fl = double(eval_ik_normal<T, T, N, OBST>(rb, w, CR_TASK_IK6, tg, sph, nob, u, At, gt));
#pragma unroll
      for (int e = 0; e < DD; ++e) Af[tid * DD + e] = At[e];
#pragma unroll
      for (int q = 0; q < D; ++q) {
        g[tid * D + q] = double(gt[q]);
        ush[tid * D + q] = u[q];
      }
    }
    __syncthreads();
    if (wthr) {
#pragma unroll
      for (int q = 0; q < D; ++q) {
        double s = 0.0, uq = double(u[q]);
        if (tid > 0) {
          double dq = uq - double(ush[(tid - 1) * D + q]);
          s += ws * dq;
          Fl += 0.5 * ws * dq * dq;
        }
        if (tid + 1 < H) s -= ws * (double(ush[(tid + 1) * D + q]) - uq);
        g[tid * D + q] += s;
      }
    }
    const double F = block_sum(Fl, red);
    __syncthreads();
    // 2. FP64 block elimination: from both ends by two warps (from 4 waypoints on), else by warp 0
    if (H >= 4 && blockDim.x >= 64) {
      const bool okw = joint_solve_twisted<T, D>(Af, g, z, Zg, col2, colr2, Zs2, reinterpret_cast<int*>(misc + 1), H,
                                                 ws, lam);
      if (tid == 0) misc[0] = okw ? 1.0 : 0.0;
    } else if (tid < 32) {
      const bool okw = joint_solve_warp<T, D>(Af, g, z, Zg, col, colr, Zs, H, ws, lam);
      if (tid == 0) misc[0] = okw ? 1.0 : 0.0;
    }
    __syncthreads();
    if (misc[0] == 0.0) {
      lam *= nu;
      nu *= 2.0;
      __syncthreads();
      continue;
    }
    // 3. trial, gain ratio 1/2 x^T (lambda D x - g), accept
    T un[D];
    double predl = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q) un[q] = wthr ? u[q] + T(z[tid * D + q]) : u[q];
    if (wthr) {
      const double nb = double((tid > 0) + (tid + 1 < H));
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const double xq = z[tid * D + q];
        const double dg = fmax(double(Af[tid * DD + tri(q, q)]) + ws * nb, 1e-12);
        predl += xq * (lam * dg * xq - g[tid * D + q]);
      }
    }
    const double pred = 0.5 * block_sum(predl, red);
    __syncthreads();
    const double Fn = path_cost(un);
    if (Fn < F) {
      double rho = (F - Fn) / pred, tt = 2.0 * rho - 1.0;
      lam *= fmax(1.0 / 3.0, 1.0 - tt * tt * tt);
      nu = 2.0;
#pragma unroll
      for (int q = 0; q < D; ++q) u[q] = un[q];
    } else {
      lam *= nu;
      nu *= 2.0;
    }
    __syncthreads();
  }
  // outputs: states, joint cost, FP64 per-waypoint metrics
  const double Ff = path_cost(u);
  double ud[D];
#pragma unroll
  for (int q = 0; q < D; ++q) ud[q] = double(u[q]);
  unsigned char flags = 3;
  if (wthr) {
#pragma unroll
    for (int q = 0; q < D; ++q) a.X_out[q * PH + p * H + tid] = ud[q];
    TargetK<double> tgd = load_target<double>(a.wp, PH, p * H + tid, CR_TASK_IK6);
    double pos, rot;
    accept_fp64<N, OBST>(rbd, wd, CR_TASK_IK6, tgd, sphd, nob, ud, a.lim_tol, pos, rot, flags);
    a.pos[p * H + tid] = pos;
    a.rot[p * H + tid] = rot;
  }
  const double lim_bad = block_max(double((flags & 1) ? 0 : 1), red);
  const double col_bad = block_max(double((flags & 2) ? 0 : 1), red);
  if (tid == 0) {
    a.F_out[p] = Ff;
    a.lim_ok[p] = lim_bad == 0.0;
    a.col_ok[p] = col_bad == 0.0;
  }
}

// ------------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------------
struct PathLaunch {
  cr_robot robot;
  cr_scene scene;
  const double* wp;
  int64_t P;
  int H;
  cr_weights w;
  int k_warm, k_joint;
  double lambda0, lim_tol;
  const double* u0;
  void* X;
  double* Z;
  double *X_out, *F_out, *pos, *rot;
  unsigned char *lim_ok, *col_ok;
  cudaStream_t stream;
};

template <typename T> cr_status launch_path(const PathLaunch& l);

template <typename T> PathArgs<T> path_args(const PathLaunch& l) {
  PathArgs<T> a{};
  a.wp = l.wp;
  a.P = l.P;
  a.H = l.H;
  a.spheres = l.scene.spheres;
  a.no = l.scene.n_o;
  a.prims = l.scene.prims;
  a.np = l.scene.n_p;
  a.sph_pp = (l.scene.per_problem && l.scene.n_o + l.scene.n_p > 0) ? 1 : 0;
  a.k_warm = l.k_warm;
  a.k_joint = l.k_joint;
  a.lambda0 = l.lambda0;
  a.lim_tol = l.lim_tol;
  a.w_s = T(l.w.w_s);
  a.u0 = l.u0;
  a.X = (T*)l.X;
  a.Z = l.Z;
  a.X_out = l.X_out;
  a.F_out = l.F_out;
  a.pos = l.pos;
  a.rot = l.rot;
  a.lim_ok = l.lim_ok;
  a.col_ok = l.col_ok;
  return a;
}

template <typename T> inline size_t path_joint_smem(int no, int np, int H, int D) {
  const size_t tsize = sizeof(T);
  size_t off = ((obstacles_smem<T>(no, np) + 15) & ~size_t(15)) + ((obstacles_smem<double>(no, np) + 15) & ~size_t(15));
  off += sizeof(double) * ((size_t)2 * H * D + 64 + (size_t)D * (D + 1) / 2 + 32 + 8 + 128 + (size_t)D * (D + 1));
  off += tsize * ((size_t)H * D * (D + 1) / 2 + (size_t)H * D);
  return off;
}

// doubles of the joint solve's block storage per waypoint (the workspace's Z region)
inline int path_z_stride(int D) { return ((D + 1) * (D + 2) / 2 + 31) / 32 * 32; }

template <typename T, int N> cr_status path_n(const PathLaunch& l) {
  constexpr int D = 3 * N, DD = D * (D + 1) / 2;
  RobotK<T> rb = crh::robot_k<T>(l.robot);
  WeightsK<T> w = crh::weights_k<T>(l.w);
  RobotK<double> rbd = crh::robot_k<double>(l.robot);
  WeightsK<double> wd = crh::weights_k<double>(l.w);
  PathArgs<T> a = path_args<T>(l);
  cr_status st;
  // exploration sweep
  size_t smw = 4 * warm_warp_bytes<T>(a.no, a.np);
  unsigned gw = (unsigned)((a.P + 3) / 4);
  if (a.np > 0) {
    if ((st = set_smem(k_path_warm<T, N, true>, smw))) return st;
    k_path_warm<T, N, true><<<gw, 128, smw, l.stream>>>(rb, w, a);
  } else if (a.no > 0) {  // spheres only: the form without primitive code
    if ((st = set_smem(k_path_warm<T, N, true, false>, smw))) return st;
    k_path_warm<T, N, true, false><<<gw, 128, smw, l.stream>>>(rb, w, a);
  } else {
    if ((st = set_smem(k_path_warm<T, N, false>, smw))) return st;
    k_path_warm<T, N, false><<<gw, 128, smw, l.stream>>>(rb, w, a);
  }
  if ((st = crh::check_launch("cr_solve_path exploration"))) return st;
  // refinement
  const int threads = ((a.H + 31) / 32) * 32;
  size_t smj = path_joint_smem<T>(a.no, a.np, a.H, D);
  if (a.np > 0) {
    if ((st = set_smem(k_path_joint<T, N, true>, smj))) return st;
    k_path_joint<T, N, true><<<(unsigned)a.P, threads, smj, l.stream>>>(rb, w, rbd, wd, a);
  } else if (a.no > 0) {
    if ((st = set_smem(k_path_joint<T, N, true, false>, smj))) return st;
    k_path_joint<T, N, true, false><<<(unsigned)a.P, threads, smj, l.stream>>>(rb, w, rbd, wd, a);
  } else {
    if ((st = set_smem(k_path_joint<T, N, false>, smj))) return st;
    k_path_joint<T, N, false><<<(unsigned)a.P, threads, smj, l.stream>>>(rb, w, rbd, wd, a);
  }
  return crh::check_launch("cr_solve_path refinement");
}

template <typename T> cr_status launch_path(const PathLaunch& l) {
  switch (l.robot.n) {
    case 1: return path_n<T, 1>(l);
    case 2: return path_n<T, 2>(l);
    case 3: return path_n<T, 3>(l);
    case 4: return path_n<T, 4>(l);
    case 5: return path_n<T, 5>(l);
    default: return path_n<T, 6>(l);
  }
}

#define CR_PATH_INSTANTIATE(EXT, T) EXT template cr_status launch_path<T>(const PathLaunch&);

}  // namespace crk
