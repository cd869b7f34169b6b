// Path following (Sec. IV-A, Eq. constrained_mp; Sec. IV-B): IK at the first waypoint, then the
// exploration sweep (waypoint t starts from the solution of t-1 and runs k_warm LM iterations on
// its own IK residual), then the refinement: joint LM over all H waypoints with the successive-
// state smoothness rows sqrt(w_s)(u_t - u_{t-1}), whose normal matrix is block tridiagonal.
//
//  k_path_warm  : one warp per path. Every lane holds the path's state and evaluates the
//                 kinematics (identical in all lanes); the backbone samples are split over the
//                 lanes for the clearance rows. Lane l owns entries l, l+32, l+64 of the packed
//                 normal matrix; lane 0 factorises it (bulk precision: this is exploration).
//  k_path_joint : one CTA per path. Thread t evaluates waypoint t's rows and its block of J^T J;
//                 the FP64 block Cholesky over t (S_t = A_t - w_s^2 S_{t-1}^-1, forward and back
//                 substitution) spreads each 12x12 step over the CTA.
#pragma once

#include "cr_traj_impl.cuh"

namespace crk {

template <typename T> struct PathArgs {
  const double* wp;       // [7][P*H]
  int64_t P;
  int H;
  const double* spheres;  // [P][no][4] when sph_pp, else [no][4]
  int no;
  int sph_pp;
  int k_warm, k_joint;
  double lambda0, lim_tol;
  T w_s;
  const double* u0;       // [D][P]   first waypoint (IK result)
  T* X;                   // [D][P*H] working states (bulk precision)
  double* Z;              // [P][H][D*D] block inverses of the joint solve
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
// Entries of the packed normal matrix owned by this lane: lane, lane + 32, lane + 64.
struct Owned {
  int r[3], c[3];
  bool on[3];
};
template <int D> CR_HD Owned owned_entries(int lane) {
  Owned o;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    int e = lane + 32 * s;
    o.on[s] = e < D * (D + 1) / 2;
    int a = 0;
    while (o.on[s] && (a + 1) * (a + 2) / 2 <= e) ++a;
    o.r[s] = a;
    o.c[s] = o.on[s] ? e - a * (a + 1) / 2 : 0;
  }
  return o;
}

// Adds the rank-1 update j j^T (and j r to g) to this lane's entries; the row goes through the
// warp's shared scratch sj[D] (every lane holds the same j).
template <typename T, int D>
__device__ void own_rank1(int lane, const Owned& ow, T* sj, T (&Aown)[3], T& gown, const T (&j)[D], T r) {
  __syncwarp();
#pragma unroll
  for (int q = 0; q < D; ++q)
    if (lane == q) sj[q] = j[q];
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 3; ++s)
    if (ow.on[s]) Aown[s] += sj[ow.r[s]] * sj[ow.c[s]];
  if (lane < D) gown += sj[lane] * r;
}

// F, and (when NORMAL) this lane's entries of J^T J and g, of the waypoint residual at u.
// Identical kinematics in every lane; samples lane, lane + 32, ... for the clearance rows.
template <typename T, int N, bool OBST, bool NORMAL>
__device__ T warp_waypoint_eval(const RobotK<T>& rb, const WeightsK<T>& w, const TargetK<T>& tg, const Sphere4<T>* sph,
                                int no, const T (&u)[3 * N], const Owned& ow, T* sj, T (&Aown)[3], T& gown) {
  constexpr int D = 3 * N;
  const int lane = threadIdx.x & 31;
  Aown[0] = Aown[1] = Aown[2] = T(0);
  gown = T(0);
  Chain<T, N> ch;
  chain_forward(rb, u, ch);
  T r[6], e[3], ang, sn, cs;
  pose_rows(CR_TASK_IK6, w, tg, ch.R, ch.p, r, e, ang, sn, cs);
  T Fonce = T(0.5) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
  T tv[N][2][3], tw[N][2][3];
  if (NORMAL) {
    segment_twists(rb, ch, tv, tw);
    // pose rows: position then rotation (J_r^-1(e) R^T applied to the angular part)
    T be = log_beta(ang);
    T E2[3][3] = {{-(e[1] * e[1] + e[2] * e[2]), e[0] * e[1], e[0] * e[2]},
                  {e[0] * e[1], -(e[0] * e[0] + e[2] * e[2]), e[1] * e[2]},
                  {e[0] * e[2], e[1] * e[2], -(e[0] * e[0] + e[1] * e[1])}};
    T Jr[3][3] = {{T(1) + be * E2[0][0], T(-0.5) * e[2] + be * E2[0][1], T(0.5) * e[1] + be * E2[0][2]},
                  {T(0.5) * e[2] + be * E2[1][0], T(1) + be * E2[1][1], T(-0.5) * e[0] + be * E2[1][2]},
                  {T(-0.5) * e[1] + be * E2[2][0], T(0.5) * e[0] + be * E2[2][1], T(1) + be * E2[2][2]}};
    T Mrot[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Mrot[a][b] = Jr[a][0] * ch.R[3 * b] + Jr[a][1] * ch.R[3 * b + 1] + Jr[a][2] * ch.R[3 * b + 2];
#pragma unroll
    for (int row = 0; row < 6; ++row) {
      T jr[D];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T ga[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          T wpv[3];
          cross(tw[i][k], ch.p, wpv);
          T jp[3] = {tv[i][k][0] + wpv[0], tv[i][k][1] + wpv[1], tv[i][k][2] + wpv[2]};
          if (row < 3) ga[k] = w.wp * jp[row];
          else {
            const int a = row - 3;
            ga[k] = w.wR * (Mrot[a][0] * tw[i][k][0] + Mrot[a][1] * tw[i][k][1] + Mrot[a][2] * tw[i][k][2]);
          }
        }
        bend_grad_to_u(rb.K[i], ga[0], ga[1], jr[3 * i], jr[3 * i + 1], jr[3 * i + 2]);
      }
      own_rank1<T, D>(lane, ow, sj, Aown, gown, jr, r[row]);
    }
  }
  // penalty rows on u (counted once: every lane adds its own entries, F is taken from lane 0)
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T su = u[3 * i] + u[3 * i + 1] + u[3 * i + 2];
    Fonce += T(0.5) * w.rho_eq * su * su;
    if (NORMAL) {
      T j[D];
#pragma unroll
      for (int q = 0; q < D; ++q) j[q] = (q / 3 == i) ? w.se : T(0);
      own_rank1<T, D>(lane, ow, sj, Aown, gown, j, w.se * su);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int q = 3 * i + a;
      T hi = u[q] - rb.umax[i], lo = -rb.umax[i] - u[q];
      if (hi > T(0) || lo > T(0)) {
        T v = hi > T(0) ? hi : lo, sgn = hi > T(0) ? T(1) : T(-1);
        Fonce += T(0.5) * w.rho_b * v * v;
        if (NORMAL) {
          T j[D];
#pragma unroll
          for (int qq = 0; qq < D; ++qq) j[qq] = qq == q ? sgn * w.sb : T(0);
          own_rank1<T, D>(lane, ow, sj, Aown, gown, j, w.sb * v);
        }
      }
    }
    if (ch.x[i] > rb.thmax[i] * rb.thmax[i]) {
      T th = c_sqrt(ch.x[i]);
      T vk = th - rb.thmax[i];
      Fonce += T(0.5) * w.rho_k * vk * vk;
      if (NORMAL) {
        T j[D];
#pragma unroll
        for (int q = 0; q < D; ++q) j[q] = T(0);
        bend_grad_to_u(rb.K[i], w.sk * ch.ax[i] / th, w.sk * ch.ay[i] / th, j[3 * i], j[3 * i + 1], j[3 * i + 2]);
        own_rank1<T, D>(lane, ow, sj, Aown, gown, j, w.sk * vk);
      }
    }
  }
  T Fsplit = T(0);
  if (OBST && no > 0) {
    const T inb = T(1) / T(rb.nb);
    const int ns = N * rb.nb;
    // active pairs found by each lane, processed one at a time by the whole warp
    for (int base = 0; base < ns; base += 32) {
      const int sidx = base + lane;
      const bool mine = sidx < ns;
      const int i = mine ? sidx / rb.nb : 0, k = mine ? sidx % rb.nb + 1 : 1;
      T q[3], wpt[3], s, c;
      T sg = T(k) * inb;
      if (mine) backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], rb.L[i], sg, q, wpt, s, c);
      for (int jsp = 0; jsp < no; ++jsp) {
        bool act = false;
        T dist = T(0), viol = T(0), dx = T(0), dy = T(0), dz = T(0);
        if (mine) {
          Sphere4<T> S = sph[jsp];
          dx = wpt[0] - S.x; dy = wpt[1] - S.y; dz = wpt[2] - S.z;
          T d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < S.reach * S.reach) {
            act = true;
            dist = c_sqrt(d2);
            viol = S.reach - dist;
            Fsplit += T(0.5) * w.rho_c * viol * viol;
          }
        }
        if (!NORMAL) continue;
        unsigned m = __ballot_sync(0xffffffffu, act);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          // the active lane's sample and normal, broadcast to the warp
          const int si = __shfl_sync(0xffffffffu, i, src), sk = __shfl_sync(0xffffffffu, k, src);
          T nx = __shfl_sync(0xffffffffu, dx / dist, src), ny = __shfl_sync(0xffffffffu, dy / dist, src),
            nz = __shfl_sync(0xffffffffu, dz / dist, src);
          T rr = w.sc * __shfl_sync(0xffffffffu, viol, src);
          T px = __shfl_sync(0xffffffffu, wpt[0], src), py = __shfl_sync(0xffffffffu, wpt[1], src),
            pz = __shfl_sync(0xffffffffu, wpt[2], src);
          T nh[3] = {nx, ny, nz}, pw[3] = {px, py, pz};
          T jr[D];
#pragma unroll
          for (int qq = 0; qq < D; ++qq) jr[qq] = T(0);
          const T sgk = T(sk) * inb;
#pragma unroll
          for (int l = 0; l < N; ++l) {
            if (l > si) break;
            T ga[2];
            if (l < si) {
#pragma unroll
              for (int kk = 0; kk < 2; ++kk) {
                T wx[3];
                cross(tw[l][kk], pw, wx);
                ga[kk] = -w.sc * (nh[0] * (tv[l][kk][0] + wx[0]) + nh[1] * (tv[l][kk][1] + wx[1]) +
                                  nh[2] * (tv[l][kk][2] + wx[2]));
              }
            } else {
              T ss, cc, s3, cp;
              seg_sc(sgk * sgk * ch.x[l], ss, cc);
              seg_deriv(sgk * sgk * ch.x[l], ss, cc, s3, cp);
              T dd[2][3], wl[2][3];
              seg_local_derivs(sgk * ch.ax[l], sgk * ch.ay[l], ss, cc, s3, cp, sgk * rb.L[l], dd, wl);
              T nl[3];
              matTvec(ch.Rb[l], nh, nl);
#pragma unroll
              for (int kk = 0; kk < 2; ++kk)
                ga[kk] = -w.sc * sgk * (nl[0] * dd[kk][0] + nl[1] * dd[kk][1] + nl[2] * dd[kk][2]);
            }
            bend_grad_to_u(rb.K[l], ga[0], ga[1], jr[3 * l], jr[3 * l + 1], jr[3 * l + 2]);
          }
          own_rank1<T, D>(lane, ow, sj, Aown, gown, jr, rr);
        }
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) Fsplit += __shfl_xor_sync(0xffffffffu, Fsplit, off);
  return __shfl_sync(0xffffffffu, Fonce, 0) + Fsplit;
}

template <typename T, int N, bool OBST>
__global__ void __launch_bounds__(128) k_path_warm(RobotK<T> rb, WeightsK<T> w, PathArgs<T> a) {
  constexpr int D = 3 * N, DD = D * (D + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * 4 + wid;
  Sphere4<T>* sph = reinterpret_cast<Sphere4<T>*>(smem_raw) + (size_t)wid * a.no;
  T* sA = reinterpret_cast<T*>(smem_raw + ((size_t)4 * a.no * sizeof(Sphere4<T>) + 15) / 16 * 16) +
          (size_t)wid * (DD + 3 * D + 2);
  T* sg = sA + DD;
  T* sd = sg + D;       // step [D], ok flag [D]
  T* sj = sd + D + 2;   // row scratch [D]
  const Owned ow = owned_entries<D>(lane);
  const bool live = p < a.P;
  if (OBST && live) {
    const double* sp = a.spheres + (a.sph_pp ? p * a.no * 4 : 0);
    for (int j = lane; j < a.no; j += 32) {
      Sphere4<T> s;
      s.x = T(sp[4 * j]); s.y = T(sp[4 * j + 1]); s.z = T(sp[4 * j + 2]);
      s.reach = T(sp[4 * j + 3]) + rb.rbody + w.delta;
      sph[j] = s;
    }
  }
  __syncwarp();
  if (!live) return;
  const int H = a.H;
  const int64_t PH = a.P * H;
  T u[D];
#pragma unroll
  for (int q = 0; q < D; ++q) u[q] = T(a.u0[q * a.P + p]);
  if (lane < D) a.X[lane * PH + p * H] = T(a.u0[lane * a.P + p]);
  for (int t = 1; t < H; ++t) {
    TargetK<T> tg = load_target<T>(a.wp, PH, p * H + t, CR_TASK_IK6);
    double lam = a.lambda0, nu = 2.0;
    for (int it = 0; it < a.k_warm; ++it) {
      T Aown[3], gown;
      T F = warp_waypoint_eval<T, N, OBST, true>(rb, w, tg, sph, a.no, u, ow, sj, Aown, gown);
#pragma unroll
      for (int s = 0; s < 3; ++s)
        if (lane + 32 * s < DD) sA[lane + 32 * s] = Aown[s];
      if (lane < D) sg[lane] = gown;
      __syncwarp();
      // lane 0: damped Cholesky and solve (exploration: bulk precision); sd[D] = step, sd[D+1] = ok
      if (lane == 0) {
        T Am[DD], Dg[D], x[D], inv[D];
#pragma unroll
        for (int e = 0; e < DD; ++e) Am[e] = sA[e];
#pragma unroll
        for (int q = 0; q < D; ++q) {
          Dg[q] = c_max(Am[tri(q, q)], T(1e-12));
          Am[tri(q, q)] += T(lam) * Dg[q];
        }
        bool ok = true;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          T s = Am[tri(j, j)];
#pragma unroll
          for (int k = 0; k < j; ++k) s -= Am[tri(j, k)] * Am[tri(j, k)];
          ok = ok && (s > T(0));
          s = s > T(0) ? s : T(1);
          T iv = c_rsqrt(s);
          inv[j] = iv;
          Am[tri(j, j)] = s * iv;
#pragma unroll
          for (int i = j + 1; i < D; ++i) {
            T t2 = Am[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) t2 -= Am[tri(i, k)] * Am[tri(j, k)];
            Am[tri(i, j)] = t2 * iv;
          }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
          T s = -sg[i];
#pragma unroll
          for (int k = 0; k < i; ++k) s -= Am[tri(i, k)] * x[k];
          x[i] = s * inv[i];
        }
#pragma unroll
        for (int i = D - 1; i >= 0; --i) {
          T s = x[i];
#pragma unroll
          for (int k = i + 1; k < D; ++k) s -= Am[tri(k, i)] * x[k];
          x[i] = s * inv[i];
        }
        T pred = T(0);
#pragma unroll
        for (int q = 0; q < D; ++q) {
          sd[q] = x[q];
          pred += x[q] * (T(lam) * Dg[q] * x[q] - sg[q]);
        }
        sA[0] = T(0.5) * pred;  // reuse: predicted reduction
        sd[D] = ok ? T(1) : T(0);
      }
      __syncwarp();
      const bool ok = sd[D] != T(0);
      if (!ok) {
        lam *= nu;
        nu *= 2.0;
        __syncwarp();
        continue;
      }
      T un[D];
#pragma unroll
      for (int q = 0; q < D; ++q) un[q] = u[q] + sd[q];
      const double pred = double(sA[0]);
      __syncwarp();
      T dummyA[3], dummyg;
      T Fn = warp_waypoint_eval<T, N, OBST, false>(rb, w, tg, sph, a.no, un, ow, sj, dummyA, dummyg);
      if (Fn < F) {
        double rho = (double(F) - double(Fn)) / pred, tt = 2.0 * rho - 1.0;
        lam *= fmax(1.0 / 3.0, 1.0 - tt * tt * tt);
        nu = 2.0;
#pragma unroll
        for (int q = 0; q < D; ++q) u[q] = un[q];
      } else {
        lam *= nu;
        nu *= 2.0;
      }
    }
    if (lane < D) {
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (q == lane) a.X[q * PH + p * H + t] = u[q];
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Refinement: joint LM over the path, FP64 block-tridiagonal Cholesky
// ------------------------------------------------------------------------------------------------
// Blocks: diagonal A_t (+ smoothness w_s I per neighbour, + lambda D), off-diagonal -w_s I.
// Forward: S_0 = A_0, S_t = A_t - w_s^2 S_{t-1}^-1, y_0 = -g_0, y_t = -g_t + w_s S_{t-1}^-1 y_{t-1};
// backward: x_{H-1} = S^-1 y_{H-1}, x_t = S_t^-1 (y_t + w_s x_{t+1}). Each S_t is factorised
// S_t = L L^T (Cholesky), its inverse Z_t = L^-T L^-1 kept for the Schur update and the back sweep.
template <typename T, int N, bool OBST>
__global__ void __launch_bounds__(160) k_path_joint(RobotK<T> rb, WeightsK<T> w, RobotK<double> rbd,
                                                     WeightsK<double> wd, PathArgs<T> a) {
  constexpr int D = 3 * N, DD = D * (D + 1) / 2, D2 = D * D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t p = blockIdx.x;
  const int tid = threadIdx.x, H = a.H;
  const int64_t PH = a.P * H;
  // shared layout: spheres (T, double) | A [H][DD] | g [H][D] | Dg [H][D] | y [H][D] | S [D2] | L [D2] | W [D2] | red
  size_t off = 0;
  Sphere4<T>* sph = reinterpret_cast<Sphere4<T>*>(smem_raw);
  off += (size_t)a.no * sizeof(Sphere4<T>);
  Sphere4<double>* sphd = reinterpret_cast<Sphere4<double>*>(smem_raw + off);
  off += (size_t)a.no * sizeof(Sphere4<double>);
  off = (off + 15) & ~size_t(15);
  double* A = reinterpret_cast<double*>(smem_raw + off);
  double* g = A + (size_t)H * DD;
  double* Dg = g + (size_t)H * D;
  double* y = Dg + (size_t)H * D;
  double* xs = y + (size_t)H * D;  // the step
  double* S = xs + (size_t)H * D;
  double* Lm = S + D2;
  double* Wm = Lm + D2;
  double* red = Wm + D2;        // [32]
  double* misc = red + 32;      // [8]: ok flag, F, Fn, pred
  T* ush = reinterpret_cast<T*>(misc + 8);  // [H][D] current states (for the smoothness coupling)
  double* Zg = a.Z + (size_t)p * H * D2;
  if (OBST) {
    const double* sp = a.spheres + (a.sph_pp ? p * a.no * 4 : 0);
    stage_spheres(sp, a.no, rb, w.delta, sph);
    stage_spheres(sp, a.no, rbd, wd.delta, sphd);
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
      Fl = double(eval_ik<T, N, OBST, false, false>(rb, w, CR_TASK_IK6, tg, sph, a.no, uu, dummy, nullptr, nullptr, nullptr));
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
    // 1. blocks of J^T J and J^T r of every waypoint, plus the smoothness rows
    double Fl = 0.0;
    if (wthr) {
      T At[DD], gt[D];
      Fl = double(eval_ik_normal<T, T, N, OBST>(rb, w, CR_TASK_IK6, tg, sph, a.no, u, At, gt));
#pragma unroll
      for (int e = 0; e < DD; ++e) A[tid * DD + e] = double(At[e]);
#pragma unroll
      for (int q = 0; q < D; ++q) {
        g[tid * D + q] = double(gt[q]);
        ush[tid * D + q] = u[q];
      }
    }
    __syncthreads();
    if (wthr) {
      const int nb = (tid > 0) + (tid + 1 < H);
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
        A[tid * DD + tri(q, q)] += ws * nb;
        double dg = fmax(A[tid * DD + tri(q, q)], 1e-12);
        Dg[tid * D + q] = dg;
        A[tid * DD + tri(q, q)] += lam * dg;
      }
    }
    const double F = block_sum(Fl, red);
    __syncthreads();
    // 2. forward elimination over t (FP64)
    if (tid == 0) misc[0] = 1.0;
    __syncthreads();
    for (int t = 0; t < H; ++t) {
      for (int e = tid; e < D2; e += blockDim.x) {
        const int i = e / D, j = e % D;
        double s = (i >= j) ? A[t * DD + tri(i, j)] : A[t * DD + tri(j, i)];
        if (t > 0) s -= ws * ws * Zg[(size_t)(t - 1) * D2 + e];
        S[e] = s;
      }
      __syncthreads();
      // Cholesky of S (right-looking; L in Lm, lower part)
      for (int j = 0; j < D; ++j) {
        if (tid == 0) {
          double s = S[j * D + j];
          if (!(s > 0.0)) { misc[0] = 0.0; s = 1.0; }
          double iv = rsqrt(s);
          Lm[j * D + j] = s * iv;
          misc[1] = iv;
        }
        __syncthreads();
        const double iv = misc[1];
        if (tid > j && tid < D) Lm[tid * D + j] = S[tid * D + j] * iv;
        __syncthreads();
        for (int e = tid; e < D2; e += blockDim.x) {
          const int i = e / D, k = e % D;
          if (k > j && i >= k) S[i * D + k] -= Lm[i * D + j] * Lm[k * D + j];
        }
        __syncthreads();
      }
      // W = L^-1 (columns in parallel), then Z_t = W^T W
      if (tid < D) {
        const int c = tid;
        for (int i = 0; i < D; ++i) {
          double v;
          if (i < c) v = 0.0;
          else if (i == c) v = 1.0 / Lm[c * D + c];
          else {
            double s = 0.0;
            for (int k = c; k < i; ++k) s += Lm[i * D + k] * Wm[k * D + c];
            v = -s / Lm[i * D + i];
          }
          Wm[i * D + c] = v;
        }
      }
      __syncthreads();
      for (int e = tid; e < D2; e += blockDim.x) {
        const int i = e / D, j = e % D;
        double s = 0.0;
        for (int k = (i > j ? i : j); k < D; ++k) s += Wm[k * D + i] * Wm[k * D + j];
        Zg[(size_t)t * D2 + e] = s;
      }
      // y_t = -g_t + w_s Z_{t-1} y_{t-1}
      if (tid < D) {
        double s = -g[t * D + tid];
        if (t > 0)
          for (int k = 0; k < D; ++k) s += ws * Zg[(size_t)(t - 1) * D2 + tid * D + k] * y[(t - 1) * D + k];
        y[t * D + tid] = s;
      }
      __syncthreads();
    }
    const bool ok = misc[0] != 0.0;
    // 3. back substitution: x_{H-1} = Z y_{H-1}; x_t = Z_t (y_t + w_s x_{t+1})
    if (!ok) {
      lam *= nu;
      nu *= 2.0;
      continue;
    }
    for (int t = H - 1; t >= 0; --t) {
      if (tid < D) {
        double xt = 0.0;
        for (int k = 0; k < D; ++k) {
          double rhs = y[t * D + k] + (t + 1 < H ? ws * xs[(t + 1) * D + k] : 0.0);
          xt += Zg[(size_t)t * D2 + tid * D + k] * rhs;
        }
        xs[t * D + tid] = xt;
      }
      __syncthreads();
    }
    // 4. trial, gain ratio 1/2 x^T (lambda D x - g), accept
    T un[D];
    double predl = 0.0;
#pragma unroll
    for (int q = 0; q < D; ++q) un[q] = wthr ? u[q] + T(xs[tid * D + q]) : u[q];
    if (wthr) {
#pragma unroll
      for (int q = 0; q < D; ++q) {
        double xq = xs[tid * D + q];
        predl += xq * (lam * Dg[tid * D + q] * xq - g[tid * D + q]);
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
    accept_fp64<N, OBST>(rbd, wd, CR_TASK_IK6, tgd, sphd, a.no, ud, a.lim_tol, pos, rot, flags);
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
  a.sph_pp = (l.scene.per_problem && l.scene.n_o > 0) ? 1 : 0;
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

inline size_t path_joint_smem(int no, int H, int D, size_t tsize) {
  size_t off = (size_t)no * (4 * tsize + 32);
  off = (off + 15) & ~size_t(15);
  off += sizeof(double) * ((size_t)H * (D * (D + 1) / 2 + 4 * D) + 3 * (size_t)D * D + 32 + 8);
  off += tsize * (size_t)H * D;
  return off;
}

template <typename T, int N> cr_status path_n(const PathLaunch& l) {
  constexpr int D = 3 * N, DD = D * (D + 1) / 2;
  RobotK<T> rb = crh::robot_k<T>(l.robot);
  WeightsK<T> w = crh::weights_k<T>(l.w);
  RobotK<double> rbd = crh::robot_k<double>(l.robot);
  WeightsK<double> wd = crh::weights_k<double>(l.w);
  PathArgs<T> a = path_args<T>(l);
  cr_status st;
  // exploration sweep
  size_t smw = (((size_t)4 * a.no * sizeof(Sphere4<T>) + 15) / 16 * 16) + (size_t)4 * (DD + 3 * D + 2) * sizeof(T);
  unsigned gw = (unsigned)((a.P + 3) / 4);
  if (a.no > 0) {
    if ((st = set_smem(k_path_warm<T, N, true>, smw))) return st;
    k_path_warm<T, N, true><<<gw, 128, smw, l.stream>>>(rb, w, a);
  } else {
    if ((st = set_smem(k_path_warm<T, N, false>, smw))) return st;
    k_path_warm<T, N, false><<<gw, 128, smw, l.stream>>>(rb, w, a);
  }
  if ((st = crh::check_launch("cr_solve_path exploration"))) return st;
  // refinement
  const int threads = a.H <= 128 ? 160 : ((a.H + 31) / 32) * 32;
  size_t smj = path_joint_smem(a.no, a.H, D, sizeof(T));
  if (a.no > 0) {
    if ((st = set_smem(k_path_joint<T, N, true>, smj))) return st;
    k_path_joint<T, N, true><<<(unsigned)a.P, threads, smj, l.stream>>>(rb, w, rbd, wd, a);
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
