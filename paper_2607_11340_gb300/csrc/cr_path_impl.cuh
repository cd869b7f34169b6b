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
//                 one warp runs the FP64 block elimination over t (S_t = M_t - w_s^2 S_{t-1}^-1,
//                 forward and back substitution), each block inverted by a symmetric sweep whose
//                 packed entries are spread over the 32 lanes, so a block step needs no CTA barrier.
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
    for (int j0 = 0; j0 < no; j0 += 64) {
    uint64_t mk[N];
    warp_segment_sphere_masks(rb, ch, sph, j0, no - j0 < 64 ? no - j0 : 64, mk);
    // active pairs found by each lane, processed one at a time by the whole warp
    for (int base = 0; base < ns; base += 32) {
      const int sidx = base + lane;
      const bool mine = sidx < ns;
      const int i = mine ? sidx / rb.nb : 0, k = mine ? sidx % rb.nb + 1 : 1;
      // candidate spheres of the segments these 32 samples belong to (the same in every lane)
      const int i_lo = base / rb.nb, i_hi = (base + 31 < ns ? base + 31 : ns - 1) / rb.nb;
      uint64_t um = 0;
#pragma unroll
      for (int ii = 0; ii < N; ++ii)
        if (ii >= i_lo && ii <= i_hi) um |= mk[ii];
      if (!um) continue;
      T q[3], wpt[3], s, c;
      T sg = T(k) * inb;
      if (mine) backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], rb.L[i], sg, q, wpt, s, c);
      for (uint64_t bits = um; bits; bits &= bits - 1) {
        const int jsp = j0 + __ffsll((long long)bits) - 1;
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
// Refinement: joint LM over the path, FP64 block-tridiagonal elimination
// ------------------------------------------------------------------------------------------------
// Entries of the augmented (D+1)x(D+1) packed lower triangle [[S, b], [b^T, *]] owned by a lane of
// the solving warp: e = lane + 32 s. Row D is the right-hand side; (D, D) is carried but unused.
template <int D> struct AugSlots {
  static constexpr int DA = (D + 1) * (D + 2) / 2;
  static constexpr int SL = (DA + 31) / 32;
  int r[SL], c[SL];
  bool on[SL];
};
template <int D> __device__ AugSlots<D> aug_slots(int lane) {
  AugSlots<D> o;
#pragma unroll
  for (int s = 0; s < AugSlots<D>::SL; ++s) {
    const int e = lane + 32 * s;
    o.on[s] = e < AugSlots<D>::DA;
    int a = 0;
    while (o.on[s] && (a + 1) * (a + 2) / 2 <= e) ++a;
    o.r[s] = a;
    o.c[s] = o.on[s] ? e - a * (a + 1) / 2 : 0;
  }
  return o;
}
// doubles of Z storage per block (the swept slots of one block, slot-major)
template <int D> constexpr int aug_stride() { return AugSlots<D>::SL * 32; }

// Symmetric sweep (Gauss-Jordan elimination without pivoting, valid for a positive definite S) of
// pivots 0..D-1 of the augmented matrix held in the warp's slots. Pivot k maps d = S_kk to -1/d, the
// rest of row and column k to S_ik / d and every other entry to S_ij - S_ik S_kj / d. Afterwards the
// S block holds -S^-1 and row D holds (S^-1 b)^T. Returns false if a pivot is not positive. col and
// colr are the warp's scratch of D + 1 doubles: column k, and column k scaled by 1/d.
template <int D>
__device__ bool sweep_aug(double (&v)[AugSlots<D>::SL], const AugSlots<D>& sl, double* col, double* colr) {
  constexpr int SL = AugSlots<D>::SL;
  const int lane = threadIdx.x & 31;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int s = 0; s < SL; ++s)
      if (sl.on[s] && (sl.r[s] == k || sl.c[s] == k)) col[sl.r[s] == k ? sl.c[s] : sl.r[s]] = v[s];
    __syncwarp();
    double d = col[k];
    ok = ok && d > 0.0;
    d = d > 0.0 ? d : 1.0;
    const double ri = recip_nr(d);
    if (lane <= D) colr[lane] = col[lane] * ri;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      if (!sl.on[s]) continue;
      const int i = sl.r[s], j = sl.c[s];
      const double upd = fma(-colr[i], col[j], v[s]);
      v[s] = (i == k) ? ((j == k) ? -ri : colr[j]) : ((j == k) ? colr[i] : upd);
    }
    __syncwarp();
  }
  return ok;
}

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
    ok = sweep_aug<D>(v, sl, col, colr) && ok;
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

// One CTA per path, one thread per waypoint (blockDim = H rounded up to a warp). Per iteration:
// every thread forms its waypoint's J^T J block and gradient (bulk precision) plus the smoothness
// terms; warp 0 solves the block system in FP64; all threads evaluate the trial path.
template <typename T, int N, bool OBST>
__global__ void __launch_bounds__(128) k_path_joint(RobotK<T> rb, WeightsK<T> w, RobotK<double> rbd,
                                                     WeightsK<double> wd, PathArgs<T> a) {
  constexpr int D = 3 * N, DD = D * (D + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t p = blockIdx.x;
  const int tid = threadIdx.x, H = a.H;
  const int64_t PH = a.P * H;
  // shared layout: spheres (T, double) | g [H][D] | z [H][D] | col, colr [32] | Zs [DD] | red [32] |
  // misc [8] | Af [H][DD] (T) | ush [H][D] (T)
  size_t off = 0;
  Sphere4<T>* sph = reinterpret_cast<Sphere4<T>*>(smem_raw);
  off += (size_t)a.no * sizeof(Sphere4<T>);
  Sphere4<double>* sphd = reinterpret_cast<Sphere4<double>*>(smem_raw + off);
  off += (size_t)a.no * sizeof(Sphere4<double>);
  off = (off + 15) & ~size_t(15);
  double* g = reinterpret_cast<double*>(smem_raw + off);
  double* z = g + (size_t)H * D;
  double* col = z + (size_t)H * D;
  double* colr = col + 32;
  double* Zs = colr + 32;
  double* red = Zs + DD;
  double* misc = red + 32;  // [8]: ok flag
  T* Af = reinterpret_cast<T*>(misc + 8);
  T* ush = Af + (size_t)H * DD;
  double* Zg = a.Z + (size_t)p * H * aug_stride<D>();
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
    // 1. J^T J block and J^T r of every waypoint, plus the smoothness rows' gradient
    double Fl = 0.0;
    if (wthr) {
      T At[DD], gt[D];
      Fl = double(eval_ik_normal<T, T, N, OBST>(rb, w, CR_TASK_IK6, tg, sph, a.no, u, At, gt));
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
    // 2. FP64 block elimination (warp 0)
    if (tid < 32) {
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
  off += sizeof(double) * ((size_t)2 * H * D + 64 + (size_t)D * (D + 1) / 2 + 32 + 8);
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
  const int threads = ((a.H + 31) / 32) * 32;
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
