// Warp-cooperative Levenberg-Marquardt pieces (Sec. IV-B, Eq. lm_step): one warp owns one state.
//
//  * The packed lower triangle of the augmented normal matrix [[A, b], [b^T, *]] ((D+1)(D+2)/2
//    entries, row D the right-hand side) is spread over the lanes: lane l holds e = l + 32 s.
//  * Residual rows are formed column-wise: lane q < D computes entry q of the row (its segment's
//    twist, its tendon), and every lane adds the products of its entries' two columns, fetched by
//    shuffles, so a row costs 2 shuffles and 1 FMA per slot and needs no shared memory.
//  * The damped system is solved by a symmetric sweep (Gauss-Jordan elimination without pivoting,
//    valid for a positive definite matrix) of the augmented matrix: D pivots, each a column
//    broadcast and one FMA per slot; the step comes out in row D.
#pragma once

#include "cr_device.cuh"

namespace crk {

template <int D> struct AugSlots {
  static constexpr int DA = (D + 1) * (D + 2) / 2;
  static constexpr int SL = (DA + 31) / 32;
  int r[SL], c[SL];  // row >= col; r == D: right-hand side; (D, D) carried but unused
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
// doubles of storage per swept block (slot-major)
template <int D> constexpr int aug_stride() { return AugSlots<D>::SL * 32; }

CR_HD float recip_fast(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}
CR_HD double recip_fast(double d) { return recip_nr(d); }

// Sweep of pivots 0..D-1 of the augmented matrix in the warp's slots. Pivot k maps d = S_kk to
// -1/d, the rest of row and column k to S_ik / d and every other entry to S_ij - S_ik S_kj / d.
// Afterwards the S block holds -S^-1 and row D holds (S^-1 b)^T. Returns false if a pivot is not
// positive. col and colr: the warp's scratch of D + 1 values (column k, and column k / d).
template <typename V, int D>
__device__ bool sweep_aug(V (&v)[AugSlots<D>::SL], const AugSlots<D>& sl, V* col, V* colr) {
  constexpr int SL = AugSlots<D>::SL;
  const int lane = threadIdx.x & 31;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int s = 0; s < SL; ++s)
      if (sl.on[s] && (sl.r[s] == k || sl.c[s] == k)) col[sl.r[s] == k ? sl.c[s] : sl.r[s]] = v[s];
    __syncwarp();
    V d = col[k];
    ok = ok && d > V(0);
    d = d > V(0) ? d : V(1);
    const V ri = recip_fast(d);
    if (lane <= D) colr[lane] = col[lane] * ri;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      if (!sl.on[s]) continue;
      const int i = sl.r[s], j = sl.c[s];
      const V upd = fma(-colr[i], col[j], v[s]);
      v[s] = (i == k) ? ((j == k) ? -ri : colr[j]) : ((j == k) ? colr[i] : upd);
    }
    __syncwarp();
  }
  return ok;
}

// Component a (tendon) of the u-space gradient of a bending gradient (gx, gy), see bend_grad_to_u.
template <typename T> CR_HD T bend_comp(T K, T gx, T gy, int a) {
  const T hx = T(0.5) * gx, ry = T(0.86602540378443864676) * gy;
  return a == 0 ? K * gx : (a == 1 ? K * (ry - hx) : K * (-ry - hx));
}

// Adds the row whose entry at this lane's column is jq (0 on lanes >= D) with residual rr.
template <typename T, int D>
__device__ void warp_row(const AugSlots<D>& sl, T (&A)[AugSlots<D>::SL], T& gq, T jq, T rr) {
#pragma unroll
  for (int s = 0; s < AugSlots<D>::SL; ++s) {
    const T a = __shfl_sync(0xffffffffu, jq, sl.r[s] < D ? sl.r[s] : 0);
    const T b = __shfl_sync(0xffffffffu, jq, sl.c[s]);
    if (sl.on[s] && sl.r[s] < D) A[s] = fma(a, b, A[s]);
  }
  gq = fma(jq, rr, gq);
}

// Full-pose IK residual of one state evaluated by a warp (every lane holds u): returns F (the same
// in every lane). NORMAL is a run-time (warp-uniform) flag, so that the LM step's two evaluations
// share one copy of this code. With NORMAL, this lane's slots of J^T J (zero in row D) and, on lane q < D, entry
// q of g = J^T r. Rows: pose (6), sum-zero per segment, active tendon bounds, active curvature
// limits, active clearance pairs (backbone samples split over the lanes).
template <typename T, int N, bool OBST>
__device__ T warp_eval(const RobotK<T>& rb, const WeightsK<T>& w, const TargetK<T>& tg, ObsK<T> ob,
                       int no, const T (&u)[3 * N], const AugSlots<3 * N>& sl, T (&A)[AugSlots<3 * N>::SL], T& gq,
                       const bool NORMAL) {
  constexpr int D = 3 * N, SL = AugSlots<D>::SL;
  const Sphere4<T>* sph = ob.s;
  const int lane = threadIdx.x & 31;
  const bool colq = lane < D;
  const int myl = colq ? lane / 3 : 0, mya = colq ? lane % 3 : 0;
  if (NORMAL) {
#pragma unroll
    for (int s = 0; s < SL; ++s) A[s] = T(0);
    gq = T(0);
  }
  Chain<T, N> ch;
  chain_forward(rb, u, ch);
  T r[6], e[3], ang, sn, cs;
  pose_rows(CR_TASK_IK6, w, tg, ch.R, ch.p, r, e, ang, sn, cs);
  T F = T(0.5) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
  // this lane's segment: twist (translational tv, angular tw for the two bending inputs), K, u
  T mtv[2][3], mtw[2][3], myK = T(0), myu = T(0), mysu = T(0);
  if (NORMAL) {
    T tv[N][2][3], tw[N][2][3];
    segment_twists(rb, ch, tv, tw);
#pragma unroll
    for (int ii = 0; ii < N; ++ii)
      if (ii == myl) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int a = 0; a < 3; ++a) { mtv[k][a] = tv[ii][k][a]; mtw[k][a] = tw[ii][k][a]; }
        myK = rb.K[ii];
        mysu = u[3 * ii] + u[3 * ii + 1] + u[3 * ii + 2];
      }
#pragma unroll
    for (int q = 0; q < D; ++q)
      if (q == lane) myu = u[q];
    // pose rows: position, then rotation through J_r^-1(e) R^T
    T be = log_beta(ang);
    T E2[3][3] = {{-(e[1] * e[1] + e[2] * e[2]), e[0] * e[1], e[0] * e[2]},
                  {e[0] * e[1], -(e[0] * e[0] + e[2] * e[2]), e[1] * e[2]},
                  {e[0] * e[2], e[1] * e[2], -(e[0] * e[0] + e[1] * e[1])}};
    T Jr[3][3] = {{T(1) + be * E2[0][0], T(-0.5) * e[2] + be * E2[0][1], T(0.5) * e[1] + be * E2[0][2]},
                  {T(0.5) * e[2] + be * E2[1][0], T(1) + be * E2[1][1], T(-0.5) * e[0] + be * E2[1][2]},
                  {T(-0.5) * e[1] + be * E2[2][0], T(0.5) * e[0] + be * E2[2][1], T(1) + be * E2[2][2]}};
    T jp[2][3];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      T wpv[3];
      cross(mtw[k], ch.p, wpv);
#pragma unroll
      for (int a = 0; a < 3; ++a) jp[k][a] = mtv[k][a] + wpv[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T jq = colq ? bend_comp(myK, w.wp * jp[0][a], w.wp * jp[1][a], mya) : T(0);
      warp_row<T, D>(sl, A, gq, jq, r[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T Mr[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) Mr[b] = Jr[a][0] * ch.R[3 * b] + Jr[a][1] * ch.R[3 * b + 1] + Jr[a][2] * ch.R[3 * b + 2];
      T g0 = w.wR * (Mr[0] * mtw[0][0] + Mr[1] * mtw[0][1] + Mr[2] * mtw[0][2]);
      T g1 = w.wR * (Mr[0] * mtw[1][0] + Mr[1] * mtw[1][1] + Mr[2] * mtw[1][2]);
      T jq = colq ? bend_comp(myK, g0, g1, mya) : T(0);
      warp_row<T, D>(sl, A, gq, jq, r[3 + a]);
    }
  }
  // sum-zero rows (segment block of ones), tendon bounds (single-entry rows)
  unsigned vmask = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T su = u[3 * i] + u[3 * i + 1] + u[3 * i + 2];
    F += T(0.5) * w.rho_eq * su * su;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int q = 3 * i + a;
      T hi = u[q] - rb.umax[i], lo = -rb.umax[i] - u[q];
      if (hi > T(0)) { F += T(0.5) * w.rho_b * hi * hi; vmask |= 1u << q; }
      if (lo > T(0)) { F += T(0.5) * w.rho_b * lo * lo; vmask |= 1u << q; }
    }
  }
  if (NORMAL) {
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int i = sl.r[s], j = sl.c[s];
      if (sl.on[s] && i < D) {
        if (i / 3 == j / 3) A[s] += w.rho_eq;
        if (i == j && ((vmask >> i) & 1u)) A[s] += w.rho_b;
      }
    }
    if (colq) {
      gq += w.rho_eq * mysu;
      T mymax = T(0);
#pragma unroll
      for (int ii = 0; ii < N; ++ii)
        if (ii == myl) mymax = rb.umax[ii];
      T hi = myu - mymax, lo = -mymax - myu;
      if (hi > T(0)) gq += w.rho_b * hi;
      if (lo > T(0)) gq -= w.rho_b * lo;
    }
  }
  // curvature limits (segment rank-1 rows)
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (ch.x[i] > rb.thmax[i] * rb.thmax[i]) {
      T th = c_sqrt(ch.x[i]);
      T vk = th - rb.thmax[i];
      F += T(0.5) * w.rho_k * vk * vk;
      if (NORMAL) {
        const T ith = c_div(w.sk, th);
        T jq = (colq && myl == i) ? bend_comp(rb.K[i], ch.ax[i] * ith, ch.ay[i] * ith, mya) : T(0);
        warp_row<T, D>(sl, A, gq, jq, w.sk * vk);
      }
    }
  }
  // clearance rows
  T Fsplit = T(0);
  if (OBST && no > 0) {
    const T inb = c_div(T(1), T(rb.nb));
    for (int j0 = 0; j0 < no; j0 += 64) {
      uint64_t mk[N];
      warp_segment_sphere_masks(rb, ch, ob, j0, no - j0 < 64 ? no - j0 : 64, mk);
#pragma unroll
      for (int ii = 0; ii < N; ++ii) {
        if (!mk[ii]) continue;
        for (int k0 = 0; k0 < rb.nb; k0 += 32) {
          const int k = k0 + lane + 1;
          const bool mine = k <= rb.nb;
          // second level: this lane's group of kCullGroup samples, then the union over the warp
          const int kg0 = (k - 1) / kCullGroup * kCullGroup + 1;
          const int kg1 = kg0 + kCullGroup - 1 < rb.nb ? kg0 + kCullGroup - 1 : rb.nb;
          const uint64_t gml = mine ? group_sphere_mask<T, N>(rb, ch, ii, kg0, kg1, ob, j0, mk[ii]) : 0ull;
          const uint64_t um = (uint64_t)__reduce_or_sync(0xffffffffu, (unsigned)gml) |
                              ((uint64_t)__reduce_or_sync(0xffffffffu, (unsigned)(gml >> 32)) << 32);
          if (!um) continue;
          T q[3], wpt[3], s, c;
          backbone_point(ch.Rb[ii], ch.pb[ii], ch.ax[ii], ch.ay[ii], ch.x[ii], ch.L[ii], T(mine ? k : 1) * inb, q,
                         wpt, s, c);
          for (uint64_t bits = um; bits; bits &= bits - 1) {
            const int jo = j0 + __ffsll((long long)bits) - 1;
            bool act;
            T viol = T(0), nvx = T(0), nvy = T(0), nvz = T(0);
            if (ob.prims() && jo >= ob.ns) {  // a primitive: the same row with sd(x) for the centre distance
              const PrimK<T>& P = ob.p[jo - ob.ns];
              T nv[3];
              act = mine && prim_active(P, wpt, P.reach, viol, nv);
              if (act) {
                nvx = nv[0]; nvy = nv[1]; nvz = nv[2];
              } else {
                viol = T(0);
              }
            } else {
              const Sphere4<T> S = sph[jo];
              const T dx = wpt[0] - S.x, dy = wpt[1] - S.y, dz = wpt[2] - S.z;
              const T d2 = dx * dx + dy * dy + dz * dz;
              act = mine && d2 < S.reach * S.reach;
              if (act) {
                const T idist = c_rsqrt(d2);
                viol = S.reach - d2 * idist;
                nvx = dx * idist; nvy = dy * idist; nvz = dz * idist;
              }
            }
            if (act) Fsplit += T(0.5) * w.rho_c * viol * viol;
            if (!NORMAL) continue;
            unsigned m = __ballot_sync(0xffffffffu, act);
            while (m) {
              const int src = __ffs(m) - 1;
              m &= m - 1;
              const T nx = __shfl_sync(0xffffffffu, nvx, src), ny = __shfl_sync(0xffffffffu, nvy, src),
                      nz = __shfl_sync(0xffffffffu, nvz, src);
              const T rr = w.sc * __shfl_sync(0xffffffffu, viol, src);
              const T px = __shfl_sync(0xffffffffu, wpt[0], src), py = __shfl_sync(0xffffffffu, wpt[1], src),
                      pz = __shfl_sync(0xffffffffu, wpt[2], src);
              const int ks = k0 + src + 1;
              T ga0 = T(0), ga1 = T(0);
              if (colq && myl < ii) {
                const T pw[3] = {px, py, pz};
                T wx0[3], wx1[3];
                cross(mtw[0], pw, wx0);
                cross(mtw[1], pw, wx1);
                ga0 = -w.sc * (nx * (mtv[0][0] + wx0[0]) + ny * (mtv[0][1] + wx0[1]) + nz * (mtv[0][2] + wx0[2]));
                ga1 = -w.sc * (nx * (mtv[1][0] + wx1[0]) + ny * (mtv[1][1] + wx1[1]) + nz * (mtv[1][2] + wx1[2]));
              } else if (colq && myl == ii) {
                const T sgk = T(ks) * inb;
                T ss, cc, s3, cp;
                seg_sc(sgk * sgk * ch.x[ii], ss, cc);
                seg_deriv(sgk * sgk * ch.x[ii], ss, cc, s3, cp);
                T dd[2][3], wl[2][3];
                seg_local_derivs(sgk * ch.ax[ii], sgk * ch.ay[ii], ss, cc, s3, cp, sgk * ch.L[ii], dd, wl);
                const T nh[3] = {nx, ny, nz};
                T nl[3];
                matTvec(ch.Rb[ii], nh, nl);
                ga0 = -w.sc * sgk * (nl[0] * dd[0][0] + nl[1] * dd[0][1] + nl[2] * dd[0][2]);
                ga1 = -w.sc * sgk * (nl[0] * dd[1][0] + nl[1] * dd[1][1] + nl[2] * dd[1][2]);
              }
              const T jq = (colq && myl <= ii) ? bend_comp(myK, ga0, ga1, mya) : T(0);
              warp_row<T, D>(sl, A, gq, jq, rr);
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) Fsplit += __shfl_xor_sync(0xffffffffu, Fsplit, off);
  return F + Fsplit;
}

// One damped LM step of the warp's state (Nielsen's lambda update, strict-decrease acceptance).
// The residual, J^T J and the costs are in the bulk precision T; the damped system is solved, and
// the gain ratio formed, in V (T for exploration, double for a refinement). Returns the cost after
// the step. The warp's scratch: col, colr, sx, sdg (D + 1 values of V each).
template <typename T, int N, bool OBST, typename V = T>
__device__ T warp_lm_step(const RobotK<T>& rb, const WeightsK<T>& w, const TargetK<T>& tg, ObsK<T> sph,
                          int no, T (&u)[3 * N], const AugSlots<3 * N>& sl, V& lam, V& nu, V* col, V* colr, V* sx,
                          V* sdg) {
  constexpr int D = 3 * N, SL = AugSlots<D>::SL;
  const int lane = threadIdx.x & 31;
  T A[SL], gq;
  T ue[D];  // the point evaluated: u (pass 0, with the normal equations), then the trial u + step
#pragma unroll
  for (int q = 0; q < D; ++q) ue[q] = u[q];
  T F = T(0), Fn = T(0);
  V pred = V(0);
  // One evaluation site for both passes (a loop that is not unrolled): the kernel carries one copy
  // of the residual code, half the instruction footprint of two inlined evaluations.
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const T Fe = warp_eval<T, N, OBST>(rb, w, tg, sph, no, ue, sl, A, gq, pass == 0);
    if (pass == 1) {
      Fn = Fe;
      break;
    }
    F = Fe;
    // damped, augmented system [A + lam D | -g]
    V Av[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int i = sl.r[s], j = sl.c[s];
      const T gj = __shfl_sync(0xffffffffu, gq, j < D ? j : 0);
      Av[s] = V(A[s]);
      if (!sl.on[s]) continue;
      if (i < D && i == j) {
        const V dg = c_max(Av[s], V(1e-12));
        sdg[i] = dg;
        Av[s] += lam * dg;
      } else if (i == D) {
        Av[s] = j < D ? -V(gj) : V(0);
      }
    }
    const bool ok = sweep_aug<V, D>(Av, sl, col, colr);
    if (!ok) {
      lam *= nu;
      nu *= V(2);
      return F;
    }
#pragma unroll
    for (int s = 0; s < SL; ++s)
      if (sl.on[s] && sl.r[s] == D && sl.c[s] < D) sx[sl.c[s]] = Av[s];
    __syncwarp();
    V predl = V(0);
    if (lane < D) {
      const V xq = sx[lane];
      predl = xq * (lam * sdg[lane] * xq - V(gq));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) predl += __shfl_xor_sync(0xffffffffu, predl, off);
    pred = V(0.5) * predl;
#pragma unroll
    for (int q = 0; q < D; ++q) ue[q] = u[q] + T(sx[q]);
    __syncwarp();
  }
  if (Fn < F) {
    const V rho = c_div(V(F) - V(Fn), pred), tt = V(2) * rho - V(1);
    lam *= c_max(V(1) / V(3), V(1) - tt * tt * tt);
    nu = V(2);
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = ue[q];
    return Fn;
  }
  lam *= nu;
  nu *= V(2);
  return F;
}

}  // namespace crk
