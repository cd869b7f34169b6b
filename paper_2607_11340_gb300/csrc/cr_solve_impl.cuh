// Kernels of Algorithm 1 (beam-search IK) and of the standalone solver steps.
//
//  k_ik_stage1 : one CTA per target, one thread per seed. SampleSeeds (counter-based), k_init
//                projected-gradient steps with the state in registers, then SelectTop by warp 0
//                with warp shuffles over the CTA's candidates staged in shared memory.
//  k_ik_refine : one thread per selected candidate: k_final LM iterations (J, r and J^T J in the
//                bulk precision; Cholesky, solve and gain ratio in FP64), then the FP64
//                re-evaluation of cost, pose error, limits and clearance.
//  k_ik_argmin : one thread per target: argmin of the FP64 cost over its candidates (costs at the
//                rounding level, <= CR_ARGMIN_TIE, tie and the first in SelectTop order wins).
#pragma once

#include <limits.h>

#include "cr_host.h"
#include "cr_warp.cuh"

namespace crk {

// ------------------------------------------------------------------------------------------------
// One projected-gradient step (stage one): trial u' = Pi(u - alpha g / |g|); accept iff F(u') < F(u).
// Returns 1 if the step was accepted.
// The trial point is feasible, so its bound and sum-zero rows are zero: the FP32 form leaves them out
// (in FP32 the sum-zero row would only contribute the projection's rounding residue); the FP64 form
// evaluates them, term by term like the FP64 definition.
// ------------------------------------------------------------------------------------------------
// first = true evaluates u itself (the seed: cost, gradient and clearance part), takes it and counts
// no step; the seed lies on the feasible set like every trial point.
template <typename T, int N, bool OBST, int MODEL = CR_MODEL_TENDON>
CR_HD int pg_step(const RobotK<T>& rb, const WeightsK<T>& w, int kind, const TargetK<T>& tg,
                   ObsK<T> sph, int no, T (&u)[3 * N], T (&g)[3 * N], T& F, T& coll, T& alpha,
                   bool first = false) {
  constexpr int D = 3 * N;
  T u1[D];
  if (first) {
#pragma unroll
    for (int q = 0; q < D; ++q) u1[q] = u[q];
  } else {
    T gn2 = T(0);
#pragma unroll
    for (int q = 0; q < D; ++q) gn2 += g[q] * g[q];
    T scale = gn2 > T(0) ? alpha * c_rsqrt(gn2) : T(0);
    T v[D];
#pragma unroll
    for (int q = 0; q < D; ++q) v[q] = u[q] - scale * g[q];
    project_state<MODEL, T, N>(rb, v, u1);
  }
  T g1[D], c1;
  T F1 = eval_ik<T, N, OBST, true, false, (sizeof(T) == 8), MODEL>(rb, w, kind, tg, sph, no, u1, g1, nullptr, nullptr,
                                                                   &c1);
  if (first || F1 < F) {
#pragma unroll
    for (int q = 0; q < D; ++q) { u[q] = u1[q]; g[q] = g1[q]; }
    F = F1;
    coll = c1;
    if (first) return 0;
    alpha *= T(1.25);
    return 1;
  }
  alpha *= T(0.5);
  return 0;
}

// ------------------------------------------------------------------------------------------------
// One Levenberg-Marquardt iteration (Sec. IV-C); returns 1 if the step was accepted.
// ------------------------------------------------------------------------------------------------
template <typename T, int N, bool OBST, int MODEL = CR_MODEL_TENDON>
CR_HD int lm_iteration(const RobotK<T>& rb, const WeightsK<T>& w, int kind, const TargetK<T>& tg,
                       ObsK<T> sph, int no, T (&u)[3 * N], double& lam, double& nu, T& Fout) {
  constexpr int D = 3 * N;
  constexpr int DD = D * (D + 1) / 2;
  double Ad[DD], Dg[D], dl[D], invd[D];
  T F;
  {
    // FP32 bulk: J^T J and J^T r accumulated exactly in two-float pairs (NormalAcc, F2)
    typedef typename NormalAcc<T>::type TA;
    TA A[DD], g[D];
    F = eval_ik_normal<T, TA, N, OBST, MODEL>(rb, w, kind, tg, sph, no, u, A, g);
#pragma unroll
    for (int a = 0; a < DD; ++a) Ad[a] = to_f64(A[a]);
#pragma unroll
    for (int q = 0; q < D; ++q) dl[q] = to_f64(g[q]);
  }
#pragma unroll
  for (int q = 0; q < D; ++q) {
    Dg[q] = fmax(Ad[tri(q, q)], 1e-12);
    Ad[tri(q, q)] += lam * Dg[q];
  }
  if (!cholesky_packed<D>(Ad, invd)) {
    lam *= nu;
    nu *= 2.0;
    Fout = F;
    return 0;
  }
  double gd[D];
#pragma unroll
  for (int q = 0; q < D; ++q) { gd[q] = dl[q]; dl[q] = -dl[q]; }
  cholesky_solve<D>(Ad, invd, dl);
  T un[D];
#pragma unroll
  for (int q = 0; q < D; ++q) un[q] = u[q] + T(dl[q]);
  T dummy[D];
  T Fn = eval_ik<T, N, OBST, false, false, true, MODEL>(rb, w, kind, tg, sph, no, un, dummy, nullptr, nullptr,
                                                       nullptr);
  double pred = 0.0;
#pragma unroll
  for (int q = 0; q < D; ++q) pred += dl[q] * (lam * Dg[q] * dl[q] - gd[q]);
  pred *= 0.5;
  if (Fn < F) {
    double rho = (double(F) - double(Fn)) / pred;
    double t = 2.0 * rho - 1.0;
    lam *= fmax(1.0 / 3.0, 1.0 - t * t * t);
    nu = 2.0;
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = un[q];
    Fout = Fn;
    return 1;
  }
  lam *= nu;
  nu *= 2.0;
  Fout = F;
  return 0;
}

// ------------------------------------------------------------------------------------------------
// SelectTop by one warp: rank (cost, coll, index) ascending with non-finite keys last, skip
// candidates within eps (max-norm) of a kept one, then fill up with the skipped ones in rank order.
// u of candidate i, component q is at u[q * ustride + i].
// ------------------------------------------------------------------------------------------------
CR_HD bool key_less(float c1, float l1, int i1, float c2, float l2, int i2) {
  if (c1 != c2) return c1 < c2;
  if (l1 != l2) return l1 < l2;
  return i1 < i2;
}

// Greedy selection with near-duplicate marking: each round keeps the best available candidate w
// and, in parallel over the lanes, marks every available candidate within eps of w as a duplicate.
// A candidate ranked below w meets w (already kept) when its turn comes in the sequential rule, so
// the kept set and order are those of the sequential rule, with at most K rounds. If fewer than K
// survive, the marked candidates fill the rest in rank order. taken: 0 available, 1 kept, 2 marked.
// Loads that bypass L1 (ld.global.cg) for candidates written by other SMs in the same launch.
template <bool CG, typename V> __device__ __forceinline__ V cand_ld(const V* p) {
  if (CG) return __ldcg(p);
  return *p;
}

template <typename T, bool CG = false>
__device__ void warp_topk(const float* cost, const float* coll, const T* u, int64_t ustride, int D, int S,
                          int K, T eps, int* sel, unsigned char* taken, int* /*unused*/) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < S; i += 32) taken[i] = 0;
  __syncwarp();
  int kept = 0;
  for (int pass = 0; pass < 2 && kept < K; ++pass) {
    const unsigned char want = pass == 0 ? 0 : 2;  // pass 0: available; pass 1: fill from marked
    while (kept < K) {
      float bc = INFINITY, bl = INFINITY;
      int bi = INT_MAX;
      for (int i = lane; i < S; i += 32) {
        if (taken[i] != want) continue;
        float c = cand_ld<CG>(cost + i), l = cand_ld<CG>(coll + i);
        c = isfinite(c) ? c : INFINITY;
        l = isfinite(l) ? l : INFINITY;
        if (key_less(c, l, i, bc, bl, bi)) { bc = c; bl = l; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        float oc = __shfl_xor_sync(FULL, bc, off);
        float ol = __shfl_xor_sync(FULL, bl, off);
        int oi = __shfl_xor_sync(FULL, bi, off);
        if (key_less(oc, ol, oi, bc, bl, bi)) { bc = oc; bl = ol; bi = oi; }
      }
      if (bi == INT_MAX) break;
      if (lane == 0) { sel[kept] = bi; taken[bi] = 1; }
      ++kept;
      __syncwarp();
      if (pass == 0) {
        for (int i = lane; i < S; i += 32) {
          if (taken[i] != 0) continue;
          T m = T(0);
          for (int q = 0; q < D; ++q)
            m = c_max(m, c_fabs(cand_ld<CG>(u + q * ustride + i) - cand_ld<CG>(u + q * ustride + bi)));
          if (m < eps) taken[i] = 2;
        }
        __syncwarp();
      }
    }
  }
  for (int k = kept; k < K; ++k)
    if (lane == 0) sel[k] = -1;
  __syncwarp();
}

// ------------------------------------------------------------------------------------------------
// Kernel parameters
// ------------------------------------------------------------------------------------------------
template <typename T> struct IkArgs {
  int kind;
  const double* targets;
  int64_t P;
  const double* spheres;
  int no;
  const double* prims;  // primitive records [np][CR_PRIM_DOUBLES] (per problem: [P][np][..])
  int np;
  int sph_pp;  // obstacles are per problem: spheres [P][no][4], primitives [P][np][CR_PRIM_DOUBLES]
  int tpb;     // per-problem obstacles: targets per refine block (their obstacle sets staged side by side)
  int S, K, k_init, k_final;
  T alpha0, eps;
  double lambda0, lim_tol, pos_tol, rot_tol;
  SeedBox box;        // seed bounds (FP64)
  uint64_t seed;
  int64_t p0;
  T* cand_u;          // [D][P*K] bulk precision
  double* cand_u64;   // [D][P*K]
  double* cand_F;     // [P*K]
  double* cand_pos;
  double* cand_rot;
  unsigned char* cand_flag;
  double* u_out;      // [D][P]
  double* cost_out;
  double* pos_out;
  double* rot_out;
  unsigned char* success;
  int* status;
  unsigned long long* pg_accepted;  // stage one adds its accepted steps here (the workspace counter)
};

// Stage one writes every seed's end state, cost and clearance part, [D][P*S] / [P*S]; SelectTop reads
// them back in a kernel of its own, so that no warp of the stage-one blocks waits on it.
template <typename T> struct StageOut {
  float* F;
  float* C;
  T* u;
};

// Stage the obstacle set of problem p (set 0 of a shared scene) at base, in precision T (PRIMS:
// stage_obstacles_as).
template <bool PRIMS = true, typename T, typename A>
__device__ ObsK<T> stage_problem_obstacles(const A& a, int64_t p, const RobotK<T>& rb, T delta, unsigned char* base) {
  const int64_t q = a.sph_pp ? p : 0;
  return stage_obstacles_as<PRIMS>(a.spheres + q * a.no * 4, a.no,
                                   a.np > 0 ? a.prims + q * a.np * CR_PRIM_DOUBLES : nullptr, a.np, rb, delta, base);
}

// Bytes of one staged obstacle set in FP64 and in T, side by side (the refine kernels').
template <typename T> __host__ __device__ inline size_t refine_set_bytes(int no, int np) {
  return ((obstacles_smem<double>(no, np) + 15) & ~(size_t)15) + ((obstacles_smem<T>(no, np) + 15) & ~(size_t)15);
}

template <typename T, int N, bool OBST, int MODEL = CR_MODEL_TENDON, bool PRIMS = true>
__global__ void __launch_bounds__(256) k_ik_stage1(RobotK<T> rb, WeightsK<T> w, IkArgs<T> a, StageOut<T> so) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = a.S;
  const int64_t p = blockIdx.x;
  const int nob = a.no + a.np;
  ObsK<T> sph(nullptr);
  if (OBST) {
    sph = stage_problem_obstacles<PRIMS>(a, p, rb, w.delta, smem_raw);
    __syncthreads();
  }
  const int s = threadIdx.x;
  int acc = 0;  // accepted steps of this seed
  if (s < S) {
    TargetK<T> tg = load_target<T>(a.targets, a.P, p, a.kind);
    T u[D], g[D], coll = T(0);
    draw_seed_m<MODEL, T, N>(a.seed, (uint64_t)(a.p0 + p), (uint64_t)s, 0, a.box, u);
    if (OBST && nob > 0) {
      for (int att = 1; att < 8; ++att) {
        if (!state_collides<T, N, MODEL>(rb, sph, nob, u)) break;
        draw_seed_m<MODEL, T, N>(a.seed, (uint64_t)(a.p0 + p), (uint64_t)s, att, a.box, u);
      }
    }
#pragma unroll
    for (int q = 0; q < D; ++q) g[q] = T(0);
    T F = T(0), alpha = a.alpha0;
    // it = -1 evaluates the seed itself (no step, always taken); it >= 0 are the projected-gradient
    // steps. One evaluation site for both keeps the kernel's code half as long.
    for (int it = -1; it < a.k_init; ++it)
      acc += pg_step<T, N, OBST, MODEL>(rb, w, a.kind, tg, sph, nob, u, g, F, coll, alpha, it < 0);
    const int64_t i = p * S + s;
    so.F[i] = float(F);
    so.C[i] = float(coll);
    const int64_t PS = a.P * S;
#pragma unroll
    for (int q = 0; q < D; ++q) so.u[q * PS + i] = u[q];
  }
  // accepted steps: one atomic per warp (every lane of the block is here: blockDim is a multiple of 32)
  acc = __reduce_add_sync(0xffffffffu, acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(a.pg_accepted, (unsigned long long)acc);
}

// SelectTop of Algorithm 1 over stage one's end states: one warp per target, its S candidates staged
// in shared memory (coalesced loads), then warp_topk; writes the K kept states (NaN for empty slots).
template <typename T> struct SelectSmem {
  __host__ __device__ static size_t per_warp(int S, int D) {
    size_t b = (size_t)D * S * sizeof(T) + (size_t)S * 2 * sizeof(float) + 32 * sizeof(int) + S;
    return (b + 15) & ~size_t(15);
  }
};

template <typename T>
__global__ void __launch_bounds__(256) k_ik_select(IkArgs<T> a, StageOut<T> so, int D) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = a.S, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
  if (p >= a.P) return;
  unsigned char* mine = smem_raw + (size_t)wid * SelectSmem<T>::per_warp(S, D);
  T* su = reinterpret_cast<T*>(mine);
  float* sF = reinterpret_cast<float*>(su + (size_t)D * S);
  float* sC = sF + S;
  int* sel = reinterpret_cast<int*>(sC + S);
  unsigned char* taken = reinterpret_cast<unsigned char*>(sel + 32);
  const int64_t PS = a.P * S, b = p * S;
  for (int j = lane; j < S; j += 32) {
    sF[j] = so.F[b + j];
    sC[j] = so.C[b + j];
  }
  for (int q = 0; q < D; ++q)
    for (int j = lane; j < S; j += 32) su[q * S + j] = so.u[q * PS + b + j];
  __syncwarp();
  warp_topk<T>(sF, sC, su, S, D, S, a.K, a.eps, sel, taken, nullptr);
  const int64_t ldc = a.P * a.K;
  for (int t = lane; t < a.K * D; t += 32) {
    const int k = t / D, q = t % D;
    const int j = sel[k];
    a.cand_u[q * ldc + p * a.K + k] = j >= 0 ? su[q * S + j] : T(NAN);
  }
}

// FP64 acceptance of one state: cost, pose errors, limit and clearance flags.
template <int N, bool OBST, int MODEL = CR_MODEL_TENDON>
CR_HD double accept_fp64(const RobotK<double>& rb, const WeightsK<double>& w, int kind,
                         const TargetK<double>& tg, ObsK<double> ob, int no,
                         const double (&u)[3 * N], double lim_tol, double& pos, double& rot,
                         unsigned char& flags) {
  const Sphere4<double>* sph = ob.s;
  double dummy[3 * N];
  double F = eval_ik<double, N, OBST, false, false, true, MODEL>(rb, w, kind, tg, ob, no, u, dummy, nullptr, nullptr,
                                                                nullptr);
  Chain<double, N> ch;
  chain_forward<double, N, MODEL>(rb, u, ch);
  double dx = ch.p[0] - tg.p[0], dy = ch.p[1] - tg.p[1], dz = ch.p[2] - tg.p[2];
  pos = sqrt(dx * dx + dy * dy + dz * dz);
  if (kind == CR_TASK_IK5) {
    double z[3] = {ch.R[2], ch.R[5], ch.R[8]}, zt[3] = {tg.R[0], tg.R[1], tg.R[2]}, cz[3];
    cross(z, zt, cz);
    rot = atan2(sqrt(dot3(cz, cz)), dot3(z, zt));
  } else {
    double E[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        E[3 * i + j] = tg.R[i] * ch.R[j] + tg.R[3 + i] * ch.R[3 + j] + tg.R[6 + i] * ch.R[6 + j];
    double e[3], sn, cs;
    so3_log(E, e, sn, cs);
    rot = sqrt(dot3(e, e));
  }
  bool lim = true;
  for (int i = 0; i < N; ++i) {
    if (MODEL == CR_MODEL_ARC) {
      if (u[3 * i + 2] > rb.lmax[i] + lim_tol || u[3 * i + 2] < rb.lmin[i] - lim_tol) lim = false;
    } else {
      double su = u[3 * i] + u[3 * i + 1] + u[3 * i + 2];
      if (fabs(su) > lim_tol) lim = false;
      for (int j = 0; j < 3; ++j)
        if (fabs(u[3 * i + j]) > rb.umax[i] + lim_tol) lim = false;
    }
    if (sqrt(ch.x[i]) > rb.thmax[i] + 1e-6) lim = false;
  }
  // clearance without the margin (radius r_o + r_body); the broad phase uses the larger reach
  bool free = true;
  if (OBST && no > 0) {
    const double inb = 1.0 / rb.nb;
    for (int j0 = 0; j0 < no && free; j0 += 64) {
      uint64_t mk[N];
      segment_sphere_masks(rb, ch, ob, j0, no - j0 < 64 ? no - j0 : 64, mk);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        if (!mk[i] || !free) continue;
        for (int k0 = 1; k0 <= rb.nb && free; k0 += kCullGroup) {
          const int k1 = k0 + kCullGroup - 1 < rb.nb ? k0 + kCullGroup - 1 : rb.nb;
          const uint64_t gm = group_sphere_mask<double, N>(rb, ch, i, k0, k1, ob, j0, mk[i]);
          for (int k = k0; k <= k1 && gm && free; ++k) {
            double q[3], wp[3], s, c;
            backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], k * inb, q, wp, s, c);
            for (uint64_t bits = gm; bits; bits &= bits - 1) {
              const int j = j0 + __ffsll((long long)bits) - 1;
              if (ob.prims() && j >= ob.ns) {
                const PrimK<double>& P = ob.p[j - ob.ns];
                double viol, nv[3];
                if (prim_active(P, wp, P.reach - w.delta, viol, nv)) { free = false; break; }
                continue;
              }
              double ddx = wp[0] - sph[j].x, ddy = wp[1] - sph[j].y, ddz = wp[2] - sph[j].z;
              double r = sph[j].reach - w.delta;
              if (ddx * ddx + ddy * ddy + ddz * ddz < r * r) { free = false; break; }
            }
          }
        }
      }
    }
  }
  // with the self-contact rows on: samples of segments two or more apart at least 2 r_body apart
  if (OBST && N >= 3 && w.rho_s > 0.0 && free) {
    const double inb = 1.0 / rb.nb, g2 = 4.0 * rb.rbody * rb.rbody;
    double mid[N][3];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double q[3], s, c;
      backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], 0.5, q, mid[i], s, c);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int j = i + 2; j < N; ++j) {
        if (!free) continue;
        const double dx = mid[i][0] - mid[j][0], dy = mid[i][1] - mid[j][1], dz = mid[i][2] - mid[j][2];
        const double lim2 = 0.5 * (ch.L[i] + ch.L[j]) + 2.0 * rb.rbody + 1e-9;
        if (!(dx * dx + dy * dy + dz * dz < lim2 * lim2)) continue;
        for (int ka = 1; ka <= rb.nb && free; ++ka) {
          double qa[3], pa[3], s_a, c_a;
          backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], ka * inb, qa, pa, s_a, c_a);
          for (int kb = 1; kb <= rb.nb; ++kb) {
            double qb[3], pb[3], s_b, c_b;
            backbone_point(ch.Rb[j], ch.pb[j], ch.ax[j], ch.ay[j], ch.x[j], ch.L[j], kb * inb, qb, pb, s_b, c_b);
            const double ex = pa[0] - pb[0], ey = pa[1] - pb[1], ez = pa[2] - pb[2];
            if (ex * ex + ey * ey + ez * ez < g2) { free = false; break; }
          }
        }
      }
    }
  }
  flags = (unsigned char)((lim ? 1 : 0) | (free ? 2 : 0));
  return F;
}

template <typename T, int N, bool OBST, int MODEL = CR_MODEL_TENDON, bool PRIMS = true>
__global__ void __launch_bounds__(128) k_ik_refine(RobotK<T> rb, WeightsK<T> w, RobotK<double> rbd,
                                                    WeightsK<double> wd, IkArgs<T> a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nob = a.no + a.np;
  ObsK<double> sphd(nullptr);
  ObsK<T> sph(nullptr);
  const int64_t PK = a.P * a.K;
  // shared sphere set: one candidate per thread; per-problem sets: tpb targets per block, K threads
  // each
  const int jt = a.sph_pp ? (int)threadIdx.x / a.K : 0;
  const int64_t c = a.sph_pp ? ((int64_t)blockIdx.x * a.tpb + jt) * a.K + (int)threadIdx.x % a.K
                             : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (OBST) {
    // the block's obstacle sets (tpb of them with per-problem scenes), each in FP64 and in T
    const size_t setb = refine_set_bytes<T>(a.no, a.np), offt = (obstacles_smem<double>(a.no, a.np) + 15) & ~(size_t)15;
    const int64_t t0 = a.sph_pp ? (int64_t)blockIdx.x * a.tpb : 0;
    const int ntb = a.sph_pp ? (int)(a.P - t0 < a.tpb ? a.P - t0 : a.tpb) : 1;
    for (int t = 0; t < ntb; ++t) {
      unsigned char* base = smem_raw + (size_t)t * setb;
      const ObsK<double> od = stage_problem_obstacles<PRIMS>(a, t0 + t, rbd, wd.delta, base);
      const ObsK<T> ot = stage_problem_obstacles<PRIMS>(a, t0 + t, rb, w.delta, base + offt);
      if (t == jt) {
        sphd = od;
        sph = ot;
      }
    }
    __syncthreads();
  }
  if (c >= PK || (a.sph_pp && jt >= a.tpb)) return;
  const int64_t p = c / a.K;
  T u[D];
#pragma unroll
  for (int q = 0; q < D; ++q) u[q] = a.cand_u[q * PK + c];
  bool valid = c_finite(u[0]);
  if (valid) {
    TargetK<T> tg = load_target<T>(a.targets, a.P, p, a.kind);
    double lam = a.lambda0, nu = 2.0;
    T F;
    for (int it = 0; it < a.k_final; ++it)
      lm_iteration<T, N, OBST, MODEL>(rb, w, a.kind, tg, sph, nob, u, lam, nu, F);
  }
  double ud[D];
#pragma unroll
  for (int q = 0; q < D; ++q) ud[q] = double(u[q]);
  double pos = NAN, rot = NAN, F = NAN;
  unsigned char flags = 0;
  if (valid) {
    TargetK<double> tgd = load_target<double>(a.targets, a.P, p, a.kind);
    F = accept_fp64<N, OBST, MODEL>(rbd, wd, a.kind, tgd, sphd, nob, ud, a.lim_tol, pos, rot, flags);
  }
#pragma unroll
  for (int q = 0; q < D; ++q) a.cand_u64[q * PK + c] = ud[q];
  a.cand_F[c] = F;
  a.cand_pos[c] = pos;
  a.cand_rot[c] = rot;
  a.cand_flag[c] = flags;
}

// Refine of problems with their own spheres and few candidates (K < 8): FP32 bulk, full pose,
// tendon model. One block per target, one warp per candidate: the warp runs the LM iterations
// cooperatively (warp_lm_step: lane q forms entry q of each residual row, the packed J^T J lives in
// slots spread over the lanes, the backbone samples of the clearance rows are split over the lanes)
// and solves the damped system in FP64 by the symmetric sweep of the augmented matrix (the pivots
// of its LDL^T factorisation); the FP64 acceptance follows. With one candidate per thread a warp of
// such a target would have K of its 32 lanes busy in both the FP32 and the FP64 work.
template <int N>
__global__ void __launch_bounds__(256, 1) k_ik_refine_warp(RobotK<float> rb, WeightsK<float> w, RobotK<double> rbd,
                                                       WeightsK<double> wd, IkArgs<float> a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nob = a.no + a.np;
  double* scr = reinterpret_cast<double*>(smem_raw + refine_set_bytes<float>(a.no, a.np));
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;  // blockDim = 32 K: warp wid, candidate wid
  double* sud = scr + (size_t)a.K * 128;                       // refined states [K][D] for the acceptance
  double* col = scr + wid * 128;
  double* colr = col + 32;
  double* sx = colr + 32;
  double* sdg = sx + 32;
  const int64_t p = blockIdx.x;
  const ObsK<double> sphd = stage_problem_obstacles(a, p, rbd, wd.delta, smem_raw);
  const ObsK<float> sph =
      stage_problem_obstacles(a, p, rb, w.delta, smem_raw + ((obstacles_smem<double>(a.no, a.np) + 15) & ~(size_t)15));
  __syncthreads();
  const int64_t PK = a.P * a.K;
  {
    const int64_t c = p * a.K + wid;
    float u[D];
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = a.cand_u[q * PK + c];
    if (c_finite(u[0])) {  // the same in every lane
      const TargetK<float> tg = load_target<float>(a.targets, a.P, p, CR_TASK_IK6);
      const AugSlots<D> sl = aug_slots<D>(lane);
      double lam = a.lambda0, nu = 2.0;
      for (int it = 0; it < a.k_final; ++it)
        warp_lm_step<float, N, true, double>(rb, w, tg, sph, nob, u, sl, lam, nu, col, colr, sx, sdg);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < D; ++q) sud[wid * D + q] = double(u[q]);
    }
  }
  __syncthreads();
  // FP64 acceptance, one lane per candidate (the FP64 pipe charges whole warps: K lanes of one warp
  // instead of K warps running the same check in all their lanes)
  if (wid == 0 && lane < a.K) {
    const int64_t c = p * a.K + lane;
    double ud[D];
#pragma unroll
    for (int q = 0; q < D; ++q) ud[q] = sud[lane * D + q];
    double pos = NAN, rot = NAN, F = NAN;
    unsigned char flags = 0;
    if (isfinite(ud[0])) {
      const TargetK<double> tgd = load_target<double>(a.targets, a.P, p, CR_TASK_IK6);
      F = accept_fp64<N, true>(rbd, wd, CR_TASK_IK6, tgd, sphd, nob, ud, a.lim_tol, pos, rot, flags);
    }
#pragma unroll
    for (int q = 0; q < D; ++q) a.cand_u64[q * PK + c] = ud[q];
    a.cand_F[c] = F;
    a.cand_pos[c] = pos;
    a.cand_rot[c] = rot;
    a.cand_flag[c] = flags;
  }
}

template <int N>
__global__ void __launch_bounds__(128) k_ik_argmin(int64_t P, int K, double pos_tol, double rot_tol,
                                                    const double* cand_u64, const double* cand_F,
                                                    const double* cand_pos, const double* cand_rot,
                                                    const unsigned char* cand_flag, double* u_out,
                                                    double* cost_out, double* pos_out, double* rot_out,
                                                    unsigned char* success, int* status) {
  constexpr int D = 3 * N;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int64_t PK = P * K;
  // key: the cost, or 0 for a solution at the rounding level (CR_ARGMIN_TIE): the first such
  // candidate in SelectTop order wins
  int best = -1;
  double bkey = INFINITY;
  for (int k = 0; k < K; ++k) {
    const double F = cand_F[p * K + k];
    const double key = F <= CR_ARGMIN_TIE ? 0.0 : F;
    if (isfinite(F) && key < bkey) { bkey = key; best = k; }
  }
  const double bF = best >= 0 ? cand_F[p * K + best] : INFINITY;
  if (best < 0) {
#pragma unroll
    for (int q = 0; q < D; ++q) u_out[q * P + p] = NAN;
    cost_out[p] = NAN;
    pos_out[p] = NAN;
    rot_out[p] = NAN;
    success[p] = 0;
    atomicOr(status, 1 << CR_ENONFINITE);
    return;
  }
  const int64_t c = p * K + best;
#pragma unroll
  for (int q = 0; q < D; ++q) u_out[q * P + p] = cand_u64[q * PK + c];
  cost_out[p] = bF;
  double pe = cand_pos[c], re = cand_rot[c];
  pos_out[p] = pe;
  rot_out[p] = re;
  unsigned char f = cand_flag[c];
  success[p] = (pe <= pos_tol && re <= rot_tol && (f & 1) && (f & 2)) ? 1 : 0;
}

// ------------------------------------------------------------------------------------------------
// Standalone steps: LM iterations, projected-gradient steps, seeds, SelectTop
// ------------------------------------------------------------------------------------------------
template <typename T> struct StepArgs {
  int kind;
  const double* targets;
  int64_t P;
  int S;
  const double* spheres;
  int no;
  const double* prims;
  int np;
  T* u;
  int64_t B;
  int iters;
  double* lam;
  double* nu;
  double* F64;
  int* acc;
  T* alpha;
  T* F;
};

template <typename T, int N, bool OBST, int MODEL = CR_MODEL_TENDON>
__global__ void __launch_bounds__(128) k_lm_steps(RobotK<T> rb, WeightsK<T> w, StepArgs<T> a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ObsK<T> sph(nullptr);
  if (OBST) {
    sph = stage_obstacles(a.spheres, a.no, a.prims, a.np, rb, w.delta, smem_raw);
    __syncthreads();
  }
  const int nob = a.no + a.np;
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.B) return;
  T u[D];
#pragma unroll
  for (int q = 0; q < D; ++q) u[q] = a.u[q * a.B + b];
  TargetK<T> tg = load_target<T>(a.targets, a.P, b / a.S, a.kind);
  double lam = a.lam[b], nu = a.nu[b];
  int nacc = 0;
  T F = T(0);
  for (int it = 0; it < a.iters; ++it)
    nacc += lm_iteration<T, N, OBST, MODEL>(rb, w, a.kind, tg, sph, nob, u, lam, nu, F);
  if (a.iters == 0 || a.F64) {
    T dummy[D];
    F = eval_ik<T, N, OBST, false, false, true, MODEL>(rb, w, a.kind, tg, sph, nob, u, dummy, nullptr, nullptr,
                                                       nullptr);
  }
#pragma unroll
  for (int q = 0; q < D; ++q) a.u[q * a.B + b] = u[q];
  a.lam[b] = lam;
  a.nu[b] = nu;
  if (a.F64) a.F64[b] = double(F);
  if (a.acc) a.acc[b] = nacc;
}

template <typename T, int N, bool OBST, int MODEL = CR_MODEL_TENDON>
__global__ void __launch_bounds__(128) k_pg_steps(RobotK<T> rb, WeightsK<T> w, StepArgs<T> a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ObsK<T> sph(nullptr);
  if (OBST) {
    sph = stage_obstacles(a.spheres, a.no, a.prims, a.np, rb, w.delta, smem_raw);
    __syncthreads();
  }
  const int nob = a.no + a.np;
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.B) return;
  T u[D], g[D], coll;
#pragma unroll
  for (int q = 0; q < D; ++q) u[q] = a.u[q * a.B + b];
  TargetK<T> tg = load_target<T>(a.targets, a.P, b / a.S, a.kind);
  T F = eval_ik<T, N, OBST, true, false, true, MODEL>(rb, w, a.kind, tg, sph, nob, u, g, nullptr, nullptr, &coll);
  T alpha = a.alpha[b];
  for (int it = 0; it < a.iters; ++it)
    pg_step<T, N, OBST, MODEL>(rb, w, a.kind, tg, sph, nob, u, g, F, coll, alpha);
#pragma unroll
  for (int q = 0; q < D; ++q) a.u[q * a.B + b] = u[q];
  a.alpha[b] = alpha;
  a.F[b] = F;
}

// sph_pp = 0: blocks of 128 consecutive seeds; sph_pp = 1: blockIdx.y = problem, its own obstacles.
template <typename T, int N, bool OBST, int MODEL = CR_MODEL_TENDON>
__global__ void __launch_bounds__(128) k_seeds(RobotK<T> rb, WeightsK<T> w, const double* spheres, int no,
                                                const double* prims, int np, int sph_pp, uint64_t key, int64_t p0,
                                                int64_t P, int S, SeedBox box, T* u_out) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ObsK<T> sph(nullptr);
  if (OBST) {
    const int64_t q = sph_pp ? (int64_t)blockIdx.y : 0;
    sph = stage_obstacles(spheres + q * no * 4, no, np > 0 ? prims + q * np * CR_PRIM_DOUBLES : nullptr, np, rb,
                          w.delta, smem_raw);
    __syncthreads();
  }
  const int64_t PS = P * S;
  const int64_t i = sph_pp ? (int64_t)blockIdx.y * S + (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                           : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= PS || (sph_pp && (int64_t)blockIdx.x * blockDim.x + threadIdx.x >= S)) return;
  const int64_t p = i / S, s = i % S;
  T u[D];
  draw_seed_m<MODEL, T, N>(key, (uint64_t)(p0 + p), (uint64_t)s, 0, box, u);
  if (OBST && no + np > 0) {
    for (int att = 1; att < 8; ++att) {
      if (!state_collides<T, N, MODEL>(rb, sph, no + np, u)) break;
      draw_seed_m<MODEL, T, N>(key, (uint64_t)(p0 + p), (uint64_t)s, att, box, u);
    }
  }
#pragma unroll
  for (int q = 0; q < D; ++q) u_out[q * PS + i] = u[q];
}

template <typename T>
__global__ void __launch_bounds__(32) k_topk(const float* cost, const float* coll, const T* u, int D, int64_t P,
                                              int S, int K, T eps, int* idx_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* skipped = reinterpret_cast<int*>(smem_raw);
  int* sel = skipped + S;
  unsigned char* taken = reinterpret_cast<unsigned char*>(sel + 32);
  const int64_t p = blockIdx.x;
  warp_topk<T>(cost + p * S, coll + p * S, u + p * S, P * S, D, S, K, eps, sel, taken, skipped);
  for (int k = threadIdx.x; k < K; k += 32) idx_out[p * K + k] = sel[k];
}

// ------------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------------
struct SolveArgs {
  cr_robot robot;
  cr_scene scene;
  cr_task task;
  cr_ik_params prm;
  void* ws;
  crh::IkLayout lay;
  double *u_out, *cost_out, *pos, *rot;
  unsigned char* success;
  // step entry points
  void* u;
  int64_t B;
  int iters;
  double *lam, *nu, *F64;
  int* acc;
  void *alpha, *F;
  // seeds / topk
  uint64_t key;
  int64_t p0, P;
  int S, K;
  double eps;
  const float *tk_cost, *tk_coll;
  int* tk_idx;
  int D;
  cudaStream_t stream;
};

template <typename T> cr_status launch_solve_ik(const SolveArgs& a, int which);
template <typename T> cr_status launch_lm_steps(const SolveArgs& a);
template <typename T> cr_status launch_pg_steps(const SolveArgs& a);
template <typename T> cr_status launch_seeds(const SolveArgs& a);
template <typename T> cr_status launch_topk(const SolveArgs& a);

inline unsigned grid1(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <typename K> cr_status set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return crh::fail(CR_ECUDA, "shared memory %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  return CR_OK;
}

template <typename T> IkArgs<T> ik_args(const SolveArgs& a) {
  IkArgs<T> k;
  const cr_ik_params& p = a.prm;
  unsigned char* ws = (unsigned char*)a.ws;
  k.kind = a.task.kind;
  k.targets = a.task.targets;
  k.P = a.task.n_targets;
  k.spheres = a.scene.spheres;
  k.no = a.scene.n_o;
  k.prims = a.scene.prims;
  k.np = a.scene.n_p;
  k.sph_pp = (a.scene.per_problem && a.scene.n_o + a.scene.n_p > 0) ? 1 : 0;
  k.tpb = 1;
  k.S = p.S;
  k.K = p.n_final;
  k.k_init = p.k_init;
  k.k_final = p.k_final;
  k.alpha0 = T(p.alpha0);
  k.eps = T(p.dedup_eps);
  k.lambda0 = p.lambda0;
  k.lim_tol = p.lim_tol;
  k.pos_tol = p.pos_tol;
  k.rot_tol = p.rot_tol;
  k.box = seed_box(a.robot);
  k.seed = p.seed;
  k.p0 = p.p0;
  k.cand_u = (T*)(ws + a.lay.cand_u);
  k.cand_u64 = (double*)(ws + a.lay.cand_u64);
  k.cand_F = (double*)(ws + a.lay.cand_F);
  k.cand_pos = (double*)(ws + a.lay.cand_pos);
  k.cand_rot = (double*)(ws + a.lay.cand_rot);
  k.cand_flag = ws + a.lay.cand_flag;
  k.u_out = a.u_out;
  k.cost_out = a.cost_out;
  k.pos_out = a.pos;
  k.rot_out = a.rot;
  k.success = a.success;
  k.status = (int*)(ws + a.lay.status);
  k.pg_accepted = (unsigned long long*)(ws + a.lay.status + 8);
  return k;
}

// which: 1 = stage one only, 2 = stage two only, 3 = both
template <typename T, int N, int MODEL = CR_MODEL_TENDON> cr_status solve_ik_n(const SolveArgs& a, int which) {
  constexpr int D = 3 * N;
  RobotK<T> rb = crh::robot_k<T>(a.robot);
  WeightsK<T> w = crh::weights_k<T>(a.task.w);
  RobotK<double> rbd = crh::robot_k<double>(a.robot);
  WeightsK<double> wd = crh::weights_k<double>(a.task.w);
  IkArgs<T> k = ik_args<T>(a);
  const int64_t P = k.P;
  const int no = k.no, np = k.np;
  const int threads = ((k.S + 31) / 32) * 32;
  const size_t sm1 = obstacles_smem<T>(no, np);
  cr_status st;
  const bool coll_rows = no + np > 0 || a.task.w.rho_s > 0;  // collision rows: obstacles and / or self-contact
  if (which & 1) {
    unsigned char* ws = (unsigned char*)a.ws;
    StageOut<T> so{(float*)(ws + a.lay.stage_F), (float*)(ws + a.lay.stage_C), (T*)(ws + a.lay.stage_u)};
    if (coll_rows) {
      // tendon-model scenes without primitives take the form compiled without primitive code
      bool done = false;
      if constexpr (MODEL == CR_MODEL_TENDON) {
        if (np == 0) {
          if ((st = set_smem(k_ik_stage1<T, N, true, MODEL, false>, sm1))) return st;
          k_ik_stage1<T, N, true, MODEL, false><<<(unsigned)P, threads, sm1, a.stream>>>(rb, w, k, so);
          done = true;
        }
      }
      if (!done) {
        if ((st = set_smem(k_ik_stage1<T, N, true, MODEL>, sm1))) return st;
        k_ik_stage1<T, N, true, MODEL><<<(unsigned)P, threads, sm1, a.stream>>>(rb, w, k, so);
      }
    } else {
      k_ik_stage1<T, N, false, MODEL><<<(unsigned)P, threads, 0, a.stream>>>(rb, w, k, so);
    }
    if ((st = crh::check_launch("cr_solve_ik stage one"))) return st;
    // SelectTop: as many warps (targets) per block as fit in 96 KB of shared memory, at most 8
    const size_t pw = SelectSmem<T>::per_warp(k.S, D);
    int wpb = (int)((96 * 1024) / pw);
    wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
    if ((st = set_smem(k_ik_select<T>, pw * wpb))) return st;
    k_ik_select<T><<<(unsigned)((P + wpb - 1) / wpb), 32 * wpb, pw * wpb, a.stream>>>(k, so, D);
    if ((st = crh::check_launch("cr_solve_ik SelectTop"))) return st;
  }
  if (!(which & 2)) return CR_OK;
  // per-problem obstacles: one warp per block. With K >= 8 it holds 32 / K (at most 4) targets, their
  // obstacle sets side by side in shared memory, so that the FP64 instructions run with all lanes busy
  // (the FP64 pipe charges a whole warp). With fewer candidates per target it holds one: more
  // targets per warp make the lanes' clearance loops diverge (the warp runs the union of their
  // trips), which costs more than the idle FP64 lanes (measured on the 4-candidate goal IK of the
  // trajectory workload).
  const size_t per_set = no + np > 0 ? refine_set_bytes<T>(no, np) : 0;
  k.tpb = 1;
  if (k.sph_pp && k.K >= 8) {
    k.tpb = 32 / k.K;
    const int cap = (int)((96 * 1024) / (per_set > 0 ? per_set : 1));
    if (k.tpb > cap) k.tpb = cap;
    if (k.tpb < 1) k.tpb = 1;
  }
  size_t sm2 = per_set * k.tpb;
  // shared (or no) spheres: one warp per block, so that the FP64-bound refine spreads evenly over all
  // SMs (128-thread blocks left the busiest SMs with 2 blocks where the average is 1.7: 1.07 ms
  // against 0.95 ms for 4096 targets x 8 candidates)
  unsigned g2 = k.sph_pp ? grid1(P, k.tpb) : grid1(P * k.K, 32);
  int b2 = k.sph_pp ? ((k.tpb * k.K + 31) / 32) * 32 : 32;
  bool warp_refine = false;
  if constexpr (sizeof(T) == 4 && MODEL == CR_MODEL_TENDON) {
    if (k.sph_pp && k.K < 8 && k.kind == CR_TASK_IK6 && !(a.task.w.rho_s > 0)) {
      const size_t smw = refine_set_bytes<float>(no, np) + (size_t)k.K * (128 + D) * sizeof(double);
      if ((st = set_smem(k_ik_refine_warp<N>, smw))) return st;
      k_ik_refine_warp<N><<<(unsigned)P, 32 * k.K, smw, a.stream>>>(rb, w, rbd, wd, k);
      warp_refine = true;
    }
  }
  if (warp_refine) {
  } else if (coll_rows) {
    bool done = false;
    if constexpr (MODEL == CR_MODEL_TENDON) {
      if (np == 0) {
        if ((st = set_smem(k_ik_refine<T, N, true, MODEL, false>, sm2))) return st;
        k_ik_refine<T, N, true, MODEL, false><<<g2, b2, sm2, a.stream>>>(rb, w, rbd, wd, k);
        done = true;
      }
    }
    if (!done) {
      if ((st = set_smem(k_ik_refine<T, N, true, MODEL>, sm2))) return st;
      k_ik_refine<T, N, true, MODEL><<<g2, b2, sm2, a.stream>>>(rb, w, rbd, wd, k);
    }
  }
  else k_ik_refine<T, N, false, MODEL><<<g2, b2, sm2, a.stream>>>(rb, w, rbd, wd, k);
  if ((st = crh::check_launch("cr_solve_ik refine"))) return st;
  k_ik_argmin<N><<<grid1(P, 128), 128, 0, a.stream>>>(P, k.K, k.pos_tol, k.rot_tol, k.cand_u64, k.cand_F,
                                                      k.cand_pos, k.cand_rot, k.cand_flag, k.u_out,
                                                      k.cost_out, k.pos_out, k.rot_out, k.success, k.status);
  return crh::check_launch("cr_solve_ik argmin");
}

template <typename T> StepArgs<T> step_args(const SolveArgs& a) {
  StepArgs<T> k;
  k.kind = a.task.kind;
  k.targets = a.task.targets;
  k.P = a.task.n_targets;
  k.S = a.task.seeds_per_target;
  k.spheres = a.scene.spheres;
  k.no = a.scene.n_o;
  k.prims = a.scene.prims;
  k.np = a.scene.n_p;
  k.u = (T*)a.u;
  k.B = a.B;
  k.iters = a.iters;
  k.lam = a.lam;
  k.nu = a.nu;
  k.F64 = a.F64;
  k.acc = a.acc;
  k.alpha = (T*)a.alpha;
  k.F = (T*)a.F;
  return k;
}

template <typename T, int N, int MODEL = CR_MODEL_TENDON> cr_status lm_steps_n(const SolveArgs& a) {
  RobotK<T> rb = crh::robot_k<T>(a.robot);
  WeightsK<T> w = crh::weights_k<T>(a.task.w);
  StepArgs<T> k = step_args<T>(a);
  size_t sm = obstacles_smem<T>(k.no, k.np);
  if (k.no + k.np > 0 || w.rho_s > T(0)) k_lm_steps<T, N, true, MODEL><<<grid1(a.B, 128), 128, sm, a.stream>>>(rb, w, k);
  else k_lm_steps<T, N, false, MODEL><<<grid1(a.B, 128), 128, sm, a.stream>>>(rb, w, k);
  return crh::check_launch("cr_lm_step");
}

template <typename T, int N, int MODEL = CR_MODEL_TENDON> cr_status pg_steps_n(const SolveArgs& a) {
  RobotK<T> rb = crh::robot_k<T>(a.robot);
  WeightsK<T> w = crh::weights_k<T>(a.task.w);
  StepArgs<T> k = step_args<T>(a);
  size_t sm = obstacles_smem<T>(k.no, k.np);
  if (k.no + k.np > 0 || w.rho_s > T(0)) k_pg_steps<T, N, true, MODEL><<<grid1(a.B, 128), 128, sm, a.stream>>>(rb, w, k);
  else k_pg_steps<T, N, false, MODEL><<<grid1(a.B, 128), 128, sm, a.stream>>>(rb, w, k);
  return crh::check_launch("cr_pg_steps");
}

template <typename T, int N, int MODEL = CR_MODEL_TENDON> cr_status seeds_n(const SolveArgs& a) {
  RobotK<T> rb = crh::robot_k<T>(a.robot);
  WeightsK<T> w = crh::weights_k<T>(a.task.w);
  const SeedBox box = seed_box(a.robot);
  int no = a.scene.n_o, np = a.scene.n_p;
  int pp = a.scene.per_problem ? 1 : 0;
  size_t sm = obstacles_smem<T>(no, np);
  dim3 g = pp ? dim3(grid1(a.S, 128), (unsigned)a.P) : dim3(grid1(a.P * a.S, 128));
  if (no + np > 0)
    k_seeds<T, N, true, MODEL><<<g, 128, sm, a.stream>>>(rb, w, a.scene.spheres, no, a.scene.prims, np, pp, a.key,
                                                         a.p0, a.P, a.S, box, (T*)a.u);
  else
    k_seeds<T, N, false, MODEL><<<g, 128, sm, a.stream>>>(rb, w, a.scene.spheres, no, a.scene.prims, np, pp, a.key,
                                                          a.p0, a.P, a.S, box, (T*)a.u);
  return crh::check_launch("cr_seeds");
}

// The arc model's launchers (1..CR_MAX_SEG_ARC segments) live in their own translation units.
template <typename T> cr_status launch_solve_ik_arc(const SolveArgs& a, int which);
template <typename T> cr_status launch_lm_steps_arc(const SolveArgs& a);
template <typename T> cr_status launch_pg_steps_arc(const SolveArgs& a);
template <typename T> cr_status launch_seeds_arc(const SolveArgs& a);

#define CR_COUPLED_DISPATCH(FN, T, N_, ...)                          \
  switch (N_) {                                                      \
    case 1: return FN<T, 1, CR_MODEL_COUPLED>(__VA_ARGS__);          \
    case 2: return FN<T, 2, CR_MODEL_COUPLED>(__VA_ARGS__);          \
    case 3: return FN<T, 3, CR_MODEL_COUPLED>(__VA_ARGS__);          \
    case 4: return FN<T, 4, CR_MODEL_COUPLED>(__VA_ARGS__);          \
    case 5: return FN<T, 5, CR_MODEL_COUPLED>(__VA_ARGS__);          \
    default: return FN<T, 6, CR_MODEL_COUPLED>(__VA_ARGS__);         \
  }

template <typename T> cr_status launch_solve_ik(const SolveArgs& a, int which) {
  if (a.robot.model == CR_MODEL_ARC) return launch_solve_ik_arc<T>(a, which);
  if (a.robot.model == CR_MODEL_COUPLED) { CR_COUPLED_DISPATCH(solve_ik_n, T, a.robot.n, a, which) }
  switch (a.robot.n) {
    case 1: return solve_ik_n<T, 1>(a, which);
    case 2: return solve_ik_n<T, 2>(a, which);
    case 3: return solve_ik_n<T, 3>(a, which);
    case 4: return solve_ik_n<T, 4>(a, which);
    case 5: return solve_ik_n<T, 5>(a, which);
    default: return solve_ik_n<T, 6>(a, which);
  }
}
template <typename T> cr_status launch_lm_steps(const SolveArgs& a) {
  if (a.robot.model == CR_MODEL_ARC) return launch_lm_steps_arc<T>(a);
  if (a.robot.model == CR_MODEL_COUPLED) { CR_COUPLED_DISPATCH(lm_steps_n, T, a.robot.n, a) }
  switch (a.robot.n) {
    case 1: return lm_steps_n<T, 1>(a);
    case 2: return lm_steps_n<T, 2>(a);
    case 3: return lm_steps_n<T, 3>(a);
    case 4: return lm_steps_n<T, 4>(a);
    case 5: return lm_steps_n<T, 5>(a);
    default: return lm_steps_n<T, 6>(a);
  }
}
template <typename T> cr_status launch_pg_steps(const SolveArgs& a) {
  if (a.robot.model == CR_MODEL_ARC) return launch_pg_steps_arc<T>(a);
  if (a.robot.model == CR_MODEL_COUPLED) { CR_COUPLED_DISPATCH(pg_steps_n, T, a.robot.n, a) }
  switch (a.robot.n) {
    case 1: return pg_steps_n<T, 1>(a);
    case 2: return pg_steps_n<T, 2>(a);
    case 3: return pg_steps_n<T, 3>(a);
    case 4: return pg_steps_n<T, 4>(a);
    case 5: return pg_steps_n<T, 5>(a);
    default: return pg_steps_n<T, 6>(a);
  }
}
template <typename T> cr_status launch_seeds(const SolveArgs& a) {
  if (a.robot.model == CR_MODEL_ARC) return launch_seeds_arc<T>(a);
  if (a.robot.model == CR_MODEL_COUPLED) { CR_COUPLED_DISPATCH(seeds_n, T, a.robot.n, a) }
  switch (a.robot.n) {
    case 1: return seeds_n<T, 1>(a);
    case 2: return seeds_n<T, 2>(a);
    case 3: return seeds_n<T, 3>(a);
    case 4: return seeds_n<T, 4>(a);
    case 5: return seeds_n<T, 5>(a);
    default: return seeds_n<T, 6>(a);
  }
}
template <typename T> cr_status launch_topk(const SolveArgs& a) {
  size_t sm = (size_t)a.S * sizeof(int) + 32 * sizeof(int) + a.S;
  k_topk<T><<<(unsigned)a.P, 32, sm, a.stream>>>(a.tk_cost, a.tk_coll, (const T*)a.u, a.D, a.P, a.S, a.K,
                                                  T(a.eps), a.tk_idx);
  return crh::check_launch("cr_topk");
}

#define CR_ARC_DISPATCH(FN, T, N_, ...)                              \
  switch (N_) {                                                      \
    case 1: return FN<T, 1, CR_MODEL_ARC>(__VA_ARGS__);              \
    case 2: return FN<T, 2, CR_MODEL_ARC>(__VA_ARGS__);              \
    case 3: return FN<T, 3, CR_MODEL_ARC>(__VA_ARGS__);              \
    default: return FN<T, 4, CR_MODEL_ARC>(__VA_ARGS__);             \
  }

template <typename T> cr_status launch_solve_ik_arc(const SolveArgs& a, int which) {
  CR_ARC_DISPATCH(solve_ik_n, T, a.robot.n, a, which)
}
template <typename T> cr_status launch_lm_steps_arc(const SolveArgs& a) { CR_ARC_DISPATCH(lm_steps_n, T, a.robot.n, a) }
template <typename T> cr_status launch_pg_steps_arc(const SolveArgs& a) { CR_ARC_DISPATCH(pg_steps_n, T, a.robot.n, a) }
template <typename T> cr_status launch_seeds_arc(const SolveArgs& a) { CR_ARC_DISPATCH(seeds_n, T, a.robot.n, a) }

#define CR_SOLVE_ARC_INSTANTIATE(EXT, T)                                \
  EXT template cr_status launch_solve_ik_arc<T>(const SolveArgs&, int); \
  EXT template cr_status launch_lm_steps_arc<T>(const SolveArgs&);      \
  EXT template cr_status launch_pg_steps_arc<T>(const SolveArgs&);      \
  EXT template cr_status launch_seeds_arc<T>(const SolveArgs&);

// Per segment count (one compilation unit each, so that the units build in parallel and ptxas
// allocates registers per kernel family).
#define CR_SOLVE_N_INSTANTIATE(EXT, T, N_, MODEL)                           \
  EXT template cr_status solve_ik_n<T, N_, MODEL>(const SolveArgs&, int); \
  EXT template cr_status lm_steps_n<T, N_, MODEL>(const SolveArgs&);      \
  EXT template cr_status pg_steps_n<T, N_, MODEL>(const SolveArgs&);      \
  EXT template cr_status seeds_n<T, N_, MODEL>(const SolveArgs&);
#define CR_SOLVE_ALL_N_EXTERN(T)                         \
  CR_SOLVE_N_INSTANTIATE(extern, T, 1, CR_MODEL_TENDON) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 2, CR_MODEL_TENDON) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 3, CR_MODEL_TENDON) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 4, CR_MODEL_TENDON) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 5, CR_MODEL_TENDON) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 6, CR_MODEL_TENDON) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 1, CR_MODEL_ARC)    \
  CR_SOLVE_N_INSTANTIATE(extern, T, 2, CR_MODEL_ARC)    \
  CR_SOLVE_N_INSTANTIATE(extern, T, 3, CR_MODEL_ARC)    \
  CR_SOLVE_N_INSTANTIATE(extern, T, 4, CR_MODEL_ARC)    \
  CR_SOLVE_N_INSTANTIATE(extern, T, 1, CR_MODEL_COUPLED) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 2, CR_MODEL_COUPLED) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 3, CR_MODEL_COUPLED) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 4, CR_MODEL_COUPLED) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 5, CR_MODEL_COUPLED) \
  CR_SOLVE_N_INSTANTIATE(extern, T, 6, CR_MODEL_COUPLED)

#define CR_SOLVE_INSTANTIATE(EXT, T)                                \
  EXT template cr_status launch_solve_ik<T>(const SolveArgs&, int); \
  EXT template cr_status launch_lm_steps<T>(const SolveArgs&);      \
  EXT template cr_status launch_pg_steps<T>(const SolveArgs&);      \
  EXT template cr_status launch_seeds<T>(const SolveArgs&);         \
  EXT template cr_status launch_topk<T>(const SolveArgs&);

}  // namespace crk
