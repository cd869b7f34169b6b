// Ragged batch: IK and path-following problems of mixed segment count n, waypoint count H, seed
// count S and obstacle count n_o (the batched form of Algorithm 1 and of the path pipeline of
// Sec. IV, for serving).
//
// Per segment count, four kernels run one after the other on one branch of the batch's CUDA graph,
// each a set of persistent warps popping work with one atomic from its own queue (queue order =
// longest estimated item first), so that the warps of one kernel all run one phase of the method:
//  k_batch_seeds:  work unit = seed group g of item i (seeds [g spu, (g + 1) spu) of the item's
//                  (first-waypoint) IK): sampling and the k_init projected-gradient steps, lanes
//                  over seeds; the end states go to the item's candidate block;
//  k_batch_refine: per item, SelectTop, the k_final LM refinement of the kept candidates (lanes
//                  over candidates, FP64 Cholesky), the FP64 argmin and acceptance; an IK item is
//                  finished here, a path item leaves waypoint 0's state in its exploration buffer;
//  k_batch_warm:   per path item, the exploration sweep (warm-started LM per waypoint) into the
//                  buffer;
//  k_batch_joint:  per path item, the joint LM over the waypoints, the FP64 acceptance of every
//                  waypoint and the outputs.
// No warp waits for another. The segment counts run as parallel branches, behind a node that
// zeroes the queue heads and stamps the batch start (%globaltimer); every item records its
// completion time.
#pragma once

#include "cr_path_impl.cuh"

namespace crk {

struct BatchItemK {
  int32_t kind, H, S, no, G, item;  // item: index in the caller's order (seed counter, outputs)
  int64_t wp;                       // first waypoint: column of targets [7][W], index into pos/rot
  int64_t sph;                      // first sphere of the item in spheres [*][4]
  int64_t st;                       // first double of the item's states in u_out ([D][H])
  int64_t cand;                     // first float of the item's candidates: u [D][S], F [S], C [S]
  int64_t xs;                       // path items: first float of the exploration states [D][H] in xbuf
};

struct BatchArgs {
  const BatchItemK* items;  // items of this segment count, queue order
  int32_t n_items;
  const int2* units;        // (item slot, seed group), queue order
  int32_t n_units;
  int32_t* head;            // queue heads (zeroed by the start node): units, then the items of the
                            // refine, exploration and joint phases
  float* xbuf;              // exploration states of the path items
  const unsigned long long* t0;
  const double* targets;    // [7][W]
  int64_t W;
  const double* spheres;    // [*][4]
  float* cand;
  unsigned char* scratch;   // per worker warp of the joint phase: path buffers
  size_t scratch_stride;
  int32_t hmax;             // waypoints the path buffers hold
  int32_t spu;              // seeds per unit
  int32_t K, k_init, k_final;
  float alpha0, eps;
  double lambda0, lim_tol, pos_tol, rot_tol;
  double umax[NMAX];
  uint64_t seed;
  int64_t p0;
  int32_t k_warm, k_joint;
  double w_s;
  double* u_out;
  double* cost;
  double* pos;
  double* rot;
  unsigned char* flags;
  unsigned long long* t_done;
};

constexpr int kBatchWarps = 4;         // warps per CTA (independent workers)
constexpr int kBatchMaxSpheres = 64;   // obstacles per item
constexpr size_t kBatchWarpSmem = 6144;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Path buffers of one worker for H waypoints (byte offsets): X0, X1 [D][H] (bulk), Af [H][DD]
// (bulk), g, z [H][D] and the swept blocks Zg [H][aug_stride] (FP64).
struct PathScratch {
  size_t x0, x1, af, g, z, zg, total;
};
__host__ __device__ inline PathScratch path_scratch(int D, int H) {
  PathScratch p;
  const int DD = D * (D + 1) / 2, ZS = ((D + 1) * (D + 2) / 2 + 31) / 32 * 32;
  size_t off = 0;
  p.x0 = off; off += (size_t)4 * D * H;
  p.x1 = off; off += (size_t)4 * D * H;
  p.af = off; off += (size_t)4 * DD * H;
  off = (off + 15) & ~size_t(15);
  p.g = off; off += (size_t)8 * D * H;
  p.z = off; off += (size_t)8 * D * H;
  p.zg = off; off += (size_t)8 * ZS * H;
  p.total = (off + 255) & ~size_t(255);
  return p;
}

template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Joint cost of the path states X ([D][H]) with the smoothness rows, summed over the warp.
template <int N>
__device__ double path_cost_warp(const RobotK<float>& rb, const WeightsK<float>& w, const double* targets, int64_t W,
                                 int64_t wp0, int H, const Sphere4<float>* sph, int no, double ws, const float* X) {
  constexpr int D = 3 * N;
  const int lane = threadIdx.x & 31;
  double Fl = 0.0;
  for (int t = lane; t < H; t += 32) {
    float u[D], dummy[D];
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = X[q * H + t];
    const TargetK<float> tg = load_target<float>(targets, W, wp0 + t, CR_TASK_IK6);
    Fl += double(eval_ik<float, N, true, false, false>(rb, w, CR_TASK_IK6, tg, sph, no, u, dummy, nullptr, nullptr,
                                                        nullptr));
    if (t >= 1) {
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const double dq = double(u[q]) - double(X[q * H + t - 1]);
        Fl += 0.5 * ws * dq * dq;
      }
    }
  }
  return warp_sum(Fl);
}

// Joint LM over the path (the refinement of k_path_joint) by one warp: waypoints over the lanes in
// rounds of 32, the block system solved by joint_solve_warp. X0 holds the exploration states on
// entry; returns the final joint cost and sets cur to the buffer holding the result.
template <int N>
__device__ double joint_lm_warp(const RobotK<float>& rb, const WeightsK<float>& w, const double* targets, int64_t W,
                                int64_t wp0, int H, const Sphere4<float>* sph, int no, int k_joint, double lam0,
                                double ws, unsigned char* scr, double* col, double* colr, double* Zs, int& cur) {
  constexpr int D = 3 * N, DD = D * (D + 1) / 2;
  const int lane = threadIdx.x & 31;
  const PathScratch ps = path_scratch(D, H);
  float* X0 = reinterpret_cast<float*>(scr + ps.x0);
  float* X1 = reinterpret_cast<float*>(scr + ps.x1);
  float* Af = reinterpret_cast<float*>(scr + ps.af);
  double* g = reinterpret_cast<double*>(scr + ps.g);
  double* z = reinterpret_cast<double*>(scr + ps.z);
  double* Zg = reinterpret_cast<double*>(scr + ps.zg);
  double lam = lam0, nu = 2.0;
  cur = 0;
  for (int itn = 0; itn < k_joint; ++itn) {
    float* Xc = cur ? X1 : X0;
    float* Xn = cur ? X0 : X1;
    double Fl = 0.0;
    for (int t = lane; t < H; t += 32) {
      float u[D], gt[D];
#pragma unroll
      for (int q = 0; q < D; ++q) u[q] = Xc[q * H + t];
      const TargetK<float> tg = load_target<float>(targets, W, wp0 + t, CR_TASK_IK6);
      float At[DD];
      Fl += double(eval_ik_normal<float, float, N, true>(rb, w, CR_TASK_IK6, tg, sph, no, u, At, gt));
#pragma unroll
      for (int e = 0; e < DD; ++e) Af[(size_t)t * DD + e] = At[e];
#pragma unroll
      for (int q = 0; q < D; ++q) g[t * D + q] = double(gt[q]);
    }
    __syncwarp();
    for (int t = lane; t < H; t += 32) {
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const double uq = double(Xc[q * H + t]);
        double s = 0.0;
        if (t > 0) {
          const double dq = uq - double(Xc[q * H + t - 1]);
          s += ws * dq;
          Fl += 0.5 * ws * dq * dq;
        }
        if (t + 1 < H) s -= ws * (double(Xc[q * H + t + 1]) - uq);
        g[t * D + q] += s;
      }
    }
    const double F = warp_sum(Fl);
    __syncwarp();
    if (!joint_solve_warp<float, D>(Af, g, z, Zg, col, colr, Zs, H, ws, lam)) {
      lam *= nu;
      nu *= 2.0;
      continue;
    }
    double predl = 0.0;
    for (int t = lane; t < H; t += 32) {
      const double nb = double((t > 0) + (t + 1 < H));
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const double xq = z[t * D + q];
        const double dg = fmax(double(Af[(size_t)t * DD + tri(q, q)]) + ws * nb, 1e-12);
        predl += xq * (lam * dg * xq - g[t * D + q]);
        Xn[q * H + t] = Xc[q * H + t] + float(xq);
      }
    }
    const double pred = 0.5 * warp_sum(predl);
    __syncwarp();
    const double Fn = path_cost_warp<N>(rb, w, targets, W, wp0, H, sph, no, ws, Xn);
    if (Fn < F) {
      const double rho = (F - Fn) / pred, tt = 2.0 * rho - 1.0;
      lam *= fmax(1.0 / 3.0, 1.0 - tt * tt * tt);
      nu = 2.0;
      cur ^= 1;
    } else {
      lam *= nu;
      nu *= 2.0;
    }
    __syncwarp();
  }
  return path_cost_warp<N>(rb, w, targets, W, wp0, H, sph, no, ws, cur ? X1 : X0);
}

// Per-warp shared layout of the phase kernels (kBatchWarpSmem bytes).
struct BatchSmem {
  Sphere4<float>* sph;     // 64 x 16
  Sphere4<double>* sphd;   // 64 x 32
  float* wsc;              // 4 x 32 floats
  double *col, *colr, *Zs; // 32, 32, up to 171 (D = 18)
  int* sel;                // 32
  unsigned char* taken;    // 256
  double* bst;             // 32
};
__device__ inline BatchSmem batch_smem_of(unsigned char* smem_raw) {
  unsigned char* sm = smem_raw + (size_t)(threadIdx.x >> 5) * kBatchWarpSmem;
  BatchSmem b;
  b.sph = reinterpret_cast<Sphere4<float>*>(sm);
  b.sphd = reinterpret_cast<Sphere4<double>*>(sm + 1024);
  b.wsc = reinterpret_cast<float*>(sm + 3072);
  b.col = reinterpret_cast<double*>(sm + 3584);
  b.colr = b.col + 32;
  b.Zs = b.colr + 32;
  b.sel = reinterpret_cast<int*>(sm + 5472);
  b.taken = sm + 5600;
  b.bst = reinterpret_cast<double*>(sm + 5856);
  return b;
}

// The item's spheres in shared memory with their reach (r_s + r_body + delta), bulk and FP64 copies.
__device__ inline void batch_spheres(const BatchArgs& a, const BatchItemK& it, const RobotK<float>& rb,
                                     const WeightsK<float>& w, Sphere4<float>* sph) {
  const int lane = threadIdx.x & 31;
  const double* sp = a.spheres + it.sph * 4;
  for (int j = lane; j < it.no; j += 32) {
    Sphere4<float> s;
    s.x = float(sp[4 * j]); s.y = float(sp[4 * j + 1]); s.z = float(sp[4 * j + 2]);
    s.reach = float(sp[4 * j + 3]) + rb.rbody + w.delta;
    sph[j] = s;
  }
}
__device__ inline void batch_spheres_d(const BatchArgs& a, const BatchItemK& it, const RobotK<double>& rbd,
                                       const WeightsK<double>& wd, Sphere4<double>* sphd) {
  const int lane = threadIdx.x & 31;
  const double* sp = a.spheres + it.sph * 4;
  for (int j = lane; j < it.no; j += 32) {
    Sphere4<double> s;
    s.x = sp[4 * j]; s.y = sp[4 * j + 1]; s.z = sp[4 * j + 2];
    s.reach = sp[4 * j + 3] + rbd.rbody + wd.delta;
    sphd[j] = s;
  }
}

// The next entry of a queue (the same for every lane), or -1 when it is exhausted.
__device__ inline int batch_pop(int32_t* head, int n) {
  int u = 0;
  if ((threadIdx.x & 31) == 0) u = atomicAdd(head, 1);
  u = __shfl_sync(0xffffffffu, u, 0);
  return u < n ? u : -1;
}

__device__ inline bool batch_is_path(const BatchItemK& it) { return it.kind == CR_ITEM_PATH && it.H > 1; }

// Register budgets of the seeds phase, picked by the planner's timing: RB = 0 the wide cap, RB = 1 a
// tight one (more resident warps per SM, at the price of spills where the state does not fit).
constexpr int batch_seeds_regs(int n, int rb) { return rb == 0 ? (n <= 4 ? 168 : 255) : (n <= 4 ? 128 : 168); }

// Phase 1: stage one of the work units (seed groups), lanes over seeds.
template <int N, int RB = 0>
__global__ void __maxnreg__(batch_seeds_regs(N, RB)) k_batch_seeds(RobotK<float> rb, WeightsK<float> w, BatchArgs a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchSmem b = batch_smem_of(smem_raw);
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int u = batch_pop(a.head, a.n_units);
    if (u < 0) break;
    const int2 un = a.units[u];
    const BatchItemK it = a.items[un.x];
    batch_spheres(a, it, rb, w, b.sph);
    __syncwarp();
    const TargetK<float> tg = load_target<float>(a.targets, a.W, it.wp, CR_TASK_IK6);
    float* cu = a.cand + it.cand;
    float* cF = cu + (size_t)D * it.S;
    float* cC = cF + it.S;
    const int s_end = (un.y + 1) * a.spu < it.S ? (un.y + 1) * a.spu : it.S;
    for (int s = un.y * a.spu + lane; s < s_end; s += 32) {
      float uu[D], g[D], coll = 0.f;
      draw_seed<float, N>(a.seed, (uint64_t)(a.p0 + it.item), (uint64_t)s, 0, a.umax, uu);
      for (int att = 1; att < 8 && it.no > 0; ++att) {
        if (!state_collides<float, N>(rb, b.sph, it.no, uu)) break;
        draw_seed<float, N>(a.seed, (uint64_t)(a.p0 + it.item), (uint64_t)s, att, a.umax, uu);
      }
      float F = eval_ik<float, N, true, true, false>(rb, w, CR_TASK_IK6, tg, b.sph, it.no, uu, g, nullptr, nullptr,
                                                      &coll);
      float alpha = a.alpha0;
      for (int k = 0; k < a.k_init; ++k)
        pg_step<float, N, true>(rb, w, CR_TASK_IK6, tg, b.sph, it.no, uu, g, F, coll, alpha);
      cF[s] = F;
      cC[s] = coll;
#pragma unroll
      for (int q = 0; q < D; ++q) cu[(size_t)q * it.S + s] = uu[q];
    }
    __syncwarp();
  }
}

// Phase 2: SelectTop, refinement, argmin and the outputs of an IK item; a path item's waypoint-0
// state goes to its exploration buffer (NaN there marks an item without any finite candidate).
template <int N>
__global__ void __maxnreg__(255)
    k_batch_refine(RobotK<float> rb, WeightsK<float> w, RobotK<double> rbd, WeightsK<double> wd, BatchArgs a) {
  constexpr int D = 3 * N;
  const unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchSmem b = batch_smem_of(smem_raw);
  const int lane = threadIdx.x & 31;
  for (;;) {
    const int i = batch_pop(a.head + 1, a.n_items);
    if (i < 0) break;
    const BatchItemK it = a.items[i];
    batch_spheres(a, it, rb, w, b.sph);
    batch_spheres_d(a, it, rbd, wd, b.sphd);
    const int S = it.S, K = S < a.K ? S : a.K;
    const float* cu = a.cand + it.cand;
    const float* cF = cu + (size_t)D * S;
    const float* cC = cF + S;
    __syncwarp();
    warp_topk<float, true>(cF, cC, cu, S, D, S, K, a.eps, b.sel, b.taken, nullptr);
    double Fk = NAN, pos = NAN, rot = NAN;
    unsigned char fl = 0;
    double ud[D];
#pragma unroll
    for (int q = 0; q < D; ++q) ud[q] = NAN;
    const TargetK<float> tg = load_target<float>(a.targets, a.W, it.wp, CR_TASK_IK6);
    const TargetK<double> tgd = load_target<double>(a.targets, a.W, it.wp, CR_TASK_IK6);
    // lane k refines candidate sel[k]: k_final LM iterations, FP64 Cholesky in registers
    const int j = lane < K ? b.sel[lane] : -1;
    if (j >= 0) {
      float uu[D];
#pragma unroll
      for (int q = 0; q < D; ++q) uu[q] = __ldcg(cu + q * S + j);
      if (c_finite(uu[0])) {
        double lam = a.lambda0, nu = 2.0;
        float Fi;
        for (int itn = 0; itn < a.k_final; ++itn)
          lm_iteration<float, N, true>(rb, w, CR_TASK_IK6, tg, b.sph, it.no, uu, lam, nu, Fi);
#pragma unroll
        for (int q = 0; q < D; ++q) ud[q] = double(uu[q]);
        Fk = accept_fp64<N, true>(rbd, wd, CR_TASK_IK6, tgd, b.sphd, it.no, ud, a.lim_tol, pos, rot, fl);
      }
    }
    // argmin of the FP64 cost (first minimum in candidate order; costs <= CR_ARGMIN_TIE count as 0)
    double bkey = isfinite(Fk) ? (Fk <= CR_ARGMIN_TIE ? 0.0 : Fk) : INFINITY;
    int bk = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double oF = __shfl_xor_sync(FULL, bkey, off);
      const int ok = __shfl_xor_sync(FULL, bk, off);
      if (oF < bkey || (oF == bkey && ok < bk)) { bkey = oF; bk = ok; }
    }
    const bool found = bkey < INFINITY;
    const double bF = __shfl_sync(FULL, Fk, bk & 31);
    if (lane == bk) {
#pragma unroll
      for (int q = 0; q < D; ++q) b.bst[q] = ud[q];
    }
    const double bpos = __shfl_sync(FULL, pos, bk & 31), brot = __shfl_sync(FULL, rot, bk & 31);
    const unsigned bfl = __shfl_sync(FULL, (unsigned)fl, bk & 31);
    __syncwarp();
    const bool path = batch_is_path(it);
    if (!found) {
      for (int e = lane; e < D * it.H; e += 32) a.u_out[it.st + e] = NAN;
      for (int t = lane; t < it.H; t += 32) { a.pos[it.wp + t] = NAN; a.rot[it.wp + t] = NAN; }
      if (path && lane == 0) a.xbuf[it.xs] = NAN;
      if (lane == 0) {
        a.cost[it.item] = NAN;
        a.flags[it.item] = 0;
        a.t_done[it.item] = global_ns() - *a.t0;
      }
    } else if (!path) {
      if (lane < D) a.u_out[it.st + lane] = b.bst[lane];
      if (lane == 0) {
        a.cost[it.item] = bF;
        a.pos[it.wp] = bpos;
        a.rot[it.wp] = brot;
        const bool lim = bfl & 1, col_ok = bfl & 2;
        const bool succ = bpos <= a.pos_tol && brot <= a.rot_tol && lim && col_ok;
        a.flags[it.item] = (unsigned char)((succ ? 1 : 0) | (lim ? 2 : 0) | (col_ok ? 4 : 0));
        a.t_done[it.item] = global_ns() - *a.t0;
      }
    } else if (lane < D) {
      a.xbuf[it.xs + (int64_t)lane * it.H] = float(b.bst[lane]);
    }
    __syncwarp();
  }
}

// Phase 3: the exploration sweep of every path item (waypoint t from the state of t - 1).
template <int N>
__global__ void __maxnreg__(255)
    k_batch_warm(RobotK<float> rb, WeightsK<float> w, BatchArgs a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchSmem b = batch_smem_of(smem_raw);
  for (;;) {
    const int i = batch_pop(a.head + 2, a.n_items);
    if (i < 0) break;
    const BatchItemK it = a.items[i];
    if (!batch_is_path(it)) continue;
    float* X = a.xbuf + it.xs;
    if (!c_finite(__ldcg(X))) continue;  // no candidate: the refine phase wrote the outputs
    batch_spheres(a, it, rb, w, b.sph);
    __syncwarp();
    float u[D];
#pragma unroll
    for (int q = 0; q < D; ++q) u[q] = __ldcg(X + (int64_t)q * it.H);
    warm_sweep_warp<float, N, true>(rb, w, a.targets, a.W, it.wp, it.H, a.k_warm, float(a.lambda0), b.sph, it.no, u,
                                    b.wsc, X, it.H);
    __syncwarp();
  }
}

// Phase 4: the joint LM of every path item, its FP64 acceptance and outputs.
template <int N>
__global__ void __maxnreg__(255)
    k_batch_joint(RobotK<float> rb, WeightsK<float> w, RobotK<double> rbd, WeightsK<double> wd, BatchArgs a) {
  constexpr int D = 3 * N;
  const unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchSmem b = batch_smem_of(smem_raw);
  const int lane = threadIdx.x & 31;
  const int64_t worker = (int64_t)blockIdx.x * kBatchWarps + (threadIdx.x >> 5);
  unsigned char* scr = a.scratch + worker * a.scratch_stride;
  for (;;) {
    const int i = batch_pop(a.head + 3, a.n_items);
    if (i < 0) break;
    const BatchItemK it = a.items[i];
    if (!batch_is_path(it)) continue;
    const float* Xi = a.xbuf + it.xs;
    if (!c_finite(__ldcg(Xi))) continue;
    batch_spheres(a, it, rb, w, b.sph);
    batch_spheres_d(a, it, rbd, wd, b.sphd);
    const int H = it.H;
    const PathScratch ps = path_scratch(D, H);
    float* X0 = reinterpret_cast<float*>(scr + ps.x0);
    for (int e = lane; e < D * H; e += 32) X0[e] = __ldcg(Xi + e);
    __syncwarp();
    int cur = 0;
    const double Ff = joint_lm_warp<N>(rb, w, a.targets, a.W, it.wp, H, b.sph, it.no, a.k_joint, a.lambda0, a.w_s,
                                       scr, b.col, b.colr, b.Zs, cur);
    const float* X = reinterpret_cast<const float*>(scr + (cur ? ps.x1 : ps.x0));
    bool all_succ = true, all_lim = true, all_col = true;
    for (int t = lane; t < H; t += 32) {
      double uw[D];
#pragma unroll
      for (int q = 0; q < D; ++q) {
        uw[q] = double(X[q * H + t]);
        a.u_out[it.st + q * H + t] = uw[q];
      }
      const TargetK<double> tgd = load_target<double>(a.targets, a.W, it.wp + t, CR_TASK_IK6);
      double pw, rw;
      unsigned char f;
      accept_fp64<N, true>(rbd, wd, CR_TASK_IK6, tgd, b.sphd, it.no, uw, a.lim_tol, pw, rw, f);
      a.pos[it.wp + t] = pw;
      a.rot[it.wp + t] = rw;
      all_lim = all_lim && (f & 1);
      all_col = all_col && (f & 2);
      all_succ = all_succ && pw <= a.pos_tol && rw <= a.rot_tol;
    }
    all_lim = __all_sync(FULL, all_lim);
    all_col = __all_sync(FULL, all_col);
    all_succ = __all_sync(FULL, all_succ) && all_lim && all_col;
    if (lane == 0) {
      a.cost[it.item] = Ff;
      a.flags[it.item] = (unsigned char)((all_succ ? 1 : 0) | (all_lim ? 2 : 0) | (all_col ? 4 : 0));
      a.t_done[it.item] = global_ns() - *a.t0;
    }
    __syncwarp();
  }
}

// Host wrappers per segment count (each instantiated in its own translation unit). phase: 0 seeds,
// 1 refine, 2 exploration, 3 joint.
struct BatchGrids {
  int g[4];
};
template <int N> cr_status batch_prepare(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_seeds<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_seeds<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_refine<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_warm<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_joint<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return crh::fail(CR_ECUDA, "k_batch phases <%d>: %s", N, cudaGetErrorString(e));
  return CR_OK;
}
template <int N> int batch_blocks_per_sm(size_t smem, int phase, int rb) {
  int nb = 0;
  cudaError_t e;
  switch (phase) {
    case 0:
      e = rb == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_seeds<N, 0>, 32 * kBatchWarps, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_seeds<N, 1>, 32 * kBatchWarps, smem);
      break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_refine<N>, 32 * kBatchWarps, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_warm<N>, 32 * kBatchWarps, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_joint<N>, 32 * kBatchWarps, smem);
  }
  return e == cudaSuccess ? nb : 0;
}
template <int N> cr_status batch_launch(const cr_robot& family, const cr_weights& wts, const BatchArgs& a,
                                        const BatchGrids& gr, size_t smem, int rb_seeds, cudaStream_t s) {
  cr_robot r = family;
  r.n = N;
  const RobotK<float> rb = crh::robot_k<float>(r);
  const WeightsK<float> w = crh::weights_k<float>(wts);
  const RobotK<double> rbd = crh::robot_k<double>(r);
  const WeightsK<double> wd = crh::weights_k<double>(wts);
  const unsigned bs = 32 * kBatchWarps;
  if (gr.g[0] > 0) {
    if (rb_seeds == 0) k_batch_seeds<N, 0><<<gr.g[0], bs, smem, s>>>(rb, w, a);
    else k_batch_seeds<N, 1><<<gr.g[0], bs, smem, s>>>(rb, w, a);
  }
  if (gr.g[1] > 0) k_batch_refine<N><<<gr.g[1], bs, smem, s>>>(rb, w, rbd, wd, a);
  if (gr.g[2] > 0) k_batch_warm<N><<<gr.g[2], bs, smem, s>>>(rb, w, a);
  if (gr.g[3] > 0) k_batch_joint<N><<<gr.g[3], bs, smem, s>>>(rb, w, rbd, wd, a);
  return crh::check_launch("k_batch phases");
}

#define CR_BATCH_INSTANTIATE(EXT, N)                                                                               \
  EXT template cr_status batch_prepare<N>(size_t);                                                                 \
  EXT template int batch_blocks_per_sm<N>(size_t, int, int);                                                       \
  EXT template cr_status batch_launch<N>(const cr_robot&, const cr_weights&, const BatchArgs&, const BatchGrids&, \
                                         size_t, int, cudaStream_t);

}  // namespace crk
