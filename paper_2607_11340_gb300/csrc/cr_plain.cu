// The plain GPU form of Algorithm 1, kept as a comparator: FP64 throughout, one launch per target,
// every iterate stored back to global memory as an array of structures after each step, SelectTop
// and argmin by a single thread. Same mathematics and outputs as cr_solve_ik.
#include "cr_solve_impl.cuh"

namespace crk {

template <int N, bool OBST>
__global__ void __launch_bounds__(256) k_plain_ik(RobotK<double> rb, WeightsK<double> w, IkArgs<double> a,
                                                   int64_t p, double* U, double* G, double* Fs, double* Cs,
                                                   double* alphas, int* sel) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ObsK<double> sph(nullptr);
  const int nob = a.no + a.np;
  if (OBST) {
    sph = stage_problem_obstacles(a, p, rb, w.delta, smem_raw);
    __syncthreads();
  }
  const int S = a.S, K = a.K;
  const int s = threadIdx.x;
  TargetK<double> tg = load_target<double>(a.targets, a.P, p, a.kind);
  if (s < S) {
    double u[D];
    draw_seed<double, N>(a.seed, (uint64_t)(a.p0 + p), (uint64_t)s, 0, a.box.umax, u);
    if (OBST && nob > 0)
      for (int att = 1; att < 8; ++att) {
        if (!state_collides<double, N>(rb, sph, nob, u)) break;
        draw_seed<double, N>(a.seed, (uint64_t)(a.p0 + p), (uint64_t)s, att, a.box.umax, u);
      }
    double g[D], coll;
    Fs[s] = eval_ik<double, N, OBST, true, false>(rb, w, a.kind, tg, sph, nob, u, g, nullptr, nullptr, &coll);
    for (int q = 0; q < D; ++q) { U[s * D + q] = u[q]; G[s * D + q] = g[q]; }
    Cs[s] = coll;
    alphas[s] = double(a.alpha0);
    for (int it = 0; it < a.k_init; ++it) {
      // the iterate, its gradient, cost and step length round-trip through global memory every step
      double uu[D], gg[D], F = Fs[s], cl = Cs[s], al = alphas[s];
      for (int q = 0; q < D; ++q) { uu[q] = U[s * D + q]; gg[q] = G[s * D + q]; }
      pg_step<double, N, OBST>(rb, w, a.kind, tg, sph, nob, uu, gg, F, cl, al);
      for (int q = 0; q < D; ++q) { U[s * D + q] = uu[q]; G[s * D + q] = gg[q]; }
      Fs[s] = F;
      Cs[s] = cl;
      alphas[s] = al;
    }
  }
  __syncthreads();
  if (s == 0) {
    // SelectTop: repeated scans for the lexicographic minimum of (cost, coll, index)
    int kept = 0, nskip = 0;
    int* skipped = sel + 32;
    unsigned char* taken = reinterpret_cast<unsigned char*>(skipped + S);
    for (int i = 0; i < S; ++i) taken[i] = 0;
    for (int round = 0; round < S && kept < K; ++round) {
      int bi = -1;
      float bc = INFINITY, bl = INFINITY;
      for (int i = 0; i < S; ++i) {
        if (taken[i]) continue;
        float c = float(Fs[i]), l = float(Cs[i]);
        c = isfinite(c) ? c : INFINITY;
        l = isfinite(l) ? l : INFINITY;
        if (bi < 0 || key_less(c, l, i, bc, bl, bi)) { bc = c; bl = l; bi = i; }
      }
      taken[bi] = 1;
      bool dup = false;
      for (int k = 0; k < kept && !dup; ++k) {
        double m = 0;
        for (int q = 0; q < D; ++q) m = fmax(m, fabs(U[bi * D + q] - U[sel[k] * D + q]));
        dup = m < double(a.eps);
      }
      if (dup) skipped[nskip++] = bi;
      else sel[kept++] = bi;
    }
    for (int q = 0; kept < K && q < nskip; ++q) sel[kept++] = skipped[q];
    for (int k = kept; k < K; ++k) sel[k] = -1;
  }
  __syncthreads();
  const int64_t PK = a.P * K;
  if (s < K) {
    const int64_t c = p * K + s;
    int j = sel[s];
    double u[D];
    for (int q = 0; q < D; ++q) u[q] = j >= 0 ? U[j * D + q] : NAN;
    double F = NAN, pos = NAN, rot = NAN;
    unsigned char flags = 0;
    if (j >= 0) {
      double lam = a.lambda0, nu = 2.0, Fi;
      for (int it = 0; it < a.k_final; ++it) {
        lm_iteration<double, N, OBST>(rb, w, a.kind, tg, sph, nob, u, lam, nu, Fi);
        for (int q = 0; q < D; ++q) a.cand_u64[q * PK + c] = u[q];
      }
      F = accept_fp64<N, OBST>(rb, w, a.kind, tg, sph, nob, u, a.lim_tol, pos, rot, flags);
    }
    for (int q = 0; q < D; ++q) a.cand_u64[q * PK + c] = u[q];
    a.cand_F[c] = F;
    a.cand_pos[c] = pos;
    a.cand_rot[c] = rot;
    a.cand_flag[c] = flags;
  }
}

template <int N> cr_status plain_n(const SolveArgs& sa) {
  RobotK<double> rb = crh::robot_k<double>(sa.robot);
  WeightsK<double> w = crh::weights_k<double>(sa.task.w);
  IkArgs<double> a = ik_args<double>(sa);
  unsigned char* ws = (unsigned char*)sa.ws;
  double* U = (double*)(ws + sa.lay.plain_u);
  double* G = (double*)(ws + sa.lay.plain_g);
  double* Fs = (double*)(ws + sa.lay.plain_F);
  double* Cs = Fs + a.S;
  double* alphas = Cs + a.S;
  int* sel = (int*)(alphas + a.S);
  // sel[32] | skipped[S] | taken[S] live after the three double arrays
  const int threads = ((a.S + 31) / 32) * 32;
  size_t sm = obstacles_smem<double>(a.no, a.np);  // at most 45 KB (CR_MAX_SPHERES obstacles)
  for (int64_t p = 0; p < a.P; ++p) {
    if (a.no + a.np > 0) k_plain_ik<N, true><<<1, threads, sm, sa.stream>>>(rb, w, a, p, U, G, Fs, Cs, alphas, sel);
    else k_plain_ik<N, false><<<1, threads, sm, sa.stream>>>(rb, w, a, p, U, G, Fs, Cs, alphas, sel);
    cr_status st = crh::check_launch("cr_solve_ik_plain");
    if (st) return st;
  }
  k_ik_argmin<N><<<grid1(a.P, 128), 128, 0, sa.stream>>>(a.P, a.K, a.pos_tol, a.rot_tol, a.cand_u64, a.cand_F,
                                                         a.cand_pos, a.cand_rot, a.cand_flag, a.u_out,
                                                         a.cost_out, a.pos_out, a.rot_out, a.success, a.status);
  return crh::check_launch("cr_solve_ik_plain argmin");
}

}  // namespace crk

using namespace crh;

extern "C" cr_status cr_solve_ik_plain(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                                       const cr_ik_params* prm, double* u_out, double* cost_out,
                                       double* pos_err, double* rot_err, uint8_t* success, void* workspace,
                                       size_t ws_bytes, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "cr_solve_ik_plain")) ||
      (st = check_scene(scene)))
    return st;
  if (!prm || !task) return fail(CR_EINVAL, "NULL params / task");
  if ((st = check_self_rows(task->w, false, "cr_solve_ik_plain"))) return st;
  if (prm->S < 1 || prm->S > CR_MAX_SEEDS || prm->n_final < 1 || prm->n_final > 32 || prm->n_final > prm->S ||
      prm->k_init < 0 || prm->k_final < 0)
    return fail(CR_EINVAL, "cr_solve_ik_plain: bad params");
  cr_task t = *task;
  t.seeds_per_target = 1;
  if ((st = check_task(&t, t.n_targets))) return st;
  if (t.n_targets == 0) return CR_OK;
  if ((st = check_ptr(u_out, 8, "u_out", true)) || (st = check_ptr(cost_out, 8, "cost_out", true)) ||
      (st = check_ptr(pos_err, 8, "pos_err", true)) || (st = check_ptr(rot_err, 8, "rot_err", true)) ||
      (st = check_ptr(success, 1, "success", true)) || (st = check_ptr(workspace, 256, "workspace", true)))
    return st;
  cr_ik_params p64 = *prm;
  p64.precision = CR_F64;
  IkLayout lay = ik_layout(*robot, t.n_targets, p64);
  if (ws_bytes < lay.total) return fail(CR_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, lay.total);
  crk::SolveArgs a{};
  a.robot = *robot;
  if (scene) a.scene = *scene;
  a.task = t;
  a.prm = p64;
  a.ws = workspace;
  a.lay = lay;
  a.u_out = u_out;
  a.cost_out = cost_out;
  a.pos = pos_err;
  a.rot = rot_err;
  a.success = success;
  a.stream = stream_of(stream);
  cudaError_t e = cudaMemsetAsync((unsigned char*)workspace + lay.status, 0, sizeof(int32_t), a.stream);
  if (e != cudaSuccess) return fail(CR_ECUDA, "cr_solve_ik_plain: %s", cudaGetErrorString(e));
  switch (robot->n) {
    case 1: return crk::plain_n<1>(a);
    case 2: return crk::plain_n<2>(a);
    case 3: return crk::plain_n<3>(a);
    case 4: return crk::plain_n<4>(a);
    case 5: return crk::plain_n<5>(a);
    default: return crk::plain_n<6>(a);
  }
}
