// C ABI of the PRM exploration of Algorithm 2: cr_prm_workspace_size, cr_prm_build, cr_prm_query.
#include "cr_prm_impl.cuh"

namespace crk {
CR_PRM_INSTANTIATE(extern, 1)
CR_PRM_INSTANTIATE(extern, 2)
CR_PRM_INSTANTIATE(extern, 3)
CR_PRM_INSTANTIATE(extern, 4)
CR_PRM_INSTANTIATE(extern, 5)
CR_PRM_INSTANTIATE(extern, 6)
}  // namespace crk

using namespace crh;

static_assert(crk::kPrmMaxN == CR_PRM_MAX_N && crk::kPrmMaxK == CR_PRM_MAX_K &&
                  crk::kPrmMaxCheck == CR_PRM_MAX_CHECK && crk::kPrmMaxAttempts == CR_PRM_MAX_ATTEMPTS,
              "PRM limits of the header and the kernels");
static_assert(CR_PRM_MAX_N <= 1024, "k_prm_csr runs one thread per node in one block");

namespace {

// Workspace of cr_prm_build: blocked flags [R*N*k] | adjacency bitset [R][N][ceil(N/32)] (uint32) |
// FP32 copy of the nodes [3n][R*N].
struct PrmWs {
  size_t blocked, adj, nodes32, total;
};
PrmWs prm_ws(int n, int64_t R, const cr_prm_params& p) {
  PrmWs w;
  size_t off = 0;
  w.blocked = off; off = align256(off + (size_t)R * p.N * p.k);
  w.adj = off; off = align256(off + (size_t)R * p.N * crk::prm_words(p.N) * 4);
  w.nodes32 = off; off = align256(off + (size_t)3 * n * R * p.N * 4);
  w.total = off;
  return w;
}

cr_status check_prm(const cr_prm_params* p) {
  if (!p) return fail(CR_EINVAL, "prm params are NULL");
  if (p->N < 2 || p->N > CR_PRM_MAX_N) return fail(CR_EINVAL, "prm: N = %d outside 2..%d", p->N, CR_PRM_MAX_N);
  if (p->k < 1 || p->k > CR_PRM_MAX_K || p->k > p->N - 1)
    return fail(CR_EINVAL, "prm: k = %d outside 1..min(%d, N - 1)", p->k, CR_PRM_MAX_K);
  if (p->n_check < 1 || p->n_check > CR_PRM_MAX_CHECK)
    return fail(CR_EINVAL, "prm: n_check = %d outside 1..%d", p->n_check, CR_PRM_MAX_CHECK);
  if (p->attempts < 1 || p->attempts > CR_PRM_MAX_ATTEMPTS)
    return fail(CR_EINVAL, "prm: attempts = %d outside 1..%d", p->attempts, CR_PRM_MAX_ATTEMPTS);
  return CR_OK;
}

cr_status check_map(const cr_roadmap* m, bool build) {
  if (!m) return fail(CR_EINVAL, "roadmap is NULL");
  if (m->R < 1 || m->R > ((int64_t)1 << 24)) return fail(CR_EINVAL, "roadmap: R = %lld outside 1..2^24", (long long)m->R);
  cr_status st;
  if ((st = check_ptr(m->nodes, 8, "roadmap.nodes", true)) || (st = check_ptr(m->node_ok, 1, "roadmap.node_ok", true)) ||
      (st = check_ptr(m->nbr, 4, "roadmap.nbr", build)) || (st = check_ptr(m->row, 4, "roadmap.row", true)) ||
      (st = check_ptr(m->col, 4, "roadmap.col", true)) || (st = check_ptr(m->wt, 8, "roadmap.wt", true)))
    return st;
  return CR_OK;
}

crk::PrmArgs prm_args(const cr_robot& r, const cr_scene* scene, const cr_weights& w, const cr_prm_params& p,
                      const cr_roadmap& m) {
  crk::PrmArgs a{};
  a.spheres = scene && scene->n_o > 0 ? scene->spheres : nullptr;
  a.no = scene ? scene->n_o : 0;
  a.sph_pp = (scene && scene->per_problem && scene->n_o > 0) ? 1 : 0;
  a.R = m.R;
  a.N = p.N;
  a.k = p.k;
  a.n_check = p.n_check;
  a.attempts = p.attempts;
  a.seed = p.seed;
  for (int i = 0; i < crk::NMAX; ++i) a.umax[i] = i < r.n ? r.u_max[i] : 0.0;
  a.coord_max = 0.0;
  for (int i = 0; i < r.n; ++i) a.coord_max = a.coord_max > r.u_max[i] ? a.coord_max : r.u_max[i];
  a.delta = w.delta;
  a.nodes = m.nodes;
  a.ok = m.node_ok;
  a.nbr = m.nbr;
  a.row = m.row;
  a.col = m.col;
  a.wt = m.wt;
  return a;
}

}  // namespace

extern "C" {

size_t cr_prm_workspace_size(const cr_robot* robot, int64_t R, const cr_prm_params* prm) {
  if (!robot || !prm || R < 1 || check_prm(prm)) return 0;
  return prm_ws(robot->n, R, *prm).total;
}

cr_status cr_prm_build(const cr_robot* robot, const cr_scene* scene, const cr_weights* w, const cr_prm_params* prm,
                       const cr_roadmap* map, void* workspace, size_t ws_bytes, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "the PRM roadmap")) ||
      (st = check_scene_spheres_only(scene, "the PRM roadmap")) || (st = check_prm(prm)) || (st = check_map(map, true)))
    return st;
  if (!w) return fail(CR_EINVAL, "weights are NULL");
  if ((st = check_self_rows(*w, false, "the PRM roadmap and query"))) return st;
  if (map->R > 65535) return fail(CR_EINVAL, "cr_prm_build: R = %lld above 65535", (long long)map->R);
  if ((st = check_ptr(workspace, 256, "workspace", true))) return st;
  const PrmWs lay = prm_ws(robot->n, map->R, *prm);
  if (ws_bytes < lay.total) return fail(CR_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, lay.total);
  crk::PrmArgs a = prm_args(*robot, scene, *w, *prm, *map);
  unsigned char* ws = (unsigned char*)workspace;
  a.blocked = ws + lay.blocked;
  a.adj = reinterpret_cast<uint32_t*>(ws + lay.adj);
  a.nodes32 = reinterpret_cast<float*>(ws + lay.nodes32);
  cudaStream_t s = stream_of(stream);
  cudaError_t e = cudaMemsetAsync(ws, 0, lay.nodes32, s);  // blocked flags and bitset
  if (e != cudaSuccess) return fail(CR_ECUDA, "cr_prm_build: %s", cudaGetErrorString(e));
  switch (robot->n) {
    case 1: return crk::prm_build_n<1>(*robot, a, s);
    case 2: return crk::prm_build_n<2>(*robot, a, s);
    case 3: return crk::prm_build_n<3>(*robot, a, s);
    case 4: return crk::prm_build_n<4>(*robot, a, s);
    case 5: return crk::prm_build_n<5>(*robot, a, s);
    default: return crk::prm_build_n<6>(*robot, a, s);
  }
}

cr_status cr_prm_query(const cr_robot* robot, const cr_scene* scene, const cr_weights* w, const cr_prm_params* prm,
                       const cr_roadmap* map, const double* u_start, const double* u_goal, int64_t P, int32_t T,
                       double* X, double* length, int32_t* hops, cr_stream stream) {
  cr_status st;
  if ((st = check_robot(robot)) || (st = check_tendon_model(robot, "the PRM query")) ||
      (st = check_scene_spheres_only(scene, "the PRM query")) || (st = check_prm(prm)) || (st = check_map(map, false)))
    return st;
  if (!w) return fail(CR_EINVAL, "weights are NULL");
  if ((st = check_self_rows(*w, false, "the PRM roadmap and query"))) return st;
  if (P < 0 || P > ((int64_t)1 << 31) - 1) return fail(CR_EINVAL, "prm query: P = %lld", (long long)P);
  if (T < 2 || T > 256) return fail(CR_EINVAL, "prm query: T = %d outside 2..256", T);
  if (map->R != 1 && map->R != P)
    return fail(CR_EINVAL, "prm query: the roadmap count R = %lld must be 1 or P = %lld", (long long)map->R,
                (long long)P);
  if (P == 0) return CR_OK;
  if ((st = check_ptr(u_start, 8, "u_start", true)) || (st = check_ptr(u_goal, 8, "u_goal", true)) ||
      (st = check_ptr(X, 8, "X", true)) || (st = check_ptr(length, 8, "length", true)) ||
      (st = check_ptr(hops, 4, "hops", true)))
    return st;
  crk::PrmArgs a = prm_args(*robot, scene, *w, *prm, *map);
  a.us = u_start;
  a.ug = u_goal;
  a.P = P;
  a.T = T;
  a.X = X;
  a.length = length;
  a.hops = hops;
  cudaStream_t s = stream_of(stream);
  switch (robot->n) {
    case 1: return crk::prm_query_n<1>(*robot, a, s);
    case 2: return crk::prm_query_n<2>(*robot, a, s);
    case 3: return crk::prm_query_n<3>(*robot, a, s);
    case 4: return crk::prm_query_n<4>(*robot, a, s);
    case 5: return crk::prm_query_n<5>(*robot, a, s);
    default: return crk::prm_query_n<6>(*robot, a, s);
  }
}

}  // extern "C"
