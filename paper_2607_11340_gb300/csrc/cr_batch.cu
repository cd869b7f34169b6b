// C ABI of the ragged batch: cr_batch_workspace_size, cr_batch_plan_create / _run / _info /
// _destroy, cr_solve_batch, and the plain per-problem form cr_solve_batch_plain.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "cr_batch_impl.cuh"

namespace crk {
CR_BATCH_INSTANTIATE(extern, 1)
CR_BATCH_INSTANTIATE(extern, 2)
CR_BATCH_INSTANTIATE(extern, 3)
CR_BATCH_INSTANTIATE(extern, 4)
CR_BATCH_INSTANTIATE(extern, 5)
CR_BATCH_INSTANTIATE(extern, 6)

// Start node: zero the queue heads (four per segment count), stamp the batch start.
__global__ void k_batch_start(int32_t* heads, int nheads, unsigned long long* t0) {
  const int i = threadIdx.x;
  if (i < nheads) heads[i] = 0;
  if (i == 0) *t0 = global_ns();
}

// Completion stamp of the plain form (one call per problem): t_done[item] = now - t0.
__global__ void k_batch_stamp(unsigned long long* t0, unsigned long long* t_done, int64_t item) {
  if (item < 0) *t0 = global_ns();
  else t_done[item] = global_ns() - *t0;
}

// Copies waypoints [w0, w0 + H) of a [7][W] target array into a [7][H] block.
__global__ void k_gather_waypoints(const double* targets, int64_t W, int64_t w0, int H, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 7 * H) out[e] = targets[(e / H) * W + w0 + e % H];
}

// Path following: the flags of one path from its waypoint errors and limit / clearance results.
__global__ void k_plain_path_flags(const double* pos, const double* rot, int H, const uint8_t* lim_ok,
                                   const uint8_t* col_ok, double pos_tol, double rot_tol, uint8_t* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool ok = true;
  for (int t = 0; t < H; ++t) ok = ok && pos[t] <= pos_tol && rot[t] <= rot_tol;
  const bool lim = *lim_ok != 0, col = *col_ok != 0;
  *flags = (uint8_t)((ok && lim && col ? 1 : 0) | (lim ? 2 : 0) | (col ? 4 : 0));
}
}  // namespace crk

using namespace crh;

struct cr_batch_plan {
  int device;
  int32_t spu;
  int32_t seed_regs;  // 1: the seeds phase's wide register budget, 2: the tight one
  int64_t units, workers;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

namespace {

constexpr int kSpuCandidates[] = {32, 64, 128, 256};

size_t batch_smem(int) { return (size_t)crk::kBatchWarps * crk::kBatchWarpSmem; }

// rb: register budget of the seeds phase (0 wide, 1 tight)
int blocks_per_sm(int n, int phase, int rb) {
  const size_t sm = batch_smem(n);
  switch (n) {
    case 1: return crk::batch_blocks_per_sm<1>(sm, phase, rb);
    case 2: return crk::batch_blocks_per_sm<2>(sm, phase, rb);
    case 3: return crk::batch_blocks_per_sm<3>(sm, phase, rb);
    case 4: return crk::batch_blocks_per_sm<4>(sm, phase, rb);
    case 5: return crk::batch_blocks_per_sm<5>(sm, phase, rb);
    default: return crk::batch_blocks_per_sm<6>(sm, phase, rb);
  }
}

cr_status prepare(int n) {
  const size_t sm = batch_smem(n);
  switch (n) {
    case 1: return crk::batch_prepare<1>(sm);
    case 2: return crk::batch_prepare<2>(sm);
    case 3: return crk::batch_prepare<3>(sm);
    case 4: return crk::batch_prepare<4>(sm);
    case 5: return crk::batch_prepare<5>(sm);
    default: return crk::batch_prepare<6>(sm);
  }
}

cr_status launch(int n, const cr_robot& fam, const cr_weights& w, const crk::BatchArgs& a, const crk::BatchGrids& g,
                 int rb, cudaStream_t s) {
  const size_t sm = batch_smem(n);
  switch (n) {
    case 1: return crk::batch_launch<1>(fam, w, a, g, sm, rb, s);
    case 2: return crk::batch_launch<2>(fam, w, a, g, sm, rb, s);
    case 3: return crk::batch_launch<3>(fam, w, a, g, sm, rb, s);
    case 4: return crk::batch_launch<4>(fam, w, a, g, sm, rb, s);
    case 5: return crk::batch_launch<5>(fam, w, a, g, sm, rb, s);
    default: return crk::batch_launch<6>(fam, w, a, g, sm, rb, s);
  }
}

cr_status check_items(const cr_robot* family, const cr_batch_item* items, int64_t N, const cr_batch_params* prm) {
  cr_status st;
  if (!family || !prm || (N > 0 && !items) || N < 0) return fail(CR_EINVAL, "batch: NULL argument or N < 0");
  if (N > (int64_t)1 << 30) return fail(CR_EINVAL, "batch: too many items");
  int nmax = 1;
  for (int64_t i = 0; i < N; ++i) {
    const cr_batch_item& it = items[i];
    if (it.kind != CR_ITEM_IK && it.kind != CR_ITEM_PATH)
      return fail(CR_EINVAL, "batch item %lld: kind %d", (long long)i, it.kind);
    if (it.n < 1 || it.n > CR_MAX_SEG) return fail(CR_EINVAL, "batch item %lld: n = %d", (long long)i, it.n);
    if (it.H < 1 || it.H > CR_BATCH_MAX_H || (it.kind == CR_ITEM_IK && it.H != 1))
      return fail(CR_EINVAL, "batch item %lld: H = %d", (long long)i, it.H);
    if (it.S < 1 || it.S > CR_MAX_SEEDS) return fail(CR_EINVAL, "batch item %lld: S = %d", (long long)i, it.S);
    if (it.n_o < 0 || it.n_o > CR_BATCH_MAX_SPHERES)
      return fail(CR_EINVAL, "batch item %lld: n_o = %d", (long long)i, it.n_o);
    nmax = std::max(nmax, it.n);
  }
  cr_robot r = *family;
  r.n = nmax;
  if ((st = check_robot(&r)) || (st = check_tendon_model(&r, "the ragged batch"))) return st;
  const cr_ik_params& p = prm->ik;
  if (p.n_final < 1 || p.n_final > 32 || p.k_init < 0 || p.k_final < 0 || prm->k_warm < 0 || prm->k_joint < 0)
    return fail(CR_EINVAL, "batch: bad iteration counts or n_final");
  const int spu = prm->seeds_per_unit;
  if (spu != 0 && spu != 32 && spu != 64 && spu != 128 && spu != 256)
    return fail(CR_EINVAL, "batch: seeds_per_unit %d not in {0, 32, 64, 128, 256}", spu);
  if (prm->seed_regs < 0 || prm->seed_regs > 2) return fail(CR_EINVAL, "batch: seed_regs %d not in {0, 1, 2}", prm->seed_regs);
  return CR_OK;
}

// Host-side plan of one batch: per-item offsets, the queues per segment count and the workspace
// layout. Estimated costs (relative warp time) order the queues longest first. grid[n-1]: the four
// phase kernels' grids; the joint phase's warps get the per-worker path buffers.
struct Layout {
  std::vector<crk::BatchItemK> items;  // grouped by n, queue order inside a group
  std::vector<int2> units;             // grouped by n
  int64_t item_begin[CR_MAX_SEG + 1], unit_begin[CR_MAX_SEG + 1];
  int hmax[CR_MAX_SEG + 1];
  crk::BatchGrids grid[CR_MAX_SEG + 1];
  size_t stride[CR_MAX_SEG + 1];
  size_t off_items, off_units, off_heads, off_t0, off_cand, off_x, off_scr[CR_MAX_SEG + 1], total;
  int64_t W, n_sph, n_states, n_cand, n_x;
  int64_t workers;
  int rb;  // register budget of the seeds phase: 0 wide, 1 tight
};
constexpr int kHeads = 4 * CR_MAX_SEG;

double est_cost(const cr_batch_item& it, const cr_batch_params& p) {
  const double n = it.n;
  double c = it.S * (p.ik.k_init + 1) * n + 8.0 * p.ik.k_final * n * n;
  if (it.kind == CR_ITEM_PATH && it.H > 1)
    c += (it.H - 1) * 3.0 * p.k_warm * n * n + p.k_joint * (4.0 * n * ((it.H + 31) / 32) + 0.5 * n * n * it.H);
  return c;
}

cr_status make_layout(const cr_batch_item* items, int64_t N, const cr_batch_params& p, int spu, int n_sm,
                      Layout& L, int rb = 0) {
  L.items.clear();
  L.units.clear();
  L.W = L.n_sph = L.n_states = L.n_cand = L.n_x = 0;
  std::vector<crk::BatchItemK> all(N);
  for (int64_t i = 0; i < N; ++i) {
    const cr_batch_item& it = items[i];
    crk::BatchItemK k{};
    const int D = 3 * it.n;
    k.kind = it.kind;
    k.H = it.H;
    k.S = it.S;
    k.no = it.n_o;
    k.G = (it.S + spu - 1) / spu;
    k.item = (int32_t)i;
    k.wp = L.W;
    k.sph = L.n_sph;
    k.st = L.n_states;
    k.cand = L.n_cand;
    k.xs = -1;
    if (it.kind == CR_ITEM_PATH && it.H > 1) {
      k.xs = L.n_x;
      L.n_x += (int64_t)D * it.H;
    }
    L.W += it.H;
    L.n_sph += it.n_o;
    L.n_states += (int64_t)D * it.H;
    L.n_cand += (int64_t)it.S * (D + 2);
    all[i] = k;
  }
  L.workers = 0;
  for (int n = 1; n <= CR_MAX_SEG; ++n) {
    std::vector<int64_t> idx;
    int hmax = 0;
    for (int64_t i = 0; i < N; ++i)
      if (items[i].n == n) {
        idx.push_back(i);
        if (items[i].kind == CR_ITEM_PATH && items[i].H > 1) hmax = std::max(hmax, items[i].H);
      }
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
      return est_cost(items[a], p) > est_cost(items[b], p);
    });
    L.item_begin[n - 1] = (int64_t)L.items.size();
    L.unit_begin[n - 1] = (int64_t)L.units.size();
    for (int64_t i : idx) {
      const int slot = (int)(L.items.size() - L.item_begin[n - 1]);
      L.items.push_back(all[i]);
      for (int g = 0; g < all[i].G; ++g) L.units.push_back(make_int2(slot, g));
    }
    L.hmax[n - 1] = hmax;
    L.stride[n - 1] = hmax > 0 ? crk::path_scratch(3 * n, hmax).total : 0;
    const int64_t nu = (int64_t)L.units.size() - L.unit_begin[n - 1];
    const int64_t ni = (int64_t)L.items.size() - L.item_begin[n - 1];
    int64_t npath = 0;
    for (int64_t i : idx) npath += (items[i].kind == CR_ITEM_PATH && items[i].H > 1) ? 1 : 0;
    const int64_t work[4] = {nu, ni, npath, npath};
    for (int ph = 0; ph < 4; ++ph) {
      const int bps = std::max(1, blocks_per_sm(n, ph, rb));
      const int64_t want = (work[ph] + crk::kBatchWarps - 1) / crk::kBatchWarps;
      L.grid[n - 1].g[ph] = work[ph] == 0 ? 0 : (int)std::min<int64_t>(want, (int64_t)bps * n_sm);
    }
    L.workers += (int64_t)L.grid[n - 1].g[0] * crk::kBatchWarps;
  }
  L.item_begin[CR_MAX_SEG] = (int64_t)L.items.size();
  L.unit_begin[CR_MAX_SEG] = (int64_t)L.units.size();
  size_t off = 0;
  L.off_items = off; off = align256(off + L.items.size() * sizeof(crk::BatchItemK));
  L.off_units = off; off = align256(off + (size_t)N * (CR_MAX_SEEDS / 32) * sizeof(int2));  // room for spu = 32
  L.off_heads = off; off = align256(off + kHeads * sizeof(int32_t));
  L.off_t0 = off; off = align256(off + sizeof(unsigned long long));
  L.off_cand = off; off = align256(off + (size_t)L.n_cand * sizeof(float));
  L.off_x = off; off = align256(off + (size_t)L.n_x * sizeof(float));
  for (int n = 1; n <= CR_MAX_SEG; ++n) {
    L.off_scr[n - 1] = off;
    off = align256(off + (size_t)L.grid[n - 1].g[3] * crk::kBatchWarps * L.stride[n - 1]);
  }
  L.total = off;
  L.rb = rb;
  return CR_OK;
}

int sm_count_of_current() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

// Upper bound over the seeds-per-unit candidates (grids do not depend on spu beyond the unit count).
size_t workspace_bound(const cr_batch_item* items, int64_t N, const cr_batch_params& p, int n_sm) {
  size_t best = 0;
  for (int spu : kSpuCandidates) {
    Layout L;
    make_layout(items, N, p, spu, n_sm, L);
    best = std::max(best, L.total);
  }
  return best;
}

struct Bound {
  const cr_robot* family;
  const cr_weights* w;
  const double* targets;
  const double* spheres;
  double *u_out, *cost, *pos, *rot;
  uint8_t* flags;
  uint64_t* t_done;
  unsigned char* ws;
};

crk::BatchArgs batch_args(const Layout& L, int n, const Bound& b, const cr_batch_params& p, int spu) {
  crk::BatchArgs a{};
  a.items = reinterpret_cast<const crk::BatchItemK*>(b.ws + L.off_items) + L.item_begin[n - 1];
  a.n_items = (int32_t)(L.item_begin[n] - L.item_begin[n - 1]);
  a.units = reinterpret_cast<const int2*>(b.ws + L.off_units) + L.unit_begin[n - 1];
  a.n_units = (int32_t)(L.unit_begin[n] - L.unit_begin[n - 1]);
  a.head = reinterpret_cast<int32_t*>(b.ws + L.off_heads) + 4 * (n - 1);
  a.xbuf = reinterpret_cast<float*>(b.ws + L.off_x);
  a.t0 = reinterpret_cast<const unsigned long long*>(b.ws + L.off_t0);
  a.targets = b.targets;
  a.W = L.W;
  a.spheres = b.spheres;
  a.cand = reinterpret_cast<float*>(b.ws + L.off_cand);
  a.scratch = b.ws + L.off_scr[n - 1];
  a.scratch_stride = L.stride[n - 1];
  a.hmax = L.hmax[n - 1];
  a.spu = spu;
  a.K = p.ik.n_final;
  a.k_init = p.ik.k_init;
  a.k_final = p.ik.k_final;
  a.alpha0 = float(p.ik.alpha0);
  a.eps = float(p.ik.dedup_eps);
  a.lambda0 = p.ik.lambda0;
  a.lim_tol = p.ik.lim_tol;
  a.pos_tol = p.ik.pos_tol;
  a.rot_tol = p.ik.rot_tol;
  for (int i = 0; i < crk::NMAX; ++i) a.umax[i] = b.family->u_max[i];
  a.seed = p.ik.seed;
  a.p0 = p.ik.p0;
  a.k_warm = p.k_warm;
  a.k_joint = p.k_joint;
  a.w_s = b.w->w_s;
  a.u_out = b.u_out;
  a.cost = b.cost;
  a.pos = b.pos;
  a.rot = b.rot;
  a.flags = b.flags;
  a.t_done = reinterpret_cast<unsigned long long*>(b.t_done);
  return a;
}

// Uploads the queues, captures the graph (start node, then per segment count the four phase
// kernels in order on one branch, the branches in parallel, largest queue first) and instantiates
// it.
cr_status build_plan(const Layout& L, const Bound& b, const cr_batch_params& p, int spu, int64_t N,
                     cudaStream_t user, cr_batch_plan* plan) {
  cudaError_t e;
  if (!L.items.empty()) {
    e = cudaMemcpyAsync(b.ws + L.off_items, L.items.data(), L.items.size() * sizeof(crk::BatchItemK),
                        cudaMemcpyHostToDevice, user);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b.ws + L.off_units, L.units.data(), L.units.size() * sizeof(int2), cudaMemcpyHostToDevice,
                          user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(user);
    if (e != cudaSuccess) return fail(CR_ECUDA, "batch plan upload: %s", cudaGetErrorString(e));
  }
  cr_status st;
  for (int n = 1; n <= CR_MAX_SEG; ++n)
    if (L.grid[n - 1].g[0] > 0 && (st = prepare(n))) return st;
  cudaStream_t cap, side[CR_MAX_SEG];
  cudaEvent_t fork, join[CR_MAX_SEG];
  if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(CR_ECUDA, "batch plan: %s", cudaGetErrorString(e));
  int made = 0;
  bool okres = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
  for (; okres && made < CR_MAX_SEG; ++made) {
    if (cudaStreamCreateWithFlags(&side[made], cudaStreamNonBlocking) != cudaSuccess) { okres = false; break; }
    if (cudaEventCreateWithFlags(&join[made], cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamDestroy(side[made]);
      okres = false;
      break;
    }
  }
  auto cleanup = [&]() {
    for (int i = 0; i < made; ++i) {
      cudaStreamDestroy(side[i]);
      cudaEventDestroy(join[i]);
    }
    cudaEventDestroy(fork);
    cudaStreamDestroy(cap);
  };
  if (!okres) {
    cleanup();
    return fail(CR_ECUDA, "batch plan: stream / event creation failed");
  }
  st = CR_OK;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cleanup();
    return fail(CR_ECUDA, "batch plan capture: %s", cudaGetErrorString(e));
  }
  {
    crk::k_batch_start<<<1, 32, 0, cap>>>(reinterpret_cast<int32_t*>(b.ws + L.off_heads), kHeads,
                                          reinterpret_cast<unsigned long long*>(b.ws + L.off_t0));
    cudaEventRecord(fork, cap);
    int order[CR_MAX_SEG];
    for (int i = 0; i < CR_MAX_SEG; ++i) order[i] = i + 1;
    std::stable_sort(order, order + CR_MAX_SEG, [&](int x, int y) {
      return L.unit_begin[x] - L.unit_begin[x - 1] > L.unit_begin[y] - L.unit_begin[y - 1];
    });
    int used = 0;
    for (int oi = 0; oi < CR_MAX_SEG && st == CR_OK; ++oi) {
      const int n = order[oi];
      if (L.grid[n - 1].g[0] == 0) continue;
      cudaStreamWaitEvent(side[used], fork, 0);
      st = launch(n, *b.family, *b.w, batch_args(L, n, b, p, spu), L.grid[n - 1], L.rb, side[used]);
      cudaEventRecord(join[used], side[used]);
      cudaStreamWaitEvent(cap, join[used], 0);
      ++used;
    }
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  cleanup();
  if (st != CR_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return st != CR_OK ? st : fail(CR_ECUDA, "batch plan capture: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(CR_ECUDA, "batch plan instantiate: %s", cudaGetErrorString(e));
  }
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  plan->graph = graph;
  plan->exec = exec;
  plan->spu = spu;
  plan->seed_regs = L.rb + 1;
  plan->units = (int64_t)L.units.size();
  plan->workers = L.workers;
  return CR_OK;
}

cr_status check_outputs(const double* targets, const double* spheres, const double* u_out, const double* cost,
                        const double* pos, const double* rot, const uint8_t* flags, const uint64_t* t_done,
                        const void* ws, bool need_sph) {
  cr_status st;
  if ((st = check_ptr(targets, 8, "targets", true)) || (st = check_ptr(spheres, 8, "spheres", need_sph)) ||
      (st = check_ptr(u_out, 8, "u_out", true)) || (st = check_ptr(cost, 8, "cost_out", true)) ||
      (st = check_ptr(pos, 8, "pos_err", true)) || (st = check_ptr(rot, 8, "rot_err", true)) ||
      (st = check_ptr(flags, 1, "flags_out", true)) || (st = check_ptr(t_done, 8, "t_done_ns", true)) ||
      (st = check_ptr(ws, 256, "workspace", true)))
    return st;
  return CR_OK;
}

bool any_spheres(const cr_batch_item* items, int64_t N) {
  for (int64_t i = 0; i < N; ++i)
    if (items[i].n_o > 0) return true;
  return false;
}

}  // namespace

extern "C" {

size_t cr_batch_workspace_size(const cr_robot* family, const cr_batch_item* items, int64_t N,
                               const cr_batch_params* prm) {
  if (check_items(family, items, N, prm)) return 0;
  const int n_sm = sm_count_of_current();
  if (n_sm <= 0) return 0;
  return workspace_bound(items, N, *prm, n_sm);
}

cr_status cr_batch_plan_create(const cr_robot* family, const cr_weights* w, const cr_batch_item* items, int64_t N,
                               const cr_batch_params* prm, const double* targets, const double* spheres,
                               double* u_out, double* cost_out, double* pos_err, double* rot_err, uint8_t* flags_out,
                               uint64_t* t_done_ns, void* workspace, size_t ws_bytes, cr_stream stream,
                               cr_batch_plan** plan_out) {
  cr_status st;
  if (w && (st = check_self_rows(*w, false, "cr_batch_plan_create"))) return st;
  if (!plan_out || !w) return fail(CR_EINVAL, "cr_batch_plan_create: NULL plan or weights");
  *plan_out = nullptr;
  if ((st = check_items(family, items, N, prm))) return st;
  if (N == 0) return fail(CR_EINVAL, "cr_batch_plan_create: empty batch");
  if ((st = check_outputs(targets, spheres, u_out, cost_out, pos_err, rot_err, flags_out, t_done_ns, workspace,
                          any_spheres(items, N))))
    return st;
  const int n_sm = sm_count_of_current();
  if (n_sm <= 0) return fail(CR_ECUDA, "cr_batch_plan_create: no device");
  const size_t need = workspace_bound(items, N, *prm, n_sm);
  if (ws_bytes < need) return fail(CR_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, need);
  cr_batch_plan* plan = static_cast<cr_batch_plan*>(std::calloc(1, sizeof(cr_batch_plan)));
  if (!plan) return fail(CR_EINVAL, "cr_batch_plan_create: out of host memory");
  cudaGetDevice(&plan->device);
  Bound b{family, w, targets, spheres, u_out, cost_out, pos_err, rot_err, flags_out, t_done_ns,
          static_cast<unsigned char*>(workspace)};
  cudaStream_t user = stream_of(stream);
  Layout L;
  // the candidates: seeds per unit x register budget of the seeds phase, each fixed by prm or open
  int spus[4], nspu = 0, rbs[2], nrb = 0;
  if (prm->seeds_per_unit != 0) spus[nspu++] = prm->seeds_per_unit;
  else for (int spu : kSpuCandidates) spus[nspu++] = spu;
  if (prm->seed_regs != 0) rbs[nrb++] = prm->seed_regs - 1;
  else { rbs[nrb++] = 0; rbs[nrb++] = 1; }
  if (nspu * nrb == 1) {
    make_layout(items, N, *prm, spus[0], n_sm, L, rbs[0]);
    if ((st = build_plan(L, b, *prm, spus[0], N, user, plan))) {
      cr_batch_plan_destroy(plan);
      return st;
    }
    *plan_out = plan;
    return CR_OK;
  }
  // by timing: each candidate is captured, run once to warm up, then timed
  float best_ms = 0.f;
  int best = 0, best_rb = 0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cr_batch_plan_destroy(plan);
    return fail(CR_ECUDA, "cr_batch_plan_create: event creation failed");
  }
  for (int c = 0; c < nspu * nrb && st == CR_OK; ++c) {
    const int spu = spus[c / nrb], rb = rbs[c % nrb];
    make_layout(items, N, *prm, spu, n_sm, L, rb);
    if ((st = build_plan(L, b, *prm, spu, N, user, plan))) break;
    cudaGraphLaunch(plan->exec, user);
    cudaEventRecord(e0, user);
    cudaGraphLaunch(plan->exec, user);
    cudaEventRecord(e1, user);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = fail(CR_ECUDA, "cr_batch_plan_create timing: %s", cudaGetErrorString(e));
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best == 0 || ms < best_ms) {
      best_ms = ms;
      best = spu;
      best_rb = rb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == CR_OK) {
    make_layout(items, N, *prm, best, n_sm, L, best_rb);
    st = build_plan(L, b, *prm, best, N, user, plan);
  }
  if (st != CR_OK) {
    cr_batch_plan_destroy(plan);
    return st;
  }
  *plan_out = plan;
  return CR_OK;
}

cr_status cr_batch_plan_run(cr_batch_plan* plan, cr_stream stream) {
  if (!plan || !plan->exec) return fail(CR_EINVAL, "cr_batch_plan_run: NULL plan");
  cudaError_t e = cudaGraphLaunch(plan->exec, stream_of(stream));
  if (e != cudaSuccess) return fail(CR_ECUDA, "cr_batch_plan_run: %s", cudaGetErrorString(e));
  return CR_OK;
}

cr_status cr_batch_plan_info(const cr_batch_plan* plan, int32_t* seeds_per_unit, int64_t* units, int64_t* workers,
                             int32_t* seed_regs) {
  if (!plan) return fail(CR_EINVAL, "cr_batch_plan_info: NULL plan");
  if (seeds_per_unit) *seeds_per_unit = plan->spu;
  if (units) *units = plan->units;
  if (workers) *workers = plan->workers;
  if (seed_regs) *seed_regs = plan->seed_regs;
  return CR_OK;
}

cr_status cr_batch_plan_destroy(cr_batch_plan* plan) {
  if (!plan) return CR_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  std::free(plan);
  return CR_OK;
}

cr_status cr_solve_batch(const cr_robot* family, const cr_weights* w, const cr_batch_item* items, int64_t N,
                         const cr_batch_params* prm, const double* targets, const double* spheres, double* u_out,
                         double* cost_out, double* pos_err, double* rot_err, uint8_t* flags_out, uint64_t* t_done_ns,
                         void* workspace, size_t ws_bytes, cr_stream stream) {
  if (!prm) return fail(CR_EINVAL, "cr_solve_batch: NULL params");
  if (w && check_self_rows(*w, false, "cr_solve_batch")) return CR_EINVAL;
  if (N == 0) return check_items(family, items, N, prm);
  cr_batch_params p = *prm;
  if (p.seeds_per_unit == 0) p.seeds_per_unit = 64;
  if (p.seed_regs == 0) p.seed_regs = 1;
  cr_batch_plan* plan = nullptr;
  cr_status st = cr_batch_plan_create(family, w, items, N, &p, targets, spheres, u_out, cost_out, pos_err, rot_err,
                                      flags_out, t_done_ns, workspace, ws_bytes, stream, &plan);
  if (st) return st;
  st = cr_batch_plan_run(plan, stream);
  cudaError_t e = cudaStreamSynchronize(stream_of(stream));
  cr_batch_plan_destroy(plan);
  if (st) return st;
  if (e != cudaSuccess) return fail(CR_ECUDA, "cr_solve_batch: %s", cudaGetErrorString(e));
  return CR_OK;
}

// ---------------------------------------------------------------------------------------------
// Plain form: one call per problem
// ---------------------------------------------------------------------------------------------
static cr_ik_params item_ik(const cr_batch_params& p, const cr_batch_item& it, int64_t i) {
  cr_ik_params q = p.ik;
  q.S = it.S;
  q.n_final = std::min(p.ik.n_final, it.S);
  q.p0 = p.ik.p0 + i;
  q.precision = CR_F32;
  return q;
}

size_t cr_batch_plain_workspace_size(const cr_robot* family, const cr_batch_item* items, int64_t N,
                                     const cr_batch_params* prm) {
  if (check_items(family, items, N, prm)) return 0;
  size_t need = 0;
  for (int64_t i = 0; i < N; ++i) {
    cr_robot r = *family;
    r.n = items[i].n;
    cr_ik_params q = item_ik(*prm, items[i], i);
    if (items[i].kind == CR_ITEM_PATH && items[i].H > 1)
      need = std::max(need, cr_path_workspace_size(&r, 1, items[i].H, &q));
    else
      need = std::max(need, cr_ik_workspace_size(&r, 1, &q));
  }
  return align256(need) + align256((size_t)7 * CR_BATCH_MAX_H * sizeof(double)) + 512;
}

cr_status cr_solve_batch_plain(const cr_robot* family, const cr_weights* w, const cr_batch_item* items, int64_t N,
                               const cr_batch_params* prm, const double* targets, const double* spheres,
                               double* u_out, double* cost_out, double* pos_err, double* rot_err, uint8_t* flags_out,
                               uint64_t* t_done_ns, void* workspace, size_t ws_bytes, cr_stream stream) {
  cr_status st;
  if (!w) return fail(CR_EINVAL, "cr_solve_batch_plain: NULL weights");
  if ((st = check_self_rows(*w, false, "cr_solve_batch_plain"))) return st;
  if ((st = check_items(family, items, N, prm))) return st;
  if (N == 0) return CR_OK;
  if ((st = check_outputs(targets, spheres, u_out, cost_out, pos_err, rot_err, flags_out, t_done_ns, workspace,
                          any_spheres(items, N))))
    return st;
  const size_t need = cr_batch_plain_workspace_size(family, items, N, prm);
  if (ws_bytes < need) return fail(CR_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, need);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const size_t tgb = align256((size_t)7 * CR_BATCH_MAX_H * sizeof(double));
  const size_t inner = need - 512 - tgb;
  double* tgt = reinterpret_cast<double*>(ws + inner);
  unsigned long long* t0 = reinterpret_cast<unsigned long long*>(ws + inner + tgb);
  uint8_t* limcol = ws + inner + tgb + 256;
  int64_t W = 0;
  for (int64_t i = 0; i < N; ++i) W += items[i].H;
  cudaStream_t s = stream_of(stream);
  unsigned long long* td = reinterpret_cast<unsigned long long*>(t_done_ns);
  crk::k_batch_stamp<<<1, 1, 0, s>>>(t0, td, -1);
  if ((st = check_launch("cr_solve_batch_plain"))) return st;
  int64_t wp = 0, so = 0, st_off = 0;
  for (int64_t i = 0; i < N; ++i) {
    const cr_batch_item& it = items[i];
    cr_robot r = *family;
    r.n = it.n;
    cr_scene sc{};
    sc.spheres = it.n_o > 0 ? spheres + so * 4 : nullptr;
    sc.n_o = it.n_o;
    sc.per_problem = 0;
    cr_ik_params q = item_ik(*prm, it, i);
    crk::k_gather_waypoints<<<(unsigned)((7 * it.H + 127) / 128), 128, 0, s>>>(targets, W, wp, it.H, tgt);
    if ((st = check_launch("cr_solve_batch_plain gather"))) return st;
    if (it.kind == CR_ITEM_PATH && it.H > 1) {
      cr_path_task pt{};
      pt.waypoints = tgt;
      pt.P = 1;
      pt.H = it.H;
      pt.w = *w;
      st = cr_solve_path(&r, &sc, &pt, &q, prm->k_warm, prm->k_joint, u_out + st_off, cost_out + i, pos_err + wp,
                         rot_err + wp, limcol, limcol + 1, ws, inner, stream);
      if (st) return st;
      crk::k_plain_path_flags<<<1, 1, 0, s>>>(pos_err + wp, rot_err + wp, it.H, limcol, limcol + 1, q.pos_tol,
                                              q.rot_tol, flags_out + i);
    } else {
      cr_task t{};
      t.kind = CR_TASK_IK6;
      t.seeds_per_target = 1;
      t.targets = tgt;
      t.n_targets = 1;
      t.w = *w;
      st = cr_solve_ik(&r, &sc, &t, &q, u_out + st_off, cost_out + i, pos_err + wp, rot_err + wp, flags_out + i, ws,
                       inner, stream);
      if (st) return st;
    }
    crk::k_batch_stamp<<<1, 1, 0, s>>>(t0, td, i);
    if ((st = check_launch("cr_solve_batch_plain"))) return st;
    wp += it.H;
    so += it.n_o;
    st_off += (int64_t)3 * it.n * it.H;
  }
  return CR_OK;
}

cr_status cr_batch_partition(const cr_batch_item* items, int64_t N, const cr_batch_params* prm, int32_t parts,
                             int64_t* bounds) {
  if (!prm || !bounds || (N > 0 && !items) || N < 0 || parts < 1)
    return fail(CR_EINVAL, "cr_batch_partition: NULL argument, N < 0 or parts < 1");
  std::vector<double> pre((size_t)N + 1, 0.0);  // prefix costs in the caller's order
  for (int64_t i = 0; i < N; ++i) {
    const cr_batch_item& it = items[i];
    if ((it.kind != CR_ITEM_IK && it.kind != CR_ITEM_PATH) || it.n < 1 || it.n > CR_MAX_SEG || it.H < 1 ||
        it.H > CR_BATCH_MAX_H || (it.kind == CR_ITEM_IK && it.H != 1) || it.S < 1 || it.S > CR_MAX_SEEDS ||
        it.n_o < 0 || it.n_o > CR_BATCH_MAX_SPHERES)
      return fail(CR_EINVAL, "cr_batch_partition: bad item %lld", (long long)i);
    pre[(size_t)i + 1] = pre[(size_t)i] + est_cost(it, *prm);
  }
  const double total = pre[(size_t)N];
  bounds[0] = 0;
  int64_t j = 0;
  for (int r = 1; r < parts; ++r) {
    const double goal = total * (double)r / (double)parts;
    while (j < N && pre[(size_t)j + 1] <= goal) ++j;  // items whose prefix cost stays within r / parts
    bounds[r] = j;
  }
  bounds[parts] = N;
  return CR_OK;
}

}  // extern "C"
