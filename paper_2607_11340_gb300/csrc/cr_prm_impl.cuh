// PRM exploration of Algorithm 2 (Sec. IV-B, "Trajectory Planning"): the roadmap of every scene
// (ParallelSample, ParallelConnect) and the per-query stage (ConnectToRoadmap, shortest path,
// ResampleLinear), all on the device.
//
//  k_prm_sample : one thread per node: up to `attempts` hexagon-uniform draws (the SampleSeeds
//                 generator with problem = roadmap, seed = node), the first collision-free one kept.
//  k_prm_knn    : one warp per node: squared distances to every node of its roadmap in shared
//                 memory, then k rounds of a warp argmin on (distance^2, index).
//  k_prm_edges  : one thread per (kNN slot, interior state): the collision test of one state of the
//                 straight segment; a colliding state marks the slot blocked.
//  k_prm_adj    : one thread per slot: a free canonical slot sets both bits of the adjacency bitset.
//  k_prm_csr    : one block per roadmap: degrees, a block scan and the rows in ascending column
//                 order (deterministic, whatever order the atomics ran in), FP64 weights.
//  k_prm_query  : one block per query: nearest nodes of the start and goal with their segment checks,
//                 synchronous relaxation rounds (every vertex takes the minimum over its neighbours
//                 of d(u) + w(u, v) until no distance changes), the canonical predecessor walk and
//                 the equal-arc-length resampling.
//
// Collision decisions are FP64 (the answer is an integer). An FP32 pass decides first with a
// margin m_j = 1e-5 (sum L + reach_j + |c_j|_1) per sphere, far above the FP32 error of the backbone
// points: a pair closer than reach - m collides for certain, a state with no pair within reach + m
// is free for certain, and only states in between are evaluated again in FP64.
//
// The relaxation reaches the same distances as Dijkstra's algorithm: with rounded additions that
// are monotone in d(u), both compute for every vertex the minimum over paths of the distance summed
// along the path from the start; the path is read back through the lowest-index neighbour u with
// d(u) < d(v) and d(u) + w(u, v) == d(v), so it is unique even when paths tie.
#pragma once

#include "cr_host.h"

namespace crk {

constexpr int kPrmMaxN = 1024;
constexpr int kPrmMaxK = 32;
constexpr int kPrmMaxCheck = 64;
constexpr int kPrmMaxAttempts = 8;  // the draw counter holds 3 bits of attempt
constexpr int kPrmQueryThreads = 256;
constexpr int kPrmKnnWarps = 4;
// Relative margin of the FP32 collision filter (about 6 um for robots and scenes of 0.3 m, some
// 60 times the FP32 error of the backbone samples).
constexpr double kPrmMargin = 1e-5;

struct PrmArgs {
  const double* spheres;  // [R or 1][no][4]
  int no, sph_pp;
  int64_t R;
  int N, k, n_check, attempts;
  uint64_t seed;
  double umax[NMAX];
  double delta;
  double coord_max;       // largest |node coordinate| (the largest u_max)
  double* nodes;          // [D][R*N]
  float* nodes32;         // [D][R*N] the nodes rounded to FP32 (build workspace: the edge filter's operands)
  unsigned char* ok;      // [R*N]
  int32_t* nbr;           // [R*N][k]
  unsigned char* blocked; // [R*N*k]
  uint32_t* adj;          // [R][N][Wd]
  int32_t* row;           // [R][N+1]
  int32_t* col;           // [R][2Nk]
  double* wt;             // [R][2Nk]
  // query
  const double* us;       // [D][P]
  const double* ug;       // [D][P]
  int64_t P;
  int T;
  double* X;              // [D][P*T]
  double* length;         // [P]
  int32_t* hops;          // [P]
};

__host__ __device__ inline int prm_words(int N) { return (N + 31) / 32; }

// Obstacles of one scene as the PRM kernels stage them: FP32 spheres with the reach widened by the
// margin (filter and broad phase), FP32 squared reach narrowed by the margin (certain collision),
// FP64 spheres with the exact reach (the decision).
struct PrmSph {
  Sphere4<float>* hi;
  float* lo2;
  Sphere4<double>* ex;
};
__host__ __device__ inline size_t prm_sph_bytes(int no) {
  return (((size_t)no * (sizeof(Sphere4<float>) + sizeof(float)) + 15) & ~size_t(15)) +
         (size_t)no * sizeof(Sphere4<double>);
}
__device__ inline PrmSph prm_sph_carve(unsigned char* base, int no) {
  PrmSph s;
  s.hi = reinterpret_cast<Sphere4<float>*>(base);
  s.lo2 = reinterpret_cast<float*>(base + (size_t)no * sizeof(Sphere4<float>));
  s.ex = reinterpret_cast<Sphere4<double>*>(
      base + (((size_t)no * (sizeof(Sphere4<float>) + sizeof(float)) + 15) & ~size_t(15)));
  return s;
}
template <int N>
__device__ void prm_stage(const double* sp, int no, const RobotK<double>& rbd, double delta, PrmSph s) {
  double lsum = 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) lsum += rbd.L[i];
  for (int j = threadIdx.x; j < no; j += blockDim.x) {
    const double x = sp[4 * j], y = sp[4 * j + 1], z = sp[4 * j + 2];
    const double reach = sp[4 * j + 3] + rbd.rbody + delta;
    const double m = kPrmMargin * (lsum + reach + fabs(x) + fabs(y) + fabs(z));
    s.hi[j] = Sphere4<float>{float(x), float(y), float(z), float(reach + m)};
    const double rl = reach - m;
    s.lo2[j] = rl > 0.0 ? float(rl * rl) : 0.0f;
    s.ex[j] = Sphere4<double>{x, y, z, reach};
  }
}

// FP32 classification of one state: 0 free, 1 colliding, 2 undecided (within the margin band).
template <int N>
__device__ int prm_class32(const RobotK<float>& rb, const PrmSph& s, int no, const float (&u)[3 * N]) {
  Chain<float, N> ch;
  chain_forward(rb, u, ch);
  const float inb = 1.0f / float(rb.nb);
  bool unsure = false;
  for (int j0 = 0; j0 < no; j0 += 64) {
    uint64_t mk[N];
    segment_sphere_masks(rb, ch, ObsK<float>(s.hi), j0, no - j0 < 64 ? no - j0 : 64, mk);
    for (int i = 0; i < N; ++i) {
      if (!mk[i]) continue;
      for (int k0 = 1; k0 <= rb.nb; k0 += kCullGroup) {
        const int k1 = k0 + kCullGroup - 1 < rb.nb ? k0 + kCullGroup - 1 : rb.nb;
        const uint64_t gm = group_sphere_mask<float, N>(rb, ch, i, k0, k1, s.hi, j0, mk[i]);
        if (!gm) continue;
        for (int k = k0; k <= k1; ++k) {
          float q[3], wp[3], sn, cs;
          backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], float(k) * inb, q, wp, sn, cs);
          for (uint64_t bits = gm; bits; bits &= bits - 1) {
            const int j = j0 + __ffsll((long long)bits) - 1;
            const Sphere4<float> S = s.hi[j];
            const float dx = wp[0] - S.x, dy = wp[1] - S.y, dz = wp[2] - S.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < s.lo2[j]) return 1;
            if (d2 < S.reach * S.reach) unsure = true;
          }
        }
      }
    }
  }
  return unsure ? 2 : 0;
}

// Collision decision of state u (FP64; the FP32 pass settles all but the margin band).
template <int N>
__device__ bool prm_collides(const RobotK<float>& rbf, const RobotK<double>& rbd, const PrmSph& s, int no,
                             const double (&u)[3 * N]) {
  if (no == 0) return false;
  float uf[3 * N];
#pragma unroll
  for (int q = 0; q < 3 * N; ++q) uf[q] = float(u[q]);
  const int c = prm_class32<N>(rbf, s, no, uf);
  if (c != 2) return c == 1;
  return state_collides<double, N>(rbd, s.ex, no, u);
}

// Squared distance summed in coordinate order, every operation rounded on its own.
template <int D> __device__ __forceinline__ double prm_dist2(const double (&a)[D], const double (&b)[D]) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    const double t = __dsub_rn(a[q], b[q]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// State c of the n_check interior states of the segment xa -> xb: xa + c/(n_check+1) (xb - xa).
template <int D>
__device__ __forceinline__ void prm_lerp(const double (&xa)[D], const double (&xb)[D], int c, int n_check,
                                         double (&x)[D]) {
  const double s = __ddiv_rn((double)c, (double)(n_check + 1));
#pragma unroll
  for (int q = 0; q < D; ++q) x[q] = __dadd_rn(xa[q], __dmul_rn(s, __dsub_rn(xb[q], xa[q])));
}

// The same state in FP32 for the filter (within a few FP32 roundings of the FP64 state, far inside
// the margin).
template <int D>
__device__ __forceinline__ void prm_lerp32(const double (&xa)[D], const double (&xb)[D], int c, int n_check,
                                           float (&x)[D]) {
  const float s = float(c) / float(n_check + 1);
#pragma unroll
  for (int q = 0; q < D; ++q) {
    const float a = float(xa[q]);
    x[q] = a + s * (float(xb[q]) - a);
  }
}

// Does the state c of the segment xa -> xb collide? FP32 filter on the FP32 interpolation; the FP64
// interpolation and decision only inside the margin band.
template <int N>
__device__ bool prm_segment_state_collides(const RobotK<float>& rbf, const RobotK<double>& rbd, const PrmSph& s,
                                           int no, const double (&xa)[3 * N], const double (&xb)[3 * N], int c,
                                           int n_check) {
  if (no == 0) return false;
  float xf[3 * N];
  prm_lerp32<3 * N>(xa, xb, c, n_check, xf);
  const int cl = prm_class32<N>(rbf, s, no, xf);
  if (cl != 2) return cl == 1;
  double x[3 * N];
  prm_lerp<3 * N>(xa, xb, c, n_check, x);
  return state_collides<double, N>(rbd, s.ex, no, x);
}

template <int D> __device__ __forceinline__ void prm_load(const double* base, int64_t ld, int64_t col, double (&x)[D]) {
#pragma unroll
  for (int q = 0; q < D; ++q) x[q] = base[q * ld + col];
}

// ------------------------------------------------------------------------------------------------
// Roadmap
// ------------------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_prm_sample(RobotK<float> rbf, RobotK<double> rbd, PrmArgs a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t r = blockIdx.y;
  const PrmSph s = prm_sph_carve(smem_raw, a.no);
  prm_stage<N>(a.spheres + (a.sph_pp ? r * a.no * 4 : 0), a.no, rbd, a.delta, s);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  double u[D];
  bool ok = false;
  for (int at = 0; at < a.attempts && !ok; ++at) {
    draw_seed<double, N>(a.seed, (uint64_t)r, (uint64_t)i, at, a.umax, u);
    ok = !prm_collides<N>(rbf, rbd, s, a.no, u);
  }
  const int64_t ld = a.R * a.N, c = r * a.N + i;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    a.nodes[q * ld + c] = u[q];
    a.nodes32[q * ld + c] = float(u[q]);
  }
  a.ok[c] = ok ? 1 : 0;
}

// k nearest valid nodes of node i, exactly by (FP64 squared distance, index). FP32 squared distances
// of the FP32 nodes first: with |coordinates| <= M, u = 2^-24, they differ from the FP64 ones by at
// most E = 24 u D M^2 + (D + 2) u d^2; t_k, the k-th smallest FP32 value, is then within E of the k-th
// smallest FP64 value, so every true neighbour has an FP32 value <= t_k + 2E. Only nodes under that
// threshold (widened 4x) get their FP64 distance; the selection runs on those.
template <int N>
__global__ void __launch_bounds__(32 * kPrmKnnWarps) k_prm_knn(PrmArgs a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = blockIdx.y;
  const int i = blockIdx.x * kPrmKnnWarps + wid;
  if (i >= a.N) return;
  // per warp: FP64 keys [N] | FP32 squared distances [N] | candidate list [N]
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_raw) + (size_t)wid * a.N;
  float* f2 = reinterpret_cast<float*>(smem_raw + (size_t)kPrmKnnWarps * a.N * 8) + (size_t)wid * a.N;
  int* cl = reinterpret_cast<int*>(smem_raw + (size_t)kPrmKnnWarps * a.N * 12) + (size_t)wid * a.N;
  const int64_t ld = a.R * a.N, base = r * a.N;
  int32_t* out = a.nbr + (base + i) * a.k;
  if (!a.ok[base + i]) {
    for (int c = lane; c < a.k; c += 32) out[c] = -1;
    return;
  }
  float fi[D];
#pragma unroll
  for (int q = 0; q < D; ++q) fi[q] = a.nodes32[q * ld + base + i];
  for (int j = lane; j < a.N; j += 32) {
    float v = INFINITY;
    if (j != i && a.ok[base + j]) {
      v = 0.0f;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const float t = fi[q] - a.nodes32[q * ld + base + j];
        v = fmaf(t, t, v);
      }
    }
    f2[j] = v;
  }
  __syncwarp();
  // t_k: k rounds of "smallest (value, index) above the previous one"
  float pv = -1.0f;
  int pj = -1;
  for (int c = 0; c < a.k; ++c) {
    float bv = INFINITY;
    int bj = 0x7fffffff;
    for (int j = lane; j < a.N; j += 32) {
      const float v = f2[j];
      const bool above = v > pv || (v == pv && j > pj);
      if (above && (v < bv || (v == bv && j < bj))) { bv = v; bj = j; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
      if (ov < bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
    }
    if (!(bv < INFINITY)) break;
    pv = bv;
    pj = bj;
  }
  const double u32 = 5.9604644775390625e-8;  // 2^-24
  float thr = -1.0f;  // FP32 threshold rounded upward
  if (pj >= 0) {
    const double t = double(pv) + 8.0 * (24.0 * u32 * D * a.coord_max * a.coord_max + (D + 2) * u32 * double(pv));
    thr = __double2float_ru(t);
  }
  // the candidates in index order (ballot compaction), then their exact FP64 squared distances with
  // the lanes over the list, kept as bit patterns: for non-negative doubles the unsigned order of the
  // bits is the order of the values
  int nc = 0;
  for (int j0 = 0; j0 < a.N; j0 += 32) {
    const int j = j0 + lane;
    const bool cand = j < a.N && f2[j] <= thr;
    const unsigned m = __ballot_sync(0xffffffffu, cand);
    if (cand) cl[nc + __popc(m & ((1u << lane) - 1u))] = j;
    nc += __popc(m);
  }
  __syncwarp();
  double xi[D];
  prm_load<D>(a.nodes, ld, base + i, xi);
  for (int e = lane; e < nc; e += 32) {
    double xj[D];
    prm_load<D>(a.nodes, ld, base + cl[e], xj);
    key[e] = (unsigned long long)__double_as_longlong(prm_dist2<D>(xi, xj));
  }
  __syncwarp();
  for (int c = 0; c < a.k; ++c) {
    unsigned long long bv = ~0ull;
    int bj = 0x7fffffff, be = -1;
    for (int e = lane; e < nc; e += 32) {
      const unsigned long long v = key[e];
      if (v < bv) { bv = v; bj = cl[e]; be = e; }  // ascending index within the lane
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
      const int oe = __shfl_xor_sync(0xffffffffu, be, off);
      if (ov < bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; be = oe; }
    }
    const bool found = bv != ~0ull;
    if (lane == 0) out[c] = found ? bj : -1;
    if (found && lane == (be & 31)) key[be] = ~0ull;
    __syncwarp();
  }
}

// Does slot e of node i name an edge that another slot checks (i > j and j lists i)?
__device__ __forceinline__ bool prm_dup(const int32_t* nbr, int64_t base, int k, int i, int j) {
  if (i < j) return false;
  const int32_t* lj = nbr + (base + j) * k;
  for (int c = 0; c < k; ++c)
    if (lj[c] == i) return true;
  return false;
}

template <int N>
__global__ void __launch_bounds__(256) k_prm_edges(RobotK<float> rbf, RobotK<double> rbd, PrmArgs a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t r = blockIdx.y;
  const PrmSph s = prm_sph_carve(smem_raw, a.no);
  prm_stage<N>(a.spheres + (a.sph_pp ? r * a.no * 4 : 0), a.no, rbd, a.delta, s);
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)a.N * a.k * a.n_check) return;
  const int slot = (int)(idx / a.n_check), c = (int)(idx % a.n_check) + 1;
  const int i = slot / a.k;
  const int64_t base = r * a.N;
  const int j = a.nbr[(base + i) * a.k + slot % a.k];
  if (j < 0 || prm_dup(a.nbr, base, a.k, i, j)) return;
  const int lo = i < j ? i : j, hi = i < j ? j : i;
  if (a.no == 0) return;
  const int64_t ld = a.R * a.N;
  // FP32 filter on the FP32 interpolation of the FP32 nodes; FP64 only inside the margin band
  const float sc = float(c) / float(a.n_check + 1);
  float xf[D];
#pragma unroll
  for (int q = 0; q < D; ++q) {
    const float fa = a.nodes32[q * ld + base + lo];
    xf[q] = fa + sc * (a.nodes32[q * ld + base + hi] - fa);
  }
  int cl = prm_class32<N>(rbf, s, a.no, xf);
  if (cl == 2) {
    double xa[D], xb[D], x[D];
    prm_load<D>(a.nodes, ld, base + lo, xa);
    prm_load<D>(a.nodes, ld, base + hi, xb);
    prm_lerp<D>(xa, xb, c, a.n_check, x);
    cl = state_collides<double, N>(rbd, s.ex, a.no, x) ? 1 : 0;
  }
  if (cl == 1) a.blocked[base * a.k + slot] = 1;
}

static __global__ void k_prm_adj(PrmArgs a) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.R * a.N * a.k) return;
  const int64_t r = idx / ((int64_t)a.N * a.k);
  const int slot = (int)(idx % ((int64_t)a.N * a.k));
  const int i = slot / a.k;
  const int64_t base = r * a.N;
  const int j = a.nbr[idx];
  if (j < 0 || prm_dup(a.nbr, base, a.k, i, j) || a.blocked[idx]) return;
  const int Wd = prm_words(a.N);
  atomicOr(a.adj + (base + i) * Wd + (j >> 5), 1u << (j & 31));
  atomicOr(a.adj + (base + j) * Wd + (i >> 5), 1u << (i & 31));
}

// Block-wide exclusive scan of one int per thread (blockDim a multiple of 32, at most 1024).
__device__ inline int prm_block_scan(int v, int* warp_tot, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= off) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;  // inclusive prefix of the warp totals
  }
  __syncthreads();
  total = warp_tot[nw - 1];
  return x - v + (wid > 0 ? warp_tot[wid - 1] : 0);
}

template <int N>
__global__ void __launch_bounds__(1024) k_prm_csr(PrmArgs a) {
  constexpr int D = 3 * N;
  __shared__ int warp_tot[32];
  const int64_t r = blockIdx.x;
  const int i = threadIdx.x;
  const int Wd = prm_words(a.N);
  const int64_t base = r * a.N;
  const uint32_t* arow = a.adj + (base + (i < a.N ? i : 0)) * Wd;
  int deg = 0;
  if (i < a.N)
    for (int w = 0; w < Wd; ++w) deg += __popc(arow[w]);
  int total;
  const int off = prm_block_scan(deg, warp_tot, total);
  int32_t* row = a.row + r * (a.N + 1);
  const int64_t cap = (int64_t)2 * a.N * a.k;
  int32_t* col = a.col + r * cap;
  double* wt = a.wt + r * cap;
  if (i == 0) row[a.N] = total;
  if (i >= a.N) return;
  row[i] = off;
  const int64_t ld = a.R * a.N;
  double xi[D];
  prm_load<D>(a.nodes, ld, base + i, xi);
  int e = off;
  for (int w = 0; w < Wd; ++w)
    for (uint32_t bits = arow[w]; bits; bits &= bits - 1) {
      const int j = w * 32 + __ffs(bits) - 1;
      double xj[D];
      prm_load<D>(a.nodes, ld, base + j, xj);
      col[e] = j;
      wt[e] = __dsqrt_rn(prm_dist2<D>(xi, xj));
      ++e;
    }
}

// ------------------------------------------------------------------------------------------------
// Query
// ------------------------------------------------------------------------------------------------
// Shared memory of one query block (byte offsets after the staged spheres).
struct PrmQuerySmem {
  size_t d0, d1, ls, lg, path, cand, cd2, blk, red, total;
};
__host__ __device__ inline PrmQuerySmem prm_query_smem(int no, int N, int k) {
  PrmQuerySmem m;
  size_t off = (prm_sph_bytes(no) + 15) & ~size_t(15);
  m.d0 = off; off += (size_t)8 * (N + 2);
  m.d1 = off; off += (size_t)8 * (N + 2);
  m.ls = off; off += (size_t)8 * N;
  m.lg = off; off += (size_t)8 * N;
  m.cd2 = off; off += (size_t)8 * 2 * k;
  m.red = off; off += (size_t)8 * 32 + 4 * 32;
  m.path = off; off += (size_t)4 * (N + 2);
  m.cand = off; off += (size_t)4 * 2 * k;
  m.blk = off; off += (size_t)2 * k;
  m.total = (off + 15) & ~size_t(15);
  return m;
}

// Block argmin of (value, index) pairs, one per thread; every thread gets the result.
__device__ inline void prm_block_argmin(double& v, int& j, double* rv, int* rj) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oj = __shfl_xor_sync(0xffffffffu, j, off);
    if (ov < v || (ov == v && oj < j)) { v = ov; j = oj; }
  }
  if (lane == 0) { rv[wid] = v; rj[wid] = j; }
  __syncthreads();
  v = rv[0];
  j = rj[0];
  for (int w = 1; w < nw; ++w)
    if (rv[w] < v || (rv[w] == v && rj[w] < j)) { v = rv[w]; j = rj[w]; }
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(kPrmQueryThreads) k_prm_query(RobotK<float> rbf, RobotK<double> rbd, PrmArgs a) {
  constexpr int D = 3 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t p = blockIdx.x;
  const int64_t r = a.R == 1 ? 0 : p;
  const int NN = a.N, S = NN, G = NN + 1, V = NN + 2;
  const PrmQuerySmem m = prm_query_smem(a.no, NN, a.k);
  const PrmSph s = prm_sph_carve(smem_raw, a.no);
  double* dA = reinterpret_cast<double*>(smem_raw + m.d0);
  double* dB = reinterpret_cast<double*>(smem_raw + m.d1);
  double* ls = reinterpret_cast<double*>(smem_raw + m.ls);
  double* lg = reinterpret_cast<double*>(smem_raw + m.lg);
  double* cd2 = reinterpret_cast<double*>(smem_raw + m.cd2);
  double* rv = reinterpret_cast<double*>(smem_raw + m.red);
  int* rj = reinterpret_cast<int*>(smem_raw + m.red + 8 * 32);
  int* path = reinterpret_cast<int*>(smem_raw + m.path);
  int* cand = reinterpret_cast<int*>(smem_raw + m.cand);
  unsigned char* blk = smem_raw + m.blk;
  __shared__ int ncand[2], hops_s;
  prm_stage<N>(a.spheres + (a.sph_pp ? p * a.no * 4 : 0), a.no, rbd, a.delta, s);
  const int64_t ld = a.R * a.N, base = r * a.N;
  const unsigned char* ok = a.ok + base;
  double xs[D], xg[D];
  prm_load<D>(a.us, a.P, p, xs);
  prm_load<D>(a.ug, a.P, p, xg);
  for (int v = threadIdx.x; v < NN; v += blockDim.x) { ls[v] = INFINITY; lg[v] = INFINITY; }
  for (int e = threadIdx.x; e < 2 * a.k; e += blockDim.x) blk[e] = 0;
  __syncthreads();
  // ConnectToRoadmap: the k nearest valid nodes of the start (side 0) and the goal (side 1)
  for (int side = 0; side < 2; ++side) {
    for (int v = threadIdx.x; v < NN; v += blockDim.x) {
      double d = INFINITY;
      if (ok[v]) {
        double xv[D];
        prm_load<D>(a.nodes, ld, base + v, xv);
        d = prm_dist2<D>(side == 0 ? xs : xg, xv);
      }
      dA[v] = d;
    }
    __syncthreads();
    int cnt = 0;
    for (int c = 0; c < a.k; ++c) {
      double bv = INFINITY;
      int bj = 0x7fffffff;
      for (int v = threadIdx.x; v < NN; v += blockDim.x)
        if (dA[v] < bv) { bv = dA[v]; bj = v; }
      prm_block_argmin(bv, bj, rv, rj);
      if (!(bv < INFINITY)) break;
      if (threadIdx.x == 0) {
        cand[side * a.k + c] = bj;
        cd2[side * a.k + c] = bv;
        dA[bj] = INFINITY;
      }
      cnt = c + 1;
      __syncthreads();
    }
    if (threadIdx.x == 0) ncand[side] = cnt;
    __syncthreads();
  }
  // segment checks of the candidate links, one state per thread
  for (int e = threadIdx.x; e < (ncand[0] + ncand[1]) * a.n_check; e += blockDim.x) {
    const int ci = e / a.n_check, c = e % a.n_check + 1;
    const int side = ci < ncand[0] ? 0 : 1, slot = side == 0 ? ci : ci - ncand[0];
    double xv[D];
    prm_load<D>(a.nodes, ld, base + cand[side * a.k + slot], xv);
    if (prm_segment_state_collides<N>(rbf, rbd, s, a.no, side == 0 ? xs : xg, xv, c, a.n_check))
      blk[side * a.k + slot] = 1;
  }
  __syncthreads();
  if (threadIdx.x < 2 * a.k) {
    const int side = threadIdx.x / a.k, slot = threadIdx.x % a.k;
    if (slot < ncand[side] && !blk[threadIdx.x])
      (side == 0 ? ls : lg)[cand[threadIdx.x]] = __dsqrt_rn(cd2[threadIdx.x]);
  }
  // synchronous relaxation from the start
  for (int v = threadIdx.x; v < V; v += blockDim.x) dA[v] = v == S ? 0.0 : INFINITY;
  __syncthreads();
  const int32_t* row = a.row + r * (NN + 1);
  const int64_t cap = (int64_t)2 * NN * a.k;
  const int32_t* col = a.col + r * cap;
  const double* wt = a.wt + r * cap;
  double* dc = dA;
  double* dn = dB;
  for (int round = 0; round <= V; ++round) {
    bool changed = false;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      double best = dc[v];
      if (v < NN) {
        for (int e = row[v]; e < row[v + 1]; ++e) {
          const double c = dc[col[e]] + wt[e];
          if (c < best) best = c;
        }
        if (ls[v] < INFINITY && dc[S] + ls[v] < best) best = dc[S] + ls[v];
        if (lg[v] < INFINITY && dc[G] + lg[v] < best) best = dc[G] + lg[v];
      } else if (v == G) {
        for (int c = 0; c < ncand[1]; ++c) {
          const int u = cand[a.k + c];
          if (lg[u] < INFINITY && dc[u] + lg[u] < best) best = dc[u] + lg[u];
        }
      }
      changed = changed || best < dc[v];
      dn[v] = best;
    }
    const int any = __syncthreads_or(changed);
    double* t = dc; dc = dn; dn = t;
    if (!any) break;
  }
  // canonical predecessor walk from the goal (one thread), then the resampling
  if (threadIdx.x == 0) {
    int M = 0;
    if (dc[G] < INFINITY) {
      int v = G, len = 0;
      path[len++] = G;
      while (v != S && len < V) {
        int best = -1;
        if (v < NN) {
          for (int e = row[v]; e < row[v + 1] && best < 0; ++e) {
            const int u = col[e];
            if (dc[u] < dc[v] && dc[u] + wt[e] == dc[v]) best = u;
          }
          if (best < 0 && ls[v] < INFINITY && dc[S] < dc[v] && dc[S] + ls[v] == dc[v]) best = S;
          if (best < 0 && lg[v] < INFINITY && dc[G] < dc[v] && dc[G] + lg[v] == dc[v]) best = G;
        } else {  // v == G: the lowest-index attached node that qualifies
          for (int c = 0; c < ncand[1]; ++c) {
            const int u = cand[a.k + c];
            if (lg[u] < INFINITY && dc[u] < dc[v] && dc[u] + lg[u] == dc[v] && (best < 0 || u < best)) best = u;
          }
        }
        if (best < 0) { len = 0; break; }
        v = best;
        path[len++] = v;
      }
      if (len > 1 && v == S) {
        M = len - 1;
        for (int e = 0; e < len / 2; ++e) {
          const int t = path[e];
          path[e] = path[len - 1 - e];
          path[len - 1 - e] = t;
        }
      }
    }
    hops_s = M;
    a.hops[p] = M;
    a.length[p] = M > 0 ? dc[G] : INFINITY;
  }
  __syncthreads();
  const int M = hops_s;
  const double Lt = dc[G];
  for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
    double x[D];
    const double ft = __ddiv_rn((double)t, (double)(a.T - 1));
    if (M == 0) {
#pragma unroll
      for (int q = 0; q < D; ++q) x[q] = __dadd_rn(xs[q], __dmul_rn(ft, __dsub_rn(xg[q], xs[q])));
    } else if (t == 0 || t == a.T - 1) {
#pragma unroll
      for (int q = 0; q < D; ++q) x[q] = t == 0 ? xs[q] : xg[q];
    } else {
      const double sl = __dmul_rn(ft, Lt);
      int j = 0;
      while (j + 1 < M && dc[path[j + 1]] <= sl) ++j;
      const int va = path[j], vb = path[j + 1];
      const double lam = __ddiv_rn(__dsub_rn(sl, dc[va]), __dsub_rn(dc[vb], dc[va]));
      double xa[D], xb[D];
      if (va == S) {
#pragma unroll
        for (int q = 0; q < D; ++q) xa[q] = xs[q];
      } else {
        prm_load<D>(a.nodes, ld, base + va, xa);
      }
      if (vb == G) {
#pragma unroll
        for (int q = 0; q < D; ++q) xb[q] = xg[q];
      } else {
        prm_load<D>(a.nodes, ld, base + vb, xb);
      }
#pragma unroll
      for (int q = 0; q < D; ++q) x[q] = __dadd_rn(xa[q], __dmul_rn(lam, __dsub_rn(xb[q], xa[q])));
    }
#pragma unroll
    for (int q = 0; q < D; ++q) a.X[q * a.P * a.T + p * a.T + t] = x[q];
  }
}

// ------------------------------------------------------------------------------------------------
// Host launchers (cr_prm_n*.cu instantiate them per segment count)
// ------------------------------------------------------------------------------------------------
inline cr_status prm_set_smem(const void* f, size_t bytes, const char* what) {
  if (bytes <= 48 * 1024) return CR_OK;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return crh::fail(CR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return CR_OK;
}

// Roadmap build: blocked flags and the adjacency bitset must be zero on entry (the caller clears
// them on the stream first).
template <int N> cr_status prm_build_n(const cr_robot& robot, const PrmArgs& a, cudaStream_t st) {
  cr_robot rr = robot;
  rr.n = N;
  const RobotK<float> rbf = crh::robot_k<float>(rr);
  const RobotK<double> rbd = crh::robot_k<double>(rr);
  const unsigned R = (unsigned)a.R;
  const size_t sb = prm_sph_bytes(a.no);
  k_prm_sample<N><<<dim3((a.N + 127) / 128, R), 128, sb, st>>>(rbf, rbd, a);
  cr_status s;
  if ((s = crh::check_launch("k_prm_sample"))) return s;
  const size_t kb = (size_t)kPrmKnnWarps * a.N * 16;
  if ((s = prm_set_smem((const void*)k_prm_knn<N>, kb, "k_prm_knn"))) return s;
  k_prm_knn<N><<<dim3((a.N + kPrmKnnWarps - 1) / kPrmKnnWarps, R), 32 * kPrmKnnWarps, kb, st>>>(a);
  if ((s = crh::check_launch("k_prm_knn"))) return s;
  const int64_t ne = (int64_t)a.N * a.k * a.n_check;
  k_prm_edges<N><<<dim3((unsigned)((ne + 255) / 256), R), 256, sb, st>>>(rbf, rbd, a);
  if ((s = crh::check_launch("k_prm_edges"))) return s;
  const int64_t ns = a.R * a.N * a.k;
  k_prm_adj<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(a);
  if ((s = crh::check_launch("k_prm_adj"))) return s;
  k_prm_csr<N><<<R, ((a.N + 31) / 32) * 32, 0, st>>>(a);
  return crh::check_launch("k_prm_csr");
}

template <int N> cr_status prm_query_n(const cr_robot& robot, const PrmArgs& a, cudaStream_t st) {
  cr_robot rr = robot;
  rr.n = N;
  const size_t sm = prm_query_smem(a.no, a.N, a.k).total;
  cr_status s;
  if ((s = prm_set_smem((const void*)k_prm_query<N>, sm, "k_prm_query"))) return s;
  k_prm_query<N><<<(unsigned)a.P, kPrmQueryThreads, sm, st>>>(crh::robot_k<float>(rr), crh::robot_k<double>(rr), a);
  return crh::check_launch("k_prm_query");
}

#define CR_PRM_INSTANTIATE(EXT, N)                                                             \
  EXT template cr_status prm_build_n<N>(const cr_robot&, const PrmArgs&, cudaStream_t);        \
  EXT template cr_status prm_query_n<N>(const cr_robot&, const PrmArgs&, cudaStream_t);

}  // namespace crk
