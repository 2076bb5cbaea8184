// Host side of the C ABI declared in include/rvea.h.
//
// The library keeps a small host handle per run; every device byte belongs
// to the caller's workspace.  The workspace holds the population pool, the
// objective and reference-vector arrays, the control block, the run's device
// descriptor and its work-item tables.  rvea_step enqueues, per generation,
// reproduction -> selection -> finalize (-> gamma on adaptation
// generations), as direct launches or as replays of a CUDA graph that covers
// one adaptation period.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <new>
#include <vector>

#include "../../include/rvea.h"
#include "rvea_device.cuh"
#include "grid_steps.cuh"
#include "metrics.cuh"
#include "nvtx_range.h"

namespace rvea {
__global__ void k_reprob_dtlz1(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_dtlz2(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_neuro(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_dtlz1s(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_dtlz2s(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_neuros(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_dtlz3(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_dtlz4(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_dtlz3s(const __grid_constant__ BatchDir dir);
__global__ void k_reprob_dtlz4s(const __grid_constant__ BatchDir dir);
__global__ void k_repro1_dtlz1(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1_dtlz2(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1_neuro(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1s_dtlz1(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1s_dtlz2(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1s_neuro(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1_dtlz3(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1_dtlz4(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1s_dtlz3(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_repro1s_dtlz4(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk);
__global__ void k_mutate_dtlz1(const __grid_constant__ BatchDir dir);
__global__ void k_mutate_dtlz2(const __grid_constant__ BatchDir dir);
__global__ void k_mutate_neuro(const __grid_constant__ BatchDir dir);
__global__ void k_mutate_dtlz3(const __grid_constant__ BatchDir dir);
__global__ void k_mutate_dtlz4(const __grid_constant__ BatchDir dir);
__global__ void k_init(const __grid_constant__ BatchDir dir);
__global__ void k_repro_de_dtlz1(const __grid_constant__ BatchDir dir);
__global__ void k_repro_de_dtlz2(const __grid_constant__ BatchDir dir);
__global__ void k_repro_de_dtlz3(const __grid_constant__ BatchDir dir);
__global__ void k_repro_de_dtlz4(const __grid_constant__ BatchDir dir);
__global__ void k_repro_rand_dtlz1(const __grid_constant__ BatchDir dir);
__global__ void k_repro_rand_dtlz2(const __grid_constant__ BatchDir dir);
__global__ void k_repro_rand_dtlz3(const __grid_constant__ BatchDir dir);
__global__ void k_repro_rand_dtlz4(const __grid_constant__ BatchDir dir);
__global__ void k_cso_mean(const __grid_constant__ BatchDir dir);
__global__ void k_cso_centre(const __grid_constant__ BatchDir dir);
__global__ void k_repro_cso_dtlz1(const __grid_constant__ BatchDir dir);
__global__ void k_repro_cso_dtlz2(const __grid_constant__ BatchDir dir);
__global__ void k_repro_cso_dtlz3(const __grid_constant__ BatchDir dir);
__global__ void k_repro_cso_dtlz4(const __grid_constant__ BatchDir dir);
__global__ void k_repro_cso_neuro(const __grid_constant__ BatchDir dir);
__global__ void k_repro_pso_dtlz1(const __grid_constant__ BatchDir dir);
__global__ void k_repro_pso_dtlz2(const __grid_constant__ BatchDir dir);
__global__ void k_repro_pso_dtlz3(const __grid_constant__ BatchDir dir);
__global__ void k_repro_pso_dtlz4(const __grid_constant__ BatchDir dir);
__global__ void k_select(const __grid_constant__ BatchDir dir);
__global__ void k_finalize(const __grid_constant__ BatchDir dir);
__global__ void k_gamma(const __grid_constant__ BatchDir dir, int force);
__global__ void k_gamma_op(const __grid_constant__ RunDesc D);
__global__ void k_init_lists(const __grid_constant__ BatchDir dir);
__global__ void k_gather_pop(const RunDesc *Rp, float *dst, uint8_t *valid);
__global__ void k_gather_obj(const RunDesc *Rp, float *dst, uint8_t *valid);
__global__ void k_gather_children(const RunDesc *Rp, float *X, float *F);
__global__ void k_gather_swarm(const RunDesc *Rp, float *vel, float *apd, float *pbest, float *fpbest);
__global__ void k_copy_selection(const RunDesc *Rp, int *assoc, int *surv);
__global__ void k_import(const RunDesc *Rp, const float *Fin, const uint8_t *vin, int t);
__global__ void k_igd_partial(const RunDesc *Rp, const float *ref, int n_ref, double *partial);
__global__ void k_igd_final(const double *partial, int nb, int n_ref, double *out);
__global__ void k_hv_compact(const RunDesc *Rp, HvRef ref, HvScratch S);
__global__ void k_hv_rank(HvScratch S);
__global__ void k_hv_slices(HvScratch S, HvRef ref);
__global__ void k_hv_final(HvScratch S, double *out);
__global__ void k_op_prep(const RunDesc *Rp);
__global__ void k_op_zstar(const RunDesc *Rp);
__global__ void k_op_finish(const RunDesc *Rp);
__global__ void k_select_pruned(const RunDesc *Rp);
__global__ void k_tiles(const RunDesc *Rp);
__global__ void k_noise(const __grid_constant__ BatchDir dir, int init);
__global__ void k_rollout(const __grid_constant__ BatchDir dir, int init);
__global__ void k_rollout_f32(const __grid_constant__ BatchDir dir, int init);
size_t rollout_f32_smem(int ns, int na);
constexpr int kRollF32Policies = 2;   // policies (warps) per CTA of the FP32 rollout
__global__ void k_select_pruned_batch(const __grid_constant__ BatchDir dir);
__global__ void k_tiles_batch(const __grid_constant__ BatchDir dir, int force);
__global__ void k_tail_dtlz1(const RunDesc *Rp);
__global__ void k_tail_dtlz2(const RunDesc *Rp);
__global__ void k_tail_dtlz3(const RunDesc *Rp);
__global__ void k_tail_dtlz4(const RunDesc *Rp);
__global__ void k_grid_scale(const RunDesc *Rp);
__global__ void k_grid_count(const RunDesc *Rp);
__global__ void k_grid_scan(const RunDesc *Rp);
__global__ void k_grid_fill(const RunDesc *Rp);
}  // namespace rvea

using namespace rvea;

// ---------------------------------------------------------------------------
// shapes, layout
// ---------------------------------------------------------------------------
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int pow2ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct Shape {
  int m, m4, d, d_pad, G, N, P, n_comb, team, ppc, nseg, sg;
  int n_repro, n_init, nblk;
  int n_sel_max;   // work items of the finest full-scan plan (table size)
  int tmax;     // tiles of the pruned selection (0: not used)
  int tglob;    // 1: tables too large for shared memory (fused tail only, from L2)
  int gG, gcells, gcap;   // direction grid of the association (gG = 0: none)
};

// Pruned selection: m <= 4 and the tile-ordered vectors plus the tile table
// fit one CTA's shared memory (about 12k vectors).
constexpr int kPruneMinN = 1000;
constexpr int kTileLeaf = 64;      // vectors per k-d tile of the pruned search (<= 64)
constexpr int kSelPerSmMax = 16;   // full scan: the finest plan (work items per SM)
constexpr int kPruneChunkHost = 2048;   // solutions per work chunk of the batched pruned search
constexpr int kRollPolicies = 2;        // policies (warps) per CTA of the rollout kernel
constexpr size_t kPruneSmemCap = 200 * 1024;
int prune_tiles_bound(int N) { return N / 16 + 2; }
constexpr int kGridMaxN = 65535;   // the grid's cell lists hold 16-bit table positions
size_t prune_smem(int N, int T) {
  const size_t bS = ((size_t)T * 8 + 15) & ~size_t(15);
  return (size_t)N * 16 + (size_t)T * 16 + 2 * bS;
}

// Reproduction teams: TS lanes (a power of two <= 32) per work unit of
// up to kLaneGroups*TS groups of 8 variables; a pair has nseg = ceil(G / (kLaneGroups TS))
// units of sg = ceil(G / nseg) groups each.
// Both depend on d only, so the reduction tree of g does too.
Shape make_shape(int m, int d, int N) {
  Shape s;
  s.m = m;
  s.m4 = (m + 3) / 4;
  s.d = d;
  s.d_pad = (d + 7) / 8 * 8;
  s.G = s.d_pad / 8;
  s.N = N;
  s.P = (N + 1) / 2;
  s.n_comb = 2 * N;
  s.team = std::min(32, std::max(1, pow2ceil((s.G + kLaneGroups - 1) / kLaneGroups)));
  s.ppc = kReproThreads / s.team;                 // work units per CTA
  s.nseg = (s.G + kLaneGroups * s.team - 1) / (kLaneGroups * s.team);
  s.sg = (s.G + s.nseg - 1) / s.nseg;   // balanced segments: no mostly idle last one
  s.n_repro = (s.P * s.nseg + s.ppc - 1) / s.ppc;
  s.n_init = (N + s.ppc - 1) / s.ppc;
  // the full-scan item table holds the finest plan of any device: every
  // solution block x every kVTileMin-vector tile
  s.nblk = (s.n_comb + kSelBlock - 1) / kSelBlock;
  s.n_sel_max = s.nblk * ((N + kVTileMin - 1) / kVTileMin);
  s.tmax = 0;
  s.tglob = 0;
  if (m <= 4 && N >= kPruneMinN && prune_smem(N, prune_tiles_bound(N)) <= kPruneSmemCap) {
    s.tmax = prune_tiles_bound(N);
  } else if (m <= 3 && N >= kPruneMinN && N <= kGridMaxN) {
    // past shared memory (N above ~12.7 k at m = 3): the tables and the
    // direction grid still serve the fused tail, read through L2
    s.tmax = prune_tiles_bound(N);
    s.tglob = 1;
  }
  // direction grid (m = 2, 3, with the tile tables it is built from): steps
  // of 1/(4H) (m = 2) or 1/(2H) (m = 3) per barycentric axis, a fraction of
  // the lattice spacing 1/H, so that a cell lists a handful of vectors
  s.gG = s.gcells = s.gcap = 0;
  if (s.tmax > 0 && (m == 2 || m == 3)) {
    const int H = m == 2 ? N - 1 : (int)std::llround((std::sqrt(8.0 * N + 1.0) - 3.0) / 2.0);
    s.gG = m == 2 ? 4 * H : 2 * H;
    s.gcells = m == 2 ? s.gG : s.gG * s.gG;
    s.gcap = std::max(4096, 2 * s.gcells);   // overflow lists (cells past 15 candidates)
  }
  return s;
}

struct Layout {
  size_t X, F, slotmap, vbits, obits, zpart, vlist, child, best, amax, assoc, surv, blk, V32, V32lo, V64, V0, g64, g32,
      ctl, desc, repro, init, sel, stage, psum, rec_par, rec_sites, otag, occ_cnt, vcnt, zacc, Vt,
      tperm, trng, tcen, tcs, gcell, gcnt, gblk, gover, selb, gscale, vrange, fcomb, noise, dynA, dynB,
      vel, kapd, xbar, xpart, pb, fpb, total;
};

// op: the run's reproduction operator; CSO (3) and PSO (4) keep velocities
// and kept APDs, CSO its centre, PSO the personal bests
Layout make_layout(const Shape &s, int steps_max, int ns_max, int na_max, int op = 0) {
  const bool swarm = op == 3 || op == 4;
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.X = take((size_t)2 * s.N * s.d_pad * sizeof(float));
  L.F = take((size_t)s.m * s.n_comb * sizeof(float));
  L.slotmap = take((size_t)2 * s.N * 4);
  L.vbits = take((size_t)((s.N + 31) / 32) * 4);
  L.obits = take((size_t)((2 * s.N + 31) / 32) * 4);
  L.zpart = take((size_t)((s.N + 1023) / 1024) * 2 * kMaxM * 4);
  L.vlist = take((size_t)s.N * 4);
  L.child = take((size_t)2 * s.N * 4);
  L.best = take((size_t)s.N * 8);
  L.amax = take((size_t)s.n_comb * 8);
  L.assoc = take((size_t)s.n_comb * 4);
  L.surv = take((size_t)s.N * 4);
  L.blk = take((size_t)s.nblk * 4);   // selection blocks of kSelBlock solutions
  L.V32 = take((size_t)s.N * s.m4 * 16);
  L.V32lo = take((size_t)s.N * s.m * 4);
  L.V64 = take((size_t)s.N * s.m * 8);
  L.V0 = take((size_t)s.N * s.m * 8);
  L.g64 = take((size_t)s.N * 8);
  L.g32 = take((size_t)s.N * 4);
  L.ctl = take(sizeof(Ctl));
  L.desc = take(sizeof(RunDesc));
  L.repro = take((size_t)s.n_repro * sizeof(ReproItem));
  L.init = take((size_t)s.n_init * sizeof(ReproItem));
  L.sel = take((size_t)s.n_sel_max * sizeof(SelItem));
  L.selb = take((size_t)s.n_sel_max * sizeof(SelItem));   // the batch's coarse table
  L.stage = take((size_t)s.N * (kMaxM + 1) * 4);
  L.psum = take((size_t)s.P * 2 * s.nseg * 4);
  L.rec_par = take((size_t)2 * s.P * 4);
  L.rec_sites = take((size_t)s.N * (1 + kMaxSites) * 4);
  L.otag = take((size_t)2 * s.N * 4);
  L.occ_cnt = take((size_t)kTailMaxCtas * 4);
  L.vcnt = take((size_t)kTailMaxCtas * 4);
  L.zacc = take((size_t)3 * kTailMaxCtas * 4 * 4);
  const size_t T = (size_t)s.tmax;
  L.Vt = take(s.tmax ? (size_t)s.N * 16 : 0);
  L.tperm = take(s.tmax ? (size_t)s.N * 4 : 0);
  L.trng = take(T * 8 + 16);
  L.tcen = take(T * 16);
  L.tcs = take(T * 8 + 16);
  L.gcell = take((size_t)s.gcells * 32);
  L.gcnt = take((size_t)s.gcells * 4);
  L.gblk = take((size_t)(s.gG > 0 ? grid_build_blocks(s.gG, s.m) + 1 : 0) * 4);
  L.gover = take(((size_t)(s.gG > 0 ? grid_build_blocks(s.gG, s.m) : 0) * kGridBlockCap + s.gcap) * 2);
  L.gscale = take(kMaxM * 4);
  L.vrange = take(kMaxM * 8);
  L.fcomb = take((size_t)2 * s.m * s.n_comb * 4);
  L.noise = take((size_t)steps_max * ns_max * 4);
  L.dynA = take((size_t)ns_max * ns_max * 4);
  L.dynB = take((size_t)ns_max * na_max * 4);
  const size_t nch = (size_t)(s.N + kMeanRows - 1) / kMeanRows;
  L.vel = take(swarm ? (size_t)2 * s.N * s.d_pad * sizeof(float) : 0);
  L.kapd = take(swarm ? (size_t)s.N * 4 : 0);
  L.xbar = take(op == 3 ? (size_t)s.d_pad * 4 : 0);
  L.xpart = take(op == 3 ? nch * s.d_pad * 4 : 0);
  L.pb = take(op == 4 ? (size_t)2 * s.N * s.d_pad * sizeof(float) : 0);
  L.fpb = take(op == 4 ? (size_t)s.m * s.n_comb * sizeof(float) : 0);
  L.total = o;
  return L;
}

int64_t lattice_size(int m, int H) {
  // C(H+m-1, m-1), saturating at 2^40
  long double c = 1.0L;
  for (int i = 1; i <= m - 1; ++i) {
    c = c * (long double)(H + i) / (long double)i;
    if (c > 1e12L) return (int64_t)1 << 40;
  }
  return (int64_t)llroundl(c);
}

// Das-Dennis lattice {k in N^m : sum k = H}, lexicographic in k_1..k_{m-1},
// each row scaled to unit length (FP64: one sqrt and one division per
// component, both correctly rounded).
void build_lattice(int m, int H, int N, std::vector<double> &V0) {
  V0.assign((size_t)N * m, 0.0);
  std::vector<int> k(m, 0);
  k[m - 1] = H;
  for (int row = 0; row < N; ++row) {
    double s = 0.0;
    for (int q = 0; q < m; ++q) s += (double)k[q] * (double)k[q];
    const double nrm = std::sqrt(s);
    for (int q = 0; q < m; ++q) V0[(size_t)row * m + q] = (double)k[q] / nrm;
    // next composition: increase the rightmost k_q (q < m-1) that can grow
    int q = m - 2;
    while (q >= 0) {
      int used = 0;
      for (int u = 0; u <= q; ++u) used += k[u];
      if (used < H) break;
      --q;
    }
    if (q < 0) break;
    k[q] += 1;
    for (int u = q + 1; u < m - 1; ++u) k[u] = 0;
    int used = 0;
    for (int u = 0; u < m - 1; ++u) used += k[u];
    k[m - 1] = H - used;
  }
}

// Spatially compact tiles of <= 32 reference vectors: recursive split of
// the initial lattice along its widest coordinate (cuts at multiples of 32
// while the part is large, then in halves).  Returns the tile-order
// permutation and each tile's (first position, count).
void build_tiles(const std::vector<double> &V0, int N, int m, std::vector<int> &perm,
                 std::vector<int2> &rng) {
  perm.resize(N);
  for (int j = 0; j < N; ++j) perm[j] = j;
  rng.clear();
  std::vector<std::pair<int, int>> todo{{0, N}};
  while (!todo.empty()) {
    const auto [a, b] = todo.back();
    todo.pop_back();
    const int n = b - a;
    if (n <= kTileLeaf) {
      rng.push_back(make_int2(a, n));
      continue;
    }
    int axis = 0;
    double spread = -1.0;
    for (int k = 0; k < m; ++k) {
      double lo = 1e300, hi = -1e300;
      for (int q = a; q < b; ++q) {
        const double v = V0[(size_t)perm[q] * m + k];
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
      if (hi - lo > spread) { spread = hi - lo; axis = k; }
    }
    std::stable_sort(perm.begin() + a, perm.begin() + b, [&](int x, int y) {
      return V0[(size_t)x * m + axis] < V0[(size_t)y * m + axis];
    });
    int h = n / 2;
    if (n > 2 * kTileLeaf) h = std::max(kTileLeaf, h / kTileLeaf * kTileLeaf);
    todo.push_back({a + h, b});
    todo.push_back({a, a + h});
  }
  std::sort(rng.begin(), rng.end(), [](int2 x, int2 y) { return x.x < y.x; });
}

uint32_t event_threshold24(double q) {
  double x = std::ceil(q * 16777216.0);
  if (x < 0.0) x = 0.0;
  if (x > 16777216.0) x = 16777216.0;
  return (uint32_t)x;
}

// Site-count thresholds of polynomial mutation.  The sites of a child row are
// independent events of probability q (Appendix B: one uniform per site
// against p_m/d); the kernel draws them as a count k ~ Binomial(d, q) and a
// uniform k-subset, the same law.  Draw 0 of the row gives the count
// k = #{i : w >= thr_i}, thr_i = floor(2^32 CDF(i)) for the i < min(d, 32)
// with CDF(i) < 1.  CDF is summed in FP64 from pmf(0) = (1-q)^d (square and
// multiply over the bits of d, least significant first) and
// pmf(i+1) = pmf(i) * (d-i) / (i+1) * (q/(1-q)); this file is compiled
// without floating-point contraction, so the sums are the plain IEEE ones.
int site_count_thresholds(double q, int d, uint32_t *thr) {
  const int K = std::min(d, kMaxSites);
  const double ratio = q / (1.0 - q);
  double b = 1.0 - q, pmf = 1.0;
  for (int e = d; e > 0; e >>= 1) {
    if (e & 1) pmf *= b;
    b *= b;
  }
  double cdf = 0.0;
  int n = 0;
  for (int i = 0; i < K; ++i) {
    if (i > 0) pmf = pmf * (double)(d - (i - 1)) / (double)i * ratio;
    cdf += pmf;
    if (cdf >= 1.0) break;
    thr[n++] = (uint32_t)std::floor(cdf * 4294967296.0);
  }
  return n;
}

std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;
int g_tail_dyn_max = 0;   // dynamic shared memory the fused tail kernel can take

thread_local cudaError_t g_last_err = cudaSuccess;
thread_local const char *g_last_where = "";

void note_error(cudaError_t e, const char *where) {
  if (e != cudaSuccess) {
    g_last_err = e;
    g_last_where = where;
  }
}

void set_kernel_attrs() {
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f) {
    // dynamic + static shared memory may not exceed the opt-in limit
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, f);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
    if (r != cudaSuccess && e == cudaSuccess) e = r;
    note_error(r, "cudaFuncSetAttribute");
  };
  set((const void *)k_reprob_dtlz1);
  set((const void *)k_reprob_dtlz2);
  set((const void *)k_reprob_neuro);
  set((const void *)k_reprob_dtlz1s);
  set((const void *)k_reprob_dtlz2s);
  set((const void *)k_reprob_neuros);
  set((const void *)k_repro1_dtlz1);
  set((const void *)k_repro1_dtlz2);
  set((const void *)k_repro1_neuro);
  set((const void *)k_repro1s_dtlz1);
  set((const void *)k_repro1s_dtlz2);
  set((const void *)k_repro1s_neuro);
  set((const void *)k_reprob_dtlz3);
  set((const void *)k_reprob_dtlz4);
  set((const void *)k_reprob_dtlz3s);
  set((const void *)k_reprob_dtlz4s);
  set((const void *)k_repro1_dtlz3);
  set((const void *)k_repro1_dtlz4);
  set((const void *)k_repro1s_dtlz3);
  set((const void *)k_repro1s_dtlz4);
  set((const void *)k_init);
  set((const void *)k_select);
  set((const void *)k_select_pruned);
  set((const void *)k_select_pruned_batch);
  set((const void *)k_rollout_f32);
  set((const void *)k_tail_dtlz1);
  {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void *)k_tail_dtlz1) == cudaSuccess)
      g_tail_dyn_max = optin - (int)fa.sharedSizeBytes;
  }
  set((const void *)k_tail_dtlz2);
  set((const void *)k_tail_dtlz3);
  set((const void *)k_tail_dtlz4);

  g_attr_err = e;
}

}  // namespace

// ---------------------------------------------------------------------------
// the run handle
// ---------------------------------------------------------------------------
struct rvea_run {
  rvea_config cfg;
  Shape sh;
  Layout lay;
  uint8_t *ws = nullptr;
  int p_adapt = 1;
  int t = 1;                      // host mirror of ctl->t
  int device = 0;
  RunDesc hd;                     // host copy of the device descriptor
  RunDesc *d_desc = nullptr;
  int repro_smem = 0, init_smem = 0, sel_smem = 0, fin_smem = 0;
  int prune_smem_bytes = 0, num_sms = 152;
  // kernel variants (the plan): none of them changes the results
  int sel_mode = 0;               // 0 full scan, 1 pruned (tables in shared memory), 2 pruned (L1)
  int sel_per_sm = 8;             // full scan: work items per SM
  int n_sel = 0;                  // full scan: work items of the current plan
  int n_selb = 0, selb_smem = 0;  // the coarse table a batch uses (8 items per SM, 512-vector tiles)
  bool tuned = false;
  double tune_repro_us = 0.0, tune_sel_us = 0.0;
  std::vector<SelItem> sel_host;  // source of the last upload of the item table
  cudaStream_t last_stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t block_graph = nullptr;
  cudaGraphExec_t plain_graph = nullptr;   // kPlainGens generations without an adaptation
  bool use_graph = true;
  bool has_last_gen = false;      // a generation ran since init / import
  bool recording = false;         // draws recorded by the generations now enqueued
  bool last_gen_recorded = false; // the last generation ran with recording on
};

namespace {

rvea_status cuerr_at(cudaError_t e, const char *where) {
  note_error(e, where);
  return e == cudaSuccess ? RVEA_OK : RVEA_ERR_CUDA;
}
#define cuerr(e) cuerr_at((e), #e)

#define RV_TRY(x)                                    \
  do {                                               \
    const cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) {                         \
      note_error(_e, #x);                            \
      return RVEA_ERR_CUDA;                          \
    }                                                \
  } while (0)

void dir_single(BatchDir &dir, const rvea_run *r, const void *items, int n_items) {
  dir.n = 1;
  dir.prefix[0] = 0;
  dir.prefix[1] = n_items;
  dir.desc[0] = r->d_desc;
  dir.items[0] = items;
  dir.key[0] = make_uint2(r->hd.key0, r->hd.key1);
}

template <class T>
T *wsp(const rvea_run *r, size_t off) {
  return reinterpret_cast<T *>(r->ws + off);
}

// Launch with programmatic stream serialisation: the kernel may start while
// its predecessor in the stream finishes; every kernel of a generation waits
// (griddepcontrol.wait) before reading its predecessor's results.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                cudaStream_t st, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_error(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...), "cudaLaunchKernelEx");
}

// Item table of the full-scan association for the run's current plan
// (sel_per_sm work items per SM), into sel_host; n_sel and the shared memory
// of one chunk follow.
void build_sel_items(rvea_run *r) {
  const Shape &sh = r->sh;
  const SelPlan sp = sel_plan(sh.n_comb, sh.N, sh.m4, r->num_sms, r->sel_per_sm);
  r->sel_host.clear();
  for (int b = 0; b < sp.nblk; ++b)
    for (int c = 0; c < sp.nch; ++c)
      r->sel_host.push_back(SelItem{b, std::min(sh.N, c * sp.chunk),
                                    std::min(sh.N, (c + 1) * sp.chunk), sp.nch});
  r->n_sel = (int)r->sel_host.size();
  r->sel_smem = std::min(sh.N, sp.chunk) * sh.m4 * 16;
}

// Reproduction of one run: the kernel instance for its problem, round keys
// in the parameter block; 32-lane teams stage the parents in shared memory.
void launch_repro1(const rvea_run *r, const BatchDir &dr, int grid, cudaStream_t st) {
  const RoundKeys rk = round_keys(r->hd.key0, r->hd.key1);
  const int sm = r->repro_smem;
  if (sm > 0) {
    switch (r->hd.problem) {
      case PROB_DTLZ1: launch_pdl(k_repro1s_dtlz1, grid, kReproThreads, sm, st, dr, rk); break;
      case PROB_DTLZ2: launch_pdl(k_repro1s_dtlz2, grid, kReproThreads, sm, st, dr, rk); break;
      case PROB_DTLZ3: launch_pdl(k_repro1s_dtlz3, grid, kReproThreads, sm, st, dr, rk); break;
      case PROB_DTLZ4: launch_pdl(k_repro1s_dtlz4, grid, kReproThreads, sm, st, dr, rk); break;
      default: launch_pdl(k_repro1s_neuro, grid, kReproThreads, sm, st, dr, rk); break;
    }
    return;
  }
  switch (r->hd.problem) {
    case PROB_DTLZ1: launch_pdl(k_repro1_dtlz1, grid, kReproThreads, 0, st, dr, rk); break;
    case PROB_DTLZ2: launch_pdl(k_repro1_dtlz2, grid, kReproThreads, 0, st, dr, rk); break;
    case PROB_DTLZ3: launch_pdl(k_repro1_dtlz3, grid, kReproThreads, 0, st, dr, rk); break;
    case PROB_DTLZ4: launch_pdl(k_repro1_dtlz4, grid, kReproThreads, 0, st, dr, rk); break;
    default: launch_pdl(k_repro1_neuro, grid, kReproThreads, 0, st, dr, rk); break;
  }
}

// Rollouts of the children (or of the initial population, init = 1) of the
// rollout-problem runs among `runs`: one directory per GEMV form.
void launch_rollouts(rvea_run *const *runs, int n, cudaStream_t st, int init, bool pdl) {
  static thread_local BatchDir dm, df;
  int nm = 0, nf = 0, pm = 0, pf = 0;
  size_t smf = 0;
  for (int q = 0; q < n; ++q) {
    const rvea_run *r = runs[q];
    if (r->hd.problem != PROB_NEURO) continue;
    const bool f32 = r->hd.roll_f32 != 0;
    BatchDir &D = f32 ? df : dm;
    int &k = f32 ? nf : nm;
    int &p = f32 ? pf : pm;
    D.prefix[k] = p;
    D.desc[k] = r->d_desc;
    D.key[k] = make_uint2(r->hd.key0, r->hd.key1);
    D.items[k] = nullptr;
    p += f32 ? (r->sh.N + kRollF32Policies - 1) / kRollF32Policies
             : (r->sh.N + kRollPolicies - 1) / kRollPolicies;
    if (f32) smf = std::max(smf, rollout_f32_smem(r->hd.ns, r->hd.na));
    ++k;
  }
  if (nm > 0) {
    dm.n = nm;
    dm.prefix[nm] = pm;
    if (pdl) launch_pdl(k_rollout, pm, 32 * kRollPolicies, 0, st, dm, init);
    else k_rollout<<<pm, 32 * kRollPolicies, 0, st>>>(dm, init);
  }
  if (nf > 0) {
    df.n = nf;
    df.prefix[nf] = pf;
    if (pdl) launch_pdl(k_rollout_f32, pf, 32 * kRollF32Policies, smf, st, df, init);
    else k_rollout_f32<<<pf, 32 * kRollF32Policies, smf, st>>>(df, init);
  }
}

// Reproduction by DE/rand/1/bin, random reproduction or CSO (the runs whose
// operator is not SBX): one kernel per (problem, CSO or not) over a
// directory of such runs, one warp per offspring.
constexpr int kOpWarps = kReproThreads / 32;
void launch_repro_op(const BatchDir &d, int problem, int grid, cudaStream_t st, int op) {
  if (op == 4) {
    switch (problem) {
      case PROB_DTLZ1: launch_pdl(k_repro_pso_dtlz1, grid, kReproThreads, 0, st, d); break;
      case PROB_DTLZ3: launch_pdl(k_repro_pso_dtlz3, grid, kReproThreads, 0, st, d); break;
      case PROB_DTLZ4: launch_pdl(k_repro_pso_dtlz4, grid, kReproThreads, 0, st, d); break;
      default: launch_pdl(k_repro_pso_dtlz2, grid, kReproThreads, 0, st, d); break;
    }
    return;
  }
  if (op == 3) {
    switch (problem) {
      case PROB_DTLZ1: launch_pdl(k_repro_cso_dtlz1, grid, kReproThreads, 0, st, d); break;
      case PROB_DTLZ3: launch_pdl(k_repro_cso_dtlz3, grid, kReproThreads, 0, st, d); break;
      case PROB_DTLZ4: launch_pdl(k_repro_cso_dtlz4, grid, kReproThreads, 0, st, d); break;
      case PROB_NEURO: launch_pdl(k_repro_cso_neuro, grid, kReproThreads, 0, st, d); break;
      default: launch_pdl(k_repro_cso_dtlz2, grid, kReproThreads, 0, st, d); break;
    }
    return;
  }
  if (op == 1) {
    switch (problem) {
      case PROB_DTLZ1: launch_pdl(k_repro_de_dtlz1, grid, kReproThreads, 0, st, d); break;
      case PROB_DTLZ3: launch_pdl(k_repro_de_dtlz3, grid, kReproThreads, 0, st, d); break;
      case PROB_DTLZ4: launch_pdl(k_repro_de_dtlz4, grid, kReproThreads, 0, st, d); break;
      default: launch_pdl(k_repro_de_dtlz2, grid, kReproThreads, 0, st, d); break;
    }
    return;
  }
  switch (problem) {
    case PROB_DTLZ1: launch_pdl(k_repro_rand_dtlz1, grid, kReproThreads, 0, st, d); break;
    case PROB_DTLZ3: launch_pdl(k_repro_rand_dtlz3, grid, kReproThreads, 0, st, d); break;
    case PROB_DTLZ4: launch_pdl(k_repro_rand_dtlz4, grid, kReproThreads, 0, st, d); break;
    default: launch_pdl(k_repro_rand_dtlz2, grid, kReproThreads, 0, st, d); break;
  }
}
// The CSO runs' swarm centres (k_cso_mean), before their reproduction; runs
// with phi = 0 do not use the centre.
int cso_mean_blocks(const rvea_run *r) {
  return (r->sh.d_pad + kMeanCols - 1) / kMeanCols * ((r->sh.N + kMeanRows - 1) / kMeanRows);
}
bool cso_needs_mean(const rvea_run *r) { return r->hd.op == 3 && r->hd.cso_phi != 0.0f; }
void launch_cso_means(rvea_run *const *runs, int n, cudaStream_t st) {
  static thread_local BatchDir d, dc;
  int nd = 0, p = 0, pc = 0;
  for (int q = 0; q < n; ++q) {
    const rvea_run *r = runs[q];
    if (!cso_needs_mean(r)) continue;
    d.prefix[nd] = p;
    dc.prefix[nd] = pc;
    d.desc[nd] = dc.desc[nd] = r->d_desc;
    d.key[nd] = dc.key[nd] = make_uint2(r->hd.key0, r->hd.key1);
    d.items[nd] = dc.items[nd] = nullptr;
    p += cso_mean_blocks(r);
    pc += (r->sh.d_pad / 4 + 7) / 8;   // one warp per float4 of variables
    ++nd;
  }
  if (nd == 0) return;
  d.n = dc.n = nd;
  d.prefix[nd] = p;
  dc.prefix[nd] = pc;
  launch_pdl(k_cso_mean, p, 256, 0, st, d);
  launch_pdl(k_cso_centre, pc, 256, 0, st, dc);
}
void launch_repro_op1(const rvea_run *r, cudaStream_t st) {
  static thread_local BatchDir d;
  rvea_run *one[1] = {const_cast<rvea_run *>(r)};
  launch_cso_means(one, 1, st);
  const int nb = (r->sh.N + kOpWarps - 1) / kOpWarps;
  dir_single(d, r, nullptr, nb);
  launch_repro_op(d, r->hd.problem, nb, st, r->hd.op);
}

// Mutation and evaluation of the children of a run reproduced by 32-lane
// teams (d > 1024), after its reproduction kernel; nothing for other runs.
void launch_mutate1(const rvea_run *r, cudaStream_t st) {
  if (r->sh.team != 32 || r->hd.op != 0) return;
  static thread_local BatchDir dm;
  const int nb = (r->sh.N + kMutThreads - 1) / kMutThreads;
  dir_single(dm, r, nullptr, nb);
  switch (r->hd.problem) {
    case PROB_DTLZ1: launch_pdl(k_mutate_dtlz1, nb, kMutThreads, 0, st, dm); break;
    case PROB_DTLZ2: launch_pdl(k_mutate_dtlz2, nb, kMutThreads, 0, st, dm); break;
    case PROB_DTLZ3: launch_pdl(k_mutate_dtlz3, nb, kMutThreads, 0, st, dm); break;
    case PROB_DTLZ4: launch_pdl(k_mutate_dtlz4, nb, kMutThreads, 0, st, dm); break;
    default: launch_pdl(k_mutate_neuro, nb, kMutThreads, 0, st, dm); break;
  }
}

// The fused tail (k_tail: mutation and evaluation, association, finalize in
// one persistent launch) serves one run of a DTLZ problem with the pruned
// search, when each CTA's share of the pool-row bitmap fits its buffer, its
// children fit its lanes (eight a child) and the search tables its shared
// memory (or, past that, the tables are read through L2).
// One CTA per SM but for the last 24 to free up: the tail's CTAs become
// resident as the reproduction kernel drains (each takes a whole SM), and the
// SMs that finish it last would start their phase A late (measured over
// 10000 generations on 152 SMs: 152 CTAs 97.5, 144 CTAs 97.07, 136 CTAs
// 96.84, 128 CTAs 96.44, 120 CTAs 96.48 us a generation).
int tail_grid(const rvea_run *r) {
  return std::min(r->num_sms > 64 ? r->num_sms - 24 : r->num_sms, kTailMaxCtas);
}
bool tail_ok(const rvea_run *r) {
  return r->hd.ntiles > 0 && r->hd.problem != PROB_NEURO &&
         (2 * r->sh.N + 31) / 32 <= 64 * tail_grid(r) &&
         r->sh.N <= 4 * (kTailThreads / 32) * tail_grid(r) &&   // a group of 8 lanes a child
         (r->hd.tables_global || r->prune_smem_bytes <= g_tail_dyn_max);
}
// dynamic shared memory of the fused tail: the staged tables, or none
int tail_smem(const rvea_run *r) { return r->hd.tables_global ? 0 : r->prune_smem_bytes; }
void launch_tail(const rvea_run *r, cudaStream_t st, bool pdl) {
  const int g = tail_grid(r), sm = tail_smem(r);
  const RunDesc *d = r->d_desc;
  void (*k)(const RunDesc *) = r->hd.problem == PROB_DTLZ1   ? k_tail_dtlz1
                               : r->hd.problem == PROB_DTLZ3 ? k_tail_dtlz3
                               : r->hd.problem == PROB_DTLZ4 ? k_tail_dtlz4
                                                             : k_tail_dtlz2;
  if (pdl) launch_pdl(k, g, kTailThreads, sm, st, d);
  else k<<<g, kTailThreads, sm, st>>>(d);
}

// Enqueue one generation of every run in `runs` (one launch per phase): the
// reproduction of all runs; the association of the pruned runs (one
// persistent launch) and of the full-scan runs; finalize; with
// gamma_by_flag, gamma and the tile tables of the runs that adapted.
rvea_status launch_generation(rvea_run *const *runs, int n, cudaStream_t st, bool gamma_by_flag,
                              cudaEvent_t *ev = nullptr) {
  static thread_local BatchDir dr, ds, dp, df, dd, dt, dg[2 * kProblems];
  int pr = 0, ps = 0, pp = 0, pd = 0, pt = 0;
  int sms = 0, smp = 0, ns = 0, np = 0, nt = 0;
  dr.n = df.n = dd.n = n;
  for (int q = 0; q < n; ++q) {
    const rvea_run *r = runs[q];
    const uint2 key = make_uint2(r->hd.key0, r->hd.key1);
    dr.prefix[q] = pr;
    df.prefix[q] = q;
    dd.prefix[q] = pd;
    dr.desc[q] = df.desc[q] = dd.desc[q] = r->d_desc;
    dr.key[q] = df.key[q] = dd.key[q] = key;
    dr.items[q] = wsp<ReproItem>(r, r->lay.repro);
    df.items[q] = dd.items[q] = nullptr;
    pd += (r->sh.N + 1023) / 1024;
    pr += r->sh.n_repro;
    // tables in L2 (too large for shared memory) serve only the fused tail,
    // which steps a run alone: in a batch such a run takes the full scan,
    // its tiles kept current
    if (r->sel_mode != 0 && r->hd.ntiles > 0) {
      dt.prefix[nt] = pt;
      dt.desc[nt] = r->d_desc;
      dt.key[nt] = key;
      dt.items[nt] = nullptr;
      pt += (r->hd.ntiles + 7) / 8;
      ++nt;
    }
    if (r->sel_mode == 0 || (n > 1 && r->hd.tables_global)) {
      ds.prefix[ns] = ps;
      ds.desc[ns] = r->d_desc;
      ds.key[ns] = key;
      // alone: the run's plan; in a batch: the coarse table (the runs fill
      // the GPU together, and finer chunks only add per-item overhead)
      ds.items[ns] = wsp<SelItem>(r, n > 1 ? r->lay.selb : r->lay.sel);
      ps += n > 1 ? r->n_selb : r->n_sel;
      sms = std::max(sms, n > 1 ? r->selb_smem : r->sel_smem);
      ++ns;
    } else {
      dp.prefix[np] = pp;
      dp.desc[np] = r->d_desc;
      dp.key[np] = key;
      dp.items[np] = nullptr;
      pp += (r->sh.n_comb + kPruneChunkHost - 1) / kPruneChunkHost;
      smp = std::max(smp, r->prune_smem_bytes);
      ++np;
    }
  }
  dr.prefix[n] = pr;
  df.prefix[n] = n;
  dd.prefix[n] = pd;
  ds.n = ns;
  ds.prefix[ns] = ps;
  dp.n = np;
  dp.prefix[np] = pp;
  dt.n = nt;
  dt.prefix[nt] = pt;
  if (ev) cudaEventRecord(ev[0], st);
  const bool fused = n == 1 && runs[0]->sel_mode == 3;
  if (n == 1) {
    if (runs[0]->hd.op != 0) {
      launch_repro_op1(runs[0], st);
    } else {
      launch_repro1(runs[0], dr, pr, st);
      if (!fused) launch_mutate1(runs[0], st);
    }
  } else {
    // one launch per (problem, load path) group, each with its own directory
    int pg[2 * kProblems] = {};
    for (int g = 0; g < 2 * kProblems; ++g) dg[g].n = 0;
    // the runs with another operator: one launch per (problem, operator:
    // DE, random, CSO, PSO)
    static thread_local BatchDir dop[4 * kProblems];
    int pop[4 * kProblems] = {};
    for (int g = 0; g < 4 * kProblems; ++g) dop[g].n = 0;
    for (int q = 0; q < n; ++q) {
      const rvea_run *r = runs[q];
      if (r->hd.op == 0) continue;
      const int g = 4 * r->hd.problem + (r->hd.op - 1);
      BatchDir &D = dop[g];
      D.prefix[D.n] = pop[g];
      D.desc[D.n] = r->d_desc;
      D.key[D.n] = make_uint2(r->hd.key0, r->hd.key1);
      D.items[D.n] = nullptr;
      pop[g] += (r->sh.N + kOpWarps - 1) / kOpWarps;
      ++D.n;
    }
    launch_cso_means(runs, n, st);
    for (int g = 0; g < 4 * kProblems; ++g) {
      if (dop[g].n == 0) continue;
      dop[g].prefix[dop[g].n] = pop[g];
      launch_repro_op(dop[g], g / 4, pop[g], st, g % 4 + 1);
    }
    for (int q = 0; q < n; ++q) {
      const rvea_run *r = runs[q];
      if (r->hd.op != 0) continue;
      const int g = r->hd.problem * 2 + (r->repro_smem > 0 ? 1 : 0);
      BatchDir &D = dg[g];
      D.prefix[D.n] = pg[g];
      D.desc[D.n] = r->d_desc;
      D.key[D.n] = make_uint2(r->hd.key0, r->hd.key1);
      D.items[D.n] = wsp<ReproItem>(r, r->lay.repro);
      pg[g] += r->sh.n_repro;
      ++D.n;
    }
    for (int g = 0; g < 2 * kProblems; ++g) {
      if (dg[g].n == 0) continue;
      dg[g].prefix[dg[g].n] = pg[g];
      const int sm = (g & 1) ? kStagedSmem : 0;
      switch (g) {
        case 0: launch_pdl(k_reprob_dtlz2, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 1: launch_pdl(k_reprob_dtlz2s, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 2: launch_pdl(k_reprob_dtlz1, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 3: launch_pdl(k_reprob_dtlz1s, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 4: launch_pdl(k_reprob_neuro, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 5: launch_pdl(k_reprob_neuros, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 6: launch_pdl(k_reprob_dtlz3, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 7: launch_pdl(k_reprob_dtlz3s, pg[g], kReproThreads, sm, st, dg[g]); break;
        case 8: launch_pdl(k_reprob_dtlz4, pg[g], kReproThreads, sm, st, dg[g]); break;
        default: launch_pdl(k_reprob_dtlz4s, pg[g], kReproThreads, sm, st, dg[g]); break;
      }
    }
    // mutation / evaluation of the 32-lane-team runs, one launch per problem
    static thread_local BatchDir dm[kProblems];
    int pm[kProblems] = {};
    for (int g = 0; g < kProblems; ++g) dm[g].n = 0;
    for (int q = 0; q < n; ++q) {
      const rvea_run *r = runs[q];
      if (r->sh.team != 32 || r->hd.op != 0) continue;
      BatchDir &D = dm[r->hd.problem];
      D.prefix[D.n] = pm[r->hd.problem];
      D.desc[D.n] = r->d_desc;
      D.key[D.n] = make_uint2(r->hd.key0, r->hd.key1);
      D.items[D.n] = nullptr;
      pm[r->hd.problem] += (r->sh.N + kMutThreads - 1) / kMutThreads;
      ++D.n;
    }
    for (int g = 0; g < kProblems; ++g) {
      if (dm[g].n == 0) continue;
      dm[g].prefix[dm[g].n] = pm[g];
      switch (g) {
        case PROB_DTLZ1: launch_pdl(k_mutate_dtlz1, pm[g], kMutThreads, 0, st, dm[g]); break;
        case PROB_DTLZ2: launch_pdl(k_mutate_dtlz2, pm[g], kMutThreads, 0, st, dm[g]); break;
        case PROB_DTLZ3: launch_pdl(k_mutate_dtlz3, pm[g], kMutThreads, 0, st, dm[g]); break;
        case PROB_DTLZ4: launch_pdl(k_mutate_dtlz4, pm[g], kMutThreads, 0, st, dm[g]); break;
        default: launch_pdl(k_mutate_neuro, pm[g], kMutThreads, 0, st, dm[g]); break;
      }
    }
  }
  {
    // evaluation of the rollout problem's children: noise of generation t,
    // then one warp per policy
    static thread_local BatchDir dn;
    int nn = 0, pn = 0;
    for (int q = 0; q < n; ++q) {
      const rvea_run *r = runs[q];
      if (r->hd.problem != PROB_NEURO) continue;
      dn.prefix[nn] = pn;
      dn.desc[nn] = r->d_desc;
      dn.key[nn] = make_uint2(r->hd.key0, r->hd.key1);
      dn.items[nn] = nullptr;
      pn += (r->hd.steps * r->hd.ns + 255) / 256;
      ++nn;
    }
    if (nn > 0) {
      dn.n = nn;
      dn.prefix[nn] = pn;
      launch_pdl(k_noise, pn, 256, 0, st, dn, 0);
      launch_rollouts(runs, n, st, 0, true);
    }
  }
  if (ev) cudaEventRecord(ev[1], st);
  if (fused) {
    launch_tail(runs[0], st, true);
  } else if (np > 0) {
    if (n == 1 && runs[0]->sel_mode == 1)
      launch_pdl(k_select_pruned, runs[0]->num_sms, 1024, runs[0]->prune_smem_bytes, st,
                 (const RunDesc *)runs[0]->d_desc);
    else
      launch_pdl(k_select_pruned_batch, runs[0]->num_sms, 1024, smp, st, dp);
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (ns > 0) launch_pdl(k_select, ps, kSelThreads, sms, st, ds);
  if (ev) cudaEventRecord(ev[3], st);
  if (!fused) launch_pdl(k_finalize, pd, 1024, 0, st, dd);
  if (ev) cudaEventRecord(ev[4], st);
  if (gamma_by_flag) {
    if (nt > 0) k_tiles_batch<<<pt, 256, 0, st>>>(dt, 0);
    // one pass: every vector of the largest run has its lanes (the tile
    // search gives each warp four vectors, a second round would double the
    // chain), between two and four CTAs per SM
    int nbg = 0;
    for (int q = 0; q < n; ++q) nbg = std::max(nbg, (runs[q]->sh.N + 31) / 32);
    nbg = std::min(std::max(nbg, 2 * runs[0]->num_sms), 4 * runs[0]->num_sms);
    k_gamma<<<nbg, 256, 0, st>>>(df, 0);
  }
  if (ev) cudaEventRecord(ev[5], st);
  return cuerr(cudaGetLastError());
}

rvea_status launch_gamma_force(rvea_run *r, cudaStream_t st) {
  static thread_local BatchDir d;
  dir_single(d, r, nullptr, 1);
  const int nb = (r->sh.N + 31) / 32;   // the tile search: 32 vectors a CTA
  k_gamma<<<std::min(nb, 4 * r->num_sms), 256, 0, st>>>(d, 1);
  return cuerr(cudaGetLastError());
}

// Tile table of the pruned selection after a change of V, then the direction
// grid built from it (marked current for this V when it fits its buffer).
rvea_status launch_tiles(rvea_run *r, cudaStream_t st) {
  if (r->hd.ntiles == 0) return RVEA_OK;
  k_tiles<<<(r->hd.ntiles + 7) / 8, 256, 0, st>>>(r->d_desc);
  if (r->hd.gG > 0) {
    const int nb = grid_build_blocks(r->hd.gG, r->sh.m);   // one CTA per block of cells
    k_grid_scale<<<1, 32, 0, st>>>(r->d_desc);
    k_grid_count<<<nb, 256, 0, st>>>(r->d_desc);
    k_grid_scan<<<1, 1024, 0, st>>>(r->d_desc);
    k_grid_fill<<<nb, 256, 0, st>>>(r->d_desc);
  }
  return cuerr(cudaGetLastError());
}

// One generation of a single run; gamma (and the tile table) are enqueued by
// the host when the generation adapts (t % p_adapt == 0), so no launch is
// spent otherwise.
rvea_status enqueue_one(rvea_run *r, cudaStream_t st) {
  rvea_run *one[1] = {r};
  rvea_status s = launch_generation(one, 1, st, false);
  if (s != RVEA_OK) return s;
  if (r->t % r->p_adapt == 0) {
    s = launch_tiles(r, st);   // the tiles first: gamma searches them
    if (s == RVEA_OK) s = launch_gamma_force(r, st);
  }
  return s;
}

// kPlainGens generations none of which adapts, captured once: rvea_step
// replays it for stretches of generations that hold no adaptation (the
// kernels read the generation index from the control block, so the same
// graph serves any such stretch).
constexpr int kPlainGens = 8;
rvea_status ensure_plain_graph(rvea_run *r) {
  if (r->plain_graph) return RVEA_OK;
  if (!r->cap_stream) RV_TRY(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
  RV_TRY(cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int t_save = r->t;
  rvea_status s = RVEA_OK;
  r->t = 1;   // p_adapt > 1: generation 1 does not adapt
  for (int q = 0; q < kPlainGens && s == RVEA_OK; ++q) s = enqueue_one(r, r->cap_stream);
  r->t = t_save;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(r->cap_stream, &g);
  if (s != RVEA_OK) { if (g) cudaGraphDestroy(g); return s; }
  if (e != cudaSuccess) return RVEA_ERR_CUDA;
  const cudaError_t e2 = cudaGraphInstantiate(&r->plain_graph, g, 0);
  cudaGraphDestroy(g);
  return cuerr(e2);
}

rvea_status ensure_block_graph(rvea_run *r) {
  if (r->block_graph) return RVEA_OK;
  if (!r->cap_stream) RV_TRY(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
  RV_TRY(cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int t_save = r->t;
  rvea_status s = RVEA_OK;
  // a period that starts at t = 1 (mod p): p-1 plain generations, then one
  // that adapts
  for (int q = 0; q < r->p_adapt && s == RVEA_OK; ++q) {
    r->t = (q == r->p_adapt - 1) ? r->p_adapt : 1;
    s = enqueue_one(r, r->cap_stream);
  }
  r->t = t_save;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(r->cap_stream, &g);
  if (s != RVEA_OK) { if (g) cudaGraphDestroy(g); return s; }
  if (e != cudaSuccess) return RVEA_ERR_CUDA;
  const cudaError_t e2 = cudaGraphInstantiate(&r->block_graph, g, 0);
  cudaGraphDestroy(g);
  return cuerr(e2);
}

// Device-usable address of a pointer that is device, managed or pinned host.
void *dev_addr(void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  if (a.type == cudaMemoryTypeUnregistered) return nullptr;
  return p;
}

rvea_status validate(const rvea_config *c) {
  if (!c) return RVEA_ERR_ARG;
  if (c->m < 2 || c->m > kMaxM || c->d < c->m || c->d > (1 << 22) || c->N < 2 || c->N > 32768)
    return RVEA_ERR_ARG;
  if (c->t_max < 1 || !(c->eta_c > 0) || !(c->eta_m > 0) || !(c->f_r > 0) || c->f_r > 1 ||
      !(c->alpha > 0) || !(c->p_c >= 0) || c->p_c > 1 || !(c->p_m >= 0) || !(c->upper > c->lower))
    return RVEA_ERR_ARG;
  // mutation: up to 8 expected sites per row (the count is capped at 32), or every site
  if (c->p_m > 8.0 && c->p_m < (double)c->d) return RVEA_ERR_ARG;
  // the DTLZ problems are defined on the unit box
  if (c->problem != PROB_NEURO && (c->lower != 0.0 || c->upper != 1.0)) return RVEA_ERR_ARG;
  if (c->problem < 0 || c->problem >= kProblems) return RVEA_ERR_ARG;
  // the other reproduction operators (DTLZ problems)
  if (c->reproduction < 0 || c->reproduction > 4) return RVEA_ERR_ARG;
  // the rollout problem: SBX with mutation or CSO (the swarm the paper's
  // neuroevolution experiment picks), whose children the rollout evaluates
  if (c->reproduction != 0 && c->reproduction != 3 && c->problem == PROB_NEURO) return RVEA_ERR_ARG;
  if (c->reproduction == 1 &&
      (!(c->de_F > 0) || c->de_F > 2 || !(c->de_CR >= 0) || c->de_CR > 1))
    return RVEA_ERR_ARG;
  if (c->reproduction == 3 && (!(c->cso_phi >= 0) || c->cso_phi > 1)) return RVEA_ERR_ARG;
  if (c->reproduction == 4 && (!(c->pso_w >= 0) || c->pso_w > 1 || !(c->pso_c1 >= 0) ||
                               c->pso_c1 > 4 || !(c->pso_c2 >= 0) || c->pso_c2 > 4))
    return RVEA_ERR_ARG;
  if (c->problem == RVEA_NEURO_LINEAR) {
    // the rollout's shape: h1 = h2 = 64 (the tensor-core tiling), ns <= 32
    // (one lane per state component), na <= 16 (one 16-row tile), and d the
    // size of the policy vector
    const rvea_neuro_dynamics *nd = c->neuro;
    if (!nd || !nd->A || !nd->B || nd->h1 != 64 || nd->h2 != 64 || nd->ns < 1 || nd->ns > 32 ||
        nd->na < 1 || nd->na > 16 || nd->steps < 1 || !(nd->sigma >= 0) || c->m != 2)
      return RVEA_ERR_ARG;
    // the FP32 form keeps eight policies' weights in shared memory
    if (nd->gemv < 0 || nd->gemv > 1 || (nd->gemv == 1 && (nd->ns > 24 || nd->na > 8)))
      return RVEA_ERR_ARG;
    if (c->d != nd->h1 * nd->ns + nd->h1 + nd->h2 * nd->h1 + nd->h2 + nd->na * nd->h2 + nd->na)
      return RVEA_ERR_ARG;
  }
  if (c->H < 0 || lattice_size(c->m, c->H) != (int64_t)c->N) return RVEA_ERR_LATTICE;
  return RVEA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

size_t rvea_workspace_bytes_ex(const rvea_config *cfg) {
  if (!cfg || validate(cfg) != RVEA_OK) return 0;
  const Shape s = make_shape(cfg->m, cfg->d, cfg->N);
  const rvea_neuro_dynamics *nd = cfg->problem == RVEA_NEURO_LINEAR ? cfg->neuro : nullptr;
  return make_layout(s, nd ? nd->steps : 0, nd ? nd->ns : 0, nd ? nd->na : 0,
                     cfg->reproduction).total;
}

int rvea_lattice_for(int m, int n) {
  if (m < 2 || m > kMaxM || lattice_size(m, 1) > (int64_t)n) return -1;
  int H = 1;
  while (lattice_size(m, H + 1) <= (int64_t)n) ++H;
  return H;
}

size_t rvea_workspace_bytes(int m, int d, int N) {
  if (m < 2 || m > kMaxM || d < m || d > (1 << 22) || N < 2 || N > 32768) return 0;
  const Shape s = make_shape(m, d, N);
  return make_layout(s, 0, 0, 0).total;
}

const char *rvea_last_cuda_error(void) {
  static thread_local char buf[256];
  if (g_last_err == cudaSuccess) return "";
  snprintf(buf, sizeof(buf), "%s: %s", g_last_where, cudaGetErrorString(g_last_err));
  return buf;
}

const char *rvea_status_str(rvea_status s) {
  switch (s) {
    case RVEA_OK: return "ok";
    case RVEA_ERR_ARG: return "invalid argument";
    case RVEA_ERR_LATTICE: return "N does not match the lattice size C(H+m-1, m-1)";
    case RVEA_ERR_NOMEM: return "workspace or scratch too small";
    case RVEA_ERR_CUDA: return "CUDA runtime error";
    case RVEA_ERR_TIMEOUT: return "a bounded device wait timed out";
    case RVEA_ERR_STATE: return "invalid in the run's current state";
    case RVEA_ERR_DEVICE: return "device-side index check failed";
  }
  return "unknown status";
}

rvea_status rvea_init_ex(const rvea_config *cfg, void *dev_workspace, size_t bytes,
                         void *cuda_stream, rvea_run **out) {
  if (!out) return RVEA_ERR_ARG;
  const rvea_status v = validate(cfg);
  if (v != RVEA_OK) return v;
  if (!dev_workspace || (reinterpret_cast<uintptr_t>(dev_workspace) & 255)) return RVEA_ERR_ARG;
  const Shape sh = make_shape(cfg->m, cfg->d, cfg->N);
  const rvea_neuro_dynamics *nd = cfg->problem == RVEA_NEURO_LINEAR ? cfg->neuro : nullptr;
  const Layout lay = make_layout(sh, nd ? nd->steps : 0, nd ? nd->ns : 0, nd ? nd->na : 0,
                                 cfg->reproduction);
  if (bytes < lay.total) return RVEA_ERR_NOMEM;
  std::call_once(g_attr_once, set_kernel_attrs);
  if (g_attr_err != cudaSuccess) return RVEA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  rvea_run *r = new (std::nothrow) rvea_run();
  if (!r) return RVEA_ERR_NOMEM;
  r->cfg = *cfg;
  r->cfg.neuro = nullptr;
  r->sh = sh;
  r->lay = lay;
  r->ws = static_cast<uint8_t *>(dev_workspace);
  r->p_adapt = std::max(1, (int)std::floor(cfg->f_r * (double)cfg->t_max + 0.5));
  r->t = 1;
  cudaGetDevice(&r->device);
  r->num_sms = current_sm_count();
  const char *ng = std::getenv("RVEA_NO_GRAPH");
  r->use_graph = !(ng && ng[0] == '1');

  RunDesc &D = r->hd;
  std::memset(&D, 0, sizeof(D));
  D.m = sh.m; D.m4 = sh.m4; D.d = sh.d; D.d_pad = sh.d_pad; D.G = sh.G;
  D.N = sh.N; D.P = sh.P; D.n_comb = sh.n_comb; D.problem = cfg->problem;
  D.t_max = cfg->t_max; D.p_adapt = r->p_adapt; D.team = sh.team; D.nseg = sh.nseg; D.sg = sh.sg;
  D.op_mode = 0;
  D.L = (float)cfg->lower; D.U = (float)cfg->upper; D.alpha = (float)cfg->alpha;
  D.inv_eta_c1 = (float)(1.0 / (cfg->eta_c + 1.0));
  D.eta_m = (float)cfg->eta_m;
  D.T_c = event_threshold24(cfg->p_c);
  D.T_m = event_threshold24(cfg->p_m / (double)cfg->d);
  D.op = cfg->reproduction;
  D.de_F = (float)cfg->de_F;
  D.T_cr = event_threshold24(cfg->de_CR);
  D.cso_phi = (float)cfg->cso_phi;
  D.pso_w = (float)cfg->pso_w;
  D.pso_c1 = (float)cfg->pso_c1;
  D.pso_c2 = (float)cfg->pso_c2;
  if (D.T_m > 0u && D.T_m < (1u << 24))
    D.n_mthr = site_count_thresholds((double)D.T_m / 16777216.0, sh.d, D.mthr);
  D.key0 = (uint32_t)cfg->seed;
  D.key1 = (uint32_t)(cfg->seed >> 32);
  D.X = wsp<float>(r, lay.X);
  D.F = wsp<float>(r, lay.F);
  std::vector<float> dynA, dynB;
  if (nd) {
    D.ns = nd->ns; D.na = nd->na; D.h1 = nd->h1; D.h2 = nd->h2; D.steps = nd->steps;
    D.sigma = (float)nd->sigma;
    D.roll_f32 = nd->gemv;
    D.noise = wsp<float>(r, lay.noise);
    D.dynA = wsp<float>(r, lay.dynA);
    D.dynB = wsp<float>(r, lay.dynB);
    dynA.assign(nd->A, nd->A + (size_t)nd->ns * nd->ns);
    dynB.assign(nd->B, nd->B + (size_t)nd->ns * nd->na);
  }
  D.slotmap = wsp<int>(r, lay.slotmap);
  D.vbits = wsp<uint32_t>(r, lay.vbits);
  D.obits = wsp<uint32_t>(r, lay.obits);
  D.zpart = wsp<uint32_t>(r, lay.zpart);
  D.vlist = wsp<int>(r, lay.vlist);
  D.child_slot = wsp<int>(r, lay.child);
  D.best = wsp<unsigned long long>(r, lay.best);
  D.amax = wsp<unsigned long long>(r, lay.amax);
  D.assoc = wsp<int>(r, lay.assoc);
  D.surv = wsp<int>(r, lay.surv);
  D.blk_cnt = wsp<int>(r, lay.blk);
  D.V32 = wsp<float>(r, lay.V32);
  D.V32lo = wsp<float>(r, lay.V32lo);
  D.V64 = wsp<double>(r, lay.V64);
  D.V0 = wsp<double>(r, lay.V0);
  D.gamma64 = wsp<double>(r, lay.g64);
  D.gamma32 = wsp<float>(r, lay.g32);
  D.ctl = wsp<Ctl>(r, lay.ctl);
  D.psum = wsp<float>(r, lay.psum);
  D.otag = wsp<int>(r, lay.otag);
  D.occ_cnt = wsp<unsigned>(r, lay.occ_cnt);
  D.vcnt = wsp<int>(r, lay.vcnt);
  D.zacc = wsp<unsigned>(r, lay.zacc);
  D.gG = sh.gG;
  D.gcells = sh.gcells;
  D.gcap = sh.gcap;
  D.gfast_off = sh.gG > 0 ? grid_build_blocks(sh.gG, sh.m) * kGridBlockCap : 0;
  D.gcell = wsp<uint16_t>(r, lay.gcell);
  D.gcnt = wsp<int>(r, lay.gcnt);
  D.gblk = wsp<int>(r, lay.gblk);
  D.gover = wsp<uint16_t>(r, lay.gover);
  D.gscale = wsp<float>(r, lay.gscale);
  D.vrange = wsp<double>(r, lay.vrange);
  D.fcomb = wsp<float>(r, lay.fcomb);
  if (cfg->reproduction == 3 || cfg->reproduction == 4) {   // the swarm state (velocities
    D.vel = wsp<float>(r, lay.vel);                             // zero from the clear below)
    D.kapd = wsp<float>(r, lay.kapd);
  }
  if (cfg->reproduction == 3) {
    D.xbar = wsp<float>(r, lay.xbar);
    D.xpart = wsp<float>(r, lay.xpart);
  }
  if (cfg->reproduction == 4) {   // personal bests: the initial positions (copied below)
    D.pb = wsp<float>(r, lay.pb);
    D.fpb = wsp<float>(r, lay.fpb);
  }
  r->d_desc = wsp<RunDesc>(r, lay.desc);

  r->repro_smem = sh.team == 32 ? kStagedSmem : 0;   // staged path (the default for 32-lane teams)
  r->init_smem = sh.ppc * std::max(1, sh.m - 1) * 4;
  r->fin_smem = 0;

  // host tables
  std::vector<ReproItem> rep(sh.n_repro), ini(sh.n_init);
  for (int q = 0; q < sh.n_repro; ++q) rep[q].pair0 = q * sh.ppc;
  for (int q = 0; q < sh.n_init; ++q) ini[q].pair0 = q * sh.ppc;
  r->sel_per_sm = 8;
  build_sel_items(r);
  std::vector<double> V0;
  build_lattice(sh.m, cfg->H, sh.N, V0);
  std::vector<int> tperm;
  std::vector<int2> trng;
  if (sh.tmax > 0) {
    build_tiles(V0, sh.N, sh.m, tperm, trng);
    if ((int)trng.size() > sh.tmax) trng.clear();   // cannot happen; keeps the bound honest
  }
  D.ntiles = (int)trng.size();
  D.tables_global = D.ntiles > 0 && sh.tglob ? 1 : 0;
  r->sel_mode = D.ntiles > 0 && !D.tables_global ? 1 : 0;
  D.repro_staged = sh.team == 32 ? 1 : 0;
  if (D.ntiles > 0) {
    D.Vt = wsp<float4>(r, lay.Vt);
    D.tperm = wsp<int>(r, lay.tperm);
    D.trng = wsp<int2>(r, lay.trng);
    D.tcen = wsp<float4>(r, lay.tcen);
    D.tcs = wsp<float2>(r, lay.tcs);
    r->prune_smem_bytes = (int)prune_smem(sh.N, D.ntiles);
  }
  if (tail_ok(r)) r->sel_mode = 3;
  std::vector<float> V32((size_t)sh.N * sh.m4 * 4, 0.0f), V32lo((size_t)sh.N * sh.m);
  for (int j = 0; j < sh.N; ++j)
    for (int k = 0; k < sh.m; ++k) {
      const double v = V0[(size_t)j * sh.m + k];
      V32[(size_t)j * sh.m4 * 4 + k] = (float)v;
      V32lo[(size_t)j * sh.m + k] = (float)(v - (double)(float)v);
    }
  Ctl c0;
  std::memset(&c0, 0, sizeof(c0));
  c0.t = 1;
  c0.K = sh.N;
  c0.grid_ver = -1;
  c0.tiles_ver = -1;
  for (int k = 0; k < kMaxM; ++k) c0.zkey[k] = 0xFFFFFFFFu;

  rvea_status s = RVEA_OK;
  auto up = [&](size_t off, const void *src, size_t n) {
    if (s == RVEA_OK) s = cuerr(cudaMemcpyAsync(r->ws + off, src, n, cudaMemcpyHostToDevice, st));
  };
  s = cuerr(cudaMemsetAsync(r->ws, 0, lay.total, st));
  up(lay.desc, &D, sizeof(D));
  up(lay.repro, rep.data(), rep.size() * sizeof(ReproItem));
  up(lay.init, ini.data(), ini.size() * sizeof(ReproItem));
  up(lay.sel, r->sel_host.data(), r->sel_host.size() * sizeof(SelItem));
  std::vector<SelItem> selb;
  {
    const SelPlan sp = sel_plan(sh.n_comb, sh.N, sh.m4, r->num_sms, 8, false);
    for (int b = 0; b < sp.nblk; ++b)
      for (int c = 0; c < sp.nch; ++c)
        selb.push_back(SelItem{b, std::min(sh.N, c * sp.chunk), std::min(sh.N, (c + 1) * sp.chunk), sp.nch});
    r->n_selb = (int)selb.size();
    r->selb_smem = std::min(sh.N, sp.chunk) * sh.m4 * 16;
  }
  up(lay.selb, selb.data(), selb.size() * sizeof(SelItem));
  up(lay.V0, V0.data(), V0.size() * 8);
  up(lay.V64, V0.data(), V0.size() * 8);
  up(lay.V32, V32.data(), V32.size() * 4);
  up(lay.V32lo, V32lo.data(), V32lo.size() * 4);
  up(lay.ctl, &c0, sizeof(c0));
  const std::vector<double> ones(kMaxM, 1.0);
  up(lay.vrange, ones.data(), kMaxM * 8);
  std::vector<float> kinf;
  if (cfg->reproduction == 3 || cfg->reproduction == 4) {   // no selection has kept a member yet
    kinf.assign(sh.N, std::numeric_limits<float>::infinity());
    up(lay.kapd, kinf.data(), kinf.size() * 4);
  }
  if (nd) {
    up(lay.dynA, dynA.data(), dynA.size() * 4);
    up(lay.dynB, dynB.data(), dynB.size() * 4);
  }
  if (D.ntiles > 0) {
    up(lay.tperm, tperm.data(), tperm.size() * 4);
    up(lay.trng, trng.data(), trng.size() * sizeof(int2));
  }
  if (s == RVEA_OK) {
    static thread_local BatchDir d;
    dir_single(d, r, wsp<ReproItem>(r, lay.init), sh.n_init);
    k_init<<<sh.n_init, kReproThreads, r->init_smem, st>>>(d);
    if (nd) {   // the initial population's rollouts (noise of t = 0)
      dir_single(d, r, nullptr, (nd->steps * nd->ns + 255) / 256);
      k_noise<<<(nd->steps * nd->ns + 255) / 256, 256, 0, st>>>(d, 1);
      rvea_run *one[1] = {r};
      launch_rollouts(one, 1, st, 1, false);
    }
    dir_single(d, r, nullptr, 1);
    k_init_lists<<<dim3((sh.N + 255) / 256, 1), 256, 0, st>>>(d);
    s = cuerr(cudaGetLastError());
    if (s == RVEA_OK && D.pb) {   // PSO: each member's personal best is where it starts
      s = cuerr(cudaMemcpyAsync(D.pb, D.X, (size_t)sh.N * sh.d_pad * 4, cudaMemcpyDeviceToDevice, st));
      if (s == RVEA_OK)
        s = cuerr(cudaMemcpyAsync(D.fpb, D.F, (size_t)sh.m * sh.n_comb * 4, cudaMemcpyDeviceToDevice, st));
    }
    if (s == RVEA_OK) s = launch_tiles(r, st);
    if (s == RVEA_OK) s = launch_gamma_force(r, st);
  }
  // pageable host sources above must stay valid until their copies are done
  if (s == RVEA_OK) s = cuerr(cudaStreamSynchronize(st));
  if (s != RVEA_OK) {
    delete r;
    return s;
  }
  r->last_stream = st;
  *out = r;
  return RVEA_OK;
}

rvea_status rvea_init(int m, int d, int N, int H, double alpha, double f_r, double eta_c,
                      double eta_m, uint64_t seed, int problem, int t_max, void *dev_workspace,
                      size_t bytes, void *cuda_stream, rvea_run **out) {
  rvea_config c;
  std::memset(&c, 0, sizeof(c));
  c.m = m; c.d = d; c.N = N; c.H = H; c.problem = problem; c.t_max = t_max;
  c.alpha = alpha; c.f_r = f_r; c.eta_c = eta_c; c.eta_m = eta_m;
  c.p_c = 1.0; c.p_m = 1.0; c.lower = 0.0; c.upper = 1.0; c.seed = seed;
  c.neuro = nullptr;
  if (problem == RVEA_NEURO_LINEAR) return RVEA_ERR_ARG;   // needs rvea_init_ex
  return rvea_init_ex(&c, dev_workspace, bytes, cuda_stream, out);
}

rvea_status rvea_step(rvea_run *r, int G, void *cuda_stream) {
  if (!r || G < 0) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  r->last_stream = st;
  if (G > 0 && r->use_graph && r->p_adapt > 1) {
    // the graphs are captured at the first step, not in the middle of a run
    // of generations that might be timed
    if (r->p_adapt > kPlainGens) {
      const rvea_status s = ensure_plain_graph(r);
      if (s != RVEA_OK) return s;
    }
    const rvea_status s = ensure_block_graph(r);
    if (s != RVEA_OK) return s;
  }
  while (G > 0) {
    const int p = r->p_adapt;
    if (r->use_graph && p > 1 && G >= p && (r->t % p) == 1) {
      const NvtxRange nr("rvea generations (one adaptation period, graph)", r->t);
      rvea_status s = ensure_block_graph(r);
      if (s != RVEA_OK) return s;
      RV_TRY(cudaGraphLaunch(r->block_graph, st));
      r->t += p;
      G -= p;
      r->has_last_gen = true;
      r->last_gen_recorded = r->recording;
      continue;
    }
    // a stretch of kPlainGens generations before the next adaptation (the
    // next multiple of p at or after t)
    if (r->use_graph && p > 1 && G >= kPlainGens && (r->t + p - 1) / p * p >= r->t + kPlainGens) {
      const NvtxRange nr("rvea generations (no adaptation, graph)", r->t);
      rvea_status s = ensure_plain_graph(r);
      if (s != RVEA_OK) return s;
      RV_TRY(cudaGraphLaunch(r->plain_graph, st));
      r->t += kPlainGens;
      G -= kPlainGens;
      r->has_last_gen = true;
      r->last_gen_recorded = r->recording;
      continue;
    }
    rvea_status s;
    {
      const NvtxRange nr("rvea generation", r->t);
      s = enqueue_one(r, st);
    }
    if (s != RVEA_OK) return s;
    r->t += 1;
    G -= 1;
    r->has_last_gen = true;
    r->last_gen_recorded = r->recording;
  }
  return RVEA_OK;
}

rvea_status rvea_step_batch(rvea_run *const *runs, int n_runs, void *cuda_stream) {
  if (!runs || n_runs < 1 || n_runs > kMaxBatch) return RVEA_ERR_ARG;
  for (int q = 0; q < n_runs; ++q) {
    if (!runs[q]) return RVEA_ERR_ARG;
    for (int u = 0; u < q; ++u)
      if (runs[u] == runs[q]) return RVEA_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const rvea_status s = launch_generation(runs, n_runs, st, true);
  if (s != RVEA_OK) return s;
  for (int q = 0; q < n_runs; ++q) {
    runs[q]->t += 1;
    runs[q]->last_stream = st;
    runs[q]->has_last_gen = true;
    runs[q]->last_gen_recorded = runs[q]->recording;
  }
  return RVEA_OK;
}

}  // extern "C"

// ---- kernel variants and the autotuner ------------------------------------

namespace {

rvea_status apply_plan(rvea_run *r, const rvea_plan &pl, cudaStream_t st) {
  if (pl.sel_mode < 0 || pl.sel_mode > 3 || (pl.sel_mode > 0 && r->hd.ntiles == 0) ||
      ((pl.sel_mode == 1 || pl.sel_mode == 2) && r->hd.tables_global) ||
      (pl.sel_mode == 3 && !tail_ok(r)))
    return RVEA_ERR_ARG;
  if (pl.sel_per_sm < 1 || pl.sel_per_sm > kSelPerSmMax) return RVEA_ERR_ARG;
  if (pl.repro_staged && r->sh.team != 32) return RVEA_ERR_ARG;
  const bool was_pruned = r->sel_mode > 0;
  r->sel_mode = pl.sel_mode;
  if (pl.sel_per_sm != r->sel_per_sm) {   // the full-scan table, kept valid in every mode
    r->sel_per_sm = pl.sel_per_sm;
    build_sel_items(r);
    RV_TRY(cudaMemcpyAsync(r->ws + r->lay.sel, r->sel_host.data(),
                           r->sel_host.size() * sizeof(SelItem), cudaMemcpyHostToDevice, st));
  }
  const int staged = pl.repro_staged ? 1 : 0;
  if (staged != r->hd.repro_staged) {
    r->hd.repro_staged = staged;
    RV_TRY(cudaMemcpyAsync(&r->d_desc->repro_staged, &r->hd.repro_staged, sizeof(int),
                           cudaMemcpyHostToDevice, st));
  }
  r->repro_smem = staged ? kStagedSmem : 0;
  // a run that was not kept up to date by the pruned path rebuilds its tiles
  if (pl.sel_mode > 0 && !was_pruned) {
    const rvea_status s = launch_tiles(r, st);
    if (s != RVEA_OK) return s;
  }
  if (r->block_graph) {   // captured with the old variants
    cudaGraphExecDestroy(r->block_graph);
    r->block_graph = nullptr;
  }
  if (r->plain_graph) {
    cudaGraphExecDestroy(r->plain_graph);
    r->plain_graph = nullptr;
  }
  // host sources of the copies above live in the run; finish them here
  RV_TRY(cudaStreamSynchronize(st));
  return RVEA_OK;
}

rvea_plan current_plan(const rvea_run *r) {
  rvea_plan pl;
  std::memset(&pl, 0, sizeof(pl));
  pl.sel_mode = r->sel_mode;
  pl.sel_per_sm = r->sel_per_sm;
  pl.repro_staged = r->hd.repro_staged;
  pl.repro_us = r->tune_repro_us;
  pl.sel_us = r->tune_sel_us;
  return pl;
}

struct TuneKey {
  int m, d, N, problem;
  bool operator<(const TuneKey &o) const {
    return std::tie(m, d, N, problem) < std::tie(o.m, o.d, o.N, o.problem);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, rvea_plan> g_tune_cache;

}  // namespace

extern "C" {

rvea_status rvea_get_plan(const rvea_run *r, rvea_plan *out) {
  if (!r || !out) return RVEA_ERR_ARG;
  *out = current_plan(r);
  return RVEA_OK;
}

rvea_status rvea_set_plan(rvea_run *r, const rvea_plan *pl, void *cuda_stream) {
  if (!r || !pl) return RVEA_ERR_ARG;
  return apply_plan(r, *pl, static_cast<cudaStream_t>(cuda_stream));
}

// Times every variant on the run's current generation without advancing it:
// the reproduction and association launches of one generation are
// idempotent (the same children, F and votes are written again; the pruned
// kernels' work counter is reset around each launch), and finalize, which
// does advance the run, is not timed.
rvea_status rvea_autotune(rvea_run *r, void *cuda_stream, int use_cache, rvea_plan *out) {
  if (!r) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const TuneKey key{r->sh.m, r->sh.d, r->sh.N, r->cfg.problem};
  if (use_cache) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      rvea_status s = apply_plan(r, it->second, st);
      if (s != RVEA_OK) return s;
      r->tune_repro_us = it->second.repro_us;
      r->tune_sel_us = it->second.sel_us;
      r->tuned = true;
      if (out) *out = current_plan(r);
      return RVEA_OK;
    }
  }
  RV_TRY(cudaStreamSynchronize(st));
  cudaEvent_t e0, e1;
  RV_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RVEA_ERR_CUDA;
  }
  rvea_status s = RVEA_OK;
  int *sel_cnt = &reinterpret_cast<Ctl *>(r->ws + r->lay.ctl)->sel_cnt;
  constexpr int kReps = 3;
  // median of kReps timed launches after one untimed one
  auto timed = [&](auto &&launch, bool reset_cnt) -> double {
    double ms[kReps];
    for (int q = -1; q < kReps && s == RVEA_OK; ++q) {
      if (reset_cnt && cudaMemsetAsync(sel_cnt, 0, sizeof(int), st) != cudaSuccess) s = RVEA_ERR_CUDA;
      cudaEventRecord(e0, st);
      launch();
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        s = RVEA_ERR_CUDA;
        break;
      }
      float f = 0.f;
      cudaEventElapsedTime(&f, e0, e1);
      if (q >= 0) ms[q] = f;
    }
    std::sort(ms, ms + kReps);
    return ms[kReps / 2] * 1e3;
  };
  static thread_local BatchDir dr, ds, dp;
  dir_single(dr, r, wsp<ReproItem>(r, r->lay.repro), r->sh.n_repro);
  dir_single(dp, r, nullptr, (r->sh.n_comb + kPruneChunkHost - 1) / kPruneChunkHost);
  const rvea_plan before = current_plan(r);
  rvea_plan best = before;
  // reproduction: direct loads, and TMA staging for 32-lane teams
  double best_rep = 1e30;
  if (r->hd.op != 0) {
    best_rep = timed([&] { launch_repro_op1(r, st); }, false);
  } else for (int staged = 0; staged <= (r->sh.team == 32 ? 1 : 0) && s == RVEA_OK; ++staged) {
    r->repro_smem = staged ? kStagedSmem : 0;
    const double us = timed([&] { launch_repro1(r, dr, r->sh.n_repro, st); }, false);
    if (us < best_rep) { best_rep = us; best.repro_staged = staged; }
  }
  // the children complete (mutated, evaluated) before the association is
  // timed on them, as the real generation will see them
  if (s == RVEA_OK) {
    launch_mutate1(r, st);
    if (cudaGetLastError() != cudaSuccess) s = RVEA_ERR_CUDA;
  }
  // association: the full scan at 4, 8 and 16 work items per SM, and the
  // pruned search with its tables in shared memory or read through L1
  double best_sel = 1e30;
  if (r->hd.ntiles > 0 && s == RVEA_OK) s = launch_tiles(r, st);
  const int per_sm[3] = {4, 8, 16};
  for (int q = 0; q < 3 && s == RVEA_OK; ++q) {
    r->sel_per_sm = per_sm[q];
    build_sel_items(r);
    if (cudaMemcpyAsync(r->ws + r->lay.sel, r->sel_host.data(), r->sel_host.size() * sizeof(SelItem),
                        cudaMemcpyHostToDevice, st) != cudaSuccess) { s = RVEA_ERR_CUDA; break; }
    dir_single(ds, r, wsp<SelItem>(r, r->lay.sel), r->n_sel);
    const double us = timed([&] { k_select<<<r->n_sel, kSelThreads, r->sel_smem, st>>>(ds); }, false);
    if (us < best_sel) { best_sel = us; best.sel_mode = 0; best.sel_per_sm = per_sm[q]; }
  }
  if (r->hd.ntiles > 0 && !r->hd.tables_global && s == RVEA_OK) {
    double us = timed([&] {
      k_select_pruned<<<r->num_sms, 1024, r->prune_smem_bytes, st>>>(r->d_desc);
    }, true);
    if (us < best_sel) { best_sel = us; best.sel_mode = 1; best.sel_per_sm = 8; }
    us = timed([&] {
      k_select_pruned_batch<<<r->num_sms, 1024, r->prune_smem_bytes, st>>>(dp);
    }, true);
    if (us < best_sel) { best_sel = us; best.sel_mode = 2; best.sel_per_sm = 8; }
    // the next real generation starts its pruned search from zero
    if (cudaMemsetAsync(sel_cnt, 0, sizeof(int), st) != cudaSuccess) s = RVEA_ERR_CUDA;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the pruned search in shared memory runs inside the fused tail where the
  // run has one (the same search, without the launch boundaries around it)
  if (best.sel_mode == 1 && tail_ok(r)) best.sel_mode = 3;
  // tables past shared memory: the fused tail's grid search (O(N) work
  // against the full scan's O(N^2)) is taken without a timing, which it
  // cannot have without advancing the run
  if (r->hd.tables_global && tail_ok(r)) best.sel_mode = 3;
  // the tables above were rebuilt for the candidates: force the chosen plan
  r->sel_per_sm = -1;
  r->repro_smem = before.repro_staged ? kStagedSmem : 0;
  if (s == RVEA_OK) s = apply_plan(r, best, st);
  if (s != RVEA_OK) return s;
  r->tune_repro_us = best_rep;
  r->tune_sel_us = best_sel;
  r->tuned = true;
  best = current_plan(r);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (out) *out = best;
  return RVEA_OK;
}

// ---- batches of runs as one CUDA graph -------------------------------------

struct rvea_batch {
  std::vector<rvea_run *> runs;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;   // kernel nodes of the captured generation
};

rvea_status rvea_batch_create(rvea_run *const *runs, int n_runs, rvea_batch **out) {
  if (!runs || !out || n_runs < 1 || n_runs > kMaxBatch) return RVEA_ERR_ARG;
  for (int q = 0; q < n_runs; ++q) {
    if (!runs[q]) return RVEA_ERR_ARG;
    for (int u = 0; u < q; ++u)
      if (runs[u] == runs[q]) return RVEA_ERR_ARG;
  }
  rvea_batch *b = new (std::nothrow) rvea_batch();
  if (!b) return RVEA_ERR_NOMEM;
  b->runs.assign(runs, runs + n_runs);
  // one batched generation (all phases; gamma and tile tables by the
  // adaptation flag), captured once and replayed per generation
  rvea_status s = RVEA_OK;
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) s = RVEA_ERR_CUDA;
  cudaGraph_t g = nullptr;
  if (s == RVEA_OK && cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    s = RVEA_ERR_CUDA;
  if (s == RVEA_OK) {
    const rvea_status sl = launch_generation(b->runs.data(), n_runs, b->cap, true);
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (sl != RVEA_OK) s = sl;
    else if (e != cudaSuccess) s = RVEA_ERR_CUDA;
  }
  if (s == RVEA_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) s = RVEA_ERR_CUDA;
  if (s == RVEA_OK) {
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) s = RVEA_ERR_CUDA;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (s == RVEA_OK && nn > 0 && cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess)
      s = RVEA_ERR_CUDA;
    for (size_t q = 0; q < nn && s == RVEA_OK; ++q) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nodes[q], &ty) != cudaSuccess) s = RVEA_ERR_CUDA;
      else if (ty == cudaGraphNodeTypeKernel) ++b->kernels;
    }
  }
  if (g) cudaGraphDestroy(g);
  if (s != RVEA_OK) {
    cudaGetLastError();
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return s;
  }
  *out = b;
  return RVEA_OK;
}

int rvea_batch_launches_per_step(const rvea_batch *b) { return b ? b->kernels : -1; }

rvea_status rvea_batch_step(rvea_batch *b, int G, void *cuda_stream) {
  if (!b || G < 0) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const NvtxRange nr("rvea batched generations", G);
  for (int q = 0; q < G; ++q) RV_TRY(cudaGraphLaunch(b->exec, st));
  for (rvea_run *r : b->runs) {
    r->t += G;
    r->last_stream = st;
    if (G > 0) { r->has_last_gen = true; r->last_gen_recorded = r->recording; }
  }
  return RVEA_OK;
}

rvea_status rvea_batch_step_profiled(rvea_batch *b, int G, void *cuda_stream, double *phase_ms,
                                     int n_phases) {
  if (!b || G < 0 || !phase_ms || n_phases < 5) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  for (int q = 0; q < n_phases; ++q) phase_ms[q] = 0.0;
  cudaEvent_t ev[6];
  for (int q = 0; q < 6; ++q)
    if (cudaEventCreate(&ev[q]) != cudaSuccess) {
      for (int u = 0; u < q; ++u) cudaEventDestroy(ev[u]);
      return RVEA_ERR_CUDA;
    }
  rvea_status s = RVEA_OK;
  for (int g = 0; g < G && s == RVEA_OK; ++g) {
    s = launch_generation(b->runs.data(), (int)b->runs.size(), st, true, ev);
    if (s == RVEA_OK && cudaEventSynchronize(ev[5]) != cudaSuccess) s = RVEA_ERR_CUDA;
    for (int q = 0; q < 5 && s == RVEA_OK; ++q) {
      float f = 0.f;
      cudaEventElapsedTime(&f, ev[q], ev[q + 1]);
      phase_ms[q] += f;
    }
    for (rvea_run *r : b->runs) {
      r->t += 1;
      r->last_stream = st;
      r->has_last_gen = true;
      r->last_gen_recorded = r->recording;
    }
  }
  for (int q = 0; q < 6; ++q) cudaEventDestroy(ev[q]);
  return s;
}

void rvea_batch_free(rvea_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

int rvea_generation(const rvea_run *r) { return r ? r->t : -1; }

int rvea_launches_per_generation(const rvea_run *r, int adapting) {
  if (!r) return -1;
  // gamma, then the tile table and the direction grid (4 launches)
  const int adapt_n = adapting ? 1 + (r->hd.ntiles > 0 ? 1 : 0) + (r->hd.gG > 0 ? 4 : 0) : 0;
  if (r->sel_mode == 3) return 2 + (cso_needs_mean(r) ? 2 : 0) + adapt_n;   // reproduction, fused tail
  int n = 3;                                        // reproduction, selection, finalize
  if (r->sh.team == 32 && r->hd.op == 0) n += 1;    // k_mutate
  if (cso_needs_mean(r)) n += 2;                    // the CSO swarm centre (two launches)
  if (r->hd.problem == PROB_NEURO) n += 2;          // noise, rollout
  n += adapt_n;
  return n;
}

rvea_status rvea_step_profiled(rvea_run *r, int G, void *cuda_stream, double *phase_ms,
                               int n_phases) {
  if (!r || G < 0 || !phase_ms || n_phases < 4) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  r->last_stream = st;
  for (int q = 0; q < n_phases; ++q) phase_ms[q] = 0.0;
  if (G == 0) return RVEA_OK;
  // events around every launch of every generation, on the launching stream
  std::vector<cudaEvent_t> ev((size_t)G * 6);
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto &x : ev) if (x) cudaEventDestroy(x);
      return RVEA_ERR_CUDA;
    }
  rvea_status s = RVEA_OK;
  static thread_local BatchDir dr, ds, df, dg, dd;
  const rvea_run *one = r;
  dir_single(dr, one, wsp<ReproItem>(r, r->lay.repro), r->sh.n_repro);
  dir_single(ds, one, wsp<SelItem>(r, r->lay.sel), r->n_sel);
  dir_single(df, one, nullptr, 1);
  dir_single(dg, one, nullptr, 1);
  static thread_local BatchDir dpb, dn1, dro1;
  dir_single(dpb, one, nullptr, (r->sh.n_comb + kPruneChunkHost - 1) / kPruneChunkHost);
  const int nbd = (r->sh.N + 1023) / 1024;
  dir_single(dd, one, nullptr, nbd);
  const int nbg = std::min((r->sh.N + 31) / 32, 4 * r->num_sms);
  for (int g = 0; g < G && s == RVEA_OK; ++g) {
    cudaEvent_t *e = &ev[(size_t)g * 6];
    cudaEventRecord(e[0], st);
    if (r->hd.op != 0) launch_repro_op1(r, st);
    else launch_repro1(r, dr, r->sh.n_repro, st);
    cudaEventRecord(e[5], st);
    if (r->sel_mode != 3) launch_mutate1(r, st);
    if (r->hd.problem == PROB_NEURO) {
      const int nb_noise = (r->hd.steps * r->hd.ns + 255) / 256;
      dir_single(dn1, one, nullptr, nb_noise);
      k_noise<<<nb_noise, 256, 0, st>>>(dn1, 0);
      launch_rollouts(&r, 1, st, 0, false);
    }
    cudaEventRecord(e[1], st);
    if (r->sel_mode == 3)   // the fused tail: mutation, association and finalize
      launch_tail(r, st, false);
    else if (r->sel_mode == 1)
      k_select_pruned<<<r->num_sms, 1024, r->prune_smem_bytes, st>>>(r->d_desc);
    else if (r->sel_mode == 2)
      k_select_pruned_batch<<<r->num_sms, 1024, r->prune_smem_bytes, st>>>(dpb);
    else
      k_select<<<r->n_sel, kSelThreads, r->sel_smem, st>>>(ds);
    cudaEventRecord(e[2], st);
    if (r->sel_mode != 3) k_finalize<<<nbd, 1024, 0, st>>>(dd);
    cudaEventRecord(e[3], st);
    if (r->t % r->p_adapt == 0) {
      launch_tiles(r, st);
      k_gamma<<<nbg, 256, 0, st>>>(dg, 1);
    }
    cudaEventRecord(e[4], st);
    s = cuerr(cudaGetLastError());
    r->t += 1;
    r->has_last_gen = true;
    r->last_gen_recorded = r->recording;
  }
  if (s == RVEA_OK) s = cuerr(cudaStreamSynchronize(st));
  // e[0] reproduction e[5] children e[1] selection e[2] finalize e[3] gamma e[4]
  const int from[5] = {0, 1, 2, 3, 5}, to[5] = {5, 2, 3, 4, 1};
  for (int g = 0; g < G && s == RVEA_OK; ++g) {
    const cudaEvent_t *e = &ev[(size_t)g * 6];
    for (int q = 0; q < 5; ++q) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e[from[q]], e[to[q]]) != cudaSuccess) { s = RVEA_ERR_CUDA; break; }
      phase_ms[(q == 4 && n_phases < 5) ? 0 : q] += ms;
    }
  }
  for (auto &x : ev) cudaEventDestroy(x);
  return s;
}

rvea_status rvea_population(const rvea_run *r, float *dst, uint8_t *valid, void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const Shape &sh = r->sh;
  float *dx = dev_addr(dst) ? static_cast<float *>(dev_addr(dst)) : nullptr;
  uint8_t *dv = dev_addr(valid) ? static_cast<uint8_t *>(dev_addr(valid)) : nullptr;
  if ((dst && !dx) || (valid && !dv)) {
    // pageable destination: flags and slot map through the staging area,
    // rows one copy each
    uint8_t *sv = wsp<uint8_t>(r, r->lay.stage);
    k_gather_pop<<<sh.N, 256, 0, st>>>(r->d_desc, nullptr, sv);
    RV_TRY(cudaGetLastError());
    std::vector<int> map(sh.N);
    RV_TRY(cudaMemcpyAsync(map.data(), r->hd.slotmap + (size_t)(r->t & 1) * sh.N, sh.N * 4,
                           cudaMemcpyDeviceToHost, st));
    RV_TRY(cudaStreamSynchronize(st));
    if (valid) {
      for (int j = 0; j < sh.N; ++j) valid[j] = map[j] >= 0 ? 1 : 0;
    }
    if (dst) {
      for (int j = 0; j < sh.N; ++j) {
        float *o = dst + (size_t)j * sh.d;
        if (map[j] < 0) {
          for (int k = 0; k < sh.d; ++k) o[k] = std::nanf("");
        } else {
          RV_TRY(cudaMemcpy(o, r->hd.X + (size_t)map[j] * sh.d_pad, sh.d * 4, cudaMemcpyDeviceToHost));
        }
      }
    }
    return RVEA_OK;
  }
  k_gather_pop<<<sh.N, 256, 0, st>>>(r->d_desc, dx, dv);
  return cuerr(cudaGetLastError());
}

rvea_status rvea_objectives(const rvea_run *r, float *dst, uint8_t *valid, void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const Shape &sh = r->sh;
  float *dx = static_cast<float *>(dev_addr(dst));
  uint8_t *dv = static_cast<uint8_t *>(dev_addr(valid));
  if ((dst && !dx) || (valid && !dv)) {
    float *sf = wsp<float>(r, r->lay.stage);
    uint8_t *sv = reinterpret_cast<uint8_t *>(sf + (size_t)sh.N * sh.m);
    k_gather_obj<<<(sh.N + 255) / 256, 256, 0, st>>>(r->d_desc, sf, sv);
    RV_TRY(cudaGetLastError());
    if (dst) RV_TRY(cudaMemcpyAsync(dst, sf, (size_t)sh.N * sh.m * 4, cudaMemcpyDeviceToHost, st));
    if (valid) RV_TRY(cudaMemcpyAsync(valid, sv, sh.N, cudaMemcpyDeviceToHost, st));
    return RVEA_OK;
  }
  k_gather_obj<<<(sh.N + 255) / 256, 256, 0, st>>>(r->d_desc, dx, dv);
  return cuerr(cudaGetLastError());
}

rvea_status rvea_igd(const rvea_run *r, const float *ref, int n_ref, double *out,
                     void *cuda_stream) {
  if (!r || !ref || !out || n_ref < 1) return RVEA_ERR_ARG;
  const float *rd = static_cast<const float *>(dev_addr(const_cast<float *>(ref)));
  if (!rd) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nb = (n_ref + 255) / 256;
  // block partials and the result in the run's staging area
  const size_t stage_bytes = (size_t)r->sh.N * (kMaxM + 1) * 4;
  if ((size_t)(nb + 1) * 8 > stage_bytes) return RVEA_ERR_ARG;
  double *part = wsp<double>(r, r->lay.stage);
  k_igd_partial<<<nb, 256, 0, st>>>(r->d_desc, rd, n_ref, part);
  RV_TRY(cudaGetLastError());
  k_igd_final<<<1, 32, 0, st>>>(part, nb, n_ref, part + nb);
  RV_TRY(cudaGetLastError());
  double v = 0.0;
  RV_TRY(cudaMemcpyAsync(&v, part + nb, sizeof(double), cudaMemcpyDeviceToHost, st));
  RV_TRY(cudaStreamSynchronize(st));
  if (!std::isfinite(v)) return RVEA_ERR_STATE;   // no valid member
  *out = v;
  return RVEA_OK;
}

rvea_status rvea_hypervolume(const rvea_run *r, const double *ref, double *out, void *cuda_stream) {
  if (!r || !ref || !out) return RVEA_ERR_ARG;
  const int m = r->sh.m, N = r->sh.N;
  if (m != 2 && m != 3) return RVEA_ERR_ARG;
  for (int k = 0; k < m; ++k)
    if (!std::isfinite(ref[k])) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // scratch in the run's staging area (N (kMaxM + 1) 4 bytes >= 44 N + 16)
  uint8_t *base = wsp<uint8_t>(r, r->lay.stage);
  double *dd = reinterpret_cast<double *>(base);
  int *ii = reinterpret_cast<int *>(base + (size_t)32 * N);
  HvScratch S{dd, dd + N, dd + 2 * (size_t)N, dd + 3 * (size_t)N,
              ii, ii + N, ii + 2 * (size_t)N, ii + 3 * (size_t)N};
  double *dout = reinterpret_cast<double *>(base + (((size_t)44 * N + 4 + 7) & ~(size_t)7));
  const HvRef hr{ref[0], ref[1], m == 3 ? ref[2] : 1.0};
  k_hv_compact<<<1, 1024, 0, st>>>(r->d_desc, hr, S);
  RV_TRY(cudaGetLastError());
  k_hv_rank<<<(N + 255) / 256, 256, 0, st>>>(S);
  RV_TRY(cudaGetLastError());
  k_hv_slices<<<(N + 7) / 8, 256, 0, st>>>(S, hr);
  RV_TRY(cudaGetLastError());
  k_hv_final<<<1, 32, 0, st>>>(S, dout);
  RV_TRY(cudaGetLastError());
  double v = 0.0;
  RV_TRY(cudaMemcpyAsync(&v, dout, sizeof(double), cudaMemcpyDeviceToHost, st));
  RV_TRY(cudaStreamSynchronize(st));
  *out = v;
  return RVEA_OK;
}

rvea_status rvea_export_state(const rvea_run *r, float *X, float *F, uint8_t *valid, double *V,
                              double *gamma, void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rvea_status s = RVEA_OK;
  if (X || valid) s = rvea_population(r, X, valid, cuda_stream);
  if (s == RVEA_OK && F) s = rvea_objectives(r, F, nullptr, cuda_stream);
  if (s != RVEA_OK) return s;
  const size_t nv = (size_t)r->sh.N * r->sh.m * 8;
  if (V) RV_TRY(cudaMemcpyAsync(V, r->hd.V64, nv, cudaMemcpyDefault, st));
  if (gamma) RV_TRY(cudaMemcpyAsync(gamma, r->hd.gamma64, (size_t)r->sh.N * 8, cudaMemcpyDefault, st));
  return RVEA_OK;
}

rvea_status rvea_import_state(rvea_run *r, const float *X, const float *F, const uint8_t *valid,
                              const double *V, const double *gamma, int t, void *cuda_stream) {
  if (!r || !X || !F || !valid || !V || !gamma || t < 1) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const Shape &sh = r->sh;
  {
    // a population without a valid member leaves mating nothing to draw
    // from: refused here, before any device state changes
    std::vector<uint8_t> hv(sh.N);
    RV_TRY(cudaStreamSynchronize(st));
    RV_TRY(cudaMemcpy(hv.data(), valid, sh.N, cudaMemcpyDefault));
    if (std::none_of(hv.begin(), hv.end(), [](uint8_t v) { return v != 0; })) return RVEA_ERR_ARG;
  }
  float *sf = wsp<float>(r, r->lay.stage);
  uint8_t *sv = reinterpret_cast<uint8_t *>(sf + (size_t)sh.N * sh.m);
  RV_TRY(cudaMemcpy2DAsync(r->hd.X, (size_t)sh.d_pad * 4, X, (size_t)sh.d * 4, (size_t)sh.d * 4,
                           sh.N, cudaMemcpyDefault, st));
  RV_TRY(cudaMemcpyAsync(sf, F, (size_t)sh.N * sh.m * 4, cudaMemcpyDefault, st));
  RV_TRY(cudaMemcpyAsync(sv, valid, sh.N, cudaMemcpyDefault, st));
  RV_TRY(cudaMemcpyAsync(r->hd.V64, V, (size_t)sh.N * sh.m * 8, cudaMemcpyDefault, st));
  RV_TRY(cudaMemcpyAsync(r->hd.gamma64, gamma, (size_t)sh.N * 8, cudaMemcpyDefault, st));
  // CSO, PSO: a new swarm (velocities zero; k_import sets the kept APDs to
  // +inf; personal bests where the members are)
  if (r->hd.vel) RV_TRY(cudaMemsetAsync(r->hd.vel, 0, (size_t)sh.N * sh.d_pad * 4, st));
  k_import<<<1, kFinThreads, 0, st>>>(r->d_desc, sf, sv, t);
  RV_TRY(cudaGetLastError());
  if (r->hd.pb) {
    RV_TRY(cudaMemcpyAsync(r->hd.pb, r->hd.X, (size_t)sh.N * sh.d_pad * 4, cudaMemcpyDeviceToDevice, st));
    RV_TRY(cudaMemcpyAsync(r->hd.fpb, r->hd.F, (size_t)sh.m * sh.n_comb * 4, cudaMemcpyDeviceToDevice, st));
  }
  if (launch_tiles(r, st) != RVEA_OK) return RVEA_ERR_CUDA;
  RV_TRY(cudaStreamSynchronize(st));
  r->t = t;
  r->last_stream = st;
  r->has_last_gen = false;
  return RVEA_OK;
}

rvea_status rvea_export_swarm(const rvea_run *r, float *vel, float *apd, float *pbest,
                              float *fpbest, void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  if (!r->hd.vel) return RVEA_ERR_STATE;
  if ((pbest || fpbest) && !r->hd.pb) return RVEA_ERR_STATE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  float *dv = static_cast<float *>(dev_addr(vel));
  float *da = static_cast<float *>(dev_addr(apd));
  float *dp = static_cast<float *>(dev_addr(pbest));
  float *df = static_cast<float *>(dev_addr(fpbest));
  if ((vel && !dv) || (apd && !da) || (pbest && !dp) || (fpbest && !df))
    return RVEA_ERR_ARG;   // device or pinned memory only
  if (!vel && !apd && !pbest && !fpbest) return RVEA_OK;
  k_gather_swarm<<<r->sh.N, 256, 0, st>>>(r->d_desc, dv, da, dp, df);
  return cuerr(cudaGetLastError());
}

rvea_status rvea_import_swarm(rvea_run *r, const float *vel, const float *apd, const float *pbest,
                              const float *fpbest, void *cuda_stream) {
  if (!r || !vel || !apd) return RVEA_ERR_ARG;
  if (!r->hd.vel) return RVEA_ERR_STATE;
  if (r->hd.pb && (!pbest || !fpbest)) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const Shape &sh = r->sh;
  // slot j's member sits in pool row j after rvea_import_state
  RV_TRY(cudaMemcpy2DAsync(r->hd.vel, (size_t)sh.d_pad * 4, vel, (size_t)sh.d * 4, (size_t)sh.d * 4,
                           sh.N, cudaMemcpyDefault, st));
  RV_TRY(cudaMemcpyAsync(r->hd.kapd, apd, (size_t)sh.N * 4, cudaMemcpyDefault, st));
  if (r->hd.pb) {
    RV_TRY(cudaMemcpy2DAsync(r->hd.pb, (size_t)sh.d_pad * 4, pbest, (size_t)sh.d * 4,
                             (size_t)sh.d * 4, sh.N, cudaMemcpyDefault, st));
    // objectives N x m (by slot) into the m x 2N table: objective k of slot j
    // (pool row j) at k 2N + j, one strided copy per objective
    for (int k = 0; k < sh.m; ++k)
      RV_TRY(cudaMemcpy2DAsync(r->hd.fpb + (size_t)k * sh.n_comb, 4, fpbest + k, (size_t)sh.m * 4, 4,
                               sh.N, cudaMemcpyDefault, st));
  }
  RV_TRY(cudaStreamSynchronize(st));
  r->last_stream = st;
  return RVEA_OK;
}

rvea_status rvea_offspring(const rvea_run *r, float *X, float *F, void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  if (!r->has_last_gen) return RVEA_ERR_STATE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  float *dx = static_cast<float *>(dev_addr(X));
  float *df = static_cast<float *>(dev_addr(F));
  if ((X && !dx) || (F && !df)) return RVEA_ERR_ARG;   // device or pinned memory only
  k_gather_children<<<r->sh.N, 256, 0, st>>>(r->d_desc, dx, df);
  return cuerr(cudaGetLastError());
}

rvea_status rvea_last_selection(const rvea_run *r, int32_t *assoc, int32_t *survivor,
                                void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  if (!r->has_last_gen) return RVEA_ERR_STATE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int *da = static_cast<int *>(dev_addr(assoc));
  int *ds = static_cast<int *>(dev_addr(survivor));
  if ((assoc && !da) || (survivor && !ds)) return RVEA_ERR_ARG;
  k_copy_selection<<<(r->sh.n_comb + 255) / 256, 256, 0, st>>>(r->d_desc, da, ds);
  return cuerr(cudaGetLastError());
}

rvea_status rvea_record_draws(rvea_run *r, int enable, void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  r->hd.rec_par = enable ? wsp<int>(r, r->lay.rec_par) : nullptr;
  r->hd.rec_sites = enable ? wsp<int>(r, r->lay.rec_sites) : nullptr;
  // the kernels read the descriptor from device memory, so direct launches
  // and graph replays both see the change; the sources live in the handle
  RV_TRY(cudaMemcpyAsync(&r->d_desc->rec_par, &r->hd.rec_par, sizeof(int *),
                         cudaMemcpyHostToDevice, st));
  RV_TRY(cudaMemcpyAsync(&r->d_desc->rec_sites, &r->hd.rec_sites, sizeof(int *),
                         cudaMemcpyHostToDevice, st));
  r->recording = enable != 0;
  return RVEA_OK;
}

rvea_status rvea_last_draws(const rvea_run *r, int32_t *parents, int32_t *sites,
                            void *cuda_stream) {
  if (!r) return RVEA_ERR_ARG;
  if (!r->has_last_gen || !r->last_gen_recorded || r->hd.op != 0) return RVEA_ERR_STATE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (parents)
    RV_TRY(cudaMemcpyAsync(parents, r->ws + r->lay.rec_par, (size_t)2 * r->sh.P * 4,
                           cudaMemcpyDefault, st));
  if (sites)
    RV_TRY(cudaMemcpyAsync(sites, r->ws + r->lay.rec_sites,
                           (size_t)r->sh.N * (1 + kMaxSites) * 4, cudaMemcpyDefault, st));
  return RVEA_OK;
}

rvea_status rvea_sync_status(rvea_run *r) {
  if (!r) return RVEA_ERR_ARG;
  if (cudaStreamSynchronize(r->last_stream) != cudaSuccess) return RVEA_ERR_CUDA;
  int status = 0;
  if (cudaMemcpy(&status, &r->hd.ctl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RVEA_ERR_CUDA;
  if (status & ST_TIMEOUT) return RVEA_ERR_TIMEOUT;
  if (status & ST_BADINDEX) return RVEA_ERR_DEVICE;
  return RVEA_OK;
}

void rvea_free(rvea_run *r) {
  if (!r) return;
  if (r->block_graph) cudaGraphExecDestroy(r->block_graph);
  if (r->plain_graph) cudaGraphExecDestroy(r->plain_graph);
  if (r->cap_stream) cudaStreamDestroy(r->cap_stream);
  delete r;
}

// ---- stateless operators --------------------------------------------------

namespace {
struct OpLayout {
  size_t ctl, desc, best, amax, blk, items, total;
};
OpLayout op_layout(int n, int r) {
  OpLayout L;
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = align256(o + b);
    return at;
  };
  const int nblk = (n + kSelBlock - 1) / kSelBlock;
  const int tiles = (r + kVTileMin - 1) / kVTileMin;   // the finest plan's chunks
  L.ctl = take(sizeof(Ctl));
  L.desc = take(sizeof(RunDesc));
  L.best = take((size_t)r * 8);
  L.amax = take((size_t)n * 8);
  L.blk = take((size_t)nblk * 4);
  L.items = take((size_t)nblk * tiles * sizeof(SelItem));
  L.total = o;
  return L;
}
}  // namespace

size_t rvea_select_scratch_bytes(int n, int r, int m) {
  if (n < 1 || r < 1 || m < 2 || m > kMaxM) return 0;
  return op_layout(n, r).total + (size_t)r * kMaxM * 16;   // + padded V copy
}

rvea_status rvea_select(int m, int n, const float *F, const uint8_t *valid, int r,
                        const float *V, const float *gamma, int t, int t_max, float alpha,
                        int32_t *assoc, int32_t *survivor, void *scratch, size_t scratch_bytes,
                        void *cuda_stream) {
  if (m < 2 || m > kMaxM || n < 1 || r < 1 || !F || !V || !gamma || !assoc || !survivor ||
      !scratch || t_max < 1 || !(alpha > 0.0f))
    return RVEA_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) & 255) return RVEA_ERR_ARG;
  if (scratch_bytes < rvea_select_scratch_bytes(n, r, m)) return RVEA_ERR_NOMEM;
  std::call_once(g_attr_once, set_kernel_attrs);
  if (g_attr_err != cudaSuccess) return RVEA_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const OpLayout L = op_layout(n, r);
  uint8_t *ws = static_cast<uint8_t *>(scratch);
  const int m4 = (m + 3) / 4;
  float *V32 = reinterpret_cast<float *>(ws + L.total);
  // zero-padded float4 rows of V
  RV_TRY(cudaMemsetAsync(V32, 0, (size_t)r * m4 * 16, st));
  RV_TRY(cudaMemcpy2DAsync(V32, (size_t)m4 * 16, V, (size_t)m * 4, (size_t)m * 4, r,
                           cudaMemcpyDeviceToDevice, st));
  RunDesc D;
  std::memset(&D, 0, sizeof(D));
  D.m = m; D.m4 = m4; D.N = r; D.n_comb = n; D.t_max = t_max; D.alpha = alpha;
  D.op_mode = 1; D.t_op = t;
  D.best = reinterpret_cast<unsigned long long *>(ws + L.best);
  D.amax = reinterpret_cast<unsigned long long *>(ws + L.amax);
  D.blk_cnt = reinterpret_cast<int *>(ws + L.blk);
  D.assoc = assoc;
  D.V32 = V32;
  D.gamma32 = const_cast<float *>(gamma);
  D.ctl = reinterpret_cast<Ctl *>(ws + L.ctl);
  D.F_aos = F;
  D.valid_in = valid;
  D.survivor_out = survivor;
  // items: every solution block x every vector chunk
  const SelPlan sp = sel_plan(n, r, m4, current_sm_count());
  std::vector<SelItem> items;
  items.reserve((size_t)sp.nblk * sp.nch);
  for (int b = 0; b < sp.nblk; ++b)
    for (int c = 0; c < sp.nch; ++c)
      items.push_back(SelItem{b, std::min(r, c * sp.chunk), std::min(r, (c + 1) * sp.chunk), sp.nch});
  RunDesc *dD = reinterpret_cast<RunDesc *>(ws + L.desc);
  RV_TRY(cudaMemcpyAsync(dD, &D, sizeof(D), cudaMemcpyHostToDevice, st));
  RV_TRY(cudaMemcpyAsync(ws + L.items, items.data(), items.size() * sizeof(SelItem),
                         cudaMemcpyHostToDevice, st));
  k_op_prep<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, st>>>(dD);
  k_op_zstar<<<(n + 255) / 256, 256, 0, st>>>(dD);
  static thread_local BatchDir d;
  d.n = 1;
  d.prefix[0] = 0;
  d.prefix[1] = (int)items.size();
  d.desc[0] = dD;
  d.items[0] = ws + L.items;
  k_select<<<(unsigned)items.size(), kSelThreads, std::min(r, sp.chunk) * m4 * 16, st>>>(d);
  k_op_finish<<<(r + 255) / 256, 256, 0, st>>>(dD);
  // the pageable host sources of the two copies above were staged before
  // cudaMemcpyAsync returned, so nothing here waits for the stream
  return cuerr(cudaGetLastError());
}

rvea_status rvea_gamma(int m, int r, const double *V, double *gamma, void *cuda_stream) {
  if (m < 2 || m > kMaxM || r < 2 || !V || !gamma) return RVEA_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the descriptor travels in the kernel parameter block: no scratch needed
  RunDesc D;
  std::memset(&D, 0, sizeof(D));
  D.m = m;
  D.N = r;
  D.V64 = const_cast<double *>(V);
  D.gamma64 = gamma;
  D.gamma32 = nullptr;
  const int nb = (r + 31) / 32;
  k_gamma_op<<<nb, 256, 0, st>>>(D);
  return cuerr(cudaGetLastError());
}

}  // extern "C"
