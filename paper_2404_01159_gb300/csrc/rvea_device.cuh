// Device-side data structures and helpers of the RVEA library (sm_103a).
//
// A run's state lives in one caller-owned workspace.  Kernels never see the
// host handle: they read a RunDesc (device memory) that holds the shape,
// the parameters and pointers into the workspace.  Every kernel is written
// for a table of runs, so one launch can serve one run or a whole batch;
// each work item touches exactly one run, so a run's arithmetic is the same
// alone and in a batch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rvea {

constexpr int kMaxM = 16;          // objectives
constexpr int kReproThreads = 256; // CTA size of the reproduction kernel
constexpr int kMutThreads = 128;   // CTA size of the mutation / evaluation kernel (one child a thread)
constexpr int kLaneGroups = 8;     // 8-variable groups per lane per reproduction unit
constexpr int kSelThreads = 128;   // selection CTA size
constexpr int kSelSols = 4;        // solutions per thread (a multiple of 2: packed pairs)
constexpr int kSelBlock = kSelSols * kSelThreads;   // solutions per selection work item
constexpr int kVTile = 512;        // reference vectors per shared-memory tile
constexpr int kVTileMin = 64;      // the smallest tile sel_plan halves kVTile to
constexpr int kFinThreads = 1024;  // CTA size of the per-run finalize kernel
constexpr int kMaxSites = 32;      // cap of the mutation-site count of one row
constexpr int kStages = 2;         // staged reproduction: chunks per warp in shared memory
constexpr int kStageWarpBytes = kStages * 2 * 1024;   // per warp: kStages x 2 parents x 1 KB
constexpr int kStagedSmem = (kReproThreads / 32) * (kStageWarpBytes + kStages * 8);
constexpr int kTailThreads = 1024;  // CTA size of the fused tail kernel (one CTA per SM)
constexpr int kTailMaxCtas = 256;   // its largest grid
constexpr int kMeanRows = 64;       // CSO swarm centre: population rows per partial sum
constexpr int kMeanCols = 1024;     // CSO swarm centre: variables per column block (256 x float4)

// Philox counter tags (word 3 of the counter).
enum : uint32_t {
  TAG_INIT = 1, TAG_MATE = 2, TAG_PAIR = 3, TAG_SBX = 4,
  TAG_MUTSITE = 5, TAG_MUTMAG = 6, TAG_NOISE = 7
};

enum : int { PROB_DTLZ2 = 0, PROB_DTLZ1 = 1, PROB_NEURO = 2, PROB_DTLZ3 = 3, PROB_DTLZ4 = 4 };
constexpr int kProblems = 5;
// DTLZ1 and DTLZ3 share the multimodal g (Rastrigin-like terms)
__host__ __device__ constexpr bool multimodal_g(int problem) {
  return problem == PROB_DTLZ1 || problem == PROB_DTLZ3;
}

// Device status word bits.
enum : int { ST_TIMEOUT = 1, ST_BADINDEX = 2 };

// Per-run control block (device memory, updated by the kernels).
struct Ctl {
  int t;               // next generation index (1-based)
  int K;               // number of valid population slots
  int status;          // ST_* bits
  int adapted;         // set by finalize on adaptation generations
  int fin_cnt;         // arrival counter of the finalize CTAs
  int sel_cnt;         // work counter of the pruned selection kernel
  unsigned zkey[kMaxM];   // ideal point z*, order-preserving uint encoding
  int v_ver;           // changes of V so far (adaptation, import)
  int fcomb_t;         // generation whose combined objectives fcomb holds (0: none)
  int grid_ver;        // the v_ver the direction grid was built for (-1: none)
  int grid_skip;       // 1: the current vectors are too skewed for the grid (not built)
  int tiles_ver;       // the v_ver the tile tables were built for (-1: none)
  unsigned long long bar;   // grid barrier of the fused tail kernel: arrivals
                            // since initialisation (a multiple of its grid
                            // between launches)
};

struct RunDesc {
  // shape
  int m, m4;           // objectives, float4s per padded vector row
  int d, d_pad, G;     // variables, row pitch (multiple of 8), 8-variable groups
  int N, P;            // population / vectors, pairs = ceil(N/2)
  int n_comb;          // solutions entering selection (2N for a run)
  int problem;
  int t_max, p_adapt;
  int team;            // threads per reproduction team (power of two <= 32, function of d)
  int nseg;            // segments per pair
  int repro_staged;    // 1: parents staged in shared memory by TMA (32-lane teams)
  int sg;              // groups per segment, ceil(G / nseg) <= kLaneGroups * team
  int op_mode;         // 1: stateless selection (identity slots, AoS F)
  int op;              // reproduction: 0 SBX + polynomial mutation, 1 DE/rand/1/bin, 2 random,
                       //               3 competitive swarm (CSO), 4 particle swarm (PSO)
  float de_F;          // DE scale factor
  uint32_t T_cr;       // DE crossover coin: fires iff (w >> 8) < T_cr
  float cso_phi;       // CSO: weight of the swarm-centre term
  float pso_w, pso_c1, pso_c2;   // PSO: inertia weight, cognitive and social weights
  // parameters
  float L, U, alpha, inv_eta_c1, eta_m;
  uint32_t T_c, T_m;   // 24-bit event thresholds (fires iff k < T)
  int n_mthr;          // site-count thresholds in use (<= kMaxSites)
  uint32_t mthr[kMaxSites];   // site count of a row = #{i < n_mthr : w >= mthr[i]}
  uint32_t key0, key1; // Philox key = seed
  // state (pointers into the workspace)
  float *X;            // [2N][d_pad] population pool (physical slots)
  float *F;            // [m][2N]    objectives per physical slot (SoA)
  int *slotmap;        // [2][N]     vector slot j -> physical slot (-1 invalid), by t & 1
  uint32_t *vbits;     // [ceil(N/32)]  valid flags of P_{t+1} (bit j)
  uint32_t *obits;     // [ceil(2N/32)] occupied pool rows of P_{t+1} (bit s)
  uint32_t *zpart;     // [ceil(N/1024)][2][kMaxM] per-block survivor min / max
  int *vlist;          // [N]        ascending valid j (K entries)
  int *child_slot;     // [2][N]     physical slot of child c, by t & 1
  unsigned long long *best;   // [N]   packed (APD bits, combined index) minima
  unsigned long long *amax;   // [n_comb] packed (cosine bits, ~vector) maxima
  int *assoc;          // [n_comb]   vector of each solution, -1 if invalid
  int *surv;           // [N]        combined index kept by vector j, -1 if none
  float *psum;         // [P][2][nseg] partial g sums of the segments of each pair
  // swarm state of the CSO and PSO operators (null for the other operators)
  float *vel;          // [2N][d_pad] velocity of each pool row (moves with its row)
  float *kapd;         // [N]        APD that kept vector slot j's member (+inf: none yet)
  float *pb;           // [2N][d_pad] PSO: personal best of each pool row's member
  float *fpb;          // [m][2N]    PSO: objectives of those personal bests
  float *xbar;         // [d_pad]    mean position of the valid members (the swarm centre)
  float *xpart;        // [ceil(N/kMeanRows)][d_pad] float partial sums of the centre
  // draw recording (inspection; null when off): the vector slot of each
  // parent draw e, and each child's mutation-site count (-1: every site)
  // followed by its sites in draw order
  int *rec_par;        // [2P]
  int *rec_sites;      // [N][1 + kMaxSites]
  // fused tail kernel (one persistent launch: mutation, association, finalize)
  int *otag;           // [2N]       generation t whose survivors occupy pool row s (0: none)
  unsigned *occ_cnt;   // [kTailMaxCtas] occupied pool rows in each CTA's row range
  int *vcnt;           // [kTailMaxCtas] valid slots in each CTA's vector range
  unsigned *zacc;      // [3][kTailMaxCtas][4] per-CTA minima of the children, minima and
                       // maxima of the survivors (order-preserving)
  float *fcomb;        // [2][m][2N] objectives of the combined population by combined
                       //            index (parents i < N in slot order, NaN when
                       //            invalid; children N + c), for generation parity t & 1
  // direction grid of the association (m = 2, 3; gG = 0: none)
  int gG, gcells, gcap;   // steps per barycentric axis, cells, candidate capacity
  int gfast_off;       // start of the fill pass's area in gover (after the blocks' shares)
  uint16_t *gcell;     // [gcells][16] record: count, then up to 15 tile-order positions
                       //              (or, past 15, the offset of the list in gover)
  int *gcnt;           // [gcells]     candidates of each cell (build)
  int *gblk;           // [build blocks] overflow candidates of each block of cells, then
                       //              their offset in gover
  uint16_t *gover;     // [gfast_off + gcap] candidate lists of the cells with more than 15
  float *gscale;       // [kMaxM]      w = 1 / range of the grid's V
  double *vrange;      // [kMaxM]      objective range of the last adaptation (1: none)
  int *blk_cnt;        // [n_comb/256] arrival counters of the selection blocks
  float *V32;          // [N][m4*4]  reference vectors, zero padded
  float *V32lo;        // [N][m]     V64 - V32 rounded to float (null: zero)
  double *V64;         // [N][m]
  double *V0;          // [N][m]     initial unit lattice
  double *gamma64;     // [N]
  float *gamma32;      // [N]
  Ctl *ctl;
  // pruned selection: reference vectors grouped into spatially compact tiles
  int ntiles;          // 0: the pruned kernel is not used for this run
  int tables_global;   // 1: the tables exceed shared memory; the fused tail reads them
                       //    from global memory (L2) and the pruned kernels are not used
  float4 *Vt;          // [N]        V32 in tile order (m <= 4)
  int *tperm;          // [N]        tile-order position -> vector index j
  int2 *trng;          // [ntiles]   (first position, count <= 64) of each tile
  float4 *tcen;        // [ntiles]   unit centre of each tile (float32)
  float2 *tcs;         // [ntiles]   (cos rho, sin rho), rho >= max angle centre-member
  // stateless-selection views (op_mode)
  const float *F_aos;  // [n][m]
  const uint8_t *valid_in;  // [n] or null
  int *survivor_out;   // [N]
  int t_op;            // generation index used by the op
  // neuroevolution rollout
  float *noise;        // [steps][ns]
  const float *dynA;   // [ns][ns]
  const float *dynB;   // [ns][na]
  int ns, na, h1, h2, steps;
  float sigma;
  int roll_f32;        // 1: policy GEMVs on the CUDA cores in FP32, 0: BF16 tensor cores
};

// Work item of the reproduction kernel: one CTA, consecutive work units of one
// run (a unit is one segment of one pair; for the initialisation kernel, one
// individual).
struct ReproItem { int pair0; };
// Work item of the selection kernel: one block of 256 solutions x one chunk
// of reference vectors (the chunk fits in shared memory).
struct SelItem { int sblk; int v0; int v1; int nchunks; };

// Runs served by one launch, passed by value as a kernel parameter: CTA b
// belongs to the run r with prefix[r] <= b < prefix[r+1] and processes item
// b - prefix[r] of that run's item table (which lives in the run's own
// workspace).  One run is a directory of size 1.
constexpr int kMaxBatch = 320;
struct BatchDir {
  int n;
  int prefix[kMaxBatch + 1];
  const RunDesc *desc[kMaxBatch];
  const void *items[kMaxBatch];
  uint2 key[kMaxBatch];   // Philox key of each run (uniform operands)
};

// Selection work plan: blocks of kSelBlock solutions x chunks of whole
// kVTile-vector tiles, at least ~per_sm CTAs per SM overall (the tuning knob
// of the full scan), each chunk small enough to sit in shared memory
// (kSelChunkBytes).
constexpr int kSelChunkBytes = 96 * 1024;
struct SelPlan {
  int nblk, nch, chunk;   // solution blocks, chunks, vectors per chunk
};
inline SelPlan sel_plan(int n, int r, int m4, int sms, int per_sm = 8, bool fine = true) {
  SelPlan p;
  p.nblk = (n + kSelBlock - 1) / kSelBlock;
  // vector tiles of kVTile, halved (fine: down to kVTileMin) while the items
  // would not reach per_sm per SM: a small run alone still spreads over the
  // GPU (a batch, many runs together, takes the coarse tiles)
  int vt = kVTile;
  while (fine && vt > kVTileMin && (long long)p.nblk * ((r + vt - 1) / vt) < (long long)per_sm * sms) vt >>= 1;
  const int tiles = (r + vt - 1) / vt;
  int cap = kSelChunkBytes / (m4 * 16) / vt;
  if (cap < 1) cap = 1;
  int nch = (per_sm * sms + p.nblk - 1) / p.nblk;
  if (nch > tiles) nch = tiles;
  if (nch < 1) nch = 1;
  int tpc = (tiles + nch - 1) / nch;
  if (tpc > cap) tpc = cap;
  p.nch = (tiles + tpc - 1) / tpc;
  p.chunk = tpc * vt;
  return p;
}

// SM count of the current device, read once per device (the grid sizes and
// the selection work plans follow it); 152, a GB300's count, if it cannot be
// read.
inline int current_sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  int n = __atomic_load_n(&cache[dev], __ATOMIC_RELAXED);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 152;
  }
  __atomic_store_n(&cache[dev], n, __ATOMIC_RELAXED);
  return n;
}

__device__ __forceinline__ int dir_find(const BatchDir &dir, int b) {
  int lo = 0, hi = dir.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (dir.prefix[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Round keys of Philox4x32-10 for one key: k_r = key + r * (W0, W1).  Passed
// by value as a kernel parameter, each round's key is a constant-bank
// operand instead of a register.
struct RoundKeys {
  uint32_t k[20];
};
inline RoundKeys round_keys(uint32_t k0, uint32_t k1) {
  RoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
    rk.k[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  return rk;
}

// Key providers for philox_k: keys from a RoundKeys parameter, or computed.
struct KeyConst {
  const RoundKeys &rk;
  __device__ __forceinline__ uint32_t k(int i) const { return rk.k[i]; }
};
struct KeyRun {
  uint32_t k0, k1;
  __device__ __forceinline__ uint32_t k(int i) const {
    return (i & 1) ? k1 + (uint32_t)(i >> 1) * 0xBB67AE85u : k0 + (uint32_t)(i >> 1) * 0x9E3779B9u;
  }
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by the two Philox constants (hi/lo halves), XORs
// the high halves with words 1/3 and the round key; the key advances by the
// golden-ratio Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2,
                                        uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = 0xD2511F53u * c0, ah = __umulhi(0xD2511F53u, c0);
    const uint32_t b = 0xCD9E8D57u * c2, bh = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = bh ^ c1 ^ k0, n2 = ah ^ c3 ^ k1;
    c0 = n0; c1 = b; c2 = n2; c3 = a;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

template <class KP>
__device__ __forceinline__ uint4 philox_k(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          const KP &kp) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = 0xD2511F53u * c0, ah = __umulhi(0xD2511F53u, c0);
    const uint32_t b = 0xCD9E8D57u * c2, bh = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = bh ^ c1 ^ kp.k(2 * r), n2 = ah ^ c3 ^ kp.k(2 * r + 1);
    c0 = n0; c1 = b; c2 = n2; c3 = a;
  }
  return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint32_t word(const uint4 &w, int i) {
  return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
}

// 24-bit uniform on [0,1): exact in float.
__device__ __forceinline__ float u24f(uint32_t w) {
  return (float)(w >> 8) * 0x1p-24f;
}

// Order-preserving map float -> uint (for atomicMin/Max on floats).
__device__ __forceinline__ unsigned f2ord(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned o) {
  const unsigned u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
  return __uint_as_float(u);
}

__device__ __forceinline__ void set_status(Ctl *ctl, int bits) {
  atomicOr(&ctl->status, bits);
}

// ---------------------------------------------------------------------------
// Packed float pairs (Blackwell .f32x2 arithmetic): one instruction does the
// same IEEE operation on both halves as two scalar instructions would.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long f2u(float2 a) {
  return *reinterpret_cast<unsigned long long *>(&a);
}
__device__ __forceinline__ float2 u2f(unsigned long long a) {
  return *reinterpret_cast<float2 *>(&a);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)));
  return u2f(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
  return u2f(d);
}
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy (TMA) helpers, inline PTX.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// APD (Eq. 4) of a solution f' (float; f' >= 0) against its unit vector v,
// APD = (1 + pen theta / gamma) |f'|.  theta comes from the chord,
// |f' - |f'| v| = |f'| 2 sin(theta / 2), not from acos of the cosine: near
// theta = 0 the cosine carries no information below float resolution, and
// the penalty divides theta by gamma (about 1e-3 rad at N = 9870).  v is a
// float pair hi + lo (the FP64 vector to ~1e-15; lo may be null), each
// chord component is formed with two fmas, and the rounding of |f'| only
// moves the chord along v, a second-order change, so theta keeps a relative
// accuracy of a few float roundings on theta <= pi/2 (f', v >= 0).
__device__ __forceinline__ float apd_chord(const float *fp, int m, const float *vhi,
                                           const float *vlo, float gam, float pen) {
  float s = 0.0f;
  for (int k = 0; k < m; ++k) s = fmaf(fp[k], fp[k], s);
  const float nf = sqrtf(s);
  if (nf == 0.0f) return 0.0f;   // f' = 0: theta = pi/2 by convention, APD = 0
  float w2 = 0.0f;
  for (int k = 0; k < m; ++k) {
    float w = fmaf(-nf, vhi[k], fp[k]);
    if (vlo) w = fmaf(-nf, vlo[k], w);
    w2 = fmaf(w, w, w2);
  }
  const float th = 2.0f * asinf(fminf(1.0f, 0.5f * sqrtf(w2) / nf));
  return (1.0f + pen * th / gam) * nf;
}

// Reference-vector adaptation of vector j (Algorithm 2, "update reference
// vectors"): V_j = V0_j (.) range / |V0_j (.) range| in FP64, written as V64,
// its float32 copy and the float32 remainder.  Every kernel that adapts calls
// this one function, and its operations are spelled out (products, sums, a
// correctly rounded square root and division, no contraction), so the bits do
// not depend on which kernel adapts.
__device__ __forceinline__ void adapt_row(const RunDesc &R, int jj, const double *rng) {
  const int m = R.m;
  const double *v0p = R.V0 + (size_t)jj * m;
  double w[kMaxM];
  double s2 = 0.0;
  for (int k = 0; k < m; ++k) {
    w[k] = __dmul_rn(v0p[k], rng[k]);
    s2 = __dadd_rn(s2, __dmul_rn(w[k], w[k]));
  }
  const double nrm = __dsqrt_rn(s2);
  float *v32 = R.V32 + (size_t)jj * R.m4 * 4;
  for (int k = 0; k < m; ++k) {
    const double v = __ddiv_rn(w[k], nrm);
    R.V64[(size_t)jj * m + k] = v;
    v32[k] = (float)v;
    R.V32lo[(size_t)jj * m + k] = (float)__dsub_rn(v, (double)(float)v);
  }
}

// Programmatic dependent launch.  The kernels of a generation are launched
// with programmatic stream serialisation, so a kernel's CTAs may start while
// its predecessor's last CTAs still run: each kernel waits (griddepcontrol
// .wait: the predecessor has completed and its writes are visible) before it
// reads anything the predecessor wrote, and only then lets its own successor
// start (launch_dependents).  Waiting before triggering keeps the ordering
// transitive; a kernel that triggers first (k_mutate) reads nothing that its
// predecessor writes before its wait.  In a kernel launched without the
// attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// One 1-D bulk copy global -> shared through the TMA engine; completion is
// signalled as transaction bytes on `bar`.  dst, src 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 policy for data streamed through once (the reproduction kernel's parent
// rows and child rows): evicted first, so that the 0.4 GB a generation
// moves does not push the selection's tables, partial sums and code out of
// L2 between the kernels.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// tma_load_1d with an L2 cache policy.
__device__ __forceinline__ void tma_load_1d_hint(void *dst, const void *src, uint32_t bytes,
                                                 uint64_t *bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// Bounded wait on phase `parity` of `bar`: returns false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

constexpr uint32_t kWaitLimit = 1u << 22;   // polls before a wait gives up

}  // namespace rvea
