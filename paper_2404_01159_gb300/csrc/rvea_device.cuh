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
constexpr int kSelThreads = 256;   // solutions per selection CTA
constexpr int kVTile = 512;        // reference vectors per shared-memory tile
constexpr int kFinThreads = 1024;  // CTA size of the per-run finalize kernel

// Philox counter tags (word 3 of the counter).
enum : uint32_t {
  TAG_INIT = 1, TAG_MATE = 2, TAG_PAIR = 3, TAG_SBX = 4,
  TAG_MUTHI = 5, TAG_MUTLO = 6, TAG_NOISE = 7
};

enum : int { PROB_DTLZ2 = 0, PROB_DTLZ1 = 1, PROB_NEURO = 2 };

// Device status word bits.
enum : int { ST_TIMEOUT = 1, ST_BADINDEX = 2 };

// Per-run control block (device memory, updated by the kernels).
struct Ctl {
  int t;               // next generation index (1-based)
  int K;               // number of valid population slots
  int status;          // ST_* bits
  int adapted;         // set by finalize on adaptation generations
  unsigned zkey[kMaxM];  // ideal point z*, order-preserving uint encoding
};

struct RunDesc {
  // shape
  int m, m4;           // objectives, float4s per padded vector row
  int d, d_pad, G;     // variables, row pitch (multiple of 8), 8-variable groups
  int N, P;            // population / vectors, pairs = ceil(N/2)
  int n_comb;          // solutions entering selection (2N for a run)
  int problem;
  int t_max, p_adapt;
  int team;            // threads per pair in reproduction (function of d)
  int op_mode;         // 1: stateless selection (identity slots, AoS F)
  // parameters
  float L, U, alpha, inv_eta_c1, eta_m;
  uint32_t T_c, T_m;   // 24-bit event thresholds (fires iff k < T)
  uint32_t key0, key1; // Philox key = seed
  // state (pointers into the workspace)
  float *X;            // [2N][d_pad] population pool (physical slots)
  float *F;            // [m][2N]    objectives per physical slot (SoA)
  int *slotmap;        // [N]        vector slot j -> physical slot, -1 invalid
  int *vlist;          // [N]        ascending valid j (K entries)
  int *child_slot;     // [2][N]     physical slot of child c, by t & 1
  unsigned long long *best;   // [N]   packed (APD bits, combined index) minima
  unsigned long long *amax;   // [n_comb] packed (cosine bits, ~vector) maxima
  int *assoc;          // [n_comb]   vector of each solution, -1 if invalid
  int *surv;           // [N]        combined index kept by vector j, -1 if none
  int *blk_cnt;        // [n_comb/256] arrival counters of selection blocks
  float *V32;          // [N][m4*4]  reference vectors, zero padded
  double *V64;         // [N][m]
  double *V0;          // [N][m]     initial unit lattice
  double *gamma64;     // [N]
  float *gamma32;      // [N]
  Ctl *ctl;
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
};

// Work item of the reproduction kernel: one CTA, consecutive pairs of one run
// (or consecutive individuals for the initialisation kernel).
struct ReproItem { int pair0; };
// Work item of the selection kernel: one block of 256 solutions x one chunk
// of reference vectors.
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
};

__device__ __forceinline__ int dir_find(const BatchDir &dir, int b) {
  int lo = 0, hi = dir.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (dir.prefix[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

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
