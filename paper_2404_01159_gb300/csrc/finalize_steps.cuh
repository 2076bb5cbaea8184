// Steps of the end of a generation (Algorithm 1 line 16; Algorithm 2,
// "update reference vectors"), run by k_finalize with CTAs of kFinDecode
// threads: every CTA decodes one block of reference vectors, the last CTA
// to arrive builds the lists.
#pragma once
#include "rvea_device.cuh"

namespace rvea {

constexpr int kFinDecode = 1024;   // threads (vectors) per finalize CTA

// Shared memory of the finalize step (one CTA of 1024 threads).
struct FinShared {
  unsigned lo[32][kMaxM], hi[32][kMaxM];   // per-warp survivor extrema
  unsigned z[2 * kMaxM];                    // next z* (min) and maximum
  int cnt[2][32];                           // per-warp valid / free counts
  double rng[kMaxM];                        // adaptation range
  uint32_t free_[2048];                     // complement of the occupied-row bitmap
};


// Writes, in ascending order, the positions of the set bits of words
// [w0, w1) of `bits` (bit b of word w is element 32 w + b) starting at
// out[base]; at most `limit` elements in total.  One warp: lane l loads word
// w0 + 32 i + l, so the loads of a round are independent (one round for up to
// 32 words); a warp scan of the popcounts gives each word its offset.
__device__ __forceinline__ int warp_compact(const uint32_t *bits, int w0, int w1, int *out,
                                           int base, int limit) {
  const int lane = threadIdx.x & 31;
  for (int r = w0; r < w1; r += 32) {
    const int w = r + lane;
    const uint32_t word = w < w1 ? bits[w] : 0u;
    const int c = __popc(word);
    int incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const int at = base + incl - c;
    // then word by word from registers: lane = bit, coalesced stores
    const uint32_t lt = (1u << lane) - 1u;
    const int nw = min(32, w1 - r);
    for (int i = 0; i < nw; ++i) {
      const uint32_t wi = __shfl_sync(0xffffffffu, word, i);
      const int pos = __shfl_sync(0xffffffffu, at, i) + __popc(wi & lt);
      if (((wi >> lane) & 1u) && pos < limit) out[pos] = 32 * (r + i) + lane;
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  return base;
}

// Decode of vectors [blk * kFinDecode, (blk + 1) * kFinDecode) by a CTA of
// kFinDecode threads: slot map, survivors, occupied-row and valid bitmaps, and
// this block's minimum / maximum of the survivors' objectives in zpart[blk].
__device__ inline void fin_decode(const RunDesc &R, int blk, FinShared &sh) {
  const int j = blk * kFinDecode + threadIdx.x;
  const int N = R.N, n2 = 2 * N, m = R.m;
  const int t = R.ctl->t;
  const int *cur = R.slotmap + (t & 1) * N;
  int *nmap = R.slotmap + ((t + 1) & 1) * N;
  const int *ccur = R.child_slot + (t & 1) * N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int s = -1;
  if (j < N) {
    const unsigned long long key = R.best[j];
    R.best[j] = ~0ull;
    int i = -1;
    if (key != ~0ull) {
      i = (int)(uint32_t)(key & 0xFFFFFFFFull);
      if (i >= 0 && i < N) s = cur[i];
      else if (i >= N && i < n2) s = ccur[i - N];
      if (s < 0 || s >= n2) { set_status(R.ctl, ST_BADINDEX); s = -1; i = -1; }
    }
    nmap[j] = s;
    R.surv[j] = i;
    if (s >= 0) atomicOr(&R.obits[s >> 5], 1u << (s & 31));
    // CSO: the APD that kept slot j's member (Eq. 4), for the next competitions
    if (R.kapd) R.kapd[j] = s >= 0 ? __uint_as_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000);
  }
  const uint32_t vmask = __ballot_sync(0xffffffffu, s >= 0);
  if (lane == 0 && j < N) R.vbits[j >> 5] = vmask;
  for (int k = 0; k < m; ++k) {
    unsigned lo = 0xFFFFFFFFu, hi = 0u;
    if (s >= 0) lo = hi = f2ord(R.F[(size_t)k * n2 + s]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) { sh.lo[warp][k] = lo; sh.hi[warp][k] = hi; }
  }
  __syncthreads();
  if (threadIdx.x < m) {
    unsigned lo = 0xFFFFFFFFu, hi = 0u;
    for (int w = 0; w < kFinDecode / 32; ++w) {
      lo = min(lo, sh.lo[w][threadIdx.x]);
      hi = max(hi, sh.hi[w][threadIdx.x]);
    }
    R.zpart[(size_t)blk * 2 * kMaxM + threadIdx.x] = lo;
    R.zpart[(size_t)blk * 2 * kMaxM + kMaxM + threadIdx.x] = hi;
  }
  __syncthreads();
}

// After every block is decoded (by this CTA, or by others whose writes this
// CTA has acquired): the ascending valid and free lists, the next z*, on
// adaptation generations the FP64 rescaling of V, and the control block.
__device__ inline void fin_lists(const RunDesc &R, int nblk, FinShared &sh) {
  const int N = R.N, n2 = 2 * N, m = R.m;
  const int t = R.ctl->t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tid = threadIdx.x;
  const int nvw = (N + 31) >> 5, now = (n2 + 31) >> 5, nzb = nblk;
  for (int w = tid; w < now; w += kFinDecode) {
    uint32_t o = __ldcg(R.obits + w);
    if (w == now - 1 && (n2 & 31)) o |= ~((1u << (n2 & 31)) - 1u);   // beyond 2N
    sh.free_[w] = ~o;
    R.obits[w] = 0u;   // empty for the next generation
  }
  if (tid < 2 * kMaxM) sh.z[tid] = tid < kMaxM ? 0xFFFFFFFFu : 0u;
  __syncthreads();
  for (int q = tid; q < nzb * m; q += kFinDecode) {
    const int b = q / m, k = q - (q / m) * m;
    atomicMin(&sh.z[k], __ldcg(R.zpart + (size_t)b * 2 * kMaxM + k));
    atomicMax(&sh.z[kMaxM + k], __ldcg(R.zpart + (size_t)b * 2 * kMaxM + kMaxM + k));
  }
  // warp w owns words [w * per, (w+1) * per) of each bitmap
  const int perv = (nvw + 31) / 32, pero = (now + 31) / 32;
  const int v0 = min(nvw, warp * perv), v1 = min(nvw, v0 + perv);
  const int o0 = min(now, warp * pero), o1 = min(now, o0 + pero);
  int cv = 0, cf = 0;
  for (int w = v0 + lane; w < v1; w += 32) cv += __popc(__ldcg(R.vbits + w));
  for (int w = o0 + lane; w < o1; w += 32) cf += __popc(sh.free_[w]);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    cv += __shfl_xor_sync(0xffffffffu, cv, off);
    cf += __shfl_xor_sync(0xffffffffu, cf, off);
  }
  if (lane == 0) { sh.cnt[0][warp] = cv; sh.cnt[1][warp] = cf; }
  __syncthreads();
  int bv = 0, bf = 0, K = 0;
  for (int w = 0; w < 32; ++w) {
    if (w < warp) { bv += sh.cnt[0][w]; bf += sh.cnt[1][w]; }
    K += sh.cnt[0][w];
  }
  warp_compact(R.vbits, v0, v1, R.vlist, bv, N);
  warp_compact(sh.free_, o0, o1, R.child_slot + ((t + 1) & 1) * N, bf, N);

  if (tid < m) R.ctl->zkey[tid] = sh.z[tid];
  const bool adapt = (t % R.p_adapt) == 0;
  if (adapt && K > 0) {
    // range_k = max - min over the survivors, floored at 1e-12, in FP64
    if (tid < m) {
      const double r = (double)ord2f(sh.z[kMaxM + tid]) - (double)ord2f(sh.z[tid]);
      sh.rng[tid] = r < 1e-12 ? 1e-12 : r;
      R.vrange[tid] = sh.rng[tid];
    }
    __syncthreads();
    for (int jj = tid; jj < N; jj += kFinDecode) adapt_row(R, jj, sh.rng);
  }
  __syncthreads();   // every thread has read t and the counters
  if (tid == 0) {
    R.ctl->K = K;
    R.ctl->adapted = adapt ? 1 : 0;
    if (adapt && K > 0) R.ctl->v_ver += 1;
    R.ctl->fin_cnt = 0;
    R.ctl->sel_cnt = 0;
    R.ctl->t = t + 1;
  }
}

}  // namespace rvea
