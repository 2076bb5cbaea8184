// Direction grid of the exact association (Algorithm 1 lines 5-6, Eq. 2)
// for m = 2, 3.
//
// The association of a solution depends only on the direction of f' = F - z*
// (f' >= 0).  A direction is the point a of the simplex (a_k = u_k / sum u,
// u = f' (.) w, w > 0 a per-run scale: 1 at first, 1 / range after each
// adaptation, so that the grid follows the rescaled reference vectors), and
// the grid cuts the first m - 1 barycentric coordinates into G equal steps.
// For each cell the build (k_grid_count / k_grid_fill) lists every reference
// vector that can be the float32 argmax of f'.v for some direction in the
// cell: with c the cell's centre direction and rho the largest angle from c
// to the cell (its corners, widened by more than the rounding of a in
// float32), a vector b found near c gives every direction d in the cell a
// best cosine of at least L = cos(angle(c, v_b) + rho); a vector j can reach
// the argmax at d only if cos(d, v_j) >= L - 2 eps (eps bounds the float32
// dot error relative to |f'|, below 1e-6), which needs
//   angle(c, v_j) <= R = rho + acos(L - 2 eps).
// Every such j is listed (the test runs in float32 with margins that only
// ever admit more vectors).  The lookup then scans the cell's list with the
// full scan's arithmetic (same products, larger dot, on equal dots the
// smaller index), so the result is the full scan's, bit for bit, after about
// half a dozen dot products instead of the tile search.
//
// The grid is valid for one set of reference vectors: the control block's
// v_ver counts changes of V (adaptation, import) and grid_ver records the V
// the grid was built for; a kernel uses the grid only when they agree (and
// the build fitted its buffer), and otherwise the tile search.
#pragma once
#include "prune_steps.cuh"

namespace rvea {

constexpr int kGridRec = 16;      // uint16 per cell record (32 bytes)
constexpr int kGridInline = 15;   // candidates held in the record itself
// Longer lists: the count pass writes a cell's list (up to kGridWarpBuf
// candidates) into its block's share of the overflow area, kGridBlockCap
// entries per block at the start of gover; a list that does not fit is left
// to the fill pass, which writes it after the shares (from gfast_off on).
constexpr int kGridBlockCap = 2048;
constexpr int kGridWarpBuf = 128;
constexpr int kGridFastBit = 1 << 30;   // gcnt flag: list written by the count pass
// cells per block of the build: one CTA lists the candidate tiles of a
// block once for all its cells (64 consecutive cells for m = 2, 8 x 8 for
// m = 3); grid_build_blocks gives the launch's CTA count
constexpr int kGridSpan2 = 64;
constexpr int kGridSpan3 = 8;
__host__ __device__ inline int grid_build_blocks(int G, int m) {
  const int span = m == 2 ? kGridSpan2 : kGridSpan3, nbx = (G + span - 1) / span;
  return m == 2 ? nbx : nbx * nbx;
}

// Cell of the direction of f' (>= 0, not 0): the first M - 1 scaled
// barycentric coordinates, each cut into G steps.
template <int M>
__device__ __forceinline__ int grid_cell(const float *f, const float *w, int G) {
  float u[M], s = 0.0f;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    u[k] = f[k] * w[k];
    s += u[k];
  }
  const float inv = (float)G / s;
  int cell = 0, mul = 1;
#pragma unroll
  for (int k = 0; k < M - 1; ++k) {
    const int c = min(G - 1, max(0, (int)(u[k] * inv)));
    cell += c * mul;
    mul *= G;
  }
  return cell;
}

// Association of solution i through the grid, then its APD vote (Eq. 4), as
// prune_group does.  One thread per solution; sV: the tile-order vectors
// (vector index in the fourth lane).
// fc: the combined objectives of this generation by combined index (NaN for
// an invalid parent), or null to read them through the slot maps.
template <int M>
__device__ __forceinline__ void grid_assoc(const RunDesc &R, int i, const float4 *sV,
                                           const float *z, const float *w, float pen,
                                           const float *fc) {
  const int N = R.N, n = R.n_comb;
  if (i >= n) return;
  float f[4] = {0.f, 0.f, 0.f, 0.f};
  if (fc) {
    float F0[M];
#pragma unroll
    for (int k = 0; k < M; ++k) F0[k] = __ldcg(fc + (size_t)k * n + i);
    if (F0[0] != F0[0]) {   // an invalid parent
      R.assoc[i] = -1;
      return;
    }
#pragma unroll
    for (int k = 0; k < M; ++k) f[k] = F0[k] - z[k];
  } else {
    const int par = R.ctl->t & 1;
    const int slot = i < N ? R.slotmap[par * N + i] : R.child_slot[par * N + (i - N)];
    if (slot < 0) {
      R.assoc[i] = -1;
      return;
    }
#pragma unroll
    for (int k = 0; k < M; ++k) f[k] = __ldcg(R.F + (size_t)k * n + slot) - z[k];
  }
  float s2 = f[0] * f[0];
#pragma unroll
  for (int k = 1; k < M; ++k) s2 = fmaf(f[k], f[k], s2);
  int bj = 0;   // f' = 0: every dot is +0, the full scan keeps vector 0
  if (sqrtf(s2) > 0.0f) {
    const int cell = grid_cell<M>(f, w, R.gG);
    // the cell's 32-byte record: count, then up to kGridInline candidates
    const uint4 *rp = reinterpret_cast<const uint4 *>(R.gcell + (size_t)cell * kGridRec);
    const uint4 r0 = __ldg(rp), r1 = __ldg(rp + 1);
    const uint32_t wd[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    const int n = (int)(wd[0] & 0xFFFFu);
    float best = -INFINITY;
    bj = 0x7FFFFFFF;
    if (n <= kGridInline) {
#pragma unroll
      for (int e = 0; e < kGridInline; ++e) {
        if (e < n) {
          const uint32_t q = (wd[(e + 1) >> 1] >> (16 * ((e + 1) & 1))) & 0xFFFFu;
          const float4 v = sV[q];
          keep(pdot<M>(f, v), __float_as_int(v.w), best, bj);
        }
      }
    } else {
      const int at = (int)((wd[0] >> 16) | ((wd[1] & 0xFFFFu) << 16));
      for (int e = 0; e < n; ++e) {
        const float4 v = sV[R.gover[at + e]];
        keep(pdot<M>(f, v), __float_as_int(v.w), best, bj);
      }
    }
  }
  if (bj < 0 || bj >= N) {
    set_status(R.ctl, ST_BADINDEX);
    return;
  }
  const float apd = apd_chord(f, M, R.V32 + (size_t)bj * R.m4 * 4, R.V32lo + (size_t)bj * M,
                              R.gamma32[bj], pen);
  R.assoc[i] = bj;
  atomicMin(&R.best[bj], ((unsigned long long)__float_as_uint(apd) << 32) | (uint32_t)i);
}

// The same association with L = 8 or 4 lanes per solution (lanes L g ..
// L g + L - 1 of a warp take solution i of group g; every lane of the warp
// must call it): each lane scans the candidates e = sub, sub + L, ... of the
// cell and fetches, for its best one, the float remainder of the vector and
// gamma, so that after the group reduces (larger dot, then smaller index)
// the lane holding the winner computes the APD and votes without another
// round trip.  Four lanes serve twice as many solutions a warp, for when
// eight would leave warps with a second round.  `pre` (or null): solution
// i's objectives from fc, loaded by the caller ahead of z*.
template <int M, int L = 8>
__device__ __forceinline__ void grid_assocL(const RunDesc &R, int i, const float4 *sV,
                                            const float *z, const float *w, float pen,
                                            const float *fc, const float *pre = nullptr) {
  static_assert(L == 8 || L == 4, "8 or 4 lanes per solution");
  constexpr int NW = 8 / L;                  // record words a lane holds
  constexpr int NE = (kGridInline + L - 1) / L;   // inline candidates a lane scans
  const int N = R.N, n = R.n_comb, lane = threadIdx.x & 31, sub = lane & (L - 1),
            gb = lane & ~(L - 1);
  const bool act = i < n;
  float f[4] = {0.f, 0.f, 0.f, 0.f};
  bool valid = false;
  if (act) {
    if (fc) {
      float F0[M];
#pragma unroll
      for (int k = 0; k < M; ++k) F0[k] = pre ? pre[k] : __ldcg(fc + (size_t)k * n + i);
      valid = F0[0] == F0[0];   // NaN: an invalid parent
#pragma unroll
      for (int k = 0; k < M; ++k) f[k] = F0[k] - z[k];
    } else {
      const int par = R.ctl->t & 1;
      const int slot = i < N ? R.slotmap[par * N + i] : R.child_slot[par * N + (i - N)];
      valid = slot >= 0;
      if (valid) {
#pragma unroll
        for (int k = 0; k < M; ++k) f[k] = __ldcg(R.F + (size_t)k * n + slot) - z[k];
      }
    }
  }
  float s2 = f[0] * f[0];
#pragma unroll
  for (int k = 1; k < M; ++k) s2 = fmaf(f[k], f[k], s2);
  const bool live = act && valid && sqrtf(s2) > 0.0f;
  // the cell record, words sub, sub + L of it on this lane
  uint32_t wd[NW];
#pragma unroll
  for (int u = 0; u < NW; ++u) wd[u] = 0u;
  if (live) {
    const int cell = grid_cell<M>(f, w, R.gG);
    const uint32_t *rw = reinterpret_cast<const uint32_t *>(R.gcell + (size_t)cell * kGridRec);
#pragma unroll
    for (int u = 0; u < NW; ++u) wd[u] = __ldg(rw + sub + L * u);
  }
  // every lane takes part in every shuffle (groups of one warp may take
  // different branches below, which hold no warp-wide operation)
  const uint32_t w0 = __shfl_sync(0xffffffffu, wd[0], gb);
  const uint32_t w1 = __shfl_sync(0xffffffffu, wd[0], gb | 1);
  uint32_t we[NE];
#pragma unroll
  for (int h = 0; h < NE; ++h) {   // the word of element e + 1, e = sub + L h (e <= 14 used)
    const int wi = min(7, (sub + L * h + 1) >> 1);
    uint32_t got = 0u;
#pragma unroll
    for (int u = 0; u < NW; ++u) {
      const uint32_t x = __shfl_sync(0xffffffffu, wd[u], gb | (wi & (L - 1)));
      if (wi / L == u) got = x;
    }
    we[h] = got;
  }
  const int cnt = live ? (int)(w0 & 0xFFFFu) : 0;
  float best = -INFINITY;
  int bj = 0x7FFFFFFF, bq = -1;
  if (cnt <= kGridInline) {
#pragma unroll
    for (int h = 0; h < NE; ++h) {
      const int e = sub + L * h;   // element e + 1 of the record
      if (e < cnt) {
        const int q = (int)((we[h] >> (16 * ((e + 1) & 1))) & 0xFFFFu);
        const float4 v = sV[q];
        const int j = __float_as_int(v.w);
        const float dt = pdot<M>(f, v);
        if (dt > best || (dt == best && j < bj)) { best = dt; bj = j; bq = q; }
      }
    }
  } else {
    const int at = (int)((w0 >> 16) | ((w1 & 0xFFFFu) << 16));
    for (int e = sub; e < cnt; e += L) {
      const int q = R.gover[at + e];
      const float4 v = sV[q];
      const int j = __float_as_int(v.w);
      const float dt = pdot<M>(f, v);
      if (dt > best || (dt == best && j < bj)) { best = dt; bj = j; bq = q; }
    }
  }
  // the remainder and gamma of this lane's best, fetched before the reduction
  float lo[4] = {0.f, 0.f, 0.f, 0.f}, gam = 1.0f;
  if (bq >= 0 && bj < N) {
#pragma unroll
    for (int k = 0; k < M; ++k) lo[k] = __ldg(R.V32lo + (size_t)bj * M + k);
    gam = __ldg(R.gamma32 + bj);
  }
  float gbest = best;
  int gbj = bj;
#pragma unroll
  for (int off = 1; off < L; off <<= 1) {
    const float od = __shfl_xor_sync(0xffffffffu, gbest, off);
    const int oj = __shfl_xor_sync(0xffffffffu, gbj, off);
    if (od > gbest || (od == gbest && oj < gbj)) { gbest = od; gbj = oj; }
  }
  if (!act) return;
  if (!valid) {
    if (sub == 0) R.assoc[i] = -1;
    return;
  }
  if (!live) {   // f' = 0: every dot is +0, the full scan keeps vector 0; APD = 0
    if (sub == 0) {
      R.assoc[i] = 0;
      atomicMin(&R.best[0], (unsigned long long)(uint32_t)i);
    }
    return;
  }
  if (gbj < 0 || gbj >= N) {
    if (sub == 0) set_status(R.ctl, ST_BADINDEX);
    return;
  }
  if (bq >= 0 && bj == gbj) {   // the lane that holds the winner
    const float4 v = sV[bq];
    const float hi[4] = {v.x, v.y, v.z, 0.0f};
    const float apd = apd_chord(f, M, hi, lo, gam, pen);
    R.assoc[i] = gbj;
    atomicMin(&R.best[gbj], ((unsigned long long)__float_as_uint(apd) << 32) | (uint32_t)i);
  }
}

// Eight lanes per solution.
template <int M>
__device__ __forceinline__ void grid_assoc8(const RunDesc &R, int i, const float4 *sV,
                                            const float *z, const float *w, float pen,
                                            const float *fc) {
  grid_assocL<M, 8>(R, i, sV, z, w, pen, fc);
}

}  // namespace rvea
