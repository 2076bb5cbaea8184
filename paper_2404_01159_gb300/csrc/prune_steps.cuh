// Exact pruned association for m <= 4 (Algorithm 1 lines 5-6, Eq. 2).
//
// The reference vectors are grouped into spatially compact tiles of <= 64
// (a k-d split of the initial lattice, fixed for the run).  Each tile has a
// float32 unit centre c and an angle rho that bounds the angle from c to
// every member.  For a solution f' (norm nf), once some vector reaches the
// float dot `best`, a tile whose centre makes an angle phi with f' can hold
// a larger dot only if phi <= acos(best / nf) + rho, i.e. only if
//   f'.c >= best cos(rho) - sqrt(nf^2 - best^2) sin(rho)      (1)
// (cos(acos(b) + rho) = b cos rho - sqrt(1 - b^2) sin rho).  The test is
// evaluated with margins that cover every float32 rounding involved -- the
// dots of f' with c and with the members (<= 1e-6 nf each for unit rows and
// m <= 16), the norms of the float32 rows, the computed square root -- and
// with cos(rho) rounded down and sin(rho) rounded up: a tile that fails it
// holds only dots strictly below `best`.  The tiles that pass are scanned
// with exactly the arithmetic of the full scan (same order of products),
// keeping the larger dot and, on equal dots, the smaller vector index.  The
// result is therefore the full scan's result bit for bit, found after
// scanning ~2 tiles instead of all of them (lattice of 9870 vectors, m = 3).
// The test itself needs f'.c of every tile, computed in the first pass (the
// closest centre); a lane keeps its kPruneKeep largest ones and the largest of
// the rest.  Every threshold (1) is at least
//   min(B, B cmin) - S smax - slack   (cmin: smallest cos(rho) of the run,
//                                       smax: largest sin(rho)),
// so when the rest stay below that bound (less a rounding margin) only the
// kept tiles can pass, and the second pass tests those alone.
//
// One persistent CTA per SM stages the tile-ordered vectors and the tile
// table in shared memory with TMA bulk copies; its warps take four solutions
// at a time from a work counter, eight lanes per solution, and cast each
// solution's APD vote (Eq. 4) directly.
#pragma once
#include "rvea_device.cuh"

namespace rvea {

constexpr int kPruneThreads = 1024;
constexpr int kPruneCand = 4;   // candidate tiles kept per lane before the fallback
constexpr int kPruneKeep = 4;   // largest centre dots a lane keeps from the first pass

// f'.v in the fixed order of the full scan: first product, then fma over k.
template <int M>
__device__ __forceinline__ float pdot(const float *f, float4 v) {
  float d = __fmul_rn(f[0], v.x);
  if (M > 1) d = fmaf(f[1], v.y, d);
  if (M > 2) d = fmaf(f[2], v.z, d);
  if (M > 3) d = fmaf(f[3], v.w, d);
  return d;
}

// Vector index of tile-order position q: kept in the unused fourth lane of
// the float4 row for m <= 3, read from the permutation for m = 4.
template <int M>
__device__ __forceinline__ int vidx(const RunDesc &R, float4 v, int q) {
  return M < 4 ? __float_as_int(v.w) : R.tperm[q];
}

// Keeps (best, bj): larger dot, then smaller vector index.
__device__ __forceinline__ void keep(float d, int j, float &best, int &bj) {
  if (d > best || (d == best && j < bj)) { best = d; bj = j; }
}

// Tables read from shared memory (staged) or through L1 (G = true).
template <bool G, class T>
__device__ __forceinline__ T tld(const T *p) {
  if constexpr (G) return __ldg(p);
  else return *p;
}

// Solutions base .. base+3 of one run, eight lanes each: association by the
// pruned search, then the APD vote.
template <int M, bool G>
__device__ __forceinline__ void prune_group(const RunDesc &R, int base, const float4 *sV,
                                            const float4 *sC, const float2 *sCS, const int2 *sR,
                                            const float *z, float pen, float2 cs_bound) {
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int T = R.ntiles, N = R.N, n = R.n_comb;
  const int t_gen = R.ctl->t;
  {
    const int i = base + (lane >> 3);
    int slot = -1;
    if (i < n) {
      const int par = t_gen & 1;
      slot = i < N ? R.slotmap[par * N + i] : R.child_slot[par * N + (i - N)];
    }
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    if (slot >= 0) {
#pragma unroll
      for (int k = 0; k < M; ++k) f[k] = __ldcg(R.F + (size_t)k * n + slot) - z[k];
    }
    float s2 = f[0] * f[0];
#pragma unroll
    for (int k = 1; k < M; ++k) s2 = fmaf(f[k], f[k], s2);
    const float nf = sqrtf(s2);
    // invalid parents take no part; f' = 0 has every dot +0, where the full
    // scan keeps vector 0 -- neither needs the search (all lanes still run
    // the shuffles below, over empty loops)
    const bool live = slot >= 0 && nf > 0.0f;
    const int TT = live ? T : 0;

    // pass 1: the tile whose centre is closest in angle; the lane's
    // kPruneKeep largest centre dots (descending) and the largest of the rest
    float kd[kPruneKeep];
    int kt[kPruneKeep];
#pragma unroll
    for (int c = 0; c < kPruneKeep; ++c) { kd[c] = -INFINITY; kt[c] = 0; }
    float rest = -INFINITY;
    for (int t = sub; t < TT; t += 8) {
      const float dc = pdot<M>(f, tld<G>(sC + t));
      if (dc > kd[kPruneKeep - 1]) {
        rest = fmaxf(rest, kd[kPruneKeep - 1]);
        float vd = dc;
        int vt = t;
#pragma unroll
        for (int c = 0; c < kPruneKeep; ++c) {   // insertion: strict, so equal dots keep order
          if (vd > kd[c]) {
            const float od = kd[c];
            const int ot = kt[c];
            kd[c] = vd; kt[c] = vt;
            vd = od; vt = ot;
          }
        }
      } else {
        rest = fmaxf(rest, dc);
      }
    }
    float dc1 = kd[0];
    int t1 = kt[0];
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, dc1, off);
      const int ot = __shfl_xor_sync(0xffffffffu, t1, off);
      if (od > dc1 || (od == dc1 && ot < t1)) { dc1 = od; t1 = ot; }
    }
    // scan that tile
    float best = -INFINITY;
    int bj = 0x7FFFFFFF;
    {
      const int2 rg = live ? tld<G>(sR + t1) : make_int2(0, 0);
      for (int q = sub; q < rg.y; q += 8) {
        const float4 v = tld<G>(sV + rg.x + q);
        keep(pdot<M>(f, v), vidx<M>(R, v, rg.x + q), best, bj);
      }
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) keep(__shfl_xor_sync(0xffffffffu, best, off),
                                               __shfl_xor_sync(0xffffffffu, bj, off), best, bj);
    // threshold (1) with margins
    const float Bn = (best - 1e-6f * nf) * (1.0f - 4e-7f);
    const float Sn = sqrtf(fmaxf(0.0f, (nf - Bn) + 4e-7f * nf) * (nf + fabsf(Bn)));
    const float slack = 3e-6f * nf;
    // a lower bound of every tile's threshold, less the rounding of the
    // thresholds' two fmas and of the bound itself
    const float lb = fminf(Bn, Bn * cs_bound.x) - Sn * cs_bound.y - slack -
                     1e-6f * (fabsf(Bn) + Sn + slack);
    // pass 2: tiles that may hold a larger (or equal) dot
    int cand[kPruneCand];
    int nc = 0;
    bool over = false;
    if (rest < lb) {   // only kept tiles can pass
#pragma unroll
      for (int k = 0; k < kPruneKeep; ++k) {
        const int t = kt[k];
        if (kd[k] == -INFINITY || t == t1) continue;
        const float2 cs = tld<G>(sCS + t);
        if (kd[k] >= fmaf(Bn, cs.x, fmaf(-Sn, cs.y, -slack))) {
#pragma unroll
          for (int c = 0; c < kPruneCand; ++c)
            if (c == nc) cand[c] = t;
          ++nc;
        }
      }
    } else for (int t = sub; t < TT; t += 8) {
      const float2 cs = tld<G>(sCS + t);
      const float thr = fmaf(Bn, cs.x, fmaf(-Sn, cs.y, -slack));
      if (t != t1 && pdot<M>(f, tld<G>(sC + t)) >= thr) {
        if (nc < kPruneCand) {
#pragma unroll
          for (int c = 0; c < kPruneCand; ++c)
            if (c == nc) cand[c] = t;
          ++nc;
        } else {
          over = true;
        }
      }
    }
    // scan the candidates: the union of the 8 lanes' lists, each tile split
    // over the solution's 8 lanes (members sub, sub + 8, ...); every group
    // of 8 walks its own list, the warp steps until all are done
    int ncmax = nc;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) ncmax = max(ncmax, __shfl_xor_sync(0xffffffffu, ncmax, off));
    const int gbase = lane & 24;
#pragma unroll
    for (int c = 0; c < kPruneCand; ++c) {
      if (c >= ncmax) break;
      const int mine = c < nc ? cand[c] : -1;
      unsigned m = (__ballot_sync(0xffffffffu, c < nc) >> gbase) & 0xFFu;
      while (__any_sync(0xffffffffu, m != 0u)) {
        const bool had = m != 0u;
        const int src = had ? __ffs(m) - 1 : 0;
        m &= m - 1u;
        const int t = __shfl_sync(0xffffffffu, mine, gbase | src);
        if (had && t >= 0) {
          const int2 rg = tld<G>(sR + t);
          for (int q = sub; q < rg.y; q += 8) {
            const float4 v = tld<G>(sV + rg.x + q);
            keep(pdot<M>(f, v), vidx<M>(R, v, rg.x + q), best, bj);
          }
        }
      }
    }
    if (over) {   // more candidates than kept: test and scan the rest here
      int seen = 0;
      for (int t = sub; t < TT; t += 8) {
        const float2 cs = tld<G>(sCS + t);
        const float thr = fmaf(Bn, cs.x, fmaf(-Sn, cs.y, -slack));
        if (t != t1 && pdot<M>(f, tld<G>(sC + t)) >= thr) {
          if (seen++ < kPruneCand) continue;   // scanned above
          const int2 rg = tld<G>(sR + t);
          for (int q = 0; q < rg.y; ++q) {
            const float4 v = tld<G>(sV + rg.x + q);
            keep(pdot<M>(f, v), vidx<M>(R, v, rg.x + q), best, bj);
          }
        }
      }
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) keep(__shfl_xor_sync(0xffffffffu, best, off),
                                               __shfl_xor_sync(0xffffffffu, bj, off), best, bj);
    if (slot >= 0 && !live) { best = 0.0f; bj = 0; }
    // APD (Eq. 4) and the vote of this solution in best[j]
    if (sub == 0 && i < n) {
      if (slot < 0) {
        R.assoc[i] = -1;
      } else if (bj < 0 || bj >= N) {
        set_status(R.ctl, ST_BADINDEX);
      } else {
        const float apd = apd_chord(f, M, R.V32 + (size_t)bj * R.m4 * 4, R.V32lo + (size_t)bj * M,
                                    R.gamma32[bj], pen);
        R.assoc[i] = bj;
        atomicMin(&R.best[bj], ((unsigned long long)__float_as_uint(apd) << 32) | (uint32_t)i);
      }
    }
  }
}

// (smallest cos(rho), largest sin(rho)) over the T tiles of the staged
// table; a barrier for the whole CTA.  (1, 0) when there are no tiles.
__device__ __forceinline__ float2 tile_bounds(const float2 *sCS, int T) {
  __shared__ unsigned s_b[2];
  if (threadIdx.x == 0) { s_b[0] = 0xFFFFFFFFu; s_b[1] = 0u; }
  __syncthreads();
  unsigned lo = 0xFFFFFFFFu, hi = 0u;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const float2 cs = sCS[t];
    lo = min(lo, f2ord(cs.x));
    hi = max(hi, f2ord(cs.y));
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&s_b[0], lo);
    atomicMax(&s_b[1], hi);
  }
  __syncthreads();
  return T > 0 ? make_float2(ord2f(s_b[0]), ord2f(s_b[1])) : make_float2(1.0f, 0.0f);
}

// One run, tables in shared memory: warps take four solutions at a time from
// the run's work counter.
template <int M>
__device__ void prune_loop(const RunDesc &R, const float4 *sV, const float4 *sC,
                           const float2 *sCS, const int2 *sR, float2 csb) {
  const int lane = threadIdx.x & 31;
  const float pen = (float)R.m * powf((float)R.ctl->t / (float)R.t_max, R.alpha);
  float z[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) z[k] = k < M ? ord2f(R.ctl->zkey[k]) : 0.f;
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&R.ctl->sel_cnt, 4);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= R.n_comb) break;
    prune_group<M, false>(R, base, sV, sC, sCS, sR, z, pen, csb);
  }
}

}  // namespace rvea
