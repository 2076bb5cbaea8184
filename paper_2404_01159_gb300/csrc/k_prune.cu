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
      for (int k = 0; k < M; ++k) f[k] = R.F[(size_t)k * n + slot] - z[k];
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

__global__ void __launch_bounds__(kPruneThreads, 1) k_select_pruned(const RunDesc *__restrict__ Rp) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar;
  const RunDesc &R = *Rp;
  const int N = R.N, T = R.ntiles;
  // layout: Vt [N] float4 | centres [T] float4 | (cos, sin) [T] float2 | ranges [T] int2
  const uint32_t bV = (uint32_t)N * 16, bC = (uint32_t)T * 16, bS = (uint32_t)T * 8;
  const uint32_t bSr = (bS + 15u) & ~15u;
  float4 *sV = reinterpret_cast<float4 *>(smem);
  float4 *sC = reinterpret_cast<float4 *>(smem + bV);
  float2 *sCS = reinterpret_cast<float2 *>(smem + bV + bC);
  int2 *sR = reinterpret_cast<int2 *>(smem + bV + bC + bSr);
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    mbar_expect_tx(&s_bar, bV + bC + 2 * bSr);
    tma_load_1d(sV, R.Vt, bV, &s_bar);
    tma_load_1d(sC, R.tcen, bC, &s_bar);
    tma_load_1d(sCS, R.tcs, bSr, &s_bar);
    tma_load_1d(sR, R.trng, bSr, &s_bar);
  }
  __syncthreads();
  const bool ok = mbar_wait(&s_bar, 0u, kWaitLimit);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      set_status(R.ctl, ST_TIMEOUT);
      mbar_wait(&s_bar, 0u, kWaitLimit);
    }
    __syncthreads();
    return;
  }
  // the tables (k_tiles, earlier than the predecessor) are staged above; the
  // population's objectives come from the reproduction kernel
  const float2 csb = tile_bounds(sCS, T);
  pdl_wait();
  pdl_trigger();
  switch (R.m) {
    case 2: prune_loop<2>(R, sV, sC, sCS, sR, csb); break;
    case 3: prune_loop<3>(R, sV, sC, sCS, sR, csb); break;
    default: prune_loop<4>(R, sV, sC, sCS, sR, csb); break;
  }
}

// A batch of runs in one persistent launch.  Work comes in chunks of
// kPruneChunk solutions of one run (dir.prefix counts chunks), taken by whole
// CTAs from the work counter of the first run; a CTA stages the tables of
// the chunk's run in shared memory with TMA unless they are already there
// (chunks come in run order, so a CTA reloads about once per run it visits).
constexpr int kPruneChunk = 2048;

__global__ void __launch_bounds__(kPruneThreads, 1) k_select_pruned_batch(const __grid_constant__ BatchDir dir) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_chunk;
  const int warp = threadIdx.x >> 5;
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  Ctl *cc = dir.desc[0]->ctl;
  const int total = dir.prefix[dir.n];
  int cached = -1;
  uint32_t phase = 0;
  float2 csb = make_float2(1.0f, 0.0f);
  for (;;) {
    __syncthreads();   // the previous chunk is done with the tables
    if (threadIdx.x == 0) s_chunk = atomicAdd(&cc->sel_cnt, 1);
    __syncthreads();
    const int c = s_chunk;
    if (c >= total) break;
    const int run = dir_find(dir, c);
    const RunDesc &R = *dir.desc[run];
    const int N = R.N, T = R.ntiles;
    const uint32_t bV = (uint32_t)N * 16, bC = (uint32_t)T * 16, bS = (uint32_t)T * 8;
    const uint32_t bSr = (bS + 15u) & ~15u;
    float4 *sV = reinterpret_cast<float4 *>(smem);
    float4 *sC = reinterpret_cast<float4 *>(smem + bV);
    float2 *sCS = reinterpret_cast<float2 *>(smem + bV + bC);
    int2 *sR = reinterpret_cast<int2 *>(smem + bV + bC + bSr);
    if (run != cached) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(&s_bar, bV + bC + 2 * bSr);
        tma_load_1d(sV, R.Vt, bV, &s_bar);
        tma_load_1d(sC, R.tcen, bC, &s_bar);
        tma_load_1d(sCS, R.tcs, bSr, &s_bar);
        tma_load_1d(sR, R.trng, bSr, &s_bar);
      }
      const bool ok = mbar_wait(&s_bar, phase, kWaitLimit);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          set_status(R.ctl, ST_TIMEOUT);
          mbar_wait(&s_bar, phase ^ 1u, kWaitLimit);
        }
        __syncthreads();
        return;
      }
      cached = run;
      csb = tile_bounds(sCS, T);
    }
    const float pen = (float)R.m * powf((float)R.ctl->t / (float)R.t_max, R.alpha);
    float z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = k < R.m ? ord2f(R.ctl->zkey[k]) : 0.f;
    const int base0 = (c - dir.prefix[run]) * kPruneChunk;
    const int nsol = min(kPruneChunk, R.n_comb - base0);
    for (int g = 4 * warp; g < nsol; g += 4 * (kPruneThreads / 32)) {
      switch (R.m) {
        case 2: prune_group<2, false>(R, base0 + g, sV, sC, sCS, sR, z, pen, csb); break;
        case 3: prune_group<3, false>(R, base0 + g, sV, sC, sCS, sR, z, pen, csb); break;
        default: prune_group<4, false>(R, base0 + g, sV, sC, sCS, sR, z, pen, csb); break;
      }
    }
  }
}

// Tile table after a change of V: members in tile order, float32 centres,
// and conservative (cos rho, sin rho) computed in FP64 from the float32 rows.
// One warp per tile.
__device__ __forceinline__ void tile_one(const RunDesc &R, int t) {
  const int lane = threadIdx.x & 31;
  if (t >= R.ntiles) return;
  const int2 rg = R.trng[t];   // up to 2 x 32 members: lane takes q = lane, lane + 32
  const int m4 = R.m4;
  float4 v[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = lane + 32 * h;
    v[h] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < rg.y) {
      const int j = R.tperm[rg.x + q];
      v[h] = reinterpret_cast<const float4 *>(R.V32)[(size_t)j * m4];
      float4 vt = v[h];
      if (R.m < 4) vt.w = __int_as_float(j);   // the member's vector index rides along
      R.Vt[rg.x + q] = vt;
    }
  }
  // centre: normalised mean of the members
  float sx = v[0].x + v[1].x, sy = v[0].y + v[1].y, sz = v[0].z + v[1].z, sw = v[0].w + v[1].w;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
    sz += __shfl_xor_sync(0xffffffffu, sz, off);
    sw += __shfl_xor_sync(0xffffffffu, sw, off);
  }
  const double cn = sqrt((double)sx * sx + (double)sy * sy + (double)sz * sz + (double)sw * sw);
  const float4 c = make_float4((float)(sx / cn), (float)(sy / cn), (float)(sz / cn), (float)(sw / cn));
  // rho: the largest angle centre-member, both float32 rows normalised in FP64
  double cmin = 1.0;
  const double ccn = sqrt((double)c.x * c.x + (double)c.y * c.y + (double)c.z * c.z + (double)c.w * c.w);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (lane + 32 * h < rg.y) {
      const float4 u = v[h];
      const double vn = sqrt((double)u.x * u.x + (double)u.y * u.y + (double)u.z * u.z + (double)u.w * u.w);
      const double cosang = ((double)u.x * c.x + (double)u.y * c.y + (double)u.z * c.z + (double)u.w * c.w) / (vn * ccn);
      cmin = fmin(cmin, cosang);
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) cmin = fmin(cmin, __shfl_xor_sync(0xffffffffu, cmin, off));
  if (lane == 0) {
    const double rho = fmin(1.5707963267948966, acos(fmax(-1.0, cmin)) + 1e-6);
    R.tcen[t] = c;
    R.tcs[t] = make_float2(__double2float_rd(cos(rho)), __double2float_ru(sin(rho)));
  }
}

__global__ void k_tiles(const RunDesc *__restrict__ Rp) {
  pdl_wait();
  tile_one(*Rp, blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
}

// The same over a batch (dir.prefix counts CTAs of 8 tiles): runs whose
// vectors were adapted this generation (all runs with force).
__global__ void k_tiles_batch(const __grid_constant__ BatchDir dir, int force) {
  pdl_wait();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  if (!force && R.ctl->adapted == 0) return;
  tile_one(R, (blockIdx.x - dir.prefix[run]) * (blockDim.x >> 5) + (threadIdx.x >> 5));
}

}  // namespace rvea
