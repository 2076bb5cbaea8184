// Build of the direction grid of the association (grid_steps.cuh): after
// every change of the reference vectors (initialisation, adaptation), once
// the tile tables are current.  One CTA per block of cells: the block's tile
// list, each cell's geometry (one thread a cell), then one warp per cell for
// its candidates.  The count pass writes every list it can hold (inline, or
// into the block's share of the overflow area); a scan and the fill pass
// place the few that do not fit.
#include "grid_steps.cuh"

namespace rvea {

constexpr float kGridPad = 4e-6f;   // cell widening in barycentric units (float rounding of a)
constexpr float kDotTol = 3e-6f;    // float32 cosine error allowance of the build's tests
constexpr float kCandEps = 2e-6f;   // 2 eps: dot error of the association relative to |f'|
constexpr float kAngTol = 2e-5f;    // allowance for the float32 angles below (radians)
constexpr int kGridBlockList = 512;  // tiles a block's list holds
constexpr double kGridMaxSkew = 16.0;  // largest range ratio the grid is built for

// The cell's candidate test: centre direction and cos / sin of R (float,
// rounded outwards), or live = false for a cell that lies outside the
// simplex (never looked up).  Every lane computes the same values.
struct CellGeom {
  float c[4];
  float cosR, sinR;
  float corner[4][3];   // the padded cell's corner directions (M - 1 <= 2 axes)
  float vb[4];          // a reference vector close to c
  float delta2;         // (largest chord centre-corner)^2, the curvature allowance
  bool live;
};

// The same for a region of cells [c0, c0 + span) per axis (a cell: span 1;
// a block of cells: its union).  The vector close to the centre is sought
// among the tiles list[0 .. nl) (every tile with list == null).  SERIAL
// false: the warp scans the tiles and members together (every lane must
// call it and gets the result); true: the calling thread scans them alone,
// in order, keeping the first maximum (the same choice as the warp's
// smaller-index tie-break), so that a warp computes 32 cells at once.
template <int M, bool SERIAL = false>
__device__ CellGeom region_geom(const RunDesc &R, const int *ck, int span, const float4 *Vt,
                                const int *list, int nl) {
  CellGeom g;
  g.live = false;
  const int G = R.gG, lane = SERIAL ? 0 : (threadIdx.x & 31), stride = SERIAL ? 1 : 32;
  float lo[2], hi[2], sl = 0.0f;
  for (int k = 0; k < M - 1; ++k) {
    lo[k] = (float)ck[k] / (float)G - kGridPad;
    hi[k] = (float)min(G, ck[k] + span) / (float)G + kGridPad;
    sl += lo[k];
  }
  if (sl > 1.0f) return g;
  float w[M];
  for (int k = 0; k < M; ++k) w[k] = R.gscale[k];
  // a point a of the scaled simplex -> unit direction a / w
  auto dir = [&](const float *a, float *x) {
    float s2 = 0.0f, last = 1.0f;
    for (int k = 0; k < M - 1; ++k) last -= a[k];
    for (int k = 0; k < M; ++k) {
      x[k] = (k < M - 1 ? a[k] : last) / w[k];
      s2 += x[k] * x[k];
    }
    const float inv = rsqrtf(s2);
    for (int k = 0; k < M; ++k) x[k] *= inv;
  };
  float a[2], c[M];
  for (int k = 0; k < M - 1; ++k) a[k] = 0.5f * (lo[k] + hi[k]);
  dir(a, c);
  // rho from the longest chord centre-corner (well conditioned for small angles)
  float chord = 0.0f;
  for (int msk = 0; msk < (1 << (M - 1)); ++msk) {
    for (int k = 0; k < M - 1; ++k) a[k] = (msk >> k) & 1 ? hi[k] : lo[k];
    float x[M], d2 = 0.0f;
    dir(a, x);
    for (int k = 0; k < M; ++k) {
      d2 += (x[k] - c[k]) * (x[k] - c[k]);
      g.corner[msk][k] = x[k];
    }
    chord = fmaxf(chord, sqrtf(d2));
  }
  g.delta2 = (chord + 1e-5f) * (chord + 1e-5f);
  const float kPi = 3.14159265f;
  const float rho = 2.0f * asinf(fminf(1.0f, 0.5f * chord)) + kAngTol;
  for (int k = 0; k < 4; ++k) g.c[k] = k < M ? c[k] : 0.0f;
  // a vector close to c: the best member of the tile whose centre is closest
  float bt = -INFINITY;
  int tb = 0;
  for (int e = lane; e < nl; e += stride) {
    const int t = list ? list[e] : e;
    const float d = pdot<M>(g.c, R.tcen[t]);
    if (d > bt || (d == bt && t < tb)) { bt = d; tb = t; }
  }
  if (!SERIAL) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, bt, off);
      const int ot = __shfl_xor_sync(0xffffffffu, tb, off);
      if (od > bt || (od == bt && ot < tb)) { bt = od; tb = ot; }
    }
  }
  const int2 rg = R.trng[tb];
  float cb = -INFINITY;
  int qb = rg.x;
  for (int q = lane; q < rg.y; q += stride) {
    const float d = pdot<M>(g.c, Vt[rg.x + q]);
    if (d > cb) { cb = d; qb = rg.x + q; }
  }
  if (!SERIAL) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, cb, off);
      const int oq = __shfl_xor_sync(0xffffffffu, qb, off);
      if (od > cb || (od == cb && oq < qb)) { cb = od; qb = oq; }
    }
  }
  {
    const float4 v = Vt[qb];
    g.vb[0] = v.x; g.vb[1] = v.y; g.vb[2] = v.z; g.vb[3] = 0.0f;
  }
  // angle to that vector (bounded above), the lower bound Lb of the best
  // cosine over the cell, the candidate radius R (bounded above)
  const float thb = acosf(fmaxf(-1.0f, fminf(1.0f, cb - kDotTol))) + kAngTol;
  const float Lb = cosf(fminf(kPi, thb + rho)) - kDotTol;
  const float Rr = fminf(kPi, rho + acosf(fmaxf(-1.0f, Lb - kCandEps)) + kAngTol);
  g.cosR = cosf(Rr) - kDotTol;
  g.sinR = fminf(1.0f, sinf(Rr) + kDotTol);
  g.live = true;
  return g;
}

// A finer necessary condition for member v (float): with u = v - v_b and any
// direction d of the cell, d.v >= d.v_b - 2 eps requires
//   c.u + max_corner (x - c).u + delta^2 |u| >= -2 eps
// ((d - c).u is at most its value at a corner of the cell, up to the
// curvature of the cell on the sphere, below delta^2 |u|).  It keeps the
// lists short where the cell is elongated in angle.
template <int M>
__device__ __forceinline__ bool support_test(const CellGeom &g, float4 v) {
  const float u[3] = {v.x - g.vb[0], v.y - g.vb[1], M > 2 ? v.z - g.vb[2] : 0.0f};
  float cu = 0.0f, uu = 0.0f;
#pragma unroll
  for (int k = 0; k < M; ++k) { cu = fmaf(g.c[k], u[k], cu); uu = fmaf(u[k], u[k], uu); }
  float sup = -INFINITY;
#pragma unroll
  for (int msk = 0; msk < (1 << (M - 1)); ++msk) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < M; ++k) s = fmaf(g.corner[msk][k] - g.c[k], u[k], s);
    sup = fmaxf(sup, s);
  }
  return cu + sup + g.delta2 * sqrtf(uu) >= -(kCandEps + 2.0f * kDotTol);
}

// Count (FILL = false) or write (FILL = true) the candidates of one cell:
// the tiles of the list whose centre lies within R + rho_t of c, then their
// members within R that pass the support test.
// The count pass also keeps the first kGridWarpBuf candidates in `buf` (the
// warp's shared-memory list), for its own write of an overflow list.
template <int M, bool FILL>
__device__ int grid_one(const RunDesc &R, const int *ck, const CellGeom &g, const int *list, int nl,
                        bool inl, int at, uint16_t *buf) {
  const int lane = threadIdx.x & 31;
  const int cell = M == 2 ? ck[0] : ck[0] + ck[1] * R.gG;
  const float4 *Vt = R.Vt;
  int n = 0;
  // inline records hold up to kGridInline candidates; longer lists go to the
  // overflow area at offset `at`
  uint16_t *rec = R.gcell + (size_t)cell * kGridRec;
  if (g.live) {
    const bool wide = g.cosR < 0.0f;   // R > pi/2: every tile of the list
    const float cR = g.cosR, sR = g.sinR;
    const float thr_m = g.cosR - kDotTol;
    for (int e0 = 0; e0 < nl; e0 += 32) {
      const int e = e0 + lane;
      bool pass = false;
      if (e < nl) {
        const int t = list ? list[e] : e;
        const float2 cs = R.tcs[t];
        const float d = pdot<M>(g.c, R.tcen[t]);
        pass = wide || d >= fmaf(cR, cs.x, -sR * cs.y) - kDotTol;
      }
      unsigned tm = __ballot_sync(0xffffffffu, pass);
      while (tm) {
        const int ee = e0 + __ffs(tm) - 1;
        tm &= tm - 1;
        const int2 rg = R.trng[list ? list[ee] : ee];
        for (int q0 = 0; q0 < rg.y; q0 += 32) {
          const int q = q0 + lane;
          bool in = false;
          if (q < rg.y) {
            const float4 v = Vt[rg.x + q];
            in = pdot<M>(g.c, v) >= thr_m && support_test<M>(g, v);
          }
          const unsigned mm = __ballot_sync(0xffffffffu, in);
          if (in) {
            const int k = n + __popc(mm & ((1u << lane) - 1u));
            if (!FILL) {   // the count pass writes the first kGridInline in place;
              if (k < kGridInline) rec[1 + k] = (uint16_t)(rg.x + q);   // the fill pass
              if (k < kGridWarpBuf) buf[k] = (uint16_t)(rg.x + q);
            } else {       // only the cells past kGridInline that the count pass left, into their list
              R.gover[at + k] = (uint16_t)(rg.x + q);
            }
          }
          n += __popc(mm);
        }
      }
    }
  }
  if (!FILL && lane == 0) {
    R.gcnt[cell] = n;
    rec[0] = (uint16_t)min(n, 0xFFFF);
  }
  return n;
}

// The count pass runs five CTAs per SM (48 registers): a chain of dependent
// table reads per cell, so resident warps set its speed (94 -> 83 us at
// N = 9870; the fill pass, which visits fewer blocks, gained nothing).
// One CTA per block of cells (kGridSpan2 cells for m = 2, kGridSpan3 x
// kGridSpan3 for m = 3): warp 0 lists the tiles that can hold a candidate
// of any cell of the block (the block taken as one region: every vector
// that can be the argmax for a direction in one of its cells lies within
// the block's radius, so its tile is listed), then the warps take the
// block's cells, each testing only the listed tiles.  A list longer than
// the buffer falls back to every tile.
template <int M, bool FILL>
__device__ void grid_block(const RunDesc &R) {
  __shared__ int s_list[kGridBlockList];
  __shared__ uint16_t s_buf[8][kGridWarpBuf];   // count: each warp's current list
  __shared__ CellGeom s_geo[kGridSpan2 > kGridSpan3 * kGridSpan3 ? kGridSpan2 : kGridSpan3 * kGridSpan3];
  __shared__ int s_n, s_ovf, s_fast;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = R.gG, span = M == 2 ? kGridSpan2 : kGridSpan3;
  const int nbx = (G + span - 1) / span;
  if (__ldcg(&R.ctl->grid_skip)) return;   // vectors too skewed: no grid for them
  if (FILL && __ldcg(&R.ctl->grid_ver) != __ldcg(&R.ctl->v_ver)) return;   // did not fit
  // fill: a block without overflow cells was finished by the count pass
  if (FILL && __ldcg(R.gblk + blockIdx.x + 1) == __ldcg(R.gblk + blockIdx.x)) return;
  // count: this block's overflow candidates (cells past kGridInline); fill:
  // the next free position of the block's range of the overflow area
  if (threadIdx.x == 0) { s_ovf = 0; s_fast = 0; }
  int b0[2] = {0, 0};
  {
    int rem = blockIdx.x;
    for (int k = 0; k < M - 1; ++k) { b0[k] = (rem % nbx) * span; rem /= nbx; }
  }
  if (warp == 0) {
    const CellGeom gb = region_geom<M>(R, b0, span, R.Vt, nullptr, R.ntiles);
    int n = 0;
    if (gb.live) {
      const bool wide = gb.cosR < 0.0f;
      for (int t0 = 0; t0 < R.ntiles; t0 += 32) {
        const int t = t0 + lane;
        bool pass = false;
        if (t < R.ntiles) {
          const float2 cs = R.tcs[t];
          const float d = pdot<M>(gb.c, R.tcen[t]);
          pass = wide || d >= fmaf(gb.cosR, cs.x, -gb.sinR * cs.y) - kDotTol;
        }
        const unsigned tm = __ballot_sync(0xffffffffu, pass);
        const int e = n + __popc(tm & ((1u << lane) - 1u));
        if (pass && e < kGridBlockList) s_list[e] = t;
        n += __popc(tm);
      }
    }
    if (lane == 0) s_n = gb.live ? n : -1;
  }
  __syncthreads();
  const int nl = s_n;
  const bool all = nl > kGridBlockList;
  const int per = M == 2 ? span : span * span;
  const int base = FILL ? __ldcg(R.gblk + blockIdx.x) : 0;
  if (nl >= 0) {   // else the block lies outside the simplex, and so do its cells
    // the cells' geometry first, one thread a cell (no lane repeats the
    // trigonometry and the scans of another's cell)
    for (int q = threadIdx.x; q < per; q += blockDim.x) {
      const int ck[2] = {b0[0] + (M == 2 ? q : q % span), M == 2 ? 0 : b0[1] + q / span};
      CellGeom g;
      g.live = false;
      if (ck[0] < G && (M == 2 || ck[1] < G))
        g = region_geom<M, true>(R, ck, 1, R.Vt, all ? nullptr : s_list, all ? R.ntiles : nl);
      s_geo[q] = g;
    }
    __syncthreads();
    for (int q = warp; q < per; q += nw) {
      int ck[2] = {b0[0] + (M == 2 ? q : q % span), M == 2 ? 0 : b0[1] + q / span};
      if (ck[0] >= G || (M == 3 && ck[1] >= G)) continue;
      const int cell = M == 2 ? ck[0] : ck[0] + ck[1] * G;
      bool inl = true;
      int at = 0;
      if (FILL) {   // an overflow cell claims its range and records it
        const int cnt = __ldcg(R.gcnt + cell);
        inl = cnt <= kGridInline || (cnt & kGridFastBit);
        if (inl) continue;   // written by the count pass
        {
          if (lane == 0) at = R.gfast_off + base + atomicAdd(&s_ovf, cnt);
          at = __shfl_sync(0xffffffffu, at, 0);
          if (lane == 0) {
            uint16_t *rec = R.gcell + (size_t)cell * kGridRec;
            rec[1] = (uint16_t)(at & 0xFFFF);
            rec[2] = (uint16_t)((uint32_t)at >> 16);
          }
        }
      }
      const int n = grid_one<M, FILL>(R, ck, s_geo[q], all ? nullptr : s_list, all ? R.ntiles : nl,
                                      inl, at, FILL ? nullptr : s_buf[warp]);
      if (!FILL && n > kGridInline) {
        // an overflow list: into this block's share when the warp holds it all
        // and the share has room, else left to the fill pass
        int fat = -1;
        if (n <= kGridWarpBuf && lane == 0) {
          const int off = atomicAdd(&s_fast, n);
          if (off + n <= kGridBlockCap) fat = blockIdx.x * kGridBlockCap + off;
        }
        fat = __shfl_sync(0xffffffffu, fat, 0);
        __syncwarp();   // the warp's list is complete in s_buf
        if (fat >= 0) {
          for (int e = lane; e < n; e += 32) R.gover[fat + e] = s_buf[warp][e];
          if (lane == 0) {
            uint16_t *rec = R.gcell + (size_t)cell * kGridRec;
            rec[1] = (uint16_t)(fat & 0xFFFF);
            rec[2] = (uint16_t)((uint32_t)fat >> 16);
            R.gcnt[cell] = n | kGridFastBit;
          }
        } else if (lane == 0) {
          atomicAdd(&s_ovf, n);
        }
        __syncwarp();   // s_buf is read before the next cell overwrites it
      }
    }
  }
  if (!FILL) {
    __syncthreads();
    if (threadIdx.x == 0) R.gblk[blockIdx.x] = s_ovf;
  }
}

__global__ void __launch_bounds__(256, 5) k_grid_count(const RunDesc *__restrict__ Rp) {
  const RunDesc &R = *Rp;
  if (R.m == 2) grid_block<2, false>(R); else grid_block<3, false>(R);
}
__global__ void __launch_bounds__(256) k_grid_fill(const RunDesc *__restrict__ Rp) {
  const RunDesc &R = *Rp;
  if (R.m == 2) grid_block<2, true>(R); else grid_block<3, true>(R);
}

// Exclusive scan of the blocks' overflow totals into their offsets in the
// overflow area (in place), one CTA.  The grid is marked current for this V
// when the overflow lists fit their buffer (and the vectors were not too
// skewed to build it).
__global__ void __launch_bounds__(1024) k_grid_scan(const RunDesc *__restrict__ Rp) {
  __shared__ int s_w[32];
  const RunDesc &R = *Rp;
  if (__ldcg(&R.ctl->grid_skip)) return;
  const int n = grid_build_blocks(R.gG, R.m), tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + 1023) / 1024, a0 = min(n, tid * per), a1 = min(n, a0 + per);
  int sum = 0;
  for (int c = a0; c < a1; ++c) sum += R.gblk[c];
  int incl = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = s_w[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += y;
    }
    s_w[lane] = v;
  }
  __syncthreads();
  int run = (warp > 0 ? s_w[warp - 1] : 0) + incl - sum;
  for (int c = a0; c < a1; ++c) {
    const int k = R.gblk[c];
    R.gblk[c] = run;
    run += k;
  }
  if (tid == 1023) {
    const int total = s_w[31];
    R.gblk[n] = total;   // the end of the last block's range
    if (total <= R.gcap) R.ctl->grid_ver = R.ctl->v_ver;
  }
}

// Grid scale w = 1 / range of the last adaptation (1 before any), as float.
// The build is skipped (grid_skip) when the ranges differ by more than
// kGridMaxSkew: the candidate lists then grow long (the vectors crowd into
// part of the cells), the build costs more than the lookups save, and the
// search falls back to the tiles.
__global__ void k_grid_scale(const RunDesc *__restrict__ Rp) {
  const RunDesc &R = *Rp;
  if (threadIdx.x < R.m) R.gscale[threadIdx.x] = (float)(1.0 / R.vrange[threadIdx.x]);
  if (threadIdx.x == 0) {
    double lo = R.vrange[0], hi = R.vrange[0];
    for (int k = 1; k < R.m; ++k) {
      lo = fmin(lo, R.vrange[k]);
      hi = fmax(hi, R.vrange[k]);
    }
    R.ctl->grid_skip = hi > kGridMaxSkew * lo ? 1 : 0;
  }
}

}  // namespace rvea
