// End of a generation, reference-vector adaptation and state transfer.
//
// k_finalize (one CTA per run) turns the per-vector minima best[j] into the
// next population P_{t+1} without copying any row: slot j of the population
// simply points at the physical pool row of its survivor.  It then builds
// the ascending list of valid slots (mating, next generation), the list of
// free pool rows that receive the next offspring, the next ideal point
// (minimum over the survivors; children lower it with atomics), and on
// adaptation generations rescales V0 by the survivors' objective range in
// FP64 (Algorithm 2, "update reference vectors").  gamma (Eq. 5) follows in
// k_gamma.
#include "finalize_steps.cuh"
#include "metrics.cuh"

namespace rvea {

// Exclusive scan of one int per thread over a CTA of kFinThreads threads.
__device__ int block_exclusive_scan(int v, int *s_warp, int *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  __syncthreads();
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < (kFinThreads >> 5)) ? s_warp[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    s_warp[lane] = w;   // inclusive prefix of warp totals
  }
  __syncthreads();
  const int before = (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
  *total = s_warp[(kFinThreads >> 5) - 1];
  __syncthreads();
  return before;
}

// ---- finalize ---------------------------------------------------------------
// Every thread decodes one reference vector j: the survivor of j (best[j])
// becomes slot j of P_{t+1}.  The CTAs publish compact bitmaps -- valid slots
// (one warp ballot per 32 vectors) and occupied pool rows (atomicOr) -- and
// their own minimum / maximum of the survivors' objectives.  The last CTA to
// finish (an arrival counter, no spinning) builds the ascending list of valid
// slots (mating of the next generation), the ascending list of free pool rows
// (its offspring), the next z*, and on adaptation generations rescales V0 by
// the survivors' objective range in FP64.

__global__ void __launch_bounds__(kFinDecode)
k_finalize(const __grid_constant__ BatchDir dir) {
  pdl_wait();
  pdl_trigger();
  __shared__ FinShared sh;
  __shared__ int s_last;
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int blk = blockIdx.x - dir.prefix[run];
  const int nblk = dir.prefix[run + 1] - dir.prefix[run];
  fin_decode(R, blk, sh);
  // the barrier (in fin_decode) orders every thread's writes before thread
  // 0's (cumulative) fence, which orders them before its arrival
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&R.ctl->fin_cnt, 1) == nblk - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  fin_lists(R, nblk, sh);
}

// gamma_j = min_{i != j} angle(v_i, v_j) (Eq. 5), FP64.  arccos is
// decreasing, so gamma_j = acos(max_{i != j} v_i.v_j) for unit rows.  A float
// pass finds max32 over reference-vector tiles staged in shared memory; only
// the i whose float dot is within 1e-5 of it (the float error of a dot of
// unit vectors is below 1e-6) are re-evaluated in FP64, so the FP64 maximum
// is exact.  One block = 32 vectors j x 8 interleaved slices of i.  Each
// thread keeps its kGKeep largest float dots from the pass: when its
// smallest kept dot is below the window, every i of its slice inside the
// window is kept and rechecked directly; otherwise (a slice with more than
// kGKeep dots in the window) the block makes a second float pass.
constexpr int kGTileF4 = 2048;   // float4s of one shared-memory tile (32 KB)
constexpr int kGKeep = 4;

__device__ __forceinline__ void gamma_load_tile(const RunDesc &R, int base, int nv, int m4,
                                                float4 *tile) {
  const int m = R.m;
  for (int q = threadIdx.x; q < nv * m4; q += blockDim.x) {
    if (R.V32) {
      tile[q] = reinterpret_cast<const float4 *>(R.V32)[(size_t)base * m4 + q];
    } else {
      const int i = base + q / m4, c = 4 * (q % m4);
      const double *v = R.V64 + (size_t)i * m;
      tile[q] = make_float4(c < m ? (float)v[c] : 0.f, c + 1 < m ? (float)v[c + 1] : 0.f,
                            c + 2 < m ? (float)v[c + 2] : 0.f, c + 3 < m ? (float)v[c + 3] : 0.f);
    }
  }
}

// FP64 dot of two rows; a call, so the rare recheck stays a real branch
// instead of being predicated into every iteration of the float scan.
__device__ __noinline__ double dot64(const double *a, const double *b, int m) {
  double e = 0.0;
  for (int k = 0; k < m; ++k) e += a[k] * b[k];
  return e;
}

template <int M>
__device__ void gamma_block_t(const RunDesc &R, int jb, float4 *tile) {
  constexpr int M4 = (M + 3) / 4;
  const int N = R.N;
  const int jl = threadIdx.x >> 3, sl = threadIdx.x & 7;
  const int j = jb * 32 + jl;
  const bool act = j < N;
  float vf[M4 * 4];
#pragma unroll
  for (int k = 0; k < M4 * 4; ++k) vf[k] = 0.f;
  if (act) {
    if (R.V32) {
#pragma unroll
      for (int k = 0; k < M; ++k) vf[k] = R.V32[(size_t)j * M4 * 4 + k];
    } else {
#pragma unroll
      for (int k = 0; k < M; ++k) vf[k] = (float)R.V64[(size_t)j * M + k];
    }
  }
  const double *vjp = R.V64 + (size_t)(act ? j : 0) * M;
  constexpr int kGTile = kGTileF4 / M4;
  float kd[kGKeep];   // the kGKeep largest float dots of this slice, descending
  int ki[kGKeep];
#pragma unroll
  for (int c = 0; c < kGKeep; ++c) { kd[c] = -INFINITY; ki[c] = 0; }
  for (int base = 0; base < N; base += kGTile) {
    const int nv = min(kGTile, N - base);
    __syncthreads();
    gamma_load_tile(R, base, nv, M4, tile);
    __syncthreads();
    if (act) {
#pragma unroll 4
      for (int u = sl; u < nv; u += 8) {
        float d = 0.f;
#pragma unroll
        for (int q = 0; q < M4; ++q) {
          const float4 v = tile[u * M4 + q];
          d = fmaf(vf[4 * q], v.x, d);
          d = fmaf(vf[4 * q + 1], v.y, d);
          d = fmaf(vf[4 * q + 2], v.z, d);
          d = fmaf(vf[4 * q + 3], v.w, d);
        }
        if (d > kd[kGKeep - 1] && base + u != j) {
          float vd = d;
          int vi = base + u;
#pragma unroll
          for (int c = 0; c < kGKeep; ++c) {
            if (vd > kd[c]) {
              const float od = kd[c];
              const int oi = ki[c];
              kd[c] = vd; ki[c] = vi;
              vd = od; vi = oi;
            }
          }
        }
      }
    }
  }
  float mx = kd[0];
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const float thr = mx - 1e-5f;
  double best = -2.0;
  if (!__syncthreads_or(act && kd[kGKeep - 1] >= thr)) {
    if (act) {
#pragma unroll
      for (int c = 0; c < kGKeep; ++c)
        if (kd[c] >= thr) best = fmax(best, dot64(R.V64 + (size_t)ki[c] * M, vjp, M));
    }
  } else for (int base = 0; base < N; base += kGTile) {
    const int nv = min(kGTile, N - base);
    __syncthreads();
    gamma_load_tile(R, base, nv, M4, tile);
    __syncthreads();
    if (act) {
      for (int u = sl; u < nv; u += 8) {
        float d = 0.f;
#pragma unroll
        for (int q = 0; q < M4; ++q) {
          const float4 v = tile[u * M4 + q];
          d = fmaf(vf[4 * q], v.x, d);
          d = fmaf(vf[4 * q + 1], v.y, d);
          d = fmaf(vf[4 * q + 2], v.z, d);
          d = fmaf(vf[4 * q + 3], v.w, d);
        }
        const int i = base + u;
        if (d >= thr && i != j) best = fmax(best, dot64(R.V64 + (size_t)i * M, vjp, M));
      }
    }
  }
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if (act && sl == 0) {
    double g = acos(fmin(1.0, fmax(-1.0, best)));
    if (!(g >= 1e-12)) g = 1e-12;
    R.gamma64[j] = g;
    if (R.gamma32) R.gamma32[j] = (float)g;
  }
}

__device__ void gamma_block(const RunDesc &R, int jb) {
  __shared__ float4 tile[kGTileF4];
  switch (R.m) {
    case 2: gamma_block_t<2>(R, jb, tile); return;
    case 3: gamma_block_t<3>(R, jb, tile); return;
    case 4: gamma_block_t<4>(R, jb, tile); return;
    case 5: gamma_block_t<5>(R, jb, tile); return;
    case 6: gamma_block_t<6>(R, jb, tile); return;
    case 7: gamma_block_t<7>(R, jb, tile); return;
    case 8: gamma_block_t<8>(R, jb, tile); return;
    case 9: gamma_block_t<9>(R, jb, tile); return;
    case 10: gamma_block_t<10>(R, jb, tile); return;
    case 11: gamma_block_t<11>(R, jb, tile); return;
    case 12: gamma_block_t<12>(R, jb, tile); return;
    case 13: gamma_block_t<13>(R, jb, tile); return;
    case 14: gamma_block_t<14>(R, jb, tile); return;
    case 15: gamma_block_t<15>(R, jb, tile); return;
    default: gamma_block_t<16>(R, jb, tile); return;
  }
}

// gamma_j through the k-d tiles of the vectors (m <= 4, tables current for
// this V): one thread per vector j.  The float pass scans the tile whose
// centre is closest to v_j, then every tile that can hold a vector i != j
// with a float dot >= b - 2e-5 (b the best so far; the tile's centre dot
// against cos(acos(b') + rho) with rho rounded outwards and 1e-5 of slack,
// which only admits more tiles); the final float maximum b is then the full
// pass's max32, and the FP64 recheck of every i with a float dot within
// 1e-5 of it (in the tiles that can hold one) gives gamma_j bit for bit as
// the full pass does: both take the FP64 maximum over a set that holds the
// true maximiser, with the same dot64.
template <int M>
__device__ __forceinline__ float gdot(const float *a, float4 b) {
  float d = a[0] * b.x;
  if (M > 1) d = fmaf(a[1], b.y, d);
  if (M > 2) d = fmaf(a[2], b.z, d);
  if (M > 3) d = fmaf(a[3], b.w, d);
  return d;
}

// kGammaLanes lanes per vector j (a group of consecutive lanes of a warp;
// every lane of the warp calls it): the lanes split the tile loops, reduce
// over the group between the passes, and the group's first lane writes
// gamma_j.
constexpr int kGammaLanes = 8;   // 16 measured slower (57 against 48 us at N = 9870)
template <int M>
__device__ void gamma_group(const RunDesc &R, int j) {
  constexpr int GL = kGammaLanes;
  const int T = R.ntiles, lane = threadIdx.x & 31, sub = lane & (GL - 1);
  const bool act = j < R.N;
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  if (act) {
#pragma unroll
    for (int k = 0; k < M; ++k) v[k] = R.V32[(size_t)j * 4 + k];   // m <= 4: one float4 a row
  }
  auto member = [&](int pos) { return M < 4 ? __float_as_int(R.Vt[pos].w) : R.tperm[pos]; };
  auto admits = [&](int t, float bt_) {
    const float Bt = fmaxf(-1.0f, bt_);
    const float S = sqrtf(fmaxf(0.0f, 1.0f - Bt * Bt));
    const float2 cs = R.tcs[t];
    return gdot<M>(v, R.tcen[t]) >= fmaf(Bt, cs.x, -S * cs.y) - 1e-5f;
  };
  // the closest centre (ties: the smaller tile)
  float bc = -INFINITY;
  int bt = 0x7FFFFFFF;
  for (int t = sub; t < T; t += GL) {
    const float d = gdot<M>(v, R.tcen[t]);
    if (d > bc) { bc = d; bt = t; }
  }
#pragma unroll
  for (int off = 1; off < GL; off <<= 1) {
    const float od = __shfl_xor_sync(0xffffffffu, bc, off);
    const int ot = __shfl_xor_sync(0xffffffffu, bt, off);
    if (od > bc || (od == bc && ot < bt)) { bc = od; bt = ot; }
  }
  float b = -2.0f;
  if (act && bt < T) {   // its members, split over the group
    const int2 rg = R.trng[bt];
    for (int q = sub; q < rg.y; q += GL)
      if (member(rg.x + q) != j) b = fmaxf(b, gdot<M>(v, R.Vt[rg.x + q]));
  }
#pragma unroll
  for (int off = 1; off < GL; off <<= 1) b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, off));
  // every other tile that can hold a dot within 2e-5 of b, one lane a tile
  const float b0 = b - 2e-5f;
  if (act) {
    for (int t = sub; t < T; t += GL) {
      if (t == bt || !admits(t, b0)) continue;
      const int2 rg = R.trng[t];
      for (int q = 0; q < rg.y; ++q)
        if (member(rg.x + q) != j) b = fmaxf(b, gdot<M>(v, R.Vt[rg.x + q]));
    }
  }
#pragma unroll
  for (int off = 1; off < GL; off <<= 1) b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, off));
  // FP64 recheck of the float maxima within 1e-5 of b
  const float thr = b - 1e-5f;
  const double *vjp = R.V64 + (size_t)(act ? j : 0) * M;
  double best = -2.0;
  if (act) {
    for (int t = sub; t < T; t += GL) {
      if (t != bt && !admits(t, thr - 1e-5f)) continue;
      const int2 rg = R.trng[t];
      for (int q = 0; q < rg.y; ++q) {
        const int i = member(rg.x + q);
        if (i != j && gdot<M>(v, R.Vt[rg.x + q]) >= thr)
          best = fmax(best, dot64(R.V64 + (size_t)i * M, vjp, M));
      }
    }
  }
#pragma unroll
  for (int off = 1; off < GL; off <<= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if (act && sub == 0) {
    double g = acos(fmin(1.0, fmax(-1.0, best)));
    if (!(g >= 1e-12)) g = 1e-12;
    R.gamma64[j] = g;
    if (R.gamma32) R.gamma32[j] = (float)g;
  }
}

__device__ void gamma_tiles(const RunDesc &R) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  constexpr int PW = 32 / kGammaLanes;   // vectors a warp
  for (int base = PW * wg; base < R.N; base += PW * nw) {   // warp-uniform
    const int j = base + lane / kGammaLanes;
    switch (R.m) {
      case 2: gamma_group<2>(R, j); break;
      case 3: gamma_group<3>(R, j); break;
      default: gamma_group<4>(R, j); break;
    }
  }
}

// Persistent over the directory: every run with ctl->adapted set (or every
// run when `force`) has its vector blocks of 32 spread over the grid.
__global__ void __launch_bounds__(256)
k_gamma(const __grid_constant__ BatchDir dir, int force) {
  pdl_wait();
  for (int r = 0; r < dir.n; ++r) {
    const RunDesc &R = *dir.desc[r];
    if (!force && R.ctl->adapted == 0) continue;
    if (R.ntiles > 0 && R.m <= 4 && R.ctl->tiles_ver == R.ctl->v_ver) {   // uniform over the grid
      gamma_tiles(R);
      continue;
    }
    const int nb = (R.N + 31) / 32;
    for (int jb = blockIdx.x; jb < nb; jb += gridDim.x) gamma_block(R, jb);
  }
}

// rvea_gamma: one caller-supplied set of vectors, descriptor by value.
__global__ void __launch_bounds__(256) k_gamma_op(const __grid_constant__ RunDesc D) {
  gamma_block(D, blockIdx.x);
}

// ---- inverted generational distance (Appendix C, the IGD equation) ----------
// One thread per reference point: the squared distance to every valid member
// of the current population (staged in shared memory kIgdTile members at a
// time, compacted), the root of the minimum in FP64, then the block's sum in
// a fixed tree into partial[blockIdx.x]; k_igd_final adds the partials in
// order.  The minimum is exact whatever the member order.
constexpr int kIgdThreads = 256;
constexpr int kIgdTile = 512;

__global__ void __launch_bounds__(kIgdThreads)
k_igd_partial(const RunDesc *__restrict__ Rp, const float *__restrict__ ref, int n_ref,
              double *__restrict__ partial) {
  __shared__ float sF[kMaxM * kIgdTile];   // objective k of member i at k * kIgdTile + i
  __shared__ int s_cnt;
  __shared__ double s_w[kIgdThreads / 32];
  const RunDesc &R = *Rp;
  const int m = R.m, N = R.N, n2 = 2 * N;
  const int *cur = R.slotmap + (R.ctl->t & 1) * N;
  const int r = blockIdx.x * kIgdThreads + threadIdx.x;
  float rv[kMaxM];
#pragma unroll
  for (int k = 0; k < kMaxM; ++k) rv[k] = (r < n_ref && k < m) ? ref[(size_t)r * m + k] : 0.0f;
  float best = INFINITY;
  for (int base = 0; base < N; base += kIgdTile) {
    __syncthreads();   // the previous tile is no longer read
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int nt = min(kIgdTile, N - base);
    for (int q = threadIdx.x; q < nt; q += kIgdThreads) {
      const int slot = cur[base + q];
      if (slot < 0 || slot >= n2) continue;
      const int pos = atomicAdd(&s_cnt, 1);
      for (int k = 0; k < m; ++k) sF[k * kIgdTile + pos] = R.F[(size_t)k * n2 + slot];
    }
    __syncthreads();
    const int c = s_cnt;
    if (r < n_ref) {
      for (int i = 0; i < c; ++i) {
        float d2 = 0.0f;
#pragma unroll
        for (int k = 0; k < kMaxM; ++k) {
          if (k < m) {
            const float e = rv[k] - sF[k * kIgdTile + i];
            d2 = fmaf(e, e, d2);
          }
        }
        best = fminf(best, d2);
      }
    }
  }
  double v = r < n_ref ? sqrt((double)best) : 0.0;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kIgdThreads / 32; ++w) s += s_w[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_igd_final(const double *__restrict__ partial, int nb, int n_ref,
                            double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[b];
  *out = s / (double)n_ref;
}

// ---- hypervolume (Appendix C, the HV equation), m = 2 or 3 -----------------
// (scratch layout: metrics.cuh)  The volume is cut into slabs along
// f3 at the members' f3 values; a slab's area is the 2-D hypervolume of the
// members at or below it, summed as bands: in f1 order, a member that lowers
// the running minimum of f2 from mprev to f2 adds (ref1 - f1) (mprev - f2).
// One CTA of 1024 threads: compaction in slot order (block scan of flags).
__global__ void __launch_bounds__(1024)
k_hv_compact(const RunDesc *__restrict__ Rp, HvRef ref, HvScratch S) {
  __shared__ int s_w[32];
  __shared__ int s_base;
  const RunDesc &R = *Rp;
  const int N = R.N, n2 = 2 * N, m = R.m;
  const int *cur = R.slotmap + (R.ctl->t & 1) * N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  for (int base = 0; base < N; base += 1024) {
    const int j = base + threadIdx.x;
    double a = 0.0, b = 0.0, c = 0.0;
    bool ok = false;
    if (j < N) {
      const int slot = cur[j];
      if (slot >= 0 && slot < n2) {
        a = (double)R.F[slot];
        b = (double)R.F[(size_t)n2 + slot];
        c = m == 3 ? (double)R.F[2 * (size_t)n2 + slot] : 0.0;
        ok = a < ref.r1 && b < ref.r2 && c < ref.r3;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    int before = s_base;
    for (int w = 0; w < warp; ++w) before += s_w[w];
    const int pos = before + __popc(bal & ((1u << lane) - 1u));
    if (ok) {
      S.f1[pos] = a;
      S.f2[pos] = b;
      S.f3[pos] = c;
    }
    __syncthreads();   // every thread has read s_base and s_w
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < 32; ++w) tot += s_w[w];
      s_base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *S.count = s_base;
}

// Member p's rank by (f1, index) and by (f3, index), and the inverse
// permutations: a count over all members.
__global__ void __launch_bounds__(256) k_hv_rank(HvScratch S) {
  const int n = *S.count;
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p >= n) return;
  const double a = S.f1[p], c = S.f3[p];
  int r1 = 0, r3 = 0;
  for (int q = 0; q < n; ++q) {
    const double aq = S.f1[q], cq = S.f3[q];
    r1 += (aq < a || (aq == a && q < p)) ? 1 : 0;
    r3 += (cq < c || (cq == c && q < p)) ? 1 : 0;
  }
  S.byF1[r1] = p;
  S.byF3[r3] = p;
  S.rank3[p] = r3;
}

// One warp per slab i (the members of f3 rank <= i, up to the next f3).
__global__ void __launch_bounds__(256) k_hv_slices(HvScratch S, HvRef ref) {
  const int n = *S.count;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;   // whole warps
  const double z = S.f3[S.byF3[i]];
  const double zn = i + 1 < n ? S.f3[S.byF3[i + 1]] : ref.r3;
  const double h = zn - z;
  if (!(h > 0.0)) {
    if (lane == 0) S.vol[i] = 0.0;
    return;
  }
  double area = 0.0, carry = ref.r2;
  for (int c0 = 0; c0 < n; c0 += 32) {
    const int sidx = c0 + lane;
    int p = 0;
    bool incl = false;
    if (sidx < n) {
      p = S.byF1[sidx];
      incl = S.rank3[p] <= i;
    }
    const double f2 = incl ? S.f2[p] : INFINITY;
    double pm = fmin(f2, carry);   // inclusive running minimum
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, pm, off);
      if (lane >= off) pm = fmin(pm, y);
    }
    double prev = __shfl_up_sync(0xffffffffu, pm, 1);
    if (lane == 0) prev = carry;
    if (incl) area += (ref.r1 - S.f1[p]) * fmax(0.0, prev - f2);
    carry = __shfl_sync(0xffffffffu, pm, 31);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) area += __shfl_xor_sync(0xffffffffu, area, off);
  if (lane == 0) S.vol[i] = h * area;
}

// The slabs' volumes in a fixed order: lane l sums slabs l, l + 32, ...,
// then a fixed tree.
__global__ void k_hv_final(HvScratch S, double *out) {
  const int n = *S.count, lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += S.vol[i];
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) *out = s;
}

// ---- state transfer -------------------------------------------------------
// Population rows in slot order -> dst (N x d); invalid rows NaN.
__global__ void k_gather_pop(const RunDesc *__restrict__ Rp, float *dst, uint8_t *valid) {
  const RunDesc &R = *Rp;
  const int j = blockIdx.x;
  const int s = R.slotmap[(R.ctl->t & 1) * R.N + j];
  if (threadIdx.x == 0 && valid) valid[j] = s >= 0 ? 1 : 0;
  if (!dst) return;
  float *o = dst + (size_t)j * R.d;
  const float *x = s >= 0 ? R.X + (size_t)s * R.d_pad : nullptr;
  for (int k = threadIdx.x; k < R.d; k += blockDim.x) o[k] = x ? x[k] : __int_as_float(0x7fc00000);
}

__global__ void k_gather_obj(const RunDesc *__restrict__ Rp, float *dst, uint8_t *valid) {
  const RunDesc &R = *Rp;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= R.N) return;
  const int s = R.slotmap[(R.ctl->t & 1) * R.N + j];
  if (valid) valid[j] = s >= 0 ? 1 : 0;
  if (!dst) return;
  for (int k = 0; k < R.m; ++k)
    dst[(size_t)j * R.m + k] = s >= 0 ? R.F[(size_t)k * R.n_comb + s] : __int_as_float(0x7fc00000);
}

// Children of the last completed generation (t - 1), child order.
__global__ void k_gather_children(const RunDesc *__restrict__ Rp, float *X, float *F) {
  const RunDesc &R = *Rp;
  const int c = blockIdx.x;
  const int t = R.ctl->t - 1;
  const int s = R.child_slot[(t & 1) * R.N + c];
  if (X) {
    const float *x = R.X + (size_t)s * R.d_pad;
    for (int k = threadIdx.x; k < R.d; k += blockDim.x) X[(size_t)c * R.d + k] = x[k];
  }
  if (F && threadIdx.x < R.m) F[(size_t)c * R.m + threadIdx.x] = R.F[(size_t)threadIdx.x * R.n_comb + s];
}

// Swarm state of a CSO or PSO run in vector-slot order: each valid slot's
// velocity row, kept APD and (PSO) personal-best row and objectives (NaN and
// +inf for invalid slots).  One CTA per slot.
__global__ void k_gather_swarm(const RunDesc *__restrict__ Rp, float *vel, float *apd, float *pbest,
                               float *fpbest) {
  const RunDesc &R = *Rp;
  const int j = blockIdx.x;
  const int s = R.slotmap[(R.ctl->t & 1) * R.N + j];
  const float qnan = __int_as_float(0x7fc00000);
  if (vel) {
    const float *v = s >= 0 ? R.vel + (size_t)s * R.d_pad : nullptr;
    for (int k = threadIdx.x; k < R.d; k += blockDim.x) vel[(size_t)j * R.d + k] = v ? v[k] : qnan;
  }
  if (pbest) {
    const float *p = s >= 0 ? R.pb + (size_t)s * R.d_pad : nullptr;
    for (int k = threadIdx.x; k < R.d; k += blockDim.x) pbest[(size_t)j * R.d + k] = p ? p[k] : qnan;
  }
  if (fpbest && threadIdx.x < R.m)
    fpbest[(size_t)j * R.m + threadIdx.x] = s >= 0 ? R.fpb[(size_t)threadIdx.x * R.n_comb + s] : qnan;
  if (apd && threadIdx.x == 0) apd[j] = s >= 0 ? R.kapd[j] : __int_as_float(0x7f800000);
}

__global__ void k_copy_selection(const RunDesc *__restrict__ Rp, int *assoc, int *surv) {
  const RunDesc &R = *Rp;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (assoc && i < R.n_comb) assoc[i] = R.assoc[i];
  if (surv && i < R.N) surv[i] = R.surv[i];
}

// Import: F (N x m, staged in device memory), valid (N), V (N x m f64) and
// gamma are in place; rebuild slot map, lists, z*, float copies.  One CTA.
__global__ void __launch_bounds__(kFinThreads)
k_import(const RunDesc *__restrict__ Rp, const float *Fin, const uint8_t *vin, int t) {
  __shared__ int s_warp[32];
  __shared__ int s_total;
  __shared__ unsigned s_z[kMaxM];
  const RunDesc &R = *Rp;
  const int N = R.N, n2 = 2 * N, m = R.m, tid = threadIdx.x;
  if (tid < kMaxM) s_z[tid] = 0xFFFFFFFFu;
  __syncthreads();
  for (int j = tid; j < N; j += kFinThreads) {
    const bool v = vin[j] != 0;
    R.slotmap[(t & 1) * N + j] = v ? j : -1;
    for (int k = 0; k < m; ++k) {
      const float f = Fin[(size_t)j * m + k];
      R.F[(size_t)k * n2 + j] = f;
      if (v) atomicMin(&s_z[k], f2ord(f));
    }
    float *v32 = R.V32 + (size_t)j * R.m4 * 4;
    for (int k = 0; k < R.m4 * 4; ++k) v32[k] = k < m ? (float)R.V64[(size_t)j * m + k] : 0.0f;
    for (int k = 0; k < m; ++k) {
      const double v = R.V64[(size_t)j * m + k];
      R.V32lo[(size_t)j * m + k] = (float)(v - (double)(float)v);
    }
    R.gamma32[j] = (float)R.gamma64[j];
    R.best[j] = ~0ull;
    R.surv[j] = -1;
    if (R.kapd) R.kapd[j] = __int_as_float(0x7f800000);   // CSO: no selection kept it yet
  }
  for (int i = tid; i < n2; i += kFinThreads) { R.amax[i] = 0ull; R.assoc[i] = -1; R.otag[i] = 0; }
  for (int w = tid; w < (n2 + 31) / 32; w += kFinThreads) R.obits[w] = 0u;
  for (int b = tid; b < (n2 + kSelBlock - 1) / kSelBlock; b += kFinThreads) R.blk_cnt[b] = 0;
  // valid list
  const int ch = (N + kFinThreads - 1) / kFinThreads;
  const int a0 = min(N, tid * ch), a1 = min(N, a0 + ch);
  int cnt = 0;
  for (int j = a0; j < a1; ++j) cnt += vin[j] != 0;
  int pos = block_exclusive_scan(cnt, s_warp, &s_total);
  const int K = s_total;
  for (int j = a0; j < a1; ++j)
    if (vin[j]) R.vlist[pos++] = j;
  // free rows: invalid slots j < N, then N..2N-1, ascending; first N
  int *cs = R.child_slot + (t & 1) * N;
  const int ch2 = (n2 + kFinThreads - 1) / kFinThreads;
  const int b0 = min(n2, tid * ch2), b1 = min(n2, b0 + ch2);
  int fc = 0;
  for (int s = b0; s < b1; ++s) fc += (s >= N || !vin[s]);
  int fpos = block_exclusive_scan(fc, s_warp, &s_total);
  for (int s = b0; s < b1 && fpos < N; ++s)
    if (s >= N || !vin[s]) cs[fpos++] = s;
  __syncthreads();
  if (tid < m) R.ctl->zkey[tid] = s_z[tid];
  if (tid == 0) {
    R.ctl->K = K;
    R.ctl->t = t;
    R.ctl->status = 0;
    R.ctl->adapted = 0;
    R.ctl->fin_cnt = 0;
    R.ctl->sel_cnt = 0;
    R.ctl->bar = 0ull;
    R.ctl->v_ver += 1;   // V was replaced
    R.ctl->fcomb_t = 0;
  }
  if (tid < m) R.vrange[tid] = 1.0;
}

// Initial slot map and lists after k_init: slot j = row j, children go to
// rows N..2N-1.
__global__ void k_init_lists(const __grid_constant__ BatchDir dir) {
  const RunDesc &R = *dir.desc[blockIdx.y];
  const int N = R.N;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) {
    R.slotmap[1 * N + j] = j;   // t = 1 reads buffer (1 & 1)
    R.vlist[j] = j;
    R.child_slot[1 * N + j] = N + j;   // t = 1 uses buffer (1 & 1)
    R.child_slot[j] = N + j;
    R.best[j] = ~0ull;
    R.surv[j] = -1;
  }
  for (int i = j; i < 2 * N; i += gridDim.x * blockDim.x) { R.amax[i] = 0ull; R.assoc[i] = -1; }
  if (j < (2 * N + kSelBlock - 1) / kSelBlock) R.blk_cnt[j] = 0;
  if (j == 0) {
    R.ctl->t = 1;
    R.ctl->K = N;
    R.ctl->status = 0;
    R.ctl->adapted = 0;
  }
}

}  // namespace rvea
