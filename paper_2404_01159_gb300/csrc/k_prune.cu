// Kernels of the exact pruned association for m <= 4 (Algorithm 1 lines
// 5-6, Eq. 2): one run with its tile tables staged in shared memory, a batch
// of runs in one persistent launch, and the tile tables after a change of V.
// The search itself (tile bounds, candidate scan, APD vote) is in
// prune_steps.cuh.
#include "grid_steps.cuh"

namespace rvea {

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
  if (R.gG > 0 && __ldcg(&R.ctl->grid_ver) == __ldcg(&R.ctl->v_ver)) {
    // the direction grid: one thread per solution
    const float pen = (float)R.m * powf((float)R.ctl->t / (float)R.t_max, R.alpha);
    float z[4], w[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = k < R.m ? ord2f(R.ctl->zkey[k]) : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = k < R.m ? R.gscale[k] : 1.0f;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = warp * gridDim.x + blockIdx.x, nw = gridDim.x * (blockDim.x >> 5);
    for (int g = gw; 4 * g < R.n_comb; g += nw) {
      if (R.m == 2) grid_assoc8<2>(R, 4 * g + (lane >> 3), sV, z, w, pen, nullptr);
      else grid_assoc8<3>(R, 4 * g + (lane >> 3), sV, z, w, pen, nullptr);
    }
    return;
  }
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
  // the kernels after this one (gamma, the grid) see the tables as current
  if (blockIdx.x == 0 && threadIdx.x == 0) Rp->ctl->tiles_ver = Rp->ctl->v_ver;
}

// The same over a batch (dir.prefix counts CTAs of 8 tiles): runs whose
// vectors were adapted this generation (all runs with force).
__global__ void k_tiles_batch(const __grid_constant__ BatchDir dir, int force) {
  pdl_wait();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  if (!force && R.ctl->adapted == 0) return;
  tile_one(R, (blockIdx.x - dir.prefix[run]) * (blockDim.x >> 5) + (threadIdx.x >> 5));
  if (blockIdx.x == dir.prefix[run] && threadIdx.x == 0) R.ctl->tiles_ver = R.ctl->v_ver;
}

}  // namespace rvea
