// Environmental selection (Algorithm 1 and Eqs. 2-5 of arXiv 2404.01159).
//
// The paper materialises n x r tensors (Theta, T_part, T_APD).  Here nothing
// of size n x r exists:
//   * association: arccos is decreasing and every v_j is a unit vector, so
//     RowMin(Theta) is the argmax over j of f'.v_j; each thread streams the
//     reference vectors of its chunk through shared memory (tiles staged by
//     1-D TMA bulk copies, double buffered on mbarriers) and keeps a running
//     (max, first index).  Chunks of the same solutions run in different CTAs
//     and merge with a 64-bit atomicMax on (order-preserving cosine bits,
//     ~j): the larger cosine wins, then the smaller j, exactly as a serial
//     first-minimum scan.
//   * APD (Eq. 4) and the per-vector argmin (lines 14-16): the last CTA of a
//     solution block to finish (an arrival counter, no spinning) computes
//     theta = acos(cos), the APD, and a 64-bit atomicMin on (APD bits,
//     combined index) into best[j]: the smaller APD wins, then the smaller
//     index -- the column argmin with ties to the first row.
// A solution equal to z* has all cosines 0 (dot = 0): it gets vector 0,
// theta = pi/2 and APD 0, as the oracle reads the 0/0 case.
#include "rvea_device.cuh"

namespace rvea {

// Solution i of run R: physical slot (or row of the op input), -1 if invalid.
__device__ __forceinline__ int sol_slot(const RunDesc &R, int i) {
  if (i >= R.n_comb) return -1;
  if (R.op_mode) return (R.valid_in == nullptr || R.valid_in[i]) ? i : -1;
  const int par = R.ctl->t & 1;
  if (i < R.N) return R.slotmap[par * R.N + i];
  return R.child_slot[par * R.N + (i - R.N)];
}

__device__ __forceinline__ float sol_f(const RunDesc &R, int slot, int k) {
  return R.op_mode ? R.F_aos[(size_t)slot * R.m + k] : R.F[(size_t)k * R.n_comb + slot];
}

// Dot product f'.v in one fixed order (first product, then fma over k);
// the scan and the rescan below evaluate it identically, bit for bit.
template <int M>
__device__ __forceinline__ float dotv(const float *fp, const float4 *v) {
  float d = __fmul_rn(fp[0], v[0].x);
#pragma unroll
  for (int k = 1; k < M; ++k) {
    const float4 q = v[k >> 2];
    const float c = (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    d = fmaf(fp[k], c, d);
  }
  return d;
}

// The dots of two solutions (a, b) with one vector, packed: lane x of each
// .f32x2 instruction is dotv of a, lane y that of b (the same IEEE
// operations in the same order, so the rescan's scalar dotv matches).
template <int M>
__device__ __forceinline__ float2 dotv2(const float2 *fab, const float4 *v) {
  float2 d = mul2(fab[0], splat2(v[0].x));
#pragma unroll
  for (int k = 1; k < M; ++k) {
    const float4 q = v[k >> 2];
    const float c = (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    d = fma2(fab[k], splat2(c), d);
  }
  return d;
}

// Chunk scan for W solutions of a thread, two per packed instruction: the
// running maximum of each 32-vector sub-tile costs one fmaxf per dot; a
// sub-tile replaces the best only on a strict improvement, so `bsub` is the
// first sub-tile holding the maximum.  Every loaded vector serves all W
// solutions.
template <int M, int W>
__device__ void scan_chunk(const float4 *__restrict__ sv, int nv, const float2 (*fab)[M],
                           float *best, int *bsub) {
  constexpr int M4 = (M + 3) / 4, NP = W / 2;
  for (int sub = 0; sub * 32 < nv; ++sub) {
    const int n = min(32, nv - sub * 32);
    const float4 *p = sv + (size_t)sub * 32 * M4;
    float mx[W];
#pragma unroll
    for (int q = 0; q < W; ++q) mx[q] = -INFINITY;
    if (n == 32) {
#pragma unroll 4
      for (int jj = 0; jj < 32; ++jj) {
        float4 v[M4];
#pragma unroll
        for (int q = 0; q < M4; ++q) v[q] = p[jj * M4 + q];
#pragma unroll
        for (int h = 0; h < NP; ++h) {
          const float2 d = dotv2<M>(fab[h], v);
          mx[2 * h] = fmaxf(mx[2 * h], d.x);
          mx[2 * h + 1] = fmaxf(mx[2 * h + 1], d.y);
        }
      }
    } else {
      for (int jj = 0; jj < n; ++jj) {
        float4 v[M4];
#pragma unroll
        for (int q = 0; q < M4; ++q) v[q] = p[jj * M4 + q];
#pragma unroll
        for (int h = 0; h < NP; ++h) {
          const float2 d = dotv2<M>(fab[h], v);
          mx[2 * h] = fmaxf(mx[2 * h], d.x);
          mx[2 * h + 1] = fmaxf(mx[2 * h + 1], d.y);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (mx[q] > best[q]) { best[q] = mx[q]; bsub[q] = sub; }
  }
}

// First vector of sub-tile `sub` whose dot equals `best` (the same
// arithmetic: lane Y of the packed pair is the solution).
template <int M, bool Y>
__device__ int find_first(const float4 *__restrict__ sv, int nv, int sub, const float2 *fab,
                          float best) {
  constexpr int M4 = (M + 3) / 4;
  float fp[M];
#pragma unroll
  for (int k = 0; k < M; ++k) fp[k] = Y ? fab[k].y : fab[k].x;
  const int j0 = sub * 32, j1 = min(nv, j0 + 32);
  for (int jj = j0; jj < j1; ++jj) {
    float4 v[M4];
#pragma unroll
    for (int q = 0; q < M4; ++q) v[q] = sv[(size_t)jj * M4 + q];
    if (dotv<M>(fp, v) == best) return jj;
  }
  return j0;
}

// APD (Eq. 4) of a solution and its vote in best[j].
__device__ __forceinline__ void apd_vote(const RunDesc &R, int i, const float *fp) {
  const int m = R.m;
  const unsigned long long key = atomicExch(&R.amax[i], 0ull);
  const int j = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
  const int t = R.op_mode ? R.t_op : R.ctl->t;
  const float pen = (float)m * powf((float)t / (float)R.t_max, R.alpha);
  if (j < 0 || j >= R.N) {
    set_status(R.ctl, ST_BADINDEX);
    return;
  }
  const float apd = apd_chord(fp, m, R.V32 + (size_t)j * R.m4 * 4,
                              R.V32lo ? R.V32lo + (size_t)j * m : nullptr, R.gamma32[j], pen);
  R.assoc[i] = j;
  atomicMin(&R.best[j], ((unsigned long long)__float_as_uint(apd) << 32) | (uint32_t)i);
}

// f' of solution `slot` (0 for an invalid one).
template <int M>
__device__ __forceinline__ void load_fp(const RunDesc &R, int slot, float *fp) {
#pragma unroll
  for (int k = 0; k < M; ++k)
    fp[k] = slot >= 0 ? sol_f(R, slot, k) - ord2f(R.ctl->zkey[k]) : 0.0f;
}

// W of the thread's solutions, from q0 on: scan, first index, merge into amax.
template <int M, int W>
__device__ __forceinline__ void select_group(const RunDesc &R, const SelItem &it, const float4 *s_v,
                                             int nv, const int *idx, const int *slot, int q0) {
  float2 fab[W / 2][M];
#pragma unroll
  for (int h = 0; h < W / 2; ++h) {
    float fa[M], fb[M];
    load_fp<M>(R, slot[q0 + 2 * h], fa);
    load_fp<M>(R, slot[q0 + 2 * h + 1], fb);
#pragma unroll
    for (int k = 0; k < M; ++k) fab[h][k] = make_float2(fa[k], fb[k]);
  }
  float best[W];
  int bsub[W];
#pragma unroll
  for (int q = 0; q < W; ++q) { best[q] = -INFINITY; bsub[q] = 0; }
  scan_chunk<M, W>(s_v, nv, fab, best, bsub);
#pragma unroll
  for (int q = 0; q < W; ++q) {
    if (slot[q0 + q] < 0) continue;
    const int j = (q & 1) ? find_first<M, true>(s_v, nv, bsub[q], fab[q >> 1], best[q])
                          : find_first<M, false>(s_v, nv, bsub[q], fab[q >> 1], best[q]);
    atomicMax(&R.amax[idx[q0 + q]], ((unsigned long long)f2ord(best[q]) << 32) |
                                        (unsigned long long)(0xFFFFFFFFu - (uint32_t)(it.v0 + j)));
  }
}

// One item: kSelBlock solutions (kSelSols per thread, kSelThreads apart) x
// one chunk of reference vectors, the chunk staged in shared memory by one
// 1-D TMA bulk copy.  Up to m = 10 one pass scans the chunk for all four
// solutions of a thread; past that, two passes of two (registers).
template <int M>
__device__ void select_item(const RunDesc &R, const SelItem &it, float4 *s_v, uint64_t *s_bar,
                            int *s_last) {
  constexpr int M4 = (M + 3) / 4;
  int idx[kSelSols], slot[kSelSols];
#pragma unroll
  for (int q = 0; q < kSelSols; ++q) {
    idx[q] = it.sblk * kSelBlock + q * kSelThreads + threadIdx.x;
    slot[q] = sol_slot(R, idx[q]);
  }
  const int nv = it.v1 - it.v0;
  const uint32_t bytes = (uint32_t)(nv * M4 * 16);
  if (threadIdx.x == 0) {
    mbar_init(s_bar, 1);
    fence_mbar_init();
    mbar_expect_tx(s_bar, bytes);
    tma_load_1d(s_v, reinterpret_cast<const float4 *>(R.V32) + (size_t)it.v0 * M4, bytes, s_bar);
  }
  __syncthreads();   // barrier initialised before anyone waits on it
  const bool ok = mbar_wait(s_bar, 0u, kWaitLimit);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      set_status(R.ctl, ST_TIMEOUT);
      mbar_wait(s_bar, 0u, kWaitLimit);   // give the copy a bounded chance to land
    }
    __syncthreads();
    return;
  }
  bool any = false;
#pragma unroll
  for (int q = 0; q < kSelSols; ++q) any |= slot[q] >= 0;
  if (any) {
    if (M <= 10) {
      select_group<M, kSelSols>(R, it, s_v, nv, idx, slot, 0);
    } else {
#pragma unroll 1
      for (int q0 = 0; q0 < kSelSols; q0 += 2) select_group<M, 2>(R, it, s_v, nv, idx, slot, q0);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();   // cumulative: orders the block's atomics before the arrival
    const int prev = atomicAdd(&R.blk_cnt[it.sblk], 1);
    *s_last = (prev == it.nchunks - 1);
  }
  __syncthreads();
  if (!*s_last) return;

  // ---- last chunk of this block: APD and per-vector argmin ---------------
  __threadfence();
#pragma unroll 1
  for (int q = 0; q < kSelSols; ++q) {
    if (slot[q] >= 0) {
      float fp[M];
      load_fp<M>(R, slot[q], fp);
      apd_vote(R, idx[q], fp);
    } else if (idx[q] < R.n_comb) {
      R.assoc[idx[q]] = -1;
    }
  }
  if (threadIdx.x == 0) R.blk_cnt[it.sblk] = 0;
}

__global__ void __launch_bounds__(kSelThreads)
k_select(const __grid_constant__ BatchDir dir) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(128) float4 s_v[];     // [chunk vectors * m4]
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_last;
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const SelItem it = static_cast<const SelItem *>(dir.items[run])[blockIdx.x - dir.prefix[run]];
  switch (R.m) {
    case 2: select_item<2>(R, it, s_v, &s_bar, &s_last); return;
    case 3: select_item<3>(R, it, s_v, &s_bar, &s_last); return;
    case 4: select_item<4>(R, it, s_v, &s_bar, &s_last); return;
    case 5: select_item<5>(R, it, s_v, &s_bar, &s_last); return;
    case 6: select_item<6>(R, it, s_v, &s_bar, &s_last); return;
    case 7: select_item<7>(R, it, s_v, &s_bar, &s_last); return;
    case 8: select_item<8>(R, it, s_v, &s_bar, &s_last); return;
    case 9: select_item<9>(R, it, s_v, &s_bar, &s_last); return;
    case 10: select_item<10>(R, it, s_v, &s_bar, &s_last); return;
    case 11: select_item<11>(R, it, s_v, &s_bar, &s_last); return;
    case 12: select_item<12>(R, it, s_v, &s_bar, &s_last); return;
    case 13: select_item<13>(R, it, s_v, &s_bar, &s_last); return;
    case 14: select_item<14>(R, it, s_v, &s_bar, &s_last); return;
    case 15: select_item<15>(R, it, s_v, &s_bar, &s_last); return;
    default: select_item<16>(R, it, s_v, &s_bar, &s_last); return;
  }
}

// ---- stateless selection: preparation and survivor extraction ------------
// Scratch of the op holds Ctl, best[r], amax[n], blk_cnt; all reset here.
__global__ void k_op_prep(const RunDesc *__restrict__ Rp) {
  const RunDesc &R = *Rp;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int j = tid; j < R.N; j += nth) R.best[j] = ~0ull;
  for (int i = tid; i < R.n_comb; i += nth) R.amax[i] = 0ull;
  const int nblk = (R.n_comb + kSelBlock - 1) / kSelBlock;
  for (int b = tid; b < nblk; b += nth) R.blk_cnt[b] = 0;
  if (tid == 0) {
    R.ctl->t = R.t_op;
    R.ctl->status = 0;
    for (int k = 0; k < kMaxM; ++k) R.ctl->zkey[k] = 0xFFFFFFFFu;
  }
}

__global__ void k_op_zstar(const RunDesc *__restrict__ Rp) {
  const RunDesc &R = *Rp;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R.n_comb) return;
  if (R.valid_in && !R.valid_in[i]) return;
  for (int k = 0; k < R.m; ++k) atomicMin(&R.ctl->zkey[k], f2ord(R.F_aos[(size_t)i * R.m + k]));
}

__global__ void k_op_finish(const RunDesc *__restrict__ Rp) {
  const RunDesc &R = *Rp;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= R.N) return;
  const unsigned long long key = R.best[j];
  R.survivor_out[j] = (key == ~0ull) ? -1 : (int)(uint32_t)(key & 0xFFFFFFFFull);
}

}  // namespace rvea
