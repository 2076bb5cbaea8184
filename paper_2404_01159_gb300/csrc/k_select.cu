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
  if (i < R.N) return R.slotmap[i];
  return R.child_slot[(R.ctl->t & 1) * R.N + (i - R.N)];
}

__device__ __forceinline__ float sol_f(const RunDesc &R, int slot, int k) {
  return R.op_mode ? R.F_aos[(size_t)slot * R.m + k] : R.F[(size_t)k * R.n_comb + slot];
}

// Running argmax of f'.v over one shared-memory tile, dot accumulated in the
// fixed order f0 v0, then fma over k = 1..m-1.
template <int M>
__device__ __forceinline__ void scan_tile(const float4 *__restrict__ tv, int nv, int jbase,
                                          const float *fpin, float &best, int &bj) {
  constexpr int M4 = (M + 3) / 4;
  float fp[M];
#pragma unroll
  for (int k = 0; k < M; ++k) fp[k] = fpin[k];
#pragma unroll 4
  for (int jj = 0; jj < nv; ++jj) {
    float v[M4 * 4];
#pragma unroll
    for (int q = 0; q < M4; ++q) {
      const float4 t4 = tv[jj * M4 + q];
      v[4 * q] = t4.x; v[4 * q + 1] = t4.y; v[4 * q + 2] = t4.z; v[4 * q + 3] = t4.w;
    }
    float dot = fp[0] * v[0];
#pragma unroll
    for (int k = 1; k < M; ++k) dot = fmaf(fp[k], v[k], dot);
    if (dot > best) { best = dot; bj = jbase + jj; }
  }
}

__device__ __forceinline__ void scan_tile_rt(const float4 *__restrict__ tv, int nv, int jbase,
                                             int m, int m4, const float *fp, float &best,
                                             int &bj) {
  switch (m) {
    case 2: scan_tile<2>(tv, nv, jbase, fp, best, bj); return;
    case 3: scan_tile<3>(tv, nv, jbase, fp, best, bj); return;
    case 4: scan_tile<4>(tv, nv, jbase, fp, best, bj); return;
    case 5: scan_tile<5>(tv, nv, jbase, fp, best, bj); return;
    case 6: scan_tile<6>(tv, nv, jbase, fp, best, bj); return;
    case 8: scan_tile<8>(tv, nv, jbase, fp, best, bj); return;
    case 10: scan_tile<10>(tv, nv, jbase, fp, best, bj); return;
    default: break;
  }
  for (int jj = 0; jj < nv; ++jj) {
    const float *v = reinterpret_cast<const float *>(tv + jj * m4);
    float dot = fp[0] * v[0];
    for (int k = 1; k < m; ++k) dot = fmaf(fp[k], v[k], dot);
    if (dot > best) { best = dot; bj = jbase + jj; }
  }
}

__global__ void __launch_bounds__(kSelThreads)
k_select(const __grid_constant__ BatchDir dir) {
  extern __shared__ __align__(128) float4 s_v[];     // [2][kVTile * m4]
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_last;

  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const SelItem it = static_cast<const SelItem *>(dir.items[run])[blockIdx.x - dir.prefix[run]];
  const int m = R.m, m4 = R.m4;
  const int i = it.sblk * kSelThreads + threadIdx.x;
  const int slot = sol_slot(R, i);

  float fp[kMaxM];
#pragma unroll
  for (int k = 0; k < kMaxM; ++k) fp[k] = 0.0f;
  if (slot >= 0) {
    for (int k = 0; k < m; ++k) fp[k] = sol_f(R, slot, k) - ord2f(R.ctl->zkey[k]);
  }

  // ---- stream reference-vector tiles of [v0, v1) -------------------------
  const int nv_all = it.v1 - it.v0;
  const int ntiles = (nv_all + kVTile - 1) / kVTile;
  const float4 *Vg = reinterpret_cast<const float4 *>(R.V32);
  const int tile_f4 = kVTile * m4;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int k) {
    const int j0 = it.v0 + k * kVTile;
    const int nv = min(kVTile, it.v1 - j0);
    const uint32_t bytes = (uint32_t)(nv * m4 * 16);
    uint64_t *bar = &s_bar[k & 1];
    mbar_expect_tx(bar, bytes);
    tma_load_1d(s_v + (k & 1) * tile_f4, Vg + (size_t)j0 * m4, bytes, bar);
  };
  if (threadIdx.x == 0) {
    if (ntiles > 0) issue(0);
    if (ntiles > 1) issue(1);
  }
  float best = -INFINITY;
  int bj = it.v0;
  bool ok = true;
  for (int k = 0; k < ntiles; ++k) {
    if (!mbar_wait(&s_bar[k & 1], (uint32_t)((k >> 1) & 1), kWaitLimit)) ok = false;
    if (__syncthreads_or(!ok)) {
      // a bulk copy never completed: flag it, then give the copies in flight
      // a bounded chance to land before this CTA's shared memory goes away
      if (threadIdx.x == 0) {
        set_status(R.ctl, ST_TIMEOUT);
        for (int q = k; q < min(k + 2, ntiles); ++q)
          mbar_wait(&s_bar[q & 1], (uint32_t)((q >> 1) & 1), kWaitLimit);
      }
      __syncthreads();
      return;
    }
    const int j0 = it.v0 + k * kVTile;
    const int nv = min(kVTile, it.v1 - j0);
    if (slot >= 0) scan_tile_rt(s_v + (k & 1) * tile_f4, nv, j0, m, m4, fp, best, bj);
    __syncthreads();   // every thread is done with this buffer
    if (threadIdx.x == 0 && k + 2 < ntiles) issue(k + 2);
  }

  if (slot >= 0) {
    const unsigned long long key =
        ((unsigned long long)f2ord(best) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)bj);
    atomicMax(&R.amax[i], key);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int prev = atomicAdd(&R.blk_cnt[it.sblk], 1);
    s_last = (prev == it.nchunks - 1);
  }
  __syncthreads();
  if (!s_last) return;

  // ---- last chunk of this block: APD and per-vector argmin ---------------
  __threadfence();
  if (slot >= 0) {
    const unsigned long long key = atomicExch(&R.amax[i], 0ull);
    const int j = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
    const float dot = ord2f((unsigned)(key >> 32));
    float s = fp[0] * fp[0];
    for (int k = 1; k < m; ++k) s = fmaf(fp[k], fp[k], s);
    const float nf = sqrtf(s);
    float theta = 1.5707963267948966f;
    if (nf > 0.0f) theta = acosf(fminf(1.0f, fmaxf(-1.0f, dot / nf)));
    const int t = R.op_mode ? R.t_op : R.ctl->t;
    const float pen = (float)m * powf((float)t / (float)R.t_max, R.alpha);
    if (j < 0 || j >= R.N) {
      set_status(R.ctl, ST_BADINDEX);
    } else {
      const float apd = (1.0f + pen * theta / R.gamma32[j]) * nf;
      R.assoc[i] = j;
      atomicMin(&R.best[j], ((unsigned long long)__float_as_uint(apd) << 32) | (uint32_t)i);
    }
  } else if (i < R.n_comb) {
    R.assoc[i] = -1;
  }
  if (threadIdx.x == 0) R.blk_cnt[it.sblk] = 0;
}

// ---- stateless selection: preparation and survivor extraction ------------
// Scratch of the op holds Ctl, best[r], amax[n], blk_cnt; all reset here.
__global__ void k_op_prep(const RunDesc *__restrict__ Rp) {
  const RunDesc &R = *Rp;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int j = tid; j < R.N; j += nth) R.best[j] = ~0ull;
  for (int i = tid; i < R.n_comb; i += nth) R.amax[i] = 0ull;
  const int nblk = (R.n_comb + kSelThreads - 1) / kSelThreads;
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
