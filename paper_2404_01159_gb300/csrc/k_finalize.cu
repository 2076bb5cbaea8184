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
#include "rvea_device.cuh"

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

__global__ void __launch_bounds__(kFinThreads)
k_finalize(const __grid_constant__ BatchDir dir) {
  extern __shared__ __align__(16) int s_map[];     // [N] new slot map, then [2N] bytes occ
  __shared__ int s_warp[32];
  __shared__ unsigned s_zmin[kMaxM], s_zmax[kMaxM];
  __shared__ int s_total;
  const RunDesc &R = *dir.desc[blockIdx.x];
  const int N = R.N, n2 = 2 * N, m = R.m;
  const int t = R.ctl->t;
  const int *cur = R.child_slot + (t & 1) * N;
  int *nxt = R.child_slot + ((t + 1) & 1) * N;
  uint8_t *occ = reinterpret_cast<uint8_t *>(s_map + N);
  const int tid = threadIdx.x;

  for (int w = tid; w < (n2 + 3) / 4; w += kFinThreads) reinterpret_cast<int *>(occ)[w] = 0;
  if (tid < kMaxM) { s_zmin[tid] = 0xFFFFFFFFu; s_zmax[tid] = 0u; }
  __syncthreads();
  for (int j = tid; j < N; j += kFinThreads) {
    const unsigned long long key = R.best[j];
    R.best[j] = ~0ull;
    int s = -1, i = -1;
    if (key != ~0ull) {
      i = (int)(uint32_t)(key & 0xFFFFFFFFull);
      if (i >= 0 && i < N) s = R.slotmap[i];
      else if (i >= N && i < n2) s = cur[i - N];
      if (s < 0 || s >= n2) { set_status(R.ctl, ST_BADINDEX); s = -1; i = -1; }
      else occ[s] = 1;
    }
    s_map[j] = s;
    R.surv[j] = i;
  }
  __syncthreads();

  // new slot map and ascending valid list
  const int ch = (N + kFinThreads - 1) / kFinThreads;
  const int a0 = min(N, tid * ch), a1 = min(N, a0 + ch);
  int cnt = 0;
  for (int j = a0; j < a1; ++j) cnt += (s_map[j] >= 0);
  int pos = block_exclusive_scan(cnt, s_warp, &s_total);
  const int K = s_total;
  for (int j = a0; j < a1; ++j) {
    const int s = s_map[j];
    R.slotmap[j] = s;
    if (s >= 0) {
      R.vlist[pos++] = j;
      for (int k = 0; k < m; ++k) {
        const unsigned o = f2ord(R.F[(size_t)k * n2 + s]);
        atomicMin(&s_zmin[k], o);
        atomicMax(&s_zmax[k], o);
      }
    }
  }
  // free rows, ascending, first N of them
  const int ch2 = (n2 + kFinThreads - 1) / kFinThreads;
  const int b0 = min(n2, tid * ch2), b1 = min(n2, b0 + ch2);
  int fc = 0;
  for (int s = b0; s < b1; ++s) fc += (occ[s] == 0);
  int fpos = block_exclusive_scan(fc, s_warp, &s_total);
  for (int s = b0; s < b1 && fpos < N; ++s)
    if (occ[s] == 0) nxt[fpos++] = s;
  __syncthreads();

  if (tid < m) R.ctl->zkey[tid] = s_zmin[tid];
  const bool adapt = (t % R.p_adapt) == 0;
  if (adapt && K > 0) {
    // range_k = max - min over the survivors, floored at 1e-12, in FP64
    __shared__ double s_rng[kMaxM];
    if (tid < m) {
      const double hi = (double)ord2f(s_zmax[tid]), lo = (double)ord2f(s_zmin[tid]);
      const double r = hi - lo;
      s_rng[tid] = r < 1e-12 ? 1e-12 : r;
    }
    __syncthreads();
    for (int j = tid; j < N; j += kFinThreads) {
      const double *v0 = R.V0 + (size_t)j * m;
      double w[kMaxM];
      double s2 = 0.0;
      for (int k = 0; k < m; ++k) {
        w[k] = v0[k] * s_rng[k];
        s2 += w[k] * w[k];
      }
      const double nrm = sqrt(s2);
      float *v32 = R.V32 + (size_t)j * R.m4 * 4;
      for (int k = 0; k < m; ++k) {
        const double v = w[k] / nrm;
        R.V64[(size_t)j * m + k] = v;
        v32[k] = (float)v;
      }
    }
  }
  if (tid == 0) {
    R.ctl->K = K;
    R.ctl->adapted = adapt ? 1 : 0;
    R.ctl->t = t + 1;
  }
}

// gamma_j = min_{i != j} angle(v_i, v_j) (Eq. 5), FP64.  arccos is
// decreasing, so gamma_j = acos(max_{i != j} v_i.v_j) for unit rows.  A float
// pass finds max32; only the i whose float dot is within 1e-5 of it (the
// float error of a dot of unit vectors is below 1e-6) are re-evaluated in
// FP64, so the FP64 maximum is exact.  One block = 32 vectors x 8 slices of i.
__device__ void gamma_block(const RunDesc &R, int jb) {
  const int N = R.N, m = R.m;
  const int jl = threadIdx.x >> 3, sl = threadIdx.x & 7;
  const int j = jb * 32 + jl;
  const bool act = j < N;
  const int per = (N + 7) / 8;
  const int i0 = sl * per, i1 = min(N, i0 + per);
  double vj[kMaxM];
  float vj32[kMaxM];
  for (int k = 0; k < kMaxM; ++k) { vj[k] = 0.0; vj32[k] = 0.f; }
  if (act)
    for (int k = 0; k < m; ++k) { vj[k] = R.V64[(size_t)j * m + k]; vj32[k] = (float)vj[k]; }
  float mx = -INFINITY;
  if (act) {
    for (int i = i0; i < i1; ++i) {
      if (i == j) continue;
      const double *vi = R.V64 + (size_t)i * m;
      float d = (float)vi[0] * vj32[0];
      for (int k = 1; k < m; ++k) d = fmaf((float)vi[k], vj32[k], d);
      mx = fmaxf(mx, d);
    }
  }
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const float thr = mx - 1e-5f;
  double best = -2.0;
  if (act) {
    for (int i = i0; i < i1; ++i) {
      if (i == j) continue;
      const double *vi = R.V64 + (size_t)i * m;
      float d = (float)vi[0] * vj32[0];
      for (int k = 1; k < m; ++k) d = fmaf((float)vi[k], vj32[k], d);
      if (d >= thr) {
        double e = 0.0;
        for (int k = 0; k < m; ++k) e += vi[k] * vj[k];
        best = fmax(best, e);
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

// Persistent over the directory: every run with ctl->adapted set (or every
// run when `force`) has its vector blocks of 32 spread over the grid.
__global__ void __launch_bounds__(256)
k_gamma(const __grid_constant__ BatchDir dir, int force) {
  for (int r = 0; r < dir.n; ++r) {
    const RunDesc &R = *dir.desc[r];
    if (!force && R.ctl->adapted == 0) continue;
    const int nb = (R.N + 31) / 32;
    for (int jb = blockIdx.x; jb < nb; jb += gridDim.x) gamma_block(R, jb);
  }
}

// rvea_gamma: one caller-supplied set of vectors, descriptor by value.
__global__ void __launch_bounds__(256) k_gamma_op(const __grid_constant__ RunDesc D) {
  gamma_block(D, blockIdx.x);
}

// ---- state transfer -------------------------------------------------------
// Population rows in slot order -> dst (N x d); invalid rows NaN.
__global__ void k_gather_pop(const RunDesc *__restrict__ Rp, float *dst, uint8_t *valid) {
  const RunDesc &R = *Rp;
  const int j = blockIdx.x;
  const int s = R.slotmap[j];
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
  const int s = R.slotmap[j];
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
    R.slotmap[j] = v ? j : -1;
    for (int k = 0; k < m; ++k) {
      const float f = Fin[(size_t)j * m + k];
      R.F[(size_t)k * n2 + j] = f;
      if (v) atomicMin(&s_z[k], f2ord(f));
    }
    float *v32 = R.V32 + (size_t)j * R.m4 * 4;
    for (int k = 0; k < R.m4 * 4; ++k) v32[k] = k < m ? (float)R.V64[(size_t)j * m + k] : 0.0f;
    R.gamma32[j] = (float)R.gamma64[j];
    R.best[j] = ~0ull;
    R.surv[j] = -1;
  }
  for (int i = tid; i < n2; i += kFinThreads) { R.amax[i] = 0ull; R.assoc[i] = -1; }
  for (int b = tid; b < (n2 + kSelThreads - 1) / kSelThreads; b += kFinThreads) R.blk_cnt[b] = 0;
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
  }
}

// Initial slot map and lists after k_init: slot j = row j, children go to
// rows N..2N-1.
__global__ void k_init_lists(const __grid_constant__ BatchDir dir) {
  const RunDesc &R = *dir.desc[blockIdx.y];
  const int N = R.N;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) {
    R.slotmap[j] = j;
    R.vlist[j] = j;
    R.child_slot[1 * N + j] = N + j;   // t = 1 uses buffer (1 & 1)
    R.child_slot[j] = N + j;
    R.best[j] = ~0ull;
    R.surv[j] = -1;
  }
  for (int i = j; i < 2 * N; i += gridDim.x * blockDim.x) { R.amax[i] = 0ull; R.assoc[i] = -1; }
  if (j < (2 * N + kSelThreads - 1) / kSelThreads) R.blk_cnt[j] = 0;
  if (j == 0) {
    R.ctl->t = 1;
    R.ctl->K = N;
    R.ctl->status = 0;
    R.ctl->adapted = 0;
  }
}

}  // namespace rvea
