// Reproduction and evaluation kernels.
//
// k_repro fuses, per pair of children (Appendix B of arXiv 2404.01159):
//   mating draw -> SBX (the two B equations and X_cross) -> clip -> polynomial
//   mutation (C, Delta, X_mut) -> clip -> DTLZ evaluation -> ideal point z*.
// A "team" of TS threads (TS a power of two fixed by d alone) owns one pair;
// thread `lane` of the team handles the 8-variable groups lane, lane+TS, ...
// Each group is two 16-byte vector loads per parent and two 16-byte stores
// per child, so a warp moves contiguous 1 KiB spans of each row.
//
// Random numbers (Philox4x32-10, counter = (c0, c1, t, tag), key = seed):
//   PAIR  (p, 0, t)      word 0    : pair gate R3 (crossover iff u24 < p_c)
//   MATE  (e/4, 0, t)    word e%4  : parent draw e -> list[(w*K) >> 32]
//   SBX   (j/4, p, t)    word j%4  : Mc = u24, sign coin bit 0, keep coin bit 1
//   MUTHI (j/8, p, t)    byte j%8 of words 0-1 / 2-3: high 8 bits of R4
//   MUTLO (j, c, t)      word 0>>16: low 16 bits of R4; word 1: M_mut = u24
// The site test R4 < p_m/d, i.e. (hi8<<16 | lo16) < T_m, is decided from hi8
// alone unless hi8 == T_m>>16; only those rare candidates (1 in 256 sites
// for d >= 256) need the MUTLO word, so they are queued in shared memory and
// resolved together before the main pass instead of diverging inside it.
#include "rvea_device.cuh"

namespace rvea {

constexpr int kQueueCap = 512;

__device__ __forceinline__ float clampf(float x, float lo, float hi) {
  return fminf(fmaxf(x, lo), hi);
}

// Deb's bounded polynomial mutation step (Appendix B, Delta), float.
__device__ __noinline__ float poly_mutate(float x, float M, float L, float U, float eta) {
  const float span = U - L;
  const float e1 = eta + 1.0f, inv = 1.0f / e1;
  float delta = 0.0f;
  if (M < 0.5f) {
    const float d1 = (x - L) / span;
    delta = span * (powf(2.0f * M + (1.0f - 2.0f * M) * powf(1.0f - d1, e1), inv) - 1.0f);
  } else if (M > 0.5f) {
    const float d2 = (U - x) / span;
    delta = span * (1.0f - powf(2.0f * (1.0f - M) + 2.0f * (M - 0.5f) * powf(1.0f - d2, e1), inv));
  }
  return clampf(x + delta, L, U);
}

// g-term of one variable.  DTLZ2: (x-1/2)^2.  DTLZ1: (x-1/2)^2 - cos(20 pi (x-1/2))
// + 1, written as y^2 + 2 sin^2(10 pi y) (identical, free of cancellation);
// the k = d-m+1 constant is absorbed by the +1 of each term.
__device__ __forceinline__ float g_term(int problem, float x) {
  const float y = x - 0.5f;
  if (problem == PROB_DTLZ1) {
    const float s = sinpif(10.0f * y);
    return fmaf(2.0f * s, s, y * y);
  }
  return y * y;
}

// Objectives from g and the first m-1 variables (standard DTLZ forms).
__device__ void dtlz_objectives(int problem, int m, float gsum, const float *head, float *f) {
  if (problem == PROB_DTLZ1) {
    const float base = 0.5f * (1.0f + 100.0f * gsum);
    for (int k = 1; k <= m; ++k) {
      float v = base;
      for (int i = 1; i <= m - k; ++i) v *= head[i - 1];
      if (k > 1) v *= 1.0f - head[m - k];
      f[k - 1] = v;
    }
  } else {
    const float base = 1.0f + gsum;
    for (int k = 1; k <= m; ++k) {
      float v = base;
      for (int i = 1; i <= m - k; ++i) v *= cospif(0.5f * head[i - 1]);
      if (k > 1) v *= sinpif(0.5f * head[m - k]);
      f[k - 1] = v;
    }
  }
}

// Sum of `v` over a team of TS threads in a fixed tree that depends on TS
// only (xor butterfly inside a warp, then warp partials in index order).
// Every thread of the CTA must call it.  Valid in the team's first thread.
__device__ __forceinline__ float2 team_sum2(float2 v, int TS, float2 *red) {
  const int lim = TS < 32 ? TS : 32;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (off < lim) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
  }
  if (TS <= 32) return v;
  const int warp = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[warp] = v;
  __syncthreads();
  float2 s = make_float2(0.f, 0.f);
  if ((threadIdx.x & (TS - 1)) == 0) {
    const int w0 = warp, nw = TS >> 5;
    s = red[w0];
    for (int w = 1; w < nw; ++w) { s.x += red[w0 + w].x; s.y += red[w0 + w].y; }
  }
  return s;
}

// Shared-memory layout of one reproduction CTA (bytes), shared with the host
// through repro_smem_bytes().
struct ReproSmem {
  int head_off, bm_off, q_off, total;
};
__host__ __device__ inline ReproSmem repro_smem_layout(int TS, int m, int G) {
  const int ppc = kReproThreads / TS;
  ReproSmem s;
  s.head_off = 0;
  const int head_bytes = ppc * 2 * (m > 1 ? m - 1 : 1) * 4;
  s.bm_off = (head_bytes + 15) & ~15;
  const int bm_bytes = ((ppc * 2 * G) + 3) & ~3;
  s.q_off = (s.bm_off + bm_bytes + 15) & ~15;
  s.total = s.q_off + kQueueCap * 4;
  return s;
}

__device__ __forceinline__ void bm_set(uint32_t *bm, int byte_index, int bit) {
  atomicOr(&bm[byte_index >> 2], 1u << (((byte_index & 3) << 3) + bit));
}
__device__ __forceinline__ uint32_t bm_get(const uint32_t *bm, int byte_index) {
  return (bm[byte_index >> 2] >> ((byte_index & 3) << 3)) & 0xFFu;
}

__global__ void __launch_bounds__(kReproThreads)
k_repro(const __grid_constant__ BatchDir dir) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ int s_par[kReproThreads][2];
  __shared__ int s_chd[kReproThreads][2];
  __shared__ int s_nocross[kReproThreads];
  __shared__ int s_qn;
  __shared__ float2 s_red[kReproThreads / 32];

  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const ReproItem it = static_cast<const ReproItem *>(dir.items[run])[blockIdx.x - dir.prefix[run]];
  const int TS = R.team, ppc = kReproThreads / TS;
  const int team = threadIdx.x / TS, lane = threadIdx.x & (TS - 1);
  const int m = R.m, d = R.d, G = R.G, N = R.N, P = R.P;
  const int p = it.pair0 + team;
  const bool active = p < P;
  const int t = R.ctl->t;
  const uint32_t k0 = R.key0, k1 = R.key1;
  const ReproSmem lay = repro_smem_layout(TS, m, G);
  float *s_head = reinterpret_cast<float *>(dyn + lay.head_off);
  uint32_t *s_bm = reinterpret_cast<uint32_t *>(dyn + lay.bm_off);
  uint32_t *s_q = reinterpret_cast<uint32_t *>(dyn + lay.q_off);
  const int *cslot = R.child_slot + (t & 1) * N;

  // ---- phase 0: mating draws and pair gate, one thread per pair ----------
  if (threadIdx.x < ppc) {
    const int q = it.pair0 + threadIdx.x;
    int a = -1, b = -1, c1 = -1, c2 = -1, nc = 1;
    if (q < P) {
      const uint32_t K = (uint32_t)R.ctl->K;
      const int e[2] = {q, q + P};
      int sl[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 w = philox((uint32_t)(e[h] >> 2), 0u, (uint32_t)t, TAG_MATE, k0, k1);
        const uint32_t idx = __umulhi(word(w, e[h] & 3), K);
        const int j = R.vlist[idx];
        int s = (j >= 0 && j < N) ? R.slotmap[j] : -1;
        if (s < 0 || s >= 2 * N) { set_status(R.ctl, ST_BADINDEX); s = 0; }
        sl[h] = s;
      }
      a = sl[0]; b = sl[1];
      const uint4 g = philox((uint32_t)q, 0u, (uint32_t)t, TAG_PAIR, k0, k1);
      nc = ((g.x >> 8) < R.T_c) ? 0 : 1;
      c1 = cslot[q];
      c2 = (q + P < N) ? cslot[q + P] : -1;
      if (c1 < 0 || c1 >= 2 * N) { set_status(R.ctl, ST_BADINDEX); c1 = 0; }
      if (c2 >= 2 * N) { set_status(R.ctl, ST_BADINDEX); c2 = -1; }
    }
    s_par[threadIdx.x][0] = a; s_par[threadIdx.x][1] = b;
    s_chd[threadIdx.x][0] = c1; s_chd[threadIdx.x][1] = c2;
    s_nocross[threadIdx.x] = nc;
  }
  // clear the mutation bitmaps
  const int bm_words = (ppc * 2 * G + 3) >> 2;
  for (int w = threadIdx.x; w < bm_words; w += kReproThreads) s_bm[w] = 0u;
  if (threadIdx.x == 0) s_qn = 0;
  __syncthreads();

  const int has2 = active ? (s_chd[team][1] >= 0) : 0;
  const uint32_t thr_hi = R.T_m >> 16, thr_lo = R.T_m & 0xFFFFu;

  // ---- phase A: mutation sites from the high byte of R4 ------------------
  if (active && R.T_m > 0) {
    for (int g = lane; g < G; g += TS) {
      const uint4 w = philox((uint32_t)g, (uint32_t)p, (uint32_t)t, TAG_MUTHI, k0, k1);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (s == 1 && !has2) break;
        const uint32_t lo = s ? w.z : w.x, hi = s ? w.w : w.y;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int j = 8 * g + b;
          if (j >= d) break;
          const uint32_t h8 = ((b < 4 ? lo : hi) >> (8 * (b & 3))) & 0xFFu;
          if (h8 < thr_hi) {
            bm_set(s_bm, (team * 2 + s) * G + g, b);
          } else if (h8 == thr_hi) {
            const int qi = atomicAdd(&s_qn, 1);
            if (qi < kQueueCap) {
              s_q[qi] = ((uint32_t)team << 24) | ((uint32_t)s << 23) | (uint32_t)j;
            } else {  // queue full: resolve here
              const int c = s ? p + P : p;
              const uint4 wl = philox((uint32_t)j, (uint32_t)c, (uint32_t)t, TAG_MUTLO, k0, k1);
              if ((wl.x >> 16) < thr_lo) bm_set(s_bm, (team * 2 + s) * G + g, b);
            }
          }
        }
      }
    }
  }
  __syncthreads();
  // ---- phase A2: resolve queued candidates with the low 16 bits ----------
  {
    const int qn = min(s_qn, kQueueCap);
    for (int qi = threadIdx.x; qi < qn; qi += kReproThreads) {
      const uint32_t e = s_q[qi];
      const int tm = (int)(e >> 24), s = (int)((e >> 23) & 1u), j = (int)(e & 0x7FFFFFu);
      const int pq = it.pair0 + tm;
      const int c = s ? pq + P : pq;
      const uint4 wl = philox((uint32_t)j, (uint32_t)c, (uint32_t)t, TAG_MUTLO, k0, k1);
      if ((wl.x >> 16) < thr_lo) bm_set(s_bm, (tm * 2 + s) * G + (j >> 3), j & 7);
    }
  }
  __syncthreads();

  // ---- phase B: SBX, clip, mutation, evaluation, store --------------------
  float2 acc = make_float2(0.f, 0.f);
  const int mh = m - 1;
  float *head = s_head + team * 2 * (mh > 0 ? mh : 1);
  if (active) {
    const float *x1p = R.X + (size_t)s_par[team][0] * R.d_pad;
    const float *x2p = R.X + (size_t)s_par[team][1] * R.d_pad;
    float *y1p = R.X + (size_t)s_chd[team][0] * R.d_pad;
    float *y2p = has2 ? R.X + (size_t)s_chd[team][1] * R.d_pad : nullptr;
    const bool nocross = s_nocross[team] != 0;
    const float L = R.L, U = R.U, ie = R.inv_eta_c1;
    const bool eval = R.problem != PROB_NEURO;
    for (int g = lane; g < G; g += TS) {
      const float4 *a4 = reinterpret_cast<const float4 *>(x1p + 8 * g);
      const float4 *b4 = reinterpret_cast<const float4 *>(x2p + 8 * g);
      const float4 xa0 = __ldg(a4), xa1 = __ldg(a4 + 1);
      const float4 xb0 = __ldg(b4), xb1 = __ldg(b4 + 1);
      const uint4 r0 = philox((uint32_t)(2 * g), (uint32_t)p, (uint32_t)t, TAG_SBX, k0, k1);
      const uint4 r1 = philox((uint32_t)(2 * g + 1), (uint32_t)p, (uint32_t)t, TAG_SBX, k0, k1);
      const float x1v[8] = {xa0.x, xa0.y, xa0.z, xa0.w, xa1.x, xa1.y, xa1.z, xa1.w};
      const float x2v[8] = {xb0.x, xb0.y, xb0.z, xb0.w, xb1.x, xb1.y, xb1.z, xb1.w};
      const uint32_t wv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
      float c1[8], c2[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const uint32_t w = wv[v];
        const float Mc = u24f(w);
        const bool lowb = Mc < 0.5f;
        const float base = lowb ? 2.0f * Mc : 2.0f - 2.0f * Mc;
        const float beta = exp2f((lowb ? ie : -ie) * __log2f(base));
        float B = (w & 1u) ? beta : -beta;
        if ((w & 2u) || nocross) B = 1.0f;
        const float x1 = x1v[v], x2 = x2v[v];
        c1[v] = clampf(0.5f * ((1.0f + B) * x1 + (1.0f - B) * x2), L, U);
        c2[v] = clampf(0.5f * ((1.0f - B) * x1 + (1.0f + B) * x2), L, U);
      }
      const uint32_t mb1 = bm_get(s_bm, (team * 2 + 0) * G + g);
      const uint32_t mb2 = has2 ? bm_get(s_bm, (team * 2 + 1) * G + g) : 0u;
      if (mb1 | mb2) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          if (mb1 & (1u << v)) {
            const uint4 wl = philox((uint32_t)(8 * g + v), (uint32_t)p, (uint32_t)t, TAG_MUTLO, k0, k1);
            c1[v] = poly_mutate(c1[v], u24f(wl.y), L, U, R.eta_m);
          }
          if (mb2 & (1u << v)) {
            const uint4 wl = philox((uint32_t)(8 * g + v), (uint32_t)(p + P), (uint32_t)t, TAG_MUTLO, k0, k1);
            c2[v] = poly_mutate(c2[v], u24f(wl.y), L, U, R.eta_m);
          }
        }
      }
      if (eval) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const int j = 8 * g + v;
          if (j < d) {
            if (j >= mh) {
              acc.x += g_term(R.problem, c1[v]);
              acc.y += g_term(R.problem, c2[v]);
            } else {
              head[j] = c1[v];
              head[mh + j] = c2[v];
            }
          }
        }
      }
      float4 *o1 = reinterpret_cast<float4 *>(y1p + 8 * g);
      o1[0] = make_float4(c1[0], c1[1], c1[2], c1[3]);
      o1[1] = make_float4(c1[4], c1[5], c1[6], c1[7]);
      if (y2p) {
        float4 *o2 = reinterpret_cast<float4 *>(y2p + 8 * g);
        o2[0] = make_float4(c2[0], c2[1], c2[2], c2[3]);
        o2[1] = make_float4(c2[4], c2[5], c2[6], c2[7]);
      }
    }
  }
  if (R.problem == PROB_NEURO) return;   // objectives come from the rollout kernel
  const float2 gs = team_sum2(acc, TS, s_red);
  __syncthreads();   // head[] written by other lanes of the team
  if (active && lane == 0) {
    float f[kMaxM];
    const int n2 = 2 * N;
    dtlz_objectives(R.problem, m, gs.x, head, f);
    const int s1 = s_chd[team][0];
    for (int k = 0; k < m; ++k) {
      R.F[(size_t)k * n2 + s1] = f[k];
      atomicMin(&R.ctl->zkey[k], f2ord(f[k]));
    }
    if (has2) {
      dtlz_objectives(R.problem, m, gs.y, head + mh, f);
      const int s2 = s_chd[team][1];
      for (int k = 0; k < m; ++k) {
        R.F[(size_t)k * n2 + s2] = f[k];
        atomicMin(&R.ctl->zkey[k], f2ord(f[k]));
      }
    }
  }
}

// Initial population (Algorithm 2, initialisation), slots 0..N-1, and its
// objectives.  DTLZ: x = L + (U-L) u24 from INIT (j/4, i, 0) word j%4.
// Rollout problem: x = clip(0.1 z), z Box-Muller from INIT (j, i, 0).
__global__ void __launch_bounds__(kReproThreads)
k_init(const __grid_constant__ BatchDir dir) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ float2 s_red[kReproThreads / 32];
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const ReproItem it = static_cast<const ReproItem *>(dir.items[run])[blockIdx.x - dir.prefix[run]];
  const int TS = R.team;
  const int team = threadIdx.x / TS, lane = threadIdx.x & (TS - 1);
  const int m = R.m, d = R.d, G = R.G, N = R.N;
  const int i = it.pair0 + team;   // one team per individual
  const bool active = i < N;
  const uint32_t k0 = R.key0, k1 = R.key1;
  const int mh = m - 1;
  float *head = reinterpret_cast<float *>(dyn) + team * (mh > 0 ? mh : 1);
  float2 acc = make_float2(0.f, 0.f);
  if (active) {
    float *y = R.X + (size_t)i * R.d_pad;
    for (int g = lane; g < G; g += TS) {
      float x[8];
      if (R.problem == PROB_NEURO) {
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const uint4 w = philox((uint32_t)(8 * g + v), (uint32_t)i, 0u, TAG_INIT, k0, k1);
          const float u1 = 1.0f - u24f(w.x), u2 = u24f(w.y);
          const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
          x[v] = clampf(0.1f * z, R.L, R.U);
        }
      } else {
        const uint4 r0 = philox((uint32_t)(2 * g), (uint32_t)i, 0u, TAG_INIT, k0, k1);
        const uint4 r1 = philox((uint32_t)(2 * g + 1), (uint32_t)i, 0u, TAG_INIT, k0, k1);
        const uint32_t wv[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
        for (int v = 0; v < 8; ++v) x[v] = R.L + (R.U - R.L) * u24f(wv[v]);
      }
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const int j = 8 * g + v;
        if (j >= d) x[v] = 0.0f;   // zero padding
        else if (R.problem != PROB_NEURO) {
          if (j >= mh) acc.x += g_term(R.problem, x[v]);
          else head[j] = x[v];
        }
      }
      float4 *o = reinterpret_cast<float4 *>(y + 8 * g);
      o[0] = make_float4(x[0], x[1], x[2], x[3]);
      o[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
  }
  if (R.problem == PROB_NEURO) return;
  const float2 gs = team_sum2(acc, TS, s_red);
  __syncthreads();
  if (active && lane == 0) {
    float f[kMaxM];
    dtlz_objectives(R.problem, m, gs.x, head, f);
    for (int k = 0; k < m; ++k) {
      R.F[(size_t)k * 2 * N + i] = f[k];
      atomicMin(&R.ctl->zkey[k], f2ord(f[k]));
    }
  }
}

int repro_smem_total(int TS, int m, int G) { return repro_smem_layout(TS, m, G).total; }

}  // namespace rvea
