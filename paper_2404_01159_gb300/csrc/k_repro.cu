// Reproduction and evaluation kernels.
//
// k_repro fuses, per pair of children (Appendix B of arXiv 2404.01159):
//   mating draw -> SBX (the two B equations and X_cross) -> clip -> polynomial
//   mutation (C, Delta, X_mut) -> clip -> DTLZ evaluation -> ideal point z*.
//
// Work decomposition.  A team of TS lanes (TS a power of two <= 32, fixed by d
// alone) owns one work unit: one segment of kLaneGroups*TS consecutive
// 8-variable groups of one pair; lane l handles groups l, l+TS, l+2TS, ...
// of the segment.  Each group is two 16-byte loads per parent and two 16-byte stores
// per child, so a warp moves contiguous 512-byte spans.  Teams never wait on
// other warps: the phases below synchronise with __syncwarp only.  A pair
// with several segments (d > 2048) combines the segments' partial sums of g
// in the last segment to finish (an arrival counter per pair, no spinning),
// always in segment order, so the reduction tree depends on d alone.
//
// Arithmetic on adjacent variables runs in packed .f32x2 instructions (the
// children of SBX and the evaluation): same IEEE operations, half the issue
// slots.  g is accumulated per lane as (even variables, odd variables).
//
// Random numbers (Philox4x32-10, counter = (c0, c1, t, tag), key = seed):
//   PAIR  (p, 0, t)      word 0    : pair gate R3 (crossover iff u24 < p_c)
//   MATE  (e/4, 0, t)    word e%4  : parent draw e -> list[(w*K) >> 32]
//   SBX   (j/4, p, t)    word j%4  : Mc = u24, sign coin bit 0, keep coin bit 1
//   MUTSITE (i/4, c, t)  word i%4  : draw i of the mutation sites of child c
//   MUTMAG  (j, c, t)    word 1    : M_mut = u24 of site j of child c
// Mutation sites: Appendix B fires each site independently with probability
// q = p_m/d (on the 24-bit grid).  The same law is drawn per child row as a
// count k ~ Binomial(d, q) (draw 0 against the host's 32-bit CDF thresholds)
// and a uniform k-subset (Floyd's sampler, draws 1..k, r = (w (J+1)) >> 32),
// so a row costs one or two Philox calls instead of one draw per site.  One
// lane per child builds the list and marks the sites of its team's segment
// in a shared-memory bitmap before the main pass.
#include "rvea_device.cuh"

namespace rvea {

constexpr int kBmWords = kLaneGroups * 16;    // per warp: 32 lanes x kLaneGroups x 16 bits

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

// Taylor coefficients of sin(pi r), through r^13 (|r| <= 1/2: the first
// omitted term is below 7e-10).
constexpr double kPI = 3.14159265358979323846;
constexpr float kS1 = (float)kPI;
constexpr float kS3 = (float)(-kPI * kPI * kPI / 6.0);
constexpr float kS5 = (float)(kPI * kPI * kPI * kPI * kPI / 120.0);
constexpr float kS7 = (float)(-kPI * kPI * kPI * kPI * kPI * kPI * kPI / 5040.0);
constexpr float kS9 = (float)(kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI / 362880.0);
constexpr float kS11 =
    (float)(-kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI / 39916800.0);
constexpr float kS13 = (float)(kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI * kPI *
                               kPI * kPI / 6227020800.0);

// g-terms of two adjacent variables x = (x_j, x_j+1), added into acc.
// DTLZ2: (x-1/2)^2.  DTLZ1: (x-1/2)^2 - cos(20 pi (x-1/2)) + 1 = y^2 + 2 sin^2(10 pi y)
// (identical, free of cancellation; the k = d-m+1 constant is the +1 of each
// term).  sin^2 has period 1 in 10y: 10y is reduced by its nearest integer
// first (one fma, one rounding), then sin(pi r) from its Taylor series.
__device__ __forceinline__ float2 g_terms2(int problem, float2 x, float2 acc) {
  const float2 y = add2(x, splat2(-0.5f));
  acc = fma2(y, y, acc);
  if (problem == PROB_DTLZ1) {
    const float2 z = mul2(y, splat2(10.0f));
    const float2 nn = make_float2(rintf(-z.x), rintf(-z.y));
    const float2 r = fma2(splat2(10.0f), y, nn);
    const float2 r2 = mul2(r, r);
    float2 p = fma2(r2, splat2(kS13), splat2(kS11));
    p = fma2(r2, p, splat2(kS9));
    p = fma2(r2, p, splat2(kS7));
    p = fma2(r2, p, splat2(kS5));
    p = fma2(r2, p, splat2(kS3));
    p = fma2(r2, p, splat2(kS1));
    const float2 s = mul2(r, p);
    acc = fma2(add2(s, s), s, acc);
  }
  return acc;
}

// Scalar form of the same terms (bit-identical per element), used where a
// group holds x_1..x_{m-1} or the ragged end of the row.
__device__ __forceinline__ float g_term1(int problem, float x, float acc) {
  const float y = x + (-0.5f);
  acc = fmaf(y, y, acc);
  if (problem == PROB_DTLZ1) {
    const float z = y * 10.0f;
    const float r = fmaf(10.0f, y, rintf(-z));
    const float r2 = r * r;
    float p = fmaf(r2, kS13, kS11);
    p = fmaf(r2, p, kS9);
    p = fmaf(r2, p, kS7);
    p = fmaf(r2, p, kS5);
    p = fmaf(r2, p, kS3);
    p = fmaf(r2, p, kS1);
    const float s = r * p;
    acc = fmaf(s + s, s, acc);
  }
  return acc;
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

// Sum over a team of TS <= 32 lanes: xor butterfly (every lane of the team
// ends with the same bits).  All 32 lanes of the warp must call it.
__device__ __forceinline__ float2 team_sum2(float2 v, int TS) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (off < TS) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
  }
  return v;
}

// Mutation sites of child row c (count, then Floyd's uniform subset), marked
// in the team's bitmap where they fall in groups [g0, g0 + SG) (16-bit entry
// gl: bits 0-7 child 1, bits 8-15 child 2).
template <class KP>
__device__ __noinline__ void mark_sites(const RunDesc &R, const KP &kp, int c, int s2, int t,
                                        int g0, int SG, uint32_t *bmw, int ebase) {
  const int d = R.d;
  uint4 w = philox_k(0u, (uint32_t)c, (uint32_t)t, TAG_MUTSITE, kp);
  const int nthr = R.n_mthr;
  int k = 0;
  while (k < nthr && w.x >= R.mthr[k]) ++k;
  int sites[kMaxSites];
  for (int i = 0; i < k; ++i) {
    const int e = i + 1;
    if ((e & 3) == 0) w = philox_k((uint32_t)(e >> 2), (uint32_t)c, (uint32_t)t, TAG_MUTSITE, kp);
    const uint32_t J = (uint32_t)(d - k + i);
    uint32_t r = __umulhi(word(w, e & 3), J + 1u);
    for (int l = 0; l < i; ++l)
      if ((uint32_t)sites[l] == r) { r = J; break; }
    sites[i] = (int)r;
    const int gl = (int)(r >> 3) - g0;
    if (gl >= 0 && gl < SG) {
      const int hw = ebase + gl;
      atomicOr(&bmw[hw >> 1], 1u << (((hw & 1) << 4) + (s2 << 3) + (r & 7)));
    }
  }
}

// 2^x with one MUFU.EX2 (PTX ex2.approx, relative error ~2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// SBX spread factor of one variable: word q carries Mc (top 24 bits), the
// sign coin (bit 0) and the keep coin (bit 1); keep or no crossover -> 1.
__device__ __forceinline__ float sbx_B(uint32_t q, bool nocross, float ie) {
  const float Mc = u24f(q);
  const bool lowb = Mc < 0.5f;
  const float base = lowb ? 2.0f * Mc : 2.0f - 2.0f * Mc;
  const float beta = ex2_approx((lowb ? ie : -ie) * __log2f(base));
  const float B = (q & 1u) ? beta : -beta;
  return ((q & 2u) || nocross) ? 1.0f : B;
}

// Children of two adjacent variables: c1 = ((1+B) x1 + (1-B) x2) / 2,
// c2 = ((1-B) x1 + (1+B) x2) / 2, clipped to [L, U].
__device__ __forceinline__ void sbx_pair(float2 x1, float2 x2, float2 B, float L, float U,
                                         float2 &c1, float2 &c2) {
  const float2 P = add2(splat2(1.0f), B), Q = sub2(splat2(1.0f), B);
  c1 = mul2(splat2(0.5f), fma2(P, x1, mul2(Q, x2)));
  c2 = mul2(splat2(0.5f), fma2(Q, x1, mul2(P, x2)));
  c1 = make_float2(clampf(c1.x, L, U), clampf(c1.y, L, U));
  c2 = make_float2(clampf(c2.x, L, U), clampf(c2.y, L, U));
}

// Four adjacent variables of both children: (a0, a1) child 1, (b0, b1) child 2.
struct Quad { float2 a0, a1, b0, b1; };

// Polynomial mutation of the marked variables of a quad (bits of h1 / h2 for
// children c1 / c2; first variable j0).  Rare (about one site per row), so
// kept out of the main loop's instruction stream.
template <class KP>
__device__ __noinline__ Quad mutate_quad(Quad q, uint32_t h1, uint32_t h2, int j0, int c1, int c2,
                                         int t, float L, float U, float eta_m, const KP &kp) {
  float x[8] = {q.a0.x, q.a0.y, q.a1.x, q.a1.y, q.b0.x, q.b0.y, q.b1.x, q.b1.y};
  const uint32_t bits = h1 | (h2 << 4);
#pragma unroll 1
  for (int b = 0; b < 8; ++b) {
    if (!(bits & (1u << b))) continue;
    const int v = b & 3, c = b < 4 ? c1 : c2;
    const uint4 w = philox_k((uint32_t)(j0 + v), (uint32_t)c, (uint32_t)t, TAG_MUTMAG, kp);
    x[b] = poly_mutate(x[b], u24f(w.y), L, U, eta_m);
  }
  return Quad{make_float2(x[0], x[1]), make_float2(x[2], x[3]), make_float2(x[4], x[5]),
              make_float2(x[6], x[7])};
}

// Evaluation terms of a quad that holds x_1..x_{m-1} (kept in hb for the
// objectives) or the ragged end of the row; returns the accumulators
// (child 1 in a0, child 2 in a1), given in acc.a0 / acc.a1.
template <int PROB>
__device__ __noinline__ Quad eval_edge(Quad q, Quad acc, int j0, int mh, int d, float *hb) {
  const float c1[4] = {q.a0.x, q.a0.y, q.a1.x, q.a1.y}, c2[4] = {q.b0.x, q.b0.y, q.b1.x, q.b1.y};
  float2 acc1 = acc.a0, acc2 = acc.a1;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int j = j0 + v;
    if (j < mh) {
      hb[j] = c1[v];
      hb[kMaxM + j] = c2[v];
    } else if (j < d) {
      if (v & 1) {
        acc1.y = g_term1(PROB, c1[v], acc1.y);
        acc2.y = g_term1(PROB, c2[v], acc2.y);
      } else {
        acc1.x = g_term1(PROB, c1[v], acc1.x);
        acc2.x = g_term1(PROB, c2[v], acc2.x);
      }
    }
  }
  return Quad{acc1, acc2, acc1, acc2};
}

// Last segment of pair p to arrive: g of both children from the segments'
// partial sums in segment order, then the objectives and the ideal point.
__device__ __noinline__ void finish_pair(const RunDesc &R, int p, int S, int ch1, int ch2) {
  __threadfence();
  const float *ps = R.psum + (size_t)p * 2 * S;
  const float *hb = R.hbuf + (size_t)p * 2 * kMaxM;
  const int m = R.m, mh = m - 1, n2 = 2 * R.N;
  float g1 = 0.f, g2 = 0.f;
  for (int sg = 0; sg < S; ++sg) {
    g1 += __ldcg(ps + sg);
    g2 += __ldcg(ps + S + sg);
  }
  float head[kMaxM], f[kMaxM];
  for (int j = 0; j < mh; ++j) head[j] = __ldcg(hb + j);
  dtlz_objectives(R.problem, m, g1, head, f);
  for (int kk = 0; kk < m; ++kk) {
    R.F[(size_t)kk * n2 + ch1] = f[kk];
    atomicMin(&R.ctl->zkey[kk], f2ord(f[kk]));
  }
  if (ch2 >= 0) {
    for (int j = 0; j < mh; ++j) head[j] = __ldcg(hb + kMaxM + j);
    dtlz_objectives(R.problem, m, g2, head, f);
    for (int kk = 0; kk < m; ++kk) {
      R.F[(size_t)kk * n2 + ch2] = f[kk];
      atomicMin(&R.ctl->zkey[kk], f2ord(f[kk]));
    }
  }
  R.pcnt[p] = 0;
}

template <int PROB, class KP>
__device__ __forceinline__ void repro_body(const BatchDir &dir, const KP &kp) {
  __shared__ uint32_t s_w[kReproThreads / 32][kBmWords];

  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const ReproItem it = static_cast<const ReproItem *>(dir.items[run])[blockIdx.x - dir.prefix[run]];
  const int TS = R.team, tpw = 32 / TS, S = R.nseg, SG = TS * kLaneGroups;
  const int m = R.m, d = R.d, G = R.G, N = R.N, P = R.P;
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  const int tw = wl / TS, lane = wl & (TS - 1), tbase = tw * TS;
  const int unit = it.pair0 + warp * tpw + tw;
  const int p = unit / S, seg = unit - p * S;
  const bool active = p < P;
  const int t = R.ctl->t;
  const int *cslot = R.child_slot + (t & 1) * N;
  uint32_t *bmw = s_w[warp];
  uint16_t *bm = reinterpret_cast<uint16_t *>(bmw) + tw * SG;   // [SG] of this team: c1 | c2 << 8

#pragma unroll
  for (int w = 0; w < kBmWords; w += 32) bmw[w + wl] = 0u;

  // ---- phase 0: the pair's two mating draws and crossover gate ------------
  uint32_t v0 = 0, v1 = 0, v2 = 0;
  if (active) {
    for (int c = lane; c < 3; c += TS) {
      if (c < 2) {
        const int e = c == 0 ? p : p + P;
        const uint4 w = philox_k((uint32_t)(e >> 2), 0u, (uint32_t)t, TAG_MATE, kp);
        const uint32_t idx = __umulhi(word(w, e & 3), (uint32_t)R.ctl->K);
        const int j = R.vlist[idx];
        int sl = (j >= 0 && j < N) ? R.slotmap[(t & 1) * N + j] : -1;
        if (sl < 0 || sl >= 2 * N) { set_status(R.ctl, ST_BADINDEX); sl = 0; }
        if (c == 0) v0 = (uint32_t)sl; else v1 = (uint32_t)sl;
      } else {
        const uint4 g = philox_k((uint32_t)p, 0u, (uint32_t)t, TAG_PAIR, kp);
        v2 = ((g.x >> 8) < R.T_c) ? 0u : 1u;
      }
    }
  }
  const int par1 = (int)__shfl_sync(0xffffffffu, v0, tbase);
  const int par2 = (int)__shfl_sync(0xffffffffu, v1, tbase + (1 & (TS - 1)));
  const bool nocross = __shfl_sync(0xffffffffu, v2, tbase + (2 & (TS - 1))) != 0u;
  int ch1 = -1, ch2 = -1;
  if (active) {
    ch1 = cslot[p];
    ch2 = (p + P < N) ? cslot[p + P] : -1;
    if (ch1 < 0 || ch1 >= 2 * N) { set_status(R.ctl, ST_BADINDEX); ch1 = 0; }
    if (ch2 >= 2 * N) { set_status(R.ctl, ST_BADINDEX); ch2 = -1; }
  }
  const bool has2 = ch2 >= 0;
  const int g0 = seg * SG;
  // run constants used inside the loops, in registers: the child-row stores
  // could alias the descriptor, which would force a reload after each store
  float4 *const X4 = reinterpret_cast<float4 *>(R.X);
  const uint32_t rq = (uint32_t)R.d_pad >> 2;      // float4s per row
  const uint32_t o1 = (uint32_t)par1 * rq, o2 = (uint32_t)par2 * rq;
  const uint32_t T_m = R.T_m;
  const float L = R.L, U = R.U, ie = R.inv_eta_c1, eta_m = R.eta_m;
  float *const hb = R.hbuf + (size_t)p * 2 * kMaxM;
  __syncwarp();

  // ---- phase A: mutation sites of this segment ----------------------------
  if (active && T_m > 0) {
    if (T_m >= (1u << 24)) {   // every site
#pragma unroll 1
      for (int k = 0; k < kLaneGroups; ++k) {
        const int gl = lane + k * TS, g = g0 + gl;
        if (g >= G) break;
        const uint32_t vmask = 8 * g + 8 <= d ? 0xFFu : (1u << (d - 8 * g)) - 1u;
        bm[gl] = (uint16_t)(vmask | (has2 ? vmask << 8 : 0u));
      }
    } else {
      for (int c = lane; c < 2; c += TS)
        if (c == 0 || has2) mark_sites(R, kp, c ? p + P : p, c, t, g0, SG, bmw, tw * SG);
    }
  }
  __syncwarp();

  // ---- phase B: SBX, clip, mutation, evaluation, store --------------------
  float2 acc1 = make_float2(0.f, 0.f), acc2 = make_float2(0.f, 0.f);
  const bool eval = PROB != PROB_NEURO;
  const int mh = m - 1;
  if (active) {
    float4 *const Y4 = X4;
    const uint32_t q1 = (uint32_t)ch1 * rq, q2 = has2 ? (uint32_t)ch2 * rq : 0u;
#pragma unroll 1
    for (int k = 0; k < kLaneGroups; ++k) {
      const int gl = lane + k * TS, g = g0 + gl;
      if (g >= G) break;
      const uint32_t mb = bm[gl];
      const bool plain = 8 * g >= mh && 8 * g + 8 <= d;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 xa = __ldg(X4 + o1 + 2 * g + h), xb = __ldg(X4 + o2 + 2 * g + h);
        const uint4 r = philox_k((uint32_t)(2 * g + h), (uint32_t)p, (uint32_t)t, TAG_SBX, kp);
        float2 a0, a1, b0, b1;   // children 1 and 2, variables (0,1) and (2,3)
        sbx_pair(make_float2(xa.x, xa.y), make_float2(xb.x, xb.y),
                 make_float2(sbx_B(r.x, nocross, ie), sbx_B(r.y, nocross, ie)), L, U, a0, b0);
        sbx_pair(make_float2(xa.z, xa.w), make_float2(xb.z, xb.w),
                 make_float2(sbx_B(r.z, nocross, ie), sbx_B(r.w, nocross, ie)), L, U, a1, b1);
        const uint32_t h1 = (mb >> (4 * h)) & 0xFu, h2 = has2 ? (mb >> (8 + 4 * h)) & 0xFu : 0u;
        if (h1 | h2) {
          const Quad o = mutate_quad(Quad{a0, a1, b0, b1}, h1, h2, 8 * g + 4 * h, p, p + P, t, L, U,
                                     eta_m, kp);
          a0 = o.a0; a1 = o.a1; b0 = o.b0; b1 = o.b1;
        }
        if (eval) {
          if (plain) {
            acc1 = g_terms2(PROB, a0, acc1);
            acc1 = g_terms2(PROB, a1, acc1);
            acc2 = g_terms2(PROB, b0, acc2);
            acc2 = g_terms2(PROB, b1, acc2);
          } else {   // a group holding x_1..x_{m-1} or the ragged end of the row
            const Quad o = eval_edge<PROB>(Quad{a0, a1, b0, b1}, Quad{acc1, acc2, acc1, acc2},
                                           8 * g + 4 * h, mh, d, hb);
            acc1 = o.a0;
            acc2 = o.a1;
          }
        }
        Y4[q1 + 2 * g + h] = make_float4(a0.x, a0.y, a1.x, a1.y);
        if (has2) Y4[q2 + 2 * g + h] = make_float4(b0.x, b0.y, b1.x, b1.y);
      }
    }
  }
  if (!eval) return;   // objectives come from the rollout kernel

  // ---- combine: team sum, then segments in order, then objectives ---------
  const float2 gs = team_sum2(make_float2(acc1.x + acc1.y, acc2.x + acc2.y), TS);
  if (active && lane == 0) {
    float *ps = R.psum + (size_t)p * 2 * S;
    ps[seg] = gs.x;
    ps[S + seg] = gs.y;
  }
  // the warp barrier orders the team's writes (child rows, head values,
  // partials) before the leader's cumulative fence and its arrival
  __syncwarp();
  if (active && lane == 0) {
    __threadfence();
    const int prev = atomicAdd(&R.pcnt[p], 1);
    if (prev == S - 1) finish_pair(R, p, S, ch1, ch2);
  }
}

template <class KP>
__device__ __forceinline__ void repro_dispatch(const BatchDir &dir, const KP &kp) {
  const int run = dir_find(dir, blockIdx.x);
  switch (dir.desc[run]->problem) {
    case PROB_DTLZ1: repro_body<PROB_DTLZ1>(dir, kp); return;
    case PROB_DTLZ2: repro_body<PROB_DTLZ2>(dir, kp); return;
    default: repro_body<PROB_NEURO>(dir, kp); return;
  }
}

// One run of a known problem: the Philox round keys come in the parameter
// block.
__global__ void __launch_bounds__(kReproThreads, 3)
k_repro1_dtlz1(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk) {
  repro_body<PROB_DTLZ1>(dir, KeyConst{rk});
}
__global__ void __launch_bounds__(kReproThreads, 3)
k_repro1_dtlz2(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk) {
  repro_body<PROB_DTLZ2>(dir, KeyConst{rk});
}
__global__ void __launch_bounds__(kReproThreads, 3)
k_repro1_neuro(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk) {
  repro_body<PROB_NEURO>(dir, KeyConst{rk});
}

// A batch of runs: each CTA's round keys follow from its run's key.
__global__ void __launch_bounds__(kReproThreads, 3)
k_repro(const __grid_constant__ BatchDir dir) {
  const int run = dir_find(dir, blockIdx.x);
  repro_dispatch(dir, KeyRun{dir.key[run].x, dir.key[run].y});
}

// Initial population (Algorithm 2, initialisation), slots 0..N-1, and its
// objectives.  DTLZ: x = L + (U-L) u24 from INIT (j/4, i, 0) word j%4.
// Rollout problem: x = clip(0.1 z), z Box-Muller from INIT (j, i, 0).
__global__ void __launch_bounds__(kReproThreads)
k_init(const __grid_constant__ BatchDir dir) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const ReproItem it = static_cast<const ReproItem *>(dir.items[run])[blockIdx.x - dir.prefix[run]];
  const int TS = R.team;
  const int team = threadIdx.x / TS, lane = threadIdx.x & (TS - 1);
  const int m = R.m, d = R.d, G = R.G, N = R.N;
  const int i = it.pair0 + team;   // one team per individual
  const bool active = i < N;
  const uint32_t k0 = dir.key[run].x, k1 = dir.key[run].y;
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
          if (j >= mh) acc.x = g_term1(R.problem, x[v], acc.x);
          else head[j] = x[v];
        }
      }
      float4 *o = reinterpret_cast<float4 *>(y + 8 * g);
      o[0] = make_float4(x[0], x[1], x[2], x[3]);
      o[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
  }
  if (R.problem == PROB_NEURO) return;
  const float2 gs = team_sum2(acc, TS);
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

}  // namespace rvea
