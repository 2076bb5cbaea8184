// Device steps shared by the reproduction, mutation and fused tail kernels:
// Deb's bounded polynomial mutation (Appendix B), the DTLZ g-terms and
// objectives (Sec. 4.1, Appendix C; DTLZ3/DTLZ4 from their published
// definitions).
#pragma once
#include "rvea_device.cuh"

namespace rvea {

__device__ __forceinline__ float clampf(float x, float lo, float hi) {
  return fminf(fmaxf(x, lo), hi);
}

// Deb's bounded polynomial mutation step (Appendix B, Delta), float.
static __device__ __noinline__ float poly_mutate(float x, float M, float L, float U, float eta) {
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

// 2 sin^2(pi r) = 1 - cos(2 pi r) = u q(u), u = r^2, |r| <= 1/2: q is the
// degree-5 minimax polynomial of the Remez exchange fit made by
// sin2_remez.py (fit error 1.2e-8; the float32 Horner evaluation stays within
// 4e-7 of the exact term, whose values run from 0 to 2).
constexpr float kQ1 = 19.739206f;
constexpr float kQ2 = -64.93916f;
constexpr float kQ3 = 85.45077f;
constexpr float kQ4 = -60.171906f;
constexpr float kQ5 = 25.98146f;
constexpr float kQ6 = -6.5458927f;
// Adding 1.5 2^23 rounds a float of magnitude below 2^22 to the nearest
// integer (ties to even), in the addition itself.
constexpr float kRound = 12582912.0f;

// g-terms of two adjacent variables x = (x_j, x_j+1), added into acc.
// DTLZ2: (x-1/2)^2.  DTLZ1: (x-1/2)^2 - cos(20 pi (x-1/2)) + 1 = y^2 + 2 sin^2(10 pi y)
// (identical, free of cancellation; the k = d-m+1 constant is the +1 of each
// term).  sin^2 has period 1 in 10y: 10y is reduced by its nearest integer n
// (n from one fused multiply-add into kRound, r = 10 y - n in one more), then
// 2 sin^2(pi r) = u q(u).
__device__ __forceinline__ float2 g_terms2(int problem, float2 x, float2 acc) {
  const float2 y = add2(x, splat2(-0.5f));
  acc = fma2(y, y, acc);
  if (multimodal_g(problem)) {
    const float2 tr = fma2(splat2(10.0f), y, splat2(kRound));
    const float2 nn = sub2(splat2(kRound), tr);          // -n
    const float2 r = fma2(splat2(10.0f), y, nn);
    const float2 u = mul2(r, r);
    float2 q = fma2(u, splat2(kQ6), splat2(kQ5));
    q = fma2(u, q, splat2(kQ4));
    q = fma2(u, q, splat2(kQ3));
    q = fma2(u, q, splat2(kQ2));
    q = fma2(u, q, splat2(kQ1));
    acc = fma2(u, q, acc);
  }
  return acc;
}

// Scalar form of the same terms (bit-identical per element), used where a
// group holds x_1..x_{m-1} or the ragged end of the row.
__device__ __forceinline__ float g_term1(int problem, float x, float acc) {
  const float y = x + (-0.5f);
  acc = fmaf(y, y, acc);
  if (multimodal_g(problem)) {
    const float tr = fmaf(10.0f, y, kRound);
    const float nn = kRound - tr;
    const float r = fmaf(10.0f, y, nn);
    const float u = r * r;
    float q = fmaf(u, kQ6, kQ5);
    q = fmaf(u, q, kQ4);
    q = fmaf(u, q, kQ3);
    q = fmaf(u, q, kQ2);
    q = fmaf(u, q, kQ1);
    acc = fmaf(u, q, acc);
  }
  return acc;
}

// Objectives from g and the first m-1 variables (standard DTLZ forms).
// gsum is the sum of the g-terms: sum (x - 1/2)^2 for DTLZ2/DTLZ4, and
// k + sum ((x - 1/2)^2 - cos 20 pi (x - 1/2)) for DTLZ1/DTLZ3 (g = 100 gsum).
// DTLZ4 maps the position variables to x^100.  One instance per problem, so
// a problem's kernels carry only its own form.  1 + 100 gsum is one explicit
// fused multiply-add, so every kernel that evaluates gets the same bits.
template <int PROB>
__device__ __forceinline__ void dtlz_objectives_t(int m, float gsum, const float *head, float *f) {
  if (PROB == PROB_DTLZ1) {
    const float base = 0.5f * __fmaf_rn(100.0f, gsum, 1.0f);
#pragma unroll
    for (int k = 1; k <= m; ++k) {
      float v = base;
#pragma unroll
      for (int i = 1; i <= m - k; ++i) v *= head[i - 1];
      if (k > 1) v *= 1.0f - head[m - k];
      f[k - 1] = v;
    }
  } else if (PROB == PROB_DTLZ4) {
    const float base = 1.0f + gsum;
    float h[kMaxM];
#pragma unroll
    for (int i = 0; i < m - 1; ++i) h[i] = powf(head[i], 100.0f);
#pragma unroll
    for (int k = 1; k <= m; ++k) {
      float v = base;
#pragma unroll
      for (int i = 1; i <= m - k; ++i) v *= cospif(0.5f * h[i - 1]);
      if (k > 1) v *= sinpif(0.5f * h[m - k]);
      f[k - 1] = v;
    }
  } else {   // DTLZ2, DTLZ3
    const float base = PROB == PROB_DTLZ3 ? __fmaf_rn(100.0f, gsum, 1.0f) : 1.0f + gsum;
#pragma unroll
    for (int k = 1; k <= m; ++k) {
      float v = base;
#pragma unroll
      for (int i = 1; i <= m - k; ++i) v *= cospif(0.5f * head[i - 1]);
      if (k > 1) v *= sinpif(0.5f * head[m - k]);
      f[k - 1] = v;
    }
  }
}

static __device__ void dtlz_objectives(int problem, int m, float gsum, const float *head, float *f) {
  switch (problem) {
    case PROB_DTLZ1: dtlz_objectives_t<PROB_DTLZ1>(m, gsum, head, f); return;
    case PROB_DTLZ3: dtlz_objectives_t<PROB_DTLZ3>(m, gsum, head, f); return;
    case PROB_DTLZ4: dtlz_objectives_t<PROB_DTLZ4>(m, gsum, head, f); return;
    default: dtlz_objectives_t<PROB_DTLZ2>(m, gsum, head, f); return;
  }
}

}  // namespace rvea
