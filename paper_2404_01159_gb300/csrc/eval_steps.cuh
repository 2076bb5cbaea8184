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
  if (multimodal_g(problem)) {
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
  if (multimodal_g(problem)) {
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
// gsum is the sum of the g-terms: sum (x - 1/2)^2 for DTLZ2/DTLZ4, and
// k + sum ((x - 1/2)^2 - cos 20 pi (x - 1/2)) for DTLZ1/DTLZ3 (g = 100 gsum).
// DTLZ4 maps the position variables to x^100.  One instance per problem, so
// a problem's kernels carry only its own form.
template <int PROB>
__device__ void dtlz_objectives_t(int m, float gsum, const float *head, float *f) {
  if (PROB == PROB_DTLZ1) {
    const float base = 0.5f * (1.0f + 100.0f * gsum);
    for (int k = 1; k <= m; ++k) {
      float v = base;
      for (int i = 1; i <= m - k; ++i) v *= head[i - 1];
      if (k > 1) v *= 1.0f - head[m - k];
      f[k - 1] = v;
    }
  } else if (PROB == PROB_DTLZ4) {
    const float base = 1.0f + gsum;
    float h[kMaxM];
    for (int i = 0; i < m - 1; ++i) h[i] = powf(head[i], 100.0f);
    for (int k = 1; k <= m; ++k) {
      float v = base;
      for (int i = 1; i <= m - k; ++i) v *= cospif(0.5f * h[i - 1]);
      if (k > 1) v *= sinpif(0.5f * h[m - k]);
      f[k - 1] = v;
    }
  } else {   // DTLZ2, DTLZ3
    const float base = 1.0f + (PROB == PROB_DTLZ3 ? 100.0f * gsum : gsum);
    for (int k = 1; k <= m; ++k) {
      float v = base;
      for (int i = 1; i <= m - k; ++i) v *= cospif(0.5f * head[i - 1]);
      if (k > 1) v *= sinpif(0.5f * head[m - k]);
      f[k - 1] = v;
    }
  }
}

__device__ void dtlz_objectives(int problem, int m, float gsum, const float *head, float *f) {
  switch (problem) {
    case PROB_DTLZ1: dtlz_objectives_t<PROB_DTLZ1>(m, gsum, head, f); return;
    case PROB_DTLZ3: dtlz_objectives_t<PROB_DTLZ3>(m, gsum, head, f); return;
    case PROB_DTLZ4: dtlz_objectives_t<PROB_DTLZ4>(m, gsum, head, f); return;
    default: dtlz_objectives_t<PROB_DTLZ2>(m, gsum, head, f); return;
  }
}

}  // namespace rvea
