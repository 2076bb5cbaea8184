// Neuroevolution objective: the synthetic linear-dynamics rollout of every
// policy (the stand-in for the paper's Brax control tasks, Sec. 4.3).
//
// Policy x = [W1 (h1 x ns), b1, W2 (h2 x h1), b2, W3 (na x h2), b3] with
// h1 = h2 = 64, ns <= 32, na <= 16; tanh on every layer; s_0 = 0,
// s_{tau+1} = A s_tau + B u_tau + sigma xi_tau for tau < steps;
// f1 = -sum_tau s_{tau+1}[0], f2 = sum_tau |u_tau|^2.  xi_tau[k] is one
// Box-Muller draw from Philox NOISE (k, tau, t), shared by every policy of
// generation t (common random numbers); t = 0 for the initial population.
//
// One warp runs one policy for all steps.  The three layers are GEMVs with a
// different matrix per policy, so they run on the tensor cores as
// mma.sync m16n8k16 (BF16 operands, FP32 accumulate) with the weights as the
// A operand and the activation vector as column 0 of B: one column of the
// eight is used, the price of a matrix-vector product on an MMA tile.
// A rollout of 1000 steps amplifies rounding: one BF16 pass misses 1e-2 on
// the objectives of sensitive policies, so both operands are split into BF16
// hi and lo parts (w = w_hi + w_lo, v = v_hi + v_lo) and every product takes
// two MMAs: B carries v_hi in column 0 and v_lo in column 1, so
// A_hi B + A_lo B accumulates W v_hi in column 0 and W v_lo in column 1, and
// their sum is W v with errors near FP32 level (FP32 accumulate).  The hi fragments of the weights stay
// in registers for the whole rollout (W1 padded to K = 32, W3 to M = 16: 112
// registers a lane), the lo fragments in shared memory (lane-major, one
// 16-byte load per tile); biases ride in the accumulator initialisers.
// Between layers the outputs (lanes 4i hold rows i and i + 8 of each 16-row
// tile, columns 0 and 1 summed) are split, packed to BF16 pairs and moved to
// the B fragments of the next layer with four shuffles per 16-row tile.  The dynamics stay in
// FP32 on the CUDA cores (lane k owns state component k; A, B rows in shared
// memory).
#include "rvea_device.cuh"

namespace rvea {

constexpr int kRollWarps = 2;      // policies per CTA (static shared memory < 48 KB)
constexpr int kRollNsMax = 32;     // state components (one per lane)
constexpr int kRollNaMax = 16;     // actions (one 16-row tile)
constexpr int kRollH = 64;         // hidden units of both hidden layers
constexpr int kRollTiles = 28;     // 16x16 weight tiles: W1 4x2, W2 4x4, W3 1x4

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// D = A (16x16, row) * B (16x8, col) + C, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma16816(float &d0, float &d1, float &d2, float &d3,
                                         const uint32_t *a, uint32_t b0, uint32_t b1, float c0,
                                         float c1, float c2, float c3) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%11,%12,%13};"
      : "=f"(d0), "=f"(d1), "=f"(d2), "=f"(d3)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1),
        "f"(c2), "f"(c3));
}

// BF16 pair (hi, lo split) of two floats: hi = bf16(a), bf16(b); lo = the
// rounded remainders a - hi_a, b - hi_b (exact in float).
__device__ __forceinline__ void split_pack(float a, float b, uint32_t &hi, uint32_t &lo) {
  hi = pack_bf16x2(a, b);
  lo = pack_bf16x2(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xFFFF0000u));
}

// A fragments (hi and lo) of the 16x16 tile (mt, kt) of a row-major matrix
// W (Mv x Kv, zero outside): lane (g = lane/4, q = lane%4) holds rows g, g+8
// and columns 2q, 2q+1, 2q+8, 2q+9 of the tile.
__device__ __forceinline__ void load_afrag(uint32_t *a, uint4 *lo, const float *W, int Mv, int Kv,
                                           int mt, int kt, int lane) {
  const int g = lane >> 2, q = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8, c0 = kt * 16 + 2 * q, c1 = c0 + 8;
  auto at = [&](int r, int c) { return (r < Mv && c < Kv) ? __ldg(W + (size_t)r * Kv + c) : 0.0f; };
  uint4 l;
  split_pack(at(r0, c0), at(r0, c0 + 1), a[0], l.x);
  split_pack(at(r1, c0), at(r1, c0 + 1), a[1], l.y);
  split_pack(at(r0, c1), at(r0, c1 + 1), a[2], l.z);
  split_pack(at(r1, c1), at(r1, c1 + 1), a[3], l.w);
  *lo = l;
}

// Two-pass product of one tile: d += A_hi B + A_lo B, B = [v_hi | v_lo | ...].
__device__ __forceinline__ void mma2(float *d, const uint32_t *ah, const uint4 &al, uint32_t b0,
                                     uint32_t b1) {
  const uint32_t a_lo[4] = {al.x, al.y, al.z, al.w};
  mma16816(d[0], d[1], d[2], d[3], ah, b0, b1, d[0], d[1], d[2], d[3]);
  mma16816(d[0], d[1], d[2], d[3], a_lo, b0, b1, d[0], d[1], d[2], d[3]);
}

// Rows r (c0 + c1: columns 0 and 1 summed) and r + 8 (c2 + c3) of a 16-row
// output tile, held by lanes 4i, after tanh, as the B fragment of the next
// layer (rows 16t..16t+15 of its input): the hi parts in column 0 (lanes
// 0..3), the lo parts in column 1 (lanes 4..7); other lanes receive values
// of unused columns.
__device__ __forceinline__ void tile_to_b(float v0, float v8, int lane, uint32_t *b) {
  uint32_t ph, pl;
  split_pack(tanh_approx(v0), tanh_approx(v8), ph, pl);
  const int q = lane & 3;
  const uint32_t xh = __shfl_sync(0xffffffffu, ph, 8 * q), yh = __shfl_sync(0xffffffffu, ph, 8 * q + 4);
  const uint32_t xl = __shfl_sync(0xffffffffu, pl, 8 * q), yl = __shfl_sync(0xffffffffu, pl, 8 * q + 4);
  const bool hi = lane < 4;
  b[0] = hi ? __byte_perm(xh, yh, 0x5410) : __byte_perm(xl, yl, 0x5410);   // rows 2q, 2q+1
  b[1] = hi ? __byte_perm(xh, yh, 0x7632) : __byte_perm(xl, yl, 0x7632);   // rows 2q+8, 2q+9
}

// Noise table of generation t for each run of the directory:
// noise[tau][k] = xi_tau[k], Box-Muller from Philox NOISE (k, tau, t) with
// u1 = 1 - u24(word 0) in (0, 1] and u2 = u24(word 1).  One thread per entry;
// dir.prefix counts CTAs of 256 entries.
__global__ void k_noise(const __grid_constant__ BatchDir dir, int init) {
  pdl_wait();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int e = (blockIdx.x - dir.prefix[run]) * blockDim.x + threadIdx.x;
  if (e >= R.steps * R.ns) return;
  const int tau = e / R.ns, k = e - tau * R.ns;
  const int t = init ? 0 : R.ctl->t;
  const uint4 w = philox((uint32_t)k, (uint32_t)tau, (uint32_t)t, TAG_NOISE, dir.key[run].x,
                         dir.key[run].y);
  const float u1 = 1.0f - u24f(w.x), u2 = u24f(w.y);
  R.noise[e] = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// Rollouts of a directory of runs: dir.prefix counts CTAs of kRollWarps
// policies.  init: the initial population (rows 0..N-1, noise of t = 0);
// otherwise the N children of generation t (rows child_slot[t & 1]).
__global__ void __launch_bounds__(kRollWarps * 32)
k_rollout(const __grid_constant__ BatchDir dir, int init) {
  pdl_wait();
  __shared__ float sA[kRollNsMax * kRollNsMax], sB[kRollNsMax * kRollNaMax];
  __shared__ uint4 sLo[kRollWarps * kRollTiles * 32];   // lo weight fragments, per warp
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ns = R.ns, na = R.na, steps = R.steps, N = R.N;
  for (int e = threadIdx.x; e < ns * ns; e += blockDim.x) sA[e] = R.dynA[e];
  for (int e = threadIdx.x; e < ns * na; e += blockDim.x) sB[e] = R.dynB[e];
  __syncthreads();
  const int c = (blockIdx.x - dir.prefix[run]) * kRollWarps + warp;
  if (c >= N) return;
  const int t = R.ctl->t;
  int slot = c;
  if (!init) slot = R.child_slot[(t & 1) * N + c];
  if (slot < 0 || slot >= 2 * N) {
    if (lane == 0) set_status(R.ctl, ST_BADINDEX);
    return;
  }
  const float *x = R.X + (size_t)slot * R.d_pad;
  const float *W1 = x, *b1 = W1 + kRollH * ns, *W2 = b1 + kRollH, *b2 = W2 + kRollH * kRollH;
  const float *W3 = b2 + kRollH, *b3 = W3 + na * kRollH;
  // weights as BF16 A fragments for the whole rollout: hi in registers, lo
  // in this warp's shared-memory slab (tile-major, lane-minor)
  uint4 *const slo = sLo + warp * (kRollTiles * 32);
  uint32_t a1[4][2][4], a2[4][4][4], a3[4][4];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
    for (int kt = 0; kt < 2; ++kt)
      load_afrag(a1[mt][kt], slo + (mt * 2 + kt) * 32 + lane, W1, kRollH, ns, mt, kt, lane);
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
      load_afrag(a2[mt][kt], slo + (8 + mt * 4 + kt) * 32 + lane, W2, kRollH, kRollH, mt, kt, lane);
  }
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) load_afrag(a3[kt], slo + (24 + kt) * 32 + lane, W3, na, kRollH, 0, kt, lane);
  __syncwarp();
  // biases in the accumulator layout (rows g, g+8 of each tile)
  const int g = lane >> 2;
  float bb1[4][2], bb2[4][2], bb3[2];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    bb1[mt][0] = __ldg(b1 + mt * 16 + g);
    bb1[mt][1] = __ldg(b1 + mt * 16 + g + 8);
    bb2[mt][0] = __ldg(b2 + mt * 16 + g);
    bb2[mt][1] = __ldg(b2 + mt * 16 + g + 8);
  }
  bb3[0] = g < na ? __ldg(b3 + g) : 0.0f;
  bb3[1] = g + 8 < na ? __ldg(b3 + g + 8) : 0.0f;

  const float sigma = R.sigma;
  const float *xi = R.noise;
  const int q = lane & 3;
  float s = 0.0f;              // lane k < ns: s[k]; other lanes 0
  float f1 = 0.0f, f2 = 0.0f;
#pragma unroll 1
  for (int tau = 0; tau < steps; ++tau) {
    // layer 1: K = ns padded to 32 (lanes >= ns hold s = 0)
    uint32_t bk[4][2];
    {
      const float v0 = __shfl_sync(0xffffffffu, s, 2 * q), v1 = __shfl_sync(0xffffffffu, s, 2 * q + 1);
      const float v2 = __shfl_sync(0xffffffffu, s, 2 * q + 8), v3 = __shfl_sync(0xffffffffu, s, 2 * q + 9);
      const float v4 = __shfl_sync(0xffffffffu, s, 2 * q + 16), v5 = __shfl_sync(0xffffffffu, s, 2 * q + 17);
      const float v6 = __shfl_sync(0xffffffffu, s, 2 * q + 24), v7 = __shfl_sync(0xffffffffu, s, 2 * q + 25);
      uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
      split_pack(v0, v1, h0, l0);
      split_pack(v2, v3, h1, l1);
      split_pack(v4, v5, h2, l2);
      split_pack(v6, v7, h3, l3);
      const bool hi = lane < 4;   // column 0: hi parts, column 1: lo parts
      bk[0][0] = hi ? h0 : l0;
      bk[0][1] = hi ? h1 : l1;
      bk[1][0] = hi ? h2 : l2;
      bk[1][1] = hi ? h3 : l3;
    }
    float h[4][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      h[mt][0] = bb1[mt][0];
      h[mt][2] = bb1[mt][1];
      h[mt][1] = h[mt][3] = 0.0f;
#pragma unroll
      for (int kt = 0; kt < 2; ++kt)
        mma2(h[mt], a1[mt][kt], slo[(mt * 2 + kt) * 32 + lane], bk[kt][0], bk[kt][1]);
    }
    // layer 2
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) tile_to_b(h[kt][0] + h[kt][1], h[kt][2] + h[kt][3], lane, bk[kt]);
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {   // two accumulation chains per tile (k-tiles 0-1, 2-3)
      float g2[4] = {0.f, 0.f, 0.f, 0.f};
      h[mt][0] = bb2[mt][0];
      h[mt][2] = bb2[mt][1];
      h[mt][1] = h[mt][3] = 0.0f;
      mma2(h[mt], a2[mt][0], slo[(8 + mt * 4 + 0) * 32 + lane], bk[0][0], bk[0][1]);
      mma2(g2, a2[mt][2], slo[(8 + mt * 4 + 2) * 32 + lane], bk[2][0], bk[2][1]);
      mma2(h[mt], a2[mt][1], slo[(8 + mt * 4 + 1) * 32 + lane], bk[1][0], bk[1][1]);
      mma2(g2, a2[mt][3], slo[(8 + mt * 4 + 3) * 32 + lane], bk[3][0], bk[3][1]);
#pragma unroll
      for (int e = 0; e < 4; ++e) h[mt][e] += g2[e];
    }
    // layer 3 (one 16-row tile, rows < na used)
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) tile_to_b(h[kt][0] + h[kt][1], h[kt][2] + h[kt][3], lane, bk[kt]);
    // four independent accumulation chains (one per k-tile), summed after
    float o[4] = {bb3[0], 0.0f, bb3[1], 0.0f}, o1[4] = {0.f, 0.f, 0.f, 0.f};
    float o2[4] = {0.f, 0.f, 0.f, 0.f}, o3[4] = {0.f, 0.f, 0.f, 0.f};
    mma2(o, a3[0], slo[24 * 32 + lane], bk[0][0], bk[0][1]);
    mma2(o1, a3[1], slo[25 * 32 + lane], bk[1][0], bk[1][1]);
    mma2(o2, a3[2], slo[26 * 32 + lane], bk[2][0], bk[2][1]);
    mma2(o3, a3[3], slo[27 * 32 + lane], bk[3][0], bk[3][1]);
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] += (o1[e] + o2[e]) + o3[e];
    // u_o = tanh(row o): lane 4o (o < 8) holds rows o and o + 8
    const float ulo = tanh_approx(o[0] + o[1]), uhi = tanh_approx(o[2] + o[3]);
    if (q == 0) {
      if (g < na) f2 = fmaf(ulo, ulo, f2);
      if (g + 8 < na) f2 = fmaf(uhi, uhi, f2);
    }
    // dynamics in FP32: lane k computes s'[k]
    float za = 0.0f, zb = 0.0f;   // two chains: A s and B u
    const float *Ar = sA + lane * ns, *Br = sB + lane * na;
    for (int i = 0; i < ns; ++i) {
      const float si = __shfl_sync(0xffffffffu, s, i);
      if (lane < ns) za = fmaf(Ar[i], si, za);
    }
    for (int oo = 0; oo < na; ++oo) {
      const float uo = __shfl_sync(0xffffffffu, oo < 8 ? ulo : uhi, 4 * (oo & 7));
      if (lane < ns) zb = fmaf(Br[oo], uo, zb);
    }
    s = lane < ns ? fmaf(sigma, __ldg(xi + (size_t)tau * ns + lane), za + zb) : 0.0f;
    f1 -= __shfl_sync(0xffffffffu, s, 0);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, off);
  if (lane == 0) {
    const int n2 = 2 * N;
    R.F[slot] = f1;
    R.F[(size_t)n2 + slot] = f2;
    atomicMin(&R.ctl->zkey[0], f2ord(f1));
    atomicMin(&R.ctl->zkey[1], f2ord(f2));
  }
}

// The same rollout with the policy GEMVs on the CUDA cores in FP32 (the
// configuration's other form, rvea_neuro_dynamics.gemv = 1): one warp per
// policy, its 64 x 64 hidden layer register-resident.  Lane l owns rows l
// and l + 32 of both hidden layers: W2's two rows (128 floats) and W3's
// columns l and l + 32 stay in its registers for the whole rollout, W1
// (transposed, float4 blocks [column / 4][row]) in shared memory, so that a
// step reads from shared memory only the broadcast input vectors and W1.
// Layer 3 reduces the lanes' partial sums of all actions at once (one
// multi-value reduce-scatter); the next step's noise is loaded a step ahead.
// The dynamics and the objectives are as in the MMA form (lane k owns state
// component k; A and B transposed in shared memory).  NS4: ns padded to a
// multiple of 4 (ns <= kRF32NsMax, na <= kRF32NaMax).
constexpr int kRF32Warps = 2;     // policies per CTA
constexpr int kRF32NsMax = 24;
constexpr int kRF32NaMax = 8;

struct RF32Shared {
  float AT[kRF32NsMax][32];                 // AT[i][k] = A[k][i], zero past ns
  float BT[kRF32NaMax][32];                 // BT[o][k] = B[k][o], zero past ns, na
  float4 w1[kRF32Warps][kRF32NsMax / 4][kRollH];
  float4 sv[kRF32Warps][kRF32NsMax / 4];    // the state (zero past ns)
  float4 h1[kRF32Warps][kRollH / 4];        // the first hidden layer's output
  float w3[kRF32Warps][kRF32NaMax][kRollH]; // W3 (zero rows past na)
  float b3[kRF32Warps][kRF32NaMax];
};

// Sum over the warp of eight values per lane, every lane ending with all
// eight sums: a reduce-scatter (each exchange halves the values a lane
// keeps: 4 + 2 + 1 shuffles), two more butterfly steps, then the eight sums
// gathered from the lanes that hold them (8 shuffles): 17 shuffles on a
// chain of 6 exchanges, where eight separate butterflies take 40.
__device__ __forceinline__ void warp_sum8(float (&v)[8], int lane) {
  // offset 16: lanes < 16 keep values 0-3, the others 4-7
  const bool hi16 = lane & 16;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float send = hi16 ? v[q] : v[q + 4];
    const float got = __shfl_xor_sync(0xffffffffu, send, 16);
    v[q] = (hi16 ? v[q + 4] : v[q]) + got;
  }
  // offset 8: keep 2 of the 4 (values 2k, 2k+1 of the kept half)
  const bool hi8 = lane & 8;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float send = hi8 ? v[q] : v[q + 2];
    const float got = __shfl_xor_sync(0xffffffffu, send, 8);
    v[q] = (hi8 ? v[q + 2] : v[q]) + got;
  }
  // offset 4: keep 1 of the 2
  {
    const bool hi4 = lane & 4;
    const float send = hi4 ? v[0] : v[1];
    const float got = __shfl_xor_sync(0xffffffffu, send, 4);
    v[0] = (hi4 ? v[1] : v[0]) + got;
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  // lane l now holds the sum of value 4 (l >> 4 & 1) + 2 (l >> 3 & 1) + (l >> 2 & 1)
  const float mine = v[0];
#pragma unroll
  for (int o = 0; o < 8; ++o)
    v[o] = __shfl_sync(0xffffffffu, mine, ((o >> 2) & 1) * 16 + ((o >> 1) & 1) * 8 + (o & 1) * 4);
}

template <int NS4>
__device__ __forceinline__ void rollout_reg(const RunDesc &R, RF32Shared &S, int c, int init) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ns = R.ns, na = R.na, steps = R.steps, N = R.N;
  const int t = R.ctl->t;
  int slot = c;
  if (!init) slot = R.child_slot[(t & 1) * N + c];
  if (slot < 0 || slot >= 2 * N) {
    if (lane == 0) set_status(R.ctl, ST_BADINDEX);
    return;
  }
  const float *x = R.X + (size_t)slot * R.d_pad;
  const float *W1 = x, *b1 = W1 + kRollH * ns, *W2 = b1 + kRollH, *b2 = W2 + kRollH * kRollH;
  const float *W3 = b2 + kRollH, *b3 = W3 + na * kRollH;
  const int r0 = lane, r1 = lane + 32;
  // W1, W3 into shared memory, W2's two rows into registers, once
  for (int e = lane; e < (NS4 / 4) * kRollH; e += 32) {
    const int c4 = e / kRollH, r = e - c4 * kRollH;
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = 4 * c4 + u < ns ? __ldg(W1 + (size_t)r * ns + 4 * c4 + u) : 0.0f;
    S.w1[warp][c4][r] = make_float4(v[0], v[1], v[2], v[3]);
  }
  for (int e = lane; e < kRF32NaMax * kRollH; e += 32)
    S.w3[warp][e / kRollH][e % kRollH] = e / kRollH < na ? __ldg(W3 + e) : 0.0f;
  if (lane < NS4 / 4) S.sv[warp][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (lane < kRF32NaMax) S.b3[warp][lane] = lane < na ? __ldg(b3 + lane) : 0.0f;
  float w2a[kRollH], w2b[kRollH];
#pragma unroll
  for (int c4 = 0; c4 < kRollH / 4; ++c4) {
    const float4 p = __ldg(reinterpret_cast<const float4 *>(W2 + (size_t)r0 * kRollH) + c4);
    const float4 q = __ldg(reinterpret_cast<const float4 *>(W2 + (size_t)r1 * kRollH) + c4);
    w2a[4 * c4] = p.x; w2a[4 * c4 + 1] = p.y; w2a[4 * c4 + 2] = p.z; w2a[4 * c4 + 3] = p.w;
    w2b[4 * c4] = q.x; w2b[4 * c4 + 1] = q.y; w2b[4 * c4 + 2] = q.z; w2b[4 * c4 + 3] = q.w;
  }
  const float bb1a = __ldg(b1 + r0), bb1b = __ldg(b1 + r1);
  const float bb2a = __ldg(b2 + r0), bb2b = __ldg(b2 + r1);
  __syncwarp();
  const float sigma = R.sigma;
  const float *xi = R.noise;
  const float4 *sv = S.sv[warp];
  const float4 *h1 = S.h1[warp];
  float *const h1f = reinterpret_cast<float *>(S.h1[warp]);
  const bool dyn = lane < ns;   // lane k owns state component k
  float f1 = 0.0f, f2 = 0.0f;
  float xin = dyn && steps > 0 ? __ldg(xi + lane) : 0.0f;   // this step's noise, loaded a step ahead
#pragma unroll 1
  for (int tau = 0; tau < steps; ++tau) {
    const float xic = xin;
    if (dyn && tau + 1 < steps) xin = __ldg(xi + (size_t)(tau + 1) * ns + lane);
    // layer 1: rows r0, r1, two accumulation chains each
    float a0 = bb1a, c0 = 0.0f, a1 = bb1b, c1 = 0.0f;
#pragma unroll
    for (int c4 = 0; c4 < NS4 / 4; ++c4) {
      const float4 v = sv[c4];
      const float4 p = S.w1[warp][c4][r0], q = S.w1[warp][c4][r1];
      a0 = fmaf(p.x, v.x, a0); c0 = fmaf(p.y, v.y, c0); a0 = fmaf(p.z, v.z, a0); c0 = fmaf(p.w, v.w, c0);
      a1 = fmaf(q.x, v.x, a1); c1 = fmaf(q.y, v.y, c1); a1 = fmaf(q.z, v.z, a1); c1 = fmaf(q.w, v.w, c1);
    }
    h1f[r0] = tanh_approx(a0 + c0);
    h1f[r1] = tanh_approx(a1 + c1);
    // the state part of the dynamics (independent of the policy): A s
    float za = 0.0f, zc = 0.0f;
#pragma unroll
    for (int c4 = 0; c4 < NS4 / 4; ++c4) {
      const float4 v = sv[c4];
      za = fmaf(S.AT[4 * c4][lane], v.x, za);
      zc = fmaf(S.AT[4 * c4 + 1][lane], v.y, zc);
      za = fmaf(S.AT[4 * c4 + 2][lane], v.z, za);
      zc = fmaf(S.AT[4 * c4 + 3][lane], v.w, zc);
    }
    __syncwarp();
    // layer 2: W2 rows from registers, four accumulation chains per row
    float e0[4] = {bb2a, 0.0f, 0.0f, 0.0f}, e1[4] = {bb2b, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int c4 = 0; c4 < kRollH / 4; ++c4) {
      const float4 v = h1[c4];
      e0[0] = fmaf(w2a[4 * c4], v.x, e0[0]); e0[1] = fmaf(w2a[4 * c4 + 1], v.y, e0[1]);
      e0[2] = fmaf(w2a[4 * c4 + 2], v.z, e0[2]); e0[3] = fmaf(w2a[4 * c4 + 3], v.w, e0[3]);
      e1[0] = fmaf(w2b[4 * c4], v.x, e1[0]); e1[1] = fmaf(w2b[4 * c4 + 1], v.y, e1[1]);
      e1[2] = fmaf(w2b[4 * c4 + 2], v.z, e1[2]); e1[3] = fmaf(w2b[4 * c4 + 3], v.w, e1[3]);
    }
    const float g0 = tanh_approx((e0[0] + e0[1]) + (e0[2] + e0[3]));
    const float g1 = tanh_approx((e1[0] + e1[1]) + (e1[2] + e1[3]));
    // layer 3: every lane's share of the actions, summed over the warp
    float pr[kRF32NaMax];
#pragma unroll
    for (int o = 0; o < kRF32NaMax; ++o) pr[o] = fmaf(S.w3[warp][o][r0], g0, S.w3[warp][o][r1] * g1);
    warp_sum8(pr, lane);
    float zb = 0.0f;
#pragma unroll
    for (int o = 0; o < kRF32NaMax; ++o) {
      const float u = o < na ? tanh_approx(pr[o] + S.b3[warp][o]) : 0.0f;
      f2 = fmaf(u, u, f2);
      zb = fmaf(S.BT[o][lane], u, zb);
    }
    // dynamics: lane k computes s'[k] = A s + B u + sigma xi
    const float s = dyn ? fmaf(sigma, xic, (za + zc) + zb) : 0.0f;
    __syncwarp();   // every lane has read the state and h1
    if (dyn) reinterpret_cast<float *>(S.sv[warp])[lane] = s;
    f1 -= __shfl_sync(0xffffffffu, s, 0);
    __syncwarp();
  }
  if (lane == 0) {
    const int n2 = 2 * N;
    R.F[slot] = f1;
    R.F[(size_t)n2 + slot] = f2;
    atomicMin(&R.ctl->zkey[0], f2ord(f1));
    atomicMin(&R.ctl->zkey[1], f2ord(f2));
  }
}

__global__ void __launch_bounds__(kRF32Warps * 32)
k_rollout_f32(const __grid_constant__ BatchDir dir, int init) {
  pdl_wait();
  __shared__ __align__(16) RF32Shared S;
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int ns = R.ns, na = R.na;
  for (int e = threadIdx.x; e < kRF32NsMax * 32; e += blockDim.x) {
    const int i = e / 32, k = e % 32;   // AT[i][k] = A[k][i]
    S.AT[i][k] = i < ns && k < ns ? R.dynA[k * ns + i] : 0.0f;
  }
  for (int e = threadIdx.x; e < kRF32NaMax * 32; e += blockDim.x) {
    const int o = e / 32, k = e % 32;   // BT[o][k] = B[k][o]
    S.BT[o][k] = o < na && k < ns ? R.dynB[k * na + o] : 0.0f;
  }
  __syncthreads();
  const int c = (blockIdx.x - dir.prefix[run]) * kRF32Warps + (threadIdx.x >> 5);
  if (c >= R.N) return;
  switch ((ns + 3) / 4) {
    case 1: rollout_reg<4>(R, S, c, init); return;
    case 2: rollout_reg<8>(R, S, c, init); return;
    case 3: rollout_reg<12>(R, S, c, init); return;
    case 4: rollout_reg<16>(R, S, c, init); return;
    case 5: rollout_reg<20>(R, S, c, init); return;
    default: rollout_reg<24>(R, S, c, init); return;
  }
}

// Dynamic shared memory of k_rollout_f32 (its tables are static).
size_t rollout_f32_smem(int, int) { return 0; }

}  // namespace rvea
