// Reproduction and evaluation kernels.
//
// k_repro fuses, per pair of children (Appendix B of arXiv 2404.01159):
//   mating draw -> SBX (the two B equations and X_cross) -> clip -> polynomial
//   mutation (C, Delta, X_mut) -> clip -> DTLZ evaluation -> ideal point z*.
//
// Work decomposition.  A team of TS lanes (TS a power of two <= 32, fixed by d
// alone) owns one work unit: one segment of sg consecutive 8-variable groups
// of one pair (the pair's G groups split into nseg near-equal segments of at
// most kLaneGroups*TS groups).  Teams never wait on other warps: the phases
// below synchronise with __syncwarp only.  Teams of fewer than 32 lanes own a
// whole pair (one segment) and finish it: mutation, g, objectives.  32-lane
// teams (d > 1024) store their segments' partial sums of g and leave the
// mutation and the evaluation to k_mutate, which adds the partials in
// segment order, so the reduction tree depends on d alone.
//
// The main pass does SBX, clip and the g-terms of both children, four
// variables (one float4) at a time, and stores the crossed children.  Only
// the float4s holding x_1..x_{m-1} (kept out of g) or the end of the row take
// an out-of-line edge path.  Mutation is sparse (about one site per row), so
// it is a second pass over the row's sites (in this kernel for teams of fewer
// than 32 lanes, in k_mutate for the others): reload the crossed value,
// mutate, store, and correct the g sum by term(new) - term(old).
// Parents are read either straight from global memory (teams of fewer than
// 32 lanes) or, for 32-lane teams, from a ring of shared-memory chunks filled
// by TMA bulk copies, so that each warp keeps its next chunk in flight.
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
// so a row costs one or two Philox calls instead of one draw per site.
#include "eval_steps.cuh"

namespace rvea {

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

// 2^x and log2 x with one MUFU instruction each (PTX ex2/lg2.approx,
// relative error ~2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// SBX spread factor of one variable (Appendix B: beta from Mc, sign from R1,
// B = 1 where R2 keeps the variable or the pair does not cross).  Word q
// carries Mc = (q >> 8) 2^-24, the sign coin (bit 0) and the keep coin
// (bit 1).  Mc < 1/2 iff bit 31 is clear; then 2 Mc = u 2^-23, otherwise
// 2 - 2 Mc = (2^24 - u) 2^-23, both exact, so log2 of the base is
// log2(integer) - 23.
__device__ __forceinline__ float sbx_B(uint32_t q, bool nocross, float ie) {
  const uint32_t u = q >> 8;
  const bool lowb = (int32_t)q >= 0;
  const float lb = lg2_approx((float)(lowb ? u : 0x1000000u - u)) - 23.0f;
  const float beta = ex2_approx((lowb ? ie : -ie) * lb);
  const float B = (q & 1u) ? beta : -beta;
  return ((q & 2u) || nocross) ? 1.0f : B;
}

// Children of two adjacent variables: with s = x1 + x2 and e = x1 - x2,
// c1 = ((1+B) x1 + (1-B) x2) / 2 = (s + B e) / 2 and c2 = s - c1, clipped to
// [L, U].  Equal parents give equal children exactly.  UNIT: the box is
// [0, 1] (the DTLZ problems), where the clip is the saturation modifier of
// the operation that makes each child, one instruction instead of three.
template <bool UNIT>
__device__ __forceinline__ void sbx_pair(float2 x1, float2 x2, float2 B, float L, float U,
                                         float2 &c1, float2 &c2) {
  const float2 sm = add2(x1, x2), df = sub2(x1, x2);
  const float2 tt = fma2(B, df, sm);
  const float2 c1u = mul2(splat2(0.5f), tt);
  if (UNIT) {
    c1 = make_float2(__saturatef(0.5f * tt.x), __saturatef(0.5f * tt.y));
    c2 = make_float2(__saturatef(sm.x - c1u.x), __saturatef(sm.y - c1u.y));
  } else {
    const float2 c2u = sub2(sm, c1u);
    c1 = make_float2(clampf(c1u.x, L, U), clampf(c1u.y, L, U));
    c2 = make_float2(clampf(c2u.x, L, U), clampf(c2u.y, L, U));
  }
}

// Main-pass work on four adjacent variables (float4 Q of the row) of both
// children: SBX from Philox SBX (Q, p, t), clip, store, accumulate g-terms.
// (EVAL false: without the g-terms, into float4s of the caller's registers rather than pool
// rows.)  The DTLZ problems live on the unit box.
template <int PROB, class KP, bool EVAL = true>
__device__ __forceinline__ void cross4(const float4 xa, const float4 xb, int Q, int p, int t,
                                       bool nocross, float ie, float L, float U, const KP &kp,
                                       float4 *y1, float4 *y2, float2 &acc1, float2 &acc2) {
  constexpr bool kUnit = PROB != PROB_NEURO;
  const uint4 r = philox_k((uint32_t)Q, (uint32_t)p, (uint32_t)t, TAG_SBX, kp);
  float2 a0, a1, b0, b1;   // children 1 and 2, variables (0,1) and (2,3)
  sbx_pair<kUnit>(make_float2(xa.x, xa.y), make_float2(xb.x, xb.y),
                  make_float2(sbx_B(r.x, nocross, ie), sbx_B(r.y, nocross, ie)), L, U, a0, b0);
  sbx_pair<kUnit>(make_float2(xa.z, xa.w), make_float2(xb.z, xb.w),
                  make_float2(sbx_B(r.z, nocross, ie), sbx_B(r.w, nocross, ie)), L, U, a1, b1);
  if (EVAL && PROB != PROB_NEURO) {
    acc1 = g_terms2(PROB, a0, acc1);
    acc1 = g_terms2(PROB, a1, acc1);
    acc2 = g_terms2(PROB, b0, acc2);
    acc2 = g_terms2(PROB, b1, acc2);
  }
  if (EVAL) {   // rows of the pool: streaming stores (evict-first in L2)
    __stcs(y1, make_float4(a0.x, a0.y, a1.x, a1.y));
    if (y2) __stcs(y2, make_float4(b0.x, b0.y, b1.x, b1.y));
  } else {      // the edge path's float4s in registers
    *y1 = make_float4(a0.x, a0.y, a1.x, a1.y);
    if (y2) *y2 = make_float4(b0.x, b0.y, b1.x, b1.y);
  }
}

// The same for a float4 that holds some of x_1..x_{m-1} (j < mh, kept out
// of g) or reaches past the last variable (j >= d): g-terms per variable.
// The accumulators travel by value (no address taken, so they stay in
// registers in the caller's loops).
struct Acc2 {
  float2 a1, a2;
};
template <int PROB>
__device__ __noinline__ Acc2 cross4_edge(const float4 xa, const float4 xb, int Q, int p, int t,
                                         bool nocross, float ie, float L, float U, const KeyRun kp,
                                         float4 *y1, float4 *y2, Acc2 acc, int mh, int d) {
  float2 z1 = make_float2(0.f, 0.f), z2 = z1;
  float4 c1, c2;
  cross4<PROB, KeyRun, false>(xa, xb, Q, p, t, nocross, ie, L, U, kp, &c1, &c2, z1, z2);
  __stcs(y1, c1);
  if (y2) __stcs(y2, c2);
  if (PROB == PROB_NEURO) return acc;
  const float u1[4] = {c1.x, c1.y, c1.z, c1.w}, u2[4] = {c2.x, c2.y, c2.z, c2.w};
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int j = 4 * Q + v;
    if (j < mh || j >= d) continue;
    if (v & 1) {
      acc.a1.y = g_term1(PROB, u1[v], acc.a1.y);
      acc.a2.y = g_term1(PROB, u2[v], acc.a2.y);
    } else {
      acc.a1.x = g_term1(PROB, u1[v], acc.a1.x);
      acc.a2.x = g_term1(PROB, u2[v], acc.a2.x);
    }
  }
  return acc;
}

// Mutation of one crossed variable in place; returns term(new) - term(old).
template <int PROB>
__device__ __forceinline__ float mutate_one(float *px, int j, int c, int t, const RunDesc &R,
                                            const KeyRun &kp) {
  const float x = __ldcg(px);
  const uint4 w = philox_k((uint32_t)j, (uint32_t)c, (uint32_t)t, TAG_MUTMAG, kp);
  const float xn = poly_mutate(x, u24f(w.y), R.L, R.U, R.eta_m);
  __stcg(px, xn);
  return (PROB != PROB_NEURO && j >= R.m - 1) ? g_term1(PROB, xn, 0.0f) - g_term1(PROB, x, 0.0f)
                                              : 0.0f;
}

// Polynomial mutation of child c (pool row `slot`) at its sites in
// [jlo, jhi): site count, then Floyd's uniform subset; returns the change
// of the row's g sum.  Every site when the per-site probability is 1.
template <int PROB>
__device__ __noinline__ float mutate_sites(const RunDesc &R, const KeyRun kp, int c, int slot, int t,
                                           int jlo, int jhi) {
  float *const row = R.X + (size_t)slot * R.d_pad;
  float dg = 0.0f;
  const int d = R.d;
  int *const rec = R.rec_sites ? R.rec_sites + (size_t)c * (1 + kMaxSites) : nullptr;
  if (R.T_m >= (1u << 24)) {
    if (rec && jlo == 0) rec[0] = -1;
    for (int j = jlo; j < min(jhi, d); ++j) dg += mutate_one<PROB>(row + j, j, c, t, R, kp);
    return dg;
  }
  uint4 w = philox_k(0u, (uint32_t)c, (uint32_t)t, TAG_MUTSITE, kp);
  const int nthr = R.n_mthr;
  int k = 0;
  while (k < nthr && w.x >= R.mthr[k]) ++k;
  if (rec) rec[0] = k;
  int sites[kMaxSites];
  for (int i = 0; i < k; ++i) {
    const int e = i + 1;
    if ((e & 3) == 0) w = philox_k((uint32_t)(e >> 2), (uint32_t)c, (uint32_t)t, TAG_MUTSITE, kp);
    const uint32_t J = (uint32_t)(d - k + i);
    uint32_t r = __umulhi(word(w, e & 3), J + 1u);
    for (int l = 0; l < i; ++l)
      if ((uint32_t)sites[l] == r) { r = J; break; }
    sites[i] = (int)r;
    if (rec) rec[1 + i] = (int)r;
    if ((int)r >= jlo && (int)r < jhi) dg += mutate_one<PROB>(row + r, (int)r, c, t, R, kp);
  }
  return dg;
}

// Objectives of one child (pool row `slot`) from its g and x_1..x_{m-1} read
// back from the row (after its mutation), and its share of the ideal point
// (into the CTA's minimum zmin in shared memory: one atomic per child on the
// same global words would serialise the kernel at large N).
template <int PROB>
__device__ __forceinline__ void evaluate_child(const RunDesc &R, int slot, float g, unsigned *zmin) {
  const int m = R.m, mh = m - 1, n2 = 2 * R.N;
  const float *row = R.X + (size_t)slot * R.d_pad;
  float head[kMaxM], f[kMaxM];
  for (int j = 0; j < mh; ++j) head[j] = __ldcg(row + j);
  dtlz_objectives_t<PROB>(m, g, head, f);
  for (int kk = 0; kk < m; ++kk) {
    R.F[(size_t)kk * n2 + slot] = f[kk];
    atomicMin(&zmin[kk], f2ord(f[kk]));
  }
}

// A pair of a team of fewer than 32 lanes (one segment): both children.
template <int PROB>
__device__ __noinline__ void finish_pair(const RunDesc &R, float g1, float g2, int ch1, int ch2,
                                         unsigned *zmin) {
  evaluate_child<PROB>(R, ch1, g1, zmin);
  if (ch2 >= 0) evaluate_child<PROB>(R, ch2, g2, zmin);
}

template <int PROB, bool STAGED, class KP>
__device__ __forceinline__ void repro_body(const BatchDir &dir, const KP &kp) {
  pdl_wait();      // the previous generation's lists and slot maps
  pdl_trigger();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const ReproItem it = static_cast<const ReproItem *>(dir.items[run])[blockIdx.x - dir.prefix[run]];
  const int TS = R.team, tpw = 32 / TS, S = R.nseg, sg = R.sg;
  const int d = R.d, G = R.G, N = R.N, P = R.P;
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  const int tw = wl / TS, lane = wl & (TS - 1), tbase = tw * TS;
  const int unit = it.pair0 + warp * tpw + tw;
  const int p = unit / S, seg = unit - p * S;
  const bool active = p < P;
  const int t = R.ctl->t;
  const int *cslot = R.child_slot + (t & 1) * N;
  // teams of fewer than 32 lanes evaluate their children here: the CTA's
  // minimum of their objectives, one global atomic per objective at the end
  __shared__ unsigned s_zmin[kMaxM];
  const bool evals = PROB != PROB_NEURO && TS < 32;   // uniform over the CTA (one run)
  if (evals) {
    if (threadIdx.x < kMaxM) s_zmin[threadIdx.x] = 0xFFFFFFFFu;
    __syncthreads();
  }

  // ---- phase 0: the pair's two mating draws and crossover gate ------------
  uint32_t v0 = 0, v1 = 0, v2 = 0;
  if (active) {
    for (int c = lane; c < 3; c += TS) {
      if (c < 2) {
        const int e = c == 0 ? p : p + P;
        const uint4 w = philox_k((uint32_t)(e >> 2), 0u, (uint32_t)t, TAG_MATE, kp);
        const uint32_t idx = __umulhi(word(w, e & 3), (uint32_t)R.ctl->K);
        const int j = R.vlist[idx];
        if (R.rec_par && seg == 0) R.rec_par[e] = j;
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
  const int g0 = seg * sg, gE = min(G, g0 + sg);
  // run constants used inside the loops, in registers: the child-row stores
  // could alias the descriptor, which would force a reload after each store
  float4 *const X4 = reinterpret_cast<float4 *>(R.X);
  const uint32_t rq = (uint32_t)R.d_pad >> 2;      // float4s per row
  const uint32_t q1 = (uint32_t)ch1 * rq, q2 = has2 ? (uint32_t)ch2 * rq : 0u;
  const float L = R.L, U = R.U, ie = R.inv_eta_c1;
  // float4s [Qs, Qe) hold neither x_1..x_{m-1} nor variables past d
  const int mh = R.m - 1, Qs = (mh + 3) >> 2, Qe = d >> 2;

  // ---- main pass: SBX, clip, g-terms, store --------------------------------
  float2 acc1 = make_float2(0.f, 0.f), acc2 = make_float2(0.f, 0.f);
  if (STAGED && active) {
    // Parent segments staged in shared memory by the TMA engine: chunks of
    // 32 groups (1 KB per parent) in a ring of kStages buffers, so each warp
    // has the next chunks in flight while it works on one.  One team per
    // warp (TS == 32): lane l takes float4s l and l + 32 of a chunk.
    extern __shared__ __align__(128) unsigned char dsm[];
    float4 *const sb = reinterpret_cast<float4 *>(dsm) + warp * (kStages * 128);
    uint64_t *const bar =
        reinterpret_cast<uint64_t *>(dsm + (kReproThreads / 32) * kStageWarpBytes) + warp * kStages;
    if (wl == 0) {
      for (int q = 0; q < kStages; ++q) mbar_init(&bar[q], 1);
      fence_mbar_init();
    }
    __syncwarp();
    const int nch = (gE - g0 + 31) >> 5;
    const float *const Xf = R.X;
    const size_t r1 = (size_t)par1 * R.d_pad, r2 = (size_t)par2 * R.d_pad;
    auto issue = [&](int c) {
      const int gs = g0 + 32 * c, q = c % kStages;
      const uint32_t bytes = (uint32_t)(min(gE, gs + 32) - gs) * 32u;
      fence_proxy_async_smem();   // this stage's earlier reads come first
      mbar_expect_tx(&bar[q], 2u * bytes);
      const uint64_t pol = policy_evict_first();
      tma_load_1d_hint(sb + q * 128, Xf + r1 + 8 * gs, bytes, &bar[q], pol);
      tma_load_1d_hint(sb + q * 128 + 64, Xf + r2 + 8 * gs, bytes, &bar[q], pol);
    };
    if (wl == 0)
      for (int c = 0; c < min(kStages - 1, nch); ++c) issue(c);
    int c = 0;
#pragma unroll 1
    for (; c < nch; ++c) {
      if (wl == 0 && c + kStages - 1 < nch) issue(c + kStages - 1);
      const int q = c % kStages;
      if (!mbar_wait(&bar[q], (uint32_t)(c / kStages) & 1u, kWaitLimit)) break;
      const int gs = g0 + 32 * c, n4 = 2 * (min(gE, gs + 32) - gs);
      const float4 *const sa = sb + q * 128;          // this chunk: parent 1, then parent 2
      float4 *const y1 = X4 + q1 + 2 * gs;            // the chunk's first float4 of each child
      float4 *const y2 = has2 ? X4 + q2 + 2 * gs : nullptr;
      if (2 * gs >= Qs && 2 * gs + n4 <= Qe) {   // an interior chunk (warp-uniform)
#pragma unroll 1
        for (int qi = wl; qi < n4; qi += 32)   // float4 2 gs + qi: variables 4Q .. 4Q+3
          cross4<PROB>(sa[qi], sa[64 + qi], 2 * gs + qi, p, t, nocross, ie, L, U, kp, y1 + qi,
                       y2 ? y2 + qi : nullptr, acc1, acc2);
      } else {
        for (int qi = wl; qi < n4; qi += 32) {
          const Acc2 a = cross4_edge<PROB>(sa[qi], sa[64 + qi], 2 * gs + qi, p, t, nocross, ie,
                                           L, U, KeyRun{R.key0, R.key1}, y1 + qi,
                                           y2 ? y2 + qi : nullptr, Acc2{acc1, acc2}, mh, d);
          acc1 = a.a1;
          acc2 = a.a2;
        }
      }
      __syncwarp();
    }
    if (c < nch) {   // a copy never arrived: flag it, let the copies in flight land
      if (wl == 0) set_status(R.ctl, ST_TIMEOUT);
      for (int e = c + 1; e < min(nch, c + kStages); ++e)
        mbar_wait(&bar[e % kStages], (uint32_t)(e / kStages) & 1u, kWaitLimit);
    }
  } else if (active) {
    const uint32_t o1 = (uint32_t)par1 * rq, o2 = (uint32_t)par2 * rq;
#pragma unroll 1
    for (int Q = 2 * g0 + lane; Q < 2 * gE; Q += TS) {
      if (Q >= Qs && Q < Qe)
        cross4<PROB>(__ldg(X4 + o1 + Q), __ldg(X4 + o2 + Q), Q, p, t, nocross, ie, L, U, kp,
                     X4 + q1 + Q, has2 ? X4 + q2 + Q : nullptr, acc1, acc2);
      else {
        const Acc2 a = cross4_edge<PROB>(__ldg(X4 + o1 + Q), __ldg(X4 + o2 + Q), Q, p, t, nocross,
                                         ie, L, U, KeyRun{R.key0, R.key1}, X4 + q1 + Q,
                                         has2 ? X4 + q2 + Q : nullptr, Acc2{acc1, acc2}, mh, d);
        acc1 = a.a1;
        acc2 = a.a2;
      }
    }
  }
  // ---- mutation pass: the sites of this segment ----------------------------
  // (32-lane teams leave their sites to k_mutate, except when every variable
  // mutates)
  __syncwarp();   // the crossed rows are visible to the whole team
  if (active && R.T_m > 0 && (TS < 32 || R.T_m >= (1u << 24))) {
    for (int c = lane; c < 2; c += TS) {
      if (c == 1 && !has2) break;
      const float dg = mutate_sites<PROB>(R, KeyRun{R.key0, R.key1}, c ? p + P : p,
                                          c ? ch2 : ch1, t, 8 * g0, 8 * gE);
      if (c == 0) acc1.x += dg; else acc2.x += dg;
    }
  } else if (active && R.T_m == 0 && TS < 32 && R.rec_sites && lane < 2 && (lane == 0 || has2)) {
    R.rec_sites[(size_t)(lane ? p + P : p) * (1 + kMaxSites)] = 0;   // no site fires
  }
  if (PROB == PROB_NEURO) return;   // objectives come from the rollout kernel

  // ---- combine: team sum; one segment finishes here, several in k_mutate --
  const float2 gs = team_sum2(make_float2(acc1.x + acc1.y, acc2.x + acc2.y), TS);
  __syncwarp();   // the team's mutations are visible to its leader
  if (active && lane == 0) {
    if (TS == 32) {
      float *ps = R.psum + (size_t)p * 2 * S;
      ps[seg] = gs.x;
      ps[S + seg] = gs.y;
    } else {
      finish_pair<PROB>(R, gs.x, gs.y, ch1, ch2, s_zmin);
    }
  }
  if (evals) {
    __syncthreads();
    if (threadIdx.x < R.m && s_zmin[threadIdx.x] != 0xFFFFFFFFu)
      atomicMin(&R.ctl->zkey[threadIdx.x], s_zmin[threadIdx.x]);
  }
}

// One run of a known problem: the Philox round keys come in the parameter
// block.  The _s instances stage the parent rows in shared memory (teams of
// 32 lanes, d > 1024); the others load them directly.
#define RVEA_REPRO1(name, PROB, STAGED)                                                    \
  __global__ void __launch_bounds__(kReproThreads, 4)                                      \
  name(const __grid_constant__ BatchDir dir, const __grid_constant__ RoundKeys rk) {       \
    repro_body<PROB, STAGED>(dir, KeyConst{rk});                                           \
  }
RVEA_REPRO1(k_repro1_dtlz1, PROB_DTLZ1, false)
RVEA_REPRO1(k_repro1_dtlz2, PROB_DTLZ2, false)
RVEA_REPRO1(k_repro1_dtlz3, PROB_DTLZ3, false)
RVEA_REPRO1(k_repro1_dtlz4, PROB_DTLZ4, false)
RVEA_REPRO1(k_repro1_neuro, PROB_NEURO, false)
RVEA_REPRO1(k_repro1s_dtlz1, PROB_DTLZ1, true)
RVEA_REPRO1(k_repro1s_dtlz2, PROB_DTLZ2, true)
RVEA_REPRO1(k_repro1s_dtlz3, PROB_DTLZ3, true)
RVEA_REPRO1(k_repro1s_dtlz4, PROB_DTLZ4, true)
RVEA_REPRO1(k_repro1s_neuro, PROB_NEURO, true)
#undef RVEA_REPRO1

// A batch of runs of one problem and one load path: each CTA's round keys
// follow from its run's key.  The host launches one instance per (problem,
// load path) group present in the batch.
#define RVEA_REPROB(name, PROB, STAGED)                                                    \
  __global__ void __launch_bounds__(kReproThreads, 4) name(const __grid_constant__ BatchDir dir) { \
    const int run = dir_find(dir, blockIdx.x);                                             \
    repro_body<PROB, STAGED>(dir, KeyRun{dir.key[run].x, dir.key[run].y});                 \
  }
RVEA_REPROB(k_reprob_dtlz1, PROB_DTLZ1, false)
RVEA_REPROB(k_reprob_dtlz2, PROB_DTLZ2, false)
RVEA_REPROB(k_reprob_dtlz3, PROB_DTLZ3, false)
RVEA_REPROB(k_reprob_dtlz4, PROB_DTLZ4, false)
RVEA_REPROB(k_reprob_neuro, PROB_NEURO, false)
RVEA_REPROB(k_reprob_dtlz1s, PROB_DTLZ1, true)
RVEA_REPROB(k_reprob_dtlz2s, PROB_DTLZ2, true)
RVEA_REPROB(k_reprob_dtlz3s, PROB_DTLZ3, true)
RVEA_REPROB(k_reprob_dtlz4s, PROB_DTLZ4, true)
RVEA_REPROB(k_reprob_neuros, PROB_NEURO, true)
#undef RVEA_REPROB

// Mutation and evaluation of the children of runs reproduced by 32-lane
// teams (d > 1024), after their reproduction kernel: one thread per child
// (draw index cd: child 1 of pair cd, or child 2 of pair cd - P), with the
// same count-then-subset sites as mutate_sites; g is the pair's segment
// partials in segment order plus the sites' term changes in draw order; then
// the objectives and the ideal point.  Moving this tail out of the
// reproduction kernel leaves its warps no serial per-pair chain and no
// cross-warp arrival.  A warp first draws its 32 children's sites into
// shared memory, then mutates them spread over its lanes (about one round of
// 32 for one site per row on average), so a child with several sites does
// not hold up the others.  Everything that does not read this generation's
// children (slots, site draws, magnitudes) runs before the wait for the
// reproduction kernel, overlapping its tail; the kernel lets its successor
// launch at once (the successor's own wait still orders it after this grid,
// and so after the reproduction kernel).  When every variable mutates
// (per-site probability 1) the reproduction kernel has already mutated.
struct MutShared {
  uint32_t j[kMutThreads / 32][32 * kMaxSites];   // site variable
  float dg[kMutThreads / 32][32 * kMaxSites];     // magnitude M, then term(new) - term(old)
  uint8_t own[kMutThreads / 32][32 * kMaxSites];  // lane of the child
  int slot[kMutThreads / 32][32];
  unsigned zmin[kMutThreads / 32][kMaxM];
};

template <int PROB>
__device__ __forceinline__ void mutate_body(const BatchDir &dir) {
  pdl_trigger();
  __shared__ MutShared sh;
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cd0 = (blockIdx.x - dir.prefix[run]) * kMutThreads + warp * 32, cd = cd0 + lane;
  const int N = R.N, P = R.P, m = R.m, d = R.d;
  // generation counter and child slots: written by the previous generation's
  // finalize, which completed before the reproduction kernel (this grid's
  // predecessor) passed its own wait; read through L2
  const int t = __ldcg(&R.ctl->t);
  const KeyRun kr{R.key0, R.key1};
  int slot = -1;
  if (cd < N) {
    slot = __ldcg(R.child_slot + (t & 1) * N + cd);
    if (slot < 0 || slot >= 2 * N) { set_status(R.ctl, ST_BADINDEX); slot = -1; }
  }
  sh.slot[warp][lane] = slot;
  // ---- the sites: count k ~ Binomial(d, q), then Floyd's subset -----------
  int k = 0;
  if (slot >= 0 && R.T_m > 0 && R.T_m < (1u << 24)) {
    uint4 w = philox_k(0u, (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr);
    const int nthr = R.n_mthr;
    while (k < nthr && w.x >= R.mthr[k]) ++k;
  }
  int incl = k;   // warp prefix of the counts: this child's entries start at off
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int off = incl - k, total = __shfl_sync(0xffffffffu, incl, 31);
  if (k > 0) {
    uint32_t *const js = sh.j[warp] + off;
    uint4 w = philox_k(0u, (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr);
    for (int i = 0; i < k; ++i) {
      const int e = i + 1;
      if ((e & 3) == 0) w = philox_k((uint32_t)(e >> 2), (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr);
      const uint32_t J = (uint32_t)(d - k + i);
      uint32_t r = __umulhi(word(w, e & 3), J + 1u);
      for (int l = 0; l < i; ++l)
        if (js[l] == r) { r = J; break; }
      js[i] = r;
      sh.own[warp][off + i] = (uint8_t)lane;
    }
  }
  if (R.rec_sites && slot >= 0) {
    int *const rec = R.rec_sites + (size_t)cd * (1 + kMaxSites);
    rec[0] = R.T_m >= (1u << 24) ? -1 : k;
    for (int i = 0; i < k; ++i) rec[1 + i] = (int)sh.j[warp][off + i];
  }
  __syncwarp();
  for (int e = lane; e < total; e += 32) {   // the magnitudes
    const uint4 w = philox_k(sh.j[warp][e], (uint32_t)(cd0 + sh.own[warp][e]), (uint32_t)t,
                             TAG_MUTMAG, kr);
    sh.dg[warp][e] = u24f(w.y);
  }
  __syncwarp();
  pdl_wait();      // the crossed children of this generation
  // ---- the mutations, one site a lane ------------------------------------
  for (int e = lane; e < total; e += 32) {
    const int o = sh.own[warp][e];
    const uint32_t j = sh.j[warp][e];
    float *const px = R.X + (size_t)sh.slot[warp][o] * R.d_pad + j;
    const float x = __ldcg(px);
    const float xn = poly_mutate(x, sh.dg[warp][e], R.L, R.U, R.eta_m);
    __stcg(px, xn);
    sh.dg[warp][e] = (PROB != PROB_NEURO && (int)j >= m - 1)
                         ? g_term1(PROB, xn, 0.0f) - g_term1(PROB, x, 0.0f) : 0.0f;
  }
  __syncwarp();   // the mutated rows and term changes are visible to the warp
  if (PROB == PROB_NEURO) return;   // objectives come from the rollout kernel
  float f[kMaxM];
  if (slot >= 0) {
    float dg = 0.0f;
    for (int i = 0; i < k; ++i) dg += sh.dg[warp][off + i];
    const int S = R.nseg, p = cd < P ? cd : cd - P;
    const float *ps = R.psum + (size_t)p * 2 * S + (cd < P ? 0 : S);
    float g = 0.0f;
    for (int q = 0; q < S; ++q) g += __ldcg(ps + q);
    const float *row = R.X + (size_t)slot * R.d_pad;
    float head[kMaxM];
    for (int jj = 0; jj < m - 1; ++jj) head[jj] = __ldcg(row + jj);
    dtlz_objectives_t<PROB>(m, g + dg, head, f);
    for (int kk = 0; kk < m; ++kk) R.F[(size_t)kk * 2 * N + slot] = f[kk];
  }
  // the ideal point: a CTA's minimum per objective, then one atomic each
  for (int kk = 0; kk < m; ++kk) {
    const unsigned v = __reduce_min_sync(0xffffffffu, slot >= 0 ? f2ord(f[kk]) : 0xFFFFFFFFu);
    if (lane == 0) sh.zmin[warp][kk] = v;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    unsigned v = 0xFFFFFFFFu;
    for (int w = 0; w < kMutThreads / 32; ++w) v = min(v, sh.zmin[w][threadIdx.x]);
    if (v != 0xFFFFFFFFu) atomicMin(&R.ctl->zkey[threadIdx.x], v);
  }
}
#define RVEA_MUTATE(name, PROB)                                                            \
  __global__ void __launch_bounds__(kMutThreads) name(const __grid_constant__ BatchDir dir) { \
    mutate_body<PROB>(dir);                                                                \
  }
RVEA_MUTATE(k_mutate_dtlz1, PROB_DTLZ1)
RVEA_MUTATE(k_mutate_dtlz2, PROB_DTLZ2)
RVEA_MUTATE(k_mutate_dtlz3, PROB_DTLZ3)
RVEA_MUTATE(k_mutate_dtlz4, PROB_DTLZ4)
RVEA_MUTATE(k_mutate_neuro, PROB_NEURO)
#undef RVEA_MUTATE

// Reproduction by the other operators of the extensibility experiment
// (Sec. 4.4 and Appendix C; the paper names them, this follows the published
// operators): DE/rand/1/bin (Storn and Price 1997) or random reproduction.
// They replace SBX and polynomial mutation and make the N offspring rows
// directly.  One warp per offspring o:
//   DE: the target is position o mod K of the valid list, r1, r2, r3 an
//       ordered triple of other distinct positions drawn one after another
//       without replacement from DE_PICK (o, 0, t) words 0..2, j_rand from
//       word 3; u_j = x_r1,j + F (x_r2,j - x_r3,j) where the CR coin of j
//       (DE_CR (j/4, o, t) word j%4, u24 < CR on the 24-bit grid) fires or
//       j = j_rand, else the target's x_j; clipped to [L, U];
//   random: x_j = L + (U - L) u24, RANDOM (j/4, o, t) word j%4.
// Then the g-terms, objectives and the ideal point, as the other kernels.
enum : uint32_t { TAG_DE_PICK = 8, TAG_DE_CR = 9, TAG_RANDOM = 10, TAG_CSO_PICK = 11, TAG_CSO_R = 12,
                  TAG_PSO_PICK = 13, TAG_PSO_R = 14 };

__device__ __forceinline__ int de_pos(uint32_t w, int n) { return (int)__umulhi(w, (uint32_t)n); }

// The g-terms of float4 Q of a child row into acc (x: its even variables, y:
// its odd ones), the position variables j < mh left out.  Past them, two
// packed steps (g_terms2 is g_term1 on each lane, and the row padding, 0.5,
// adds an exact zero), else element by element: the same bits either way.
template <int PROB>
__device__ __forceinline__ float2 gterms4(const float *u, int Q, int mh, int d, float2 acc) {
  if (4 * Q >= mh) {
    acc = g_terms2(PROB, make_float2(u[0], u[1]), acc);
    return g_terms2(PROB, make_float2(u[2], u[3]), acc);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int j = 4 * Q + v;
    if (j >= mh && j < d) {
      if (v & 1) acc.y = g_term1(PROB, u[v], acc.y);
      else acc.x = g_term1(PROB, u[v], acc.x);
    }
  }
  return acc;
}

template <int PROB, int OP>   // OP 1: DE/rand/1/bin, 2: random reproduction
__device__ __forceinline__ void repro_op_body(const BatchDir &dir) {
  __shared__ unsigned s_z[kMaxM];
  pdl_wait();      // the previous generation's lists and slot maps
  pdl_trigger();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o = (blockIdx.x - dir.prefix[run]) * (kReproThreads / 32) + warp;
  const int N = R.N, d = R.d, m = R.m, t = R.ctl->t, K = R.ctl->K;
  const KeyRun kr{dir.key[run].x, dir.key[run].y};
  if (threadIdx.x < kMaxM) s_z[threadIdx.x] = 0xFFFFFFFFu;
  __syncthreads();
  float f[kMaxM];
  bool have = false;
  if (o < N) {
    int slot = R.child_slot[(t & 1) * N + o];
    if (slot < 0 || slot >= 2 * N) { set_status(R.ctl, ST_BADINDEX); slot = -1; }
    // DE: the four rows (physical slots) and j_rand, drawn by lane 0
    int rows[4] = {0, 0, 0, 0}, jr = -1;
    if (OP == 1 && lane == 0 && K > 0) {
      const uint4 w = philox_k((uint32_t)o, 0u, (uint32_t)t, TAG_DE_PICK, kr);
      const int tp = o % K;
      int pos[4];
      pos[0] = tp;
      if (K >= 4) {
        const int a = de_pos(w.x, K - 1);
        int bq = de_pos(w.y, K - 2), c = de_pos(w.z, K - 3);
        if (bq >= a) bq += 1;
        const int lo = min(a, bq), hi = max(a, bq);
        if (c >= lo) c += 1;
        if (c >= hi) c += 1;
        pos[1] = a < tp ? a : a + 1;
        pos[2] = bq < tp ? bq : bq + 1;
        pos[3] = c < tp ? c : c + 1;
      } else {
        pos[1] = de_pos(w.x, K);
        pos[2] = de_pos(w.y, K);
        pos[3] = de_pos(w.z, K);
      }
      jr = de_pos(w.w, d);
      for (int q = 0; q < 4; ++q) {
        const int j = R.vlist[pos[q]];
        int sl = (j >= 0 && j < N) ? R.slotmap[(t & 1) * N + j] : -1;
        if (sl < 0 || sl >= 2 * N) { set_status(R.ctl, ST_BADINDEX); sl = 0; }
        rows[q] = sl;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) rows[q] = __shfl_sync(0xffffffffu, rows[q], 0);
    jr = __shfl_sync(0xffffffffu, jr, 0);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    float2 acc = make_float2(0.f, 0.f);
    if (slot >= 0) {
      const float L = R.L, U = R.U, Fde = R.de_F;
      const int mh = m - 1;
      const float4 *X4 = reinterpret_cast<const float4 *>(R.X);
      float4 *Y4 = reinterpret_cast<float4 *>(R.X + (size_t)slot * R.d_pad);
      const int rq = R.d_pad >> 2;
      // DE: the four rows streamed in, the next float4s loaded while the
      // current ones are processed (four more loads in flight per lane)
      const float4 *T0 = X4 + (size_t)rows[0] * rq, *T1 = X4 + (size_t)rows[1] * rq;
      const float4 *T2 = X4 + (size_t)rows[2] * rq, *T3 = X4 + (size_t)rows[3] * rq;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 c0 = z4, c1 = z4, c2 = z4, c3 = z4;
      if (OP == 1 && lane < rq) {
        c0 = __ldg(T0 + lane);
        c1 = __ldg(T1 + lane);
        c2 = __ldg(T2 + lane);
        c3 = __ldg(T3 + lane);
      }
      for (int Q = lane; Q < rq; Q += 32) {
        float u[4];
        if (OP == 1) {
          float4 n0 = z4, n1 = z4, n2 = z4, n3 = z4;
          if (Q + 32 < rq) {
            n0 = __ldg(T0 + Q + 32);
            n1 = __ldg(T1 + Q + 32);
            n2 = __ldg(T2 + Q + 32);
            n3 = __ldg(T3 + Q + 32);
          }
          const uint4 w = philox_k((uint32_t)Q, (uint32_t)o, (uint32_t)t, TAG_DE_CR, kr);
          const float a0[4] = {c0.x, c0.y, c0.z, c0.w}, a1[4] = {c1.x, c1.y, c1.z, c1.w};
          const float a2[4] = {c2.x, c2.y, c2.z, c2.w}, a3[4] = {c3.x, c3.y, c3.z, c3.w};
          const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int j = 4 * Q + v;
            const bool take = (ww[v] >> 8) < R.T_cr || j == jr;
            const float val = take ? fmaf(Fde, a2[v] - a3[v], a1[v]) : a0[v];
            u[v] = clampf(val, L, U);
          }
          c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        } else {
          const uint4 w = philox_k((uint32_t)Q, (uint32_t)o, (uint32_t)t, TAG_RANDOM, kr);
          const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int v = 0; v < 4; ++v) u[v] = L + (U - L) * u24f(ww[v]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (4 * Q + v >= d) u[v] = 0.5f;   // row padding: a g-term of exactly zero
        acc = gterms4<PROB>(u, Q, mh, d, acc);
        Y4[Q] = make_float4(u[0], u[1], u[2], u[3]);
      }
      const float2 gs = team_sum2(acc, 32);
      __syncwarp();   // the row is visible to lane 0
      if (lane == 0) {
        float head[kMaxM];
        const float *row = R.X + (size_t)slot * R.d_pad;
        for (int jj = 0; jj < mh; ++jj) head[jj] = __ldcg(row + jj);
        dtlz_objectives_t<PROB>(m, gs.x + gs.y, head, f);
        for (int kk = 0; kk < m; ++kk) R.F[(size_t)kk * 2 * N + slot] = f[kk];
        have = true;
      }
    }
  }
  if (have)
    for (int kk = 0; kk < m; ++kk) atomicMin(&s_z[kk], f2ord(f[kk]));
  __syncthreads();
  if (threadIdx.x < m && s_z[threadIdx.x] != 0xFFFFFFFFu)
    atomicMin(&R.ctl->zkey[threadIdx.x], s_z[threadIdx.x]);
}
// The swarm centre of the CSO operator, xbar = the mean position of the K
// valid members (the oracle's order: a sum over the valid list, then / K),
// in two launches.  k_cso_mean: CTA (chunk, column block) adds the rows
// [kMeanRows chunk, +kMeanRows) of the valid list over its kMeanCols
// variables in float, in list order, into xpart (grid per run: column blocks
// x ceil(N / kMeanRows) chunks; chunks past K write zeros).  k_cso_centre:
// one warp per float4 of variables adds the chunks' partials in FP64, lane l
// taking chunks l, l + 32, ... in order and the lanes combined by a fixed
// butterfly, then divides by K: the same bits on every run.
__global__ void __launch_bounds__(256) k_cso_mean(const __grid_constant__ BatchDir dir) {
  __shared__ int s_rows[kMeanRows];
  pdl_wait();      // the previous generation's lists and slot maps
  pdl_trigger();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int N = R.N, t = R.ctl->t, K = R.ctl->K;
  const int rq = R.d_pad >> 2;
  const int ncb = (R.d_pad + kMeanCols - 1) / kMeanCols;
  const int b = blockIdx.x - dir.prefix[run];
  const int cb = b % ncb, ch = b / ncb;
  const int r0 = ch * kMeanRows, nr = max(0, min(kMeanRows, K - r0));
  if (threadIdx.x < kMeanRows) {
    int s = 0;
    if ((int)threadIdx.x < nr) {
      const int j = R.vlist[r0 + threadIdx.x];
      s = (j >= 0 && j < N) ? R.slotmap[(t & 1) * N + j] : -1;
      if (s < 0 || s >= 2 * N) { set_status(R.ctl, ST_BADINDEX); s = 0; }
    }
    s_rows[threadIdx.x] = s;
  }
  __syncthreads();
  const int Q = cb * (kMeanCols / 4) + (int)threadIdx.x;
  if (Q >= rq) return;
  const float4 *X4 = reinterpret_cast<const float4 *>(R.X);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
  for (int r = 0; r < nr; ++r) {
    const float4 x = __ldcs(X4 + (size_t)s_rows[r] * rq + Q);
    acc.x += x.x; acc.y += x.y; acc.z += x.z; acc.w += x.w;
  }
  reinterpret_cast<float4 *>(R.xpart)[(size_t)ch * rq + Q] = acc;
}

__global__ void __launch_bounds__(256) k_cso_centre(const __grid_constant__ BatchDir dir) {
  pdl_wait();      // the partial sums
  pdl_trigger();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int lane = threadIdx.x & 31;
  const int Q = (blockIdx.x - dir.prefix[run]) * 8 + (int)(threadIdx.x >> 5);
  const int rq = R.d_pad >> 2;
  if (Q >= rq) return;   // warp-uniform
  const int K = R.ctl->K;
  const int nk = (K + kMeanRows - 1) / kMeanRows;
  const float4 *P4 = reinterpret_cast<const float4 *>(R.xpart);
  double sx = 0.0, sy = 0.0, sz = 0.0, sw = 0.0;
  for (int c = lane; c < nk; c += 32) {
    const float4 p = __ldcg(P4 + (size_t)c * rq + Q);
    sx += p.x; sy += p.y; sz += p.z; sw += p.w;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
    sz += __shfl_xor_sync(0xffffffffu, sz, off);
    sw += __shfl_xor_sync(0xffffffffu, sw, off);
  }
  if (lane == 0) {
    const double k = (double)max(K, 1);
    reinterpret_cast<float4 *>(R.xbar)[Q] =
        make_float4((float)(sx / k), (float)(sy / k), (float)(sz / k), (float)(sw / k));
  }
}

#define RVEA_REPRO_OP(name, PROB, OP)                                                      \
  __global__ void __launch_bounds__(kReproThreads) name(const __grid_constant__ BatchDir dir) { \
    repro_op_body<PROB, OP>(dir);                                                          \
  }
RVEA_REPRO_OP(k_repro_de_dtlz1, PROB_DTLZ1, 1)
RVEA_REPRO_OP(k_repro_de_dtlz2, PROB_DTLZ2, 1)
RVEA_REPRO_OP(k_repro_de_dtlz3, PROB_DTLZ3, 1)
RVEA_REPRO_OP(k_repro_de_dtlz4, PROB_DTLZ4, 1)
RVEA_REPRO_OP(k_repro_rand_dtlz1, PROB_DTLZ1, 2)
RVEA_REPRO_OP(k_repro_rand_dtlz2, PROB_DTLZ2, 2)
RVEA_REPRO_OP(k_repro_rand_dtlz3, PROB_DTLZ3, 2)
RVEA_REPRO_OP(k_repro_rand_dtlz4, PROB_DTLZ4, 2)
#undef RVEA_REPRO_OP

// Reproduction by the competitive swarm optimizer (CSO; Cheng and Jin 2015),
// the operator the paper's neuroevolution experiment picks (Sec. 4.4).  One
// warp per offspring o: a competition between two distinct valid members,
// positions a then b of the valid list (CSO_PICK (o, 0, t) words 0 and 1, b
// drawn over the positions other than a); the smaller kept APD wins (ties:
// the smaller slot), and the loser learns
//   v' = r1 v_l + r2 (x_w - x_l) + phi r3 (xbar - x_l),   x' = x_l + v',
// r1, r2, r3 of variable j from word j%4 of CSO_R (3 (j/4) + k, o, t),
// k = 0, 1, 2 (r3 only when phi > 0), xbar the swarm centre (k_cso_mean);
// x' is clipped to [L, U] and (x', v') goes to the child's pool row and its
// velocity row.  Each lane streams float4s of the winner's and loser's rows
// and the loser's velocity, the next float4s loaded while the current ones
// are processed (the centre, read by every offspring, comes from L1 / L2).  Then the g-terms, objectives and the ideal point.
template <int PROB>
__device__ __forceinline__ void repro_cso_body(const BatchDir &dir) {
  __shared__ unsigned s_z[kMaxM];
  pdl_wait();      // the previous generation's lists, slot maps and kept APDs; the centre
  pdl_trigger();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o = (blockIdx.x - dir.prefix[run]) * (kReproThreads / 32) + warp;
  const int N = R.N, d = R.d, m = R.m, t = R.ctl->t, K = R.ctl->K;
  const KeyRun kr{dir.key[run].x, dir.key[run].y};
  if (threadIdx.x < kMaxM) s_z[threadIdx.x] = 0xFFFFFFFFu;
  __syncthreads();
  float f[kMaxM];
  bool have = false;
  if (o < N) {
    int slot = R.child_slot[(t & 1) * N + o];
    if (slot < 0 || slot >= 2 * N) { set_status(R.ctl, ST_BADINDEX); slot = -1; }
    int rw = 0, rl = 0;   // pool rows of the winner and the loser
    if (lane == 0 && K > 0) {
      const uint4 w = philox_k((uint32_t)o, 0u, (uint32_t)t, TAG_CSO_PICK, kr);
      const int a = de_pos(w.x, K);
      int bq = a;
      if (K > 1) {
        bq = de_pos(w.y, K - 1);
        if (bq >= a) bq += 1;
      }
      int ia = R.vlist[a], ib = R.vlist[bq];
      if (ia < 0 || ia >= N || ib < 0 || ib >= N) { set_status(R.ctl, ST_BADINDEX); ia = ib = 0; }
      const float pa = R.kapd[ia], pb = R.kapd[ib];
      const bool a_wins = pa < pb || (pa == pb && ia <= ib);
      rw = R.slotmap[(t & 1) * N + (a_wins ? ia : ib)];
      rl = R.slotmap[(t & 1) * N + (a_wins ? ib : ia)];
      if (rw < 0 || rw >= 2 * N || rl < 0 || rl >= 2 * N) { set_status(R.ctl, ST_BADINDEX); rw = rl = 0; }
    }
    rw = __shfl_sync(0xffffffffu, rw, 0);
    rl = __shfl_sync(0xffffffffu, rl, 0);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    float2 acc = make_float2(0.f, 0.f);
    if (slot >= 0) {
      const float L = R.L, U = R.U, phi = R.cso_phi;
      const int mh = m - 1, rq = R.d_pad >> 2;
      const float4 *X4 = reinterpret_cast<const float4 *>(R.X);
      const float4 *V4 = reinterpret_cast<const float4 *>(R.vel);
      const float4 *XW = X4 + (size_t)rw * rq, *XL = X4 + (size_t)rl * rq, *VL = V4 + (size_t)rl * rq;
      const float4 *XB = reinterpret_cast<const float4 *>(R.xbar);
      float4 *Y4 = reinterpret_cast<float4 *>(R.X + (size_t)slot * R.d_pad);
      float4 *VY = reinterpret_cast<float4 *>(R.vel + (size_t)slot * R.d_pad);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 cw = z4, cl = z4, cv = z4;
      if (lane < rq) {
        cw = __ldg(XW + lane);
        cl = __ldg(XL + lane);
        cv = __ldg(VL + lane);
      }
      for (int Q = lane; Q < rq; Q += 32) {
        float4 nw = z4, nl = z4, nv = z4;
        if (Q + 32 < rq) {
          nw = __ldg(XW + Q + 32);
          nl = __ldg(XL + Q + 32);
          nv = __ldg(VL + Q + 32);
        }
        // the centre (d_pad floats, shared by every offspring) stays in L1 / L2
        const float4 cb = phi != 0.0f ? __ldg(XB + Q) : z4;
        const float aw[4] = {cw.x, cw.y, cw.z, cw.w}, al[4] = {cl.x, cl.y, cl.z, cl.w};
        const float av[4] = {cv.x, cv.y, cv.z, cv.w}, ab[4] = {cb.x, cb.y, cb.z, cb.w};
        // the three terms in turn, one Philox call each (one call's words live at a time)
        float vv[4];
        {
          const uint4 w = philox_k(3u * (uint32_t)Q, (uint32_t)o, (uint32_t)t, TAG_CSO_R, kr);
#pragma unroll
          for (int v = 0; v < 4; ++v) vv[v] = u24f(word(w, v)) * av[v];
        }
        {
          const uint4 w = philox_k(3u * (uint32_t)Q + 1u, (uint32_t)o, (uint32_t)t, TAG_CSO_R, kr);
#pragma unroll
          for (int v = 0; v < 4; ++v) vv[v] = fmaf(u24f(word(w, v)), aw[v] - al[v], vv[v]);
        }
        if (phi != 0.0f) {
          const uint4 w = philox_k(3u * (uint32_t)Q + 2u, (uint32_t)o, (uint32_t)t, TAG_CSO_R, kr);
#pragma unroll
          for (int v = 0; v < 4; ++v) vv[v] = fmaf(phi * u24f(word(w, v)), ab[v] - al[v], vv[v]);
        }
        float u[4], nvel[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int j = 4 * Q + v;
          if (j >= d) {   // row padding: a g-term of exactly zero, no velocity
            u[v] = 0.5f;
            nvel[v] = 0.0f;
          } else {
            u[v] = clampf(al[v] + vv[v], L, U);
            nvel[v] = vv[v];
          }
        }
        if (PROB != PROB_NEURO) acc = gterms4<PROB>(u, Q, mh, d, acc);
        Y4[Q] = make_float4(u[0], u[1], u[2], u[3]);
        __stcs(VY + Q, make_float4(nvel[0], nvel[1], nvel[2], nvel[3]));
        cw = nw; cl = nl; cv = nv;
      }
      const float2 gs = team_sum2(acc, 32);
      __syncwarp();   // the row is visible to lane 0
      // the rollout problem's children are evaluated by the rollout kernel
      if (PROB != PROB_NEURO && lane == 0) {
        float head[kMaxM];
        const float *row = R.X + (size_t)slot * R.d_pad;
        for (int jj = 0; jj < mh; ++jj) head[jj] = __ldcg(row + jj);
        dtlz_objectives_t<PROB>(m, gs.x + gs.y, head, f);
        for (int kk = 0; kk < m; ++kk) R.F[(size_t)kk * 2 * N + slot] = f[kk];
        have = true;
      }
    }
  }
  if (have)
    for (int kk = 0; kk < m; ++kk) atomicMin(&s_z[kk], f2ord(f[kk]));
  __syncthreads();
  if (threadIdx.x < m && s_z[threadIdx.x] != 0xFFFFFFFFu)
    atomicMin(&R.ctl->zkey[threadIdx.x], s_z[threadIdx.x]);
}
#define RVEA_REPRO_CSO(name, PROB)                                                         \
  __global__ void __launch_bounds__(kReproThreads, 3) name(const __grid_constant__ BatchDir dir) { \
    repro_cso_body<PROB>(dir);                                                             \
  }
RVEA_REPRO_CSO(k_repro_cso_dtlz1, PROB_DTLZ1)
RVEA_REPRO_CSO(k_repro_cso_dtlz2, PROB_DTLZ2)
RVEA_REPRO_CSO(k_repro_cso_dtlz3, PROB_DTLZ3)
RVEA_REPRO_CSO(k_repro_cso_dtlz4, PROB_DTLZ4)
RVEA_REPRO_CSO(k_repro_cso_neuro, PROB_NEURO)
#undef RVEA_REPRO_CSO

// Reproduction by particle swarm optimization (PSO; Kennedy and Eberhart
// 1995, the inertia weight of Shi and Eberhart 1998, the personal-best rule
// of the multiobjective PSO of Coello, Pulido and Lechuga 2004).  One warp
// per offspring o: the particle is the member at position o mod K of the
// valid list, its leader the winner of a binary tournament on the kept APD
// between two distinct valid members (PSO_PICK (o, 0, t) words 0 and 1; ties:
// the smaller slot), and it moves
//   v' = w v + c1 r1 (p - x) + c2 r2 (g - x),   x' = clip(x + v'),
// r1, r2 of variable j from word j%4 of PSO_R (2 (j/4) + k, o, t), k = 0, 1.
// (x', v') goes to the child's pool row and velocity row, and x' to its
// personal-best row; after the evaluation, when the particle's personal
// best dominates f(x') (no worse in every objective, better in one), the
// warp copies that best (row and objectives) over the child's instead.
template <int PROB>
__device__ __forceinline__ void repro_pso_body(const BatchDir &dir) {
  __shared__ unsigned s_z[kMaxM];
  pdl_wait();      // the previous generation's lists, slot maps and kept APDs
  pdl_trigger();
  const int run = dir_find(dir, blockIdx.x);
  const RunDesc &R = *dir.desc[run];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o = (blockIdx.x - dir.prefix[run]) * (kReproThreads / 32) + warp;
  const int N = R.N, d = R.d, m = R.m, t = R.ctl->t, K = R.ctl->K, n2 = 2 * N;
  const KeyRun kr{dir.key[run].x, dir.key[run].y};
  if (threadIdx.x < kMaxM) s_z[threadIdx.x] = 0xFFFFFFFFu;
  __syncthreads();
  float f[kMaxM];
  bool have = false;
  if (o < N) {
    int slot = R.child_slot[(t & 1) * N + o];
    if (slot < 0 || slot >= n2) { set_status(R.ctl, ST_BADINDEX); slot = -1; }
    int rp = 0, rg = 0;   // pool rows of the particle and its leader
    if (lane == 0 && K > 0) {
      const uint4 w = philox_k((uint32_t)o, 0u, (uint32_t)t, TAG_PSO_PICK, kr);
      const int a = de_pos(w.x, K);
      int bq = a;
      if (K > 1) {
        bq = de_pos(w.y, K - 1);
        if (bq >= a) bq += 1;
      }
      int ip = R.vlist[o % K], ia = R.vlist[a], ib = R.vlist[bq];
      if (ip < 0 || ip >= N || ia < 0 || ia >= N || ib < 0 || ib >= N) {
        set_status(R.ctl, ST_BADINDEX);
        ip = ia = ib = 0;
      }
      const float pa = R.kapd[ia], pbv = R.kapd[ib];
      const int ig = (pa < pbv || (pa == pbv && ia <= ib)) ? ia : ib;
      rp = R.slotmap[(t & 1) * N + ip];
      rg = R.slotmap[(t & 1) * N + ig];
      if (rp < 0 || rp >= n2 || rg < 0 || rg >= n2) { set_status(R.ctl, ST_BADINDEX); rp = rg = 0; }
    }
    rp = __shfl_sync(0xffffffffu, rp, 0);
    rg = __shfl_sync(0xffffffffu, rg, 0);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    float2 acc = make_float2(0.f, 0.f);
    if (slot >= 0) {
      const float L = R.L, U = R.U, w = R.pso_w, c1 = R.pso_c1, c2 = R.pso_c2;
      const int mh = m - 1, rq = R.d_pad >> 2;
      const float4 *X4 = reinterpret_cast<const float4 *>(R.X);
      const float4 *XP = X4 + (size_t)rp * rq, *XG = X4 + (size_t)rg * rq;
      const float4 *VP = reinterpret_cast<const float4 *>(R.vel) + (size_t)rp * rq;
      const float4 *PP = reinterpret_cast<const float4 *>(R.pb) + (size_t)rp * rq;
      float4 *Y4 = reinterpret_cast<float4 *>(R.X + (size_t)slot * R.d_pad);
      float4 *VY = reinterpret_cast<float4 *>(R.vel + (size_t)slot * R.d_pad);
      float4 *PY = reinterpret_cast<float4 *>(R.pb + (size_t)slot * R.d_pad);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 cx = z4, cv = z4, cp = z4, cg = z4;
      if (lane < rq) {
        cx = __ldg(XP + lane);
        cv = __ldg(VP + lane);
        cp = __ldg(PP + lane);
        cg = __ldg(XG + lane);
      }
      for (int Q = lane; Q < rq; Q += 32) {
        float4 nx = z4, nv = z4, np = z4, ng = z4;
        if (Q + 32 < rq) {
          nx = __ldg(XP + Q + 32);
          nv = __ldg(VP + Q + 32);
          np = __ldg(PP + Q + 32);
          ng = __ldg(XG + Q + 32);
        }
        const float ax[4] = {cx.x, cx.y, cx.z, cx.w}, av[4] = {cv.x, cv.y, cv.z, cv.w};
        const float ap[4] = {cp.x, cp.y, cp.z, cp.w}, ag[4] = {cg.x, cg.y, cg.z, cg.w};
        float vv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) vv[v] = w * av[v];
        {
          const uint4 r = philox_k(2u * (uint32_t)Q, (uint32_t)o, (uint32_t)t, TAG_PSO_R, kr);
#pragma unroll
          for (int v = 0; v < 4; ++v) vv[v] = fmaf(c1 * u24f(word(r, v)), ap[v] - ax[v], vv[v]);
        }
        {
          const uint4 r = philox_k(2u * (uint32_t)Q + 1u, (uint32_t)o, (uint32_t)t, TAG_PSO_R, kr);
#pragma unroll
          for (int v = 0; v < 4; ++v) vv[v] = fmaf(c2 * u24f(word(r, v)), ag[v] - ax[v], vv[v]);
        }
        float u[4], nvel[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int j = 4 * Q + v;
          if (j >= d) {   // row padding: a g-term of exactly zero, no velocity
            u[v] = 0.5f;
            nvel[v] = 0.0f;
          } else {
            u[v] = clampf(ax[v] + vv[v], L, U);
            nvel[v] = vv[v];
          }
        }
        acc = gterms4<PROB>(u, Q, mh, d, acc);
        const float4 xo = make_float4(u[0], u[1], u[2], u[3]);
        Y4[Q] = xo;
        __stcs(VY + Q, make_float4(nvel[0], nvel[1], nvel[2], nvel[3]));
        PY[Q] = xo;
        cx = nx; cv = nv; cp = np; cg = ng;
      }
      const float2 gs = team_sum2(acc, 32);
      __syncwarp();   // the row is visible to lane 0
      int keep_old = 0;
      if (lane == 0) {
        float head[kMaxM];
        const float *row = R.X + (size_t)slot * R.d_pad;
        for (int jj = 0; jj < mh; ++jj) head[jj] = __ldcg(row + jj);
        dtlz_objectives_t<PROB>(m, gs.x + gs.y, head, f);
        bool le = true, lt = false;
        for (int kk = 0; kk < m; ++kk) {
          R.F[(size_t)kk * n2 + slot] = f[kk];
          const float fp = R.fpb[(size_t)kk * n2 + rp];
          le = le && fp <= f[kk];
          lt = lt || fp < f[kk];
        }
        keep_old = le && lt;
        for (int kk = 0; kk < m; ++kk)
          R.fpb[(size_t)kk * n2 + slot] = keep_old ? R.fpb[(size_t)kk * n2 + rp] : f[kk];
        have = true;
      }
      keep_old = __shfl_sync(0xffffffffu, keep_old, 0);
      if (keep_old)   // the particle's best stays its best: over the child's best row
        for (int Q = lane; Q < rq; Q += 32) PY[Q] = __ldg(PP + Q);
    }
  }
  if (have)
    for (int kk = 0; kk < m; ++kk) atomicMin(&s_z[kk], f2ord(f[kk]));
  __syncthreads();
  if (threadIdx.x < m && s_z[threadIdx.x] != 0xFFFFFFFFu)
    atomicMin(&R.ctl->zkey[threadIdx.x], s_z[threadIdx.x]);
}
#define RVEA_REPRO_PSO(name, PROB)                                                         \
  __global__ void __launch_bounds__(kReproThreads, 3) name(const __grid_constant__ BatchDir dir) { \
    repro_pso_body<PROB>(dir);                                                             \
  }
RVEA_REPRO_PSO(k_repro_pso_dtlz1, PROB_DTLZ1)
RVEA_REPRO_PSO(k_repro_pso_dtlz2, PROB_DTLZ2)
RVEA_REPRO_PSO(k_repro_pso_dtlz3, PROB_DTLZ3)
RVEA_REPRO_PSO(k_repro_pso_dtlz4, PROB_DTLZ4)
#undef RVEA_REPRO_PSO

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
        if (j >= d) x[v] = 0.5f;   // padding: a g-term of exactly zero on [0, 1]
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
