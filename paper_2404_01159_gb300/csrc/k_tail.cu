// Fused tail of a generation for one run: one persistent launch, one CTA per
// SM, that takes the children from the reproduction kernel to the next
// population (Algorithm 2, one loop iteration after X_cross):
//
//   A  mutation and evaluation of the children (Appendix B, C / X_mut, and
//      the DTLZ objectives; only for runs whose reproduction leaves them to a
//      second kernel, d > 1024), and their share of the ideal point z*
//      (Algorithm 1 lines 3-4);
//   -- grid barrier: z* is final --
//   B  association and APD votes (Algorithm 1 lines 5-15, Eqs. 2, 4): the
//      exact pruned search, its tables staged in shared memory by TMA while
//      the reproduction kernel still runs;
//   -- grid barrier: every vote is in --
//   C  decode of the per-vector minima into the next slot map (Algorithm 1
//      line 16), the valid bits, the pool rows the survivors occupy, the
//      survivors' objective minimum and maximum;
//   -- grid barrier: the decode is complete --
//   D  the ascending lists of valid slots (next mating) and free pool rows
//      (next offspring), from per-CTA counts published in C; the next z*;
//      on adaptation generations the FP64 rescaling of V (Algorithm 2,
//      "update reference vectors"); the control block.
//
// The arithmetic of every step is that of the separate kernels (k_mutate,
// k_select_pruned, k_finalize), so the results are the same bit for bit;
// only the launch boundaries, the last-CTA list building and the per-CTA
// arrival chain are gone.  The grid barriers wait with a time limit (1 s):
// a wait that gives up sets ST_TIMEOUT in the status word and its CTA
// returns, so a broken barrier ends in an error status, never in a hang.
// Every CTA is resident at once by construction (grid <= SM count, one
// 1024-thread CTA per SM), and the kernel lets its successor launch only
// after its last barrier.
//
// Data written by another CTA inside this launch is read through L2
// (__ldcg) after the barrier that orders it.
#include "eval_steps.cuh"
#include "grid_steps.cuh"

namespace rvea {

constexpr unsigned long long kBarrierNs = 1000000000ull;   // 1 s
constexpr int kTailFreeWords = 64;   // pool-row words (32 rows each) per CTA, at most

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long add_release_gpu(unsigned long long *p,
                                                              unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier over the launch's nb CTAs (all resident).  The arrival
// counter only grows: every launch adds exactly 3 nb, so an instance's
// arrivals are the nb values [k nb, (k + 1) nb) and it is complete once the
// counter reaches `target` = (k + 1) nb.  The launch reads the counter once
// before its first arrival (floor to a multiple of nb: the launch's base)
// and derives its three targets, so that an arrival is one release-add
// with no reply to wait for, then acquire polls; no reset, so nothing is
// serialised behind the last arrival.  Returns false, for the whole CTA,
// when the wait gave up.
__device__ __forceinline__ void red_release_gpu(unsigned long long *p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ bool grid_barrier(Ctl *ctl, unsigned long long target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_gpu(&ctl->bar, 1ull);
    if (ld_acquire_gpu(&ctl->bar) < target) {
      const unsigned long long t0 = global_ns();
      for (unsigned it = 1;; ++it) {
        if (ld_acquire_gpu(&ctl->bar) >= target) break;
        if ((it & 63u) == 0 && global_ns() - t0 > kBarrierNs) {
          ok = 0;
          set_status(ctl, ST_TIMEOUT);
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Phase A (the same draws and operations as k_mutate): the path of a child
// with more sites than its group has lanes: the draws again, the mutations
// one after another; returns the change of the child's g sum.
template <int PROB, int M>
__device__ __noinline__ float child_serial(const RunDesc &R, const KeyRun kr, int cd, int t,
                                           int slot, int k) {
  const int d = R.d;
  int js[kMaxSites];
  uint4 w = philox_k(0u, (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr);
  for (int i = 0; i < k; ++i) {
    const int e = i + 1;
    if ((e & 3) == 0) w = philox_k((uint32_t)(e >> 2), (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr);
    const uint32_t J = (uint32_t)(d - k + i);
    uint32_t r = __umulhi(word(w, e & 3), J + 1u);
    for (int l = 0; l < i; ++l)
      if ((uint32_t)js[l] == r) { r = J; break; }
    js[i] = (int)r;
  }
  if (R.rec_sites) {
    int *const rec = R.rec_sites + (size_t)cd * (1 + kMaxSites);
    rec[0] = k;
    for (int i = 0; i < k; ++i) rec[1 + i] = js[i];
  }
  float *const row = R.X + (size_t)slot * R.d_pad;
  float dg = 0.0f;
  for (int i = 0; i < k; ++i) {
    const int j = js[i];
    const float Mm = u24f(philox_k((uint32_t)j, (uint32_t)cd, (uint32_t)t, TAG_MUTMAG, kr).y);
    const float x = __ldcg(row + j);
    const float xn = poly_mutate(x, Mm, R.L, R.U, R.eta_m);
    __stcg(row + j, xn);
    dg += j >= M - 1 ? g_term1(PROB, xn, 0.0f) - g_term1(PROB, x, 0.0f) : 0.0f;
  }
  return dg;
}

// Ascending positions of the set bits of words [w0, w1) (word w from
// getw(w), bit b = element 32 w + b), written from out[base] on, at most
// `limit` in total.  One warp.
template <class GetW>
__device__ __forceinline__ void warp_compact_by(GetW getw, int w0, int w1, int *out, int base,
                                                int limit) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  for (int r = w0; r < w1; r += 32) {
    const int w = r + lane;
    const uint32_t word = w < w1 ? getw(w) : 0u;
    const int c = __popc(word);
    int incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const int at = base + incl - c;
    const int nw = min(32, w1 - r);
    for (int i = 0; i < nw; ++i) {
      const uint32_t wi = __shfl_sync(0xffffffffu, word, i);
      const int pos = __shfl_sync(0xffffffffu, at, i) + __popc(wi & lt);
      if (((wi >> lane) & 1u) && pos < limit) out[pos] = 32 * (r + i) + lane;
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// Static shared memory of the kernel, declared once for its three m
// instances.
struct TailShared {
  RunDesc desc;
  uint64_t bar;
  unsigned lo[kMaxM], hi[kMaxM];
  int red[2][32];
  uint32_t free_[kTailFreeWords];
  uint32_t vb_[kTailFreeWords];   // this CTA's valid-flag words of P_{t+1} (C -> D)
  double rng[kMaxM];
  unsigned z[4];          // z* of the combined population (order-preserving)
  unsigned zr[8];         // survivors' minimum (0..3) and maximum (4..7)
  unsigned zpar[4];       // the parents' z*, read before the dependency wait
  float gw[4];            // direction-grid scale of the current vectors
  float pen;              // the APD penalty M (t / t_max)^alpha (Eq. 4)
  unsigned long long bar0; // the grid barrier counter at this launch's start
  int grid_ok;            // the direction grid matches the current vectors
};

template <int PROB, int M>
__device__ __forceinline__ void tail_body(const RunDesc &R, TailShared &S) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t &s_bar = S.bar;
  unsigned *const s_lo = S.lo, *const s_hi = S.hi;
  int (*const s_red)[32] = S.red;
  const int N = R.N, n2 = 2 * N, m = R.m, T = R.ntiles;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = gridDim.x, b = blockIdx.x;
  Ctl *const ctl = R.ctl;

  // ---- prologue: the search tables into shared memory (written by k_tiles,
  // earlier than the reproduction kernel), unless they exceed it: then the
  // kernel reads them where they are, through L2 --------------------------------
  const bool gtab = R.tables_global != 0;
  const uint32_t bV = (uint32_t)N * 16, bC = (uint32_t)T * 16, bS = (uint32_t)T * 8;
  const uint32_t bSr = (bS + 15u) & ~15u;
  const float4 *sV = gtab ? R.Vt : reinterpret_cast<const float4 *>(smem);
  const float4 *sC = gtab ? R.tcen : reinterpret_cast<const float4 *>(smem + bV);
  const float2 *sCS = gtab ? R.tcs : reinterpret_cast<const float2 *>(smem + bV + bC);
  const int2 *sR = gtab ? R.trng : reinterpret_cast<const int2 *>(smem + bV + bC + bSr);
  // (the copies land while phase A runs: phase B is the first to read them)
  if (!gtab && tid == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    mbar_expect_tx(&s_bar, bV + bC + 2 * bSr);
    tma_load_1d(smem, R.Vt, bV, &s_bar);
    tma_load_1d(smem + bV, R.tcen, bC, &s_bar);
    tma_load_1d(smem + bV + bC, R.tcs, bSr, &s_bar);
    tma_load_1d(smem + bV + bC + bSr, R.trng, bSr, &s_bar);
  }
  // the generation index and the child slots were written by the previous
  // generation's tail, which completed before the reproduction kernel (this
  // grid's predecessor) passed its own wait; read through L2
  const int t = __ldcg(&ctl->t);
  const KeyRun kr{R.key0, R.key1};
  // children are finished here when SBX left them to a second kernel
  const bool tail_mut = R.team == 32 && R.op == 0 && PROB != PROB_NEURO;
  // this generation's combined objectives by combined index: the parents
  // written by the previous generation's decode (when it was this kernel),
  // the children by phase A below
  const float *fcur = (tail_mut && __ldcg(&ctl->fcomb_t) == t)
                          ? R.fcomb + (size_t)(t & 1) * M * n2 : nullptr;
  // Also final before the wait: the parents' z* (set by the previous
  // generation's decode; when SBX finished the children, the reproduction
  // kernel adds theirs to it, so it is read after the wait instead), and
  // whether the direction grid matches the vectors (its build ran after the
  // previous tail) with its scale.
  if (tid == kTailThreads - 32) {   // the last warp, which serves no child below 19 k children
    // the launch's barrier base: the previous launches' arrivals, completed
    // (a CTA of this launch that arrived already adds less than nb)
    S.bar0 = (__ldcg(&ctl->bar) / (unsigned long long)nb) * (unsigned long long)nb;
    S.pen = (float)m * powf((float)t / (float)R.t_max, R.alpha);
    S.grid_ok = M <= 3 && R.gG > 0 && __ldcg(&ctl->grid_ver) == __ldcg(&ctl->v_ver);
    for (int q = 0; q < 4; ++q) {
      S.gw[q] = q < M && M <= 3 && R.gG > 0 ? __ldcg(R.gscale + q) : 1.0f;
      S.zpar[q] = tail_mut && q < M ? __ldcg(&ctl->zkey[q]) : 0xFFFFFFFFu;
    }
  }
  // Phase A takes each child with a group of eight lanes (four children a
  // warp, spread over the CTAs first).  Before the wait: the child's slot,
  // its site count and sites (Floyd's sampler, every lane of the group
  // computing the same draws and lane i keeping site i) and lane i's
  // magnitude; a child with more than eight sites is left to lane 0 alone
  // after the wait.
  const int sub = lane & 7, gl = lane & 24;
  const int cd = 4 * (warp * nb + b) + (lane >> 3);   // this group's child
  const bool child = tail_mut && cd < N;
  int slot = -1, k = 0;
  if (child) {
    slot = __ldcg(R.child_slot + (t & 1) * N + cd);
    if (slot < 0 || slot >= n2) {
      if (sub == 0) set_status(ctl, ST_BADINDEX);
      slot = -1;
    }
    if (slot >= 0 && R.T_m > 0 && R.T_m < (1u << 24)) {
      const uint4 w = philox_k(0u, (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr);
      const int nthr = R.n_mthr;
      while (k < nthr && w.x >= R.mthr[k]) ++k;
    }
  }
  const bool ovf = k > 8;                 // the child's sites do not fit its lanes
  const int kin = ovf ? 0 : k;
  const int kmax = __reduce_max_sync(0xffffffffu, kin);
  uint32_t js = 0u;                        // site sub of the child (sub < kin)
  {
    uint4 w = kin > 0 ? philox_k(0u, (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr) : make_uint4(0, 0, 0, 0);
    for (int i = 0; i < kmax; ++i) {       // every lane of the warp takes every step
      const int e = i + 1;
      if ((e & 3) == 0 && i < kin)
        w = philox_k((uint32_t)(e >> 2), (uint32_t)cd, (uint32_t)t, TAG_MUTSITE, kr);
      const uint32_t J = (uint32_t)(R.d - kin + i);
      uint32_t r = i < kin ? __umulhi(word(w, e & 3), J + 1u) : 0u;
      const bool hit = sub < i && js == r;   // drawn already by this child
      if ((__ballot_sync(0xffffffffu, hit) >> gl) & 0xFFu) r = J;
      if (sub == i) js = r;
    }
  }
  const float mag = sub < kin ? u24f(philox_k(js, (uint32_t)cd, (uint32_t)t, TAG_MUTMAG, kr).y) : 0.0f;
  if (R.rec_sites && slot >= 0 && !ovf) {
    int *const rec = R.rec_sites + (size_t)cd * (1 + kMaxSites);
    if (sub == 0) rec[0] = R.T_m >= (1u << 24) ? -1 : k;
    if (sub < kin) rec[1 + sub] = (int)js;
  }

  pdl_wait();   // the reproduction kernel's children

  // ---- A: mutation and evaluation of the children, z* ----------------------
  if (tid < kMaxM) { s_lo[tid] = 0xFFFFFFFFu; s_hi[tid] = 0u; }
  if (b == 0)
    for (int q = tid; q < nb; q += kTailThreads) R.occ_cnt[q] = 0u;
  __syncthreads();
  if (tail_mut && cd - (lane >> 3) < N) {   // a warp with at least one child (warp-uniform)
    const bool live = slot >= 0;
    float *const row = live ? R.X + (size_t)slot * R.d_pad : nullptr;
    // the pair's segment partials, added in segment order (lanes load eight
    // at a time, every lane adds); the position variables
    const int S = R.nseg, pp = cd < R.P ? cd : cd - R.P;
    const float *ps = R.psum + (size_t)pp * 2 * S + (cd < R.P ? 0 : S);
    // the group's loads first, all in flight together: the first eight
    // partials, the position variables and the sites' values
    const float v0 = live && sub < S ? __ldcg(ps + sub) : 0.0f;
    float hv = live && sub < M - 1 ? __ldcg(row + sub) : 0.0f;
    float *const px = live ? row + js : nullptr;
    const float x = live && sub < kin ? __ldcg(px) : 0.0f;
    float g = 0.0f;
    for (int q0 = 0; q0 < S; q0 += 8) {
      const float v = q0 == 0 ? v0 : (live && q0 + sub < S ? __ldcg(ps + q0 + sub) : 0.0f);
      for (int u = 0; u < 8 && q0 + u < S; ++u) g += __shfl_sync(0xffffffffu, v, gl | u);
    }
    // the mutations, site i on lane i of the group
    float dgi = 0.0f;
    bool hhit = false;
    if (live && sub < kin) {
      const float xn = poly_mutate(x, mag, R.L, R.U, R.eta_m);
      __stcg(px, xn);
      dgi = (int)js >= M - 1 ? g_term1(PROB, xn, 0.0f) - g_term1(PROB, x, 0.0f) : 0.0f;
      hhit = (int)js < M - 1;
    }
    float dg = 0.0f;   // the term changes in draw order
    for (int i = 0; i < kmax; ++i) {
      const float v = __shfl_sync(0xffffffffu, dgi, gl | i);
      if (i < kin) dg += v;
    }
    if (live && ovf && sub == 0) {
      dg = child_serial<PROB, M>(R, kr, cd, t, slot, k);
      hhit = true;
    }
    // a site among x_1..x_{m-1}: read them back, mutated
    const bool ghit = ((__ballot_sync(0xffffffffu, hhit) >> gl) & 0xFFu) != 0u;
    __syncwarp();   // the group's stores above are visible to its lanes
    if (ghit && live && sub < M - 1) hv = __ldcg(row + sub);
    dg = __shfl_sync(0xffffffffu, dg, gl);
    float head[M > 1 ? M - 1 : 1];
#pragma unroll
    for (int jj = 0; jj < M - 1; ++jj) head[jj] = __shfl_sync(0xffffffffu, hv, gl | jj);
    if (live && sub == 0) {
      float f[M];
      dtlz_objectives_t<PROB>(M, g + dg, head, f);
      float *const fc = R.fcomb + (size_t)(t & 1) * M * n2 + N + cd;
#pragma unroll
      for (int kk = 0; kk < M; ++kk) {
        R.F[(size_t)kk * n2 + slot] = f[kk];
        fc[(size_t)kk * n2] = f[kk];
        atomicMin(&s_lo[kk], f2ord(f[kk]));
      }
    }
  }
  // this CTA's minimum of its children (plane 0 of zacc): a plain store per
  // CTA, where one atomic per CTA on the same words would queue the loads
  // of z* after the barrier behind all of them
  __syncthreads();
  if (tid < 4) R.zacc[b * 4 + tid] = s_lo[tid];
  if (!grid_barrier(ctl, S.bar0 + (unsigned long long)nb)) return;
  if (tid < kMaxM) s_lo[tid] = 0xFFFFFFFFu;   // for the survivors' minimum in C
  // ---- B: association and APD votes ----------------------------------------
  {
    // the direction grid's first group of solutions (the only one, unless
    // the population outgrows the grid's lanes): their objectives are loaded
    // here, in flight while warp 0 gathers z*
    constexpr int MG = M <= 3 ? M : 3;
    const int gw = warp * nb + b, nw = nb * (kTailThreads / 32);
    const bool l8 = R.n_comb <= 4 * nw;
    const int i0 = l8 ? 4 * gw + (lane >> 3) : 8 * gw + (lane >> 2);
    const bool use_pre = S.grid_ok && fcur != nullptr && i0 < R.n_comb;
    float pre[MG];
#pragma unroll
    for (int k = 0; k < MG; ++k) pre[k] = use_pre ? __ldcg(fcur + (size_t)k * n2 + i0) : 0.0f;
    if (warp == 0) {   // z* = min(the parents' z*, every CTA's children)
      // lane l reads the four minima of CTAs l, l + 32, ... (all loads in
      // flight together, nb <= kTailMaxCtas = 8 x 32, and in flight while
      // the CTA waits for its tables below)
      uint4 v[kTailMaxCtas / 32];
#pragma unroll
      for (int i = 0; i < kTailMaxCtas / 32; ++i) {
        const int q = lane + 32 * i;
        v[i] = q < nb ? __ldcg(reinterpret_cast<const uint4 *>(R.zacc) + q)
                      : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
      }
      unsigned z0 = v[0].x, z1 = v[0].y, z2 = v[0].z, z3 = v[0].w;
#pragma unroll
      for (int i = 1; i < kTailMaxCtas / 32; ++i) {
        z0 = min(z0, v[i].x); z1 = min(z1, v[i].y); z2 = min(z2, v[i].z); z3 = min(z3, v[i].w);
      }
      z0 = __reduce_min_sync(0xffffffffu, z0);
      z1 = __reduce_min_sync(0xffffffffu, z1);
      z2 = __reduce_min_sync(0xffffffffu, z2);
      z3 = __reduce_min_sync(0xffffffffu, z3);
      if (lane < 4) {
        const unsigned zp = tail_mut ? S.zpar[lane] : __ldcg(&ctl->zkey[lane]);
        S.z[lane] = min(zp, lane == 0 ? z0 : lane == 1 ? z1 : lane == 2 ? z2 : z3);
      }
    }
    if (!gtab) {   // the tables staged in the prologue
      const bool staged = mbar_wait(&s_bar, 0u, kWaitLimit);
      if (__syncthreads_or(!staged)) {
        // a copy never arrived: flag it, let the copies land, give up (the
        // other CTAs' next barrier then times out and reports the same status)
        if (tid == 0) {
          set_status(ctl, ST_TIMEOUT);
          mbar_wait(&s_bar, 0u, kWaitLimit);
        }
        __syncthreads();
        return;
      }
    }
    const float pen = S.pen;
    __syncthreads();
    float z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] = k < m ? ord2f(S.z[k]) : 0.f;
    if (S.grid_ok) {
      // the direction grid
      float w[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) w[k] = S.gw[k];
      // eight lanes per solution (groups of four solutions spread over the
      // CTAs), or four where eight would give some warps a second group
      if (l8) {
        for (int g = gw; 4 * g < R.n_comb; g += nw)
          grid_assocL<MG, 8>(R, 4 * g + (lane >> 3), sV, z, w, pen, fcur,
                             g == gw && use_pre ? pre : nullptr);
      } else {
        for (int g = gw; 8 * g < R.n_comb; g += nw)
          grid_assocL<MG, 4>(R, 8 * g + (lane >> 2), sV, z, w, pen, fcur,
                             g == gw && use_pre ? pre : nullptr);
      }
    } else {   // the tile search (a CTA-uniform branch)
      const float2 csb = tile_bounds(sCS, T);
      const int groups = (R.n_comb + 3) >> 2;
      for (int g = gw; g < groups; g += nw) prune_group<M, false>(R, 4 * g, sV, sC, sCS, sR, z, pen, csb);
    }
  }
  if (!grid_barrier(ctl, S.bar0 + 2ull * nb)) return;

  // ---- C: decode of this CTA's vector words --------------------------------
  // vector words [v0, v1) (32 vectors each) and pool-row words [o0, o1) (32
  // rows each) belong to this CTA in C and D
  const int nvw = (N + 31) >> 5, now = (n2 + 31) >> 5;
  const int pv = (nvw + nb - 1) / nb, po = (now + nb - 1) / nb;
  const int v0 = min(nvw, b * pv), v1 = min(nvw, v0 + pv);
  const int o0 = min(now, b * po), o1 = min(now, o0 + po);
  {
    const int *cur = R.slotmap + (t & 1) * N;
    int *nmap = R.slotmap + ((t + 1) & 1) * N;
    const int *ccur = R.child_slot + (t & 1) * N;
    int nvalid = 0;
    float *const fnext = R.fcomb + (size_t)((t + 1) & 1) * M * n2;
    for (int vw = v0 + warp; vw < v1; vw += kTailThreads / 32) {
      const int j = 32 * vw + lane;
      int s = -1, i = -1;
      float fci[M];   // the winner's objectives by combined index, loaded with its slot
#pragma unroll
      for (int k = 0; k < M; ++k) fci[k] = 0.0f;
      if (j < N) {
        const unsigned long long key = __ldcg(R.best + j);
        R.best[j] = ~0ull;
        if (key != ~0ull) {
          i = (int)(uint32_t)(key & 0xFFFFFFFFull);
          if (fcur && i >= 0 && i < n2) {
#pragma unroll
            for (int k = 0; k < M; ++k) fci[k] = __ldcg(fcur + (size_t)k * n2 + i);
          }
          if (i >= 0 && i < N) s = cur[i];
          else if (i >= N && i < n2) s = ccur[i - N];
          if (s < 0 || s >= n2) { set_status(ctl, ST_BADINDEX); s = -1; i = -1; }
        }
        nmap[j] = s;
        R.surv[j] = i;
        // CSO: the APD that kept slot j's member (Eq. 4), for the next competitions
        if (R.kapd) R.kapd[j] = s >= 0 ? __uint_as_float((uint32_t)(key >> 32)) : __int_as_float(0x7f800000);
        if (s >= 0) {
          R.otag[s] = t;
          atomicAdd(&R.occ_cnt[min(nb - 1, (s >> 5) / po)], 1u);
        }
      }
      const uint32_t vmask = __ballot_sync(0xffffffffu, s >= 0);
      if (lane == 0) {
        R.vbits[vw] = vmask;
        S.vb_[vw - v0] = vmask;   // v1 - v0 <= the pool-row words a CTA holds
      }
      nvalid += __popc(vmask);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        unsigned lo = 0xFFFFFFFFu, hi = 0u;
        float fv = __int_as_float(0x7fffffff);   // NaN: an invalid slot of P_{t+1}
        if (s >= 0) {
          fv = fcur ? fci[k] : __ldcg(R.F + (size_t)k * n2 + s);
          lo = hi = f2ord(fv);
        }
        if (j < N) fnext[(size_t)k * n2 + j] = fv;
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0) { atomicMin(&s_lo[k], lo); atomicMax(&s_hi[k], hi); }
      }
    }
    if (lane == 0) s_red[0][warp] = nvalid;
  }
  __syncthreads();
  if (tid < 4) {   // planes 1 and 2 of zacc: this CTA's survivors' minimum and maximum
    R.zacc[(nb + b) * 4 + tid] = s_lo[tid];
    R.zacc[(2 * nb + b) * 4 + tid] = s_hi[tid];
  }
  if (tid == 0) {
    int c = 0;
    for (int w = 0; w < kTailThreads / 32; ++w) c += s_red[0][w];
    R.vcnt[b] = c;
  }
  if (!grid_barrier(ctl, S.bar0 + 3ull * nb)) return;

  // ---- D: lists, next z*, adaptation, control block ------------------------
  // prefix of the valid slots and of the free rows over the CTAs before this
  // one, and the totals
  int pre_v, tot_v, pre_f;
  if (warp == 0) {   // one warp reads the nb counts, the others wait
    int a = 0, av = 0, af = 0;
    for (int q = lane; q < nb; q += 32) {
      const int vq = __ldcg(R.vcnt + q);
      const int q0 = min(now, q * po), q1 = min(now, q0 + po);
      const int rows = max(0, min(n2, 32 * q1) - 32 * q0);
      const int fq = rows - (int)__ldcg(R.occ_cnt + q);
      a += vq;
      if (q < b) { av += vq; af += fq; }
    }
    a = __reduce_add_sync(0xffffffffu, a);
    av = __reduce_add_sync(0xffffffffu, av);
    af = __reduce_add_sync(0xffffffffu, af);
    if (lane == 0) { s_red[1][0] = a; s_red[1][1] = av; s_red[1][2] = af; }
  } else if (warp == 1) {   // meanwhile: the free pool rows of this CTA's row words
    uint32_t *const s_free = S.free_;
    for (int w = o0; w < o1; ++w) {
      const int row = 32 * w + lane;
      const bool occ = row >= n2 || __ldcg(R.otag + row) == t;
      const uint32_t fw = __ballot_sync(0xffffffffu, !occ);
      if (lane == 0) s_free[w - o0] = fw;
    }
  }
  const bool adapt = (t % R.p_adapt) == 0;
  if (warp == 2 && (b == 0 || adapt)) {   // the survivors' minimum and maximum over the CTAs
    unsigned lo = 0xFFFFFFFFu, hi = 0u;      // of objective lane % 4, as in B
    for (int e = lane; e < 4 * nb; e += 32) {
      lo = min(lo, __ldcg(R.zacc + 4 * nb + e));
      hi = max(hi, __ldcg(R.zacc + 8 * nb + e));
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane < 4) { S.zr[lane] = lo; S.zr[4 + lane] = hi; }
  }
  __syncthreads();
  tot_v = s_red[1][0];
  pre_v = s_red[1][1];
  pre_f = s_red[1][2];
  const int K = tot_v;
  if (warp == 0) {   // ascending valid slots of this CTA's vector words (from C)
    warp_compact_by([&](int w) { return S.vb_[w - v0]; }, v0, v1, R.vlist, pre_v, N);
  } else if (warp == 1) {   // ascending free pool rows of this CTA's row words
    uint32_t *const s_free = S.free_;
    warp_compact_by([&](int w) { return s_free[w - o0]; }, o0, o1,
                    R.child_slot + ((t + 1) & 1) * N, pre_f, N);
  }
  if (b == 0 && tid < m) ctl->zkey[tid] = S.zr[tid];
  if (adapt && K > 0) {
    // range_k = max - min over the survivors, floored at 1e-12, in FP64
    double *const s_rng = S.rng;
    if (tid < m) {
      const double r = (double)ord2f(S.zr[4 + tid]) - (double)ord2f(S.zr[tid]);
      s_rng[tid] = r < 1e-12 ? 1e-12 : r;
      if (b == 0) R.vrange[tid] = s_rng[tid];
    }
    __syncthreads();
    const int pj = (N + nb - 1) / nb;
    const int j0 = min(N, b * pj), j1 = min(N, j0 + pj);
    for (int jj = j0 + tid; jj < j1; jj += kTailThreads) adapt_row(R, jj, s_rng);
  }
  if (b == 0 && tid == 0) {
    ctl->K = K;
    ctl->adapted = adapt ? 1 : 0;
    if (adapt && K > 0) ctl->v_ver += 1;
    ctl->fin_cnt = 0;
    ctl->sel_cnt = 0;
    ctl->fcomb_t = t + 1;
    ctl->t = t + 1;
  }
  pdl_trigger();
}

// The descriptor is copied into shared memory first: its fields are read in
// every phase, and after each wait and barrier a global load of them would
// go back to L2.
__device__ __forceinline__ void stage_desc(const RunDesc *Rp, RunDesc *sD) {
  const int *src = reinterpret_cast<const int *>(Rp);
  int *dst = reinterpret_cast<int *>(sD);
  for (int q = threadIdx.x; q < (int)(sizeof(RunDesc) / 4); q += blockDim.x) dst[q] = src[q];
  __syncthreads();
}
#define RVEA_TAIL(name, PROB)                                                              \
  __global__ void __launch_bounds__(kTailThreads, 1) name(const RunDesc *__restrict__ Rp) { \
    __shared__ __align__(16) TailShared S;                                                 \
    stage_desc(Rp, &S.desc);                                                               \
    switch (S.desc.m) {                                                                    \
      case 2: tail_body<PROB, 2>(S.desc, S); break;                                        \
      case 3: tail_body<PROB, 3>(S.desc, S); break;                                        \
      default: tail_body<PROB, 4>(S.desc, S); break;                                       \
    }                                                                                      \
  }
RVEA_TAIL(k_tail_dtlz1, PROB_DTLZ1)
RVEA_TAIL(k_tail_dtlz2, PROB_DTLZ2)
RVEA_TAIL(k_tail_dtlz3, PROB_DTLZ3)
RVEA_TAIL(k_tail_dtlz4, PROB_DTLZ4)
#undef RVEA_TAIL

}  // namespace rvea
