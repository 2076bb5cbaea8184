/*
 * FP64 CPU oracle of one generation of tensorized RVEA (arXiv 2404.01159).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline legs of bench.py.  The CUDA library never includes or loads it.
 *
 * This file is deliberately plain: every step is the paper's formula written
 * out in double precision, in the paper's order, with no blocking or fusion.
 * Loops over independent rows carry an OpenMP pragma; no reduction crosses
 * threads, so results do not depend on the thread count.
 *
 * Parity pins (tests/test_oracle_*.py) check this file against closed forms,
 * invariants, known-answer vectors and brute force; see the header of each
 * function for what it follows.
 */
#include "rvea_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void orc_set_threads(int32_t n) { g_threads = n < 1 ? 1 : n; }
int32_t orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon et al. SC'11, Sec. 3-4: ten rounds of the S-box     */
/* (two 32x32->64 multiplies by 0xD2511F53 and 0xCD9E8D57, XOR with the      */
/* other counter words and the round key), key bumped by the Weyl constants  */
/* 0x9E3779B9 / 0xBB67AE85 between rounds.                                   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox(const orc_params *p, uint32_t c0, uint32_t c1, uint32_t c2,
                   uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* A uniform on [0,1) with 24 random bits: exact in float and double. */
static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* Box-Muller (Box & Muller 1958): N(0,1) from two uniforms, u1 in (0,1]. */
static double box_muller(uint32_t w0, uint32_t w1)
{
    double u1 = 1.0 - u24(w0);
    double u2 = u24(w1);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Event of probability q fires iff R < q, for R = k * 2^-24:
 * k < ceil(q * 2^24).  q = 0 never fires, q >= 1 always fires. */
static uint32_t event_threshold(double q)
{
    double x = ceil(q * 16777216.0);
    if (x < 0.0) x = 0.0;
    if (x > 16777216.0) x = 16777216.0;
    return (uint32_t)x;
}

/* ------------------------------------------------------------------------ */
/* Reference vectors.  The paper takes unit vectors V0 as input (Algorithm 2 */
/* and Sec. 3.1) without fixing their construction; the reading used is the  */
/* Das-Dennis simplex lattice {k / H : k_i >= 0, sum k_i = H} of the original */
/* RVEA, listed in lexicographic order of (k_1..k_{m-1}), then normalised.   */
/* ------------------------------------------------------------------------ */
int64_t orc_lattice_count(int32_t m, int32_t H)
{
    /* C(H + m - 1, m - 1) */
    int64_t c = 1;
    for (int32_t i = 1; i <= m - 1; ++i)
        c = c * (int64_t)(H + i) / i;
    return c;
}

/* Population size n that is not a lattice size (the speed sweeps of Sec.
 * 4.1 use n = 2^5 .. 2^14): the reference vectors are the largest Das-Dennis
 * lattice with at most n points, as a uniform-point generator gives them,
 * and the population is that lattice's size.  Returns its H (>= 1), or -1
 * when even H = 1 has more than n points. */
int32_t orc_lattice_for(int32_t m, int32_t n)
{
    if (m < 2 || orc_lattice_count(m, 1) > n) return -1;
    int32_t H = 1;
    while (orc_lattice_count(m, H + 1) <= n) ++H;
    return H;
}

static int32_t lattice_rec(int32_t m, int32_t pos, int32_t left, int32_t *cur,
                           int32_t *K, int32_t N, int32_t row)
{
    if (pos == m - 1) {
        if (row >= N) return row + 1;
        cur[pos] = left;
        for (int32_t k = 0; k < m; ++k) K[(int64_t)row * m + k] = cur[k];
        return row + 1;
    }
    for (int32_t k = 0; k <= left; ++k) {
        cur[pos] = k;
        row = lattice_rec(m, pos + 1, left - k, cur, K, N, row);
    }
    return row;
}

int32_t orc_lattice(int32_t m, int32_t H, int32_t N, int32_t *K)
{
    if (m < 1 || H < 0 || orc_lattice_count(m, H) != N) return -1;
    int32_t *cur = (int32_t *)calloc((size_t)m, sizeof(int32_t));
    int32_t rows = lattice_rec(m, 0, H, cur, K, N, 0);
    free(cur);
    return rows;
}

void orc_lattice_unit(int32_t m, int32_t N, const int32_t *K, double *V0)
{
    for (int32_t j = 0; j < N; ++j) {
        double s = 0.0;
        for (int32_t k = 0; k < m; ++k) {
            double v = (double)K[(int64_t)j * m + k];
            s += v * v;
        }
        double nrm = sqrt(s);
        for (int32_t k = 0; k < m; ++k)
            V0[(int64_t)j * m + k] = (double)K[(int64_t)j * m + k] / nrm;
    }
}

static double dot(const double *a, const double *b, int32_t m)
{
    double s = 0.0;
    for (int32_t k = 0; k < m; ++k) s += a[k] * b[k];
    return s;
}

static double clamp1(double c)
{
    if (c > 1.0) return 1.0;
    if (c < -1.0) return -1.0;
    return c;
}

/* Eq. 5 and Algorithm 1 (Gamma line): gamma_j = min over i != j of the angle
 * between v_i and v_j.  The printed Gamma line takes a row minimum over the
 * full arccos matrix, whose diagonal is zero; Eq. 5 excludes i = j, which is
 * the reading used.  Clamped below at 1e-12 so the APD division is finite. */
void orc_gamma(int32_t m, int32_t r, const double *V, double *gamma)
{
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int32_t j = 0; j < r; ++j) {
        const double *vj = V + (int64_t)j * m;
        double nj = sqrt(dot(vj, vj, m));
        double best = INFINITY;
        for (int32_t i = 0; i < r; ++i) {
            if (i == j) continue;
            const double *vi = V + (int64_t)i * m;
            double ni = sqrt(dot(vi, vi, m));
            double a = acos(clamp1(dot(vi, vj, m) / (ni * nj)));
            if (a < best) best = a;
        }
        if (!(best >= 1e-12)) best = 1e-12;
        gamma[j] = best;
    }
}

/* Objective range of the current population, used by the adaptation. */
void orc_objective_range(int32_t m, int32_t n, const double *F, const uint8_t *valid,
                         double *range)
{
    for (int32_t k = 0; k < m; ++k) {
        double lo = INFINITY, hi = -INFINITY;
        for (int32_t i = 0; i < n; ++i) {
            if (valid && !valid[i]) continue;
            double f = F[(int64_t)i * m + k];
            if (f < lo) lo = f;
            if (f > hi) hi = f;
        }
        range[k] = (hi >= lo) ? hi - lo : 0.0;
    }
}

/* Algorithm 2 ("update reference vectors ... from V_t and V0"): the formula is
 * not printed; the reading is the original RVEA adaptation, V_j = V0_j (.)
 * range / ||V0_j (.) range||, with each range component floored at 1e-12. */
void orc_adapt(int32_t m, int32_t r, const double *V0, const double *range, double *V)
{
    for (int32_t j = 0; j < r; ++j) {
        double s = 0.0;
        for (int32_t k = 0; k < m; ++k) {
            double rk = range[k] < 1e-12 ? 1e-12 : range[k];
            double v = V0[(int64_t)j * m + k] * rk;
            s += v * v;
        }
        double nrm = sqrt(s);
        for (int32_t k = 0; k < m; ++k) {
            double rk = range[k] < 1e-12 ? 1e-12 : range[k];
            V[(int64_t)j * m + k] = V0[(int64_t)j * m + k] * rk / nrm;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Initialisation (Algorithm 2, "initialize population P0 with n randomized  */
/* individuals").  DTLZ: uniform on [L,U]; neuroevolution: N(0, 0.1^2)      */
/* weights clipped to [L,U].                                                 */
/* ------------------------------------------------------------------------ */
void orc_init_population(const orc_params *p, double *X)
{
    const int32_t N = p->N, d = p->d;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int32_t i = 0; i < N; ++i) {
        for (int32_t j = 0; j < d; ++j) {
            uint32_t w[4];
            double x;
            if (p->problem == ORC_NEURO) {
                philox(p, (uint32_t)j, (uint32_t)i, 0u, ORC_TAG_INIT, w);
                x = 0.1 * box_muller(w[0], w[1]);
                if (x < p->L) x = p->L;
                if (x > p->U) x = p->U;
            } else {
                philox(p, (uint32_t)(j / 4), (uint32_t)i, 0u, ORC_TAG_INIT, w);
                x = p->L + (p->U - p->L) * u24(w[j % 4]);
            }
            X[(int64_t)i * d + j] = x;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Objectives.  The paper names DTLZ1/DTLZ2 (Sec. 4.1, Appendix C) without   */
/* printing them; the formulas are the standard DTLZ definitions with        */
/* 1-based x, g over x_m..x_d, k = d - m + 1.  DTLZ3/DTLZ4 (the rest of the  */
/* suite of Sec. 4.1's benchmark family) follow the same published source.  */
/* ------------------------------------------------------------------------ */
static void dtlz2(int32_t m, int32_t d, const double *x, double *f)
{
    double g = 0.0;
    for (int32_t j = m - 1; j < d; ++j) g += (x[j] - 0.5) * (x[j] - 0.5);
    for (int32_t k = 1; k <= m; ++k) {
        /* f_k = (1+g) prod_{i < m-k+1} cos(x_i pi/2) [* sin(x_{m-k+1} pi/2) if k>1] */
        double v = 1.0 + g;
        for (int32_t i = 1; i <= m - k; ++i) v *= cos(x[i - 1] * M_PI / 2.0);
        if (k > 1) v *= sin(x[m - k] * M_PI / 2.0);
        f[k - 1] = v;
    }
}

static void dtlz1(int32_t m, int32_t d, const double *x, double *f)
{
    int32_t kk = d - m + 1;
    double s = 0.0;
    for (int32_t j = m - 1; j < d; ++j) {
        double y = x[j] - 0.5;
        s += y * y - cos(20.0 * M_PI * y);
    }
    double g = 100.0 * ((double)kk + s);
    for (int32_t k = 1; k <= m; ++k) {
        double v = 0.5 * (1.0 + g);
        for (int32_t i = 1; i <= m - k; ++i) v *= x[i - 1];
        if (k > 1) v *= 1.0 - x[m - k];
        f[k - 1] = v;
    }
}

/* DTLZ3 (Deb, Thiele, Laumanns, Zitzler 2005): the spherical shape of DTLZ2
 * with the multimodal g of DTLZ1 (3^k - 1 local fronts). */
static void dtlz3(int32_t m, int32_t d, const double *x, double *f)
{
    int32_t kk = d - m + 1;
    double s = 0.0;
    for (int32_t j = m - 1; j < d; ++j) {
        double y = x[j] - 0.5;
        s += y * y - cos(20.0 * M_PI * y);
    }
    double g = 100.0 * ((double)kk + s);
    for (int32_t k = 1; k <= m; ++k) {
        double v = 1.0 + g;
        for (int32_t i = 1; i <= m - k; ++i) v *= cos(x[i - 1] * M_PI / 2.0);
        if (k > 1) v *= sin(x[m - k] * M_PI / 2.0);
        f[k - 1] = v;
    }
}

/* DTLZ4 (same source): DTLZ2 with the position variables x_1..x_{m-1}
 * mapped to x_i^alpha, alpha = 100 (a front biased towards the f_m axis). */
static void dtlz4(int32_t m, int32_t d, const double *x, double *f)
{
    double g = 0.0;
    for (int32_t j = m - 1; j < d; ++j) g += (x[j] - 0.5) * (x[j] - 0.5);
    for (int32_t k = 1; k <= m; ++k) {
        double v = 1.0 + g;
        for (int32_t i = 1; i <= m - k; ++i) v *= cos(pow(x[i - 1], 100.0) * M_PI / 2.0);
        if (k > 1) v *= sin(pow(x[m - k], 100.0) * M_PI / 2.0);
        f[k - 1] = v;
    }
}

/* Process noise of the synthetic rollout: xi[s][k] ~ N(0,1), one draw per
 * step s and state component k, shared by every policy of generation t
 * (common random numbers). */
void orc_neuro_noise(const orc_params *p, const orc_neuro *nd, int32_t t, double *xi)
{
    for (int32_t s = 0; s < nd->steps; ++s)
        for (int32_t k = 0; k < nd->ns; ++k) {
            uint32_t w[4];
            philox(p, (uint32_t)k, (uint32_t)s, (uint32_t)t, ORC_TAG_NOISE, w);
            xi[(int64_t)s * nd->ns + k] = box_muller(w[0], w[1]);
        }
}

/* Neuroevolution objective (the linear-dynamics stand-in for the paper's
 * Brax tasks, Sec. 4.3): policy x = [W1 (h1 x ns), b1, W2 (h2 x h1), b2,
 * W3 (na x h2), b3], tanh on every layer, s_0 = 0,
 * s_{tau+1} = A s_tau + B u_tau + sigma xi_tau;
 * f1 = -sum_tau s_{tau+1}[0], f2 = sum_tau ||u_tau||^2. */
static void neuro_rollout(const orc_neuro *nd, const double *x, const double *xi,
                          double *f)
{
    const int32_t ns = nd->ns, na = nd->na, h1 = nd->h1, h2 = nd->h2;
    const double *W1 = x, *b1 = W1 + (int64_t)h1 * ns;
    const double *W2 = b1 + h1, *b2 = W2 + (int64_t)h2 * h1;
    const double *W3 = b2 + h2, *b3 = W3 + (int64_t)na * h2;
    double s[64], sn[64], a1[256], a2[256], u[64];
    for (int32_t k = 0; k < ns; ++k) s[k] = 0.0;
    double f1 = 0.0, f2 = 0.0;
    for (int32_t tau = 0; tau < nd->steps; ++tau) {
        for (int32_t o = 0; o < h1; ++o) {
            double z = b1[o];
            for (int32_t i = 0; i < ns; ++i) z += W1[(int64_t)o * ns + i] * s[i];
            a1[o] = tanh(z);
        }
        for (int32_t o = 0; o < h2; ++o) {
            double z = b2[o];
            for (int32_t i = 0; i < h1; ++i) z += W2[(int64_t)o * h1 + i] * a1[i];
            a2[o] = tanh(z);
        }
        for (int32_t o = 0; o < na; ++o) {
            double z = b3[o];
            for (int32_t i = 0; i < h2; ++i) z += W3[(int64_t)o * h2 + i] * a2[i];
            u[o] = tanh(z);
        }
        for (int32_t k = 0; k < ns; ++k) {
            double z = 0.0;
            for (int32_t i = 0; i < ns; ++i) z += nd->A[(int64_t)k * ns + i] * s[i];
            for (int32_t i = 0; i < na; ++i) z += nd->B[(int64_t)k * na + i] * u[i];
            sn[k] = z + nd->sigma * xi[(int64_t)tau * ns + k];
        }
        for (int32_t k = 0; k < ns; ++k) s[k] = sn[k];
        f1 -= s[0];
        for (int32_t o = 0; o < na; ++o) f2 += u[o] * u[o];
    }
    f[0] = f1;
    f[1] = f2;
}

void orc_evaluate(const orc_params *p, int32_t n, const double *X, double *F,
                  const orc_neuro *nd, int32_t t)
{
    const int32_t m = p->m, d = p->d;
    double *xi = NULL;
    if (p->problem == ORC_NEURO) {
        xi = (double *)malloc(sizeof(double) * (size_t)nd->steps * (size_t)nd->ns);
        orc_neuro_noise(p, nd, t, xi);
    }
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
    for (int32_t i = 0; i < n; ++i) {
        const double *x = X + (int64_t)i * d;
        double *f = F + (int64_t)i * m;
        if (p->problem == ORC_DTLZ2) dtlz2(m, d, x, f);
        else if (p->problem == ORC_DTLZ1) dtlz1(m, d, x, f);
        else if (p->problem == ORC_DTLZ3) dtlz3(m, d, x, f);
        else if (p->problem == ORC_DTLZ4) dtlz4(m, d, x, f);
        else neuro_rollout(nd, x, xi, f);
    }
    free(xi);
}

/* ------------------------------------------------------------------------ */
/* Reproduction, Appendix B.                                                 */
/* ------------------------------------------------------------------------ */

/* Mating: Appendix B partitions X into X1, X2 without saying how parents are
 * chosen.  Reading: 2*ceil(N/2) draws uniformly with replacement from the K
 * valid members (ascending slot order); draws 0..P-1 form X1 and P..2P-1
 * form X2.  Index of draw e = (w_e * K) >> 32 on the 32-bit word w_e. */
void orc_mating(const orc_params *p, int32_t t, int32_t K, const int32_t *vlist,
                int32_t *parents)
{
    const int32_t P = (p->N + 1) / 2;
    for (int32_t e = 0; e < 2 * P; ++e) {
        uint32_t w[4];
        philox(p, (uint32_t)(e / 4), 0u, (uint32_t)t, ORC_TAG_MATE, w);
        uint32_t idx = (uint32_t)(((uint64_t)w[e % 4] * (uint64_t)(uint32_t)K) >> 32);
        parents[e] = vlist[idx];
    }
}

/* ------------------------------------------------------------------------ */
/* Alternative reproduction operators of the extensibility experiment (Sec.  */
/* 4.4 and Appendix C: GA, PSO, DE, CSO and random reproduction inside the   */
/* same environmental selection).  The paper cites them without printing     */
/* them; these follow the published operators.  Offspring o = 0..N-1 fill   */
/* the N offspring rows as SBX's do.                                         */
/* ------------------------------------------------------------------------ */

/* Random reproduction (the experiment's baseline): x_oj = L + (U - L) u24,
 * u24 from RANDOM (j/4, o, t) word j%4. */
void orc_random_offspring(const orc_params *p, int32_t t, double *Xout)
{
    const int32_t N = p->N, d = p->d;
    for (int32_t o = 0; o < N; ++o)
        for (int32_t j = 0; j < d; ++j) {
            uint32_t w[4];
            philox(p, (uint32_t)(j / 4), (uint32_t)o, (uint32_t)t, ORC_TAG_RANDOM, w);
            Xout[(int64_t)o * d + j] = p->L + (p->U - p->L) * u24(w[j % 4]);
        }
}

/* DE/rand/1/bin draws of offspring o (Storn and Price 1997): out[0] = the
 * target's position o mod K in the valid list, out[1..3] = the positions of
 * r1, r2, r3, out[4] = j_rand.  With K >= 4 the three are a uniformly random
 * ordered triple of distinct positions other than the target's, drawn one
 * after another without replacement from DE_PICK (o, 0, t) words 0..2
 * (a in [0, K-1), b in [0, K-2), c in [0, K-3), each index = (w n) >> 32,
 * counted over the positions not yet taken); with K < 4 each is drawn with
 * replacement over all K.  j_rand = (w d) >> 32 of word 3. */
void orc_de_picks(const orc_params *p, int32_t t, int32_t K, int32_t o, int32_t *out)
{
    uint32_t w[4];
    philox(p, (uint32_t)o, 0u, (uint32_t)t, ORC_TAG_DE_PICK, w);
    const int32_t tpos = o % K;
    out[0] = tpos;
    if (K >= 4) {
        /* positions 0..K-2 of the list without the target */
        int32_t a = (int32_t)(((uint64_t)w[0] * (uint64_t)(K - 1)) >> 32);
        int32_t b = (int32_t)(((uint64_t)w[1] * (uint64_t)(K - 2)) >> 32);
        int32_t c = (int32_t)(((uint64_t)w[2] * (uint64_t)(K - 3)) >> 32);
        if (b >= a) b += 1;
        const int32_t lo = a < b ? a : b, hi = a < b ? b : a;
        if (c >= lo) c += 1;
        if (c >= hi) c += 1;
        const int32_t q[3] = {a, b, c};
        for (int32_t k = 0; k < 3; ++k) out[1 + k] = q[k] < tpos ? q[k] : q[k] + 1;
    } else {
        for (int32_t k = 0; k < 3; ++k)
            out[1 + k] = (int32_t)(((uint64_t)w[k] * (uint64_t)K) >> 32);
    }
    out[4] = (int32_t)(((uint64_t)w[3] * (uint64_t)p->d) >> 32);
}

/* DE/rand/1/bin as the reproduction operator: offspring o takes the target
 * x_t = X[vlist[o mod K]] and v = x_r1 + F (x_r2 - x_r3) (orc_de_picks);
 * u_j = v_j where the CR coin of j fires or j = j_rand, else x_t,j; the coin
 * fires iff u24 < ceil(CR 2^24) / 2^24, u24 from DE_CR (j/4, o, t) word j%4;
 * then u is clipped to [L, U].  X: population rows by slot. */
void orc_de_offspring(const orc_params *p, int32_t t, const double *X, int32_t K,
                      const int32_t *vlist, double F, double CR, double *Xout)
{
    const int32_t N = p->N, d = p->d;
    const uint32_t thr = (uint32_t)ceil(CR * 16777216.0);
    for (int32_t o = 0; o < N; ++o) {
        int32_t pk[5];
        orc_de_picks(p, t, K, o, pk);
        const double *xt = X + (int64_t)vlist[pk[0]] * d;
        const double *x1 = X + (int64_t)vlist[pk[1]] * d;
        const double *x2 = X + (int64_t)vlist[pk[2]] * d;
        const double *x3 = X + (int64_t)vlist[pk[3]] * d;
        double *u = Xout + (int64_t)o * d;
        for (int32_t j = 0; j < d; ++j) {
            uint32_t w[4];
            philox(p, (uint32_t)(j / 4), (uint32_t)o, (uint32_t)t, ORC_TAG_DE_CR, w);
            const int take = (w[j % 4] >> 8) < thr || j == pk[4];
            double v = take ? x1[j] + F * (x2[j] - x3[j]) : xt[j];
            if (v < p->L) v = p->L;
            if (v > p->U) v = p->U;
            u[j] = v;
        }
    }
}

/* The competitive swarm optimizer (CSO; Cheng and Jin, "A competitive swarm
 * optimizer for large scale optimization", IEEE T-Cyb 2015) as the
 * reproduction operator.  The paper names it and plugs it into the same
 * selection without printing it; the reading (listed with the others in the
 * design notes): each of the N offspring comes from one competition between
 * two distinct valid members (positions a then b of the valid list, drawn
 * without replacement: a = (w0 K) >> 32, b = (w1 (K-1)) >> 32 counted over
 * the positions other than a, CSO_PICK (o, 0, t) words 0 and 1; with K = 1
 * the member meets itself).  The winner has the smaller APD from the
 * selection that kept it (Eq. 4; +inf before any selection), ties to the
 * smaller population index.  The loser learns (Cheng and Jin's update):
 *   v' = r1 v_l + r2 (x_w - x_l) + phi r3 (xbar - x_l),   x' = x_l + v',
 * with r1, r2, r3 of variable j the u24 of word j%4 of CSO_R (3 (j/4) + k,
 * o, t) for k = 0, 1, 2 (each Philox call serves four consecutive variables),
 * xbar the mean position of the valid members; x' is clipped to [L, U] (v' is
 * kept as computed).  Offspring o is (x', v'); winners pass on only as
 * parents. */
void orc_cso_picks(const orc_params *p, int32_t t, int32_t K, int32_t o, int32_t *out)
{
    uint32_t w[4];
    philox(p, (uint32_t)o, 0u, (uint32_t)t, ORC_TAG_CSO_PICK, w);
    const int32_t a = (int32_t)(((uint64_t)w[0] * (uint64_t)K) >> 32);
    int32_t b = a;
    if (K > 1) {
        b = (int32_t)(((uint64_t)w[1] * (uint64_t)(K - 1)) >> 32);
        if (b >= a) b += 1;
    }
    out[0] = a;
    out[1] = b;
}

void orc_cso_offspring(const orc_params *p, int32_t t, const double *X, const double *Vel,
                       const double *apd, int32_t K, const int32_t *vlist, const double *xbar,
                       double *Xout, double *Vout)
{
    const int32_t N = p->N, d = p->d;
    for (int32_t o = 0; o < N; ++o) {
        int32_t pk[2];
        orc_cso_picks(p, t, K, o, pk);
        const int32_t ia = vlist[pk[0]], ib = vlist[pk[1]];
        const int a_wins = apd[ia] < apd[ib] || (apd[ia] == apd[ib] && ia <= ib);
        const int32_t iw = a_wins ? ia : ib, il = a_wins ? ib : ia;
        const double *xw = X + (int64_t)iw * d, *xl = X + (int64_t)il * d;
        const double *vl = Vel + (int64_t)il * d;
        for (int32_t j = 0; j < d; ++j) {
            double r[3];
            for (int32_t k = 0; k < 3; ++k) {
                uint32_t w[4];
                philox(p, (uint32_t)(3 * (j / 4) + k), (uint32_t)o, (uint32_t)t, ORC_TAG_CSO_R, w);
                r[k] = u24(w[j % 4]);
            }
            const double v = r[0] * vl[j] + r[1] * (xw[j] - xl[j]) +
                             p->cso_phi * r[2] * (xbar[j] - xl[j]);
            double x = xl[j] + v;
            if (x < p->L) x = p->L;
            if (x > p->U) x = p->U;
            Xout[(int64_t)o * d + j] = x;
            Vout[(int64_t)o * d + j] = v;
        }
    }
}

/* Particle swarm optimization (PSO; Kennedy and Eberhart 1995, with the
 * inertia weight of Shi and Eberhart 1998) as the reproduction operator.  The
 * paper names it and plugs it into the same selection without printing it;
 * the reading (listed with the others in the design notes), after the
 * multiobjective PSO of Coello, Pulido and Lechuga (2004) with the archive's
 * role taken by RVEA's population: particle o is the member at position
 * o mod K of the valid list, with its velocity v and personal best p
 * (carried with the member, like the velocity); its leader g is the winner
 * of a binary tournament on the kept APD (Eq. 4) between two distinct valid
 * members (positions a, then b over the others: PSO_PICK (o, 0, t) words 0
 * and 1, as the CSO competitors; ties to the smaller slot; with K = 1 the
 * member itself).  The particle moves:
 *   v' = w v + c1 r1 (p - x) + c2 r2 (g - x),   x' = clip(x + v'),
 * r1, r2 of variable j the u24 of word j%4 of PSO_R (2 (j/4) + k, o, t),
 * k = 0, 1.  out[0] = the particle's position in the list, out[1] = the
 * leader's. */
void orc_pso_picks(const orc_params *p, int32_t t, int32_t K, int32_t o, int32_t *out)
{
    uint32_t w[4];
    philox(p, (uint32_t)o, 0u, (uint32_t)t, ORC_TAG_PSO_PICK, w);
    const int32_t a = (int32_t)(((uint64_t)w[0] * (uint64_t)K) >> 32);
    int32_t b = a;
    if (K > 1) {
        b = (int32_t)(((uint64_t)w[1] * (uint64_t)(K - 1)) >> 32);
        if (b >= a) b += 1;
    }
    out[0] = o % K;
    out[1] = a;   /* the tournament is decided by the caller from the kept APDs */
    out[2] = b;
}

void orc_pso_offspring(const orc_params *p, int32_t t, const double *X, const double *Vel,
                       const double *Pb, const double *apd, int32_t K, const int32_t *vlist,
                       double *Xout, double *Vout)
{
    const int32_t N = p->N, d = p->d;
    for (int32_t o = 0; o < N; ++o) {
        int32_t pk[3];
        orc_pso_picks(p, t, K, o, pk);
        const int32_t ip = vlist[pk[0]], ia = vlist[pk[1]], ib = vlist[pk[2]];
        const int32_t ig = (apd[ia] < apd[ib] || (apd[ia] == apd[ib] && ia <= ib)) ? ia : ib;
        const double *x = X + (int64_t)ip * d, *v = Vel + (int64_t)ip * d;
        const double *pb = Pb + (int64_t)ip * d, *g = X + (int64_t)ig * d;
        for (int32_t j = 0; j < d; ++j) {
            double r[2];
            for (int32_t k = 0; k < 2; ++k) {
                uint32_t w[4];
                philox(p, (uint32_t)(2 * (j / 4) + k), (uint32_t)o, (uint32_t)t, ORC_TAG_PSO_R, w);
                r[k] = u24(w[j % 4]);
            }
            const double vn = p->pso_w * v[j] + p->pso_c1 * r[0] * (pb[j] - x[j]) +
                              p->pso_c2 * r[1] * (g[j] - x[j]);
            double xn = x[j] + vn;
            if (xn < p->L) xn = p->L;
            if (xn > p->U) xn = p->U;
            Xout[(int64_t)o * d + j] = xn;
            Vout[(int64_t)o * d + j] = vn;
        }
    }
}

/* Personal best of offspring o after its evaluation (the MOPSO rule of
 * Coello et al.): its new position x' unless the particle's personal best p
 * dominates it (f(p) <= f(x') in every objective and < in one), when p is
 * kept.  Pb / FPb: personal bests and their objectives by slot; Xc / Fc: the
 * offspring and their objectives; Pout / FPout: the offspring's bests. */
void orc_pso_pbest(const orc_params *p, int32_t t, int32_t K, const int32_t *vlist,
                   const double *Pb, const double *FPb, const double *Xc, const double *Fc,
                   double *Pout, double *FPout)
{
    const int32_t N = p->N, d = p->d, m = p->m;
    (void)t;
    for (int32_t o = 0; o < N; ++o) {
        const int32_t ip = vlist[o % K];
        const double *fp = FPb + (int64_t)ip * m, *fx = Fc + (int64_t)o * m;
        int le = 1, lt = 0;
        for (int32_t k = 0; k < m; ++k) {
            if (fp[k] > fx[k]) le = 0;
            if (fp[k] < fx[k]) lt = 1;
        }
        const int keep_old = le && lt;
        memcpy(Pout + (int64_t)o * d, keep_old ? Pb + (int64_t)ip * d : Xc + (int64_t)o * d,
               sizeof(double) * (size_t)d);
        memcpy(FPout + (int64_t)o * m, keep_old ? fp : fx, sizeof(double) * (size_t)m);
    }
}

/* Tensorized SBX, Appendix B (the two B equations and X_cross):
 *   B  = sgn(R1 - 1/2) [H(1/2 - Mc)(2Mc)^(1/(eta+1)) + (1 - H(1/2 - Mc))(2 - 2Mc)^(-1/(eta+1))]
 *   B  = [1 - rep(H(R3 - p_c))] [(1 - H(R2 - 1/2)) B + H(R2 - 1/2)] + rep(H(R3 - p_c))
 *   X_cross = [((1+B) X1 + (1-B) X2)/2 ; ((1-B) X1 + (1+B) X2)/2]
 * R1 and R2 enter only through sgn(R1 - 1/2) and H(R2 - 1/2): each is read as
 * a fair coin (bit 0 and bit 1 of the word that carries Mc).  The pair gate
 * H(R3 - p_c) is 0 (crossover happens) iff R3 < p_c.
 * X1, X2: P x d; Xcross: 2P x d. */
void orc_sbx(const orc_params *p, int32_t t, const double *X1, const double *X2,
             double *Xcross)
{
    const int32_t P = (p->N + 1) / 2, d = p->d;
    const double eta = p->eta_c;
    const uint32_t Tc = event_threshold(p->p_c);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int32_t pr = 0; pr < P; ++pr) {
        uint32_t g[4];
        philox(p, (uint32_t)pr, 0u, (uint32_t)t, ORC_TAG_PAIR, g);
        double no_cross = ((g[0] >> 8) < Tc) ? 0.0 : 1.0;   /* H(R3 - p_c) */
        for (int32_t j = 0; j < d; ++j) {
            uint32_t w[4];
            philox(p, (uint32_t)(j / 4), (uint32_t)pr, (uint32_t)t, ORC_TAG_SBX, w);
            uint32_t word = w[j % 4];
            double Mc = u24(word);
            double sgn = (word & 1u) ? 1.0 : -1.0;               /* sgn(R1 - 1/2) */
            double keep = (word & 2u) ? 1.0 : 0.0;               /* H(R2 - 1/2)   */
            double h = (Mc < 0.5) ? 1.0 : 0.0;                   /* H(1/2 - Mc)   */
            double beta = h * pow(2.0 * Mc, 1.0 / (eta + 1.0))
                        + (1.0 - h) * pow(2.0 - 2.0 * Mc, -1.0 / (eta + 1.0));
            double B = sgn * beta;
            B = (1.0 - no_cross) * ((1.0 - keep) * B + keep) + no_cross;
            double x1 = X1[(int64_t)pr * d + j], x2 = X2[(int64_t)pr * d + j];
            Xcross[(int64_t)pr * d + j] = ((1.0 + B) * x1 + (1.0 - B) * x2) / 2.0;
            Xcross[(int64_t)(pr + P) * d + j] = ((1.0 - B) * x1 + (1.0 + B) * x2) / 2.0;
        }
    }
}

/* Tensorized polynomial mutation, Appendix B (C, X_mut and Delta):
 *   C = H(p_m/d - R4),  X_mut = X_cross + Delta (.) C,
 *   Delta = (U-L)[(2M + (1-2M)(1-d1)^(xi+1))^(1/(xi+1)) - 1]   if M < 1/2
 *         = (U-L)[1 - (2(1-M) + 2(M-1/2)(1-d2)^(xi+1))^(1/(xi+1))]  if M > 1/2
 *   d1 = (x-L)/(U-L), d2 = (U-x)/(U-L).
 * The formula assumes x in [L,U] while SBX can leave the box: the reading
 * clips to [L,U] before and after.
 *
 * The mask C.  Appendix B draws one uniform R4 per site: the sites of a row
 * are independent events of probability q.  Here q is p_m/d on the 24-bit
 * grid, q = ceil(2^24 p_m/d) 2^-24 (q >= 1: every site; q = 0: none), and the
 * mask of row c is drawn in the equivalent count-then-subset form of that
 * law: the number of sites k ~ Binomial(d, q), then a uniform k-subset of
 * the d positions (given its size, the set of independent Bernoulli events
 * is a uniform subset).  Both steps use Philox at counter (i/4, c, t, MUTSITE),
 * word i%4, for draw i = 0, 1, 2, ...:
 *   draw 0:  k = #{ i < min(d, 32) : w >= thr_i },  thr_i = floor(2^32 CDF(i))
 *            (saturated at 2^32), CDF of Binomial(d, q) summed in FP64 from
 *            pmf(0) = (1-q)^d (square-and-multiply over the bits of d, least
 *            significant first) and pmf(i+1) = pmf(i) * (d-i) / (i+1) * (q/(1-q));
 *   draws 1..k: Floyd's subset sampler: for i = 0..k-1, J = d-k+i,
 *            r = (w * (J+1)) >> 32 (uniform in [0, J]); add J if r is already
 *            in the set, else add r.
 * Counts are capped at 32 (the caller keeps p_m <= 8, where the mass above 32
 * is below 2^-32).  The magnitude of site (c, j) is M = u24(word 1) of Philox
 * at (j, c, t, MUTMAG).
 * Xc holds the N kept offspring rows (the first N rows of X_cross), mutated
 * in place; mask (N x d, may be NULL) receives C. */
static double pow_uint(double b, int32_t e)
{
    double r = 1.0;
    while (e > 0) {
        if (e & 1) r *= b;
        b *= b;
        e >>= 1;
    }
    return r;
}

/* thresholds of the site count; returns how many are below 2^32 (<= 32) */
static int32_t site_count_thresholds(double q, int32_t d, uint64_t thr[32])
{
    const int32_t K = d < 32 ? d : 32;
    const double ratio = q / (1.0 - q);
    double pmf = pow_uint(1.0 - q, d), cdf = 0.0;
    int32_t n = 0;
    for (int32_t i = 0; i < K; ++i) {
        if (i > 0) pmf = pmf * (double)(d - (i - 1)) / (double)i * ratio;
        cdf += pmf;
        if (cdf >= 1.0) break;
        thr[n++] = (uint64_t)floor(cdf * 4294967296.0);
    }
    return n;
}

/* mutation sites of child row c (count-then-subset form above); returns k */
static int32_t mutation_sites(const orc_params *p, int32_t t, int32_t c, int32_t n_thr,
                              const uint64_t *thr, int32_t *sites)
{
    const int32_t d = p->d;
    uint32_t w[4];
    philox(p, 0u, (uint32_t)c, (uint32_t)t, ORC_TAG_MUTSITE, w);
    int32_t k = 0;
    for (int32_t i = 0; i < n_thr; ++i)
        if ((uint64_t)w[0] >= thr[i]) k = i + 1;
    for (int32_t i = 0; i < k; ++i) {
        const int32_t e = i + 1;
        if (e % 4 == 0) philox(p, (uint32_t)(e / 4), (uint32_t)c, (uint32_t)t, ORC_TAG_MUTSITE, w);
        const uint32_t J = (uint32_t)(d - k + i);
        uint32_t r = (uint32_t)(((uint64_t)w[e % 4] * (uint64_t)(J + 1u)) >> 32);
        for (int32_t l = 0; l < i; ++l)
            if ((uint32_t)sites[l] == r) { r = J; break; }
        sites[i] = (int32_t)r;
    }
    return k;
}

void orc_mutation(const orc_params *p, int32_t t, double *Xc, uint8_t *mask)
{
    const int32_t N = p->N, d = p->d;
    const double L = p->L, U = p->U, xi = p->eta_m;
    const uint32_t Tm = event_threshold(p->p_m / (double)d);
    const double q = (double)Tm / 16777216.0;
    uint64_t thr[32];
    const int32_t n_thr = (Tm > 0u && Tm < (1u << 24)) ? site_count_thresholds(q, d, thr) : 0;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int32_t c = 0; c < N; ++c) {
        uint8_t *C = (uint8_t *)calloc((size_t)d, 1);
        if (Tm >= (1u << 24)) {
            memset(C, 1, (size_t)d);
        } else if (Tm > 0u) {
            int32_t sites[32];
            const int32_t k = mutation_sites(p, t, c, n_thr, thr, sites);
            for (int32_t i = 0; i < k; ++i) C[sites[i]] = 1;
        }
        for (int32_t j = 0; j < d; ++j) {
            double x = Xc[(int64_t)c * d + j];
            if (x < L) x = L;
            if (x > U) x = U;
            double delta = 0.0;
            if (C[j]) {
                uint32_t wm[4];
                philox(p, (uint32_t)j, (uint32_t)c, (uint32_t)t, ORC_TAG_MUTMAG, wm);
                const double M = u24(wm[1]);
                const double d1 = (x - L) / (U - L), d2 = (U - x) / (U - L);
                if (M < 0.5)          /* H(0.5 - M) */
                    delta = (U - L) * (pow(2.0 * M + (1.0 - 2.0 * M) * pow(1.0 - d1, xi + 1.0),
                                           1.0 / (xi + 1.0)) - 1.0);
                else if (M > 0.5)     /* H(M - 0.5) */
                    delta = (U - L) * (1.0 - pow(2.0 * (1.0 - M) + 2.0 * (M - 0.5) * pow(1.0 - d2, xi + 1.0),
                                                 1.0 / (xi + 1.0)));
            }
            x = x + delta * (double)C[j];
            if (x < L) x = L;
            if (x > U) x = U;
            Xc[(int64_t)c * d + j] = x;
            if (mask) mask[(int64_t)c * d + j] = C[j];
        }
        free(C);
    }
}

/* ------------------------------------------------------------------------ */
/* Selection, Algorithm 1 with Eqs. 2-5.                                     */
/*   z* = min over the population (lines 3-4), F' = F - z*                   */
/*   Theta = arccos(F' V^T / (||F'|| ||V||)) (line 5)                        */
/*   A = RowMin index of Theta (line 6, Eq. 2), ties to the lower index      */
/*   APD_i = (1 + m (t/t_max)^alpha theta_i / gamma_{A_i}) ||f'_i|| (Eq. 4)  */
/*   survivor_j = column argmin of APD over {i : A_i = j}, inf elsewhere     */
/*   (lines 7-15); a column with no member is an invalid slot (Sec. 3.2).    */
/* Theta is evaluated one row at a time; only its row minimum is kept.       */
/* A solution equal to z* has 0/0 cosines: read as cos = 0 for every j, so   */
/* A_i = 0, theta_i = pi/2 and APD_i = 0.                                    */
/* ------------------------------------------------------------------------ */
void orc_select(int32_t m, int32_t n, const double *F, const uint8_t *valid,
                int32_t r, const double *V, const double *gamma,
                int32_t t, int32_t t_max, double alpha,
                double *zstar, int32_t *assoc, double *theta, double *apd,
                int32_t *survivor)
{
    double z[64];
    for (int32_t k = 0; k < m; ++k) {
        z[k] = INFINITY;
        for (int32_t i = 0; i < n; ++i) {
            if (valid && !valid[i]) continue;
            double f = F[(int64_t)i * m + k];
            if (f < z[k]) z[k] = f;
        }
        if (zstar) zstar[k] = z[k];
    }
    const double pen = (double)m * pow((double)t / (double)t_max, alpha);
    double *vn = (double *)malloc(sizeof(double) * (size_t)r);
    double *th_all = (double *)malloc(sizeof(double) * (size_t)n);
    double *apd_all = (double *)malloc(sizeof(double) * (size_t)n);
    for (int32_t j = 0; j < r; ++j)
        vn[j] = sqrt(dot(V + (int64_t)j * m, V + (int64_t)j * m, m));

#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        if (valid && !valid[i]) {
            assoc[i] = -1;
            th_all[i] = NAN;
            apd_all[i] = INFINITY;
            continue;
        }
        double fp[64];
        for (int32_t k = 0; k < m; ++k) fp[k] = F[(int64_t)i * m + k] - z[k];
        double nf = sqrt(dot(fp, fp, m));
        int32_t best_j = 0;
        double best_th = INFINITY;
        for (int32_t j = 0; j < r; ++j) {
            double c = (nf > 0.0) ? dot(fp, V + (int64_t)j * m, m) / (nf * vn[j]) : 0.0;
            double th = acos(clamp1(c));
            if (th < best_th) { best_th = th; best_j = j; }
        }
        assoc[i] = best_j;
        th_all[i] = best_th;
        apd_all[i] = (1.0 + pen * best_th / gamma[best_j]) * nf;
    }

    /* column argmin, scanned serially in increasing i: ties go to lower i */
    double *best = (double *)malloc(sizeof(double) * (size_t)r);
    for (int32_t j = 0; j < r; ++j) { best[j] = INFINITY; survivor[j] = -1; }
    for (int32_t i = 0; i < n; ++i) {
        int32_t j = assoc[i];
        if (j < 0) continue;
        if (survivor[j] < 0 || apd_all[i] < best[j]) {
            best[j] = apd_all[i];
            survivor[j] = i;
        }
    }
    if (theta) memcpy(theta, th_all, sizeof(double) * (size_t)n);
    if (apd) memcpy(apd, apd_all, sizeof(double) * (size_t)n);
    free(best);
    free(apd_all);
    free(th_all);
    free(vn);
}

/* ------------------------------------------------------------------------ */
/* One generation of Algorithm 2 on a population held in vector-slot order:  */
/* X (N x d), F (N x m), valid (N); V, gamma (N = r).  Offspring Q_t, union   */
/* with the valid parents (parents take combined indices j, children N + c), */
/* selection with V_t, then, every round(f_r t_max) generations, adaptation  */
/* of V from V0 and gamma.  Inspection outputs may be NULL.  Returns the     */
/* number of surviving slots.                                                */
/* ------------------------------------------------------------------------ */
int32_t orc_generation(const orc_params *p, int32_t t, const double *V0,
                       const orc_neuro *nd,
                       double *X, double *F, uint8_t *valid, double *V, double *gamma,
                       double *Xchild, double *Fchild, int32_t *parents,
                       int32_t *assoc, int32_t *survivor)
{
    return orc_generation_ex(p, t, V0, nd, X, F, valid, V, gamma, NULL, NULL, NULL, NULL,
                             Xchild, Fchild, parents, assoc, survivor);
}

/* The same with the swarm state of the CSO and PSO operators: Vel (N x d,
 * velocities by slot), apd (N, the APD that kept each member; +inf before
 * any selection), and for PSO Pb (N x d, personal bests) and FPb (N x m,
 * their objectives), all updated with the population.  They may be NULL for
 * the operators that do not use them (apd is then not kept). */
int32_t orc_generation_ex(const orc_params *p, int32_t t, const double *V0,
                          const orc_neuro *nd,
                          double *X, double *F, uint8_t *valid, double *V, double *gamma,
                          double *Vel, double *apd, double *Pb, double *FPb,
                          double *Xchild, double *Fchild, int32_t *parents,
                          int32_t *assoc, int32_t *survivor)
{
    const int32_t N = p->N, d = p->d, m = p->m, P = (p->N + 1) / 2;
    int32_t *vlist = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t K = 0;
    for (int32_t j = 0; j < N; ++j)
        if (valid[j]) vlist[K++] = j;
    if (K == 0) { free(vlist); return -1; }

    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * P));
    double *Xc = (double *)malloc(sizeof(double) * (size_t)(2 * P) * d);
    double *Vc = NULL;   /* the offspring's velocities (CSO, PSO) */
    double *Pc = NULL, *FPc = NULL;   /* the offspring's personal bests (PSO) */
    if (p->op == ORC_OP_DE) {
        /* the extensibility experiment's operators replace SBX and mutation */
        for (int32_t e = 0; e < 2 * P; ++e) par[e] = -1;
        orc_de_offspring(p, t, X, K, vlist, p->de_F, p->de_CR, Xc);
    } else if (p->op == ORC_OP_RANDOM) {
        for (int32_t e = 0; e < 2 * P; ++e) par[e] = -1;
        orc_random_offspring(p, t, Xc);
    } else if (p->op == ORC_OP_CSO) {
        for (int32_t e = 0; e < 2 * P; ++e) par[e] = -1;
        if (!Vel || !apd) { free(vlist); free(par); free(Xc); return -1; }
        double *xbar = (double *)calloc((size_t)d, sizeof(double));
        for (int32_t k = 0; k < K; ++k)
            for (int32_t j = 0; j < d; ++j) xbar[j] += X[(int64_t)vlist[k] * d + j];
        for (int32_t j = 0; j < d; ++j) xbar[j] /= (double)K;
        Vc = (double *)malloc(sizeof(double) * (size_t)N * d);
        orc_cso_offspring(p, t, X, Vel, apd, K, vlist, xbar, Xc, Vc);
        free(xbar);
    } else if (p->op == ORC_OP_PSO) {
        for (int32_t e = 0; e < 2 * P; ++e) par[e] = -1;
        if (!Vel || !apd || !Pb || !FPb) { free(vlist); free(par); free(Xc); return -1; }
        Vc = (double *)malloc(sizeof(double) * (size_t)N * d);
        orc_pso_offspring(p, t, X, Vel, Pb, apd, K, vlist, Xc, Vc);
    } else {
        orc_mating(p, t, K, vlist, par);
        double *X1 = (double *)malloc(sizeof(double) * (size_t)P * d);
        double *X2 = (double *)malloc(sizeof(double) * (size_t)P * d);
        for (int32_t q = 0; q < P; ++q) {
            memcpy(X1 + (int64_t)q * d, X + (int64_t)par[q] * d, sizeof(double) * (size_t)d);
            memcpy(X2 + (int64_t)q * d, X + (int64_t)par[P + q] * d, sizeof(double) * (size_t)d);
        }
        orc_sbx(p, t, X1, X2, Xc);
        free(X1);
        free(X2);
        /* keep the first N rows of X_cross */
        orc_mutation(p, t, Xc, NULL);
    }
    double *Fc = (double *)malloc(sizeof(double) * (size_t)N * m);
    orc_evaluate(p, N, Xc, Fc, nd, t);
    if (p->op == ORC_OP_PSO) {
        Pc = (double *)malloc(sizeof(double) * (size_t)N * d);
        FPc = (double *)malloc(sizeof(double) * (size_t)N * m);
        orc_pso_pbest(p, t, K, vlist, Pb, FPb, Xc, Fc, Pc, FPc);
    }

    /* combined population: parents (slot order) then children */
    const int32_t n = 2 * N;
    double *Fall = (double *)malloc(sizeof(double) * (size_t)n * m);
    uint8_t *vall = (uint8_t *)malloc((size_t)n);
    memcpy(Fall, F, sizeof(double) * (size_t)N * m);
    memcpy(Fall + (int64_t)N * m, Fc, sizeof(double) * (size_t)N * m);
    for (int32_t j = 0; j < N; ++j) { vall[j] = valid[j]; vall[N + j] = 1; }
    int32_t *as = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sv = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    double *apd_all = (double *)malloc(sizeof(double) * (size_t)n);
    orc_select(m, n, Fall, vall, N, V, gamma, t, p->t_max, p->alpha,
               NULL, as, NULL, apd_all, sv);

    if (Xchild) memcpy(Xchild, Xc, sizeof(double) * (size_t)N * d);
    if (Fchild) memcpy(Fchild, Fc, sizeof(double) * (size_t)N * m);
    if (parents) memcpy(parents, par, sizeof(int32_t) * (size_t)(2 * P));
    if (assoc) memcpy(assoc, as, sizeof(int32_t) * (size_t)n);
    if (survivor) memcpy(survivor, sv, sizeof(int32_t) * (size_t)N);

    /* P_{t+1}: slot j holds the survivor of vector j (with its velocity and
     * the APD it was kept with) */
    double *Xn = (double *)malloc(sizeof(double) * (size_t)N * d);
    double *Fn = (double *)malloc(sizeof(double) * (size_t)N * m);
    double *Vn = Vel ? (double *)malloc(sizeof(double) * (size_t)N * d) : NULL;
    double *Pn = Pb ? (double *)malloc(sizeof(double) * (size_t)N * d) : NULL;
    double *FPn = FPb ? (double *)malloc(sizeof(double) * (size_t)N * m) : NULL;
    int32_t alive = 0;
    for (int32_t j = 0; j < N; ++j) {
        int32_t i = sv[j];
        if (i < 0) {
            valid[j] = 0;
            for (int32_t k = 0; k < d; ++k) Xn[(int64_t)j * d + k] = NAN;
            for (int32_t k = 0; k < m; ++k) Fn[(int64_t)j * m + k] = NAN;
            if (Vn) for (int32_t k = 0; k < d; ++k) Vn[(int64_t)j * d + k] = NAN;
            if (Pn) for (int32_t k = 0; k < d; ++k) Pn[(int64_t)j * d + k] = NAN;
            if (FPn) for (int32_t k = 0; k < m; ++k) FPn[(int64_t)j * m + k] = NAN;
            if (apd) apd[j] = INFINITY;
            continue;
        }
        valid[j] = 1;
        ++alive;
        const double *xs = (i < N) ? X + (int64_t)i * d : Xc + (int64_t)(i - N) * d;
        const double *fs = Fall + (int64_t)i * m;
        memcpy(Xn + (int64_t)j * d, xs, sizeof(double) * (size_t)d);
        memcpy(Fn + (int64_t)j * m, fs, sizeof(double) * (size_t)m);
        if (Vn) {
            double *vd = Vn + (int64_t)j * d;
            if (i < N) memcpy(vd, Vel + (int64_t)i * d, sizeof(double) * (size_t)d);
            else if (Vc) memcpy(vd, Vc + (int64_t)(i - N) * d, sizeof(double) * (size_t)d);
            else for (int32_t k = 0; k < d; ++k) vd[k] = 0.0;
        }
        if (Pn) {   /* a parent keeps its personal best; a child carries its own */
            double *pd = Pn + (int64_t)j * d, *fpd = FPn + (int64_t)j * m;
            const double *ps = (i < N) ? Pb + (int64_t)i * d
                             : Pc ? Pc + (int64_t)(i - N) * d : Xc + (int64_t)(i - N) * d;
            const double *fps = (i < N) ? FPb + (int64_t)i * m
                              : FPc ? FPc + (int64_t)(i - N) * m : Fc + (int64_t)(i - N) * m;
            memcpy(pd, ps, sizeof(double) * (size_t)d);
            memcpy(fpd, fps, sizeof(double) * (size_t)m);
        }
        if (apd) apd[j] = apd_all[i];
    }
    memcpy(X, Xn, sizeof(double) * (size_t)N * d);
    memcpy(F, Fn, sizeof(double) * (size_t)N * m);
    if (Vn) { memcpy(Vel, Vn, sizeof(double) * (size_t)N * d); free(Vn); }
    if (Pn) { memcpy(Pb, Pn, sizeof(double) * (size_t)N * d); free(Pn); }
    if (FPn) { memcpy(FPb, FPn, sizeof(double) * (size_t)N * m); free(FPn); }

    /* reference-vector adaptation every round(f_r * t_max) generations */
    int32_t period = (int32_t)floor(p->f_r * (double)p->t_max + 0.5);
    if (period < 1) period = 1;
    if (t % period == 0) {
        double range[64];
        orc_objective_range(m, N, F, valid, range);
        orc_adapt(m, N, V0, range, V);
        orc_gamma(m, N, V, gamma);
    }

    free(Xn); free(Fn); free(as); free(sv); free(vall); free(Fall); free(apd_all);
    free(Fc); free(Xc); free(Vc); free(Pc); free(FPc); free(par); free(vlist);
    return alive;
}
