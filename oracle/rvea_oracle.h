/*
 * FP64 CPU oracle of one generation of tensorized RVEA.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this code: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py use it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Every function states the passage of arXiv 2404.01159 ("GPU-accelerated
 * Evolutionary Multiobjective Optimization Using Tensorized RVEA") it follows.
 * Where the paper is silent the reading used is stated beside the function.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11), written here from that definition.
 * Counter layout (key = seed lo/hi 32 bits; c2 = generation t; c3 = tag):
 *   INIT   (j/4, i, 0, 1)  word j%4   -> x_ij = L + (U-L) * u24
 *   MATE   (e/4, 0, t, 2)  word e%4   -> parent draw e, index (w*K)>>32
 *   PAIR   (p,   0, t, 3)  word 0     -> R3 of pair p (u24)
 *   SBX    (j/4, p, t, 4)  word j%4   -> Mc = u24(w), sign coin bit0, keep coin bit1
 *   MUTSITE(i/4, c, t, 5)  word i%4 -> draw i of child c's mutation sites:
 *                          draw 0 the site count, draws 1..k Floyd's subset
 *   MUTMAG (j,   c, t, 6)  word1 -> M_mut (u24) of site j of child c
 *   INIT   (j,   i, 0, 1)  words 0,1 -> Box-Muller N(0,1) (neuroevolution weights)
 *   NOISE  (k,   s, t, 7)  words 0,1 -> Box-Muller N(0,1), state component k, step s
 *   CSO_PICK (o, 0, t, 11) words 0,1 -> the two competitors of offspring o
 *   CSO_R  (3(j/4)+k, o, t, 12) word j%4 -> r_{k+1} (u24), k = 0,1,2, of variable j of
 *                          offspring o
 *   PSO_PICK (o, 0, t, 13) words 0,1 -> the two candidates for offspring o's leader
 *   PSO_R  (2(j/4)+k, o, t, 14) word j%4 -> r_{k+1} (u24), k = 0,1, of variable j of
 *                          offspring o
 * where u24(w) = (w >> 8) * 2^-24.
 */
#ifndef RVEA_ORACLE_H
#define RVEA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_DTLZ2 = 0, ORC_DTLZ1 = 1, ORC_NEURO = 2, ORC_DTLZ3 = 3, ORC_DTLZ4 = 4 };
enum { ORC_TAG_INIT = 1, ORC_TAG_MATE = 2, ORC_TAG_PAIR = 3, ORC_TAG_SBX = 4,
       ORC_TAG_MUTSITE = 5, ORC_TAG_MUTMAG = 6, ORC_TAG_NOISE = 7,
       ORC_TAG_DE_PICK = 8, ORC_TAG_DE_CR = 9, ORC_TAG_RANDOM = 10,
       ORC_TAG_CSO_PICK = 11, ORC_TAG_CSO_R = 12, ORC_TAG_PSO_PICK = 13, ORC_TAG_PSO_R = 14 };

typedef struct {
    int32_t m, d, N, H;
    int32_t problem;
    int32_t t_max;
    double alpha, f_r, eta_c, eta_m, p_c, p_m, L, U;
    uint64_t seed;
    int32_t op;               /* reproduction: ORC_OP_SBX_PM, ORC_OP_DE, ORC_OP_RANDOM */
    double de_F, de_CR;       /* DE/rand/1/bin scale factor and crossover rate   */
    double cso_phi;           /* CSO: weight of the swarm-centre term            */
    double pso_w, pso_c1, pso_c2;   /* PSO: inertia weight, cognitive and social  */
} orc_params;

/* Reproduction operators (Sec. 4.4, the extensibility experiment): SBX with
 * polynomial mutation (Appendix B), DE/rand/1/bin, random reproduction, the
 * competitive swarm optimizer. */
enum { ORC_OP_SBX_PM = 0, ORC_OP_DE = 1, ORC_OP_RANDOM = 2, ORC_OP_CSO = 3, ORC_OP_PSO = 4 };

/* Synthetic linear-dynamics rollout used as the neuroevolution objective. */
typedef struct {
    int32_t ns, na, h1, h2;   /* state, action, hidden sizes (17, 6, 64, 64)   */
    int32_t steps;            /* rollout length                                */
    double sigma;             /* process-noise standard deviation              */
    const double *A;          /* ns x ns, row-major                            */
    const double *B;          /* ns x na, row-major                            */
} orc_neuro;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

int64_t orc_lattice_count(int32_t m, int32_t H);
int32_t orc_lattice_for(int32_t m, int32_t n);
int32_t orc_lattice(int32_t m, int32_t H, int32_t N, int32_t *K);
void orc_lattice_unit(int32_t m, int32_t N, const int32_t *K, double *V0);
void orc_gamma(int32_t m, int32_t r, const double *V, double *gamma);
void orc_objective_range(int32_t m, int32_t n, const double *F, const uint8_t *valid,
                         double *range);
void orc_adapt(int32_t m, int32_t r, const double *V0, const double *range, double *V);

void orc_init_population(const orc_params *p, double *X);
void orc_evaluate(const orc_params *p, int32_t n, const double *X, double *F,
                  const orc_neuro *nd, int32_t t);
void orc_neuro_noise(const orc_params *p, const orc_neuro *nd, int32_t t, double *xi);
void orc_mating(const orc_params *p, int32_t t, int32_t K, const int32_t *vlist,
                int32_t *parents);
void orc_sbx(const orc_params *p, int32_t t, const double *X1, const double *X2,
             double *Xcross);
void orc_mutation(const orc_params *p, int32_t t, double *Xc, uint8_t *mask);
void orc_select(int32_t m, int32_t n, const double *F, const uint8_t *valid,
                int32_t r, const double *V, const double *gamma,
                int32_t t, int32_t t_max, double alpha,
                double *zstar, int32_t *assoc, double *theta, double *apd,
                int32_t *survivor);
int32_t orc_generation(const orc_params *p, int32_t t, const double *V0,
                       const orc_neuro *nd,
                       double *X, double *F, uint8_t *valid, double *V, double *gamma,
                       double *Xchild, double *Fchild, int32_t *parents,
                       int32_t *assoc, int32_t *survivor);

void orc_random_offspring(const orc_params *p, int32_t t, double *Xout);
void orc_de_picks(const orc_params *p, int32_t t, int32_t K, int32_t o, int32_t *out);
void orc_de_offspring(const orc_params *p, int32_t t, const double *X, int32_t K,
                      const int32_t *vlist, double F, double CR, double *Xout);
void orc_cso_picks(const orc_params *p, int32_t t, int32_t K, int32_t o, int32_t *out);
void orc_cso_offspring(const orc_params *p, int32_t t, const double *X, const double *Vel,
                       const double *apd, int32_t K, const int32_t *vlist, const double *xbar,
                       double *Xout, double *Vout);
void orc_pso_picks(const orc_params *p, int32_t t, int32_t K, int32_t o, int32_t *out);
void orc_pso_offspring(const orc_params *p, int32_t t, const double *X, const double *Vel,
                       const double *Pb, const double *apd, int32_t K, const int32_t *vlist,
                       double *Xout, double *Vout);
void orc_pso_pbest(const orc_params *p, int32_t t, int32_t K, const int32_t *vlist,
                   const double *Pb, const double *FPb, const double *Xc, const double *Fc,
                   double *Pout, double *FPout);
int32_t orc_generation_ex(const orc_params *p, int32_t t, const double *V0,
                          const orc_neuro *nd,
                          double *X, double *F, uint8_t *valid, double *V, double *gamma,
                          double *Vel, double *apd, double *Pb, double *FPb,
                          double *Xchild, double *Fchild, int32_t *parents,
                          int32_t *assoc, int32_t *survivor);
void orc_set_threads(int32_t n);
int32_t orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
