/*
 * rvea.h -- C ABI of the GB300 (sm_103a) tensorized-RVEA library.
 *
 * One call of rvea_step runs whole generations of RVEA (arXiv 2404.01159,
 * Algorithm 2) for a population resident in device memory:
 *   reproduction  -- SBX crossover and polynomial mutation, Appendix B
 *   evaluation    -- DTLZ1 / DTLZ2 (Sec. 4.1) or a policy rollout (Sec. 4.3)
 *   selection     -- ideal point, angle association, APD and per-vector
 *                    argmin, Algorithm 1 with Eqs. 2-5
 *   adaptation    -- reference-vector rescaling and gamma (Eq. 5) every
 *                    round(f_r * t_max) generations
 *
 * Conventions shared by every entry point:
 *  - Memory: the caller owns all device memory.  It allocates the workspace
 *    (rvea_workspace_bytes) and every output buffer; the library allocates
 *    nothing on the device and keeps only a small host handle.  A workspace
 *    must stay allocated, untouched, until rvea_free.
 *  - Pointers: an argument documented as "host or device" may be a device
 *    pointer, a pinned (page-locked) host pointer or ordinary pageable host
 *    memory; the kind is found with cudaPointerGetAttributes.
 *  - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 *    All work is enqueued asynchronously on it; results written to host
 *    memory are complete only after the stream is synchronised.
 *  - Layouts: row-major, C order.  Population rows and reference vectors are
 *    reported in reference-vector slot order: row j holds the survivor kept
 *    by vector j, or an invalid slot (valid[j] = 0, values NaN) when no
 *    solution associated with vector j (Sec. 3.2, end of Algorithm 1).
 *  - Errors: status codes only; nothing throws across this boundary.  Faults
 *    found on the device (a timed-out wait, an out-of-range index) set a
 *    device status word that rvea_sync_status reports.
 */
#ifndef RVEA_H
#define RVEA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rvea_run rvea_run;   /* opaque host handle */

typedef enum {
    RVEA_OK = 0,
    RVEA_ERR_ARG = -1,      /* an argument is out of range                 */
    RVEA_ERR_LATTICE = -2,  /* N != C(H+m-1, m-1)                           */
    RVEA_ERR_NOMEM = -3,    /* workspace or scratch smaller than required  */
    RVEA_ERR_CUDA = -4,     /* a CUDA runtime call failed                  */
    RVEA_ERR_TIMEOUT = -5,  /* a bounded device wait gave up               */
    RVEA_ERR_STATE = -6,    /* call not valid in the run's current state   */
    RVEA_ERR_DEVICE = -7    /* a device-side check failed (bad index)      */
} rvea_status;

typedef enum {
    RVEA_DTLZ2_SPHERE = 0,  /* spherical front, |f| = 1 on the front       */
    RVEA_DTLZ1_LINEAR = 1,  /* multimodal linear front, sum f = 1/2        */
    RVEA_NEURO_LINEAR = 2,  /* MLP policy rollout on linear dynamics       */
    RVEA_DTLZ3_SPHERE = 3,  /* DTLZ1's multimodal g on DTLZ2's sphere      */
    RVEA_DTLZ4_SPHERE = 4   /* DTLZ2 with x_i^100 position variables       */
} rvea_problem;

/* Synthetic linear dynamics of the neuroevolution objective (the stand-in
 * for the paper's Brax tasks, Sec. 4.3 and Appendix C):
 *   policy x = [W1 (h1 x ns), b1 (h1), W2 (h2 x h1), b2 (h2), W3 (na x h2), b3 (na)],
 *   u = tanh(W3 tanh(W2 tanh(W1 s + b1) + b2) + b3), s_0 = 0,
 *   s' = A s + B u + sigma * xi,  xi ~ N(0, I) per step, shared by all
 *   policies of one generation;
 *   f1 = -sum_steps s'[0],  f2 = sum_steps |u|^2.
 * A (ns x ns) and B (ns x na) are host pointers, row-major, read during the
 * rvea_init_ex call only.  Supported sizes: ns <= 32, na <= 16, h1 = h2 = 64. */
typedef struct {
    int ns, na, h1, h2;
    int steps;
    double sigma;
    const double *A;
    const double *B;
    int gemv;         /* 0: the policy GEMVs on the tensor cores, BF16 operands
                         split in hi and lo parts, FP32 accumulate; 1: on the
                         CUDA cores in FP32, the hidden layer's weights held
                         in registers (needs ns <= 24 and na <= 8, else
                         RVEA_ERR_ARG); the faster of the two on a GB300
                         (7.3 against 13.0 ms for 10^4 1000-step rollouts)  */
} rvea_neuro_dynamics;

/* All parameters of one optimisation run. */
typedef struct {
    int m;            /* objectives, 2..16                                   */
    int d;            /* decision variables, m..(1<<22)                      */
    int N;            /* population = number of reference vectors, 2..32768 */
    int H;            /* lattice divisions; N must equal C(H+m-1, m-1)        */
    int problem;      /* rvea_problem                                        */
    int t_max;        /* generations of the run (APD penalty schedule), >= 1 */
    double alpha;     /* APD penalty exponent, Eq. 4, > 0                    */
    double f_r;       /* adaptation frequency: every round(f_r*t_max) gens  */
    double eta_c;     /* SBX distribution index, > 0                         */
    double eta_m;     /* mutation distribution index xi, > 0                 */
    double p_c;       /* crossover probability per pair, [0,1]               */
    double p_m;       /* mutation rate: per-site probability p_m / d, >= 0   */
    double lower;     /* box [lower, upper] of every decision variable; the
                         DTLZ problems require [0, 1], their domain          */
    double upper;
    uint64_t seed;    /* Philox4x32-10 key                                   */
    const rvea_neuro_dynamics *neuro;   /* required iff problem == NEURO     */
    int reproduction; /* rvea_reproduction (0: SBX + polynomial mutation)   */
    double de_F;      /* DE/rand/1/bin scale factor, (0, 2]                  */
    double de_CR;     /* DE/rand/1/bin crossover rate, [0, 1]                */
    double cso_phi;   /* CSO: weight of the swarm-centre term, [0, 1]        */
    double pso_w;     /* PSO: inertia weight, [0, 1] (0.7298 is Clerc's)     */
    double pso_c1;    /* PSO: cognitive weight, [0, 4] (1.49618)             */
    double pso_c2;    /* PSO: social weight, [0, 4] (1.49618)                */
} rvea_config;

/* Reproduction operators (Sec. 4.4, the extensibility experiment: the same
 * selection with another offspring generator).  RVEA_REPRO_DE and
 * RVEA_REPRO_RANDOM replace SBX and polynomial mutation: DE/rand/1/bin (Storn
 * and Price) makes offspring o from the target at position o mod K of the
 * valid list and an ordered triple of other distinct members, v = x_r1 +
 * F (x_r2 - x_r3), binomial crossover with rate CR and one forced variable,
 * clipped to the box; random reproduction draws every variable uniformly on
 * the box.  RVEA_REPRO_CSO is the competitive swarm optimizer (Cheng and
 * Jin, IEEE T-Cyb 2015), which the paper names among the operators it plugs
 * into the same selection without printing it; read here as: offspring o is
 * one competition between two distinct valid members (uniform, drawn one
 * after the other), the one kept with the smaller APD (Eq. 4) wins (ties:
 * the smaller slot), and the loser learns, v' = r1 v_l + r2 (x_w - x_l) +
 * phi r3 (xbar - x_l), x' = clip(x_l + v'), with r1..r3 uniform per
 * variable and xbar the mean position of the valid members.  Velocities
 * (zero at first) and kept APDs (+inf before the first selection) stay
 * with the survivors.  RVEA_REPRO_PSO is particle swarm optimization
 * (Kennedy and Eberhart 1995, Shi and Eberhart's inertia weight), also named
 * by the paper and not printed; read here after the multiobjective PSO of
 * Coello, Pulido and Lechuga (2004), the population taking the archive's
 * role: particle o is the member at position o mod K of the valid list, its
 * leader g the winner of an APD tournament between two distinct valid
 * members, v' = w v + c1 r1 (p - x) + c2 r2 (g - x), x' = clip(x + v');
 * the offspring's personal best p is x' unless the particle's personal best
 * dominates f(x') (then that best is kept).  Velocities (zero at first),
 * personal bests (the initial positions at first), their objectives and the
 * kept APDs stay with the survivors.  DE, random reproduction and PSO serve
 * the DTLZ problems; CSO serves them and the rollout problem (whose
 * children the rollout evaluates). */
typedef enum {
    RVEA_REPRO_SBX_PM = 0,
    RVEA_REPRO_DE = 1,
    RVEA_REPRO_RANDOM = 2,
    RVEA_REPRO_CSO = 3,
    RVEA_REPRO_PSO = 4
} rvea_reproduction;

/* Lattice divisions H for a requested population size n that need not be a
 * lattice size (the speed sweeps of Sec. 4.1 use n = 2^5 .. 2^14 and n =
 * 100): the largest H with C(H+m-1, m-1) <= n, so that the reference
 * vectors are the largest Das-Dennis lattice with at most n points -- what a
 * uniform-point generator gives -- and the run's N is that lattice's size.
 * -1 if m < 2 or even H = 1 has more than n points.  Host only. */
int rvea_lattice_for(int m, int n);

/* Bytes of device workspace a run of this shape needs (0 if invalid).
 * DTLZ problems only; the rollout problem adds its noise table and dynamics:
 * use rvea_workspace_bytes_ex. */
size_t rvea_workspace_bytes(int m, int d, int N);

/* Bytes of device workspace the run `cfg` needs (0 if cfg is invalid). */
size_t rvea_workspace_bytes_ex(const rvea_config *cfg);

/* Create a run: builds the Das-Dennis lattice V0 (unit vectors), gamma(V0),
 * draws and evaluates the initial population (Algorithm 2, initialisation)
 * on `cuda_stream`.  The population uses p_c = 1, p_m = 1 (per-site 1/d),
 * box [0,1] for DTLZ and [-1,1] for the rollout problem.
 * dev_workspace: device pointer, 256-byte aligned, >= rvea_workspace_bytes.
 * Errors: RVEA_ERR_LATTICE if N != C(H+m-1,m-1); RVEA_ERR_ARG for m < 2,
 * d < m, t_max < 1, eta <= 0, f_r outside (0,1], unknown problem;
 * RVEA_ERR_NOMEM if `bytes` is too small.  *out is set only on success. */
rvea_status rvea_init(int m, int d, int N, int H, double alpha, double f_r,
                      double eta_c, double eta_m, uint64_t seed,
                      int problem, int t_max, void *dev_workspace, size_t bytes,
                      void *cuda_stream, rvea_run **out);

/* As rvea_init with every parameter explicit (needed for the rollout).
 * Also RVEA_ERR_ARG for a DTLZ problem on a box other than [0, 1]. */
rvea_status rvea_init_ex(const rvea_config *cfg, void *dev_workspace, size_t bytes,
                         void *cuda_stream, rvea_run **out);

/* Enqueue n_generations >= 0 generations on `cuda_stream` (asynchronous;
 * no host synchronisation).  Generation t is the run's next generation
 * index (1-based); a run may continue past t_max, the penalty term
 * (t/t_max)^alpha then exceeding 1. */
rvea_status rvea_step(rvea_run *run, int n_generations, void *cuda_stream);

/* One generation of each of n_runs distinct runs, packed into one launch
 * per phase.  Every run's result is identical to what rvea_step(run, 1)
 * gives.  All runs must live on the current device. */
rvea_status rvea_step_batch(rvea_run *const *runs, int n_runs, void *cuda_stream);

/* Kernel variants of a run (its "plan").  None of them changes a result bit:
 *   sel_mode   0: association by the full scan of every reference vector
 *                 (Algorithm 1, lines 5-6), tiled into work items of
 *                 (256 solutions x a chunk of vectors), sel_per_sm items per
 *                 SM (1..16): the chunk size;
 *              (the full-scan table is kept for every mode, so sel_per_sm
 *              is always 1..16);
 *              1: the exact pruned search with its tile tables in shared
 *                 memory (one run per launch); 2: the same search with the
 *                 tables read through L1 (the form batches use);
 *              3: mode 1's search inside one persistent launch (one CTA per
 *                 SM) that also mutates and evaluates the children and
 *                 builds the next population (the "fused tail"), grid
 *                 phases separated by time-limited grid barriers; DTLZ
 *                 problems, stepped alone (in a batch it runs as mode 2).
 *                 Modes 1-3 need m <= 4 and N >= 1000; a run that has mode 3
 *                 starts in it;
 *   repro_staged 1: parents staged in shared memory by TMA bulk copies
 *                 (runs with d > 1024), 0: loaded directly.
 * repro_us / sel_us: the autotuner's median launch times (0 if untuned). */
typedef struct {
    int sel_mode;
    int sel_per_sm;
    int repro_staged;
    double repro_us;
    double sel_us;
} rvea_plan;

/* The run's current plan. */
rvea_status rvea_get_plan(const rvea_run *run, rvea_plan *out);

/* Sets the plan (synchronises `cuda_stream`).  RVEA_ERR_ARG for a variant
 * the run's shape does not have (see rvea_plan). */
rvea_status rvea_set_plan(rvea_run *run, const rvea_plan *plan, void *cuda_stream);

/* Autotuner: times every variant of the run's plan on its current
 * generation -- the reproduction and association launches of a generation
 * are idempotent, so the run is neither advanced nor changed -- and keeps
 * the fastest of each phase.  Synchronous.  With use_cache != 0 a plan
 * already tuned for the same (m, d, N, problem) in this process is reused
 * without timing.  out (may be NULL) receives the plan and its times. */
rvea_status rvea_autotune(rvea_run *run, void *cuda_stream, int use_cache, rvea_plan *out);

/* A fixed set of runs stepped together: one batched generation (the
 * reproduction of all runs, the pruned association of the runs whose plan
 * uses it, the full scan of the others, finalize, and gamma plus the tile
 * tables of the runs that adapt) captured once as a CUDA graph and replayed
 * once per generation.  Each run's results are the bits rvea_step gives.
 * The plans are read at creation: re-create the batch after rvea_set_plan
 * or rvea_autotune.  1 <= n_runs <= 320, runs distinct; the runs must not
 * be stepped otherwise while the batch is in use. */
typedef struct rvea_batch rvea_batch;
rvea_status rvea_batch_create(rvea_run *const *runs, int n_runs, rvea_batch **out);

/* Enqueue n_generations >= 0 batched generations on `cuda_stream`. */
rvea_status rvea_batch_step(rvea_batch *batch, int n_generations, void *cuda_stream);

/* Kernel launches of one batched generation (the kernel nodes of its graph;
 * gamma and the tile tables launch every generation and act on their flag);
 * -1 if batch is NULL. */
int rvea_batch_launches_per_step(const rvea_batch *batch);

/* As rvea_batch_step with direct launches (no graph) and CUDA events around
 * every phase; synchronous.  phase_ms[0..4] (n_phases >= 5) receive the
 * summed device time of: reproduction, pruned association, full-scan
 * association, finalize, gamma plus tile tables. */
rvea_status rvea_batch_step_profiled(rvea_batch *batch, int n_generations, void *cuda_stream,
                                     double *phase_ms, int n_phases);

void rvea_batch_free(rvea_batch *batch);

/* Copy the population (N x d float32, slot order) and the valid flags
 * (N uint8, may be NULL).  dst, valid: host or device. */
rvea_status rvea_population(const rvea_run *run, float *dst, uint8_t *valid,
                            void *cuda_stream);

/* Copy the objective values (N x m float32, slot order) and valid flags. */
rvea_status rvea_objectives(const rvea_run *run, float *dst, uint8_t *valid,
                            void *cuda_stream);

/* Synchronise `run`'s last stream and report the device status word:
 * RVEA_OK, RVEA_ERR_TIMEOUT or RVEA_ERR_DEVICE. */
rvea_status rvea_sync_status(rvea_run *run);

/* Release the host handle (the caller frees the workspace afterwards). */
void rvea_free(rvea_run *run);

const char *rvea_status_str(rvea_status s);

/* The CUDA call and error string behind the calling thread's most recent
 * RVEA_ERR_CUDA ("" if none).  Valid until the next call on this thread. */
const char *rvea_last_cuda_error(void);

/* ---- inspection, checkpoint and teacher forcing ---------------------- */

/* Index of the next generation rvea_step will run (1 after init). */
int rvea_generation(const rvea_run *run);

/* As rvea_step with direct launches, a CUDA event recorded on `cuda_stream`
 * around every kernel, and a synchronisation at the end; adds the measured
 * device milliseconds per phase into phase_ms: [0] the reproduction kernel
 * (with mutation and evaluation when d <= 1024), [1] selection, [2]
 * finalize, [3] gamma and the tile table, [4] the kernels that finish the
 * children after it (mutation and evaluation when d > 1024, the rollout
 * evaluation of the neuroevolution problem).  With n_phases == 4, [4] is
 * added into [0].  phase_ms: host, n_phases >= 4.  Same results as
 * rvea_step. */
rvea_status rvea_step_profiled(rvea_run *run, int n_generations, void *cuda_stream,
                               double *phase_ms, int n_phases);

/* Inverted generational distance (Appendix C, the IGD equation) of the
 * run's current population against n_ref reference points: the mean over
 * the points of the Euclidean distance to the nearest objective vector of a
 * valid member.  ref: n_ref x m float32, row-major, device memory (or mapped
 * host memory); *out (host) receives the value; synchronises `cuda_stream`
 * and uses the run's staging area (stream-ordered with the run's other
 * calls).  Distances in float32, their roots and sum in FP64.  RVEA_ERR_ARG
 * for a NULL or non-device pointer, n_ref < 1, or more than about 2048 N
 * points; RVEA_ERR_STATE when the population has no valid member. */
rvea_status rvea_igd(const rvea_run *run, const float *ref, int n_ref, double *out,
                     void *cuda_stream);

/* Hypervolume (Appendix C, the HV equation) of the run's current population,
 * m = 2 or 3: the measure of the union of the boxes [f, ref] over the valid
 * members f that dominate ref (f < ref in every objective); objectives as
 * stored (normalise through ref).  ref: host, m finite values; *out (host)
 * receives the value; synchronises `cuda_stream` and uses the run's staging
 * area.  O(N^2) work (members ranked by counting, one warp per f3 slab), in
 * FP64 from the float32 objectives.  RVEA_ERR_ARG for NULL pointers, m > 3
 * or a non-finite ref. */
rvea_status rvea_hypervolume(const rvea_run *run, const double *ref, double *out,
                             void *cuda_stream);

/* Failure-detection self-test: one kernel waits, with a limit of `polls`
 * (1..2^20) mbarrier polls, on a barrier that nothing arrives at, as the
 * reproduction and association kernels wait for their copies.  Returns
 * RVEA_ERR_TIMEOUT when the wait gave up and reported it (the designed
 * outcome; the context stays usable), RVEA_OK if the barrier completed
 * (cannot happen), RVEA_ERR_ARG for polls out of range, RVEA_ERR_CUDA on a
 * launch or copy error.  Synchronises `cuda_stream`; uses no run. */
rvea_status rvea_selftest_wait(int polls, void *cuda_stream);

/* Kernel launches rvea_step enqueues for one generation of `run` (adapting:
 * a generation with t % round(f_r t_max) == 0, which also rescales V); -1 if
 * run is NULL. */
int rvea_launches_per_generation(const rvea_run *run, int adapting);

/* Full run state in slot order: X (N x d f32), F (N x m f32), valid (N u8),
 * V (N x m f64, current reference vectors), gamma (N f64).  Any output may
 * be NULL.  Host or device pointers.  Together with rvea_generation (and,
 * for the CSO and PSO operators, rvea_export_swarm) this is a checkpoint:
 * Philox is counter-based, so no generator state exists. */
rvea_status rvea_export_state(const rvea_run *run, float *X, float *F, uint8_t *valid,
                              double *V, double *gamma, void *cuda_stream);

/* Replace the run state (same layouts as rvea_export_state; all required)
 * and set the next generation index to t >= 1.  F is taken as given.
 * RVEA_ERR_ARG, with the run unchanged, when no member is valid (mating
 * would have nothing to draw from).  Synchronises `cuda_stream`. */
rvea_status rvea_import_state(rvea_run *run, const float *X, const float *F,
                              const uint8_t *valid, const double *V,
                              const double *gamma, int t, void *cuda_stream);

/* Swarm state of a run reproduced by CSO or PSO, in vector-slot order like
 * rvea_export_state: vel (N x d f32, the velocity of each slot's member),
 * apd (N f32, the APD of Eq. 4 with which the last selection kept the
 * member; +inf before any selection), and for PSO pbest (N x d f32, the
 * member's personal best) and fpbest (N x m f32, its objectives); NaN rows
 * and +inf for invalid slots.  Any may be NULL.  Device or pinned host memory
 * only (RVEA_ERR_ARG otherwise); RVEA_ERR_STATE for a run of another
 * operator, or for pbest / fpbest of a CSO run.  Asynchronous on
 * `cuda_stream`. */
rvea_status rvea_export_swarm(const rvea_run *run, float *vel, float *apd, float *pbest,
                              float *fpbest, void *cuda_stream);

/* Replace the swarm state of a CSO or PSO run (same layouts as
 * rvea_export_swarm; vel and apd required, pbest and fpbest required for PSO
 * and ignored for CSO; device or host memory).  Call it after
 * rvea_import_state, which starts a new swarm: velocities zero, kept APDs
 * +inf, personal bests the imported positions and objectives.  Synchronises
 * `cuda_stream`.  RVEA_ERR_STATE for a run of another operator. */
rvea_status rvea_import_swarm(rvea_run *run, const float *vel, const float *apd,
                              const float *pbest, const float *fpbest, void *cuda_stream);

/* Offspring of the last completed generation, in child order c = 0..N-1
 * (c < ceil(N/2): first child of pair c; otherwise second child of pair
 * c - ceil(N/2)): X (N x d f32), F (N x m f32).  Valid until the next step. */
rvea_status rvea_offspring(const rvea_run *run, float *X, float *F, void *cuda_stream);

/* Selection of the last completed generation over the 2N combined
 * solutions (parents i = j in slot order, then children i = N + c):
 * assoc (2N i32; reference vector of each solution, -1 for an invalid
 * parent) and survivor (N i32; combined index kept by vector j, or -1). */
rvea_status rvea_last_selection(const rvea_run *run, int32_t *assoc, int32_t *survivor,
                                void *cuda_stream);

/* Draw recording, for inspection and bit-exact testing of the random
 * decisions of Appendix B: with enable != 0 every later generation of the
 * run also writes, into its workspace, (i) the vector slot drawn for each
 * parent (the mating draws that partition X into X1 and X2; draw e < P is
 * the first parent of pair e, draw P + e its second, P = ceil(N/2)) and
 * (ii) the mutation sites of each child c = 0..N-1 (the variables where the
 * mask C of the polynomial mutation is 1).  Off by default; recording costs
 * about 4 (2P + 33 N) bytes of writes per generation.  Enqueued on
 * `cuda_stream`; applies to direct launches and graph replays alike. */
rvea_status rvea_record_draws(rvea_run *run, int enable, void *cuda_stream);

/* The draws of the last completed generation, which must have run with
 * recording on and with SBX reproduction (else RVEA_ERR_STATE).  parents: 2P int32, the vector slot
 * (0..N-1, slot order of the parent population) of each draw.  sites:
 * N x 33 int32, row c = [k, s_1..s_k, unused...]: k the number of mutation
 * sites of child c (-1 when every variable mutates: per-site probability 1)
 * and s_i the 0-based variables in draw order (distinct).  Host or device
 * pointers, either may be NULL. */
rvea_status rvea_last_draws(const rvea_run *run, int32_t *parents, int32_t *sites,
                            void *cuda_stream);

/* ---- stateless operators ---------------------------------------------- */

/* Scratch bytes rvea_select needs for n solutions, r vectors. */
size_t rvea_select_scratch_bytes(int n, int r, int m);

/* Environmental selection of Algorithm 1 on n solutions:
 * F (n x m f32, device), valid (n u8, device, NULL = all valid),
 * V (r x m f32, device, unit rows), gamma (r f32, device) -> assoc (n i32,
 * device), survivor (r i32, device: index of the solution kept by vector j
 * or -1).  t, t_max, alpha enter the APD penalty (Eq. 4).  scratch: device,
 * >= rvea_select_scratch_bytes(n, r, m), contents need no initialisation.
 * Limits: m <= 16, n < 2^31. */
rvea_status rvea_select(int m, int n, const float *F, const uint8_t *valid,
                        int r, const float *V, const float *gamma,
                        int t, int t_max, float alpha,
                        int32_t *assoc, int32_t *survivor,
                        void *scratch, size_t scratch_bytes, void *cuda_stream);

/* rvea_select for callers that cannot allocate device memory -- for example
 * an execution step of an inference-server or framework plugin whose host
 * owns every device byte and forbids allocation while work is enqueued, or a
 * process whose device memory is all reserved by another caching allocator.
 * (The paper has no counterpart: this is a deployment variant of rvea_select.)
 * Same arguments and results as rvea_select, bit for bit, without the
 * scratch argument: the scratch is a 4 MiB array inside the library.
 * Limits: n <= 65536, r <= 16384, and the shape's scratch must fit the
 * 4 MiB; larger sizes return RVEA_ERR_NOMEM before any GPU work.
 * Set-up: the array lives in its own GPU module of the library, which CUDA
 * loads on a device -- reserving the 4 MiB there until the process exits --
 * at the first call on that device (lazy module loading, CUDA's default;
 * with CUDA_MODULE_LOADING=EAGER, when the process first uses the device).
 * That first call also looks up the array's device address and sets the
 * selection kernel's shared-memory limit, with the device current: make it
 * before the caller's device memory is fully reserved and before any stream
 * capture.  After it, a call allocates no device memory and no host memory
 * (no cudaMalloc/cudaFree, no allocating library call).  Every call shares
 * the one array and clears what it reads; calls whose GPU work overlaps (e.g.
 * on unordered streams) race and corrupt each other's results. */
rvea_status rvea_select_noalloc(int m, int n, const float *F, const uint8_t *valid,
                                int r, const float *V, const float *gamma,
                                int t, int t_max, float alpha,
                                int32_t *assoc, int32_t *survivor, void *cuda_stream);

/* ---- serving loop (continuous batching) ---------------------------------
 * Not in the paper: a request loop over independent runs.  Requests (a run
 * configuration and a generation budget) queue on the host.  Each
 * rvea_server_step first enqueues one generation of every live run, packed
 * into batched launches (rvea_step_batch, 320 runs each), on the caller's
 * stream; runs whose budget is spent leave the batch.  Then, while the GPU
 * works on that step, it admits queued requests whose workspaces fit the
 * caller's device arena (the HBM budget) while fewer than max_live runs are
 * live: in arrival order, and past a head request that does not fit yet
 * (backfill, looking at up to 64 requests) unless that head has been passed
 * over for 32 steps, when admission waits for the arena to drain for it.
 * Admission initialises the run and, with autotune != 0, picks its kernel
 * variants (rvea_autotune, cached per shape), on a stream of the server's
 * own; the next step's launches wait for that work on the device.  A
 * finished run's state stays in the arena until rvea_server_fetch copies
 * the result out and frees the memory.  Every run's result is the bits it
 * gets stepped alone.  Not thread-safe. */
typedef struct rvea_server rvea_server;
typedef struct {
    int live;             /* runs in the batch after this step            */
    int queued;           /* requests waiting for admission               */
    int finished;         /* budgets spent, results not yet fetched       */
    int admitted;         /* requests admitted by this step               */
    size_t arena_used;    /* arena bytes held by live and finished runs   */
    long long generations;/* run-generations enqueued since creation      */
} rvea_server_stats;

/* dev_arena: device memory owned by the caller, 256-byte aligned, used for
 * every run's workspace; max_live >= 1. */
rvea_status rvea_server_create(void *dev_arena, size_t arena_bytes, int max_live, int autotune,
                               rvea_server **out);

/* Queue a request (DTLZ problems; cfg->neuro must be NULL); *id_out gets its
 * id (1, 2, ...).  cfg is validated here, on the host: RVEA_ERR_ARG for an
 * invalid configuration (rvea_workspace_bytes_ex returns 0, a lattice
 * mismatch included) or generations < 1, RVEA_ERR_NOMEM when its workspace
 * exceeds the whole arena; nothing is queued then. */
rvea_status rvea_server_submit(rvea_server *srv, const rvea_config *cfg, int generations,
                               int64_t *id_out);

/* One generation of every live run on `cuda_stream`, then admission (see
 * above; it synchronises the server's own stream, not cuda_stream).  stats
 * may be NULL; stats->live counts the runs after admission.  A request whose
 * admission fails (initialisation or tuning returns an error) ends there:
 * rvea_server_poll reports its id like a finished one and rvea_server_fetch
 * returns its error; the step goes on with the other requests.  The step's
 * own return value reports the batched generations and the stream wiring. */
rvea_status rvea_server_step(rvea_server *srv, void *cuda_stream, rvea_server_stats *stats);

/* Ids of runs whose budget was spent since the last poll (up to cap); their
 * results are complete once the stream of the step that finished them is. */
rvea_status rvea_server_poll(rvea_server *srv, int64_t *ids, int cap, int *n_out);

/* Copy a finished run's population (N x d) and objectives (N x m, valid
 * flags N) to X / F / valid (host or device; each may be NULL), synchronise
 * the stream and release the run.  For a request whose admission failed,
 * its error (nothing is copied).  RVEA_ERR_STATE if id is not finished or
 * already fetched. */
rvea_status rvea_server_fetch(rvea_server *srv, int64_t id, float *X, float *F, uint8_t *valid,
                              void *cuda_stream);

void rvea_server_free(rvea_server *srv);

/* gamma_j = min over i != j of the angle between v_i and v_j (Eq. 5), FP64.
 * V (r x m f64, device, unit rows) -> gamma (r f64, device). */
rvea_status rvea_gamma(int m, int r, const double *V, double *gamma, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RVEA_H */
