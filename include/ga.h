/*
 * ga.h -- C ABI of the device-resident GA operators (libga): one generation of
 * the paper's genetic algorithm over a whole population of dose vectors,
 * computed on the GPU so that a GA loop never leaves the device
 * (arxiv 2303.08123, "The Genetic Algorithm (GA)", "The Main GA Loop" and the
 * GA operator details: selection, elitism, crossover, mutation, guards).
 *
 * Genotype ("Protocol Representation"): a row of n_slots bytes; byte i is the
 * dose given i * 30 min after the start, in dose units (the caller's unit, the
 * paper's resolution is 0.25 Gy), 0 for no fraction.  A population is P rows,
 * row-major, P * n_slots bytes.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 * seed, counter (draw index, generation, purpose, individual), one draw per
 * counter, uniform u = (x0 >> 8) * 2^-24 and integer pick(n) = ((x0 >> 8) * n)
 * >> 24.  Purposes 3 (parent selection), 4 (children), 5 (initial population)
 * never collide with the simulator's 0..2.
 *
 * One generation (ga_generation), given fitness f (higher is better):
 *  rank      individuals ordered by f descending, ties by lower index;
 *  elitism   rows 0 .. n_elite-1 of the next population are the n_elite best,
 *            unchanged;
 *  parents   n_parents picks: simple = the n_parents best; roulette = p_i
 *            proportional to f_i - min(0, min f) (FP64 prefix sum in index
 *            order, first index whose prefix reaches u * total); tournament =
 *            k entrants drawn without replacement (Floyd's method) from the
 *            ranking, best first, the r-th best wins with probability
 *            q (1 - q)^r (walk: advance while u >= q);
 *  children  pair m fills rows n_elite + 2m and n_elite + 2m + 1 (the second
 *            dropped past row P-1): two distinct parent-list positions, then
 *            single-point (cut in [S/4, 3S/4]), two-point (cuts in [S/4, S/2]
 *            and [S/2, 3S/4]) or uniform (one draw per slot) crossover; then per
 *            child each enabled mutation with probability p_mut, in the order
 *            swap, split, dose-time, dose-value; then the guards;
 *  guards    clip to [0, d_max]; while some fraction sits closer than min_gap
 *            slots to the previous one, move the first such dose to a random
 *            slot that keeps every gap (none free: fold it into the previous
 *            fraction, capped at d_max); then take one unit from the largest
 *            dose (earliest on ties) until the total is within total_cap.
 * The exact draw sequence of every operator is fixed by the kernels in
 * csrc/ga_kernels.cuh and restated by the CPU oracle; results are bit-exact.
 *
 * Conventions as in sim.h: the caller owns all memory; work is enqueued on the
 * given stream (asynchronous); return values are sim_status codes (0 ok, -1 bad
 * argument, -2 workspace too small, -3 CUDA error).
 */
#ifndef GPUGA_GA_H
#define GPUGA_GA_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { GA_SEL_SIMPLE = 0, GA_SEL_ROULETTE = 1, GA_SEL_TOURNAMENT = 2 };
enum { GA_X_SINGLE_POINT = 0, GA_X_TWO_POINT = 1, GA_X_UNIFORM = 2 };
enum { GA_MUT_SWAP = 1, GA_MUT_SPLIT = 2, GA_MUT_DOSE_TIME = 4, GA_MUT_DOSE_VALUE = 8 };
enum { GA_MAX_SLOTS = 1024, GA_MAX_TOURNAMENT = 64, GA_MAX_POPULATION = 1 << 16 };

typedef struct {
    int32_t n_slots;      /* S, 1 .. GA_MAX_SLOTS */
    int32_t d_max;        /* largest single fraction in dose units, 1 .. 255 */
    int32_t total_cap;    /* total dose cap in dose units, >= 0 */
    int32_t min_gap;      /* minimum slots between fractions, >= 1 */
    int32_t n_elite;      /* 0 .. P */
    int32_t n_parents;    /* 1 .. P */
    int32_t selection;    /* GA_SEL_* */
    int32_t crossover;    /* GA_X_* */
    uint32_t mutations;   /* bit set of GA_MUT_* */
    float p_mut;          /* per enabled mutation and child; compared with u in FP32 */
    int32_t tournament_k; /* entrants, 1 .. min(P, GA_MAX_TOURNAMENT) */
    float tournament_q;   /* compared with u in FP32 */
} ga_params;

/* Device scratch for populations of up to P individuals. */
int ga_workspace_size(int P, size_t* bytes);

/* d_pop (device, P * n_slots bytes) = P random protocols: 1 + pick(S / min_gap)
 * fractions, each adding 1 + pick(d_max) units at slot pick(S), then the
 * guards.  Draws: purpose 5, generation word 0, individual = row.  Async. */
int ga_random_population(const ga_params* prm, int P, uint64_t seed, uint8_t* d_pop, void* cuda_stream);

/* d_next (device, P rows) = next generation of d_pop (device, P rows) under
 * fitness d_fitness (device FP32, P entries, higher is better), as described
 * above.  d_pop and d_next must not overlap.  Optional d_order (device i32,
 * P entries, may be NULL) receives the ranking (d_order[r] = index of the
 * r-th best).  Async. */
int ga_generation(const ga_params* prm, int P, const uint8_t* d_pop, const float* d_fitness, uint64_t seed,
                  uint32_t generation, uint8_t* d_next, int32_t* d_order, void* d_workspace, size_t bytes,
                  void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
