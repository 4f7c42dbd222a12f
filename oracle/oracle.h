/*
 * oracle.h -- FP64 CPU oracle of the EMT6/Ro spheroid cellular automaton under
 * a radiotherapy protocol (arxiv 2303.08123, "Underlying model", "The tumour
 * case library", "GA Resolution, constraints", "Protocol Representation",
 * Eq. final_fit_fun).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * restatement of the simulation that the CUDA library is checked against.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code with the CUDA path.
 *
 * Site index s = x + L*(y + L*z).  Cell word: bits 0..2 kind (0 empty, 1 G1,
 * 2 S, 3 G2, 4 M, 5 Q), bit 3 DOOMED, bits 4..31 age in steps within the phase.
 */
#ifndef GPUGA_ORACLE_H
#define GPUGA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_DIRICHLET = 0, OR_BC_PERIODIC = 1, OR_BC_NOFLUX = 2 };
enum { OR_PURPOSE_INIT = 0, OR_PURPOSE_IRR = 1, OR_PURPOSE_DIV = 2 };

/* near-threshold flags written per site by or_step (tests count these) */
enum { OR_NEAR_IRR = 1, OR_NEAR_DEATH = 2, OR_NEAR_QUIESCENCE = 4 };

typedef struct {
    int32_t dur[4];       /* steps in G1, S, G2, M */
    int32_t n_sub;        /* diffusion substeps per CA step */
    int32_t flags;        /* model switches, see synth/params.py */
    double lam[3];        /* per-substep diffusion numbers O, G, H */
    double medium_O, medium_G, medium_pH;
    double q_O, K_O, q_G, K_G, k_an, O_an, q_H, f_Q;
    double alpha, beta, omf_m, omf_K;
    double phi[5];        /* G1, S, G2, M, Q */
    double O_q, G_q, pH_q, G_d, pH_d;
    double repair_half_h; /* sublethal-damage repair half-time (h); 0: complete repair */
    double near_tol;      /* relative tolerance that defines near-threshold */
} or_params;

typedef struct {
    int64_t n_live;
    int64_t n_deaths;       /* necrosis + mitotic catastrophe in this step */
    int64_t n_divisions;    /* daughters placed */
    int64_t n_intents;      /* cells that completed M and tried to divide */
    int64_t n_doomed_new;   /* cells newly marked DOOMED by irradiation */
    int64_t n_decisions;    /* threshold decisions taken (irradiation, death, quiescence) */
    int64_t n_near;         /* of which near-threshold */
} or_stats;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Seeded spheroid: medium fields everywhere; cells on interior sites within
 * radius R of (L/2, L/2, L/2); phase and age drawn by Philox (purpose INIT,
 * protocol word init_word).  Returns the number of cells placed. */
int64_t or_init(const or_params* P, int L, int R, int bc, const uint32_t key[2],
                uint32_t init_word, double* O, double* G, double* H, uint32_t* cell);

/* One CA step (irradiate if dose > 0, n_sub diffusion substeps, cell update,
 * division).  unrepaired: dose of earlier fractions still unrepaired at this
 * step (the H of the incomplete-repair LQ term; 0 with complete repair).
 * near (nullable) receives OR_NEAR_* bits per site.  Returns 0. */
int or_step(const or_params* P, int L, int bc, const uint32_t key[2], uint32_t protocol,
            uint32_t step, double dose, double unrepaired, double* O, double* G, double* H,
            uint32_t* cell, uint8_t* near, or_stats* st);

/* Fraction schedule: step of fraction j = round(600 * sum_{i<=j} wait_i). */
int64_t or_fraction_step(const double* wait_h, int j);

/* Whole run of one protocol from the seeded spheroid.
 * counts (nullable, hours+1 entries): live cells at every whole hour 0..hours.
 * t_end_steps > 0 fixes the horizon; otherwise last fraction + regrowth_h.
 * Final state is written to O, G, H, cell (caller-allocated, L^3 each).
 * cum_dose (nullable) receives the delivered dose in Gy.
 * Returns the number of steps taken. */
int64_t or_run(const or_params* P, int L, int R, const uint32_t key[2], uint32_t protocol,
               uint32_t init_word, int n_frac, const double* dose_gy, const double* wait_h,
               int64_t t_end_steps, int regrowth_h, int32_t* counts, int hours,
               double* O, double* G, double* H, uint32_t* cell, double* cum_dose,
               or_stats* total);

/* or_run, and near_any (L^3 entries) receives per site the OR of the
 * OR_NEAR_* bits of every step of the run: the sites where some decision of
 * the run fell inside the near-threshold band. */
int64_t or_run_near(const or_params* P, int L, int R, const uint32_t key[2], uint32_t protocol,
                    uint32_t init_word, int n_frac, const double* dose_gy, const double* wait_h,
                    int64_t t_end_steps, int regrowth_h, int32_t* counts, int hours,
                    double* O, double* G, double* H, uint32_t* cell, double* cum_dose,
                    or_stats* total, uint8_t* near_any);

/* Many protocols on n_threads host threads (one protocol per thread at a time).
 * Per protocol p: lattice L[p], radius R[p], fractions off[p]..off[p+1]-1,
 * protocol word p_word[p]; init_word 0xFFFFFFFE seeds each protocol's spheroid
 * with its own protocol word.  Outputs: final live count n_final[p], steps[p] and
 * (nullable) counts[p*(hours+1) + h].  max_steps > 0 stops every run after that
 * many steps (used to time a bounded sample).  Returns 0. */
int or_run_batch(const or_params* P, int n, const int32_t* L, const int32_t* R,
                 const uint32_t key[2], const uint32_t* p_word, uint32_t init_word,
                 const int32_t* off, const double* dose_gy, const double* wait_h,
                 int64_t t_end_steps, int regrowth_h, int64_t max_steps,
                 int64_t* n_final, int64_t* steps, int32_t* counts, int hours, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
