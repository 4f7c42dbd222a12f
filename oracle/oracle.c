/*
 * oracle.c -- FP64 CPU oracle of the EMT6/Ro spheroid cellular automaton
 * (arxiv 2303.08123).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * The paper names the model's ingredients (diffusing oxygen, glucose and
 * metabolic waste; cell-cycle phases; aerobic/anaerobic and proliferating/
 * quiescent metabolism driven by local nutrients and pH; division; radiation
 * damage; "Underlying model" section), the medium ("The tumour case library"),
 * the time step of 600 steps per hour ("GA Resolution, constraints"), the
 * protocol as (dose, wait) pairs with the first wait counted from t = 0
 * ("Defining the search problem") and the fitness 1500 - n (Eq.
 * final_fit_fun).  Everything else is the build's reading, written out step by
 * step below in the order the step is defined:
 *   1. irradiate (fraction steps only), 2. n_sub diffusion-reaction substeps,
 *   3. cell update, 4. division.
 * No blocking, fusion or reordering: every loop runs over all sites in index
 * order, every substep reads only the previous substep's arrays.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define KIND_MASK 7u
#define DOOM_BIT 8u
#define AGE_SHIFT 4
enum { EMPTY = 0, G1 = 1, S_PH = 2, G2 = 3, M_PH = 4, Q_PH = 5 };
enum {
    F_DIVISION = 1, F_DEATH = 2, F_QUIESCENCE = 4, F_REACTION = 8, F_DIFFUSION = 16,
    F_DOOM_IMMEDIATE = 32
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10, as defined by Salmon et al., SC'11: ten rounds of two */
/* 32x32->64 multiplications with the key bumped by the Weyl constants */
/* between rounds.                                                      */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24-bit uniform in [0,1): exact in binary64 and binary32 */
static double uniform24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
/* floor(u * n) for the uniform above, in exact integer arithmetic */
static uint32_t pick24(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)(x >> 8) * n) >> 24); }

static double h_of_ph(double ph) { return pow(10.0, 3.0 - ph); } /* pH -> mM of H+ */

static int is_face(int L, int x, int y, int z) {
    return x == 0 || y == 0 || z == 0 || x == L - 1 || y == L - 1 || z == L - 1;
}

static int64_t sidx(int L, int x, int y, int z) { return (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z); }

/* neighbour coordinate along one axis under the boundary mode; -1 = none */
static int nb(int L, int bc, int v) {
    if (v >= 0 && v < L) return v;
    if (bc == OR_BC_PERIODIC) return (v + L) % L;
    return -1;
}

static int near_cmp(double x, double theta, double scale, double tol) {
    return fabs(x - theta) <= tol * scale;
}

/* ------------------------------------------------------------------ */
int64_t or_init(const or_params* P, int L, int R, int bc, const uint32_t key[2], uint32_t init_word,
                double* O, double* G, double* H, uint32_t* cell) {
    const double Hm = h_of_ph(P->medium_pH);
    const int c = L / 2;
    int64_t placed = 0;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t s = sidx(L, x, y, z);
                O[s] = P->medium_O;
                G[s] = P->medium_G;
                H[s] = Hm;
                cell[s] = EMPTY;
                if (bc == OR_BC_DIRICHLET && is_face(L, x, y, z)) continue;
                int dx = x - c, dy = y - c, dz = z - c;
                if (R < 0 || dx * dx + dy * dy + dz * dz > R * R) continue;
                uint32_t ctr[4] = {(uint32_t)s, 0u, (uint32_t)OR_PURPOSE_INIT, init_word};
                uint32_t r[4];
                or_philox4x32_10(ctr, key, r);
                uint32_t kind = 1u + pick24(r[0], 4u);
                uint32_t age = pick24(r[1], (uint32_t)P->dur[kind - 1]);
                cell[s] = kind | (age << AGE_SHIFT);
                ++placed;
            }
    return placed;
}

/* ------------------------------------------------------------------ */
/* Step 1: irradiation.  Survival of a cell of phase k at oxygen O under dose D
 * is the linear-quadratic S = exp(-a D - b D^2) with a = alpha*phi_k*OMF(O) and
 * b = beta*(phi_k*OMF(O))^2, OMF(O) = (m O + K) / (m (O + K)).  With incomplete
 * repair between fractions the quadratic term also pairs D with the unrepaired
 * dose Hu of earlier fractions: -ln S = a D + b (D^2 + 2 D Hu) (Thames 1985).  A
 * cell whose Philox uniform u satisfies u >= S is lethally hit (DOOMED). */
static void irradiate(const or_params* P, int L, const uint32_t key[2], uint32_t protocol, uint32_t step,
                      double dose, double unrepaired, const double* O, uint32_t* cell, uint8_t* near,
                      or_stats* st) {
    const int64_t N = (int64_t)L * L * L;
    for (int64_t s = 0; s < N; ++s) {
        uint32_t w = cell[s];
        uint32_t kind = w & KIND_MASK;
        if (kind == EMPTY) continue;
        double omf = (P->omf_m * O[s] + P->omf_K) / (P->omf_m * (O[s] + P->omf_K));
        double mod = P->phi[kind - 1] * omf;
        double a = P->alpha * mod;
        double b = P->beta * mod * mod;
        double S = exp(-a * dose - b * (dose * dose + 2.0 * dose * unrepaired));
        uint32_t ctr[4] = {(uint32_t)s, step, (uint32_t)OR_PURPOSE_IRR, protocol};
        uint32_t r[4];
        or_philox4x32_10(ctr, key, r);
        double u = uniform24(r[0]);
        st->n_decisions++;
        if (fabs(u - S) <= P->near_tol) {
            st->n_near++;
            if (near) near[s] |= OR_NEAR_IRR;
        }
        if (u >= S) {
            if (P->flags & F_DOOM_IMMEDIATE) {
                cell[s] = EMPTY;
                st->n_deaths++;
            } else if (!(w & DOOM_BIT)) {
                cell[s] = w | DOOM_BIT;
                st->n_doomed_new++;
            }
        }
    }
}

/* Step 2: one explicit (FTCS) diffusion-reaction substep for the three fields.
 *   c' = c + lambda_c * (sum of 6 face neighbours - 6 c) - R_c,  then c' >= 0.
 * Uptake by a cell of consumption weight f (1 cycling, f_Q quiescent, 0 empty):
 *   U_O = f q_O O/(O+K_O)
 *   g   = f q_G G/(G+K_G),   w = O_an/(O+O_an)   (anaerobic weight)
 *   U_G = g (1 + (k_an-1) w)
 *   P_H = q_H g k_an w        (H+ released, enters with + sign)
 * Dirichlet faces keep their medium values. */
static void substep(const or_params* P, int L, int bc, const uint32_t* cell,
                    const double* const in[3], double* const out[3]) {
    const int diff = (P->flags & F_DIFFUSION) != 0;
    const int react = (P->flags & F_REACTION) != 0;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t s = sidx(L, x, y, z);
                if (bc == OR_BC_DIRICHLET && is_face(L, x, y, z)) {
                    for (int f = 0; f < 3; ++f) out[f][s] = in[f][s];
                    continue;
                }
                int xm = nb(L, bc, x - 1), xp = nb(L, bc, x + 1);
                int ym = nb(L, bc, y - 1), yp = nb(L, bc, y + 1);
                int zm = nb(L, bc, z - 1), zp = nb(L, bc, z + 1);
                double lap[3] = {0.0, 0.0, 0.0};
                if (diff) {
                    for (int f = 0; f < 3; ++f) {
                        const double* c = in[f];
                        double cs = c[s];
                        /* a missing neighbour (no-flux) contributes c[s] itself */
                        double sum = (xm >= 0 ? c[sidx(L, xm, y, z)] : cs) + (xp >= 0 ? c[sidx(L, xp, y, z)] : cs) +
                                     (ym >= 0 ? c[sidx(L, x, ym, z)] : cs) + (yp >= 0 ? c[sidx(L, x, yp, z)] : cs) +
                                     (zm >= 0 ? c[sidx(L, x, y, zm)] : cs) + (zp >= 0 ? c[sidx(L, x, y, zp)] : cs);
                        lap[f] = sum - 6.0 * cs;
                    }
                }
                double uO = 0.0, uG = 0.0, pH = 0.0;
                uint32_t kind = cell[s] & KIND_MASK;
                if (react && kind != EMPTY) {
                    double fw = (kind == Q_PH) ? P->f_Q : 1.0;
                    double Ov = in[0][s], Gv = in[1][s];
                    uO = fw * P->q_O * Ov / (Ov + P->K_O);
                    double g = fw * P->q_G * Gv / (Gv + P->K_G);
                    double w = P->O_an / (Ov + P->O_an);
                    uG = g * (1.0 + (P->k_an - 1.0) * w);
                    pH = P->q_H * g * P->k_an * w;
                }
                double nO = in[0][s] + P->lam[0] * lap[0] - uO;
                double nG = in[1][s] + P->lam[1] * lap[1] - uG;
                double nH = in[2][s] + P->lam[2] * lap[2] + pH;
                out[0][s] = nO > 0.0 ? nO : 0.0;
                out[1][s] = nG > 0.0 ? nG : 0.0;
                out[2][s] = nH > 0.0 ? nH : 0.0;
            }
}

/* Step 3: cell update from the step-start cell words and the post-diffusion
 * fields.  Death (necrosis) when G < G_d or H > H_d (pH below pH_d); a G1 cell
 * turns quiescent when O < O_q, G < G_q or H > H_q; a quiescent cell returns to
 * G1 (age 0) when all three are restored.  Cycling cells age by one step and
 * move to the next phase when age reaches the phase duration.  A cell that
 * completes M dies if DOOMED (death at the next mitosis after a lethal hit),
 * otherwise it stays at the end of M with capped age and wants to divide. */
static void cell_update(const or_params* P, int L, const double* O, const double* G, const double* H,
                        const uint32_t* cell, uint32_t* next, uint8_t* near, or_stats* st) {
    const int64_t N = (int64_t)L * L * L;
    const double Hm = h_of_ph(P->medium_pH);
    const double Hq = h_of_ph(P->pH_q), Hd = h_of_ph(P->pH_d);
    const double tol = P->near_tol;
    for (int64_t s = 0; s < N; ++s) {
        uint32_t w = cell[s];
        next[s] = w;
        uint32_t kind = w & KIND_MASK;
        if (kind == EMPTY) continue;
        uint32_t doomed = w & DOOM_BIT;
        uint32_t age = w >> AGE_SHIFT;
        double Ov = O[s], Gv = G[s], Hv = H[s];
        if (P->flags & F_DEATH) {
            st->n_decisions++;
            if (near_cmp(Gv, P->G_d, P->medium_G, tol) || near_cmp(Hv, Hd, Hm, tol)) {
                st->n_near++;
                if (near) near[s] |= OR_NEAR_DEATH;
            }
            if (Gv < P->G_d || Hv > Hd) {
                next[s] = EMPTY;
                st->n_deaths++;
                continue;
            }
        }
        int qnear = near_cmp(Ov, P->O_q, P->medium_O, tol) || near_cmp(Gv, P->G_q, P->medium_G, tol) ||
                    near_cmp(Hv, Hq, Hm, tol);
        if (kind == Q_PH) {
            if (P->flags & F_QUIESCENCE) {
                st->n_decisions++;
                if (qnear) {
                    st->n_near++;
                    if (near) near[s] |= OR_NEAR_QUIESCENCE;
                }
                if (Ov >= P->O_q && Gv >= P->G_q && Hv <= Hq) next[s] = (uint32_t)G1 | doomed;
            }
            continue;
        }
        if (kind == G1 && (P->flags & F_QUIESCENCE)) {
            st->n_decisions++;
            if (qnear) {
                st->n_near++;
                if (near) near[s] |= OR_NEAR_QUIESCENCE;
            }
            if (Ov < P->O_q || Gv < P->G_q || Hv > Hq) {
                next[s] = (uint32_t)Q_PH | doomed;
                continue;
            }
        }
        age += 1;
        if (age >= (uint32_t)P->dur[kind - 1]) {
            if (kind < M_PH) {
                kind += 1;
                age = 0;
            } else {
                if (doomed) {
                    next[s] = EMPTY;
                    st->n_deaths++;
                    continue;
                }
                age = (uint32_t)P->dur[M_PH - 1];
            }
        }
        next[s] = kind | doomed | (age << AGE_SHIFT);
    }
}

/* Step 4: division.  Every cell at the end of M (not DOOMED) lists its free
 * Moore-26 neighbours (empty after step 3, not a Dirichlet face) in (dz, dy,
 * dx) lexicographic order and picks the k-th, k = floor(u * n_free) with u its
 * Philox uniform (purpose DIV).  Among several claimants of one site the
 * smallest parent index wins; the winner and its daughter restart in G1 at age
 * 0.  Losers and cells without a free neighbour retry at the next step. */
static void divide(const or_params* P, int L, int bc, const uint32_t key[2], uint32_t protocol,
                   uint32_t step, uint32_t* cell, or_stats* st) {
    const int64_t N = (int64_t)L * L * L;
    const uint32_t durM = (uint32_t)P->dur[M_PH - 1];
    uint32_t* claim = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
    int64_t* target = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t s = 0; s < N; ++s) {
        claim[s] = UINT32_MAX;
        target[s] = -1;
    }
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t s = sidx(L, x, y, z);
                uint32_t w = cell[s];
                if ((w & KIND_MASK) != M_PH || (w & DOOM_BIT) || (w >> AGE_SHIFT) != durM) continue;
                st->n_intents++;
                int64_t freelist[26];
                int nf = 0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (dx == 0 && dy == 0 && dz == 0) continue;
                            int xx = nb(L, bc, x + dx), yy = nb(L, bc, y + dy), zz = nb(L, bc, z + dz);
                            if (xx < 0 || yy < 0 || zz < 0) continue;
                            if (bc == OR_BC_DIRICHLET && is_face(L, xx, yy, zz)) continue;
                            int64_t t = sidx(L, xx, yy, zz);
                            if ((cell[t] & KIND_MASK) != EMPTY) continue;
                            freelist[nf++] = t;
                        }
                if (nf == 0) continue;
                uint32_t ctr[4] = {(uint32_t)s, step, (uint32_t)OR_PURPOSE_DIV, protocol};
                uint32_t r[4];
                or_philox4x32_10(ctr, key, r);
                int64_t t = freelist[pick24(r[0], (uint32_t)nf)];
                target[s] = t;
                if ((uint32_t)s < claim[t]) claim[t] = (uint32_t)s;
            }
    for (int64_t s = 0; s < N; ++s) {
        int64_t t = target[s];
        if (t < 0 || claim[t] != (uint32_t)s) continue;
        cell[s] = G1;
        cell[t] = G1;
        st->n_divisions++;
    }
    free(claim);
    free(target);
}

int or_step(const or_params* P, int L, int bc, const uint32_t key[2], uint32_t protocol, uint32_t step,
            double dose, double unrepaired, double* O, double* G, double* H, uint32_t* cell, uint8_t* near,
            or_stats* st_out) {
    const int64_t N = (int64_t)L * L * L;
    or_stats st;
    memset(&st, 0, sizeof st);
    if (near) memset(near, 0, (size_t)N);

    if (dose > 0.0) irradiate(P, L, key, protocol, step, dose, unrepaired, O, cell, near, &st);

    double* bufA[3] = {O, G, H};
    double* tmp = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* bufB[3] = {tmp, tmp + N, tmp + 2 * N};
    for (int sub = 0; sub < P->n_sub; ++sub) {
        const double* in[3] = {bufA[0], bufA[1], bufA[2]};
        substep(P, L, bc, cell, in, bufB);
        for (int f = 0; f < 3; ++f) {
            double* t = bufA[f];
            bufA[f] = bufB[f];
            bufB[f] = t;
        }
    }
    if (bufA[0] != O) { /* odd substep count: result sits in the scratch buffer */
        memcpy(O, bufA[0], sizeof(double) * (size_t)N);
        memcpy(G, bufA[1], sizeof(double) * (size_t)N);
        memcpy(H, bufA[2], sizeof(double) * (size_t)N);
    }
    free(tmp);

    uint32_t* next = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
    cell_update(P, L, O, G, H, cell, next, near, &st);
    memcpy(cell, next, sizeof(uint32_t) * (size_t)N);
    free(next);

    if (P->flags & F_DIVISION) divide(P, L, bc, key, protocol, step, cell, &st);

    int64_t live = 0;
    for (int64_t s = 0; s < N; ++s) live += (cell[s] & KIND_MASK) != EMPTY;
    st.n_live = live;
    if (st_out) *st_out = st;
    return 0;
}

int64_t or_fraction_step(const double* wait_h, int j) {
    double t = 0.0;
    for (int i = 0; i <= j; ++i) t += wait_h[i];
    return llround(600.0 * t);
}

static void add_stats(or_stats* a, const or_stats* b) {
    a->n_deaths += b->n_deaths;
    a->n_divisions += b->n_divisions;
    a->n_intents += b->n_intents;
    a->n_doomed_new += b->n_doomed_new;
    a->n_decisions += b->n_decisions;
    a->n_near += b->n_near;
    a->n_live = b->n_live;
}

static int64_t run_impl(const or_params* P, int L, int R, const uint32_t key[2], uint32_t protocol,
                        uint32_t init_word, int n_frac, const double* dose_gy, const double* wait_h,
                        int64_t t_end_steps, int regrowth_h, int64_t max_steps, int32_t* counts, int hours,
                        double* O, double* G, double* H, uint32_t* cell, double* cum_dose, or_stats* total,
                        uint8_t* near_any) {
    const int64_t N = (int64_t)L * L * L;
    uint8_t* near = near_any ? (uint8_t*)malloc((size_t)N) : NULL;
    if (near_any) memset(near_any, 0, (size_t)N);
    int64_t* fstep = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_frac > 0 ? n_frac : 1));
    for (int j = 0; j < n_frac; ++j) fstep[j] = or_fraction_step(wait_h, j);
    int64_t T = t_end_steps > 0 ? t_end_steps : (n_frac > 0 ? fstep[n_frac - 1] : 0) + 600LL * regrowth_h;
    if (max_steps > 0 && max_steps < T) T = max_steps;
    int64_t live = or_init(P, L, R, OR_BC_DIRICHLET, key, init_word, O, G, H, cell);
    if (counts)
        for (int h = 0; h <= hours; ++h) counts[h] = -1;
    or_stats tot;
    memset(&tot, 0, sizeof tot);
    double cum = 0.0;
    for (int64_t s = 0; s < T; ++s) {
        if (counts && s % 600 == 0 && s / 600 <= hours) counts[s / 600] = (int32_t)live;
        double dose = 0.0, unrepaired = 0.0;
        for (int j = 0; j < n_frac; ++j) {
            if (fstep[j] == s) dose += dose_gy[j];
            /* earlier fractions, decayed with the repair half-time (none left if repair is complete) */
            if (fstep[j] < s && P->repair_half_h > 0.0)
                unrepaired += dose_gy[j] * pow(2.0, -(double)(s - fstep[j]) / 600.0 / P->repair_half_h);
        }
        cum += dose;
        or_stats st;
        or_step(P, L, OR_BC_DIRICHLET, key, protocol, (uint32_t)s, dose, unrepaired, O, G, H, cell, near, &st);
        if (near_any)
            for (int64_t i = 0; i < N; ++i) near_any[i] |= near[i];
        add_stats(&tot, &st);
        live = st.n_live;
    }
    if (counts && T % 600 == 0 && T / 600 <= hours) counts[T / 600] = (int32_t)live;
    tot.n_live = live;
    free(near);
    free(fstep);
    if (cum_dose) *cum_dose = cum;
    if (total) *total = tot;
    return T;
}

int64_t or_run(const or_params* P, int L, int R, const uint32_t key[2], uint32_t protocol, uint32_t init_word,
               int n_frac, const double* dose_gy, const double* wait_h, int64_t t_end_steps, int regrowth_h,
               int32_t* counts, int hours, double* O, double* G, double* H, uint32_t* cell, double* cum_dose,
               or_stats* total) {
    return run_impl(P, L, R, key, protocol, init_word, n_frac, dose_gy, wait_h, t_end_steps, regrowth_h, 0,
                    counts, hours, O, G, H, cell, cum_dose, total, NULL);
}

int64_t or_run_near(const or_params* P, int L, int R, const uint32_t key[2], uint32_t protocol,
                    uint32_t init_word, int n_frac, const double* dose_gy, const double* wait_h,
                    int64_t t_end_steps, int regrowth_h, int32_t* counts, int hours, double* O, double* G,
                    double* H, uint32_t* cell, double* cum_dose, or_stats* total, uint8_t* near_any) {
    return run_impl(P, L, R, key, protocol, init_word, n_frac, dose_gy, wait_h, t_end_steps, regrowth_h, 0,
                    counts, hours, O, G, H, cell, cum_dose, total, near_any);
}

/* ------------------------------------------------------------------ */
typedef struct {
    const or_params* P;
    int n;
    const int32_t *L, *R, *off;
    const uint32_t* key;
    const uint32_t* p_word;
    uint32_t init_word;
    const double *dose, *wait;
    int64_t t_end, max_steps;
    int regrowth_h, hours;
    int64_t *n_final, *steps;
    int32_t* counts;
    int next; /* shared work counter */
} batch_job;

static void* batch_worker(void* arg) {
    batch_job* J = (batch_job*)arg;
    for (;;) {
        int p = __atomic_fetch_add(&J->next, 1, __ATOMIC_SEQ_CST);
        if (p >= J->n) break;
        int L = J->L[p];
        int64_t N = (int64_t)L * L * L;
        double* f = (double*)malloc(sizeof(double) * 3 * (size_t)N);
        uint32_t* cell = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
        or_stats tot;
        int32_t* cnt = J->counts ? J->counts + (int64_t)p * (J->hours + 1) : NULL;
        int nf = J->off[p + 1] - J->off[p];
        /* init word 0xFFFFFFFE: every protocol grows its own spheroid (init word = its protocol word) */
        const uint32_t iw = J->init_word == 0xFFFFFFFEu ? J->p_word[p] : J->init_word;
        int64_t T = run_impl(J->P, L, J->R[p], J->key, J->p_word[p], iw, nf, J->dose + J->off[p],
                             J->wait + J->off[p], J->t_end, J->regrowth_h, J->max_steps, cnt, J->hours, f,
                             f + N, f + 2 * N, cell, NULL, &tot, NULL);
        J->n_final[p] = tot.n_live;
        J->steps[p] = T;
        free(f);
        free(cell);
    }
    return NULL;
}

int or_run_batch(const or_params* P, int n, const int32_t* L, const int32_t* R, const uint32_t key[2],
                 const uint32_t* p_word, uint32_t init_word, const int32_t* off, const double* dose_gy,
                 const double* wait_h, int64_t t_end_steps, int regrowth_h, int64_t max_steps, int64_t* n_final,
                 int64_t* steps, int32_t* counts, int hours, int n_threads) {
    batch_job J = {P, n, L, R, off, key, p_word, init_word, dose_gy, wait_h, t_end_steps, max_steps,
                   regrowth_h, hours, n_final, steps, counts, 0};
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n) n_threads = n;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, batch_worker, &J);
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    free(th);
    return 0;
}
