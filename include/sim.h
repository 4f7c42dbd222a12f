/*
 * sim.h -- C ABI of the batched EMT6/Ro spheroid simulator (libsim).
 *
 * Computes, for a batch of radiotherapy protocols, the time-stepped cellular
 * automaton of an EMT6/Ro tumour spheroid (arxiv 2303.08123, "Underlying model"):
 * reaction-diffusion of oxygen, glucose and H+ with per-cell metabolism,
 * cell-cycle progression, death, division into free neighbouring sites and the
 * irradiation kill at each dose fraction, on a cubic lattice with 600 steps per
 * simulated hour ("GA Resolution, constraints").  A protocol is a list of
 * (dose Gy, wait h) pairs whose first wait counts from t = 0 ("Defining the
 * search problem"); the output is the live-cell count over time and the
 * fitness f = n_max - n at the end of the run (Eq. final_fit_fun).
 *
 * Conventions
 *  - Every call returns sim_status; nothing is thrown across the ABI.
 *  - The caller owns every buffer.  Host pointers are borrowed for the call.
 *    The device workspace given to sim_create is borrowed for the context's
 *    lifetime; the library never allocates device memory.
 *  - Work is enqueued on the CUDA stream given to sim_create.  Calls marked
 *    "synchronises" wait for that stream and report device-side errors.
 *  - A context is not thread-safe; use one context per host thread.
 *  - Conditions found on the device are recorded in the context's status word
 *    and returned by the next synchronising call: a protocol loaded from device
 *    dose vectors that breaks a limit (SIM_EINVAL) and, in the index-checking
 *    debug build of this library (libsim_check.so, compiled with SIM_CHECK), a
 *    kernel addressing a site outside the batch (SIM_ECUDA; the access is
 *    skipped).  sim_reset and the protocol loaders clear the word.
 *  - Lattice site index s = x + L*(y + L*z); sites with a coordinate equal to
 *    0 or L-1 are faces that hold the medium values and never hold cells.
 *  - Cell word: bits 0..2 kind (0 empty, 1 G1, 2 S, 3 G2, 4 M, 5 quiescent),
 *    bit 3 DOOMED (lethally irradiated), bits 4..31 age in steps in the phase.
 */
#ifndef GPUGA_SIM_H
#define GPUGA_SIM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = -1,   /* bad argument or protocol (message in sim_last_error) */
    SIM_ENOSPC = -2,   /* workspace or host buffer too small */
    SIM_ECUDA = -3,    /* a CUDA call failed */
    SIM_ETIMEOUT = -4, /* a bounded device wait ran out */
    SIM_ESTATE = -5    /* call not valid in the context's current state */
} sim_status;

enum { SIM_FP32 = 0, SIM_BF16 = 1, SIM_FP16 = 2 };         /* field storage precision */
enum { SIM_F_DIVISION = 1, SIM_F_DEATH = 2, SIM_F_QUIESCENCE = 4, SIM_F_REACTION = 8,
       SIM_F_DIFFUSION = 16, SIM_F_DOOM_IMMEDIATE = 32 };  /* model switches */

/* Model parameters (host doubles; the library converts them to FP32). */
typedef struct {
    double dur_h[4];      /* phase durations G1, S, G2, M in hours (600 steps per hour) */
    int32_t n_sub;        /* explicit diffusion substeps per CA step */
    int32_t flags;        /* SIM_F_* */
    double lam[3];        /* per-substep diffusion numbers for O2, glucose, H+ (<= 1/6) */
    double medium_O, medium_G, medium_pH; /* medium: mM, mM, pH */
    double q_O, K_O, q_G, K_G, k_an, O_an, q_H, f_Q; /* metabolism (mM per substep) */
    double alpha, beta, omf_m, omf_K;     /* LQ survival and oxygen modification */
    double phi[5];        /* radiosensitivity factors G1, S, G2, M, quiescent */
    double O_q, G_q, pH_q, G_d, pH_d;     /* quiescence and death thresholds */
    double repair_half_h; /* sublethal-damage repair half-time in hours.  0: repair is complete
                             between fractions (each fraction an independent LQ kill).  > 0:
                             incomplete repair -- a fraction of dose D at time t is scored with
                             -ln S = a D + b D (D + 2 H), H = sum over earlier fractions of
                             D_i 2^(-(t - t_i) / repair_half_h), the interaction term of the
                             LQ model extended to incompletely repaired damage (Thames 1985) */
} sim_params;

typedef struct {
    sim_params params;
    uint64_t seed;          /* Philox key */
    int32_t precision;      /* SIM_FP32 / SIM_BF16 / SIM_FP16 field storage */
    int32_t regrowth_h;     /* horizon = last fraction + regrowth_h (paper: 5 days) */
    int64_t t_end_steps;    /* > 0: fixed horizon for every protocol instead */
    double n_max_fitness;   /* fitness = n_max - n (paper: 1500) */
    double dose_cap_gy;     /* reject protocols whose total dose exceeds this */
    int32_t hours;          /* hourly counts kept per protocol for hours 0..hours */
    int32_t max_fractions;  /* capacity of each protocol's fraction table */
    uint32_t init_word;     /* Philox protocol word of the seeded spheroid; 0xFFFFFFFE: each
                               slot seeds its own spheroid with its slot index */
    int32_t use_graphs;     /* 1: replay each simulated hour as one CUDA graph */
    int32_t path;           /* SIM_PATH_FUSED (default) or SIM_PATH_SUBSTEP */
    int32_t tile_shape;     /* fused tile: 0 auto; 1 = 32 x 16, 2 = 16 x 16 with two columns per
                               thread (packed FP32); 3 = 32 x 16, 4 = 16 x 16 with one column per
                               thread; 5 = 32 x 16, 6 = 16 x 16 with one column per thread and the
                               planes staged by TMA (FP32 storage, every lattice side a multiple of
                               4); 7 = 32 x 16, 8 = 16 x 16 as 5 and 6 with passes of four
                               substeps instead of two (n_sub even; the last pass two deep when
                               n_sub is not a multiple of 4).  For a given storage precision every
                               shape gives the same results bit for bit */
    int32_t z_chunk;        /* fused z range per CTA: 0 auto, else planes per CTA */
} sim_config;

/* Kernel paths (same results, bit for bit, with FP32 storage):
 *  SIM_PATH_FUSED    temporally blocked passes of two substeps each, the last one
 *                    fused with the cell update (each site read and written once
 *                    per pass);
 *  SIM_PATH_SUBSTEP  one kernel per substep plus a separate cell-update kernel.
 * With BF16/FP16 storage the fused path needs even lattice sides and an even
 * n_sub; other contexts run the substep path. */
enum { SIM_PATH_FUSED = 0, SIM_PATH_SUBSTEP = 1 };

typedef struct sim_ctx sim_ctx;

/*
 * Device workspace needed for n protocols on lattices L[0..n-1] (each 8..1024).
 * Fields and cell words are stored double-buffered (fields in the configured
 * precision); per site the workspace holds 2 x 3 field values, 2 x 4-byte cell
 * words, an 8-byte division claim and 8 bytes of division work list.  Errors: SIM_EINVAL on NULL or
 * out-of-range arguments.
 */
sim_status sim_workspace_size(const sim_config* cfg, int n, const int32_t* L, size_t* bytes);

/*
 * Create a context over a caller-allocated device workspace (at least
 * sim_workspace_size bytes, 256-byte aligned) and a CUDA stream (NULL = the
 * legacy default stream).  L and R (host, n entries) give each protocol's
 * lattice size and initial spheroid radius (R < 0: empty lattice).  Seeds every
 * spheroid (asynchronously).  *out receives the context.
 * Errors: SIM_EINVAL, SIM_ENOSPC (workspace too small), SIM_ECUDA.
 */
sim_status sim_create(const sim_config* cfg, int n, const int32_t* L, const int32_t* R, void* d_workspace,
                      size_t bytes, void* cuda_stream, sim_ctx** out);

/*
 * Load one protocol per slot (host CSR: offsets[n+1], dose_gy[], wait_h[]) and
 * reset every slot to its seeded spheroid at step 0.  n must equal the
 * context's protocol count.  Fraction j of a protocol fires at step
 * round(600 * sum_{i<=j} wait_i); doses landing on one step add up.
 * Rejected (SIM_EINVAL): negative dose or wait, a wait not on the 30 min grid,
 * total dose above dose_cap_gy, more than max_fractions fractions.
 */
sim_status sim_load_protocols(sim_ctx* ctx, int n, const int32_t* offsets, const double* dose_gy,
                              const double* wait_h);

/*
 * Load one protocol per slot from dose vectors already on the device ("Protocol
 * Representation"): d_units (device, n x n_slots bytes, row p = slot p) holds
 * in entry i the dose given i * 30 min after the start (step 300 i), in units
 * of unit_gy; 0 = no fraction.  Resets every slot to its seeded spheroid at
 * step 0 like sim_load_protocols.  Needs a fixed horizon (t_end_steps > 0):
 * the host never learns the protocols.  A row with more than max_fractions
 * fractions or a total above dose_cap_gy runs without fractions and the next
 * synchronising call returns SIM_EINVAL.  With repair_half_h > 0 the
 * quadratic partners of the fractions are computed on the device.
 * Asynchronous (the caller keeps d_units unchanged until the stream passes
 * this call).  Errors: SIM_EINVAL (arguments), SIM_ESTATE (no fixed horizon).
 */
sim_status sim_load_dose_vectors(sim_ctx* ctx, const uint8_t* d_units, int n_slots, double unit_gy);

/* Final live count (device i32, n entries, may be NULL) and fitness
 * n_max - n (device FP32, n entries, may be NULL) of every protocol, written
 * on the stream without synchronising (the device-resident GA reads them). */
sim_status sim_fitness_device(sim_ctx* ctx, int32_t* d_count, float* d_fitness);

/* Re-seed every spheroid and set the clock to step 0 (asynchronous). */
sim_status sim_reset(sim_ctx* ctx);

/*
 * Advance every protocol by up to max_steps steps (max_steps <= 0: until every
 * protocol reaches its horizon).  A protocol past its horizon stays frozen.
 * Asynchronous; device errors surface at the next synchronising call.
 */
sim_status sim_run(sim_ctx* ctx, int64_t max_steps);

/* Final live count n and fitness n_max - n per protocol (host outputs, n
 * entries each; either may be NULL).  Synchronises. */
sim_status sim_fitness(sim_ctx* ctx, int32_t* out_count, double* out_fitness);

/* Hourly live counts (host, n x (hours+1), row-major; -1 where the hour lies
 * beyond the protocol's horizon or has not been reached).  Synchronises. */
sim_status sim_counts(sim_ctx* ctx, int32_t* out, int hours);

/* Total substrate per protocol and field (sum over all L^3 sites of O2,
 * glucose and H+ in mM, row-major n x 3): out64 summed in FP64 on the device,
 * out32 in FP32 with Kahan compensation; either may be NULL.  Deterministic
 * (blocks are added in a fixed order).  Synchronises. */
sim_status sim_field_totals(sim_ctx* ctx, double* out64, float* out32);

/* Delivered dose per protocol in Gy (host, n entries, FP64).  Synchronises. */
sim_status sim_delivered_dose(sim_ctx* ctx, double* out);

/* Current step and horizon of every protocol (host, n entries; either may be
 * NULL). */
sim_status sim_clock(sim_ctx* ctx, int64_t* step, int64_t* t_end);

/* Set the step counter of every protocol (parity tests start a step at a
 * chosen Philox step index). */
sim_status sim_set_clock(sim_ctx* ctx, int64_t step);

/* Copy protocol p's lattice to / from host arrays (FP32 fields in mM, L^3
 * each, converted from / to the storage precision; cell words).  Any pointer
 * may be NULL to skip that array.  Synchronises. */
sim_status sim_get_state(sim_ctx* ctx, int p, float* O, float* G, float* H, uint32_t* cell);
sim_status sim_set_state(sim_ctx* ctx, int p, const float* O, const float* G, const float* H,
                         const uint32_t* cell);

/* Copy protocol slot ps of context src (fields and cell words) into slot pd
 * of context dst on the device.  Both slots must have the same lattice side
 * and both contexts the same storage precision; src must not be running work
 * that changes that slot (the copy is ordered on dst's stream only).  Used to
 * start many evaluations from one grown tumour (a tumour case library). */
sim_status sim_copy_lattice(sim_ctx* dst, int pd, const sim_ctx* src, int ps);

/* Checkpoint the whole batch (fields, cells, clock, delivered dose, counts)
 * into a host buffer; with buf == NULL only *bytes is set to the size needed.
 * Philox is counter-based, so a restored run continues bit for bit.
 * Synchronises.  SIM_ENOSPC if the buffer is too small. */
sim_status sim_save_state(sim_ctx* ctx, void* buf, size_t* bytes);
sim_status sim_load_state(sim_ctx* ctx, const void* buf, size_t bytes);

/*
 * Advance every protocol by n_steps steps with plain launches (no graph) and
 * time each kernel class with CUDA events on the context's stream.  ms (4
 * entries) receives the summed device time in milliseconds of: [0] the
 * reaction-diffusion work before the cell update (fused path: every pass but
 * the last; substep path: the n_sub substep kernels), [1] the cell update
 * (fused path: the last pass, which also runs its substeps; substep path: the
 * cell-update kernel), [2] the division claims, [3] the division resolution;
 * launches (4 entries, may be NULL) the number of kernel launches of each
 * class.  Same results as sim_run.  Synchronises.
 */
sim_status sim_profile_steps(sim_ctx* ctx, int n_steps, double* ms, int64_t* launches);

/*
 * Allocation-free reaction-diffusion step for one FP32 lattice (no
 * counterpart in the paper; this is a service for callers that cannot
 * allocate device memory).  Some hosts hand every byte of device memory to
 * their own pool allocator and forbid stray cudaMalloc calls, and some
 * latency-bound loops cannot afford the device-wide synchronisation a
 * cudaMalloc/cudaFree may cause; such callers cannot provide the workspace
 * sim_create needs.  This entry point needs none: it runs the n_sub
 * substeps of one CA step (with the dose fraction of that step applied to
 * the cell words first, exactly as sim_run does for protocol slot 0) on the
 * caller's device arrays O, G, H (mM, L^3 floats each) and cell (L^3 words),
 * in place, on `cuda_stream` (NULL = legacy default stream).  The ping-pong
 * field buffer and the small launch tables live in one fixed device array
 * inside the library, 3 MiB + 64 KiB, that every GPU which loads the library
 * keeps until the process exits.
 *  - Sizes: 8 <= L <= 64.  A larger lattice is rejected with SIM_ENOSPC
 *    before any work is enqueued; cfg->precision must be SIM_FP32.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current, and looks it up again
 *    when the device's context has changed (after a cudaDeviceReset).
 *  - The small launch tables are copied from host memory that lives only
 *    during the call, so a call on a stream that is being captured is
 *    refused with SIM_EINVAL before any work is enqueued.
 *  - All calls share the one array and each call overwrites it (it keeps the
 *    last call's contents): calls that overlap on the GPU, e.g. on two
 *    streams, race and corrupt each other's results.  Serialise them.
 *  - No device memory is allocated or freed; the call is asynchronous.
 * Errors: SIM_EINVAL (NULL pointer, bad config, negative dose or step, a
 * stream under capture), SIM_ENOSPC (L > 64), SIM_ECUDA (a failed copy or
 * launch of this call; errors pending from earlier work are left untouched).
 */
sim_status sim_diffuse_noalloc(const sim_config* cfg, int L, int64_t step, double dose_gy, float* O, float* G,
                               float* H, uint32_t* cell, void* cuda_stream);

/*
 * Autotuner of the fused path: time n_steps plain steps of this context's own
 * batch with every applicable tile shape (sim_config.tile_shape 1..8) -- on a
 * batch with too few column tiles to fill the GPU (split in z unless
 * sim_config.z_chunk fixes the split) each shape also with a finer z split of
 * 2 planes per CTA -- keep the fastest, then re-seed every spheroid and set the
 * clock to 0 (call it right after sim_load_protocols).  *best (may be NULL)
 * receives the chosen shape (0 on the substep path); ms (8 entries, may be
 * NULL) the device milliseconds per step of each shape (its faster split), -1
 * where a shape does not apply.  Synchronises.
 */
sim_status sim_autotune(sim_ctx* ctx, int n_steps, int* best, double* ms);

/* Message of the last failed call on this context ("" if none). */
const char* sim_last_error(const sim_ctx* ctx);
const char* sim_status_string(sim_status s);

/* Release the context (the workspace stays the caller's).  NULL is a no-op. */
void sim_destroy(sim_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
