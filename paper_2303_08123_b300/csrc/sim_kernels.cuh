// sim_kernels.cuh -- the per-step kernels of libsim (sm_103a).
//
// One CA step of every protocol in the batch (paper: 600 steps per hour):
//   k_substep  x n_sub  explicit reaction-diffusion of O2, glucose, H+; the
//                       first substep also applies the dose fraction (LQ kill)
//   k_cell              necrosis / quiescence / cell-cycle ageing, and the
//                       warp-ballot compaction of cells that want to divide
//   k_claim             each dividing cell picks a free Moore neighbour and
//                       claims it with a 64-bit atomicMax (smallest parent wins)
//   k_resolve           winners place their daughter
// Every kernel reads the step index from the device clock (+ k_off), so a whole
// simulated hour can be captured once as a CUDA graph and replayed.
#pragma once
#include "sim_device.cuh"

namespace simdev {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Seeded spheroid: medium everywhere (both field buffers), cells on interior
// sites within radius R of the centre (L/2, L/2, L/2), phase uniform over
// G1..M and age uniform in [0, duration) from Philox (purpose INIT).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_init(const Block* __restrict__ blocks, const Proto* __restrict__ protos,
                                                   T* O0, T* G0, T* H0, T* O1, T* G1, T* H1, uint32_t* cell,
                                                   unsigned long long* claim, Params P) {
    const Block b = blocks[blockIdx.x];
    const Proto pr = protos[b.p];
    const int L = pr.L, c = L / 2;
    const T o = cvt<T>(P.med[0]), gl = cvt<T>(P.med[1]), h = cvt<T>(P.med[2]);
    for (int i = threadIdx.x; i < b.n; i += blockDim.x) {
        const int64_t s = b.begin + i;
        const int64_t g = pr.site0 + s;
        const int x = (int)(s % L), y = (int)((s / L) % L), z = (int)(s / ((int64_t)L * L));
        O0[g] = o; G0[g] = gl; H0[g] = h;
        O1[g] = o; G1[g] = gl; H1[g] = h;
        claim[g] = 0ull;
        uint32_t w = kEmpty;
        const int dx = x - c, dy = y - c, dz = z - c;
        if (!is_face(L, x, y, z) && pr.R >= 0 && dx * dx + dy * dy + dz * dz <= pr.R * pr.R) {
            // init word 0xFFFFFFFE: every slot grows its own spheroid (init word = slot index)
            const uint32_t iw = P.init_word == 0xFFFFFFFEu ? (uint32_t)b.p : P.init_word;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)s, 0u, kPurposeInit, iw), P.key0, P.key1);
            const uint32_t kind = 1u + pick24(r.x, 4u);
            const uint32_t age = pick24(r.y, (uint32_t)P.dur[kind - 1]);
            w = kind | (age << kAgeShift);
        }
        cell[g] = w;
    }
}

// ---------------------------------------------------------------------------
// One explicit substep  c' = max(0, c + lam_c (sum6 - 6c) - R_c(cell, O, G, H)).
// Uptake of a cell with weight f (1 cycling, f_Q quiescent):
//   U_O = f q_O O/(O+K_O);  g = f q_G G/(G+K_G);  w = O_an/(O+O_an)
//   U_G = g (1 + (k_an-1) w);  H+ release = q_H g k_an w.
// Faces are Dirichlet (medium) and are never written.  In substep 0 the
// step's dose fraction is applied before diffusion from the step-start O2:
// survival S = exp(-a D - b D^2), a = alpha phi OMF(O), b = beta (phi OMF)^2,
// OMF(O) = (m O + K)/(m (O + K)); a cell with Philox uniform u >= S is DOOMED.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_substep(const Block* __restrict__ blocks, const Proto* __restrict__ protos,
                                                      const int64_t* __restrict__ clock, int k_off, int sub,
                                                      const T* __restrict__ iO, const T* __restrict__ iG,
                                                      const T* __restrict__ iH, T* __restrict__ oO, T* __restrict__ oG,
                                                      T* __restrict__ oH, uint32_t* __restrict__ cell,
                                                      const int64_t* __restrict__ fstep,
                                                      const double* __restrict__ fdose, double* __restrict__ cum_dose,
                                                      Params P) {
    const Block b = blocks[blockIdx.x];
    const Proto pr = protos[b.p];
    const int64_t step = *clock + k_off;
    if (step >= pr.t_end) return;
    float dose = 0.f, dq = 0.f;
    if (sub == 0) {  // the step's fraction is applied in its first substep
        __shared__ float s_dose, s_dq;
        if (threadIdx.x == 0) {
            double q;
            const double d = dose_at(pr, fstep, fdose, step, P.frac_cap, &q);
            s_dose = (float)d;
            s_dq = (float)q;
            if (d > 0.0 && b.begin == 0) cum_dose[b.p] += d;  // exactly one block per protocol has begin == 0
        }
        __syncthreads();
        dose = s_dose;
        dq = s_dq;
    }
    const int L = pr.L;
    const int64_t LL = (int64_t)L * L;
    const bool diffuse = (P.flags & kFDiffusion) != 0, react = (P.flags & kFReaction) != 0;
    for (int i = threadIdx.x; i < b.n; i += blockDim.x) {
        const int64_t s = b.begin + i;
        const int x = (int)(s % L), y = (int)((s / L) % L), z = (int)(s / LL);
        if (is_face(L, x, y, z)) continue;
        const int64_t g = pr.site0 + s;
        if (!site_ok(P, g - LL) || !site_ok(P, g + LL)) continue;  // SIM_CHECK build only
        const float O = ld(iO + g), Gv = ld(iG + g), H = ld(iH + g);
        uint32_t w = cell[g];
        const uint32_t kind = w & kKindMask;
        if (dose > 0.f && kind != kEmpty) {
            const float S = lq_survival(kind, O, dose, dq, P);
            const uint4 r = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)step, kPurposeIrr, (uint32_t)b.p),
                                          P.key0, P.key1);
            if (u24(r.x) >= S) {
                if (P.flags & kFDoomImmediate) w = kEmpty;
                else w |= kDoomed;
                cell[g] = w;
            }
        }
        float tO = O, tG = Gv, tH = H;
        if (diffuse) {
            const int64_t xm = g - 1, xp = g + 1, ym = g - L, yp = g + L, zm = g - LL, zp = g + LL;
            tO = stencil_t(O, ld(iO + xm), ld(iO + xp), ld(iO + ym), ld(iO + yp), ld(iO + zm), ld(iO + zp), P.lam[0]);
            tG = stencil_t(Gv, ld(iG + xm), ld(iG + xp), ld(iG + ym), ld(iG + yp), ld(iG + zm), ld(iG + zp),
                           P.lam[1]);
            tH = stencil_t(H, ld(iH + xm), ld(iH + xp), ld(iH + ym), ld(iH + yp), ld(iH + zm), ld(iH + zp), P.lam[2]);
        }
        float uO = 0.f, uG = 0.f, pH = 0.f;
        // uptake follows the kind after irradiation: a DOOMED cell keeps consuming,
        // an immediately killed one (variant switch) does not
        const uint32_t kr = w & kKindMask;
        if (react && kr != kEmpty) uptake(kr, O, Gv, P, uO, uG, pH);
        // stochastic-rounding bits per (site, step, substep), one hash for the three fields; unused with FP32
        const Dither3 r = sizeof(T) != 4 ? dither3((uint32_t)g, (uint32_t)step, (uint32_t)sub) : Dither3{0u, 0u, 0u};
        oO[g] = cvt_sr<T>(fmaxf(__fsub_rn(tO, uO), 0.f), r.o);
        oG[g] = cvt_sr<T>(fmaxf(__fsub_rn(tG, uG), 0.f), r.g);
        oH[g] = cvt_sr<T>(fmaxf(__fadd_rn(tH, pH), 0.f), r.h);
    }
}

// ---------------------------------------------------------------------------
// Cell update from the step-start cell word and the post-diffusion fields:
// necrosis if G < G_d or H > H_d; a G1 cell turns quiescent when O < O_q,
// G < G_q or H > H_q and a quiescent cell returns to G1 once all three are
// restored; cycling cells age and move on at the end of each phase; a cell
// completing M dies if DOOMED, else it stays at the end of M (age capped) and
// is appended to the division work list.  The append is warp-aggregated: one
// ballot, one atomicAdd per warp, each lane writes at base + rank.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cell(const Block* __restrict__ blocks, const Proto* __restrict__ protos,
                                                   const int64_t* __restrict__ clock, int k_off,
                                                   const T* __restrict__ O_, const T* __restrict__ G_,
                                                   const T* __restrict__ H_, uint32_t* __restrict__ cell,
                                                   uint32_t* __restrict__ intents, uint32_t* __restrict__ icount,
                                                   Params P) {
    const Block b = blocks[blockIdx.x];
    const Proto pr = protos[b.p];
    const int64_t step = *clock + k_off;
    if (step >= pr.t_end) return;
    uint32_t* cnt = icount + (step & 1);
    const uint32_t lane = threadIdx.x & 31u;
    for (int base = 0; base < b.n; base += blockDim.x) {  // uniform trip count per warp (ballot below)
        const int i = base + threadIdx.x;
        bool want = false;
        int64_t g = 0;
        if (i < b.n && site_ok(P, pr.site0 + b.begin + i)) {
            g = pr.site0 + b.begin + i;
            const uint32_t w = cell[g];
            if ((w & kKindMask) != kEmpty) {
                const uint32_t nw = update_cell(w, ld(O_ + g), ld(G_ + g), ld(H_ + g), P, want);
                if (nw != w) cell[g] = nw;
            }
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, want);
        if (mask) {
            const uint32_t leader = __ffs(mask) - 1;
            uint32_t slot = 0;
            if (lane == leader) slot = atomicAdd(cnt, (uint32_t)__popc(mask));
            slot = __shfl_sync(0xffffffffu, slot, leader);
            const uint32_t at = slot + __popc(mask & ((1u << lane) - 1u));
            if (want && site_ok(P, at)) intents[at] = (uint32_t)g;
        }
    }
}

// ---------------------------------------------------------------------------
// Division claim: a cell at the end of M lists its free Moore-26 neighbours
// (empty after the cell update, not a face) in (dz, dy, dx) lexicographic
// order, picks the k-th with k = floor(u n_free) from its Philox uniform
// (purpose DIV) and claims it with atomicMax on (step << 32 | ~parent): within
// one step the smallest parent index wins, and claims of earlier steps always
// lose, so the claim array never needs clearing between steps.
__global__ void __launch_bounds__(kThreads) k_claim(const Proto* __restrict__ protos, int n_protos,
                                                    const int64_t* __restrict__ clock, int k_off,
                                                    const uint32_t* __restrict__ cell,
                                                    const uint32_t* __restrict__ intents,
                                                    const uint32_t* __restrict__ icount, uint32_t* __restrict__ target,
                                                    unsigned long long* __restrict__ claim, Params P) {
    const int64_t step = *clock + k_off;
    const uint32_t n = icount[step & 1];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t g = intents[i];
        if (!site_ok(P, g)) {
            target[i] = 0xffffffffu;
            continue;
        }
        const int p = owner(protos, n_protos, g);
        const Proto pr = protos[p];
        const int L = pr.L;
        const int64_t s = g - pr.site0;
        const int x = (int)(s % L), y = (int)((s / L) % L), z = (int)(s / ((int64_t)L * L));
        if (is_face(L, x, y, z)) {  // cells never sit on faces; never read past the lattice
            target[i] = 0xffffffffu;
            continue;
        }
        uint32_t freebits = 0;  // bit j: j-th Moore neighbour in lexicographic order is free
        int j = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0 && dz == 0) continue;
                    const int xx = x + dx, yy = y + dy, zz = z + dz;
                    const int64_t t = g + dx + (int64_t)L * (dy + (int64_t)L * dz);
                    if (!is_face(L, xx, yy, zz) && site_ok(P, t) && (cell[t] & kKindMask) == kEmpty)
                        freebits |= 1u << j;
                    ++j;
                }
        const uint32_t nf = __popc(freebits);
        if (nf == 0) {
            target[i] = 0xffffffffu;
            continue;
        }
        const uint4 r = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)step, kPurposeDiv, (uint32_t)p), P.key0, P.key1);
        uint32_t k = pick24(r.x, nf);
        uint32_t bits = freebits;
        for (; k > 0; --k) bits &= bits - 1;     // drop the k lowest set bits
        const int jj = __ffs(bits) - 1;          // rank of the chosen neighbour among the 26
        const int q = (jj >= 13) ? jj + 1 : jj;  // its position in the 27-point cube (centre = 13)
        const int qz = q / 9 - 1, qy = (q / 3) % 3 - 1, qx = q % 3 - 1;
        const int64_t t = g + qx + (int64_t)L * (qy + (int64_t)L * qz);
        if (!site_ok(P, t)) {
            target[i] = 0xffffffffu;
            continue;
        }
        target[i] = (uint32_t)t;
        atomicMax(claim + t, ((unsigned long long)(uint32_t)step << 32) | (unsigned long long)(0xffffffffu - (uint32_t)s));
    }
}

// Winners (their key is the target's maximum) place the daughter; both cells
// restart in G1 at age 0.  The block-0 leader clears the work-list counter of
// the next step.
__global__ void __launch_bounds__(kThreads) k_resolve(const Proto* __restrict__ protos, int n_protos,
                                                      const int64_t* __restrict__ clock, int k_off,
                                                      uint32_t* __restrict__ cell, const uint32_t* __restrict__ intents,
                                                      uint32_t* __restrict__ icount,
                                                      const uint32_t* __restrict__ target,
                                                      const unsigned long long* __restrict__ claim,
                                                      uint32_t* __restrict__ tile_ctr, int n_pass, int slots,
                                                      Params P) {
    const int64_t step = *clock + k_off;
    const uint32_t n = icount[step & 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) icount[(step + 1) & 1] = 0;
    // tile tickets of the next step's fused passes (slots per step parity)
    if (tile_ctr && blockIdx.x == 0 && (int)threadIdx.x < n_pass)
        tile_ctr[(int)((step + 1) & 1) * slots + threadIdx.x] = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t t = target[i];
        if (t == 0xffffffffu) continue;
        const int64_t g = intents[i];
        if (!site_ok(P, g) || !site_ok(P, t)) continue;
        const int p = owner(protos, n_protos, g);
        const uint32_t s = (uint32_t)(g - protos[p].site0);
        const unsigned long long key = ((unsigned long long)(uint32_t)step << 32) | (unsigned long long)(0xffffffffu - s);
        if (claim[t] == key) {
            cell[g] = kG1;
            cell[t] = kG1;
        }
    }
}

// ---------------------------------------------------------------------------
// Live cells per protocol: warp shuffle + block reduce + one atomicAdd per block.
// hourly != 0: adds into out[p * stride + step / 600] for protocols whose
// horizon has not passed; otherwise into out[p] unconditionally.
__global__ void __launch_bounds__(kThreads) k_count(const Block* __restrict__ blocks, const Proto* __restrict__ protos,
                                                   const int64_t* __restrict__ clock, const uint32_t* __restrict__ cell,
                                                   int32_t* __restrict__ out, int stride, int hourly) {
    const Block b = blocks[blockIdx.x];
    const Proto pr = protos[b.p];
    const int64_t step = *clock;
    int64_t dst = b.p;
    if (hourly) {
        if (step > pr.t_end) return;
        dst = (int64_t)b.p * stride + step / kStepsPerHour;
    }
    int c = 0;
    for (int i = threadIdx.x; i < b.n; i += blockDim.x) c += (cell[pr.site0 + b.begin + i] & kKindMask) != kEmpty;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __shared__ int warp_sum[kThreads / 32];
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        c = (threadIdx.x < (blockDim.x >> 5)) ? warp_sum[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (threadIdx.x == 0 && c) atomicAdd(out + dst, c);
    }
}

__global__ void k_tick(int64_t* clock, int64_t by) { *clock += by; }

// ---------------------------------------------------------------------------
// Field totals per protocol (substrate mass): each work-list block reduces its
// sites in FP64 and, separately, in FP32 with Kahan compensation per thread;
// k_totals_finish then adds the blocks of each protocol in order (FP64, and
// FP32 Kahan), so the result does not depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_totals_part(const Block* __restrict__ blocks,
                                                          const Proto* __restrict__ protos, const T* __restrict__ O_,
                                                          const T* __restrict__ G_, const T* __restrict__ H_,
                                                          double* __restrict__ part64, float* __restrict__ part32) {
    const Block b = blocks[blockIdx.x];
    const Proto pr = protos[b.p];
    const T* f[3] = {O_, G_, H_};
    __shared__ double s64[3][kThreads];
    __shared__ float s32[3][kThreads];
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        float sum = 0.f, comp = 0.f;  // Kahan: sum + comp carries the low-order bits
        for (int i = threadIdx.x; i < b.n; i += blockDim.x) {
            const float v = ld(f[k] + pr.site0 + b.begin + i);
            acc += (double)v;
            const float yk = __fsub_rn(v, comp);
            const float t = __fadd_rn(sum, yk);
            comp = __fsub_rn(__fsub_rn(t, sum), yk);
            sum = t;
        }
        s64[k][threadIdx.x] = acc;
        s32[k][threadIdx.x] = sum;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int k = threadIdx.x;
        double a = 0.0;
        float sum = 0.f, comp = 0.f;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            a += s64[k][t];
            const float yk = __fsub_rn(s32[k][t], comp);
            const float tt = __fadd_rn(sum, yk);
            comp = __fsub_rn(__fsub_rn(tt, sum), yk);
            sum = tt;
        }
        part64[(size_t)blockIdx.x * 3 + k] = a;
        part32[(size_t)blockIdx.x * 3 + k] = sum;
    }
}

__global__ void k_totals_finish(const int32_t* __restrict__ first_block, int n, const double* __restrict__ part64,
                                const float* __restrict__ part32, double* __restrict__ out64,
                                float* __restrict__ out32) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * n) return;
    const int p = idx / 3, k = idx % 3;
    double a = 0.0;
    float sum = 0.f, comp = 0.f;
    for (int b = first_block[p]; b < first_block[p + 1]; ++b) {
        a += part64[(size_t)b * 3 + k];
        const float yk = __fsub_rn(part32[(size_t)b * 3 + k], comp);
        const float t = __fadd_rn(sum, yk);
        comp = __fsub_rn(__fsub_rn(t, sum), yk);
        sum = t;
    }
    out64[idx] = a;
    out32[idx] = sum;
}

// ---------------------------------------------------------------------------
// Dose vectors on the device -> fraction tables ("Protocol Representation":
// entry i of a protocol's vector is the dose i * 30 min after the start, i.e.
// at step 300 i).  One warp per protocol compacts the non-zero entries in slot
// order (ballot + popc), checks the fraction count and the dose cap, and
// fills the quadratic LQ partner of each fraction (incomplete repair with
// half-time half_h > 0, the dose itself otherwise).  A protocol that breaks a
// limit gets no fractions and raises bit kStatusBadProtocol of *status.
constexpr int kStepsPerSlot = 300;

__global__ void k_load_vectors(const uint8_t* __restrict__ units, int S, double unit_gy, int n,
                               Proto* __restrict__ protos, int64_t* __restrict__ fstep, double* __restrict__ fdose,
                               int F, int cap, double dose_cap, double half_h, int64_t t_end,
                               uint32_t* __restrict__ status) {
    const int p = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (p >= n) return;
    const uint8_t* row = units + (size_t)p * S;
    const int f0 = protos[p].frac0;
    int nf = 0, total = 0;
    for (int base = 0; base < S; base += 32) {
        const int s = base + lane;
        const int u = s < S ? row[s] : 0;
        const unsigned m = __ballot_sync(0xffffffffu, u != 0);
        const int pos = nf + __popc(m & ((1u << lane) - 1u));
        if (u && pos < F) {
            fstep[f0 + pos] = (int64_t)s * kStepsPerSlot;
            fdose[f0 + pos] = u * unit_gy;
        }
        nf += __popc(m);
        total += __reduce_add_sync(0xffffffffu, u);
    }
    const bool bad = nf > F || total * unit_gy > dose_cap + 1e-9;
    if (bad) nf = 0;
    __syncwarp();
    for (int j = lane; j < nf; j += 32) {
        double h = 0.0;
        for (int i = 0; half_h > 0.0 && i < j; ++i) {
            const double dt_h = (double)(fstep[f0 + j] - fstep[f0 + i]) / kStepsPerHour;
            h += fdose[f0 + i] * exp2(-dt_h / half_h);
        }
        fdose[cap + f0 + j] = fdose[f0 + j] + 2.0 * h;
    }
    if (lane == 0) {
        protos[p].nfrac = nf;
        protos[p].t_end = t_end;
        if (bad) atomicOr(status, kStatusBadProtocol);
    }
}

// final count and fitness n_max - n per protocol into device arrays
__global__ void k_fitness_out(const int32_t* __restrict__ count, int n, float n_max, int32_t* __restrict__ d_count,
                              float* __restrict__ d_fit) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (d_count) d_count[p] = count[p];
    if (d_fit) d_fit[p] = n_max - (float)count[p];
}

}  // namespace simdev
