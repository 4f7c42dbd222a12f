// sim_tma.cuh -- TMA-staged temporally blocked reaction-diffusion pass (FP32 storage, sm_103a).
//
// The same pass as k_fused1 (K explicit substeps per pass over a column tile
// streamed through z, one lattice column per thread, register z-rings, the
// pinned arithmetic of stencil_t), with the level-0 planes staged by the
// tensor memory accelerator instead of per-thread copies:
//   * one thread issues, per plane, four 3-D tiled bulk-tensor loads (O2,
//     glucose, H+, cell word) of a (TX + 8) x (TY + 4) box into a ring of
//     shared-memory stages; each stage completes on its own mbarrier
//     (expect-tx bytes), and every thread waits on it with a bounded spin;
//   * the box starts 4 columns left of the tile (a 16-byte aligned x
//     coordinate) and HY rows above it (HY = 2 for passes of up to two
//     substeps, 4 for the deep shapes' passes of up to four); rows, columns and
//     planes outside the lattice arrive as zeros, which is what the cell-word
//     and field halo of a lattice edge needs (such sites are faces and never
//     feed an interior site);
//   * the thread grid covers only the level-1 region (the tile plus K - 1
//     columns), not the outer halo the copies used to need a thread for;
//   * on the 32 x 16 tiles, whose CTA has an SM to itself, no CTA-wide
//     barrier per plane: the level planes the threads exchange live in a ring
//     of three slots per level, every thread arrives on one mbarrier after its
//     level-plane stores of a plane iteration and, in the next iteration,
//     waits for that phase only before its own first store (and before the
//     stage refill), so warps may drift apart by most of an iteration instead
//     of meeting at the top of each one (9-10 % faster); the 16 x 16 tiles run
//     three CTAs per SM, which hide each other's barrier waits, and keep one
//     __syncthreads per plane (the mbarrier measured 11-13 % slower there);
//     both use the three-slot ring, whose slot offsets the x3 unrolled z loop
//     fixes at compile time (2 % faster than two slots indexed by plane parity).
// One tensor map per (lattice side, array, tile shape) addresses each array as
// an L x L x Z volume; every protocol's first site is a multiple of L^2, so the
// protocol's planes are whole z-slices of that volume.
// Every substep uses the pinned operation sequence, so this path gives the same
// FP32 results, bit for bit, as k_fused1 and the one-kernel-per-substep path.
#pragma once
#include <cudaTypedefs.h>

#include "sim_fused.cuh"

namespace simdev {

constexpr int kTmaArrays = 8;        // tensor maps per (side, shape): O0, G0, H0, O1, G1, H1, C0, C1
constexpr int kTmaHaloX = 4;         // box x origin: 4 columns left of the tile (x * 4 B stays 16-byte aligned)
constexpr int kTmaStages = 8;        // shared-memory stages (a power of two >= kDepth + 2)
constexpr uint32_t kStatusTmaTimeout = 8u;  // a stage's copies did not land within the bounded wait

// HY: rows of halo the staged box carries above and below the tile (the deepest pass it serves)
template <int TX, int TY, int K, int HY>
struct TmaShape {
    static constexpr bool PLANE_BAR = TX * TY > 256;  // mbarrier-paced planes (see above), else a CTA barrier
    static constexpr int SLOTS = 3;                    // level-plane slots per level: plane (q - zl0) mod 3
    static constexpr int BX = TX + 2 * kTmaHaloX;  // staged box (x extent)
    static constexpr int BY = TY + 2 * HY;         // staged box (y extent)
    static constexpr int NB = BX * BY;             // sites of one staged plane
    static constexpr int RX = TX + 2 * (K - 1);    // level-1 region = thread grid
    static constexpr int RY = TY + 2 * (K - 1);
    static constexpr int NR = RX * RY;
    static constexpr int THREADS = (NR + 31) / 32 * 32;
    static_assert((NB * 4) % 128 == 0, "every staged array must start 128-byte aligned");
    static_assert(K >= 1 && K <= HY && K <= kTmaHaloX, "a pass of K substeps needs a box halo of K sites");
};

// dynamic shared memory: stages (4 planar arrays each) + level planes (float2 O2/glucose, float H+) + alignment slack
template <int TX, int TY, int K, int HY>
constexpr size_t tma_smem_bytes() {
    using S = TmaShape<TX, TY, K, HY>;
    return 128 + (size_t)kTmaStages * 4 * S::NB * sizeof(float) +
           (size_t)((K > 1) ? K - 1 : 1) * S::SLOTS * S::THREADS * (sizeof(float2) + sizeof(float));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed; false after the spin bound (2^22 tries)
// (a loop written in PTX instead measured 1-3 % slower on every tile shape)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 3-D tiled bulk-tensor load of one box into shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

#ifndef SIM_TMA_MIN_BLOCKS_SMALL
#define SIM_TMA_MIN_BLOCKS_SMALL 3  // CTAs per SM the 16 x 16 TMA kernel is register-budgeted for
#endif
#ifndef SIM_TMA_MIN_BLOCKS_DEEP
#define SIM_TMA_MIN_BLOCKS_DEEP 1  // the same for its passes of four substeps
#endif

// FULL: diffusion and reaction both on (the model as run), so their switches
// are compile-time constants; other switch settings run the FULL = false instance.
template <int TX, int TY, int K, int HY, bool EPI, bool FULL>
__global__ void __launch_bounds__(TmaShape<TX, TY, K, HY>::THREADS,
                                  (TX * TY > 256) ? 1 : (K > 2 ? SIM_TMA_MIN_BLOCKS_DEEP : SIM_TMA_MIN_BLOCKS_SMALL))
    k_tma(const Tile* __restrict__ tiles, const Proto* __restrict__ protos, const int64_t* __restrict__ clock,
          int k_off, int first, const CUtensorMap* __restrict__ maps, int map_in, float* __restrict__ oO,
          float* __restrict__ oG, float* __restrict__ oH, int map_cin, uint32_t* cout,
          const int64_t* __restrict__ fstep, const double* __restrict__ fdose, double* __restrict__ cum_dose,
          uint32_t* __restrict__ intents, uint32_t* __restrict__ icount, uint32_t* __restrict__ tile_ctr, int n_tiles,
          int pass, Params P) {
    using S = TmaShape<TX, TY, K, HY>;
    constexpr int BX = S::BX, NB = S::NB, RX = S::RX, RY = S::RY, NR = S::NR;
    constexpr int NT = S::THREADS;  // stride of the level planes: one slot per thread, the idle tail included
    constexpr int kS = kTmaStages;
    constexpr uint32_t kStageBytes = 4u * NB * sizeof(float);
    extern __shared__ unsigned char smem_raw[];
    // the stages need 128-byte aligned starts
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float* stage = reinterpret_cast<float*>(base);  // stage s: O2 [NB], glucose [NB], H+ [NB], cell words [NB]
    float2* lv_og = reinterpret_cast<float2*>(base + (size_t)kS * kStageBytes);
    float* lv_h = reinterpret_cast<float*>(base + (size_t)kS * kStageBytes +
                                           (size_t)((K > 1) ? K - 1 : 1) * S::SLOTS * NT * sizeof(float2));
    __shared__ __align__(8) uint64_t full[kS];
    __shared__ __align__(8) uint64_t plane_bar;  // every thread arrives once per plane iteration
    __shared__ float s_dose, s_dq;
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    const bool act = tid < NR;
    const int rx = tid % RX, ry = tid / RX;
    // per-thread constants of the tile-independent geometry
    bool inreg[K + 1];
#pragma unroll
    for (int l = 1; l <= K; ++l) inreg[l] = act && rx >= l - 1 && rx < RX - (l - 1) && ry >= l - 1 && ry < RY - (l - 1);
    const bool outtile = inreg[K];
    // this thread's site in a staged plane (idle threads read thread 0's, so the loads need no guard)
    const int sb0 = (HY - (K - 1)) * BX + kTmaHaloX - (K - 1);  // the level-1 region's first site
    const int sb = act ? sb0 + ry * BX + rx : sb0;
    float2* const my_lvog = lv_og + tid;  // + ((l - 1) * 3 + slot) * NT
    float* const my_lvh = lv_h + tid;
    const float2 lam_og = f2(P.lam[0], P.lam[1]);
    const uint32_t lane = threadIdx.x & 31u;
    const bool diffuse = FULL || (P.flags & kFDiffusion) != 0, react = FULL || (P.flags & kFReaction) != 0;
    bool timed_out = false;

    if (tid == 0) {
        for (int s = 0; s < kS; ++s) mbar_init(&full[s], 1);
        if (S::PLANE_BAR) mbar_init(&plane_bar, NT);
    }
    uint32_t n_sync = 0;  // plane iterations this thread has arrived for (plane_bar phases)
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncthreads();

    const int64_t step = *clock + k_off;
    uint32_t* cnt = icount + (step & 1);
    uint32_t loaded_planes = 0;  // planes this CTA has staged so far: stage = n % kS, phase parity = (n / kS) & 1
    for (;;) {
    const int ti = next_tile(tile_ctr, step, pass, &s_tile);
    if (ti >= n_tiles) break;
    const Tile tl = tiles[ti];
    const Proto pr = protos[tl.p];
    if (step >= pr.t_end) continue;
    if (threadIdx.x == 0) {
        double q = 0.0;
        const double d = first ? dose_at(pr, fstep, fdose, step, P.frac_cap, &q) : 0.0;
        s_dose = (float)d;
        s_dq = (float)q;
        if (d > 0.0 && tl.x0 == 0 && tl.y0 == 0 && tl.z0 == 0) cum_dose[tl.p] += d;
    }
    const int L = pr.L;
    const int LL = L * L;
    const int x = tl.x0 - (K - 1) + rx, y = tl.y0 - (K - 1) + ry;
    const bool in = act && x >= 0 && x < L && y >= 0 && y < L;
    const bool fxy = !in || x == 0 || y == 0 || x == L - 1 || y == L - 1;
    const bool outc = outtile && in;
    const int col = in ? x + L * y : 0;
    const int z0 = tl.z0, z1 = tl.z1;
    const int zl0 = max(0, z0 - K), zl1 = min(L - 1, z1 - 1 + K);
    float* const d0 = oO + pr.site0 + col;  // this column's outputs: plane q at offset q * L^2
    float* const d1 = oG + pr.site0 + col;
    float* const d2 = oH + pr.site0 + col;
    uint32_t* const dC = cout + pr.site0 + col;
    // tensor maps of this protocol's lattice side; the protocol's planes start at z = site0 / L^2
    const CUtensorMap* mf = maps + (size_t)pr.tmap * kTmaArrays;
    const int zb = (int)(pr.site0 / LL);
    const int bx0 = tl.x0 - kTmaHaloX, by0 = tl.y0 - HY;
    const uint32_t g0 = loaded_planes;

    // thread 0 stages level-0 plane j (all four arrays) into its ring slot
    auto issue = [&](int j) {
        if (tid == 0 && j <= zl1) {
            const uint32_t n = g0 + (uint32_t)(j - zl0);
            uint64_t* bar = &full[n & (kS - 1)];
            float* dst = stage + (size_t)(n & (kS - 1)) * 4 * NB;
            mbar_expect_tx(bar, kStageBytes);
#pragma unroll
            for (int a = 0; a < 3; ++a) tma_load_3d(dst + a * NB, mf + map_in + a, bx0, by0, zb + j, bar);
            tma_load_3d(dst + 3 * NB, mf + map_cin, bx0, by0, zb + j, bar);
        }
    };

    float2 rog[K][3];  // z-rings per level: (O2, glucose) and H+
    float rh[K][3];
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rog[l][j] = f2(0.f, 0.f);
            rh[l][j] = 0.f;
        }
    // cell words of the planes in flight: while a pass is at most two substeps deep, planes i, i - 1 and
    // i - 2 fit one ring of three; a deeper pass hands each plane's word on from level to level
    constexpr int kWr = (K <= 2) ? 1 : K;
    uint32_t wr[kWr][3];
#pragma unroll
    for (int l = 0; l < kWr; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j) wr[l][j] = 0u;
    uint32_t hit = 0;  // planes whose word irradiation changed (passes of at most two substeps)

#pragma unroll
    for (int j = 0; j < kDepth; ++j) issue(zl0 + j);
    __syncthreads();
    const float dose = s_dose;
    const int n_it = zl1 + K - zl0 + 1;
    // planes i in [i_lo, i_hi] need none of the z-boundary checks
    const int i_lo = max(max(zl0 + 2 * K, z0 + K), K + 1);
    const int i_hi = min(min(zl1, z1 - 1 + K), L - 2);
    auto iteration = [&](auto phc, auto chkc, const int i) {
        constexpr int ph = decltype(phc)::value;
        constexpr bool CHK = decltype(chkc)::value;
        if constexpr (!S::PLANE_BAR) {
            __syncthreads();  // iteration i - 1 is done everywhere: its stage reads and level-plane writes
            issue(i + kDepth);
        }
        const bool loaded = !CHK || i <= zl1;
        const uint32_t n = g0 + (uint32_t)(i - zl0);
        const float* st = stage + (size_t)(n & (kS - 1)) * 4 * NB;
        if (loaded && !timed_out && !mbar_wait(&full[n & (kS - 1)], (n / kS) & 1u)) {
            timed_out = true;
            if (P.status) atomicOr(P.status, kStatusTmaTimeout);
        }
        float2 v0og = f2(0.f, 0.f);
        float v0h = 0.f;
        uint32_t w = 0;
        if (loaded) {
            v0og = f2(st[sb], st[NB + sb]);
            v0h = st[2 * NB + sb];
            w = __float_as_uint(st[3 * NB + sb]);
        }
        if (dose > 0.f && loaded && !fxy && (!CHK || (i > 0 && i < L - 1)) && (w & kKindMask) != kEmpty) {
            const float Sv = lq_survival(w & kKindMask, v0og.x, dose, s_dq, P);
            const int s = x + L * y + LL * i;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)step, kPurposeIrr, (uint32_t)tl.p),
                                          P.key0, P.key1);
            if (u24(r.x) >= Sv) {
                const uint32_t nw = (P.flags & kFDoomImmediate) ? kEmpty : (w | kDoomed);
                if (nw != w) hit |= 1u << ph;
                w = nw;
            }
        }
        wr[0][ph] = w;
        rog[0][ph] = v0og;
        rh[0][ph] = v0h;
#pragma unroll
        for (int l = 1; l <= K; ++l) {
            const int q = i - l;
            const int sq = (ph - l + 6) % 3, sm = (ph - l - 1 + 6) % 3, sp = (ph - l + 1 + 6) % 3;
            const uint32_t wq = wr[(K <= 2) ? 0 : l - 1][sq];  // the cell word of plane q
            if constexpr (K > 2) {
                if (l < K) wr[l][sq] = wq;
            }
            bool reg = inreg[l];
            if constexpr (CHK) {
                const int lo = (zl0 == 0) ? 0 : zl0 + l;
                const int hi = (zl1 == L - 1) ? L - 1 : zl1 - l;
                reg = reg && q >= lo && q <= hi;
            }
            // outside the level's region 0; on a face the value carried unchanged; else one substep
            const float2 cog = rog[l - 1][sq];
            const float ch = rh[l - 1][sq];
            const bool face_q = fxy || (CHK && (q == 0 || q == L - 1));
            float2 vog = reg ? cog : f2(0.f, 0.f);
            float vh = reg ? ch : 0.f;
            if (reg && !face_q) {
                if (diffuse) {
                    float2 xm, xp, ym, yp;
                    float hxm, hxp, hym, hyp;
                    if (l == 1) {  // level-0 neighbours from the staged plane q (planar arrays)
                        const float* pq = stage + (size_t)((g0 + (uint32_t)(q - zl0)) & (kS - 1)) * 4 * NB + sb;
                        xm = f2(pq[-1], pq[NB - 1]);
                        xp = f2(pq[1], pq[NB + 1]);
                        ym = f2(pq[-BX], pq[NB - BX]);
                        yp = f2(pq[BX], pq[NB + BX]);
                        hxm = pq[2 * NB - 1];
                        hxp = pq[2 * NB + 1];
                        hym = pq[2 * NB - BX];
                        hyp = pq[2 * NB + BX];
                    } else {  // level l-1 neighbours from its shared plane
                        const int pj = (l >= 2 ? l - 2 : 0) * S::SLOTS + sq;
                        const float2* pog = my_lvog + pj * NT;
                        const float* phh = my_lvh + pj * NT;
                        xm = pog[-1];
                        xp = pog[1];
                        ym = pog[-RX];
                        yp = pog[RX];
                        hxm = phh[-1];
                        hxp = phh[1];
                        hym = phh[-RX];
                        hyp = phh[RX];
                    }
                    vog = stencil_t2l(cog, xm, xp, ym, yp, rog[l - 1][sm], rog[l - 1][sp], lam_og);
                    vh = stencil_t(ch, hxm, hxp, hym, hyp, rh[l - 1][sm], rh[l - 1][sp], P.lam[2]);
                } else {
                    vog = cog;
                    vh = ch;
                }
                float uO = 0.f, uG = 0.f, pHv = 0.f;
                const uint32_t kq = wq & kKindMask;
                if (react && kq != kEmpty) uptake(kq, cog.x, cog.y, P, uO, uG, pHv);
                const float2 o2 = __fadd2_rn(vog, f2(-uO, -uG));  // v - u, lane by lane
                vog = f2(fmaxf(o2.x, 0.f), fmaxf(o2.y, 0.f));
                vh = fmaxf(__fadd_rn(vh, pHv), 0.f);
            }
            if (S::PLANE_BAR && l == 1) {
                // every thread has finished the previous iteration (its stage reads, level-plane stores and
                // reads): the level-plane slots of plane q - 3 and the stage of plane i - 4 are free again
                if (n_sync > 0 && !timed_out && !mbar_wait(&plane_bar, (n_sync - 1) & 1u)) {
                    timed_out = true;
                    if (P.status) atomicOr(P.status, kStatusTmaTimeout);
                }
                issue(i + kDepth);
            }
            if (l < K) {
                const int pj = (l - 1) * S::SLOTS + sq;  // level l, plane q: slot (q - zl0) mod 3
                rog[l][sq] = vog;
                rh[l][sq] = vh;
                my_lvog[pj * NT] = vog;  // idle threads write their own (never read) slot
                my_lvh[pj * NT] = vh;
            } else {
                bool want = false;
                const int o = q * LL;
                if (outc && (!CHK || (q >= z0 && q < z1)) && site_ok(P, pr.site0 + col + o)) {
                    const bool face = fxy || (CHK && (q == 0 || q == L - 1));
                    if (!face) {
                        d0[o] = vog.x;
                        d1[o] = vog.y;
                        d2[o] = vh;
                    }
                    const uint32_t w0 = wq;
                    // only irradiation changes words here; a deeper pass stores every word of a dose step
                    if (EPI) dC[o] = face ? w0 : update_cell(w0, vog.x, vog.y, vh, P, want);
                    else if (dose > 0.f && (K > 2 || (hit >> sq & 1u))) dC[o] = w0;
                }
                if (K <= 2 && !EPI && dose > 0.f) hit &= ~(1u << sq);
                if (EPI) {
                    const uint32_t mask = __ballot_sync(0xffffffffu, want);
                    if (mask) {
                        const uint32_t leader = __ffs(mask) - 1;
                        uint32_t slot = 0;
                        if (lane == leader) slot = atomicAdd(cnt, (uint32_t)__popc(mask));
                        slot = __shfl_sync(0xffffffffu, slot, leader);
                        const uint32_t at = slot + __popc(mask & ((1u << lane) - 1u));
                        if (want && site_ok(P, at)) intents[at] = (uint32_t)(pr.site0 + col + o);
                    }
                }
            }
            if (S::PLANE_BAR && l == (K > 1 ? K - 1 : 1)) {  // this thread's level-plane stores and stage reads
                mbar_arrive(&plane_bar);
                ++n_sync;
            }
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using Checked = std::integral_constant<bool, true>;
    using Unchecked = std::integral_constant<bool, false>;
    int ib = 0;
    for (; ib < n_it && zl0 + ib < i_lo; ib += 3) {
        iteration(I0{}, Checked{}, zl0 + ib);
        if (ib + 1 < n_it) iteration(I1{}, Checked{}, zl0 + ib + 1);
        if (ib + 2 < n_it) iteration(I2{}, Checked{}, zl0 + ib + 2);
    }
    for (; ib + 2 < n_it && zl0 + ib + 2 <= i_hi; ib += 3) {
        iteration(I0{}, Unchecked{}, zl0 + ib);
        iteration(I1{}, Unchecked{}, zl0 + ib + 1);
        iteration(I2{}, Unchecked{}, zl0 + ib + 2);
    }
    for (; ib < n_it; ib += 3) {
        iteration(I0{}, Checked{}, zl0 + ib);
        if (ib + 1 < n_it) iteration(I1{}, Checked{}, zl0 + ib + 1);
        if (ib + 2 < n_it) iteration(I2{}, Checked{}, zl0 + ib + 2);
    }
    loaded_planes = g0 + (uint32_t)(zl1 - zl0 + 1);
    }
    // every staged plane was waited for inside its tile; a CTA that gave up on a wait drains what may still
    // be in flight (bounded) before it exits
    if (timed_out && tid == 0)
        for (uint32_t n = (loaded_planes > kS ? loaded_planes - kS : 0); n < loaded_planes; ++n)
            (void)mbar_wait(&full[n & (kS - 1)], (n / kS) & 1u);
}


}  // namespace simdev
