// sim_fused1h.cuh -- the one-column-per-thread fused pass for 2-byte field
// storage (BF16 / FP16 values, FP32 arithmetic), sm_103a.
//
// Same pipeline as k_fused1 (sim_fused.cuh): a CTA streams a column tile with a
// halo of K through z, level l is computed at plane i - l while plane i lands,
// z neighbours live in register rings, x/y neighbours come from shared memory.
// What changes with 2-byte storage:
//   * cp.async moves at least 4 bytes, so the thread of an even column stages
//     the element pair (x, x+1) of each field; with even lattice sides and even
//     tile origins a pair is either wholly inside the lattice or wholly outside,
//     and its global address is 4-byte aligned.  Cell words are staged per
//     thread as before.
//   * stage values are widened to FP32 when read; computed levels stay FP32 in
//     shared memory;
//   * every stored field value rounds stochastically with the bits of the same
//     counter-based hash (site, step, pass salt; one hash per site) as the column-pair
//     kernel, so both kernels give bit-identical results.
#pragma once
#include "sim_fused.cuh"

namespace simdev {

template <typename T>
__device__ __forceinline__ float widen(T v);
template <>
__device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float widen<__half>(__half v) { return __half2float(v); }

// stages: 3 fields of T and a cell word per site; level planes: float2 + float per thread, three slots per level
template <typename T, int TX, int TY, int K>
constexpr size_t fused1h_smem_bytes() {
    using S = FusedShape1<TX, TY, K>;
    return (size_t)kStages1 * S::NC * (3 * sizeof(T) + sizeof(uint32_t)) +
           (size_t)((K > 1) ? K - 1 : 1) * 3 * 3 * S::THREADS * sizeof(float);
}

#ifndef SIM_FUSED1H_MIN_BLOCKS_SMALL
#define SIM_FUSED1H_MIN_BLOCKS_SMALL 2  // CTAs per SM the 16 x 16 two-byte kernel is register-budgeted for
#endif

// FULL as in k_fused1: diffusion and reaction switches fixed on at compile time.
template <typename T, int TX, int TY, int K, bool EPI, bool FULL>
__global__ void __launch_bounds__(FusedShape1<TX, TY, K>::THREADS,
                                  (TX * TY <= 256) ? SIM_FUSED1H_MIN_BLOCKS_SMALL : SIM_FUSED1_MIN_BLOCKS_LARGE)
    k_fused1h(const Tile* __restrict__ tiles, const Proto* __restrict__ protos, const int64_t* __restrict__ clock,
              int k_off, int first, const T* __restrict__ iO, const T* __restrict__ iG, const T* __restrict__ iH,
              T* __restrict__ oO, T* __restrict__ oG, T* __restrict__ oH, const uint32_t* cin, uint32_t* cout,
              const int64_t* __restrict__ fstep, const double* __restrict__ fdose, double* __restrict__ cum_dose,
              uint32_t* __restrict__ intents, uint32_t* __restrict__ icount, uint32_t* __restrict__ tile_ctr,
              int n_tiles, int pass, Params P) {
    using S = FusedShape1<TX, TY, K>;
    constexpr int HX = S::HX, HY = S::HY, NC = S::NC;
    constexpr int NT = S::THREADS;  // stride of the level planes: one slot per thread, the idle tail included
    static_assert(HX % 2 == 0 && NC % 2 == 0, "element pairs must not straddle rows or planes");
    constexpr int kS1 = kStages1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* stage_t = reinterpret_cast<T*>(smem_raw);  // [stage][field][site]
    uint32_t* stage_c = reinterpret_cast<uint32_t*>(smem_raw + (size_t)kS1 * 3 * NC * sizeof(T));
    unsigned char* lv_raw = smem_raw + (size_t)kS1 * NC * (3 * sizeof(T) + sizeof(uint32_t));
    float2* lv_og = reinterpret_cast<float2*>(lv_raw);
    float* lv_h = reinterpret_cast<float*>(lv_raw + (size_t)((K > 1) ? K - 1 : 1) * 3 * NT * sizeof(float2));
    __shared__ float s_dose, s_dq;
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    const bool act = tid < NC;
    const int cx = tid % HX, cy = tid / HX;
    const bool pair_head = (cx & 1) == 0;  // this thread stages the element pair (cx, cx + 1)
    bool inreg[K + 1];
#pragma unroll
    for (int l = 1; l <= K; ++l) inreg[l] = act && cx >= l && cx < HX - l && cy >= l && cy < HY - l;
    const bool outtile = act && cx >= K && cx < K + TX && cy >= K && cy < K + TY;
    T* const my_t = stage_t + tid;             // + (s * 3 + f) * NC
    uint32_t* const my_cell = stage_c + tid;   // + s * NC
    float2* const my_lvog = lv_og + tid;       // + ((l - 1) * 3 + slot) * NT
    float* const my_lvh = lv_h + tid;
    const int me = act ? tid : 0;              // idle threads read thread 0's staged site: no guard on the loads
    const float2 lam_og = f2(P.lam[0], P.lam[1]);
    const uint32_t lane = threadIdx.x & 31u;
    const bool diffuse = FULL || (P.flags & kFDiffusion) != 0, react = FULL || (P.flags & kFReaction) != 0;
    // stochastic-rounding salt of this pass, as in the column-pair kernel
    const uint32_t salt = (EPI ? (uint32_t)P.n_sub - 1u : (uint32_t)K - 1u) + 100u;

    const int64_t step = *clock + k_off;
    uint32_t* cnt = icount + (step & 1);
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
    const int x = tl.x0 - K + cx, y = tl.y0 - K + cy;
    const bool in = act && x >= 0 && x < L && y >= 0 && y < L;
    const bool fxy = !in || x == 0 || y == 0 || x == L - 1 || y == L - 1;
    const bool outc = outtile && in;
    const int col = in ? x + L * y : 0;
    const int z0 = tl.z0, z1 = tl.z1;
    const int zl0 = max(0, z0 - K), zl1 = min(L - 1, z1 - 1 + K);
    const T* gf[3] = {iO + pr.site0 + col, iG + pr.site0 + col, iH + pr.site0 + col};
    const uint32_t* gC = cin + pr.site0 + col;
    T* const d0 = oO + pr.site0 + col;
    T* const d1 = oG + pr.site0 + col;
    T* const d2 = oH + pr.site0 + col;
    uint32_t* const dC = cout + pr.site0 + col;

    auto prefetch = [&](int j) {
        if (act && j <= zl1) {
            const int s = (j - zl0) & (kS1 - 1);
            const int o = j * LL;
            if (site_ok(P, pr.site0 + col + o)) {  // SIM_CHECK build only
                if (pair_head) {
#pragma unroll
                    for (int f = 0; f < 3; ++f) cp_async(my_t + (s * 3 + f) * NC, gf[f] + o, 4, in);
                }
                cp_async(my_cell + s * NC, gC + o, 4, in);
            }
        }
        cp_async_commit();
    };

    float2 rog[K][3];
    float rh[K][3];
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rog[l][j] = f2(0.f, 0.f);
            rh[l][j] = 0.f;
        }
    uint32_t wr[3] = {0u, 0u, 0u};
    uint32_t hit = 0;

#pragma unroll
    for (int j = 0; j < kDepth; ++j) prefetch(zl0 + j);
    __syncthreads();
    const float dose = s_dose;
    const int n_it = zl1 + K - zl0 + 1;
    const int i_lo = max(max(zl0 + 2 * K, z0 + K), K + 1);
    const int i_hi = min(min(zl1, z1 - 1 + K), L - 2);
    auto iteration = [&](auto phc, auto chkc, const int i) {
        constexpr int ph = decltype(phc)::value;
        constexpr bool CHK = decltype(chkc)::value;
        cp_async_wait<kDepth - 1>();
        __syncthreads();
        prefetch(i + kDepth);
        const bool loaded = !CHK || i <= zl1;
        const int st = (i - zl0) & (kS1 - 1);
        float2 v0og = f2(0.f, 0.f);
        float v0h = 0.f;
        uint32_t w = 0;
        if (loaded) {
            const T* sf = stage_t + me + st * 3 * NC;
            v0og = f2(widen<T>(sf[0]), widen<T>(sf[NC]));
            v0h = widen<T>(sf[2 * NC]);
            w = stage_c[me + st * NC];
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
        wr[ph] = w;
        rog[0][ph] = v0og;
        rh[0][ph] = v0h;
#pragma unroll
        for (int l = 1; l <= K; ++l) {
            const int q = i - l;
            const int sq = (ph - l + 6) % 3, sm = (ph - l - 1 + 6) % 3, sp = (ph - l + 1 + 6) % 3;
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
                    if (l == 1) {  // neighbours from the stage of plane q, widened to FP32
                        const T* so = my_t + ((q - zl0) & (kS1 - 1)) * 3 * NC;
                        const T* sg = so + NC;
                        const T* sh = so + 2 * NC;
                        vog = stencil_t2l(cog, f2(widen<T>(so[-1]), widen<T>(sg[-1])),
                                          f2(widen<T>(so[1]), widen<T>(sg[1])),
                                          f2(widen<T>(so[-HX]), widen<T>(sg[-HX])),
                                          f2(widen<T>(so[HX]), widen<T>(sg[HX])), rog[l - 1][sm],
                                          rog[l - 1][sp], lam_og);
                        vh = stencil_t(ch, widen<T>(sh[-1]), widen<T>(sh[1]), widen<T>(sh[-HX]),
                                       widen<T>(sh[HX]), rh[l - 1][sm], rh[l - 1][sp], P.lam[2]);
                    } else {  // neighbours from the shared plane of level l-1 (FP32)
                        const int pj = (l >= 2 ? l - 2 : 0) * 3 + sq;
                        const float2* pog = my_lvog + pj * NT;
                        const float* phh = my_lvh + pj * NT;
                        vog = stencil_t2l(cog, pog[-1], pog[1], pog[-HX], pog[HX], rog[l - 1][sm],
                                          rog[l - 1][sp], lam_og);
                        vh = stencil_t(ch, phh[-1], phh[1], phh[-HX], phh[HX], rh[l - 1][sm], rh[l - 1][sp],
                                       P.lam[2]);
                    }
                } else {
                    vog = cog;
                    vh = ch;
                }
                float uO = 0.f, uG = 0.f, pHv = 0.f;
                const uint32_t kq = wr[sq] & kKindMask;
                if (react && kq != kEmpty) uptake(kq, cog.x, cog.y, P, uO, uG, pHv);
                const float2 o2 = __fadd2_rn(vog, f2(-uO, -uG));
                vog = f2(fmaxf(o2.x, 0.f), fmaxf(o2.y, 0.f));
                vh = fmaxf(__fadd_rn(vh, pHv), 0.f);
            }
            if (l < K) {
                const int pj = (l - 1) * 3 + sq;  // level l, plane q: slot (q - zl0) mod 3, fixed by the unroll
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
                        const Dither3 r = dither3((uint32_t)(pr.site0 + col + o), (uint32_t)step, salt);
                        d0[o] = cvt_sr<T>(vog.x, r.o);
                        d1[o] = cvt_sr<T>(vog.y, r.g);
                        d2[o] = cvt_sr<T>(vh, r.h);
                    }
                    const uint32_t w0 = wr[sq];
                    if (EPI) dC[o] = face ? w0 : update_cell(w0, vog.x, vog.y, vh, P, want);
                    else if (dose > 0.f && (hit >> sq & 1u)) dC[o] = w0;
                }
                if (!EPI && dose > 0.f) hit &= ~(1u << sq);
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
    cp_async_wait<0>();
    __syncthreads();
    }
}

}  // namespace simdev
