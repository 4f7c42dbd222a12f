// sim_fused.cuh -- temporally blocked reaction-diffusion + cell update (sm_103a).
//
// One CTA owns a TX x TY column tile of one protocol's lattice and streams it
// through z.  A pass applies K explicit substeps at once: the CTA loads the tile
// plus a halo of K columns; plane i of level 0 is loaded while level l is
// computed at plane i - l, so each site's fields are read and written once per
// pass instead of once per substep.
//   * every thread owns two adjacent columns (a, b) and computes them together
//     with Blackwell's packed FP32 instructions (add / fma on f32x2);
//   * the z neighbours of each level live in per-thread register rings indexed
//     by (plane - first plane) mod 3, with the z loop unrolled by three so every
//     ring index is a compile-time constant;
//   * the x/y neighbours come from the current plane of each level in shared
//     memory (8-byte accesses for the pair, 4-byte for the two outer columns).
//   first pass: applies the step's dose fraction at load time (LQ kill, Philox)
//   last pass (EPI): cell update of the finished plane + division work list
// Every substep uses the pinned operation sequence of stencil_t, so this path
// and the one-kernel-per-substep path give bit-identical FP32 results.
#pragma once
#include <type_traits>

#include "sim_device.cuh"

#ifndef SIM_FUSED_MIN_BLOCKS
#define SIM_FUSED_MIN_BLOCKS 1  // CTAs per SM the register budget is sized for
#endif

namespace simdev {

// Work list entry of the fused kernels: one column tile and a z range.
struct Tile {
    int32_t p;
    int16_t x0, y0;
    int16_t z0, z1;
    int32_t pad;
};

template <int TX, int TY, int K>
struct FusedShape {
    static constexpr int HX = TX + 2 * K, HY = TY + 2 * K, NC = HX * HY, PX = HX / 2;
    static constexpr int THREADS = (PX * HY + 31) / 32 * 32;
    static_assert(HX % 2 == 0, "the halo row must hold whole column pairs");
};

// store a column pair; 2-byte types round stochastically with the bits ra, rb
template <typename T>
__device__ __forceinline__ void st_pair(T* p, float2 v, bool vec, bool sa, bool sb, uint32_t ra, uint32_t rb) {
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float2*>(p) = v;
        } else {
            T pair[2] = {cvt_sr<T>(v.x, ra), cvt_sr<T>(v.y, rb)};
            *reinterpret_cast<uint32_t*>(p) = *reinterpret_cast<uint32_t*>(pair);
        }
        return;
    }
    if (sa) p[0] = cvt_sr<T>(v.x, ra);
    if (sb) p[1] = cvt_sr<T>(v.y, rb);
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// the pinned substep sequence of stencil_t on a column pair
__device__ __forceinline__ float2 stencil_t2(float2 c, float2 xm, float2 xp, float2 ym, float2 yp, float2 zm,
                                             float2 zp, float lam) {
    const float2 s = __fadd2_rn(__fadd2_rn(__fadd2_rn(xm, xp), __fadd2_rn(ym, yp)), __fadd2_rn(zm, zp));
    const float2 lap = __ffma2_rn(f2(-6.f, -6.f), c, s);
    return __ffma2_rn(f2(lam, lam), lap, c);
}

// the same sequence on two fields of one site (O2 and glucose), each with its own lambda
__device__ __forceinline__ float2 stencil_t2l(float2 c, float2 xm, float2 xp, float2 ym, float2 yp, float2 zm,
                                              float2 zp, float2 lam) {
    const float2 s = __fadd2_rn(__fadd2_rn(__fadd2_rn(xm, xp), __fadd2_rn(ym, yp)), __fadd2_rn(zm, zp));
    const float2 lap = __ffma2_rn(f2(-6.f, -6.f), c, s);
    return __ffma2_rn(lam, lap, c);
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async), zero-filled where the source
// lies outside the lattice.  Used to keep kDepth planes in flight per CTA.
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? bytes : 0;
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ float2 lds_pair(const T* p);
template <>
__device__ __forceinline__ float2 lds_pair<float>(const float* p) { return *reinterpret_cast<const float2*>(p); }
template <>
__device__ __forceinline__ float2 lds_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
template <>
__device__ __forceinline__ float2 lds_pair<__half>(const __half* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
}
template <typename T>
__device__ __forceinline__ float lds1(const T* p) { return (float)(*p); }
template <>
__device__ __forceinline__ float lds1<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <>
__device__ __forceinline__ float lds1<__half>(const __half* p) { return __half2float(*p); }

constexpr int kDepth = 4;              // planes in flight per CTA
constexpr int kMaxPasses = 128;        // tile-ticket slots per step parity (n_sub <= 256)

// Persistent scheduling: each CTA takes tiles by atomic ticket from the slot
// of this (step parity, pass); the division-resolve kernel of a step clears
// the slots of the next one.  Tiles are sorted longest first.
__device__ __forceinline__ int next_tile(uint32_t* ctr, int64_t step, int pass, int* s_tile) {
    if (threadIdx.x == 0) *s_tile = (int)atomicAdd(ctr + (int)(step & 1) * kMaxPasses + pass, 1u);
    __syncthreads();
    const int t = *s_tile;
    __syncthreads();  // every thread has read the ticket before thread 0 draws the next one
    return t;
}
constexpr int kStages = kDepth + 2;    // a plane's stage is reused once its x/y neighbours were consumed

// dynamic shared memory of a fused pass
template <typename T, int TX, int TY, int K>
constexpr size_t fused_smem_bytes() {
    using S = FusedShape<TX, TY, K>;
    return (size_t)kStages * S::NC * (3 * sizeof(T) + sizeof(uint32_t)) +
           (size_t)((K > 1) ? K - 1 : 1) * 2 * 3 * S::NC * sizeof(float);
}

template <typename T, int TX, int TY, int K, bool EPI>
__global__ void __launch_bounds__(FusedShape<TX, TY, K>::THREADS, SIM_FUSED_MIN_BLOCKS)
    k_fused(const Tile* __restrict__ tiles, const Proto* __restrict__ protos, const int64_t* __restrict__ clock,
            int k_off, int first, int vec_ok, const T* __restrict__ iO, const T* __restrict__ iG,
            const T* __restrict__ iH, T* __restrict__ oO, T* __restrict__ oG, T* __restrict__ oH, const uint32_t* cin,
            uint32_t* cout, const int64_t* __restrict__ fstep, const double* __restrict__ fdose,
            double* __restrict__ cum_dose, uint32_t* __restrict__ intents, uint32_t* __restrict__ icount,
            uint32_t* __restrict__ tile_ctr, int n_tiles, int pass, Params P) {
    using S = FusedShape<TX, TY, K>;
    constexpr int HX = S::HX, HY = S::HY, NC = S::NC, PX = S::PX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // stage s: fields (3 x NC of T) then cell words (NC of u32) of one level-0 plane
    T* stage_f = reinterpret_cast<T*>(smem_raw);
    uint32_t* stage_c = reinterpret_cast<uint32_t*>(smem_raw + (size_t)kStages * 3 * NC * sizeof(T));
    float* slv = reinterpret_cast<float*>(smem_raw + (size_t)kStages * NC * (3 * sizeof(T) + sizeof(uint32_t)));
    __shared__ float s_dose, s_dq;  // the step's dose and its quadratic partner
    __shared__ int s_tile;

    const int64_t step = *clock + k_off;
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
        if (d > 0.0 && tl.x0 == 0 && tl.y0 == 0 && tl.z0 == 0) cum_dose[tl.p] += d;  // one tile per protocol
    }
    const int L = pr.L;
    const int LL = L * L;  // L <= 1024: a lattice holds < 2^31 sites, so 32-bit offsets suffice
    const int tid = threadIdx.x;
    const bool act = tid < PX * HY;
    const int cx = 2 * (tid % PX), cy = tid / PX;  // column a = cx, column b = cx + 1
    const int xa = tl.x0 - K + cx, y = tl.y0 - K + cy;
    const bool yin = act && y >= 0 && y < L;
    const bool ina = yin && xa >= 0 && xa < L, inb = yin && xa + 1 >= 0 && xa + 1 < L;
    // columns outside the lattice behave like faces: pinned, never fed into an interior site
    const bool ya_face = y == 0 || y == L - 1;
    const bool fa = !ina || ya_face || xa == 0 || xa == L - 1;
    const bool fb = !inb || ya_face || xa + 1 == 0 || xa + 1 == L - 1;
    const bool tyin = cy >= K && cy < K + TY;
    const bool outa = ina && tyin && cx >= K && cx < K + TX;
    const bool outb = inb && tyin && cx + 1 >= K && cx + 1 < K + TX;
    const bool vec = vec_ok && ina && inb;  // both lanes in the lattice and an even element index
    // element offset of column a; when only column b lies in the lattice the pointer sits one element before
    // it and only the second element is accessed
    const int col = (ina || inb) ? xa + L * y : 0;
    const int z0 = tl.z0, z1 = tl.z1;
    const int zl0 = max(0, z0 - K), zl1 = min(L - 1, z1 - 1 + K);
    const bool diffuse = (P.flags & kFDiffusion) != 0, react = (P.flags & kFReaction) != 0;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t* cnt = icount + (step & 1);
    const int sidx = cy * HX + cx;  // shared-memory index of column a
    const T* gO = iO + pr.site0 + col;
    const T* gG = iG + pr.site0 + col;
    const T* gH = iH + pr.site0 + col;
    const uint32_t* gC = cin + pr.site0 + col;

    // queue the copies of level-0 plane j into its stage (one commit group per plane, even when empty)
    auto prefetch = [&](int j) {
        if (act && j <= zl1 && (!ina || site_ok(P, pr.site0 + col + (int64_t)j * LL)) &&
            (!inb || site_ok(P, pr.site0 + col + (int64_t)j * LL + 1))) {  // site checks: SIM_CHECK build only
            const int s = (j - zl0) % kStages;
            const int o = j * LL;
            T* sf = stage_f + (size_t)s * 3 * NC + sidx;
            uint32_t* sc = stage_c + (size_t)s * NC + sidx;
            const T* src[3] = {gO + o, gG + o, gH + o};
            if (vec) {
#pragma unroll
                for (int f = 0; f < 3; ++f) cp_async(sf + f * NC, src[f], 2 * sizeof(T), true);
                cp_async(sc, gC + o, 8, true);
            } else if (sizeof(T) == 4) {
                const T* base = iO + pr.site0;  // a valid address for zero-filled lanes
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    cp_async(sf + f * NC, ina ? src[f] : base, 4, ina);
                    cp_async(sf + f * NC + 1, inb ? src[f] + 1 : base, 4, inb);
                }
                cp_async(sc, ina ? gC + o : cin + pr.site0, 4, ina);
                cp_async(sc + 1, inb ? gC + o + 1 : cin + pr.site0, 4, inb);
            }
        }
        cp_async_commit();
    };

    float2 ring[K][3][3];  // ring[l][f][(plane - zl0) mod 3]: level l of field f, columns (a, b)
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int j = 0; j < 3; ++j) ring[l][f][j] = f2(0.f, 0.f);
    uint2 wr[3] = {make_uint2(0, 0), make_uint2(0, 0), make_uint2(0, 0)};  // cell words (post-irradiation)
    uint32_t hit = 0;  // bit 2*slot + lane: the word was changed by irradiation

#pragma unroll
    for (int j = 0; j < kDepth; ++j) prefetch(zl0 + j);
    __syncthreads();  // s_dose
    const float dose = s_dose;

    const int n_it = zl1 + K - zl0 + 1;  // the same trip count in every thread
    // one z iteration; `phc` carries (i - zl0) mod 3 as a compile-time constant so that every register-ring
    // index below is static
    auto iteration = [&](auto phc, const int i) {
        constexpr int ph = decltype(phc)::value;
        cp_async_wait<kDepth - 1>();  // this thread's copies of plane i have landed
        __syncthreads();              // ... and everyone's; stages of planes < i - 1 are free again
        prefetch(i + kDepth);
        // ---- level 0 at plane i
        const bool loaded = i <= zl1;
        const int st = (i - zl0) % kStages;
        float2 v0[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
        uint2 w = make_uint2(0, 0);
        if (loaded && act) {
            const T* sf = stage_f + (size_t)st * 3 * NC + sidx;
#pragma unroll
            for (int f = 0; f < 3; ++f) v0[f] = lds_pair(sf + f * NC);
            w = *reinterpret_cast<const uint2*>(stage_c + (size_t)st * NC + sidx);
        }
        if (dose > 0.f && loaded && i > 0 && i < L - 1) {
#pragma unroll
            for (int ln = 0; ln < 2; ++ln) {
                uint32_t& wl = ln ? w.y : w.x;
                const bool fl = ln ? fb : fa;
                const uint32_t kind = wl & kKindMask;
                if (fl || kind == kEmpty) continue;
                const float Sv = lq_survival(kind, ln ? v0[0].y : v0[0].x, dose, s_dq, P);
                const int s = xa + ln + L * y + LL * i;
                const uint4 r = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)step, kPurposeIrr, (uint32_t)tl.p),
                                              P.key0, P.key1);
                if (u24(r.x) >= Sv) {
                    const uint32_t nw = (P.flags & kFDoomImmediate) ? kEmpty : (wl | kDoomed);
                    if (nw != wl) hit |= 1u << (2 * ph + ln);
                    wl = nw;
                }
            }
        }
        wr[ph] = w;
#pragma unroll
        for (int f = 0; f < 3; ++f) ring[0][f][ph] = v0[f];
        // ---- level l at plane q = i - l
#pragma unroll
        for (int l = 1; l <= K; ++l) {
            const int q = i - l;
            const int sq = (ph - l + 6) % 3;      // ring slot of plane q
            const int sm = (ph - l - 1 + 6) % 3;  // ring slot of plane q - 1
            const int sp = (ph - l + 1 + 6) % 3;  // ring slot of plane q + 1
            const int lo = (zl0 == 0) ? 0 : zl0 + l;
            const int hi = (zl1 == L - 1) ? L - 1 : zl1 - l;
            const bool rowreg = act && cy >= l && cy < HY - l && q >= lo && q <= hi;
            const bool ra = rowreg && cx >= l && cx < HX - l;
            const bool rb = rowreg && cx + 1 >= l && cx + 1 < HX - l;
            float2 v[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
            if (ra || rb) {
                const bool zface = q == 0 || q == L - 1;
                const bool pa = fa || zface, pb = fb || zface;  // pinned (Dirichlet) lanes
                const uint32_t ka = wr[sq].x & kKindMask, kb = wr[sq].y & kKindMask;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const float2 c = ring[l - 1][f][sq];
                    float2 t = c;
                    if (diffuse && !(pa && pb)) {
                        float2 up, dn;
                        float left, right;
                        if (l == 1) {  // level 0 neighbours from the plane's stage
                            const T* pf = stage_f + (size_t)((q - zl0) % kStages) * 3 * NC + f * NC + sidx;
                            up = lds_pair(pf - HX);
                            dn = lds_pair(pf + HX);
                            left = lds1(pf - 1);
                            right = lds1(pf + 2);
                        } else {       // level l-1 neighbours from its shared plane
                            const float* pf = slv + ((size_t)((l >= 2) ? l - 2 : 0) * 2 + (q & 1)) * 3 * NC + f * NC + sidx;
                            up = *reinterpret_cast<const float2*>(pf - HX);
                            dn = *reinterpret_cast<const float2*>(pf + HX);
                            left = pf[-1];
                            right = pf[2];
                        }
                        t = stencil_t2(c, f2(left, c.x), f2(c.y, right), up, dn, ring[l - 1][f][sm],
                                       ring[l - 1][f][sp], P.lam[f]);
                    }
                    v[f] = t;
                }
                float uOa = 0.f, uGa = 0.f, pHa = 0.f, uOb = 0.f, uGb = 0.f, pHb = 0.f;
                if (react && !pa && ka != kEmpty)
                    uptake(ka, ring[l - 1][0][sq].x, ring[l - 1][1][sq].x, P, uOa, uGa, pHa);
                if (react && !pb && kb != kEmpty)
                    uptake(kb, ring[l - 1][0][sq].y, ring[l - 1][1][sq].y, P, uOb, uGb, pHb);
                const float2 o0 = __fadd2_rn(v[0], f2(-uOa, -uOb));
                const float2 o1 = __fadd2_rn(v[1], f2(-uGa, -uGb));
                const float2 o2 = __fadd2_rn(v[2], f2(pHa, pHb));
                const float2 c0 = ring[l - 1][0][sq], c1 = ring[l - 1][1][sq], c2 = ring[l - 1][2][sq];
                v[0] = f2(pa ? c0.x : fmaxf(o0.x, 0.f), pb ? c0.y : fmaxf(o0.y, 0.f));
                v[1] = f2(pa ? c1.x : fmaxf(o1.x, 0.f), pb ? c1.y : fmaxf(o1.y, 0.f));
                v[2] = f2(pa ? c2.x : fmaxf(o2.x, 0.f), pb ? c2.y : fmaxf(o2.y, 0.f));
            }
            if (l < K) {
                // level l at plane q: ring slot sq; shared plane by parity (read at iteration i + 1)
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    ring[l][f][sq] = v[f];
                    if (act)
                        *reinterpret_cast<float2*>(slv + ((size_t)(l - 1) * 2 + (q & 1)) * 3 * NC + f * NC + sidx) =
                            v[f];
                }
            } else {
                // ---- epilogue: plane q is finished for this pass
                const bool oz = q >= z0 && q < z1;
                const bool oa = outa && oz, ob = outb && oz;
                bool wa = false, wb = false;
                const int o = q * LL;
                if ((oa || ob) && (!oa || site_ok(P, pr.site0 + col + o)) && (!ob || site_ok(P, pr.site0 + col + o + 1))) {
                    const bool zface = q == 0 || q == L - 1;
                    const bool sa = oa && !fa && !zface, sb = ob && !fb && !zface;  // interior sites written
                    const bool vw = vec && sa && sb;
                    if (sa || sb) {
                        // stochastic-rounding bits per (site, step, pass): one hash per site serves its
                        // three fields; the substep path salts with the substep, a fused pass with
                        // 100 + its last substep
                        uint32_t r[6] = {0, 0, 0, 0, 0, 0};
                        if constexpr (sizeof(T) != 4) {
                            const uint32_t ga = (uint32_t)(pr.site0 + col + o), stp = (uint32_t)step;
                            const uint32_t salt = (EPI ? (uint32_t)P.n_sub - 1u : (uint32_t)K - 1u) + 100u;
                            const Dither3 da = dither3(ga, stp, salt), db = dither3(ga + 1, stp, salt);
                            r[0] = da.o, r[1] = db.o, r[2] = da.g, r[3] = db.g, r[4] = da.h, r[5] = db.h;
                        }
                        st_pair(oO + pr.site0 + col + o, v[0], vw, sa, sb, r[0], r[1]);
                        st_pair(oG + pr.site0 + col + o, v[1], vw, sa, sb, r[2], r[3]);
                        st_pair(oH + pr.site0 + col + o, v[2], vw, sa, sb, r[4], r[5]);
                    }
                    const uint2 w0 = wr[sq];
                    uint32_t* pc = cout + pr.site0 + col + o;
                    if (EPI) {
                        const uint32_t na = sa ? update_cell(w0.x, v[0].x, v[1].x, v[2].x, P, wa) : w0.x;
                        const uint32_t nb = sb ? update_cell(w0.y, v[0].y, v[1].y, v[2].y, P, wb) : w0.y;
                        if (vec && oa && ob) *reinterpret_cast<uint2*>(pc) = make_uint2(na, nb);
                        else {
                            if (oa) pc[0] = na;
                            if (ob) pc[1] = nb;
                        }
                    } else {
                        if (oa && (hit >> (2 * sq) & 1u)) pc[0] = w0.x;
                        if (ob && (hit >> (2 * sq + 1) & 1u)) pc[1] = w0.y;
                    }
                }
                hit &= ~(3u << (2 * sq));  // the slot is reused by plane q + 3
                if (EPI) {
                    const uint32_t ma = __ballot_sync(0xffffffffu, wa), mb = __ballot_sync(0xffffffffu, wb);
                    if (ma | mb) {
                        const uint32_t leader = __ffs(ma | mb) - 1;
                        uint32_t slot = 0;
                        if (lane == leader) slot = atomicAdd(cnt, (uint32_t)(__popc(ma) + __popc(mb)));
                        slot = __shfl_sync(0xffffffffu, slot, leader);
                        const uint32_t lt = (1u << lane) - 1u;
                        const uint32_t g = (uint32_t)(pr.site0 + col + o);
                        const uint32_t ata = slot + __popc(ma & lt), atb = slot + __popc(ma) + __popc(mb & lt);
                        if (wa && site_ok(P, ata)) intents[ata] = g;
                        if (wb && site_ok(P, atb)) intents[atb] = g + 1;
                    }
                }
            }
        }
    };
    for (int ib = 0; ib < n_it; ib += 3) {
        iteration(std::integral_constant<int, 0>{}, zl0 + ib);
        if (ib + 1 < n_it) iteration(std::integral_constant<int, 1>{}, zl0 + ib + 1);
        if (ib + 2 < n_it) iteration(std::integral_constant<int, 2>{}, zl0 + ib + 2);
    }
    cp_async_wait<0>();  // no copy may still target this CTA's shared memory after the tile
    __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// One column per thread (FP32 storage only): the same pipeline as k_fused with
// twice the threads per tile, for latency-bound shapes where more resident
// warps matter more than column pairs.  O2 and glucose of a site sit side by
// side in shared memory (float2), so one 8-byte load fetches both and their
// stencils run as packed f32x2 operations; H+ stays scalar.  Same pinned
// arithmetic, so the results are bit-identical to the other paths.
template <int TX, int TY, int K>
struct FusedShape1 {
    static constexpr int HX = TX + 2 * K, HY = TY + 2 * K, NC = HX * HY;
    static constexpr int THREADS = (NC + 31) / 32 * 32;
};

constexpr int kStages1 = 8;  // stages of the one-column kernel (a power of two >= kDepth + 2)

// stages: (O2, glucose) float2, H+ float, cell word per site; level planes: float2 + float per thread, three
// slots per level (plane (q - zl0) mod 3)
template <int TX, int TY, int K>
constexpr size_t fused1_smem_bytes() {
    using S = FusedShape1<TX, TY, K>;
    return (size_t)kStages1 * S::NC * 4 * sizeof(float) +
           (size_t)((K > 1) ? K - 1 : 1) * 3 * 3 * S::THREADS * sizeof(float);
}

#ifndef SIM_FUSED1_MIN_BLOCKS_SMALL
#define SIM_FUSED1_MIN_BLOCKS_SMALL 2  // CTAs per SM the 16 x 16 column kernel is register-budgeted for
#endif
#ifndef SIM_FUSED1_MIN_BLOCKS_LARGE
#define SIM_FUSED1_MIN_BLOCKS_LARGE 1  // the same for the 32 x 16 column kernel
#endif

// FULL: diffusion and reaction both on (the model as run), so their switches
// are compile-time constants; other switch settings run the FULL = false instance.
template <int TX, int TY, int K, bool EPI, bool FULL>
__global__ void __launch_bounds__(FusedShape1<TX, TY, K>::THREADS,
                                  (TX * TY <= 256) ? SIM_FUSED1_MIN_BLOCKS_SMALL : SIM_FUSED1_MIN_BLOCKS_LARGE)
    k_fused1(const Tile* __restrict__ tiles, const Proto* __restrict__ protos, const int64_t* __restrict__ clock,
             int k_off, int first, const float* __restrict__ iO, const float* __restrict__ iG,
             const float* __restrict__ iH, float* __restrict__ oO, float* __restrict__ oG, float* __restrict__ oH,
             const uint32_t* cin, uint32_t* cout, const int64_t* __restrict__ fstep, const double* __restrict__ fdose,
             double* __restrict__ cum_dose, uint32_t* __restrict__ intents, uint32_t* __restrict__ icount,
             uint32_t* __restrict__ tile_ctr, int n_tiles, int pass, Params P) {
    using S = FusedShape1<TX, TY, K>;
    constexpr int HX = S::HX, HY = S::HY, NC = S::NC;
    constexpr int NT = S::THREADS;  // stride of the level planes: one slot per thread, the idle tail included
    constexpr int kS1 = kStages1;  // power of two: stage index = (plane - zl0) & (kS1 - 1)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* stage_og = reinterpret_cast<float2*>(smem_raw);
    float* stage_h = reinterpret_cast<float*>(smem_raw + (size_t)kS1 * NC * sizeof(float2));
    uint32_t* stage_c = reinterpret_cast<uint32_t*>(smem_raw + (size_t)kS1 * NC * 3 * sizeof(float));
    float2* lv_og = reinterpret_cast<float2*>(smem_raw + (size_t)kS1 * NC * 4 * sizeof(float));
    float* lv_h = reinterpret_cast<float*>(smem_raw + (size_t)kS1 * NC * 4 * sizeof(float) +
                                           (size_t)((K > 1) ? K - 1 : 1) * 3 * NT * sizeof(float2));
    __shared__ float s_dose, s_dq;  // the step's dose and its quadratic partner
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    const bool act = tid < NC;
    const int cx = tid % HX, cy = tid / HX;
    // per-thread constants of the tile-independent geometry
    bool inreg[K + 1];
#pragma unroll
    for (int l = 1; l <= K; ++l) inreg[l] = act && cx >= l && cx < HX - l && cy >= l && cy < HY - l;
    const bool outtile = act && cx >= K && cx < K + TX && cy >= K && cy < K + TY;
    float2* const my_og = stage_og + tid;      // + s * NC
    float* const my_h = stage_h + tid;         // + s * NC
    uint32_t* const my_cell = stage_c + tid;   // + s * NC
    float2* const my_lvog = lv_og + tid;       // + ((l - 1) * 3 + slot) * NT
    float* const my_lvh = lv_h + tid;          // + ((l - 1) * 3 + slot) * NT
    const int me = act ? tid : 0;              // idle threads read thread 0's staged site: no guard on the loads
    const float2 lam_og = f2(P.lam[0], P.lam[1]);
    const uint32_t lane = threadIdx.x & 31u;
    const bool diffuse = FULL || (P.flags & kFDiffusion) != 0, react = FULL || (P.flags & kFReaction) != 0;

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
    const float* g0 = iO + pr.site0 + col;
    const float* g1 = iG + pr.site0 + col;
    const float* g2 = iH + pr.site0 + col;
    const uint32_t* gC = cin + pr.site0 + col;
    float* const d0 = oO + pr.site0 + col;  // this column's outputs: plane q at offset q * L^2
    float* const d1 = oG + pr.site0 + col;
    float* const d2 = oH + pr.site0 + col;
    uint32_t* const dC = cout + pr.site0 + col;
    const bool fetch = act;  // every active thread copies (zero-filled outside the lattice)

    auto prefetch = [&](int j) {
        if (fetch && j <= zl1) {
            const int s = (j - zl0) & (kS1 - 1);
            const int o = j * LL;
            float2* sog = my_og + s * NC;
            if (site_ok(P, pr.site0 + col + o)) {  // SIM_CHECK build only
                cp_async(&sog->x, g0 + o, 4, in);
                cp_async(&sog->y, g1 + o, 4, in);
                cp_async(my_h + s * NC, g2 + o, 4, in);
                cp_async(my_cell + s * NC, gC + o, 4, in);
            }
        }
        cp_async_commit();
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
    uint32_t wr[3] = {0u, 0u, 0u};
    uint32_t hit = 0;

#pragma unroll
    for (int j = 0; j < kDepth; ++j) prefetch(zl0 + j);
    __syncthreads();
    const float dose = s_dose;
    const int n_it = zl1 + K - zl0 + 1;
    // Planes i in [i_lo, i_hi] need none of the z-boundary checks (loaded, in
    // the level ranges, no face plane, inside the tile's output range); the
    // iterations there run a CHK = false instance without them.
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
            v0og = stage_og[me + st * NC];
            v0h = stage_h[me + st * NC];
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
                // level l-1 plane q: the stage of plane q (l = 1) or the shared plane of level l-1
                const int pj = (l == 1) ? ((q - zl0) & (kS1 - 1)) : ((l >= 2 ? l - 2 : 0) * 3 + sq);
                const float2* pog = ((l == 1) ? my_og : my_lvog) + pj * ((l == 1) ? NC : NT);
                const float* phh = ((l == 1) ? my_h : my_lvh) + pj * ((l == 1) ? NC : NT);
                if (diffuse) {
                    vog = stencil_t2l(cog, pog[-1], pog[1], pog[-HX], pog[HX], rog[l - 1][sm], rog[l - 1][sp],
                                      lam_og);
                    vh = stencil_t(ch, phh[-1], phh[1], phh[-HX], phh[HX], rh[l - 1][sm], rh[l - 1][sp],
                                   P.lam[2]);
                } else {
                    vog = cog;
                    vh = ch;
                }
                float uO = 0.f, uG = 0.f, pHv = 0.f;
                const uint32_t kq = wr[sq] & kKindMask;
                if (react && kq != kEmpty) uptake(kq, cog.x, cog.y, P, uO, uG, pHv);
                const float2 o2 = __fadd2_rn(vog, f2(-uO, -uG));  // v - u, lane by lane
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
                        d0[o] = vog.x;
                        d1[o] = vog.y;
                        d2[o] = vh;
                    }
                    const uint32_t w0 = wr[sq];
                    if (EPI) dC[o] = face ? w0 : update_cell(w0, vog.x, vog.y, vh, P, want);
                    else if (dose > 0.f && (hit >> sq & 1u)) dC[o] = w0;  // only irradiation changes words here
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
    for (; ib + 2 < n_it && zl0 + ib + 2 <= i_hi; ib += 3) {  // every plane of the triple in [i_lo, i_hi]
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
