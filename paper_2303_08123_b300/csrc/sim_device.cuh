// sim_device.cuh -- device-side types and helpers of libsim (sm_103a).
//
// Lattice state lives in HBM as structure-of-arrays over the whole batch: one
// array per field (O2, glucose, H+), double-buffered, plus one 32-bit cell
// word, one 64-bit division claim and the division work list.  Protocol p owns
// sites [site0[p], site0[p] + L_p^3) of every array, index x + L (y + L z).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace simdev {

// Cell word: bits 0..2 kind, bit 3 DOOMED, bits 4.. age (steps in the phase).
constexpr uint32_t kEmpty = 0, kG1 = 1, kS = 2, kG2 = 3, kM = 4, kQ = 5;
constexpr uint32_t kKindMask = 7u, kDoomed = 8u;
constexpr int kAgeShift = 4;
// Philox counter word 2 ("purpose") separates the streams of one site and step.
constexpr uint32_t kPurposeInit = 0, kPurposeIrr = 1, kPurposeDiv = 2;
// model switches
constexpr int kFDivision = 1, kFDeath = 2, kFQuiescence = 4, kFReaction = 8, kFDiffusion = 16,
              kFDoomImmediate = 32;

constexpr int kStepsPerHour = 600;  // paper: 600 CA steps per simulated hour

// FP32 model parameters as the kernels use them (pH thresholds already turned
// into H+ concentrations in mM so no kernel takes a logarithm).
struct Params {
    int dur[4];
    int n_sub;
    int flags;
    float lam[3];
    float med[3];  // medium O2, glucose, H+ (mM)
    float q_O, K_O, q_G, K_G, k_an, O_an, q_H, f_Q;
    float alpha, beta, omf_m, omf_K;
    float phi[5];
    float O_q, G_q, H_q, G_d, H_d;
    uint32_t key0, key1, init_word;
    int frac_cap;  // fraction-table entries per array: doses at [0, cap), quadratic partners at [cap, 2 cap)
    uint64_t n_sites;  // sites of the batch (index checks of the SIM_CHECK build)
    uint32_t* status;  // the context's device status word (may be null)
};

// Device status bits (read back by every synchronising call).
constexpr uint32_t kStatusBadProtocol = 2u;  // a protocol loaded on the device broke a limit
constexpr uint32_t kStatusBounds = 4u;       // SIM_CHECK build: an index fell outside the batch

// Debug build (-DSIM_CHECK): every global site index of the kernels is checked
// against the batch; a violation sets kStatusBounds and the access is skipped
// (nothing traps).  Compiled out otherwise.
#ifdef SIM_CHECK
__device__ __forceinline__ bool site_ok(const Params& P, int64_t idx) {
    if ((uint64_t)idx < P.n_sites) return true;
    if (P.status) atomicOr(P.status, kStatusBounds);
    return false;
}
#else
__device__ __forceinline__ bool site_ok(const Params&, int64_t) { return true; }
#endif

struct Proto {
    int32_t L;
    int32_t R;
    int64_t site0;   // first site of this protocol in the batch arrays (a multiple of L^2)
    int64_t t_end;   // horizon in steps; the protocol is frozen from then on
    int32_t frac0;   // first entry in the fraction table
    int32_t nfrac;   // fractions (distinct steps)
    int32_t tmap;    // lattice-side class: index of this side's tensor maps (TMA-staged passes)
    int32_t pad;
};

// Work list entry: `n` consecutive sites of protocol `p` starting at local
// index `begin`.  Ragged batches are just lists of such entries.
struct Block {
    int32_t p;
    int32_t n;
    int64_t begin;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based, so every
// (site, step, purpose, protocol) tuple has its own independent draw and a run
// resumed from a checkpoint repeats itself exactly.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform in [0,1) from the top 24 bits: exact in FP32
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }
// floor(u24(x) * n) in exact integer arithmetic
__device__ __forceinline__ uint32_t pick24(uint32_t x, uint32_t n) {
    return (uint32_t)(((uint64_t)(x >> 8) * (uint64_t)n) >> 24);
}

// ---------------------------------------------------------------------------
// storage precision of the fields: FP32 compute, FP32 / BF16 / FP16 storage
template <typename T>
__device__ __forceinline__ float ld(const T* p);
template <>
__device__ __forceinline__ float ld<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <>
__device__ __forceinline__ float ld<__half>(const __half* p) { return __half2float(*p); }

template <typename T>
__device__ __forceinline__ T cvt(float v);
template <>
__device__ __forceinline__ float cvt<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half cvt<__half>(float v) { return __float2half_rn(v); }

// Stochastic rounding for 2-byte field storage.  Round-to-nearest loses every
// per-substep increment below half an ulp of the stored value (a BF16 ulp of
// 0.28 mM is 1e-3 mM, above the O2 uptake of one substep), so the fields
// stagnate.  Rounding up with probability equal to the remainder keeps the
// stored value unbiased.  The random bits come from a counter-based integer
// hash of (site, step, salt), so runs remain reproducible.
__device__ __forceinline__ uint32_t dither_bits(uint32_t site, uint32_t step, uint32_t salt) {
    uint32_t x = site * 0x9E3779B1u ^ (step + 0x632BE5ABu) * 0x85EBCA77u ^ salt * 0xC2B2AE3Du;
    x ^= x >> 16;  // integer avalanche: alternating xor-shifts and odd multiplications
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

// The rounding bits of one site's three fields from one hash: each stored
// value needs 16 random bits (the rounding probability resolved to 2^-16), so
// O2 takes the low and glucose the high half of the hash, and H+ the low half
// of one more xor-shift-multiply round of it.
struct Dither3 {
    uint32_t o, g, h;
};
__device__ __forceinline__ Dither3 dither3(uint32_t site, uint32_t step, uint32_t salt) {
    const uint32_t x = dither_bits(site, step, salt);
    uint32_t y = x ^ (x >> 15);
    y *= 0x2C1B3C6Du;
    y ^= y >> 12;
    return {x & 0xFFFFu, x >> 16, y & 0xFFFFu};
}

template <typename T>
__device__ __forceinline__ T cvt_sr(float v, uint32_t r);
template <>
__device__ __forceinline__ float cvt_sr<float>(float v, uint32_t) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_sr<__nv_bfloat16>(float v, uint32_t r) {
    // BF16 keeps the top 16 bits of an FP32: adding 16 random low bits before truncation rounds up with
    // probability (dropped bits) / 2^16 (values here are finite and >= 0)
    const uint32_t b = __float_as_uint(v) + (r & 0xFFFFu);
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
}
template <>
__device__ __forceinline__ __half cvt_sr<__half>(float v, uint32_t r) {
    const __half lo = __float2half_rd(v), hi = __float2half_ru(v);
    const float flo = __half2float(lo), fhi = __half2float(hi);
    if (fhi == flo) return lo;
    const float u = (float)(r & 0xFFFFu) * 0x1p-16f;  // uniform in [0, 1) from the 16 rounding bits
    // fhi - flo is one FP16 spacing, a power of two: its reciprocal and the product are exact
    return (u < (v - flo) * __frcp_rn(fhi - flo)) ? hi : lo;
}

__device__ __forceinline__ bool is_face(int L, int x, int y, int z) {
    return x == 0 || y == 0 || z == 0 || x == L - 1 || y == L - 1 || z == L - 1;
}

// Dose delivered to protocol `pr` at `step` (fractions on one step were merged
// on the host); *dq receives the dose the quadratic LQ term pairs it with (the
// dose itself, plus twice the unrepaired dose of earlier fractions when repair
// is incomplete).  Fraction tables hold at most a few hundred entries.
__device__ __forceinline__ double dose_at(const Proto& pr, const int64_t* __restrict__ fstep,
                                          const double* __restrict__ fdose, int64_t step, int cap, double* dq) {
    for (int j = 0; j < pr.nfrac; ++j)
        if (fstep[pr.frac0 + j] == step) {
            *dq = fdose[cap + pr.frac0 + j];
            return fdose[pr.frac0 + j];
        }
    *dq = 0.0;
    return 0.0;
}

// Protocol owning global site g (site0 is ascending).
__device__ __forceinline__ int owner(const Proto* __restrict__ protos, int n, int64_t g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (protos[mid].site0 <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Arithmetic of one explicit substep, written with explicit round-to-nearest
// intrinsics so that every kernel (scalar or packed f32x2) performs the same
// operations in the same order and gets bit-identical FP32 results:
//   s = ((xm + xp) + (ym + yp)) + (zm + zp);  lap = fma(-6, c, s);  t = fma(lam, lap, c)
// (a pairwise sum: three dependent additions instead of five)
__device__ __forceinline__ float stencil_t(float c, float xm, float xp, float ym, float yp, float zm, float zp,
                                           float lam) {
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
    const float lap = __fmaf_rn(-6.f, c, s);
    return __fmaf_rn(lam, lap, c);
}

// Uptake of one substep by a cell of the given kind:
//   U_O = f q_O O/(O+K_O);  g = f q_G G/(G+K_G);  w = O_an/(O+O_an)
//   U_G = g (1 + (k_an-1) w);  H+ release = q_H g k_an w
// with f = 1 for cycling and f_Q for quiescent cells.  The three quotients
// share one fast reciprocal: with a = O+K_O, b = O+O_an, c = G+K_G and
// r ~ 1/(a b c), O/a = O (b c) r, G/c = G (a b) r and O_an/b = O_an (a c) r.
// a b c lies in [K_O O_an K_G, ~0.5] (normal floats), so the relative error
// stays at a few FP32 ulps, far inside the per-step field tolerance.
__device__ __forceinline__ void uptake(uint32_t kind, float O, float Gv, const Params& P, float& uO, float& uG,
                                       float& pH) {
    const float f = (kind == kQ) ? P.f_Q : 1.f;
    const float a = __fadd_rn(O, P.K_O), b = __fadd_rn(O, P.O_an), c = __fadd_rn(Gv, P.K_G);
    const float ab = __fmul_rn(a, b);
    const float r = __fdividef(1.f, __fmul_rn(ab, c));
    uO = __fmul_rn(__fmul_rn(__fmul_rn(f, P.q_O), O), __fmul_rn(__fmul_rn(b, c), r));
    const float gg = __fmul_rn(__fmul_rn(__fmul_rn(f, P.q_G), Gv), __fmul_rn(ab, r));
    const float wa = __fmul_rn(P.O_an, __fmul_rn(__fmul_rn(a, c), r));
    uG = __fmul_rn(gg, __fmaf_rn(__fsub_rn(P.k_an, 1.f), wa, 1.f));
    pH = __fmul_rn(__fmul_rn(__fmul_rn(P.q_H, gg), P.k_an), wa);
}

// Cell update of one site from its step-start word and post-diffusion fields:
// necrosis if G < G_d or H > H_d; a G1 cell turns quiescent when O < O_q,
// G < G_q or H > H_q and a quiescent cell returns to G1 once all three are
// restored; cycling cells age and move on at the end of each phase; a cell
// completing M dies if DOOMED, else it stays at the end of M (age capped) and
// sets `want` (division intent).
__device__ __forceinline__ uint32_t update_cell(uint32_t w, float O, float Gv, float H, const Params& P, bool& want) {
    uint32_t kind = w & kKindMask;
    if (kind == kEmpty) return w;
    const uint32_t doomed = w & kDoomed;
    uint32_t age = w >> kAgeShift;
    if ((P.flags & kFDeath) && (Gv < P.G_d || H > P.H_d)) return kEmpty;
    if (kind == kQ) {
        if ((P.flags & kFQuiescence) && O >= P.O_q && Gv >= P.G_q && H <= P.H_q) return kG1 | doomed;
        return w;
    }
    if (kind == kG1 && (P.flags & kFQuiescence) && (O < P.O_q || Gv < P.G_q || H > P.H_q)) return kQ | doomed;
    age += 1;
    if (age >= (uint32_t)P.dur[kind - 1]) {
        if (kind < kM) {
            kind += 1;
            age = 0;
        } else if (doomed) {
            return kEmpty;  // mitotic catastrophe
        } else {
            age = (uint32_t)P.dur[kM - 1];
            want = (P.flags & kFDivision) != 0;
        }
    }
    return kind | doomed | (age << kAgeShift);
}

// LQ survival of a cell of the given kind at O2 level O under dose D:
// S = exp(-a D - b D dq), a = alpha phi OMF(O), b = beta (phi OMF)^2,
// OMF(O) = (m O + K)/(m (O + K)); dq = D with complete repair between
// fractions, D + 2 H (H the unrepaired earlier dose) with incomplete repair.
__device__ __forceinline__ float lq_survival(uint32_t kind, float O, float dose, float dq, const Params& P) {
    const float omf = (P.omf_m * O + P.omf_K) / (P.omf_m * (O + P.omf_K));
    const float mod = P.phi[kind - 1] * omf;
    const float a = P.alpha * mod, bq = P.beta * mod * mod;
    return expf(-a * dose - bq * dose * dq);
}

}  // namespace simdev
