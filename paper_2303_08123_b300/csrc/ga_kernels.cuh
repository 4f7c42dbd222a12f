// ga_kernels.cuh -- one generation of the paper's GA on the device (sm_103a).
//
// ("The Genetic Algorithm (GA)", "The Main GA Loop" and the GA operator
// details.)  The population is P rows of S dose-unit bytes.  The work is small
// and branchy (a few hundred byte operations per child), so each child pair is
// one thread working on its two rows in shared memory, laid out interleaved
// (byte s of thread t at s * T + t) so that a warp's accesses to the same slot
// fall into distinct banks.  Ranking is an all-pairs count (P <= 65536), the
// roulette prefix sum runs in one thread in index order so its FP64 rounding
// is fixed.  Every random decision is one Philox draw with an explicit counter.
#pragma once
#include "sim_device.cuh"

namespace gadev {

using simdev::philox4x32_10;
using simdev::pick24;

constexpr uint32_t kPurposeSelect = 3, kPurposeChild = 4, kPurposeInit = 5;

struct GaParams {
    int S, d_max, cap, gap, n_elite, n_par, selection, crossover;
    uint32_t mutations;
    float p_mut;
    int tk;
    float tq;
    uint32_t key0, key1;
};

// one draw of the stream (individual, generation, purpose): word x0 of counter (k, gen, purpose, who)
struct Stream {
    uint32_t who, gen, purpose, k;
    uint32_t key0, key1;
    __device__ __forceinline__ uint32_t next() {
        return philox4x32_10(make_uint4(k++, gen, purpose, who), key0, key1).x;
    }
    __device__ __forceinline__ float u() { return (float)(next() >> 8) * 0x1p-24f; }
    __device__ __forceinline__ int pick(int n) { return (int)pick24(next(), (uint32_t)n); }
};

// sortable key of a fitness value: larger key = fitter; NaN ranks last
__device__ __forceinline__ uint32_t fit_key(float f) {
    const uint32_t b = __float_as_uint(f);
    if (f != f) return 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// rank of i = number of individuals fitter than i (ties: lower index first);
// order[rank] = i.  Fitness keys are staged through shared memory in chunks.
__global__ void k_rank(const float* __restrict__ fit, int P, int32_t* __restrict__ order) {
    __shared__ uint32_t sk[1024];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t ki = i < P ? fit_key(fit[i]) : 0u;
    int rank = 0;
    for (int base = 0; base < P; base += 1024) {
        __syncthreads();
        for (int j = threadIdx.x; j < 1024 && base + j < P; j += blockDim.x) sk[j] = fit_key(fit[base + j]);
        __syncthreads();
        const int n = min(1024, P - base);
        if (i < P)
            for (int j = 0; j < n; ++j) {
                const uint32_t kj = sk[j];
                rank += (kj > ki) || (kj == ki && base + j < i);
            }
    }
    if (i < P) order[rank] = i;
}

// parents[t], t < n_par: simple / roulette / tournament selection
__global__ void k_select(const float* __restrict__ fit, int P, const int32_t* __restrict__ order,
                         double* __restrict__ cum, int32_t* __restrict__ parents, GaParams g, uint32_t gen) {
    if (g.selection == 1) {  // roulette: FP64 prefix sum of the shifted fitness, in index order, one thread
        if (threadIdx.x == 0) {
            double lo = 0.0;
            for (int i = 0; i < P; ++i) {
                const float f = fit[i];
                const double v = (f == f) ? (double)f : 0.0;
                lo = v < lo ? v : lo;
            }
            double c = 0.0;
            for (int i = 0; i < P; ++i) {
                const float f = fit[i];
                const double v = (f == f) ? (double)f : 0.0;
                c += v - lo;
                cum[i] = c;
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < g.n_par; t += blockDim.x) {
        Stream rs{(uint32_t)t, gen, kPurposeSelect, 0u, g.key0, g.key1};
        int who;
        if (g.selection == 0) {
            who = order[t];
        } else if (g.selection == 1) {
            const double total = cum[P - 1];
            if (!(total > 0.0)) {
                who = rs.pick(P);
            } else {
                const double target = (double)(rs.next() >> 8) * 0x1p-24 * total;
                int lo = 0, hi = P;  // first i with cum[i] >= target (P if none)
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cum[mid] >= target) hi = mid;
                    else lo = mid + 1;
                }
                who = lo < P ? lo : P - 1;
            }
        } else {
            // k entrants among the ranking positions 0..P-1, without replacement (Floyd), best first
            int ent[64];
            const int K = g.tk;
            int n = 0;
            for (int j = P - K; j < P; ++j) {
                const int r = rs.pick(j + 1);
                bool seen = false;
                for (int e = 0; e < n; ++e) seen |= ent[e] == r;
                ent[n++] = seen ? j : r;
            }
            for (int a = 1; a < K; ++a) {  // insertion sort, ascending position = fitter first
                const int v = ent[a];
                int b = a - 1;
                while (b >= 0 && ent[b] > v) {
                    ent[b + 1] = ent[b];
                    --b;
                }
                ent[b + 1] = v;
            }
            int r = 0;
            while (r < K - 1 && rs.u() >= g.tq) ++r;
            who = order[ent[r]];
        }
        parents[t] = who;
    }
}

// rows 0..n_elite-1 of the next population: the n_elite best, unchanged
__global__ void k_elites(const uint8_t* __restrict__ pop, const int32_t* __restrict__ order, int n_elite, int S,
                         uint8_t* __restrict__ next) {
    const int r = blockIdx.x;
    if (r >= n_elite) return;
    const uint8_t* src = pop + (size_t)order[r] * S;
    for (int s = threadIdx.x; s < S; s += blockDim.x) next[(size_t)r * S + s] = src[s];
}

// A child row in shared memory: byte s at base[s * T].
struct Row {
    uint8_t* base;
    int T;
    __device__ __forceinline__ uint8_t& operator[](int s) const { return base[s * T]; }
};

__device__ __forceinline__ int row_total(const Row& v, int S) {
    int t = 0;
    for (int s = 0; s < S; ++s) t += v[s];
    return t;
}

// k-th occupied slot (k < count) among slots with value > above
__device__ __forceinline__ int kth_above(const Row& v, int S, int above, int k) {
    for (int s = 0; s < S; ++s)
        if (v[s] > above && k-- == 0) return s;
    return -1;
}

__device__ __forceinline__ int count_above(const Row& v, int S, int above) {
    int n = 0;
    for (int s = 0; s < S; ++s) n += v[s] > above;
    return n;
}

// slots at distance >= gap from every occupied slot; k < 0: count them, else return the k-th
__device__ int free_slots(const Row& v, int S, int gap, int k) {
    constexpr int kFar = 1 << 20;
    int last = -kFar, nx = 0, n = 0;
    while (nx < S && !v[nx]) ++nx;
    if (nx >= S) nx = kFar;
    for (int s = 0; s < S; ++s) {
        if (nx < s) {  // next occupied slot at or after s
            nx = s;
            while (nx < S && !v[nx]) ++nx;
            if (nx >= S) nx = kFar;
        }
        if (s - last >= gap && nx - s >= gap) {
            if (k == n) return s;
            ++n;
        }
        if (v[s]) last = s;
    }
    return k < 0 ? n : -1;
}

// guards: clip to d_max, minimum interval (relocate or fold), total cap
__device__ void repair(const Row& v, const GaParams& g, Stream& rs) {
    const int S = g.S;
    for (int s = 0; s < S; ++s)
        if (v[s] > g.d_max) v[s] = (uint8_t)g.d_max;
    for (int guard = 0; guard < S; ++guard) {  // each pass removes at least one violation
        int prev = -1, j = -1;
        for (int s = 0; s < S; ++s)
            if (v[s]) {
                if (prev >= 0 && s - prev < g.gap) {
                    j = s;
                    break;
                }
                prev = s;
            }
        if (j < 0) break;
        const int d = v[j];
        v[j] = 0;
        const int nf = free_slots(v, S, g.gap, -1);
        if (nf > 0) {
            v[free_slots(v, S, g.gap, rs.pick(nf))] = (uint8_t)d;
        } else {
            const int f = v[prev] + d;
            v[prev] = (uint8_t)(f < g.d_max ? f : g.d_max);
        }
    }
    int total = row_total(v, S);
    while (total > g.cap) {
        int j = 0;
        for (int s = 1; s < S; ++s)
            if (v[s] > v[j]) j = s;
        v[j] = (uint8_t)(v[j] - 1);
        --total;
    }
}

__device__ void mutate(const Row& v, const GaParams& g, Stream& rs) {
    const int S = g.S;
    for (int kind = 0; kind < 4; ++kind) {
        if (!(g.mutations & (1u << kind))) continue;
        if (!(rs.u() < g.p_mut)) continue;
        if (kind == 0) {  // swap: a fraction trades places with a random slot
            const int n = count_above(v, S, 0);
            if (!n) continue;
            const int i = kth_above(v, S, 0, rs.pick(n)), j = rs.pick(S);
            const uint8_t t = v[i];
            v[i] = v[j];
            v[j] = t;
        } else if (kind == 1) {  // split: a dose > 1 unit becomes two parts placed within d_max
            const int n = count_above(v, S, 1);
            if (!n) continue;
            const int i = kth_above(v, S, 1, rs.pick(n));
            const int part = 1 + rs.pick(v[i] - 1), rest = v[i] - part;
            v[i] = 0;
            for (int h = 0; h < 2; ++h) {
                const int d = h ? rest : part;
                bool placed = false;
                for (int tries = 0; tries < 8 && !placed; ++tries) {
                    const int j = rs.pick(S);
                    if (v[j] + d <= g.d_max) {
                        v[j] = (uint8_t)(v[j] + d);
                        placed = true;
                    }
                }
                if (!placed) v[i] = (uint8_t)(v[i] + d);
            }
        } else if (kind == 2) {  // dose-time: move a dose, at most up to d_max at the target
            const int n = count_above(v, S, 0);
            if (!n) continue;
            const int i = kth_above(v, S, 0, rs.pick(n)), j = rs.pick(S);
            int moved = (j != i) ? min((int)v[i], g.d_max - (int)v[j]) : 0;
            moved = max(0, moved);
            v[j] = (uint8_t)(v[j] + moved);
            v[i] = (uint8_t)(v[i] - moved);
        } else {  // dose-value: raise a dose into the slack under the cap
            const int slack = g.cap - row_total(v, S);
            const int n = count_above(v, S, 0);
            if (slack <= 0 || !n) continue;
            const int i = kth_above(v, S, 0, rs.pick(n));
            const int room = min(slack, g.d_max - (int)v[i]);
            if (room > 0) v[i] = (uint8_t)(v[i] + 1 + rs.pick(room));
        }
    }
}

// children: thread m builds pair m (rows n_elite + 2m, n_elite + 2m + 1)
__global__ void k_children(const uint8_t* __restrict__ pop, const int32_t* __restrict__ parents, int P,
                           uint8_t* __restrict__ next, GaParams g, uint32_t gen) {
    extern __shared__ uint8_t sm[];
    const int T = blockDim.x, t = threadIdx.x;
    const int m = blockIdx.x * T + t;
    const int n_children = P - g.n_elite;
    const int n_pairs = (n_children + 1) / 2;
    if (m >= n_pairs) return;
    const int S = g.S;
    const Row c0{sm + t, T}, c1{sm + (size_t)S * T + t, T};
    Stream rs{(uint32_t)m, gen, kPurposeChild, 0u, g.key0, g.key1};
    const int ap = rs.pick(g.n_par);
    const int bq = rs.pick(g.n_par > 1 ? g.n_par - 1 : 1);
    const int bp = g.n_par > 1 ? bq + (bq >= ap) : ap;
    const uint8_t* A = pop + (size_t)parents[ap] * S;
    const uint8_t* B = pop + (size_t)parents[bp] * S;
    int cut1 = S, cut2 = S;
    if (g.crossover == 0) {
        cut1 = S / 4 + rs.pick(3 * S / 4 - S / 4 + 1);
    } else if (g.crossover == 1) {
        cut1 = S / 4 + rs.pick(S / 2 - S / 4 + 1);
        cut2 = S / 2 + rs.pick(3 * S / 4 - S / 2 + 1);
    }
    for (int s = 0; s < S; ++s) {
        bool fromA;
        if (g.crossover == 2) fromA = rs.u() < 0.5f;
        else fromA = s < cut1 || s >= cut2;
        c0[s] = fromA ? A[s] : B[s];
        c1[s] = fromA ? B[s] : A[s];
    }
    const int r0 = g.n_elite + 2 * m;
    for (int h = 0; h < 2; ++h) {
        if (r0 + h >= P) break;
        const Row& c = h ? c1 : c0;
        mutate(c, g, rs);
        repair(c, g, rs);
        uint8_t* dst = next + (size_t)(r0 + h) * S;
        for (int s = 0; s < S; ++s) dst[s] = c[s];
    }
}

// random initial population: row i gets 1 + pick(S / gap) fractions of 1 + pick(d_max) units
__global__ void k_random_population(int P, uint8_t* __restrict__ pop, GaParams g) {
    extern __shared__ uint8_t sm[];
    const int T = blockDim.x, t = threadIdx.x;
    const int i = blockIdx.x * T + t;
    if (i >= P) return;
    const int S = g.S;
    const Row v{sm + t, T};
    for (int s = 0; s < S; ++s) v[s] = 0;
    Stream rs{(uint32_t)i, 0u, kPurposeInit, 0u, g.key0, g.key1};
    const int nf = 1 + rs.pick(S / g.gap);
    for (int f = 0; f < nf; ++f) {
        const int s = rs.pick(S);
        const int add = 1 + rs.pick(g.d_max);
        v[s] = (uint8_t)min(255, (int)v[s] + add);
    }
    repair(v, g, rs);
    for (int s = 0; s < S; ++s) pop[(size_t)i * S + s] = v[s];
}

}  // namespace gadev
