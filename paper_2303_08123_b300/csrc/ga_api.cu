// ga_api.cu -- extern "C" entry points of libga (include/ga.h).
#include <atomic>

#include "ga.h"
#include "ga_kernels.cuh"

namespace {

constexpr size_t kAlign = 256;
constexpr int kSmemBudget = 100 * 1024;  // dynamic shared memory of the child kernels

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct GaLayout {
    size_t order, parents, cum, total;
};

GaLayout ga_layout(int P) {
    GaLayout l{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    l.order = take(sizeof(int32_t) * (size_t)P);
    l.parents = take(sizeof(int32_t) * (size_t)P);
    l.cum = take(sizeof(double) * (size_t)P);
    l.total = off;
    return l;
}

bool valid(const ga_params* p, int P) {
    if (!p || P < 1 || P > GA_MAX_POPULATION) return false;
    if (p->n_slots < 1 || p->n_slots > GA_MAX_SLOTS) return false;
    if (p->d_max < 1 || p->d_max > 255 || p->total_cap < 0 || p->min_gap < 1) return false;
    if (p->n_elite < 0 || p->n_elite > P || p->n_parents < 1 || p->n_parents > P) return false;
    if (p->selection < GA_SEL_SIMPLE || p->selection > GA_SEL_TOURNAMENT) return false;
    if (p->crossover < GA_X_SINGLE_POINT || p->crossover > GA_X_UNIFORM) return false;
    if (p->mutations & ~0xFu) return false;
    if (!(p->p_mut >= 0.f && p->p_mut <= 1.f)) return false;
    if (p->selection == GA_SEL_TOURNAMENT) {
        if (p->tournament_k < 1 || p->tournament_k > GA_MAX_TOURNAMENT || p->tournament_k > P) return false;
        if (!(p->tournament_q >= 0.f && p->tournament_q <= 1.f)) return false;
    }
    return true;
}

gadev::GaParams to_device(const ga_params* p, uint64_t seed) {
    gadev::GaParams g{};
    g.S = p->n_slots;
    g.d_max = p->d_max;
    g.cap = p->total_cap;
    g.gap = p->min_gap;
    g.n_elite = p->n_elite;
    g.n_par = p->n_parents;
    g.selection = p->selection;
    g.crossover = p->crossover;
    g.mutations = p->mutations;
    g.p_mut = p->p_mut;
    g.tk = p->tournament_k;
    g.tq = p->tournament_q;
    g.key0 = (uint32_t)(seed & 0xffffffffu);
    g.key1 = (uint32_t)(seed >> 32);
    return g;
}

// threads per block of the per-row kernels: two (children) or one row of S bytes each in shared memory
int row_threads(int S, int rows) {
    for (int t = 128; t > 32; t /= 2)
        if ((size_t)t * rows * S <= (size_t)kSmemBudget) return t;
    return 32;
}

// dynamic shared memory above 48 KB must be allowed once per device
cudaError_t set_smem_attrs() {
    static std::atomic<uint64_t> done{0};  // bit d: device d is set up (devices 0..63; others every call)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 64 && ((done.load() >> dev) & 1u)) return cudaSuccess;
    e = cudaFuncSetAttribute(gadev::k_children, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
    if (!e) e = cudaFuncSetAttribute(gadev::k_random_population, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kSmemBudget);
    if (!e && dev < 64) done.fetch_or(1ull << dev);
    return e;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? 0 : -3; }

}  // namespace

extern "C" {

int ga_workspace_size(int P, size_t* bytes) {
    if (!bytes || P < 1 || P > GA_MAX_POPULATION) return -1;
    *bytes = ga_layout(P).total;
    return 0;
}

int ga_random_population(const ga_params* prm, int P, uint64_t seed, uint8_t* d_pop, void* cuda_stream) {
    if (!valid(prm, P) || !d_pop) return -1;
    if (cudaError_t e = set_smem_attrs()) return status_of(e);
    const gadev::GaParams g = to_device(prm, seed);
    const int T = row_threads(g.S, 1);
    gadev::k_random_population<<<(P + T - 1) / T, T, (size_t)T * g.S, (cudaStream_t)cuda_stream>>>(P, d_pop, g);
    return status_of(cudaGetLastError());
}

int ga_generation(const ga_params* prm, int P, const uint8_t* d_pop, const float* d_fitness, uint64_t seed,
                  uint32_t generation, uint8_t* d_next, int32_t* d_order, void* d_workspace, size_t bytes,
                  void* cuda_stream) {
    if (!valid(prm, P) || !d_pop || !d_fitness || !d_next || !d_workspace) return -1;
    const size_t rowb = (size_t)P * prm->n_slots;
    const uintptr_t a = (uintptr_t)d_pop, b = (uintptr_t)d_next;
    if (a < b + rowb && b < a + rowb) return -1;  // overlapping populations
    if ((uintptr_t)d_workspace % kAlign) return -1;
    const GaLayout l = ga_layout(P);
    if (bytes < l.total) return -2;
    if (cudaError_t e = set_smem_attrs()) return status_of(e);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    char* ws = (char*)d_workspace;
    int32_t* order = (int32_t*)(ws + l.order);
    int32_t* parents = (int32_t*)(ws + l.parents);
    double* cum = (double*)(ws + l.cum);
    const gadev::GaParams g = to_device(prm, seed);
    gadev::k_rank<<<(P + 255) / 256, 256, 0, s>>>(d_fitness, P, order);
    gadev::k_select<<<1, 1024, 0, s>>>(d_fitness, P, order, cum, parents, g, generation);
    if (g.n_elite > 0) gadev::k_elites<<<g.n_elite, 128, 0, s>>>(d_pop, order, g.n_elite, g.S, d_next);
    const int n_pairs = (P - g.n_elite + 1) / 2;
    if (n_pairs > 0) {
        const int T = row_threads(g.S, 2);
        gadev::k_children<<<(n_pairs + T - 1) / T, T, (size_t)2 * T * g.S, s>>>(d_pop, parents, P, d_next, g,
                                                                                 generation);
    }
    cudaError_t e = cudaGetLastError();
    if (!e && d_order) e = cudaMemcpyAsync(d_order, order, sizeof(int32_t) * P, cudaMemcpyDeviceToDevice, s);
    return status_of(e);
}

}  // extern "C"
