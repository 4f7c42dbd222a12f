// sim_api.cu -- the C ABI of libsim (declared in include/sim.h).
//
// Host side of the batched simulator: validates protocols, lays the batch out
// in the caller's workspace, builds the ragged work list, launches the step
// kernels (or replays one captured CUDA graph per simulated hour) and moves
// results back.  No device memory is allocated here.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sim.h"
#include "sim_kernels.cuh"
#include "sim_fused.cuh"
#include "sim_fused1h.cuh"
#include "sim_tma.cuh"

using namespace simdev;

namespace {

constexpr int kSitesPerBlock = 1024;  // work-list granularity (sites per CTA)
constexpr int kMaxL = 1024;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t elem_size(int precision) { return precision == SIM_FP32 ? 4 : 2; }

// Byte offsets of every region of the workspace.
struct Layout {
    size_t proto, blocks, tiles, fstep, fdose, field[2][3], cell[2], claim, intents, target, icount, counts, cum,
        clock, status, final_count, first_block, part64, part32, tot64, tot32, tile_ctr, tmaps, total;
};

constexpr int kTmaShapes = 4;  // tile shapes 5-8 stage their planes by TMA (one set of tensor maps each)

// Number of distinct lattice sides (one set of tensor maps each).
int side_classes(int n, const int32_t* L) {
    std::vector<int32_t> u(L, L + n);
    std::sort(u.begin(), u.end());
    return (int)(std::unique(u.begin(), u.end()) - u.begin());
}

Layout make_layout(const sim_config& cfg, int n, int64_t total_sites, int64_t nblocks, int64_t ntiles,
                   int n_sides) {
    Layout l{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    const size_t es = elem_size(cfg.precision);
    const int64_t nf = (int64_t)n * cfg.max_fractions;
    l.proto = take(sizeof(Proto) * n);
    l.blocks = take(sizeof(Block) * nblocks);
    l.tiles = take(sizeof(Tile) * (ntiles > 0 ? ntiles : 1));
    l.fstep = take(sizeof(int64_t) * (nf > 0 ? nf : 1));
    l.fdose = take(sizeof(double) * 2 * (nf > 0 ? nf : 1));  // doses, then their quadratic partners
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < 3; ++f) l.field[b][f] = take(es * total_sites);
    l.cell[0] = take(4 * total_sites);
    l.cell[1] = take(4 * total_sites);
    l.claim = take(8 * total_sites);
    l.intents = take(4 * total_sites);
    l.target = take(4 * total_sites);
    l.icount = take(4 * 2);
    l.counts = take(sizeof(int32_t) * n * (size_t)(cfg.hours + 1));
    l.cum = take(sizeof(double) * n);
    l.clock = take(sizeof(int64_t));
    l.status = take(sizeof(uint32_t));
    l.final_count = take(sizeof(int32_t) * n);
    l.first_block = take(sizeof(int32_t) * (n + 1));
    l.part64 = take(sizeof(double) * 3 * nblocks);
    l.part32 = take(sizeof(float) * 3 * nblocks);
    l.tot64 = take(sizeof(double) * 3 * n);
    l.tot32 = take(sizeof(float) * 3 * n);
    l.tile_ctr = take(sizeof(uint32_t) * 2 * kMaxPasses);
    l.tmaps = take(sizeof(CUtensorMap) * kTmaShapes * (size_t)n_sides * kTmaArrays);
    l.total = off;
    return l;
}

bool valid_config(const sim_config* cfg, std::string* why) {
    const sim_params& p = cfg->params;
    if (cfg->precision < SIM_FP32 || cfg->precision > SIM_FP16) return *why = "precision must be 0, 1 or 2", false;
    if (p.n_sub < 1 || p.n_sub > 256) return *why = "n_sub must be in 1..256", false;
    for (int i = 0; i < 4; ++i) {
        const double st = p.dur_h[i] * kStepsPerHour;
        if (!(st >= 1.0) || st > 1e8) return *why = "phase durations must be at least one step", false;
    }
    for (int i = 0; i < 3; ++i)
        if (!(p.lam[i] >= 0.0 && p.lam[i] <= 1.0 / 6.0 + 1e-12))
            return *why = "diffusion numbers must lie in [0, 1/6] (FTCS stability in 3-D)", false;
    if (cfg->hours < 0 || cfg->hours > 1000000) return *why = "hours out of range", false;
    if (cfg->max_fractions < 0 || cfg->max_fractions > 100000) return *why = "max_fractions out of range", false;
    if (!std::isfinite(cfg->params.repair_half_h) || cfg->params.repair_half_h < 0.0)
        return *why = "repair_half_h must be finite and >= 0", false;
    if (cfg->regrowth_h < 0) return *why = "regrowth_h must be >= 0", false;
    if (cfg->path < SIM_PATH_FUSED || cfg->path > SIM_PATH_SUBSTEP) return *why = "unknown kernel path", false;
    if (cfg->tile_shape < 0 || cfg->tile_shape > 8) return *why = "tile_shape must be in 0..8", false;
    if (cfg->z_chunk < 0) return *why = "z_chunk must be >= 0", false;
    return true;
}

// Tile shapes of the fused kernels: (x extent, y extent); shapes 1-2 run two
// columns per thread (packed f32x2), shapes 3-4 one column per thread, shapes
// 5-6 one column per thread with the planes staged by TMA (FP32 storage),
// shapes 7-8 the same with passes of four substeps (deep temporal blocking;
// an even substep count, the last pass two deep when it is not a multiple of 4).
constexpr int kNumShapes = 8;
constexpr int kTileShapes[kNumShapes + 1][2] = {{0, 0},   {32, 16}, {16, 16}, {32, 16}, {16, 16},
                                                {32, 16}, {16, 16}, {32, 16}, {16, 16}};
bool tma_shape(int sh) { return sh >= 5 && sh <= 8; }
bool deep_shape(int sh) { return sh == 7 || sh == 8; }
int tma_halo_y(int sh) { return deep_shape(sh) ? 4 : 2; }  // rows of halo in the staged box

// First site of each protocol: the running total rounded up to a multiple of
// L^2, so that a protocol's planes are whole z-slices of the L x L x Z volume a
// tensor map of its side describes.  Returns the padded total.
int64_t place_protocols(int n, const int32_t* L, int64_t* site0) {
    int64_t at = 0;
    for (int p = 0; p < n; ++p) {
        const int64_t LL = (int64_t)L[p] * L[p];
        at = (at + LL - 1) / LL * LL;
        if (site0) site0[p] = at;
        at += LL * L[p];
    }
    return at;
}
constexpr int kTargetCtas = 2 * 148;  // at least two CTAs per SM when the batch allows it

// Default tile shape (the autotuner may pick any): one column per thread, the
// tile covering the fewest sites; on a tie the larger tile, unless the batch
// then has too few tiles to give every SM two CTAs' worth of work.
int pick_shape(const sim_config& cfg, int n, const int32_t* L) {
    if (cfg.tile_shape) return cfg.tile_shape;
    int64_t area[kNumShapes + 1] = {}, tiles[kNumShapes + 1] = {};
    for (int sh = 3; sh <= 4; ++sh)
        for (int p = 0; p < n; ++p) {
            const int64_t tx = (L[p] + kTileShapes[sh][0] - 1) / kTileShapes[sh][0];
            const int64_t ty = (L[p] + kTileShapes[sh][1] - 1) / kTileShapes[sh][1];
            area[sh] += tx * kTileShapes[sh][0] * ty * kTileShapes[sh][1] * (int64_t)L[p];
            tiles[sh] += tx * ty;
        }
    if (area[4] < area[3]) return 4;
    if (area[3] < area[4]) return 3;
    return tiles[3] >= kTargetCtas ? 3 : 4;
}

constexpr int kFineZ = 2;  // the finer z split the autotuner also tries on batches with too few columns

// Fused work list: column tiles of every protocol still running (live[p] != 0;
// live == nullptr: all), split in z when those have too few columns to fill the
// GPU (chunks of at least 8 planes, or of fine_z planes when fine_z > 0).
std::vector<Tile> make_tiles(const sim_config& cfg, int n, const int32_t* L, int shape,
                             const uint8_t* live = nullptr, int fine_z = 0) {
    const int TX = kTileShapes[shape][0], TY = kTileShapes[shape][1];
    int64_t cols = 0;
    for (int p = 0; p < n; ++p)
        if (!live || live[p]) cols += (int64_t)((L[p] + TX - 1) / TX) * ((L[p] + TY - 1) / TY);
    std::vector<Tile> t;
    for (int p = 0; p < n; ++p) {
        if (live && !live[p]) continue;
        int zc = L[p];
        if (cfg.z_chunk > 0) zc = cfg.z_chunk;
        else if (cols < kTargetCtas) {
            const int64_t nz = (kTargetCtas + cols - 1) / cols;
            zc = (int)((L[p] + nz - 1) / nz);
            if (fine_z > 0) zc = fine_z;
            else if (zc < 8) zc = 8;
        }
        for (int z = 0; z < L[p]; z += zc)
            for (int y = 0; y < L[p]; y += TY)
                for (int x = 0; x < L[p]; x += TX) {
                    Tile e{};
                    e.p = p;
                    e.x0 = (int16_t)x;
                    e.y0 = (int16_t)y;
                    e.z0 = (int16_t)z;
                    e.z1 = (int16_t)((z + zc) < L[p] ? z + zc : L[p]);
                    t.push_back(e);
                }
    }
    // longest z ranges first, so the persistent CTAs finish together (ties keep their order)
    std::stable_sort(t.begin(), t.end(), [](const Tile& a, const Tile& b) { return a.z1 - a.z0 > b.z1 - b.z0; });
    return t;
}

// True if the batch has too few columns to fill the GPU, so that its work list is split in z.
bool z_split_applies(const sim_config& cfg, int n, const int32_t* L, int shape) {
    if (cfg.z_chunk > 0) return false;
    const int TX = kTileShapes[shape][0], TY = kTileShapes[shape][1];
    int64_t cols = 0;
    for (int p = 0; p < n; ++p) cols += (int64_t)((L[p] + TX - 1) / TX) * ((L[p] + TY - 1) / TY);
    return cols < kTargetCtas;
}

}  // namespace

struct sim_ctx {
    sim_config cfg{};
    Params P{};
    int n = 0;
    std::vector<Proto> proto;
    std::vector<Block> blocks;
    std::vector<Tile> tiles;
    std::vector<uint8_t> tile_live;  // protocols the fused work list covers
    int shape = 1;
    int fine_z = 0;  // > 0: the autotuner chose the finer z split (chunks of this many planes)
    int vec_ok = 1;  // every lattice side even: column pairs start on even elements
    int64_t total_sites = 0;
    Layout lay{};
    char* ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    int64_t clock = 0;          // host mirror of the device clock
    int cur = 0;                // field buffer holding the current state
    int ccur = 0;               // cell-word buffer holding the current state
    int64_t counted_hour = -1;  // last hour whose counts were recorded
    bool loaded = false;
    cudaGraphExec_t hour_graph[4] = {nullptr, nullptr, nullptr, nullptr};  // by (field, cell) start buffers
    bool tma_ok = false;  // tensor maps encoded: shapes 5-8 may run
    int n_sides = 0;      // distinct lattice sides (tensor-map classes)
    std::string err;

    template <typename T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
    void* field(int buf, int f) const { return ws + lay.field[buf][f]; }
    uint32_t* cells(int buf) const { return reinterpret_cast<uint32_t*>(ws + lay.cell[buf]); }
    bool fused() const { return cfg.path == SIM_PATH_FUSED; }
    // substeps per fused pass: passes of two (of four on the deep shapes), the last one shorter by the remainder
    int depth() const { return deep_shape(shape) ? 4 : 2; }
    int passes() const { return (P.n_sub + depth() - 1) / depth(); }
    int pass_k(int j) const { return j < passes() - 1 ? depth() : P.n_sub - depth() * (passes() - 1); }
    int field_flips() const { return fused() ? passes() : P.n_sub; }
    int cell_flips() const { return fused() ? 1 : 0; }
};

namespace {

sim_status fail(sim_ctx* c, sim_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

sim_status cuda_check(sim_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SIM_OK;
    return fail(c, SIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

Params make_params(const sim_config& cfg) {
    const sim_params& p = cfg.params;
    Params P{};
    for (int i = 0; i < 4; ++i) P.dur[i] = (int)llround(p.dur_h[i] * kStepsPerHour);
    P.n_sub = p.n_sub;
    P.flags = p.flags;
    for (int i = 0; i < 3; ++i) P.lam[i] = (float)p.lam[i];
    P.med[0] = (float)p.medium_O;
    P.med[1] = (float)p.medium_G;
    P.med[2] = (float)std::pow(10.0, 3.0 - p.medium_pH);  // pH -> mM of H+
    P.q_O = (float)p.q_O; P.K_O = (float)p.K_O; P.q_G = (float)p.q_G; P.K_G = (float)p.K_G;
    P.k_an = (float)p.k_an; P.O_an = (float)p.O_an; P.q_H = (float)p.q_H; P.f_Q = (float)p.f_Q;
    P.alpha = (float)p.alpha; P.beta = (float)p.beta; P.omf_m = (float)p.omf_m; P.omf_K = (float)p.omf_K;
    for (int i = 0; i < 5; ++i) P.phi[i] = (float)p.phi[i];
    P.O_q = (float)p.O_q; P.G_q = (float)p.G_q; P.G_d = (float)p.G_d;
    P.H_q = (float)std::pow(10.0, 3.0 - p.pH_q);
    P.H_d = (float)std::pow(10.0, 3.0 - p.pH_d);
    P.key0 = (uint32_t)(cfg.seed & 0xffffffffu);
    P.key1 = (uint32_t)(cfg.seed >> 32);
    P.init_word = cfg.init_word;
    return P;
}

template <typename T>
sim_status launch_init(sim_ctx* c) {
    k_init<T><<<(unsigned)c->blocks.size(), kThreads, 0, c->stream>>>(
        c->at<Block>(c->lay.blocks), c->at<Proto>(c->lay.proto), (T*)c->field(0, 0), (T*)c->field(0, 1),
        (T*)c->field(0, 2), (T*)c->field(1, 0), (T*)c->field(1, 1), (T*)c->field(1, 2), c->cells(0),
        c->at<unsigned long long>(c->lay.claim), c->P);
    return cuda_check(c, cudaGetLastError(), "k_init launch");
}

sim_status reset_device(sim_ctx* c) {
    sim_status st;
    switch (c->cfg.precision) {
        case SIM_BF16: st = launch_init<__nv_bfloat16>(c); break;
        case SIM_FP16: st = launch_init<__half>(c); break;
        default: st = launch_init<float>(c); break;
    }
    if (st) return st;
    cudaError_t e = cudaMemsetAsync(c->ws + c->lay.icount, 0, 8, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.tile_ctr, 0, sizeof(uint32_t) * 2 * kMaxPasses, c->stream);
    if (!e)
        e = cudaMemsetAsync(c->ws + c->lay.counts, 0, sizeof(int32_t) * c->n * (size_t)(c->cfg.hours + 1), c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.cum, 0, sizeof(double) * c->n, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.clock, 0, sizeof(int64_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.status, 0, sizeof(uint32_t), c->stream);
    c->clock = 0;
    c->cur = 0;
    c->ccur = 0;
    c->counted_hour = -1;
    return cuda_check(c, e, "reset");
}

// One CA step for every protocol, reading the step index as clock + k_off.
// Persistent grid: as many CTAs as fit on the device at once (at most one per tile).
template <typename Kern>
unsigned persistent_grid(Kern kern, int threads, size_t smem, size_t n_tiles) {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    const size_t g = (size_t)sms * (size_t)(per_sm > 0 ? per_sm : 1);
    return (unsigned)(g < n_tiles ? g : n_tiles);
}

template <typename T, int TX, int TY, int K, bool EPI>
void launch_fused_t(sim_ctx* c, cudaStream_t s, int k_off, int first, int buf, const uint32_t* cin, uint32_t* cout,
                    int pass) {
    using Sh = FusedShape<TX, TY, K>;
    static unsigned grid = 0;  // per instantiation: the occupancy does not depend on the batch
    if (!grid) grid = persistent_grid(k_fused<T, TX, TY, K, EPI>, Sh::THREADS, fused_smem_bytes<T, TX, TY, K>(), ~0ull);
    const unsigned g = grid < c->tiles.size() ? grid : (unsigned)c->tiles.size();
    k_fused<T, TX, TY, K, EPI><<<g, Sh::THREADS, fused_smem_bytes<T, TX, TY, K>(), s>>>(
        c->at<Tile>(c->lay.tiles), c->at<Proto>(c->lay.proto), c->at<int64_t>(c->lay.clock), k_off, first,
        (c->vec_ok && K % 2 == 0) ? 1 : 0, (const T*)c->field(buf, 0), (const T*)c->field(buf, 1), (const T*)c->field(buf, 2), (T*)c->field(buf ^ 1, 0),
        (T*)c->field(buf ^ 1, 1), (T*)c->field(buf ^ 1, 2), cin, cout, c->at<int64_t>(c->lay.fstep),
        c->at<double>(c->lay.fdose), c->at<double>(c->lay.cum), c->at<uint32_t>(c->lay.intents),
        c->at<uint32_t>(c->lay.icount), c->at<uint32_t>(c->lay.tile_ctr), (int)c->tiles.size(), pass, c->P);
}

// the one-column-per-thread kernel of storage type T: k_fused1 for FP32, k_fused1h for 2-byte types
template <typename T, int TX, int TY, int K, bool EPI, bool FULL>
constexpr auto fused1_kernel() {
    if constexpr (std::is_same<T, float>::value) return k_fused1<TX, TY, K, EPI, FULL>;
    else return k_fused1h<T, TX, TY, K, EPI, FULL>;
}
template <typename T, int TX, int TY, int K>
constexpr size_t fused1_bytes() {
    if constexpr (std::is_same<T, float>::value) return fused1_smem_bytes<TX, TY, K>();
    else return fused1h_smem_bytes<T, TX, TY, K>();
}

template <typename T, int TX, int TY, int K, bool EPI, bool FULL>
void launch_fused1_f(sim_ctx* c, cudaStream_t s, int k_off, int first, int buf, const uint32_t* cin,
                     uint32_t* cout, int pass) {
    using Sh = FusedShape1<TX, TY, K>;
    constexpr auto kern = fused1_kernel<T, TX, TY, K, EPI, FULL>();
    static unsigned grid = 0;
    if (!grid) grid = persistent_grid(kern, Sh::THREADS, fused1_bytes<T, TX, TY, K>(), ~0ull);
    const unsigned g = grid < c->tiles.size() ? grid : (unsigned)c->tiles.size();
    kern<<<g, Sh::THREADS, fused1_bytes<T, TX, TY, K>(), s>>>(
        c->at<Tile>(c->lay.tiles), c->at<Proto>(c->lay.proto), c->at<int64_t>(c->lay.clock), k_off, first,
        (const T*)c->field(buf, 0), (const T*)c->field(buf, 1), (const T*)c->field(buf, 2),
        (T*)c->field(buf ^ 1, 0), (T*)c->field(buf ^ 1, 1), (T*)c->field(buf ^ 1, 2), cin, cout,
        c->at<int64_t>(c->lay.fstep), c->at<double>(c->lay.fdose), c->at<double>(c->lay.cum),
        c->at<uint32_t>(c->lay.intents), c->at<uint32_t>(c->lay.icount), c->at<uint32_t>(c->lay.tile_ctr),
        (int)c->tiles.size(), pass, c->P);
}

// diffusion and reaction on (the model as run): the instance with both switches fixed at compile time
template <typename T, int TX, int TY, int K, bool EPI>
void launch_fused1_t(sim_ctx* c, cudaStream_t s, int k_off, int first, int buf, const uint32_t* cin,
                     uint32_t* cout, int pass) {
    if ((c->P.flags & (kFDiffusion | kFReaction)) == (kFDiffusion | kFReaction))
        launch_fused1_f<T, TX, TY, K, EPI, true>(c, s, k_off, first, buf, cin, cout, pass);
    else
        launch_fused1_f<T, TX, TY, K, EPI, false>(c, s, k_off, first, buf, cin, cout, pass);
}

template <int TX, int TY, int K, int HY, bool EPI, bool FULL>
void launch_tma_f(sim_ctx* c, cudaStream_t s, int k_off, int first, int buf, int cbuf, uint32_t* cout, int pass) {
    using Sh = TmaShape<TX, TY, K, HY>;
    constexpr auto kern = k_tma<TX, TY, K, HY, EPI, FULL>;
    constexpr size_t smem = tma_smem_bytes<TX, TY, K, HY>();
    static unsigned grid = 0;
    if (!grid) grid = persistent_grid(kern, Sh::THREADS, smem, ~0ull);
    const unsigned g = grid < c->tiles.size() ? grid : (unsigned)c->tiles.size();
    const CUtensorMap* maps =
        c->at<CUtensorMap>(c->lay.tmaps) + (size_t)(c->shape - 5) * c->n_sides * kTmaArrays;
    kern<<<g, Sh::THREADS, smem, s>>>(
        c->at<Tile>(c->lay.tiles), c->at<Proto>(c->lay.proto), c->at<int64_t>(c->lay.clock), k_off, first, maps,
        3 * buf, (float*)c->field(buf ^ 1, 0), (float*)c->field(buf ^ 1, 1), (float*)c->field(buf ^ 1, 2), 6 + cbuf,
        cout, c->at<int64_t>(c->lay.fstep), c->at<double>(c->lay.fdose), c->at<double>(c->lay.cum),
        c->at<uint32_t>(c->lay.intents), c->at<uint32_t>(c->lay.icount), c->at<uint32_t>(c->lay.tile_ctr),
        (int)c->tiles.size(), pass, c->P);
}

template <int TX, int TY, int K, int HY, bool EPI>
void launch_tma_t(sim_ctx* c, cudaStream_t s, int k_off, int first, int buf, const uint32_t* cin, uint32_t* cout,
                  int pass) {
    const int cbuf = cin == c->cells(0) ? 0 : 1;
    if ((c->P.flags & (kFDiffusion | kFReaction)) == (kFDiffusion | kFReaction))
        launch_tma_f<TX, TY, K, HY, EPI, true>(c, s, k_off, first, buf, cbuf, cout, pass);
    else
        launch_tma_f<TX, TY, K, HY, EPI, false>(c, s, k_off, first, buf, cbuf, cout, pass);
}

// a pass of four substeps: the deep TMA shapes only
template <bool EPI>
void launch_deep(sim_ctx* c, cudaStream_t s, int k_off, int first, int buf, const uint32_t* cin, uint32_t* cout,
                 int pass) {
    if (c->shape == 7) launch_tma_t<32, 16, 4, 4, EPI>(c, s, k_off, first, buf, cin, cout, pass);
    else launch_tma_t<16, 16, 4, 4, EPI>(c, s, k_off, first, buf, cin, cout, pass);
}

template <typename T, int K, bool EPI>
void launch_fused_k(sim_ctx* c, cudaStream_t s, int k_off, int first, int buf, const uint32_t* cin, uint32_t* cout,
                    int pass) {
    if constexpr (std::is_same<T, float>::value) {  // TMA staging: FP32 storage only
        if (c->shape == 5) return launch_tma_t<32, 16, K, 2, EPI>(c, s, k_off, first, buf, cin, cout, pass);
        if (c->shape == 6) return launch_tma_t<16, 16, K, 2, EPI>(c, s, k_off, first, buf, cin, cout, pass);
        if constexpr (K == 2) {  // the two-substep remainder pass of a deep shape
            if (c->shape == 7) return launch_tma_t<32, 16, 2, 4, EPI>(c, s, k_off, first, buf, cin, cout, pass);
            if (c->shape == 8) return launch_tma_t<16, 16, 2, 4, EPI>(c, s, k_off, first, buf, cin, cout, pass);
        }
    }
    if (c->shape == 3) return launch_fused1_t<T, 32, 16, K, EPI>(c, s, k_off, first, buf, cin, cout, pass);
    if (c->shape == 4) return launch_fused1_t<T, 16, 16, K, EPI>(c, s, k_off, first, buf, cin, cout, pass);
    if (c->shape == 2) launch_fused_t<T, 16, 16, K, EPI>(c, s, k_off, first, buf, cin, cout, pass);
    else launch_fused_t<T, 32, 16, K, EPI>(c, s, k_off, first, buf, cin, cout, pass);
}

// allow the dynamic shared memory of every fused instantiation of type T (done once, outside any capture)
template <typename T, int TX, int TY>
cudaError_t fused_attrs_shape() {
    cudaError_t e = cudaFuncSetAttribute(k_fused<T, TX, TY, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_smem_bytes<T, TX, TY, 1>());
    if (!e)
        e = cudaFuncSetAttribute(k_fused<T, TX, TY, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes<T, TX, TY, 1>());
    if (!e)
        e = cudaFuncSetAttribute(k_fused<T, TX, TY, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes<T, TX, TY, 2>());
    if (!e)
        e = cudaFuncSetAttribute(k_fused<T, TX, TY, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes<T, TX, TY, 2>());
    return e;
}

template <typename T, int TX, int TY, bool FULL>
cudaError_t fused1_attrs_full() {
    cudaError_t e = cudaFuncSetAttribute(fused1_kernel<T, TX, TY, 1, false, FULL>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused1_bytes<T, TX, TY, 1>());
    if (!e)
        e = cudaFuncSetAttribute(fused1_kernel<T, TX, TY, 1, true, FULL>(),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused1_bytes<T, TX, TY, 1>());
    if (!e)
        e = cudaFuncSetAttribute(fused1_kernel<T, TX, TY, 2, false, FULL>(),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused1_bytes<T, TX, TY, 2>());
    if (!e)
        e = cudaFuncSetAttribute(fused1_kernel<T, TX, TY, 2, true, FULL>(),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused1_bytes<T, TX, TY, 2>());
    return e;
}

template <typename T, int TX, int TY>
cudaError_t fused1_attrs_shape() {
    cudaError_t e = fused1_attrs_full<T, TX, TY, true>();
    if (!e) e = fused1_attrs_full<T, TX, TY, false>();
    return e;
}

template <int TX, int TY, int K, int HY, bool FULL>
cudaError_t tma_attrs_k() {
    constexpr int smem = (int)tma_smem_bytes<TX, TY, K, HY>();
    cudaError_t e =
        cudaFuncSetAttribute(k_tma<TX, TY, K, HY, false, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (!e)
        e = cudaFuncSetAttribute(k_tma<TX, TY, K, HY, true, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

// the pass depths a shape runs: 1 and 2 on the two-row halo, 2 and 4 on the deep (four-row) one
template <int TX, int TY, int HY>
cudaError_t tma_attrs_shape() {
    constexpr int K0 = HY > 2 ? 2 : 1, K1 = HY > 2 ? 4 : 2;
    cudaError_t e = tma_attrs_k<TX, TY, K0, HY, true>();
    if (!e) e = tma_attrs_k<TX, TY, K1, HY, true>();
    if (!e) e = tma_attrs_k<TX, TY, K0, HY, false>();
    if (!e) e = tma_attrs_k<TX, TY, K1, HY, false>();
    return e;
}

template <typename T>
cudaError_t fused_attrs() {
    cudaError_t e = fused_attrs_shape<T, 32, 16>();
    if (!e) e = fused_attrs_shape<T, 16, 16>();
    if (!e) e = fused1_attrs_shape<T, 32, 16>();
    if (!e) e = fused1_attrs_shape<T, 16, 16>();
    if constexpr (std::is_same<T, float>::value) {
        if (!e) e = tma_attrs_shape<32, 16, 2>();
        if (!e) e = tma_attrs_shape<16, 16, 2>();
        if (!e) e = tma_attrs_shape<32, 16, 4>();
        if (!e) e = tma_attrs_shape<16, 16, 4>();
    }
    return e;
}

// Tensor maps of the TMA-staged passes: per tile shape (5-8), lattice-side
// class and array (O, G, H of both field buffers, both cell-word buffers), an
// L x L x Z volume over the whole array (Z = planes of L^2 sites it spans) with
// a (TX + 8) x (TY + 2 HY) x 1 box (HY = 2, or 4 on the deep shapes); sites
// outside the volume read as zero.  The
// encoder is the driver's, reached through the runtime so that the library
// links against the runtime only.  False if any map cannot be encoded (the TMA
// shapes are then unavailable).
bool encode_tensor_maps(sim_ctx* c, const std::vector<int32_t>& sides) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)f;
    }();
    if (!encode) return false;
    std::vector<CUtensorMap> maps((size_t)kTmaShapes * sides.size() * kTmaArrays);
    for (int sh = 0; sh < kTmaShapes; ++sh) {
        const int TX = kTileShapes[5 + sh][0], TY = kTileShapes[5 + sh][1];
        for (size_t k = 0; k < sides.size(); ++k) {
            const cuuint64_t Lk = (cuuint64_t)sides[k];
            const cuuint64_t dims[3] = {Lk, Lk, (cuuint64_t)c->total_sites / (Lk * Lk)};
            const cuuint64_t strides[2] = {Lk * 4, Lk * Lk * 4};  // bytes, dimensions 1 and 2
            const cuuint32_t box[3] = {(cuuint32_t)(TX + 2 * kTmaHaloX), (cuuint32_t)(TY + 2 * tma_halo_y(5 + sh)),
                                       1};
            const cuuint32_t estr[3] = {1, 1, 1};
            for (int a = 0; a < kTmaArrays; ++a) {
                void* base = a < 6 ? c->field(a / 3, a % 3) : (void*)c->cells(a - 6);
                const CUtensorMapDataType dt =
                    a < 6 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
                CUtensorMap* m = &maps[((size_t)sh * sides.size() + k) * kTmaArrays + a];
                if (encode(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    return false;
            }
        }
    }
    cudaError_t e = cudaMemcpyAsync(c->ws + c->lay.tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);  // the staging vector dies with this call
    return e == cudaSuccess;
}

template <typename T>
void launch_fused(sim_ctx* c, cudaStream_t s, int k_off, int K, bool epi, int first, int buf, const uint32_t* cin,
                  uint32_t* cout, int pass) {
    if (K == 1) {
        if (epi) launch_fused_k<T, 1, true>(c, s, k_off, first, buf, cin, cout, pass);
        else launch_fused_k<T, 1, false>(c, s, k_off, first, buf, cin, cout, pass);
    } else if (K == 4) {
        if (epi) launch_deep<true>(c, s, k_off, first, buf, cin, cout, pass);
        else launch_deep<false>(c, s, k_off, first, buf, cin, cout, pass);
    } else {
        if (epi) launch_fused_k<T, 2, true>(c, s, k_off, first, buf, cin, cout, pass);
        else launch_fused_k<T, 2, false>(c, s, k_off, first, buf, cin, cout, pass);
    }
}

// Events (profiling): ev[0] start, ev[1] after the reaction-diffusion work
// without the cell update, ev[2] after the cell update (last fused pass or
// k_cell), ev[3] after the claims, ev[4] after the resolution.
template <typename T>
sim_status enqueue_step(sim_ctx* c, cudaStream_t s, int k_off, int start_buf, int start_cell,
                        cudaEvent_t* ev = nullptr) {
    const unsigned nb = (unsigned)c->blocks.size();
    const Block* blocks = c->at<Block>(c->lay.blocks);
    const Proto* protos = c->at<Proto>(c->lay.proto);
    const int64_t* clock = c->at<int64_t>(c->lay.clock);
    const unsigned ng = 148 * 4;  // the division work list is short: a fixed grid strides over it
    if (c->fused()) {
        int buf = start_buf;
        const int np = c->passes();
        if (ev) cudaEventRecord(ev[0], s);
        for (int j = 0; j < np; ++j) {
            const bool epi = j == np - 1;
            if (epi && ev) cudaEventRecord(ev[1], s);
            uint32_t* cout = epi ? c->cells(start_cell ^ 1) : c->cells(start_cell);
            launch_fused<T>(c, s, k_off, c->pass_k(j), epi, j == 0, buf, c->cells(start_cell), cout, j);
            buf ^= 1;
        }
        if (ev) cudaEventRecord(ev[2], s);
        uint32_t* cell = c->cells(start_cell ^ 1);
        k_claim<<<ng, kThreads, 0, s>>>(protos, c->n, clock, k_off, cell, c->at<uint32_t>(c->lay.intents),
                                        c->at<uint32_t>(c->lay.icount), c->at<uint32_t>(c->lay.target),
                                        c->at<unsigned long long>(c->lay.claim), c->P);
        if (ev) cudaEventRecord(ev[3], s);
        k_resolve<<<ng, kThreads, 0, s>>>(protos, c->n, clock, k_off, cell, c->at<uint32_t>(c->lay.intents),
                                          c->at<uint32_t>(c->lay.icount), c->at<uint32_t>(c->lay.target),
                                          c->at<unsigned long long>(c->lay.claim), c->at<uint32_t>(c->lay.tile_ctr),
                                          c->passes(), kMaxPasses, c->P);
        if (ev) cudaEventRecord(ev[4], s);
        return cuda_check(c, cudaGetLastError(), "step launch");
    }
    uint32_t* cell = c->cells(start_cell);
    int buf = start_buf;
    if (ev) cudaEventRecord(ev[0], s);
    for (int sub = 0; sub < c->P.n_sub; ++sub) {
        k_substep<T><<<nb, kThreads, 0, s>>>(blocks, protos, clock, k_off, sub, (const T*)c->field(buf, 0),
                                             (const T*)c->field(buf, 1), (const T*)c->field(buf, 2),
                                             (T*)c->field(buf ^ 1, 0), (T*)c->field(buf ^ 1, 1),
                                             (T*)c->field(buf ^ 1, 2), cell, c->at<int64_t>(c->lay.fstep),
                                             c->at<double>(c->lay.fdose), c->at<double>(c->lay.cum), c->P);
        buf ^= 1;
    }
    if (ev) cudaEventRecord(ev[1], s);
    k_cell<T><<<nb, kThreads, 0, s>>>(blocks, protos, clock, k_off, (const T*)c->field(buf, 0),
                                      (const T*)c->field(buf, 1), (const T*)c->field(buf, 2), cell,
                                      c->at<uint32_t>(c->lay.intents), c->at<uint32_t>(c->lay.icount), c->P);
    if (ev) cudaEventRecord(ev[2], s);
    k_claim<<<ng, kThreads, 0, s>>>(protos, c->n, clock, k_off, cell, c->at<uint32_t>(c->lay.intents),
                                    c->at<uint32_t>(c->lay.icount), c->at<uint32_t>(c->lay.target),
                                    c->at<unsigned long long>(c->lay.claim), c->P);
    if (ev) cudaEventRecord(ev[3], s);
    k_resolve<<<ng, kThreads, 0, s>>>(protos, c->n, clock, k_off, cell, c->at<uint32_t>(c->lay.intents),
                                      c->at<uint32_t>(c->lay.icount), c->at<uint32_t>(c->lay.target),
                                      c->at<unsigned long long>(c->lay.claim), nullptr, 0, kMaxPasses, c->P);
    if (ev) cudaEventRecord(ev[4], s);
    return cuda_check(c, cudaGetLastError(), "step launch");
}

sim_status step_dispatch(sim_ctx* c, cudaStream_t s, int k_off, int start_buf, int start_cell,
                         cudaEvent_t* ev = nullptr) {
    switch (c->cfg.precision) {
        case SIM_BF16: return enqueue_step<__nv_bfloat16>(c, s, k_off, start_buf, start_cell, ev);
        case SIM_FP16: return enqueue_step<__half>(c, s, k_off, start_buf, start_cell, ev);
        default: return enqueue_step<float>(c, s, k_off, start_buf, start_cell, ev);
    }
}

// advance the host mirror of the buffer parities by `steps` steps
void advance(sim_ctx* c, int64_t steps) {
    c->clock += steps;
    c->cur ^= (int)((steps * c->field_flips()) & 1);
    c->ccur ^= (int)((steps * c->cell_flips()) & 1);
}

sim_status tick(sim_ctx* c, cudaStream_t s, int64_t by) {
    k_tick<<<1, 1, 0, s>>>(c->at<int64_t>(c->lay.clock), by);
    return cuda_check(c, cudaGetLastError(), "k_tick launch");
}

sim_status count_hour(sim_ctx* c) {
    const int64_t h = c->clock / kStepsPerHour;
    if (c->clock % kStepsPerHour != 0 || h > c->cfg.hours || h <= c->counted_hour) return SIM_OK;
    k_count<<<(unsigned)c->blocks.size(), kThreads, 0, c->stream>>>(
        c->at<Block>(c->lay.blocks), c->at<Proto>(c->lay.proto), c->at<int64_t>(c->lay.clock),
        c->cells(c->ccur), c->at<int32_t>(c->lay.counts), c->cfg.hours + 1, 1);
    c->counted_hour = h;
    return cuda_check(c, cudaGetLastError(), "k_count launch");
}

// Capture one simulated hour (600 steps + clock advance) starting from field
// buffer `start` as a CUDA graph.  Captured on a private stream; replayed on
// the context's stream.
sim_status build_hour_graph(sim_ctx* c, int start, int cstart) {
    const int key = start * 2 + cstart;
    if (c->hour_graph[key]) return SIM_OK;
    cudaError_t e = cudaSuccess;
    if (!c->capture_stream) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e) return cuda_check(c, e, "capture stream");
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e) return cuda_check(c, e, "begin capture");
    int buf = start, cb = cstart;
    sim_status st = SIM_OK;
    for (int k = 0; k < kStepsPerHour && st == SIM_OK; ++k) {
        st = step_dispatch(c, c->capture_stream, k, buf, cb);
        buf ^= (c->field_flips() & 1);
        cb ^= (c->cell_flips() & 1);
    }
    if (st == SIM_OK) st = tick(c, c->capture_stream, kStepsPerHour);
    e = cudaStreamEndCapture(c->capture_stream, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e) return cuda_check(c, e, "end capture");
    e = cudaGraphInstantiate(&c->hour_graph[key], g, 0);
    cudaGraphDestroy(g);
    return cuda_check(c, e, "graph instantiate");
}

void drop_graphs(sim_ctx* c) {
    for (auto& g : c->hour_graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

int64_t max_t_end(const sim_ctx* c) {
    int64_t m = 0;
    for (const Proto& p : c->proto) m = p.t_end > m ? p.t_end : m;
    return m;
}

sim_status read_status(sim_ctx* c) {
    uint32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c->ws + c->lay.status, sizeof st, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_check(c, e, "synchronise");
    if (st & kStatusBounds)
        return fail(c, SIM_ECUDA, "index check failed: a kernel addressed a site outside the batch (SIM_CHECK build)");
    if (st & kStatusBadProtocol)
        return fail(c, SIM_EINVAL,
                    "a protocol loaded from device dose vectors exceeds max_fractions or the dose cap "
                    "(it was run without fractions)");
    if (st) return fail(c, SIM_ETIMEOUT, "device reported status " + std::to_string(st));
    return SIM_OK;
}

template <typename T>
void to_float(const void* src, float* dst, int64_t n) {
    const T* s = (const T*)src;
    for (int64_t i = 0; i < n; ++i) dst[i] = (float)s[i];
}

struct CkptHeader {
    char magic[8];
    int32_t n, precision;
    int64_t total_sites, clock, counted_hour;
    int32_t cur, hours;
};

size_t ckpt_bytes(const sim_ctx* c) {
    const size_t es = elem_size(c->cfg.precision);
    const size_t ncnt = (size_t)c->n * (c->cfg.hours + 1);
    return sizeof(CkptHeader) + 3 * es * c->total_sites + 4 * c->total_sites + 8 * c->n + 4 * ncnt;
}

}  // namespace

namespace {

template <typename T>
void launch_totals(sim_ctx* c) {
    k_totals_part<T><<<(unsigned)c->blocks.size(), kThreads, 0, c->stream>>>(
        c->at<Block>(c->lay.blocks), c->at<Proto>(c->lay.proto), (const T*)c->field(c->cur, 0),
        (const T*)c->field(c->cur, 1), (const T*)c->field(c->cur, 2), c->at<double>(c->lay.part64),
        c->at<float>(c->lay.part32));
}

// Switch the fused work list to tile shape `sh` (rebuilds and uploads the tiles; drops captured graphs).
sim_status set_shape(sim_ctx* c, int sh, const std::vector<int32_t>& L) {
    c->shape = sh;
    c->tiles = make_tiles(c->cfg, c->n, L.data(), sh, c->tile_live.data(), c->fine_z);
    drop_graphs(c);
    cudaError_t e = cudaMemcpyAsync(c->ws + c->lay.tiles, c->tiles.data(), sizeof(Tile) * c->tiles.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.tile_ctr, 0, sizeof(uint32_t) * 2 * kMaxPasses, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "set shape");
}

// At an hour boundary, drop protocols that have reached their horizon from the
// fused work list: their tiles would only be skipped, and once the survivors'
// columns no longer fill the GPU make_tiles splits them in z again.
sim_status refresh_tiles(sim_ctx* c) {
    if (!c->fused() || !c->loaded) return SIM_OK;
    std::vector<uint8_t> live(c->n);
    bool any = false;
    for (int p = 0; p < c->n; ++p) any |= (live[p] = c->proto[p].t_end > c->clock) != 0;
    if (!any || live == c->tile_live) return SIM_OK;
    c->tile_live = live;
    std::vector<int32_t> L(c->n);
    for (int p = 0; p < c->n; ++p) L[p] = c->proto[p].L;
    return set_shape(c, c->shape, L);
}

}  // namespace

extern "C" {

const char* sim_status_string(sim_status s) {
    switch (s) {
        case SIM_OK: return "ok";
        case SIM_EINVAL: return "invalid argument";
        case SIM_ENOSPC: return "buffer too small";
        case SIM_ECUDA: return "CUDA error";
        case SIM_ETIMEOUT: return "device wait timed out";
        case SIM_ESTATE: return "invalid state";
    }
    return "unknown status";
}

const char* sim_last_error(const sim_ctx* c) { return c ? c->err.c_str() : "null context"; }

sim_status sim_workspace_size(const sim_config* cfg, int n, const int32_t* L, size_t* bytes) {
    if (!cfg || !L || !bytes || n < 1) return SIM_EINVAL;
    std::string why;
    if (!valid_config(cfg, &why)) return SIM_EINVAL;
    int64_t nb = 0;
    for (int p = 0; p < n; ++p) {
        if (L[p] < 8 || L[p] > kMaxL) return SIM_EINVAL;
        if (cfg->z_chunk > 0 && cfg->z_chunk > L[p]) return SIM_EINVAL;
        const int64_t sites = (int64_t)L[p] * L[p] * L[p];
        nb += (sites + kSitesPerBlock - 1) / kSitesPerBlock;
    }
    const int64_t total = place_protocols(n, L, nullptr);
    if (total >= (int64_t)0xffffffffLL) return SIM_EINVAL;  // work list holds 32-bit site indices
    int64_t nt = 0;  // room for the work list of any shape and z split the autotuner may pick
    for (int sh = 1; sh <= kNumShapes; ++sh)
        for (int fz : {0, kFineZ}) {
            const int64_t t = (int64_t)make_tiles(*cfg, n, L, sh, nullptr, fz).size();
            nt = t > nt ? t : nt;
        }
    *bytes = make_layout(*cfg, n, total, nb, nt, side_classes(n, L)).total;
    return SIM_OK;
}

sim_status sim_create(const sim_config* cfg, int n, const int32_t* L, const int32_t* R, void* d_workspace,
                      size_t bytes, void* cuda_stream, sim_ctx** out) {
    if (!out) return SIM_EINVAL;
    *out = nullptr;
    if (!cfg || !L || !R || !d_workspace || n < 1) return SIM_EINVAL;
    if (((uintptr_t)d_workspace) % kAlign) return SIM_EINVAL;
    size_t need = 0;
    if (sim_workspace_size(cfg, n, L, &need) != SIM_OK) return SIM_EINVAL;
    if (bytes < need) return SIM_ENOSPC;
    sim_ctx* c = new sim_ctx();
    c->cfg = *cfg;
    c->n = n;
    c->P = make_params(*cfg);
    c->P.frac_cap = n * cfg->max_fractions;
    c->ws = (char*)d_workspace;
    c->stream = (cudaStream_t)cuda_stream;
    std::vector<int64_t> first_site(n);
    const int64_t site0 = place_protocols(n, L, first_site.data());
    std::vector<int32_t> sides(L, L + n);  // tensor-map classes: the distinct sides in ascending order
    std::sort(sides.begin(), sides.end());
    sides.erase(std::unique(sides.begin(), sides.end()), sides.end());
    c->n_sides = (int)sides.size();
    for (int p = 0; p < n; ++p) {
        Proto pr{};
        pr.L = L[p];
        pr.R = R[p];
        pr.site0 = first_site[p];
        pr.t_end = 0;
        pr.frac0 = p * cfg->max_fractions;
        pr.nfrac = 0;
        pr.tmap = (int32_t)(std::lower_bound(sides.begin(), sides.end(), L[p]) - sides.begin());
        const int64_t sites = (int64_t)L[p] * L[p] * L[p];
        for (int64_t b = 0; b < sites; b += kSitesPerBlock) {
            Block bl{};
            bl.p = p;
            bl.begin = b;
            bl.n = (int)((sites - b) < kSitesPerBlock ? (sites - b) : kSitesPerBlock);
            c->blocks.push_back(bl);
        }
        c->proto.push_back(pr);
    }
    c->total_sites = site0;
    c->shape = pick_shape(*cfg, n, L);
    for (int p = 0; p < n; ++p)
        if (L[p] % 2) c->vec_ok = 0;
    // 2-byte storage is staged in shared memory as aligned element pairs, which needs even lattice sides and
    // passes of two substeps: other cases take the substep path
    if (c->cfg.path == SIM_PATH_FUSED && c->cfg.precision != SIM_FP32 && (!c->vec_ok || (c->P.n_sub & 1)))
        c->cfg.path = SIM_PATH_SUBSTEP;
    if (c->cfg.path == SIM_PATH_FUSED) {
        cudaError_t ea = c->cfg.precision == SIM_BF16   ? fused_attrs<__nv_bfloat16>()
                         : c->cfg.precision == SIM_FP16 ? fused_attrs<__half>()
                                                        : fused_attrs<float>();
        if (ea) {
            delete c;
            return SIM_ECUDA;
        }
    }
    c->tiles = make_tiles(*cfg, n, L, c->shape);
    c->tile_live.assign(n, 1);
    int64_t nt = 0;
    for (int sh = 1; sh <= kNumShapes; ++sh)
        for (int fz : {0, kFineZ}) {
            const int64_t t = (int64_t)make_tiles(*cfg, n, L, sh, nullptr, fz).size();
            nt = t > nt ? t : nt;
        }
    c->lay = make_layout(*cfg, n, site0, (int64_t)c->blocks.size(), nt, c->n_sides);
    c->P.n_sites = (uint64_t)site0;
    c->P.status = c->at<uint32_t>(c->lay.status);
    std::vector<int32_t> first_block(n + 1, 0);
    for (size_t b = 0; b < c->blocks.size(); ++b) first_block[c->blocks[b].p + 1] = (int32_t)(b + 1);
    cudaError_t e = cudaMemcpyAsync(c->ws + c->lay.blocks, c->blocks.data(), sizeof(Block) * c->blocks.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (!e)
        e = cudaMemcpyAsync(c->ws + c->lay.first_block, first_block.data(), sizeof(int32_t) * (n + 1),
                            cudaMemcpyHostToDevice, c->stream);
    if (!e)
        e = cudaMemcpyAsync(c->ws + c->lay.tiles, c->tiles.data(), sizeof(Tile) * c->tiles.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (!e)
        e = cudaMemcpyAsync(c->ws + c->lay.proto, c->proto.data(), sizeof(Proto) * n, cudaMemcpyHostToDevice,
                            c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);  // host vectors may change before the copy would run
    sim_status st = cuda_check(c, e, "create copies");
    // TMA-staged shapes: FP32 storage on the fused path, every side a multiple of 4 (16-byte row strides)
    bool tma_fit = c->cfg.path == SIM_PATH_FUSED && c->cfg.precision == SIM_FP32;
    for (int p = 0; p < n; ++p) tma_fit = tma_fit && L[p] % 4 == 0;
    if (!st && tma_fit) c->tma_ok = encode_tensor_maps(c, sides);
    // without the autotuner a 16 x 16 one-column context runs the TMA-staged kernel of the same tiles
    if (!st && cfg->tile_shape == 0 && c->tma_ok && c->shape == 4) c->shape = 6;
    if (!st && c->cfg.path == SIM_PATH_FUSED && tma_shape(c->shape) && !c->tma_ok)
        st = fail(c, SIM_EINVAL, "tile shapes 5-8 need FP32 storage and lattice sides that are multiples of 4");
    if (!st && c->cfg.path == SIM_PATH_FUSED && deep_shape(c->shape) && (c->P.n_sub & 1))
        st = fail(c, SIM_EINVAL, "tile shapes 7 and 8 run passes of four and two substeps: n_sub must be even");
    if (!st) st = reset_device(c);
    if (st) {
        delete c;
        return st;
    }
    *out = c;
    return SIM_OK;
}

sim_status sim_load_protocols(sim_ctx* c, int n, const int32_t* offsets, const double* dose_gy,
                              const double* wait_h) {
    if (!c) return SIM_EINVAL;
    if (n != c->n || !offsets) return fail(c, SIM_EINVAL, "protocol count must equal the context's slots");
    if (offsets[0] != 0) return fail(c, SIM_EINVAL, "offsets[0] must be 0");
    const int F = c->cfg.max_fractions;
    const size_t cap = (size_t)n * (F > 0 ? F : 1);
    std::vector<int64_t> fstep(cap, -1);
    std::vector<double> fdose(2 * cap, 0.0);  // doses, then their quadratic partners
    std::vector<Proto> proto = c->proto;
    for (int p = 0; p < n; ++p) {
        const int a = offsets[p], b = offsets[p + 1];
        if (b < a) return fail(c, SIM_EINVAL, "offsets must be non-decreasing");
        if ((a != b) && (!dose_gy || !wait_h)) return fail(c, SIM_EINVAL, "dose/wait arrays missing");
        double t_h = 0.0, total = 0.0;
        int nf = 0;
        int64_t last = -1;
        for (int j = a; j < b; ++j) {
            const double d = dose_gy[j], w = wait_h[j];
            if (!std::isfinite(d) || !std::isfinite(w) || d < 0.0 || w < 0.0)
                return fail(c, SIM_EINVAL, "protocol " + std::to_string(p) + ": negative or non-finite dose/wait");
            if (std::fabs(w * 2.0 - std::round(w * 2.0)) > 1e-9)
                return fail(c, SIM_EINVAL, "protocol " + std::to_string(p) + ": wait not on the 30 min grid");
            t_h += w;
            total += d;
            const int64_t st = llround(kStepsPerHour * t_h);
            last = st;
            if (d == 0.0) continue;
            if (nf > 0 && fstep[(size_t)p * F + nf - 1] == st) {  // fractions on one step add up
                fdose[(size_t)p * F + nf - 1] += d;
                continue;
            }
            if (nf >= F) return fail(c, SIM_EINVAL, "protocol " + std::to_string(p) + ": too many fractions");
            fstep[(size_t)p * F + nf] = st;
            fdose[(size_t)p * F + nf] = d;
            ++nf;
        }
        if (total > c->cfg.dose_cap_gy + 1e-9)
            return fail(c, SIM_EINVAL, "protocol " + std::to_string(p) + ": total dose above the cap");
        // quadratic partner of each fraction: D_j + 2 sum_{i<j} D_i 2^(-(t_j - t_i) / T_half) under
        // incomplete repair, D_j alone when repair completes between fractions
        const double th = c->cfg.params.repair_half_h;
        for (int j = 0; j < nf; ++j) {
            const size_t at = (size_t)p * F + j;
            double h = 0.0;
            for (int i = 0; th > 0.0 && i < j; ++i) {
                const double dt_h = (double)(fstep[at] - fstep[(size_t)p * F + i]) / kStepsPerHour;
                h += fdose[(size_t)p * F + i] * std::exp2(-dt_h / th);
            }
            fdose[cap + at] = fdose[at] + 2.0 * h;
        }
        proto[p].nfrac = nf;
        proto[p].t_end = c->cfg.t_end_steps > 0
                             ? c->cfg.t_end_steps
                             : (last > 0 ? last : 0) + (int64_t)kStepsPerHour * c->cfg.regrowth_h;
    }
    cudaError_t e = cudaSuccess;
    if (F > 0) {
        e = cudaMemcpyAsync(c->ws + c->lay.fstep, fstep.data(), sizeof(int64_t) * cap, cudaMemcpyHostToDevice,
                            c->stream);
        if (!e)
            e = cudaMemcpyAsync(c->ws + c->lay.fdose, fdose.data(), sizeof(double) * 2 * cap,
                                cudaMemcpyHostToDevice, c->stream);
    }
    if (!e)
        e = cudaMemcpyAsync(c->ws + c->lay.proto, proto.data(), sizeof(Proto) * n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);  // the staging vectors die with this call
    if (e) return cuda_check(c, e, "load protocols");
    c->proto = proto;
    c->loaded = true;
    return reset_device(c);
}

sim_status sim_load_dose_vectors(sim_ctx* c, const uint8_t* d_units, int n_slots, double unit_gy) {
    if (!c) return SIM_EINVAL;
    if (!d_units || n_slots < 1 || n_slots > (1 << 20) || !std::isfinite(unit_gy) || unit_gy <= 0.0)
        return fail(c, SIM_EINVAL, "dose vectors: need a device pointer, 1..2^20 slots and a positive unit");
    if (c->cfg.t_end_steps <= 0)
        return fail(c, SIM_ESTATE, "dose vectors loaded on the device need a fixed horizon (t_end_steps > 0)");
    if (c->cfg.max_fractions < 1) return fail(c, SIM_ESTATE, "max_fractions must be >= 1");
    for (Proto& pr : c->proto) {
        pr.t_end = c->cfg.t_end_steps;
        pr.nfrac = 0;  // known on the device only
    }
    c->loaded = true;
    sim_status st = reset_device(c);  // clears the status word before the loader may set it
    if (st) return st;
    k_load_vectors<<<(unsigned)((c->n * 32 + 255) / 256), 256, 0, c->stream>>>(
        d_units, n_slots, unit_gy, c->n, c->at<Proto>(c->lay.proto), c->at<int64_t>(c->lay.fstep),
        c->at<double>(c->lay.fdose), c->cfg.max_fractions, c->P.frac_cap, c->cfg.dose_cap_gy,
        c->cfg.params.repair_half_h, c->cfg.t_end_steps, c->at<uint32_t>(c->lay.status));
    return cuda_check(c, cudaGetLastError(), "k_load_vectors launch");
}

sim_status sim_fitness_device(sim_ctx* c, int32_t* d_count, float* d_fitness) {
    if (!c) return SIM_EINVAL;
    cudaError_t e = cudaMemsetAsync(c->ws + c->lay.final_count, 0, sizeof(int32_t) * c->n, c->stream);
    if (e) return cuda_check(c, e, "fitness memset");
    k_count<<<(unsigned)c->blocks.size(), kThreads, 0, c->stream>>>(
        c->at<Block>(c->lay.blocks), c->at<Proto>(c->lay.proto), c->at<int64_t>(c->lay.clock),
        c->cells(c->ccur), c->at<int32_t>(c->lay.final_count), 1, 0);
    if (sim_status st = cuda_check(c, cudaGetLastError(), "k_count launch")) return st;
    k_fitness_out<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(
        c->at<int32_t>(c->lay.final_count), c->n, (float)c->cfg.n_max_fitness, d_count, d_fitness);
    return cuda_check(c, cudaGetLastError(), "k_fitness_out launch");
}

sim_status sim_reset(sim_ctx* c) {
    if (!c) return SIM_EINVAL;
    return reset_device(c);
}

// NVTX range for the duration of a host call (visible in Nsight timelines)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

sim_status sim_run(sim_ctx* c, int64_t max_steps) {
    if (!c) return SIM_EINVAL;
    if (!c->loaded) return fail(c, SIM_ESTATE, "load protocols before running");
    NvtxRange nvtx("sim_run");
    int64_t target = max_t_end(c);
    if (max_steps > 0 && c->clock + max_steps < target) target = c->clock + max_steps;
    const bool graphs = c->cfg.use_graphs != 0;
    sim_status st = SIM_OK;
    while (c->clock < target && st == SIM_OK) {
        st = count_hour(c);
        if (!st && c->clock % kStepsPerHour == 0) st = refresh_tiles(c);
        if (st) break;
        if (graphs && c->clock % kStepsPerHour == 0 && c->clock + kStepsPerHour <= target) {
            st = build_hour_graph(c, c->cur, c->ccur);
            if (st) break;
            cudaError_t e = cudaGraphLaunch(c->hour_graph[c->cur * 2 + c->ccur], c->stream);
            if (e) return cuda_check(c, e, "graph launch");
            advance(c, kStepsPerHour);
        } else {
            st = step_dispatch(c, c->stream, 0, c->cur, c->ccur);
            if (!st) st = tick(c, c->stream, 1);
            advance(c, 1);
        }
    }
    if (!st) st = count_hour(c);
    return st;
}

sim_status sim_profile_steps(sim_ctx* c, int n_steps, double* ms, int64_t* launches) {
    if (!c || !ms || n_steps < 0) return SIM_EINVAL;
    if (!c->loaded) return fail(c, SIM_ESTATE, "load protocols before running");
    for (int k = 0; k < 4; ++k) {
        ms[k] = 0.0;
        if (launches) launches[k] = 0;
    }
    cudaEvent_t ev[5];
    for (int k = 0; k < 5; ++k)
        if (cudaError_t e = cudaEventCreate(&ev[k])) return cuda_check(c, e, "event create");
    sim_status st = SIM_OK;
    for (int i = 0; i < n_steps && st == SIM_OK; ++i) {
        st = count_hour(c);
        if (!st) st = step_dispatch(c, c->stream, 0, c->cur, c->ccur, ev);
        if (!st) st = tick(c, c->stream, 1);
        if (st) break;
        advance(c, 1);
        cudaError_t e = cudaEventSynchronize(ev[4]);
        if (e) {
            st = cuda_check(c, e, "event sync");
            break;
        }
        for (int k = 0; k < 4; ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            ms[k] += t;
        }
        if (launches) {
            launches[0] += c->fused() ? c->passes() - 1 : c->P.n_sub;
            launches[1] += 1;
            launches[2] += 1;
            launches[3] += 1;
        }
    }
    for (int k = 0; k < 5; ++k) cudaEventDestroy(ev[k]);
    if (!st) st = count_hour(c);
    if (!st) st = read_status(c);
    return st;
}

sim_status sim_autotune(sim_ctx* c, int n_steps, int* best, double* ms) {
    if (!c || n_steps < 1) return SIM_EINVAL;
    NvtxRange nvtx("sim_autotune");
    if (!c->loaded) return fail(c, SIM_ESTATE, "load protocols before autotuning");
    for (int k = 0; k < kNumShapes; ++k)
        if (ms) ms[k] = -1.0;
    if (!c->fused()) {
        if (best) *best = 0;
        return reset_device(c);
    }
    std::vector<int32_t> L(c->n);
    for (int p = 0; p < c->n; ++p) L[p] = c->proto[p].L;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) || cudaEventCreate(&b)) return fail(c, SIM_ECUDA, "event create");
    double best_ms = -1.0;
    int pick = c->shape, pick_z = 0;
    sim_status st = SIM_OK;
    // every applicable shape; on a batch split in z to fill the GPU, each shape also with the finer split
    // (shorter z ranges per CTA: more halo work, less latency per pass)
    for (int sh = 1; sh <= kNumShapes && st == SIM_OK; ++sh)
        for (int fz : {0, kFineZ}) {
            if (tma_shape(sh) && !c->tma_ok) continue;
            if (deep_shape(sh) && (c->P.n_sub & 1)) continue;
            if (fz && !z_split_applies(c->cfg, c->n, L.data(), sh)) continue;
            c->fine_z = fz;
            st = set_shape(c, sh, L);
            // one untimed step (first touch), then n_steps timed plain steps
            for (int i = 0; i <= n_steps && st == SIM_OK; ++i) {
                if (i == 1) cudaEventRecord(a, c->stream);
                st = step_dispatch(c, c->stream, 0, c->cur, c->ccur);
                if (!st) st = tick(c, c->stream, 1);
                advance(c, 1);
            }
            if (st) break;
            cudaEventRecord(b, c->stream);
            cudaError_t e = cudaEventSynchronize(b);
            if (e) {
                st = cuda_check(c, e, "autotune sync");
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, a, b);
            if (ms && (ms[sh - 1] < 0 || t / n_steps < ms[sh - 1])) ms[sh - 1] = t / n_steps;
            if (best_ms < 0 || t < best_ms) best_ms = t, pick = sh, pick_z = fz;
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    c->fine_z = pick_z;
    st = set_shape(c, pick, L);
    if (best) *best = pick;
    if (!st) st = reset_device(c);  // the timing steps advanced the batch: start it again from step 0
    if (!st) st = read_status(c);
    return st;
}

sim_status sim_field_totals(sim_ctx* c, double* out64, float* out32) {
    if (!c) return SIM_EINVAL;
    switch (c->cfg.precision) {
        case SIM_BF16: launch_totals<__nv_bfloat16>(c); break;
        case SIM_FP16: launch_totals<__half>(c); break;
        default: launch_totals<float>(c); break;
    }
    k_totals_finish<<<(3 * c->n + 127) / 128, 128, 0, c->stream>>>(
        c->at<int32_t>(c->lay.first_block), c->n, c->at<double>(c->lay.part64), c->at<float>(c->lay.part32),
        c->at<double>(c->lay.tot64), c->at<float>(c->lay.tot32));
    if (sim_status st = cuda_check(c, cudaGetLastError(), "totals launch")) return st;
    cudaError_t e = cudaSuccess;
    if (out64) e = cudaMemcpyAsync(out64, c->ws + c->lay.tot64, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost,
                                   c->stream);
    if (!e && out32)
        e = cudaMemcpyAsync(out32, c->ws + c->lay.tot32, sizeof(float) * 3 * c->n, cudaMemcpyDeviceToHost, c->stream);
    if (e) return cuda_check(c, e, "totals copy");
    return read_status(c);
}

sim_status sim_fitness(sim_ctx* c, int32_t* out_count, double* out_fitness) {
    if (!c) return SIM_EINVAL;
    cudaError_t e = cudaMemsetAsync(c->ws + c->lay.final_count, 0, sizeof(int32_t) * c->n, c->stream);
    if (e) return cuda_check(c, e, "fitness memset");
    k_count<<<(unsigned)c->blocks.size(), kThreads, 0, c->stream>>>(
        c->at<Block>(c->lay.blocks), c->at<Proto>(c->lay.proto), c->at<int64_t>(c->lay.clock),
        c->cells(c->ccur), c->at<int32_t>(c->lay.final_count), 1, 0);
    if (sim_status st = cuda_check(c, cudaGetLastError(), "k_count launch")) return st;
    std::vector<int32_t> cnt(c->n);
    e = cudaMemcpyAsync(cnt.data(), c->ws + c->lay.final_count, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost,
                        c->stream);
    if (e) return cuda_check(c, e, "fitness copy");
    if (sim_status st = read_status(c)) return st;
    for (int p = 0; p < c->n; ++p) {
        if (out_count) out_count[p] = cnt[p];
        if (out_fitness) out_fitness[p] = c->cfg.n_max_fitness - (double)cnt[p];
    }
    return SIM_OK;
}

sim_status sim_counts(sim_ctx* c, int32_t* out, int hours) {
    if (!c || !out) return SIM_EINVAL;
    if (hours != c->cfg.hours) return fail(c, SIM_EINVAL, "hours must equal the configured count length");
    const size_t n = (size_t)c->n * (hours + 1);
    cudaError_t e =
        cudaMemcpyAsync(out, c->ws + c->lay.counts, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e) return cuda_check(c, e, "counts copy");
    if (sim_status st = read_status(c)) return st;
    for (int p = 0; p < c->n; ++p) {
        const int64_t last = c->proto[p].t_end < c->clock ? c->proto[p].t_end : c->clock;
        for (int h = 0; h <= hours; ++h)
            if ((int64_t)h * kStepsPerHour > last || h > c->counted_hour) out[(size_t)p * (hours + 1) + h] = -1;
    }
    return SIM_OK;
}

sim_status sim_delivered_dose(sim_ctx* c, double* out) {
    if (!c || !out) return SIM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(out, c->ws + c->lay.cum, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream);
    if (e) return cuda_check(c, e, "dose copy");
    return read_status(c);
}

sim_status sim_clock(sim_ctx* c, int64_t* step, int64_t* t_end) {
    if (!c) return SIM_EINVAL;
    for (int p = 0; p < c->n; ++p) {
        if (step) step[p] = c->clock < c->proto[p].t_end ? c->clock : c->proto[p].t_end;
        if (t_end) t_end[p] = c->proto[p].t_end;
    }
    return SIM_OK;
}

sim_status sim_set_clock(sim_ctx* c, int64_t step) {
    if (!c || step < 0 || step >= (int64_t)0xffffffffLL) return SIM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(c->ws + c->lay.clock, &step, sizeof step, cudaMemcpyHostToDevice, c->stream);
    // stale claims carry step tags that could outrank the new clock: clear them with the work-list counters
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.claim, 0, 8 * (size_t)c->total_sites, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.icount, 0, 8, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.tile_ctr, 0, sizeof(uint32_t) * 2 * kMaxPasses, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_check(c, e, "set clock");
    c->clock = step;
    c->counted_hour = step / kStepsPerHour - (step % kStepsPerHour == 0 ? 1 : 0);
    return SIM_OK;
}

sim_status sim_get_state(sim_ctx* c, int p, float* O, float* G, float* H, uint32_t* cell) {
    if (!c || p < 0 || p >= c->n) return SIM_EINVAL;
    const Proto& pr = c->proto[p];
    const int64_t n = (int64_t)pr.L * pr.L * pr.L;
    const size_t es = elem_size(c->cfg.precision);
    std::vector<char> tmp((size_t)(n * es));
    float* dst[3] = {O, G, H};
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 3 && !e; ++f) {
        if (!dst[f]) continue;
        e = cudaMemcpyAsync(tmp.data(), (char*)c->field(c->cur, f) + pr.site0 * es, n * es, cudaMemcpyDeviceToHost,
                            c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) break;
        if (c->cfg.precision == SIM_FP32) std::memcpy(dst[f], tmp.data(), n * 4);
        else if (c->cfg.precision == SIM_BF16) to_float<__nv_bfloat16>(tmp.data(), dst[f], n);
        else to_float<__half>(tmp.data(), dst[f], n);
    }
    if (!e && cell)
        e = cudaMemcpyAsync(cell, c->cells(c->ccur) + pr.site0, n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_check(c, e, "get state");
    return read_status(c);
}

sim_status sim_copy_lattice(sim_ctx* dst, int pd, const sim_ctx* src, int ps) {
    if (!dst || !src || pd < 0 || pd >= dst->n || ps < 0 || ps >= src->n) return SIM_EINVAL;
    const Proto& a = dst->proto[pd];
    const Proto& b = src->proto[ps];
    if (a.L != b.L || dst->cfg.precision != src->cfg.precision)
        return fail(dst, SIM_EINVAL, "lattice side or precision differ");
    const int64_t n = (int64_t)a.L * a.L * a.L;
    const size_t es = elem_size(dst->cfg.precision);
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 3 && !e; ++f)
        for (int k = 0; k < 2 && !e; ++k)  // both buffers: faces are read from either
            e = cudaMemcpyAsync((char*)dst->field(k, f) + a.site0 * es, (const char*)src->field(src->cur, f) + b.site0 * es,
                                n * es, cudaMemcpyDeviceToDevice, dst->stream);
    if (!e)
        e = cudaMemcpyAsync(dst->cells(dst->ccur) + a.site0, src->cells(src->ccur) + b.site0, 4 * n,
                            cudaMemcpyDeviceToDevice, dst->stream);
    return cuda_check(dst, e, "copy lattice");
}

sim_status sim_set_state(sim_ctx* c, int p, const float* O, const float* G, const float* H, const uint32_t* cell) {
    if (!c || p < 0 || p >= c->n) return SIM_EINVAL;
    const Proto& pr = c->proto[p];
    const int64_t n = (int64_t)pr.L * pr.L * pr.L;
    const size_t es = elem_size(c->cfg.precision);
    const float* src[3] = {O, G, H};
    if (cell) {  // cells only on interior sites and with a valid kind
        const int L = pr.L;
        for (int64_t s = 0; s < n; ++s) {
            const uint32_t k = cell[s] & kKindMask;
            if (k == kEmpty) continue;
            const int x = (int)(s % L), y = (int)((s / L) % L), z = (int)(s / ((int64_t)L * L));
            if (k > kQ || x == 0 || y == 0 || z == 0 || x == L - 1 || y == L - 1 || z == L - 1)
                return fail(c, SIM_EINVAL, "cell word at site " + std::to_string(s) + " is invalid or on a face");
        }
    }
    std::vector<char> tmp((size_t)(n * es));
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 3 && !e; ++f) {
        if (!src[f]) continue;
        if (c->cfg.precision == SIM_FP32) std::memcpy(tmp.data(), src[f], n * 4);
        else if (c->cfg.precision == SIM_BF16)
            for (int64_t i = 0; i < n; ++i) ((__nv_bfloat16*)tmp.data())[i] = __float2bfloat16_rn(src[f][i]);
        else
            for (int64_t i = 0; i < n; ++i) ((__half*)tmp.data())[i] = __float2half_rn(src[f][i]);
        for (int b = 0; b < 2 && !e; ++b)  // both buffers: faces are read from either
            e = cudaMemcpyAsync((char*)c->field(b, f) + pr.site0 * es, tmp.data(), n * es, cudaMemcpyHostToDevice,
                                c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
    }
    if (!e && cell)
        e = cudaMemcpyAsync(c->cells(c->ccur) + pr.site0, cell, n * 4, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "set state");
}

sim_status sim_save_state(sim_ctx* c, void* buf, size_t* bytes) {
    if (!c || !bytes) return SIM_EINVAL;
    const size_t es = elem_size(c->cfg.precision);
    const size_t ncnt = (size_t)c->n * (c->cfg.hours + 1);
    const size_t need = ckpt_bytes(c);
    if (!buf) {
        *bytes = need;
        return SIM_OK;
    }
    if (*bytes < need) return fail(c, SIM_ENOSPC, "checkpoint buffer too small");
    CkptHeader h{};
    std::memcpy(h.magic, "GPUGACK1", 8);
    h.n = c->n;
    h.precision = c->cfg.precision;
    h.total_sites = c->total_sites;
    h.clock = c->clock;
    h.counted_hour = c->counted_hour;
    h.cur = c->cur;
    h.hours = c->cfg.hours;
    char* out = (char*)buf;
    std::memcpy(out, &h, sizeof h);
    size_t off = sizeof h;
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 3 && !e; ++f, off += es * c->total_sites)
        e = cudaMemcpyAsync(out + off, c->field(c->cur, f), es * c->total_sites, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(out + off, c->cells(c->ccur), 4 * c->total_sites, cudaMemcpyDeviceToHost, c->stream);
    off += 4 * c->total_sites;
    if (!e) e = cudaMemcpyAsync(out + off, c->ws + c->lay.cum, 8 * c->n, cudaMemcpyDeviceToHost, c->stream);
    off += 8 * c->n;
    if (!e) e = cudaMemcpyAsync(out + off, c->ws + c->lay.counts, 4 * ncnt, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_check(c, e, "save state");
    *bytes = need;
    return read_status(c);
}

sim_status sim_load_state(sim_ctx* c, const void* buf, size_t bytes) {
    if (!c || !buf || bytes < sizeof(CkptHeader)) return SIM_EINVAL;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    const size_t es = elem_size(c->cfg.precision);
    const size_t ncnt = (size_t)c->n * (c->cfg.hours + 1);
    if (std::memcmp(h.magic, "GPUGACK1", 8) || h.n != c->n || h.precision != c->cfg.precision ||
        h.total_sites != c->total_sites || h.hours != c->cfg.hours || bytes < ckpt_bytes(c))
        return fail(c, SIM_EINVAL, "checkpoint does not match this context");
    const char* in = (const char*)buf;
    size_t off = sizeof h;
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 3 && !e; ++f, off += es * c->total_sites)
        for (int b = 0; b < 2 && !e; ++b)
            e = cudaMemcpyAsync(c->field(b, f), in + off, es * c->total_sites, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(c->cells(0), in + off, 4 * c->total_sites, cudaMemcpyHostToDevice, c->stream);
    off += 4 * c->total_sites;
    if (!e) e = cudaMemcpyAsync(c->ws + c->lay.cum, in + off, 8 * c->n, cudaMemcpyHostToDevice, c->stream);
    off += 8 * c->n;
    if (!e) e = cudaMemcpyAsync(c->ws + c->lay.counts, in + off, 4 * ncnt, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(c->ws + c->lay.clock, &h.clock, sizeof h.clock, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.claim, 0, 8 * (size_t)c->total_sites, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.icount, 0, 8, c->stream);
    if (!e) e = cudaMemsetAsync(c->ws + c->lay.tile_ctr, 0, sizeof(uint32_t) * 2 * kMaxPasses, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_check(c, e, "load state");
    c->clock = h.clock;
    c->counted_hour = h.counted_hour;
    c->cur = 0;  // both field buffers hold the restored state
    c->ccur = 0;
    return SIM_OK;
}

void sim_destroy(sim_ctx* c) {
    if (!c) return;
    drop_graphs(c);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free reaction-diffusion step (sim_diffuse_noalloc).  For callers
// that cannot allocate device memory: the ping-pong field buffer and the
// launch tables live in this fixed file-scope device array, which every GPU
// that loads the library holds until the process exits.  Host code must not
// use the array's name as a device address (on the host it is only a
// stand-in); the real address comes from cudaGetSymbolAddress, looked up once
// per device and context (a cudaDeviceReset makes a new context, whose copy of
// the array lives elsewhere, so the cached address is looked up again).
namespace {
constexpr int kNoallocMaxL = 64;
constexpr size_t kNoallocMaxSites = (size_t)kNoallocMaxL * kNoallocMaxL * kNoallocMaxL;
constexpr size_t kNoallocFieldBytes = 3 * sizeof(float) * kNoallocMaxSites;  // 3 MiB
constexpr size_t kNoallocTableBytes = 64 * 1024;
constexpr int kNoallocMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocFieldBytes + kNoallocTableBytes];

namespace {
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_base[kNoallocMaxDevices] = {};
void* g_noalloc_ctx[kNoallocMaxDevices] = {};  // context the cached address belongs to

// The calling thread's current driver context (nullptr if none or if the query
// fails), through the runtime's driver entry point so that the library links
// against the runtime only.
void* current_context() {
    using GetCurrent = int (*)(void**);
    static GetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (GetCurrent)f;
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

// byte offsets of the launch tables behind the field buffer
constexpr size_t kNaProto = kNoallocFieldBytes;
constexpr size_t kNaBlocks = kNaProto + 256;
constexpr size_t kNaMaxBlocks = (kNoallocMaxSites + kSitesPerBlock - 1) / kSitesPerBlock;
constexpr size_t kNaFstep = kNaBlocks + sizeof(Block) * kNaMaxBlocks;
constexpr size_t kNaFdose = kNaFstep + 64;
constexpr size_t kNaClock = kNaFdose + 64;
constexpr size_t kNaCum = kNaClock + 64;
static_assert(kNaCum + 64 <= kNoallocFieldBytes + kNoallocTableBytes, "no-alloc tables overflow the scratch array");
}  // namespace

extern "C" sim_status sim_diffuse_noalloc(const sim_config* cfg, int L, int64_t step, double dose_gy, float* O,
                                          float* G, float* H, uint32_t* cell, void* cuda_stream) {
    if (!cfg || !O || !G || !H || !cell) return SIM_EINVAL;
    std::string why;
    if (!valid_config(cfg, &why) || cfg->precision != SIM_FP32) return SIM_EINVAL;
    if (L < 8) return SIM_EINVAL;
    if (L > kNoallocMaxL) return SIM_ENOSPC;  // the fixed scratch holds at most 64^3 sites
    if (step < 0 || step >= (int64_t)0xffffffffLL || !(dose_gy >= 0.0) || !std::isfinite(dose_gy)) return SIM_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // The launch tables are copied from host memory that lives only during this call: a captured copy node
    // would read it after it is gone, so a call on a stream under capture is refused before any work.
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &capturing) != cudaSuccess || capturing != cudaStreamCaptureStatusNone)
        return SIM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return SIM_ECUDA;
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        void* ctx = current_context();
        if (!g_noalloc_base[dev] || !ctx || ctx != g_noalloc_ctx[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SIM_ECUDA;
            g_noalloc_base[dev] = (unsigned char*)p;
            g_noalloc_ctx[dev] = ctx ? ctx : current_context();  // the lookup may have created the context
        }
        base = g_noalloc_base[dev];
    }
    Params P = make_params(*cfg);  // frac_cap 0: the one fraction is its own quadratic partner
    const int64_t sites = (int64_t)L * L * L;
    P.n_sites = (uint64_t)sites;  // no status word here: index checks of a SIM_CHECK build skip silently
    Proto pr{};
    pr.L = L;
    pr.R = -1;
    pr.site0 = 0;
    pr.t_end = step + 1;
    pr.frac0 = 0;
    pr.nfrac = dose_gy > 0.0 ? 1 : 0;
    std::vector<Block> blocks;
    for (int64_t b = 0; b < sites; b += kSitesPerBlock) {
        Block bl{};
        bl.p = 0;
        bl.begin = b;
        bl.n = (int)((sites - b) < kSitesPerBlock ? (sites - b) : kSitesPerBlock);
        blocks.push_back(bl);
    }
    const double zero = 0.0;
    // host-to-device copies from pageable memory return once the source has been staged
    cudaError_t e = cudaMemcpyAsync(base + kNaProto, &pr, sizeof pr, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(base + kNaBlocks, blocks.data(), sizeof(Block) * blocks.size(), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(base + kNaFstep, &step, sizeof step, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(base + kNaFdose, &dose_gy, sizeof dose_gy, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(base + kNaClock, &step, sizeof step, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(base + kNaCum, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
    // the scratch buffer starts as a copy of the caller's fields so both buffers hold the same Dirichlet faces
    float* buf[2][3] = {{O, G, H},
                        {(float*)base, (float*)base + kNoallocMaxSites, (float*)base + 2 * kNoallocMaxSites}};
    for (int f = 0; f < 3 && !e; ++f)
        e = cudaMemcpyAsync(buf[1][f], buf[0][f], sizeof(float) * sites, cudaMemcpyDeviceToDevice, s);
    if (e) return SIM_ECUDA;
    int cur = 0;
    const Block* blk = (const Block*)(base + kNaBlocks);
    const Proto* prot = (const Proto*)(base + kNaProto);
    const int64_t* clk = (const int64_t*)(base + kNaClock);
    const int64_t* fst = (const int64_t*)(base + kNaFstep);
    const double* fds = (const double*)(base + kNaFdose);
    double* cum = (double*)(base + kNaCum);
    int k_off = 0;
    for (int sub = 0; sub < P.n_sub && !e; ++sub) {
        const float *iO = buf[cur][0], *iG = buf[cur][1], *iH = buf[cur][2];
        float *oO = buf[cur ^ 1][0], *oG = buf[cur ^ 1][1], *oH = buf[cur ^ 1][2];
        void* args[] = {&blk, &prot, &clk, &k_off, &sub, &iO, &iG, &iH, &oO, &oG, &oH, &cell, &fst, &fds, &cum, &P};
        // the launch's own status: an error left pending by earlier, unrelated work is neither reported nor cleared
        e = cudaLaunchKernel((const void*)k_substep<float>, dim3((unsigned)blocks.size()), dim3(kThreads), args, 0, s);
        cur ^= 1;
    }
    for (int f = 0; f < 3 && cur == 1 && !e; ++f)  // odd n_sub: the result sits in the scratch buffer
        e = cudaMemcpyAsync(buf[0][f], buf[1][f], sizeof(float) * sites, cudaMemcpyDeviceToDevice, s);
    return e ? SIM_ECUDA : SIM_OK;
}
