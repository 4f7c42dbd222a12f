// tc_gemm.cuh -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores
// (tcgen05, sm_103a), written with inline PTX.
//
//   C[M x N] (FP32, row-major) = A[M x K] * B[N x K]^T   (A, B BF16, K contiguous)
//
// One CTA (4 warps) owns a 128-row x (up to) 64-column tile of C, so that a
// 4,096 x 256 product runs on 128 CTAs.  The accumulator lives in tensor memory
// (TMEM): lane = row, column = output column.  K advances in chunks of 64,
// double-buffered and staged by the tensor memory accelerator: per chunk one
// thread issues one 2-D tiled bulk-tensor load per 8 K-columns of A (a 8 x 128
// box) and of B (a 8 x 64 box).  A box lands as rows of 16 bytes, which is the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
// 128 bytes between 8-row groups, one box between K groups).  The same thread
// issues the tcgen05.mma instructions (M = 128, N, K = 16 each) once the
// chunk's mbarrier reports its bytes, and tcgen05.commit makes a second
// mbarrier arrive when they have finished reading the buffer, which is then
// restaged with chunk c + 2 while chunk c + 1 is multiplied.  The epilogue reads
// TMEM with tcgen05.ld (each warp its 32 lanes) into shared memory and writes the
// FP32 tile with TMA stores.
#pragma once
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

namespace tcg {

constexpr int kRows = 128;     // M per CTA
constexpr int kChunk = 64;     // K per staged chunk
constexpr int kThreads = 128;  // 4 warps: one per 32 TMEM lanes
constexpr int kCoreBytes = 128;  // 8 rows x 16 bytes: a core matrix, and the distance between 8-row groups
constexpr uint32_t kSpinLimit = 1u << 26;     // bounded mbarrier wait

constexpr int kCols = 64;      // N per CTA (columns of C)
// bytes of one staged A (128 x 64) and B (64 x 64) chunk; one box of 8 K-columns is kRows (kCols) rows of 16 B
constexpr int kABox = kRows * 16, kBBox = kCols * 16;
constexpr int kABytes = (kChunk / 8) * kABox;
constexpr int kBBytes = (kChunk / 8) * kBBox;
constexpr int kBufBytes = kABytes + kBBytes;
// requested dynamic shared memory: two buffers and the barriers; at most four
// CTAs fit on one SM, so their 4 x 64 TMEM columns never exceed the SM's 512 and
// tcgen05.alloc never waits
constexpr int kSmemBytes = 52 * 1024;
static_assert(2 * kBufBytes + 1024 + 64 <= kSmemBytes, "staging buffers exceed the shared-memory request");
static_assert(5 * kSmemBytes > 228 * 1024, "more than four CTAs per SM could exhaust the tensor memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start address, the
// byte offset between core matrices adjacent in K (leading) and in M/N
// (stride), all in 16-byte units; bits 46-47 carry the descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;  // base offset 0, relative leading offset, layout type 0 (no swizzle)
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// wait for the phase with the given parity to complete; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (thread t <- lane t)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 2-D tiled bulk-tensor load (x = K column, y = row) into shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 2-D tiled bulk-tensor store of one box from shared memory (bulk-group completion)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// C = A * B^T for one tile: rows 128 blockIdx.x.., columns 64 blockIdx.y..; N a
// multiple of 16 (<= 256), K a multiple of 16, M a multiple of 128.  mapA / mapB
// describe A [M x K] and B [N x K] (BF16, K innermost) with boxes of 8 K-columns
// by 128 / 64 rows.  *status != 0 after a timed-out wait.
__global__ void __launch_bounds__(kThreads) k_gemm_bf16(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapB,
                                                        const __grid_constant__ CUtensorMap mapC, int M, int N,
                                                        int K, uint32_t* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // buffers start 1024-byte aligned: buffer b holds A at +0 and B at +kABytes, each as one box per 8 K-columns
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * kBufBytes);   // chunk landed, per buffer
    uint64_t* done = full + 2;                                            // chunk's MMAs finished, per buffer
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 2);
    __shared__ int s_fail;
    const int warp = threadIdx.x / 32;
    const int n0 = blockIdx.y * kCols;
    const int nt = (N - n0) < kCols ? (N - n0) : kCols;  // columns of this tile (a multiple of 16)
    const uint32_t ncols = nt <= 32 ? 32u : 64u;
    if (warp == 0) tmem_alloc(tslot, ncols);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&done[b], 1);
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int m0 = blockIdx.x * kRows;
    const int n_chunks = (K + kChunk - 1) / kChunk;
    if (threadIdx.x == 0) {
        const uint32_t idesc = instr_desc(kRows, nt);
        const uint32_t base = smem_u32(smem);
        // stage chunk c into buffer c & 1 (its boxes beyond K are not loaded; rows beyond N read as zeros)
        auto load = [&](int c) {
            const int b = c & 1, k0 = c * kChunk;
            const int groups = ((K - k0) < kChunk ? (K - k0) : kChunk) / 8;
            mbar_expect_tx(&full[b], (uint32_t)groups * (kABox + kBBox));
            for (int j = 0; j < groups; ++j) {
                tma_load_2d(base + b * kBufBytes + j * kABox, &mapA, k0 + 8 * j, m0, &full[b]);
                tma_load_2d(base + b * kBufBytes + kABytes + j * kBBox, &mapB, k0 + 8 * j, n0, &full[b]);
            }
        };
        uint32_t ph_full0 = 0u, ph_full1 = 0u, ph_done0 = 0u, ph_done1 = 0u;  // parities of the next completions
        auto wait = [&](uint64_t* bar, uint32_t& ph) {
            const bool r = mbar_wait(bar, ph);
            ph ^= 1u;
            return r;
        };
        load(0);
        if (n_chunks > 1) load(1);
        bool ok = true;
        for (int c = 0; c < n_chunks && ok; ++c) {
            const int b = c & 1;
            ok = wait(&full[b], b ? ph_full1 : ph_full0);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int kc = (K - c * kChunk) < kChunk ? (K - c * kChunk) : kChunk;
            for (int ks = 0; ks < kc / 16; ++ks) {
                const uint32_t a = base + b * kBufBytes + ks * 2 * kABox;
                const uint32_t bb = base + b * kBufBytes + kABytes + ks * 2 * kBBox;
                mma_bf16(tmem, smem_desc(a, kABox, kCoreBytes), smem_desc(bb, kBBox, kCoreBytes), idesc,
                         (c > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&done[b]);
            // chunk c + 1 goes into the other buffer once chunk c - 1's MMAs have read it (chunk 1: already loaded)
            if (c >= 1 && c + 1 < n_chunks) {
                ok = wait(&done[b ^ 1], b ? ph_done0 : ph_done1);
                if (ok) load(c + 1);
            }
        }
        // the last commits: every MMA has finished and the accumulator is complete
        for (int c = n_chunks >= 2 ? n_chunks - 2 : 0; c < n_chunks && ok; ++c)
            ok = wait(&done[c & 1], (c & 1) ? ph_done1 : ph_done0);
        if (!ok) {
            s_fail = 1;
            // give copies and MMAs that may still be in flight a bounded time to land before the CTA exits
            for (int b = 0; b < 2; ++b) {
                (void)mbar_wait(&full[b], b ? ph_full1 : ph_full0, 1u << 16);
                (void)mbar_wait(&done[b], b ? ph_done1 : ph_done0, 1u << 16);
            }
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        // Epilogue: the tile goes through shared memory (the staging buffers are free now) as up to two boxes of
        // 32 columns x 128 rows, each row 128 bytes with its 16-byte units XOR-swizzled by row % 8 (the TMA 128-byte
        // swizzle, which also spreads a warp's stores over all banks), then one TMA store per box writes it out;
        // columns beyond N are clipped by the tensor map.
        const int r = warp * 32 + (threadIdx.x & 31);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int cb = 0; cb < nt; cb += 32) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)cb, v);
            float4* box = reinterpret_cast<float4*>(smem + (cb / 32) * (kRows * 128) + r * 128);
#pragma unroll
            for (int j = 0; j < 8; ++j) box[j ^ (r & 7)] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy stores -> the TMA store
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int cb = 0; cb < nt; cb += 32) tma_store_2d(&mapC, n0 + cb, m0, smem_u32(smem) + (cb / 32) * (kRows * 128));
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // shared memory read before the CTA exits
        }
    } else if (threadIdx.x == 0) {
        atomicExch(status, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Failure-path probe: waits on an mbarrier that nothing will ever arrive at,
// with `limit` polls, and reports the timeout through *status exactly as the
// GEMM does.  Lets a test exercise the error path without hanging the GPU.
__global__ void k_wait_probe(uint32_t limit, uint32_t* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(&bar, 0, limit)) atomicExch(status, 1u);
    }
}

}  // namespace tcg
