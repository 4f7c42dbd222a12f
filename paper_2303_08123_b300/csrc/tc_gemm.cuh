// tc_gemm.cuh -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores
// (tcgen05, sm_103a), written with inline PTX.
//
//   C[M x N] (FP32, row-major) = A[M x K] * B[N x K]^T   (A, B BF16, K contiguous)
//
// One CTA (4 warps) owns a 128-row x (up to) 64-column tile of C, so that a
// 4,096 x 256 product runs on 128 CTAs.  The accumulator lives in tensor memory
// (TMEM): lane = row, column = output column.  K advances in chunks of 64,
// double-buffered: all threads stage chunk c + 1 of A and B in shared memory (in
// the no-swizzle K-major core-matrix layout, 8 rows x 16 bytes per core matrix)
// while the tensor cores work on chunk c; one elected thread issues the
// tcgen05.mma instructions (M = 128, N, K = 16 each), and tcgen05.commit makes
// the buffer's mbarrier arrive when they have finished reading it.  A buffer is
// restaged only after that arrival.  The epilogue reads TMEM with tcgen05.ld
// (each warp its 32 lanes) and stores FP32 rows.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace tcg {

constexpr int kRows = 128;     // M per CTA
constexpr int kChunk = 64;     // K per staged chunk
constexpr int kThreads = 128;  // 4 warps: one per 32 TMEM lanes
constexpr int kCoreBytes = 128;               // 8 rows x 16 bytes
constexpr int kSbo = (kChunk / 8) * kCoreBytes;  // bytes between 8-row groups (1024)
constexpr uint32_t kSpinLimit = 1u << 26;     // bounded mbarrier wait

constexpr int kCols = 64;      // N per CTA (columns of C)
// bytes of one staged A (128 x 64) and B (<= 64 x 64) chunk
constexpr int kABytes = (kRows / 8) * kSbo;
constexpr int kBBytes = (kCols / 8) * kSbo;
constexpr int kBufBytes = kABytes + kBBytes;
// requested dynamic shared memory: two buffers and the barriers; at most four
// CTAs fit on one SM, so their 4 x 64 TMEM columns never exceed the SM's 512 and
// tcgen05.alloc never waits
constexpr int kSmemBytes = 52 * 1024;
static_assert(2 * kBufBytes + 64 <= kSmemBytes, "staging buffers exceed the shared-memory request");
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

// Stage rows [0, rows) x K-columns [k0, k0 + kc) of a row-major BF16 matrix
// (leading dimension ld) into the core-matrix layout: 16-byte unit (r, u)
// (u = 8-column group) goes to (r / 8) * kSbo + u * 128 + (r % 8) * 16.
__device__ __forceinline__ void stage(unsigned char* dst, const __nv_bfloat16* __restrict__ src, int rows, int ld,
                                      int k0, int kc) {
    const int units = rows * (kc / 8);
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
        const int r = u / (kc / 8), cu = u % (kc / 8);
        const uint4 v = *reinterpret_cast<const uint4*>(src + (size_t)r * ld + k0 + cu * 8);
        *reinterpret_cast<uint4*>(dst + (r / 8) * kSbo + cu * kCoreBytes + (r % 8) * 16) = v;
    }
}

// C = A * B^T for one tile: rows 128 blockIdx.x.., columns 64 blockIdx.y..; N a
// multiple of 16 (<= 256), K a multiple of 16, M a multiple of 128.  *status != 0
// after a timed-out wait.
__global__ void __launch_bounds__(kThreads) k_gemm_bf16(const __nv_bfloat16* __restrict__ A,
                                                        const __nv_bfloat16* __restrict__ B, float* __restrict__ C,
                                                        int M, int N, int K, uint32_t* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // buffer b: A chunk at smem + b * kBufBytes, B chunk kABytes after it
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kBufBytes);  // one per buffer
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * kBufBytes + 16);
    __shared__ int s_fail;
    const int warp = threadIdx.x / 32;
    const int n0 = blockIdx.y * kCols;
    const int nt = (N - n0) < kCols ? (N - n0) : kCols;  // columns of this tile (a multiple of 16)
    const uint32_t ncols = nt <= 32 ? 32u : 64u;
    if (warp == 0) tmem_alloc(tslot, ncols);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int m0 = blockIdx.x * kRows;
    const uint32_t idesc = instr_desc(kRows, nt);
    const int n_chunks = (K + kChunk - 1) / kChunk;
    uint32_t phase0 = 0u, phase1 = 0u;  // parity of the next completion of each buffer's barrier
    int committed = 0;  // chunks whose MMAs were issued
    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        if (c >= 2) {  // the MMAs of chunk c - 2 must be done reading this buffer
            if (threadIdx.x == 0 && !mbar_wait(&bar[buf], buf ? phase1 : phase0)) s_fail = 1;
            (buf ? phase1 : phase0) ^= 1u;
            __syncthreads();
            if (s_fail) break;
        }
        const int k0 = c * kChunk;
        const int kc = (K - k0) < kChunk ? (K - k0) : kChunk;
        unsigned char* sA = smem + buf * kBufBytes;
        unsigned char* sB = sA + kABytes;
        stage(sA, A + (size_t)m0 * K, kRows, K, k0, kc);
        stage(sB, B + (size_t)n0 * K, nt, K, k0, kc);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy stores -> async proxy
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < kc / 16; ++ks) {
                const uint64_t da = smem_desc(smem_u32(sA) + ks * 2 * kCoreBytes, kCoreBytes, kSbo);
                const uint64_t db = smem_desc(smem_u32(sB) + ks * 2 * kCoreBytes, kCoreBytes, kSbo);
                mma_bf16(tmem, da, db, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&bar[buf]);
        }
        committed = c + 1;
    }
    // the last (up to two) commits: every MMA has finished and the accumulator is complete
    if (threadIdx.x == 0)
        for (int c = committed >= 2 ? committed - 2 : 0; c < committed; ++c) {
            const int buf = c & 1;
            if (!mbar_wait(&bar[buf], buf ? phase1 : phase0)) s_fail = 1;
            (buf ? phase1 : phase0) ^= 1u;
        }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        const int row = m0 + warp * 32 + (threadIdx.x & 31);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int cb = 0; cb < nt; cb += 32) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)cb, v);
            const int nv = (nt - cb) < 32 ? (nt - cb) : 32;
            float* dst = C + (size_t)row * N + n0 + cb;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < nv) dst[j] = v[j];
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
