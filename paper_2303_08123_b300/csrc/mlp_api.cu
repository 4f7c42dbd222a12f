// mlp_api.cu -- the surrogate network behind include/mlp.h (sm_103a).
//
// Forward:  Z_l = A_{l-1} W_l^T + b_l,  A_l = GELU(Z_l)  (l = 1..3),  y = A_3 w_4 + b_4
// Backward: mean squared error, dZ_l = dA_l * GELU'(Z_l),
//           dW_l = dZ_l^T A_{l-1},  dA_{l-1} = dZ_l W_l,  db_l = column sums of dZ_l
// Every product above is one call of the tcgen05 GEMM (C = A B^T with both
// operands K-major): the forward stores each activation both row-major and
// transposed, and each weight is kept in BF16 both as W and as W^T, so no
// GEMM ever needs a transposed operand.  Elementwise work (bias, GELU and its
// derivative, the 256 -> 1 output layer, loss, Adam) runs in small kernels.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mlp.h"
#include "tc_gemm.cuh"

namespace {

constexpr int H = MLP_HIDDEN, IP = MLP_IN_PAD, IN = MLP_IN;
constexpr int kEw = 256;  // threads of the elementwise kernels

// parameter offsets (floats)
constexpr int oW1 = 0, oB1 = oW1 + H * IP, oW2 = oB1 + H, oB2 = oW2 + H * H, oW3 = oB2 + H, oB3 = oW3 + H * H,
              oW4 = oB3 + H, oB4 = oW4 + H, kNP = oB4 + 1;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
    size_t p, g, m, v, w16[3], wt16[3], x16, xt16, z[3], h16[3], ht16[3], h3, y, dy, dz, dz16, dzt16, c, red, status,
        total;
};

Layout layout(int B) {
    Layout l{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    const int in_l[3] = {IP, H, H};
    l.p = take(4 * kNP);
    l.g = take(4 * kNP);
    l.m = take(4 * kNP);
    l.v = take(4 * kNP);
    for (int i = 0; i < 3; ++i) {
        l.w16[i] = take(2 * H * in_l[i]);
        l.wt16[i] = take(2 * H * in_l[i]);
    }
    l.x16 = take(2 * (size_t)B * IP);
    l.xt16 = take(2 * (size_t)B * IP);
    for (int i = 0; i < 3; ++i) {
        l.z[i] = take(4 * (size_t)B * H);
        l.h16[i] = take(2 * (size_t)B * H);
        l.ht16[i] = take(2 * (size_t)B * H);
    }
    l.h3 = take(4 * (size_t)B * H);
    l.y = take(4 * (size_t)B);
    l.dy = take(4 * (size_t)B);
    l.dz = take(4 * (size_t)B * H);
    l.dz16 = take(2 * (size_t)B * H);
    l.dzt16 = take(2 * (size_t)B * H);
    l.c = take(4 * (size_t)(B > H ? B : H) * H);
    l.red = take(4 * 8);
    l.status = take(4);
    l.total = off;
    return l;
}

// splitmix64 (Steele, Lea, Flood, OOPSLA 2014): host-side weight initialisation
uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// X (B x 45 FP32) -> X16 (B x 48 BF16, zero-padded) and its transpose (48 x B)
__global__ void k_prep_x(const float* __restrict__ X, int B, __nv_bfloat16* __restrict__ x16,
                         __nv_bfloat16* __restrict__ xt16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * IP) return;
    const int r = i / IP, c = i % IP;
    const __nv_bfloat16 v = __float2bfloat16_rn(c < IN ? X[(size_t)r * IN + c] : 0.f);
    x16[i] = v;
    xt16[(size_t)c * B + r] = v;
}

// Z = C + b (kept in FP32), A = GELU(Z): BF16 row-major and transposed, FP32 optionally
__global__ void k_bias_gelu(const float* __restrict__ C, const float* __restrict__ b, int B, float* __restrict__ Z,
                            __nv_bfloat16* __restrict__ a16, __nv_bfloat16* __restrict__ at16, float* __restrict__ a32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * H) return;
    const int r = i / H, c = i % H;
    const float z = C[i] + b[c];
    Z[i] = z;
    const float a = gelu(z);
    const __nv_bfloat16 a_b = __float2bfloat16_rn(a);
    a16[i] = a_b;
    at16[(size_t)c * B + r] = a_b;
    if (a32) a32[i] = a;
}

// y = A3 w4 + b4 (one warp per row)
__global__ void k_out(const float* __restrict__ a3, const float* __restrict__ p, int B, float* __restrict__ y) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= B) return;
    float s = 0.f;
    for (int j = lane; j < H; j += 32) s = fmaf(a3[(size_t)row * H + j], p[oW4 + j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s + p[oB4];
}

// loss = mean (y - t)^2 (FP64 accumulation) and dy = 2 (y - t) / B
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, int B, float* __restrict__ dy,
                       double* __restrict__ loss) {
    __shared__ double part[kEw];
    double s = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const float e = y[i] - t[i];
        dy[i] = 2.f * e / (float)B;
        s += (double)e * (double)e;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) a += part[k];
        *loss = a / (double)B;
    }
}

// output layer gradients: g_w4[j] = sum_b dy_b A3[b][j], g_b4 = sum_b dy_b (one block per j, one for b4)
__global__ void k_grad_out(const float* __restrict__ dy, const float* __restrict__ a3, int B, float* __restrict__ g) {
    __shared__ float part[kEw];
    const int j = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += dy[b] * (j < H ? a3[(size_t)b * H + j] : 1.f);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int k = 0; k < (int)blockDim.x; ++k) a += part[k];
        g[j < H ? oW4 + j : oB4] = a;
    }
}

// dZ = dA * GELU'(Z) where dA = dy (x) w4 (last hidden layer) or the GEMM output C
__global__ void k_back(const float* __restrict__ C, const float* __restrict__ dy, const float* __restrict__ p,
                       const float* __restrict__ Z, int B, float* __restrict__ dz, __nv_bfloat16* __restrict__ dz16,
                       __nv_bfloat16* __restrict__ dzt16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * H) return;
    const int r = i / H, c = i % H;
    const float da = dy ? dy[r] * p[oW4 + c] : C[i];
    const float d = da * gelu_grad(Z[i]);
    dz[i] = d;
    const __nv_bfloat16 d_b = __float2bfloat16_rn(d);
    dz16[i] = d_b;
    dzt16[(size_t)c * B + r] = d_b;
}

// db[c] = sum_b dz[b][c] (one block per column)
__global__ void k_colsum(const float* __restrict__ dz, int B, float* __restrict__ db) {
    __shared__ float part[kEw];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += dz[(size_t)b * H + c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int k = 0; k < (int)blockDim.x; ++k) a += part[k];
        db[c] = a;
    }
}

// dW (C, H x in) -> gradient slot (W1 keeps its 48 padded columns, their gradient is zeroed)
__global__ void k_copy_grad(const float* __restrict__ C, int n_in, int n_real, float* __restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * n_in) return;
    g[i] = (i % n_in) < n_real ? C[i] : 0.f;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// BF16 copies of W (out x in) and W^T (in x out)
__global__ void k_refresh(const float* __restrict__ W, int n_in, __nv_bfloat16* __restrict__ w16,
                          __nv_bfloat16* __restrict__ wt16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * n_in) return;
    const int r = i / n_in, c = i % n_in;
    const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
    w16[i] = v;
    wt16[(size_t)c * H + r] = v;
}

unsigned blocks(size_t n) { return (unsigned)((n + kEw - 1) / kEw); }

}  // namespace

struct mlp_ctx {
    int batch_max = 0;
    Layout lay{};
    char* ws = nullptr;
    cudaStream_t stream = nullptr;
    int64_t adam_t = 0;
    template <typename T>
    T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? 0 : -3; }

// Tensor map of a row-major BF16 matrix [rows x K] for the GEMM's staging: x = K
// column, y = row, a box of 8 K-columns by box_rows rows (rows beyond the matrix
// read as zeros).  The driver's encoder is reached through the runtime.
bool encode_operand(CUtensorMap* m, const void* base, int rows, int K, int box_rows) {
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
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the FP32 result C [M x N] for the epilogue's stores: boxes of 32
// columns (128 bytes) by 128 rows in the 128-byte swizzle; columns beyond N are
// not written.
bool encode_result(CUtensorMap* m, float* base, int M, int N) {
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
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
    const cuuint64_t strides[1] = {(cuuint64_t)N * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)tcg::kRows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int gemm(const void* A, const void* B, float* C, int M, int N, int K, uint32_t* status, cudaStream_t s) {
    if (M <= 0 || M % tcg::kRows || N < 16 || N > 256 || N % 16 || K <= 0 || K % 16) return -1;
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16 || (uintptr_t)C % 16) return -1;  // tensor-map bases: 16-byte aligned
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(tcg::k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, tcg::kSmemBytes))
            return -3;
        attr = true;
    }
    CUtensorMap mapA, mapB, mapC;
    if (!encode_operand(&mapA, A, M, K, tcg::kRows) || !encode_operand(&mapB, B, N, K, tcg::kCols) ||
        !encode_result(&mapC, C, M, N))
        return -3;
    const dim3 grid((unsigned)(M / tcg::kRows), (unsigned)((N + tcg::kCols - 1) / tcg::kCols));
    tcg::k_gemm_bf16<<<grid, tcg::kThreads, tcg::kSmemBytes, s>>>(mapA, mapB, mapC, M, N, K, status);
    return cuda_status(cudaGetLastError());
}

void refresh(mlp_ctx* c) {
    const int in_l[3] = {IP, H, H};
    const int off[3] = {oW1, oW2, oW3};
    for (int l = 0; l < 3; ++l)
        k_refresh<<<blocks((size_t)H * in_l[l]), kEw, 0, c->stream>>>(
            c->at<float>(c->lay.p) + off[l], in_l[l], c->at<__nv_bfloat16>(c->lay.w16[l]),
            c->at<__nv_bfloat16>(c->lay.wt16[l]));
}

int forward(mlp_ctx* c, const float* X, int B) {
    uint32_t* st = c->at<uint32_t>(c->lay.status);
    float* p = c->at<float>(c->lay.p);
    float* C = c->at<float>(c->lay.c);
    k_prep_x<<<blocks((size_t)B * IP), kEw, 0, c->stream>>>(X, B, c->at<__nv_bfloat16>(c->lay.x16),
                                                              c->at<__nv_bfloat16>(c->lay.xt16));
    const int boff[3] = {oB1, oB2, oB3};
    const int in_l[3] = {IP, H, H};
    const __nv_bfloat16* a_prev = c->at<__nv_bfloat16>(c->lay.x16);
    for (int l = 0; l < 3; ++l) {
        int r = gemm(a_prev, c->at<__nv_bfloat16>(c->lay.w16[l]), C, B, H, in_l[l], st, c->stream);
        if (r) return r;
        k_bias_gelu<<<blocks((size_t)B * H), kEw, 0, c->stream>>>(
            C, p + boff[l], B, c->at<float>(c->lay.z[l]), c->at<__nv_bfloat16>(c->lay.h16[l]),
            c->at<__nv_bfloat16>(c->lay.ht16[l]), l == 2 ? c->at<float>(c->lay.h3) : nullptr);
        a_prev = c->at<__nv_bfloat16>(c->lay.h16[l]);
    }
    k_out<<<(B + 7) / 8, 256, 0, c->stream>>>(c->at<float>(c->lay.h3), p, B, c->at<float>(c->lay.y));
    return cuda_status(cudaGetLastError());
}

// forward + backward into the gradient buffer; loss (FP64) left on the device
int backward(mlp_ctx* c, const float* X, const float* t, int B) {
    if (int r = forward(c, X, B)) return r;
    uint32_t* st = c->at<uint32_t>(c->lay.status);
    float* p = c->at<float>(c->lay.p);
    float* g = c->at<float>(c->lay.g);
    float* C = c->at<float>(c->lay.c);
    float* dy = c->at<float>(c->lay.dy);
    k_loss<<<1, kEw, 0, c->stream>>>(c->at<float>(c->lay.y), t, B, dy, c->at<double>(c->lay.red));
    k_grad_out<<<H + 1, kEw, 0, c->stream>>>(dy, c->at<float>(c->lay.h3), B, g);
    const int woff[3] = {oW1, oW2, oW3}, boff[3] = {oB1, oB2, oB3};
    const int in_l[3] = {IP, H, H};
    for (int l = 2; l >= 0; --l) {
        // dZ_l from dA_l (the output layer for l = 2, else the GEMM result of the layer above)
        k_back<<<blocks((size_t)B * H), kEw, 0, c->stream>>>(C, l == 2 ? dy : nullptr, p, c->at<float>(c->lay.z[l]),
                                                            B, c->at<float>(c->lay.dz),
                                                            c->at<__nv_bfloat16>(c->lay.dz16),
                                                            c->at<__nv_bfloat16>(c->lay.dzt16));
        k_colsum<<<H, kEw, 0, c->stream>>>(c->at<float>(c->lay.dz), B, g + boff[l]);
        // dW_l = dZ_l^T A_{l-1}: A operand dZ^T (H x B), B operand A_{l-1}^T (in x B)
        const __nv_bfloat16* at_prev =
            l == 0 ? c->at<__nv_bfloat16>(c->lay.xt16) : c->at<__nv_bfloat16>(c->lay.ht16[l - 1]);
        int r = gemm(c->at<__nv_bfloat16>(c->lay.dzt16), at_prev, C, H, in_l[l], B, st, c->stream);
        if (r) return r;
        k_copy_grad<<<blocks((size_t)H * in_l[l]), kEw, 0, c->stream>>>(C, in_l[l], l == 0 ? IN : H, g + woff[l]);
        if (l > 0) {
            // dA_{l-1} = dZ_l W_l: A operand dZ (B x H), B operand W_l^T (in x H)
            r = gemm(c->at<__nv_bfloat16>(c->lay.dz16), c->at<__nv_bfloat16>(c->lay.wt16[l]), C, B, in_l[l], H, st,
                     c->stream);
            if (r) return r;
        }
    }
    return cuda_status(cudaGetLastError());
}

int check_batch(const mlp_ctx* c, int B) { return (B <= 0 || B % tcg::kRows || B > c->batch_max) ? -1 : 0; }

int fetch_loss(mlp_ctx* c, float* loss) {
    double l = 0.0;
    uint32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&l, c->at<double>(c->lay.red), 8, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(&st, c->at<uint32_t>(c->lay.status), 4, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return -3;
    if (st) return -4;
    if (loss) *loss = (float)l;
    return 0;
}

}  // namespace

extern "C" {

int mlp_num_params(void) { return kNP; }

int mlp_workspace_size(int batch_max, size_t* bytes) {
    if (!bytes || batch_max <= 0 || batch_max % tcg::kRows) return -1;
    *bytes = layout(batch_max).total;
    return 0;
}

int mlp_create(int batch_max, uint64_t seed, void* d_ws, size_t bytes, void* stream, mlp_ctx** out) {
    if (!out || !d_ws || batch_max <= 0 || batch_max % tcg::kRows) return -1;
    *out = nullptr;
    if (((uintptr_t)d_ws) % 256) return -1;
    const Layout l = layout(batch_max);
    if (bytes < l.total) return -2;
    mlp_ctx* c = new mlp_ctx();
    c->batch_max = batch_max;
    c->lay = l;
    c->ws = (char*)d_ws;
    c->stream = (cudaStream_t)stream;
    std::vector<float> p(kNP, 0.f);
    uint64_t s = seed;
    auto fill = [&](int off, int rows, int fan_in, int cols_real, int cols) {
        const float a = std::sqrt(6.0f / (float)fan_in);
        for (int r = 0; r < rows; ++r)
            for (int k = 0; k < cols; ++k) {
                const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
                p[off + r * cols + k] = k < cols_real ? (float)((2.0 * u - 1.0) * a) : 0.f;
            }
    };
    fill(oW1, H, IN, IN, IP);
    fill(oW2, H, H, H, H);
    fill(oW3, H, H, H, H);
    fill(oW4, 1, H, H, H);
    int r = mlp_set_params(c, p.data());
    if (r) {
        delete c;
        return r;
    }
    *out = c;
    return 0;
}

int mlp_set_params(mlp_ctx* c, const float* host) {
    if (!c || !host) return -1;
    cudaError_t e = cudaMemcpyAsync(c->at<float>(c->lay.p), host, 4 * kNP, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemsetAsync(c->at<float>(c->lay.m), 0, 4 * kNP, c->stream);
    if (!e) e = cudaMemsetAsync(c->at<float>(c->lay.v), 0, 4 * kNP, c->stream);
    if (!e) e = cudaMemsetAsync(c->at<uint32_t>(c->lay.status), 0, 4, c->stream);
    if (e) return -3;
    refresh(c);
    c->adam_t = 0;
    return cuda_status(cudaStreamSynchronize(c->stream));
}

int mlp_get_params(mlp_ctx* c, float* host) {
    if (!c || !host) return -1;
    cudaError_t e = cudaMemcpyAsync(host, c->at<float>(c->lay.p), 4 * kNP, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return cuda_status(e);
}

int mlp_forward(mlp_ctx* c, const float* d_X, int B, float* d_y) {
    if (!c || !d_X || !d_y || check_batch(c, B)) return -1;
    if (int r = forward(c, d_X, B)) return r;
    return cuda_status(cudaMemcpyAsync(d_y, c->at<float>(c->lay.y), 4 * (size_t)B, cudaMemcpyDeviceToDevice,
                                       c->stream));
}

int mlp_gradients(mlp_ctx* c, const float* d_X, const float* d_t, int B, float* d_grad, float* loss) {
    if (!c || !d_X || !d_t || !d_grad || check_batch(c, B)) return -1;
    if (int r = backward(c, d_X, d_t, B)) return r;
    cudaError_t e = cudaMemcpyAsync(d_grad, c->at<float>(c->lay.g), 4 * kNP, cudaMemcpyDeviceToDevice, c->stream);
    if (e) return -3;
    return loss ? fetch_loss(c, loss) : 0;
}

int mlp_train_step(mlp_ctx* c, const float* d_X, const float* d_t, int B, float lr, float* loss) {
    if (!c || !d_X || !d_t || check_batch(c, B) || !(lr > 0.f)) return -1;
    if (int r = backward(c, d_X, d_t, B)) return r;
    c->adam_t += 1;
    const float c1 = 1.f - (float)std::pow(0.9, (double)c->adam_t);
    const float c2 = 1.f - (float)std::pow(0.999, (double)c->adam_t);
    k_adam<<<blocks(kNP), kEw, 0, c->stream>>>(c->at<float>(c->lay.p), c->at<float>(c->lay.g),
                                                c->at<float>(c->lay.m), c->at<float>(c->lay.v), kNP, lr, c1, c2);
    refresh(c);
    if (cudaGetLastError()) return -3;
    return loss ? fetch_loss(c, loss) : 0;
}

int mlp_gemm_bf16(const void* d_A, const void* d_B, float* d_C, int M, int N, int K, uint32_t* d_status,
                  void* stream) {
    if (!d_A || !d_B || !d_C || !d_status) return -1;
    return gemm(d_A, d_B, d_C, M, N, K, d_status, (cudaStream_t)stream);
}

int mlp_wait_probe(uint32_t spin_limit, uint32_t* d_status, void* stream) {
    if (!d_status || spin_limit == 0 || spin_limit > (1u << 26)) return -1;
    tcg::k_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(spin_limit, d_status);
    return cuda_status(cudaGetLastError());
}

void mlp_destroy(mlp_ctx* c) { delete c; }

}  // extern "C"
