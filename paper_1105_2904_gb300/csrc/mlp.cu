// Learned drag / torque closure: a small multilayer perceptron trained and evaluated on the
// GPU (the C-ABI lbm_mlp_* of include/lbmp.h). The paper has no network; this is an addition
// that corrects the force and torque a coarse-resolution particle feels.
//
// Precision: weights and activations in bfloat16, products accumulated in FP32 on the tensor
// cores (mma.sync m16n8k16 bf16 -> f32), FP32 master weights and Adam moments, FP32 loss.
// Each layer's output gradient is kept in bfloat16 (it is a tensor-core operand).
//
// Kernels:
//   k_gemm        C[M][N] = sum_k A(m,k) B(k,n) with arbitrary element strides for A and B
//                 (so X W^T, dY W and dY^T X are one kernel), fused epilogue: + bias, relu,
//                 relu' mask, bfloat16 and / or FP32 output; or FP32 split-K partials
//   k_sum_splits  fixed-order sum of split-K partials (weight gradients)
//   k_colsum      fixed-order column sums (bias gradients)
//   k_loss        mean-squared error, its output gradient (bfloat16) and per-block partial sums
//   k_gather      minibatch rows (by index) of the FP32 inputs as bfloat16, and their targets
//   k_adam        Adam on the FP32 masters, refreshing the bfloat16 copies
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "lbmp.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 32, PADK = BK + 8;
constexpr int GEMM_THREADS = 128;

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A;
    long long sam, sak;  // A(m,k) = A[m*sam + k*sak]
    const __nv_bfloat16* B;
    long long sbk, sbn;  // B(k,n) = B[k*sbk + n*sbn]
    const float* bias;   // [N] or null
    int relu;            // 1: max(v, 0)
    const __nv_bfloat16* mask;  // relu' mask: v *= (mask(m,n) > 0), mask(m,n) = mask[m*ldo + n]
    __nv_bfloat16* out16;       // C as bfloat16, out16[m*ldo + n] (or null)
    float* out32;               // C as FP32 (or null)
    long long ldo;
    int ksplit;                 // > 1: blockIdx.z takes K range z; out32 = partials [ksplit][M][N]
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One 64 x 64 output tile per block, four warps of 32 x 32; K in steps of 32 staged in shared
// memory as As[m][k] and Bs[n][k] (zero outside the matrices).
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm(const GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][PADK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][PADK];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    int k_begin = 0, k_end = g.K;
    if (g.ksplit > 1) {
        const int per = ((g.K + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
        k_begin = blockIdx.z * per;
        k_end = min(g.K, k_begin + per);
    }
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = k_begin; k0 < k_end; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += GEMM_THREADS) {
            const int r = e / BK, c = e % BK;
            const int m = m0 + r, k = k0 + c, n = n0 + r;
            As[r][c] = (m < g.M && k < k_end) ? g.A[(long long)m * g.sam + (long long)k * g.sak] : zero;
            Bs[r][c] = (n < g.N && k < k_end) ? g.B[(long long)k * g.sbk + (long long)n * g.sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gq;
                a[i][0] = ld_pair(&As[r][kk + 2 * tq]);
                a[i][1] = ld_pair(&As[r + 8][kk + 2 * tq]);
                a[i][2] = ld_pair(&As[r][kk + 2 * tq + 8]);
                a[i][3] = ld_pair(&As[r + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + gq;
                b[j][0] = ld_pair(&Bs[n][kk + 2 * tq]);
                b[j][1] = ld_pair(&Bs[n][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    // epilogue: c0, c1 at (row gq, cols 2tq, 2tq+1); c2, c3 at row gq + 8
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + i * 16 + gq + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * tq + (q & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][q];
                if (g.ksplit > 1) {
                    g.out32[((long long)blockIdx.z * g.M + m) * g.N + n] = v;
                    continue;
                }
                if (g.bias) v += g.bias[n];
                if (g.relu) v = fmaxf(v, 0.f);
                if (g.mask && !(__bfloat162float(g.mask[(long long)m * g.ldo + n]) > 0.f)) v = 0.f;
                if (g.out16) g.out16[(long long)m * g.ldo + n] = __float2bfloat16(v);
                if (g.out32) g.out32[(long long)m * g.ldo + n] = v;
            }
}

// out[i] = sum over s of part[s][i], s in order.
__global__ void k_sum_splits(const float* __restrict__ part, int splits, long long n, float* __restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + i];
        out[i] = s;
    }
}

// out[n] = sum over rows m of d[m][n] (bfloat16 values, FP32 sum): one block per column,
// a fixed-order tree over the block.
__global__ void k_colsum(const __nv_bfloat16* __restrict__ d, int M, int N, float* __restrict__ out)
{
    __shared__ float part[256];
    const int n = blockIdx.x;
    float s = 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) s += __bfloat162float(d[(long long)m * N + n]);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = part[0];
}

// Mean-squared error over the B x O outputs: d = 2 (y - t) / (B O) as bfloat16, and one FP32
// partial sum of (y - t)^2 per block (block b covers entries b*256 .. b*256 + 255).
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, long long n, float scale,
                       __nv_bfloat16* __restrict__ d, float* __restrict__ partial)
{
    __shared__ float part[256];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float r2 = 0.f;
    if (i < n) {
        const float r = y[i] - t[i];
        d[i] = __float2bfloat16(2.f * r * scale);
        r2 = r * r;
    }
    part[threadIdx.x] = r2;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = part[0];
}

// loss_out[slot] = scale * sum of the partials, in order (one thread).
__global__ void k_loss_total(const float* __restrict__ partial, int nparts, double scale, double* loss_out, int slot)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += (double)partial[i];
    loss_out[slot] += s * scale;
}

// Rows idx[r] of X (FP32, [n][K]) as bfloat16 rows r of Xb, each input standardised as
// (x - shift[c]) * scale[c] when shift / scale are given, and of T ([n][O]) as rows of Tb.
__global__ void k_gather(const float* __restrict__ X, const float* __restrict__ T, const int* __restrict__ idx,
                         int rows, int K, int O, const float* __restrict__ shift, const float* __restrict__ scale,
                         __nv_bfloat16* __restrict__ Xb, float* __restrict__ Tb)
{
    const long long nx = (long long)rows * K, total = nx + (long long)rows * O;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        if (e < nx) {
            const long long r = e / K, c = e % K;
            const long long src = idx ? idx[r] : r;
            float v = X[src * K + c];
            if (shift) v = (v - shift[c]) * scale[c];
            Xb[e] = __float2bfloat16(v);
        } else if (T) {
            const long long f = e - nx, r = f / O, c = f % O;
            const long long src = idx ? idx[r] : r;
            Tb[f] = T[src * O + c];
        }
    }
}

// Adam (Kingma & Ba, 2015) on FP32 masters p with moments m, v; t_dev holds the number of
// steps taken so far (this is step t_dev + 1; k_adam_tick advances it afterwards).
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       long long n, const int* __restrict__ t_dev, float lr, float b1, float b2, float eps,
                       __nv_bfloat16* __restrict__ p16)
{
    const int t = *t_dev + 1;
    const float c1 = 1.f - powf(b1, (float)t);
    const float c2 = 1.f - powf(b2, (float)t);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (p16) p16[i] = __float2bfloat16(pi);
    }
}

__global__ void k_adam_tick(int* t_dev)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t_dev += 1;
}

__global__ void k_to_bf16(const float* __restrict__ a, long long n, __nv_bfloat16* __restrict__ b)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

int blocks_for(long long n, int t = 256) { return (int)std::max<long long>(1, std::min<long long>(4096, (n + t - 1) / t)); }

}  // namespace

struct lbm_mlp {
    int L = 0;
    std::vector<int> sizes;
    cudaStream_t stream = nullptr;
    // parameters, layer-major: W[l] (sizes[l+1] x sizes[l], row-major) then b[l]
    std::vector<long long> w_off, b_off;
    long long nparam = 0;
    float* p = nullptr;   // FP32 masters
    float* m = nullptr;
    float* v = nullptr;
    float* g = nullptr;   // gradients
    __nv_bfloat16* p16 = nullptr;  // bfloat16 copies (W entries used; b entries unused)
    int* t = nullptr;
    // workspace for up to `cap` rows
    int cap = 0;
    __nv_bfloat16* xb = nullptr;
    float* tb = nullptr;
    std::vector<__nv_bfloat16*> h;   // activations of hidden layers
    std::vector<__nv_bfloat16*> d;   // output gradients of every layer
    float* y = nullptr;
    float* partial = nullptr;        // split-K partials and loss partial sums
    size_t partial_floats = 0;
    int* idx = nullptr;
    int idx_cap = 0;
    double* loss_dev = nullptr;
    int loss_cap = 0;
    float* in_shift = nullptr;       // input standardisation (null: none)
    float* in_scale = nullptr;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

lbm_status mfail(lbm_mlp* n, lbm_status s, const std::string& msg)
{
    if (n) n->err = msg;
    return s;
}

#define MK(call)                                                                                              \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return mfail(net, LBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
lbm_status malloc_dev(lbm_mlp* net, T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(16, count * sizeof(T)));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mfail(net, LBM_E_OOM, "cudaMalloc failed");
    }
    net->allocs.push_back(q);
    *p = (T*)q;
    return LBM_OK;
}

void free_dev(lbm_mlp* net, void* p)
{
    if (!p) return;
    auto it = std::find(net->allocs.begin(), net->allocs.end(), p);
    if (it != net->allocs.end()) net->allocs.erase(it);
    cudaFree(p);
}

const int SPLITS = 16;

lbm_status ensure_rows(lbm_mlp* net, int rows)
{
    if (rows <= net->cap) return LBM_OK;
    int cap = 1;
    while (cap < rows) cap <<= 1;
    free_dev(net, net->xb);
    free_dev(net, net->tb);
    free_dev(net, net->y);
    free_dev(net, net->partial);
    for (auto* q : net->h) free_dev(net, q);
    for (auto* q : net->d) free_dev(net, q);
    net->h.assign(net->L - 1, nullptr);
    net->d.assign(net->L, nullptr);
    const int K = net->sizes[0], O = net->sizes[net->L];
    lbm_status s;
    if ((s = malloc_dev(net, &net->xb, (size_t)cap * K)) != LBM_OK) return s;
    if ((s = malloc_dev(net, &net->tb, (size_t)cap * O)) != LBM_OK) return s;
    if ((s = malloc_dev(net, &net->y, (size_t)cap * O)) != LBM_OK) return s;
    for (int l = 0; l + 1 < net->L; ++l)
        if ((s = malloc_dev(net, &net->h[(size_t)l], (size_t)cap * net->sizes[(size_t)l + 1])) != LBM_OK) return s;
    for (int l = 0; l < net->L; ++l)
        if ((s = malloc_dev(net, &net->d[(size_t)l], (size_t)cap * net->sizes[(size_t)l + 1])) != LBM_OK) return s;
    size_t pf = (size_t)(cap * (long long)O + 255) / 256 + 16;
    for (int l = 0; l < net->L; ++l)
        pf = std::max(pf, (size_t)SPLITS * net->sizes[(size_t)l] * net->sizes[(size_t)l + 1]);
    if ((s = malloc_dev(net, &net->partial, pf)) != LBM_OK) return s;
    net->partial_floats = pf;
    net->cap = cap;
    return LBM_OK;
}

void gemm(cudaStream_t s, int M, int N, int K, const __nv_bfloat16* A, long long sam, long long sak,
          const __nv_bfloat16* B, long long sbk, long long sbn, const float* bias, int relu,
          const __nv_bfloat16* mask, __nv_bfloat16* out16, float* out32, long long ldo, int ksplit = 1)
{
    GemmArgs g{M, N, K, A, sam, sak, B, sbk, sbn, bias, relu, mask, out16, out32, ldo, ksplit};
    const dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, ksplit);
    k_gemm<<<grid, GEMM_THREADS, 0, s>>>(g);
}

// Forward pass of `rows` rows already in net->xb; output in net->y (FP32).
void forward(lbm_mlp* net, int rows)
{
    const __nv_bfloat16* in = net->xb;
    for (int l = 0; l < net->L; ++l) {
        const int K = net->sizes[(size_t)l], N = net->sizes[(size_t)l + 1];
        const __nv_bfloat16* W = net->p16 + net->w_off[(size_t)l];
        const float* b = net->p + net->b_off[(size_t)l];
        const bool last = l == net->L - 1;
        gemm(net->stream, rows, N, K, in, K, 1, W, 1, K, b, last ? 0 : 1, nullptr, last ? nullptr : net->h[(size_t)l],
             last ? net->y : nullptr, N);
        if (!last) in = net->h[(size_t)l];
    }
}

// Loss and gradients of `rows` rows in net->xb / net->tb (forward included). The loss is
// added to net->loss_dev[slot] (FP64).
void backward(lbm_mlp* net, int rows, int slot)
{
    const int O = net->sizes[(size_t)net->L];
    const long long n = (long long)rows * O;
    const int lb = (int)((n + 255) / 256);
    forward(net, rows);
    k_loss<<<lb, 256, 0, net->stream>>>(net->y, net->tb, n, 1.f / (float)n, net->d[(size_t)net->L - 1], net->partial);
    k_loss_total<<<1, 32, 0, net->stream>>>(net->partial, lb, 1.0 / (double)n, net->loss_dev, slot);
    for (int l = net->L - 1; l >= 0; --l) {
        const int K = net->sizes[(size_t)l], N = net->sizes[(size_t)l + 1];
        const __nv_bfloat16* din = net->d[(size_t)l];
        const __nv_bfloat16* hin = l == 0 ? net->xb : net->h[(size_t)l - 1];
        // dW[N][K] = d^T h: A(m=j, k=r) = d[r][j], B(k=r, n=c) = h[r][c]; split over the rows
        gemm(net->stream, N, K, rows, din, 1, N, hin, K, 1, nullptr, 0, nullptr, nullptr, net->partial, K, SPLITS);
        k_sum_splits<<<blocks_for((long long)N * K), 256, 0, net->stream>>>(net->partial, SPLITS, (long long)N * K,
                                                                           net->g + net->w_off[(size_t)l]);
        k_colsum<<<N, 256, 0, net->stream>>>(din, rows, N, net->g + net->b_off[(size_t)l]);
        if (l > 0) {
            // d_{l-1} = (d_l W_l) * relu'(h_{l-1}): A = d (rows x N), B(k=j, n=c) = W[j][c]
            const __nv_bfloat16* W = net->p16 + net->w_off[(size_t)l];
            gemm(net->stream, rows, K, N, din, N, 1, W, K, 1, nullptr, 0, net->h[(size_t)l - 1], net->d[(size_t)l - 1],
                 nullptr, K);
        }
    }
}

void adam(lbm_mlp* net, float lr, float b1, float b2, float eps)
{
    k_adam<<<blocks_for(net->nparam), 256, 0, net->stream>>>(net->p, net->m, net->v, net->g, net->nparam, net->t, lr, b1,
                                                              b2, eps, net->p16);
    k_adam_tick<<<1, 32, 0, net->stream>>>(net->t);
}

lbm_status ensure_loss_slots(lbm_mlp* net, int n)
{
    if (n <= net->loss_cap) return LBM_OK;
    free_dev(net, net->loss_dev);
    net->loss_dev = nullptr;
    lbm_status s = malloc_dev(net, &net->loss_dev, (size_t)n);
    if (s != LBM_OK) return s;
    net->loss_cap = n;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_mlp_create(lbm_mlp** out, int nlayers, const int* sizes, void* cuda_stream)
{
    if (!out) return LBM_E_INVALID;
    *out = nullptr;
    if (nlayers < 1 || nlayers > 8 || !sizes) return LBM_E_INVALID;
    for (int l = 0; l <= nlayers; ++l)
        if (sizes[l] < 1 || sizes[l] > 4096) return LBM_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    lbm_mlp* net = new lbm_mlp();
    net->L = nlayers;
    net->sizes.assign(sizes, sizes + nlayers + 1);
    net->stream = (cudaStream_t)cuda_stream;
    long long off = 0;
    for (int l = 0; l < nlayers; ++l) {
        net->w_off.push_back(off);
        off += (long long)sizes[l] * sizes[l + 1];
        net->b_off.push_back(off);
        off += sizes[l + 1];
    }
    net->nparam = off;
    lbm_status s = LBM_OK;
    if ((s = malloc_dev(net, &net->p, (size_t)off)) != LBM_OK || (s = malloc_dev(net, &net->m, (size_t)off)) != LBM_OK ||
        (s = malloc_dev(net, &net->v, (size_t)off)) != LBM_OK || (s = malloc_dev(net, &net->g, (size_t)off)) != LBM_OK ||
        (s = malloc_dev(net, &net->p16, (size_t)off)) != LBM_OK || (s = malloc_dev(net, &net->t, 1)) != LBM_OK) {
        lbm_mlp_destroy(net);
        return s;
    }
    cudaMemsetAsync(net->p, 0, sizeof(float) * off, net->stream);
    cudaMemsetAsync(net->m, 0, sizeof(float) * off, net->stream);
    cudaMemsetAsync(net->v, 0, sizeof(float) * off, net->stream);
    cudaMemsetAsync(net->g, 0, sizeof(float) * off, net->stream);
    cudaMemsetAsync(net->p16, 0, sizeof(__nv_bfloat16) * off, net->stream);
    cudaMemsetAsync(net->t, 0, sizeof(int), net->stream);
    if (cudaStreamSynchronize(net->stream) != cudaSuccess) {
        cudaGetLastError();
        lbm_mlp_destroy(net);
        return LBM_E_CUDA;
    }
    *out = net;
    return LBM_OK;
}

long long lbm_mlp_num_params(const lbm_mlp* net) { return net ? net->nparam : -1; }

lbm_status lbm_mlp_set_params(lbm_mlp* net, const double* params)
{
    if (!net || !params) return LBM_E_INVALID;
    std::vector<float> h((size_t)net->nparam);
    for (long long i = 0; i < net->nparam; ++i) h[(size_t)i] = (float)params[i];
    MK(cudaMemcpyAsync(net->p, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, net->stream));
    k_to_bf16<<<blocks_for(net->nparam), 256, 0, net->stream>>>(net->p, net->nparam, net->p16);
    MK(cudaGetLastError());
    MK(cudaMemsetAsync(net->m, 0, sizeof(float) * net->nparam, net->stream));
    MK(cudaMemsetAsync(net->v, 0, sizeof(float) * net->nparam, net->stream));
    MK(cudaMemsetAsync(net->t, 0, sizeof(int), net->stream));
    MK(cudaStreamSynchronize(net->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_set_input_scaling(lbm_mlp* net, const double* shift, const double* scale)
{
    if (!net || (!shift) != (!scale)) return LBM_E_INVALID;
    const int K = net->sizes[0];
    if (!shift) {
        free_dev(net, net->in_shift);
        free_dev(net, net->in_scale);
        net->in_shift = net->in_scale = nullptr;
        return LBM_OK;
    }
    std::vector<float> h((size_t)2 * K);
    for (int c = 0; c < K; ++c) {
        if (!std::isfinite(shift[c]) || !std::isfinite(scale[c])) return mfail(net, LBM_E_INVALID, "non-finite scaling");
        h[(size_t)c] = (float)shift[c];
        h[(size_t)K + c] = (float)scale[c];
    }
    lbm_status s = LBM_OK;
    if (!net->in_shift && ((s = malloc_dev(net, &net->in_shift, (size_t)K)) != LBM_OK ||
                           (s = malloc_dev(net, &net->in_scale, (size_t)K)) != LBM_OK))
        return s;
    MK(cudaMemcpyAsync(net->in_shift, h.data(), sizeof(float) * K, cudaMemcpyHostToDevice, net->stream));
    MK(cudaMemcpyAsync(net->in_scale, h.data() + K, sizeof(float) * K, cudaMemcpyHostToDevice, net->stream));
    MK(cudaStreamSynchronize(net->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp* net, double* params, double* grads)
{
    if (!net || (!params && !grads)) return LBM_E_INVALID;
    std::vector<float> h((size_t)net->nparam);
    if (params) {
        MK(cudaMemcpyAsync(h.data(), net->p, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, net->stream));
        MK(cudaStreamSynchronize(net->stream));
        for (long long i = 0; i < net->nparam; ++i) params[i] = h[(size_t)i];
    }
    if (grads) {
        MK(cudaMemcpyAsync(h.data(), net->g, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, net->stream));
        MK(cudaStreamSynchronize(net->stream));
        for (long long i = 0; i < net->nparam; ++i) grads[i] = h[(size_t)i];
    }
    return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp* net, const float* x, int rows, float* y)
{
    if (!net || !x || !y || rows < 0) return LBM_E_INVALID;
    if (rows == 0) return LBM_OK;
    lbm_status s = ensure_rows(net, rows);
    if (s != LBM_OK) return s;
    const int K = net->sizes[0], O = net->sizes[(size_t)net->L];
    k_gather<<<blocks_for((long long)rows * K), 256, 0, net->stream>>>(x, nullptr, nullptr, rows, K, O, net->in_shift,
                                                                         net->in_scale, net->xb, nullptr);
    forward(net, rows);
    MK(cudaMemcpyAsync(y, net->y, sizeof(float) * (size_t)rows * O, cudaMemcpyDeviceToDevice, net->stream));
    MK(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_mlp_loss_grad(lbm_mlp* net, const float* x, const float* t, int rows, double* loss)
{
    if (!net || !x || !t || rows < 1) return LBM_E_INVALID;
    lbm_status s = ensure_rows(net, rows);
    if (s == LBM_OK) s = ensure_loss_slots(net, 1);
    if (s != LBM_OK) return s;
    const int K = net->sizes[0], O = net->sizes[(size_t)net->L];
    MK(cudaMemsetAsync(net->loss_dev, 0, sizeof(double), net->stream));
    k_gather<<<blocks_for((long long)rows * (K + O)), 256, 0, net->stream>>>(x, t, nullptr, rows, K, O, net->in_shift,
                                                                               net->in_scale, net->xb, net->tb);
    backward(net, rows, 0);
    MK(cudaGetLastError());
    if (loss) {
        MK(cudaMemcpyAsync(loss, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, net->stream));
        MK(cudaStreamSynchronize(net->stream));
    }
    return LBM_OK;
}

lbm_status lbm_mlp_adam_step(lbm_mlp* net, double lr, double beta1, double beta2, double eps)
{
    if (!net || !(lr > 0.0)) return LBM_E_INVALID;
    adam(net, (float)lr, (float)beta1, (float)beta2, (float)eps);
    MK(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp* net, const float* x, const float* t, int n, int batch, int epochs, double lr,
                         unsigned seed, double* epoch_loss)
{
    if (!net || !x || !t || n < 1 || batch < 1 || epochs < 1 || !(lr > 0.0)) return LBM_E_INVALID;
    batch = std::min(batch, n);
    lbm_status s = ensure_rows(net, batch);
    if (s == LBM_OK) s = ensure_loss_slots(net, epochs);
    if (s != LBM_OK) return s;
    if (net->idx_cap < n) {
        free_dev(net, net->idx);
        net->idx = nullptr;
        if ((s = malloc_dev(net, &net->idx, (size_t)n)) != LBM_OK) return s;
        net->idx_cap = n;
    }
    const int K = net->sizes[0], O = net->sizes[(size_t)net->L];
    MK(cudaMemsetAsync(net->loss_dev, 0, sizeof(double) * epochs, net->stream));
    std::mt19937 rng(seed);
    std::vector<int> perm((size_t)n);
    const int nb = n / batch;  // full minibatches per epoch
    for (int e = 0; e < epochs; ++e) {
        for (int i = 0; i < n; ++i) perm[(size_t)i] = i;
        std::shuffle(perm.begin(), perm.end(), rng);
        MK(cudaMemcpyAsync(net->idx, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, net->stream));
        for (int bi = 0; bi < nb; ++bi) {
            k_gather<<<blocks_for((long long)batch * (K + O)), 256, 0, net->stream>>>(x, t, net->idx + (size_t)bi * batch,
                                                                                      batch, K, O, net->in_shift,
                                                                                      net->in_scale, net->xb, net->tb);
            backward(net, batch, e);
            adam(net, (float)lr, 0.9f, 0.999f, 1e-8f);
        }
        // the host permutation buffer is reused next epoch: wait for its copy
        MK(cudaStreamSynchronize(net->stream));
    }
    MK(cudaGetLastError());
    if (epoch_loss) {
        std::vector<double> h((size_t)epochs);
        MK(cudaMemcpy(h.data(), net->loss_dev, sizeof(double) * epochs, cudaMemcpyDeviceToHost));
        for (int e = 0; e < epochs; ++e) epoch_loss[e] = h[(size_t)e] / nb;
    }
    return LBM_OK;
}

const char* lbm_mlp_last_error(const lbm_mlp* net) { return net ? net->err.c_str() : "null network"; }

void lbm_mlp_destroy(lbm_mlp* net)
{
    if (!net) return;
    if (net->stream) cudaStreamSynchronize(net->stream);
    else cudaDeviceSynchronize();
    for (void* p : net->allocs) cudaFree(p);
    delete net;
}

}  // extern "C"
