// State diagnostics (lbm_diagnostics in include/lbmp.h): totals of mass and momentum, the
// largest speed and the number of sites whose moments are not finite, at the current step
// boundary. The moments are those lbm_get_fields returns (rho = sum f, u = (sum f c + F/2) / rho
// of the pulled populations with the pending IS imposition and wall momentum), in either
// streaming scheme. The sums run in a fixed order (per-thread strided partials, a fixed tree per
// block, then the blocks in index order), so the result does not depend on scheduling.
#include <cmath>

#include "ctx.h"
#include "sweep.cuh"

using namespace lbmp;
using namespace lbmp::host;

namespace {

constexpr int DIAG_BLOCKS = 1216;  // 8 blocks per SM on 152 SMs
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_VALUES = 6;     // mass, momentum x, y, z, max |u|, non-finite sites

template <class L, typename S, bool WALLS>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(const MaterializeArgs a, double* __restrict__ part)
{
    __shared__ double sh[DIAG_VALUES][DIAG_THREADS];
    double acc[DIAG_VALUES] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride) {
        double rho, u[3];
        site_moments<L, S, WALLS>(a, idx, rho, u);
        if (!(isfinite(rho) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
            acc[5] += 1.0;
            continue;
        }
        acc[0] += rho;
        for (int k = 0; k < 3; ++k) acc[1 + k] += rho * u[k];
        acc[4] = fmax(acc[4], sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    }
    for (int q = 0; q < DIAG_VALUES; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int h = DIAG_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            for (int q = 0; q < DIAG_VALUES; ++q) {
                const double o = sh[q][threadIdx.x + h];
                sh[q][threadIdx.x] = q == 4 ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < DIAG_VALUES) part[(size_t)blockIdx.x * DIAG_VALUES + threadIdx.x] = sh[threadIdx.x][0];
}

// One thread per value, the blocks' partials in block order.
__global__ void k_diag_final(const double* __restrict__ part, double* __restrict__ out)
{
    const int q = threadIdx.x;
    if (q >= DIAG_VALUES) return;
    double t = 0.0;
    for (int b = 0; b < DIAG_BLOCKS; ++b) {
        const double v = part[(size_t)b * DIAG_VALUES + q];
        t = q == 4 ? fmax(t, v) : t + v;
    }
    out[q] = t;
}

template <class L, typename S>
void launch_diag_l(const MaterializeArgs& a, double* part, double* out, cudaStream_t s)
{
    const bool walls = a.g.wall[0] || a.g.wall[1] || a.g.wall[2];
    if (walls) k_diag_partial<L, S, true><<<DIAG_BLOCKS, DIAG_THREADS, 0, s>>>(a, part);
    else k_diag_partial<L, S, false><<<DIAG_BLOCKS, DIAG_THREADS, 0, s>>>(a, part);
    k_diag_final<<<1, 32, 0, s>>>(part, out);
}

template <typename S>
void launch_diag(const MaterializeArgs& a, double* part, double* out, cudaStream_t s)
{
    if (a.lattice == 0) launch_diag_l<D2Q9, S>(a, part, out, s);
    else launch_diag_l<D3Q19, S>(a, part, out, s);
}

}  // namespace

extern "C" {

lbm_status lbm_diagnostics(lbm_ctx* ctx, double out[7])
{
    if (!ctx || !out) return LBM_E_INVALID;
    CS(ensure_alloc(ctx));
    CS(sync_status(ctx));
    MaterializeArgs a{};
    a.lattice = ctx->lattice;
    a.g = ctx->g;
    a.fin = ctx->f[ctx->inplace ? 0 : ctx->cur];
    a.aa = ctx->inplace ? ctx->cur : 0;
    a.is_rho = ctx->inplace ? ctx->is_rho[ctx->cur] : nullptr;
    a.pv = part_view(ctx);
    for (int k = 0; k < 3; ++k) a.F[k] = ctx->F[k];
    wall_args(ctx, a);
    double* part = ctx->staging;                              // [DIAG_BLOCKS][6]
    double* dout = ctx->staging + (size_t)DIAG_BLOCKS * DIAG_VALUES;
    switch (ctx->precision) {
    case LBM_FP64: launch_diag<double>(a, part, dout, ctx->stream); break;
    case LBM_FP32: launch_diag<float>(a, part, dout, ctx->stream); break;
    case LBM_FP16DEV: launch_diag<__half>(a, part, dout, ctx->stream); break;
    default: launch_diag<__nv_bfloat16>(a, part, dout, ctx->stream); break;
    }
    CK(cudaGetLastError());
    double v[DIAG_VALUES];
    CK(cudaMemcpyAsync(v, dout, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < 5; ++q) out[q] = v[q];
    out[5] = v[4] * std::sqrt(3.0);  // lattice Mach number: c_s = 1 / sqrt(3)
    out[6] = v[5];
    if (v[5] > 0.0)
        return fail(ctx, LBM_E_NAN, std::to_string((long long)v[5]) + " sites with non-finite density or velocity");
    return LBM_OK;
}

}  // extern "C"
