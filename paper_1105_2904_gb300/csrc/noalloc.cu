// lbm_bs_exchange_noalloc: the boundary-site momentum exchange and its per-particle sums
// for callers that cannot allocate device memory (see include/lbmp.h).
//
// The per-particle accumulators live in a file-scope device array of fixed size instead of
// memory obtained from cudaMalloc. Host code cannot use that array's name as a device
// address, so its address is looked up with cudaGetSymbolAddress once per device (on the
// first call made with that device current) and handed to the kernels.
#include <mutex>

#include "kernels.h"
#include "lbmp.h"
#include "sweep.cuh"

namespace {

using namespace lbmp;

// Every GPU that loads the library holds this array (3 MiB) until the process exits.
static __device__ __align__(256) double g_noalloc_acc[(size_t)LBM_NOALLOC_MAX_PARTICLES * 6];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_acc_addr[kMaxDevices] = {nullptr};

struct ExchangeArgs {
    Geom g;
    const float* gdev;       // [Q][N] deviations f - w at the start of the step
    const unsigned* tags;    // [N] owner map
    int n;
    const double* centers;   // [n][3] centre of each particle's site set
    const double* vel;       // [n][3]
    const double* omega;     // [n][3]
    float F[3];
    double* acc;             // [n][6] accumulators (the static array)
};

__global__ void k_noalloc_clear(double* acc, int count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) acc[i] = 0.0;
}

// One site per thread. At a BS site of particle p: the forced collision keeps rho and adds F
// to the momentum, so the post-collision density and momentum are rho and j + F; the site
// takes the rigid-body velocity u_p + omega_p x r (Eq. 5) and hands the fluid
// dp = rho u' - (j + F) (Eq. 6) and dl = r x dp (Eq. 7), summed per particle (Eqs. 8-9).
template <class L>
__global__ void __launch_bounds__(128) k_noalloc_exchange(const ExchangeArgs a)
{
    constexpr int Q = L::Q;
    const Geom& g = a.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool valid = x < g.nx;
    const unsigned idx = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx + (unsigned)(valid ? x : 0);
    const unsigned t = valid ? a.tags[idx] : TAG_FLUID;
    const unsigned pid = t & PID_MASK;
    const bool bs = valid && (t >> 30) == CLS_BS && pid < (unsigned)a.n;
    float dv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (bs) {
        float drho = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const float v = a.gdev[(size_t)i * g.N + idx];
            drho += v;
            if constexpr (L::c(i, 0) != 0) j0 += (float)L::c(i, 0) * v;
            if constexpr (L::c(i, 1) != 0) j1 += (float)L::c(i, 1) * v;
            if constexpr (L::c(i, 2) != 0) j2 += (float)L::c(i, 2) * v;
        });
        const float rho = 1.0f + drho;
        const int s[3] = {x, y, z};
        const int nn[3] = {g.nx, g.ny, g.nz};
        float r[3], u[3], om[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double d = (double)s[k] - a.centers[(size_t)pid * 3 + k];
            if (!g.wall[k] && k < L::D) d -= (double)nn[k] * floor(d / (double)nn[k] + 0.5);
            r[k] = (float)d;
            u[k] = (float)a.vel[(size_t)pid * 3 + k];
            om[k] = (float)a.omega[(size_t)pid * 3 + k];
        }
        const float ub[3] = {u[0] + (om[1] * r[2] - om[2] * r[1]), u[1] + (om[2] * r[0] - om[0] * r[2]),
                             u[2] + (om[0] * r[1] - om[1] * r[0])};
        const float pB[3] = {j0 + a.F[0], j1 + a.F[1], j2 + a.F[2]};
#pragma unroll
        for (int k = 0; k < 3; ++k) dv[k] = rho * ub[k] - pB[k];
        dv[3] = r[1] * dv[2] - r[2] * dv[1];
        dv[4] = r[2] * dv[0] - r[0] * dv[2];
        dv[5] = r[0] * dv[1] - r[1] * dv[0];
    }
    // Lanes of a warp that share a particle add their values first; one FP64 atomic per
    // (warp, particle, component).
    const unsigned lane = threadIdx.x & 31u;
    unsigned m = __ballot_sync(0xffffffffu, bs);
    while (m) {
        const int leader = __ffs(m) - 1;
        const unsigned lp = __shfl_sync(0xffffffffu, pid, leader);
        const bool mine = bs && pid == lp;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float v = mine ? dv[q] : 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if ((int)lane == leader) atomicAdd(&a.acc[(size_t)lp * 6 + q], (double)v);
        }
        m &= ~__ballot_sync(0xffffffffu, mine);
    }
}

__global__ void k_noalloc_finish(const double* acc, int n, double* force, double* torque)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            force[(size_t)p * 3 + k] = -acc[(size_t)p * 6 + k];
            torque[(size_t)p * 3 + k] = -acc[(size_t)p * 6 + 3 + k];
        }
}

// Address of the static accumulator array on the current device, looked up once per device
// ordinal and kept for the life of the process (a device reset, which would move the array,
// is not supported after the first call on that device).
lbm_status accumulator_address(double** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LBM_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_acc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_acc) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_E_CUDA;
        }
        g_acc_addr[dev] = (double*)p;
    }
    *out = g_acc_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_bs_exchange_noalloc(int lattice, int nx, int ny, int nz, const int walls[3],
                                              const double body_force[3], const float* g,
                                              const unsigned* tags, int n, const double* centers,
                                              const double* velocities, const double* omegas, double* force,
                                              double* torque, void* cuda_stream)
{
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) return LBM_E_INVALID;
    if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535 || (lattice == LBM_D2Q9 && nz != 1))
        return LBM_E_INVALID;
    if ((unsigned long long)nx * ny * nz >= (1ull << 31)) return LBM_E_INVALID;
    if (n < 0 || n > LBM_NOALLOC_MAX_PARTICLES) return LBM_E_INVALID;
    if (!g || !tags || (n > 0 && (!centers || !velocities || !omegas || !force || !torque))) return LBM_E_INVALID;
    if (n == 0) return LBM_OK;
    // An error left by earlier work is not this call's: report it without clearing it, and
    // launch nothing, so that every error read after a launch below belongs to that launch.
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_E_CUDA;
    double* acc = nullptr;
    const lbm_status st = accumulator_address(&acc);
    if (st != LBM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    ExchangeArgs a{};
    a.g.nx = nx;
    a.g.ny = ny;
    a.g.nz = nz;
    for (int k = 0; k < 3; ++k) {
        a.g.wall[k] = walls ? (walls[k] ? 1 : 0) : 0;
        a.F[k] = body_force ? (float)body_force[k] : 0.0f;
    }
    if (lattice == LBM_D2Q9) {
        a.g.wall[2] = 0;
        a.F[2] = 0.0f;
    }
    a.g.N = (unsigned)((unsigned long long)nx * ny * nz);
    a.gdev = g;
    a.tags = tags;
    a.n = n;
    a.centers = centers;
    a.vel = velocities;
    a.omega = omegas;
    a.acc = acc;
    k_noalloc_clear<<<(6 * n + 255) / 256, 256, 0, s>>>(acc, 6 * n);
    if (cudaGetLastError() != cudaSuccess) return LBM_E_CUDA;
    const dim3 grid((nx + 127) / 128, ny, nz);
    if (lattice == LBM_D2Q9)
        k_noalloc_exchange<D2Q9><<<grid, 128, 0, s>>>(a);
    else
        k_noalloc_exchange<D3Q19><<<grid, 128, 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return LBM_E_CUDA;
    k_noalloc_finish<<<(n + 127) / 128, 128, 0, s>>>(acc, n, force, torque);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}
