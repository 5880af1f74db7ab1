// Shared definitions of the CUDA path: lattice velocity sets, storage formats, the owner
// (tag) encoding and the device-side particle records.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmp {

// ---- lattice velocity sets (D2Q9 of Fig. 1; D3Q19 for 3D) --------------------------------
// Velocity order is part of the C-ABI (include/lbmp.h).
struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    __host__ __device__ static constexpr int c(int i, int k)
    {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        return t[i][k];
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    __host__ __device__ static constexpr int c(int i, int k)
    {
        constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[i][k];
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// ---- storage formats -------------------------------------------------------------------
// double : f itself (FP64 arithmetic).
// float  : g = f - w_i (FP32 arithmetic on deviations).
// half / bfloat16 : h = (f - w_i) / w_i, converted to g = h * w_i for FP32 arithmetic.
template <typename S> struct Store;
template <> struct Store<double> {
    using C = double;
    static constexpr bool deviation = false;
    __device__ static double load(double v, double) { return v; }
    __device__ static double save(double v, double) { return v; }
};
template <> struct Store<float> {
    using C = float;
    static constexpr bool deviation = true;
    __device__ static float load(float v, float) { return v; }
    __device__ static float save(float v, float) { return v; }
};
template <> struct Store<__half> {
    using C = float;
    static constexpr bool deviation = true;
    __device__ static float load(__half v, float w) { return __half2float(v) * w; }
    __device__ static __half save(float g, float w) { return __float2half_rn(g * (1.0f / w)); }
};
template <> struct Store<__nv_bfloat16> {
    using C = float;
    static constexpr bool deviation = true;
    __device__ static float load(__nv_bfloat16 v, float w) { return __bfloat162float(v) * w; }
    __device__ static __nv_bfloat16 save(float g, float w)
    {
        return __float2bfloat16_rn(g * (1.0f / w));
    }
};

// ---- owner map ---------------------------------------------------------------------------
// tag = (class << 30) | particle id; the lowest value owns a site (IS < BS < IN < fluid).
constexpr unsigned CLS_IS = 0u;
constexpr unsigned CLS_BS = 1u;
constexpr unsigned CLS_IN = 2u;
constexpr unsigned TAG_FLUID = 0xFFFFFFFFu;
constexpr unsigned PID_MASK = (1u << 30) - 1u;

// Template entry: int8 offsets (x, y, z) from floor(x_p0) and the class, packed in 32 bits.
__host__ __device__ inline int tmpl_ox(int e) { return (int)(signed char)(e & 0xFF); }
__host__ __device__ inline int tmpl_oy(int e) { return (int)(signed char)((e >> 8) & 0xFF); }
__host__ __device__ inline int tmpl_oz(int e) { return (int)(signed char)((e >> 16) & 0xFF); }
__host__ __device__ inline unsigned tmpl_cls(int e) { return (unsigned)((e >> 24) & 0x3); }
inline int tmpl_pack(int ox, int oy, int oz, unsigned cls)
{
    return (int)((unsigned)(ox & 0xFF) | ((unsigned)(oy & 0xFF) << 8) | ((unsigned)(oz & 0xFF) << 16) |
                 (cls << 24));
}

// ---- particle records ----------------------------------------------------------------------
// What the sweep needs of each particle (read-only there; written by the particle phase).
struct __align__(16) PKern {
    double u[3];   // translational velocity u_p
    double om[3];  // angular velocity omega_p
    double phi[3]; // x_p0 - floor(x_p0): lever arm of offset o is o - phi
    int K[3];      // anchor floor(x_p0) + shift: site of offset o is K + o
    int Kw[3];     // K wrapped into [0, n) on periodic axes (= K on wall axes)
};

// FP32 copy of the same record for the reduced-precision sweeps (no FP64 conversions in
// the hot loop), refreshed by the particle phase every step.
struct __align__(16) PKernF {
    float u[3];
    float om[3];
    float phi[3];
    int Kw[3];
};

// Lever-arm offset of site coordinate s from a wrapped anchor kw (|o| < n/2 is guaranteed
// by the particle-size check): minimum image without a division.
__device__ __forceinline__ int offset_from_wrapped(int s, int kw, int n, bool periodic)
{
    int o = s - kw;
    if (periodic) {
        const int h = n / 2;
        if (o < -h) o += n;
        else if (o >= n - h) o -= n;
    }
    return o;
}

// Constants of each particle.
struct __align__(16) PConst {
    double x0[3];  // centre when added
    double r, inv_m, inv_I;
    double ext[3]; // external velocity increment per step (buoyant gravity, body force)
    int A[3];      // floor(x0)
    int tmpl_off;  // first template entry; entries are grouped BS, IS, then interior, each
                   // group in z, y, x lexicographic order of the offsets
    int tmpl_n;    // number of template entries
    int n_bs;      // entries [tmpl_off, tmpl_off + n_bs) are BS
    int n_is;      // the next n_is entries are IS
};

// Device status word values (mirrors lbm_status codes).
constexpr int ERR_CAPACITY = 8;
constexpr int ERR_UNSTABLE = 9;
constexpr int ERR_BOUNDS = 10;

// Index checks of the bounds-checked build (compiled with -DLBM_DEBUG): an index that is out
// of range records ERR_BOUNDS in the device status word (the first fault wins) and the caller
// skips or redirects the access; nothing traps. In the normal build the checks compile to
// nothing (true).
#ifdef LBM_DEBUG
__device__ __forceinline__ bool debug_check(int* status, bool ok)
{
    if (!ok && status) atomicCAS(status, 0, ERR_BOUNDS);
    return ok;
}
#define LBM_DCHECK(status, ok) ::lbmp::debug_check((status), (ok))
#else
#define LBM_DCHECK(status, ok) true
#endif

// Per-step work-list sizes, cleared at the start of every particle phase.
struct Counters {
    int npairs;
    int nchanged;
    int nrestamp;
    int pad;
};

// Tangential velocity of each wall face (-x,+x,-y,+y,-z,+z), in FP64 and FP32.
struct WallVel {
    double u[6][3];
    float uf[6][3];
};

struct Geom {
    int nx, ny, nz;
    int wall[3];     // 1 = halfway bounce-back walls on both ends of the axis
    unsigned N;      // number of sites
    int eqface;      // bit f: face f (-x,+x,-y,+y,-z,+z) imposes its velocity by equilibrium
};

// Index of the FP32 BS record of site (x, y, z). FP32 storage keeps the 16-byte records in
// bricks of 2 x 2 x 2 sites (2 x 2 x 1 in 2D): a sphere's records then share more DRAM pages
// than in rows of the whole box, and the per-particle sums read them faster (512^3 suspension:
// 0.247 -> 0.221 ms per step). The 16-bit storages keep the records at the site index: the
// index arithmetic costs their instruction-bound sweep more than that.
__host__ __device__ __forceinline__ unsigned rec_brick_index(const Geom& g, int x, int y, int z)
{
    const int zb = g.nz > 1 ? 1 : 0;
    const unsigned bx = (unsigned)(g.nx + 1) >> 1, by = (unsigned)(g.ny + 1) >> 1;
    const unsigned brick = ((unsigned)(z >> zb) * by + (unsigned)(y >> 1)) * bx + (unsigned)(x >> 1);
    return (brick << (2 + zb)) | (((unsigned)z & (unsigned)zb) << 2) | (((unsigned)y & 1u) << 1) | ((unsigned)x & 1u);
}
__host__ __device__ __forceinline__ size_t rec_brick_count(const Geom& g)
{
    const int zb = g.nz > 1 ? 1 : 0;
    return ((size_t)((g.nx + 1) >> 1) * (size_t)((g.ny + 1) >> 1) * (size_t)((g.nz + zb) >> zb)) << (2 + zb);
}

// Everything the sweep and the getters read of the particle side.
struct PartView {
    const unsigned* tag;  // owner map [N] (nullptr when there are no particles)
    const PKern* pk;      // [np]
    const PKernF* pkf;    // [np] FP32 copy
    const int* pending;   // 1: the IS imposition of the previous step is still to apply
    // Per-site mask of pull directions whose source is an IS site of the site's own owner
    // (bit i), and bit 31 when some source is an IS site of another particle.
    const unsigned* ismask;
    int np;                   // particles (index checks of the LBM_DEBUG build)
    int* status;              // device status word (the same)
};

constexpr unsigned MASK_OTHER = 1u << 31;

__device__ inline int wrap_offset(int o, int n, bool periodic)
{
    if (!periodic) return o;
    o %= n;
    const int h = n / 2;
    if (o < -h) o += n;
    else if (o >= n - h) o -= n;
    return o;
}

// Anchor wrapped into [0, n) on periodic axes (once per particle).
__device__ __forceinline__ void wrap_anchor(const Geom& g, const int K[3], int Kw[3])
{
    const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k) Kw[k] = g.wall[k] ? K[k] : ((K[k] % n[k]) + n[k]) % n[k];
}

// Site index of offset o of a particle with wrapped anchor Kw (|o| < n on periodic axes, so
// one correction suffices); false when the site lies beyond a wall.
__device__ __forceinline__ bool site_fast(const Geom& g, const int Kw[3], int ox, int oy, int oz,
                                          unsigned& idx)
{
    int v[3] = {Kw[0] + ox, Kw[1] + oy, Kw[2] + oz};
    const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (v[k] < 0) {
            if (g.wall[k]) return false;
            v[k] += n[k];
        } else if (v[k] >= n[k]) {
            if (g.wall[k]) return false;
            v[k] -= n[k];
        }
    }
    idx = ((unsigned)v[2] * (unsigned)g.ny + (unsigned)v[1]) * (unsigned)g.nx + (unsigned)v[0];
    return true;
}

// Same, also returning the site's coordinates.
__device__ __forceinline__ bool site_fast_xyz(const Geom& g, const int Kw[3], int ox, int oy, int oz,
                                              unsigned& idx, int v[3])
{
    v[0] = Kw[0] + ox;
    v[1] = Kw[1] + oy;
    v[2] = Kw[2] + oz;
    const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (v[k] < 0) {
            if (g.wall[k]) return false;
            v[k] += n[k];
        } else if (v[k] >= n[k]) {
            if (g.wall[k]) return false;
            v[k] -= n[k];
        }
    }
    idx = ((unsigned)v[2] * (unsigned)g.ny + (unsigned)v[1]) * (unsigned)g.nx + (unsigned)v[0];
    return true;
}

// Site index of offset o of a particle anchored at K; false when it lies beyond a wall.
__device__ __forceinline__ bool site_of(const Geom& g, const int K[3], int ox, int oy, int oz,
                                        unsigned& idx)
{
    int v[3] = {K[0] + ox, K[1] + oy, K[2] + oz};
    const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (g.wall[k]) {
            if (v[k] < 0 || v[k] >= n[k]) return false;
        } else {
            v[k] %= n[k];
            if (v[k] < 0) v[k] += n[k];
        }
    }
    idx = ((unsigned)v[2] * (unsigned)g.ny + (unsigned)v[1]) * (unsigned)g.nx + (unsigned)v[0];
    return true;
}

}  // namespace lbmp
