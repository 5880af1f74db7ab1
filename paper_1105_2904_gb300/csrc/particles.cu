// Particle phase of one step, FP64 throughout (built with -fmad=false so that the
// arithmetic is evaluated exactly as written):
//   reduction of the exchanged momentum in a fixed order (FP64 storage mode only),
//   acceleration (Eqs. 10-11), hard-core contacts (Sec. 2.3, Eqs. 16-19; predicted-overlap
//   trigger, pairs processed in (i, j) order), position update (Eq. 13) and the integer
//   shift of each site set (Eqs. 14-15), then the incremental re-marking of the owner map
//   for the particles whose shift changed and their neighbours.
#include <algorithm>

#include "kernels.h"

namespace lbmp {

namespace {

constexpr int PT = 128;  // threads per block of the per-particle kernels

__device__ inline void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// Arguments of the simulation a block works on: the kernel parameter for a single context,
// entry blockIdx.y of a device array for a batch of cells (each entry's pointers address
// that cell's own arrays, so particle and site indices stay local to the cell).
template <bool B>
__device__ __forceinline__ ParticleArgs cell_args(const ParticleArgs& a0, const ParticleArgs* __restrict__ cells)
{
    if constexpr (B)
        return cells[blockIdx.y];
    else
        return a0;
}

// Per-step clearing of the work-list counters, the contact cell counts and cursors, and the
// re-stamp flags.
template <bool B>
__global__ void k_phase_clear(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, T = gridDim.x * blockDim.x;
    if (t0 == 0) *a.cnt = Counters{0, 0, 0, 0};
    for (int i = t0; i < a.cg.total; i += T) {
        a.cell_count[i] = 0;
        a.cell_cursor[i] = 0;
    }
    for (int i = t0; i < a.np; i += T) {
        a.restamp_flag[i] = 0;
        a.pk_prev[i] = a.pk[i];
        a.pkf_prev[i] = a.pkf[i];
    }
    if (t0 == 0) *a.pending_prev = *a.pending;
}

// d - n floor(d/n + 1/2). For |d| < n/4, d/n + 1/2 lies in (1/4, 3/4) whatever the
// rounding, so the floor is 0 and the result is d itself: skip the FP64 division.
__device__ inline double min_image(double d, int n, bool periodic)
{
    if (!periodic) return d;
    const double q = 0.25 * (double)n;
    if (d > -q && d < q) return d;
    return d - (double)n * floor(d / (double)n + 0.5);
}

__device__ inline int axis_len(const Geom& g, int k) { return k == 0 ? g.nx : (k == 1 ? g.ny : g.nz); }

__device__ inline bool periodic_axis(const Geom& g, int k, int D) { return k < D && !g.wall[k]; }

// Fixed-order sums of the per-site momentum exchange of each particle (Eqs. 8-9) over the
// sites it owns as BS, in template order (z, y, x lexicographic offsets). FP64 mode: one
// thread per particle, strictly sequential, the order a direct implementation uses.
template <bool B>
__global__ void k_reduce_ordered(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const PConst pc = a.pc[p];
    const int Kw[3] = {a.pk[p].Kw[0], a.pk[p].Kw[1], a.pk[p].Kw[2]};
    const unsigned code = (CLS_BS << 30) | (unsigned)p;
    const double* sc = (const double*)a.bs_scratch;
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int e = 0; e < pc.n_bs; ++e) {
        const int ent = a.tmpl[pc.tmpl_off + e];
        unsigned site;
        if (!site_fast(a.g, Kw, tmpl_ox(ent), tmpl_oy(ent), tmpl_oz(ent), site)) continue;
        if (a.tag[site] != code) continue;
#pragma unroll
        for (int q = 0; q < 6; ++q) s[q] += sc[(size_t)site * 6 + q];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) a.acc[(size_t)p * 6 + q] = s[q];
}

// FP32 modes: one block of RT threads per particle. Thread t sums entries t, t + RT, ... in
// FP32 (loads of four entries in flight), then a fixed tree combines the threads
// (deterministic), and the total is stored in FP64. A site's 16-byte record holds dp and the
// owner tag it was written under; the torque dl = r x dp (Eq. 7) is formed here, with
// r = o - phi from the entry's template offset o (the sweep's lever arm). A record counts when
// its tag is this particle's BS code: the sweep rewrites the record of every BS site each
// step, and a site that stops being a BS site of its particle has the tag word of its record
// cleared at that moment (k_mark_clear, stamp_particle), so a matching record is this step's.
// The records sit at their sites' indices, so a particle's ~890 come from as many scattered
// sectors; 128 threads per block measured faster than 256 or 512.
constexpr int RT = 128;
template <bool B>
__global__ void __launch_bounds__(RT) k_reduce_block(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    __shared__ float part[RT / 32][6];
    const int p = blockIdx.x;
    if (p >= a.np) return;
    const PConst pc = a.pc[p];
    const int Kw[3] = {a.pk[p].Kw[0], a.pk[p].Kw[1], a.pk[p].Kw[2]};
    const float phi[3] = {a.pkf[p].phi[0], a.pkf[p].phi[1], a.pkf[p].phi[2]};
    const unsigned code = (CLS_BS << 30) | (unsigned)p;
    const float4* sc = (const float4*)a.bs_scratch;
    float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int e0 = threadIdx.x; e0 < pc.n_bs; e0 += 4 * RT) {
        unsigned site[4];
        int ent[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * RT;
            ok[u] = false;
            ent[u] = 0;
            if (e < pc.n_bs) {
                ent[u] = a.tmpl[pc.tmpl_off + e];
                int v[3];
                ok[u] = site_fast_xyz(a.g, Kw, tmpl_ox(ent[u]), tmpl_oy(ent[u]), tmpl_oz(ent[u]), site[u], v);
                if (a.rec_brick) site[u] = rec_brick_index(a.g, v[0], v[1], v[2]);
            }
        }
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = ok[u] ? sc[site[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (ok[u] && __float_as_uint(v[u].w) == code) {
                const float r0 = (float)tmpl_ox(ent[u]) - phi[0];
                const float r1 = (float)tmpl_oy(ent[u]) - phi[1];
                const float r2 = (float)tmpl_oz(ent[u]) - phi[2];
                s[0] += v[u].x;
                s[1] += v[u].y;
                s[2] += v[u].z;
                s[3] += r1 * v[u].z - r2 * v[u].y;
                s[4] += r2 * v[u].x - r0 * v[u].z;
                s[5] += r0 * v[u].y - r1 * v[u].x;
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
        if (lane == 0) part[warp][q] = s[q];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float tot = 0.f;
        for (int w = 0; w < RT / 32; ++w) tot += part[w][threadIdx.x];
        a.acc[(size_t)p * 6 + threadIdx.x] = (double)tot;
    }
}

// Clears the tag word of the float4 BS record of site (index site, coordinates v) when the site
// stops being a BS site of the particle that wrote it (the FP64 mode checks the owner map
// instead).
__device__ inline void drop_record(const ParticleArgs& a, unsigned site, const int v[3])
{
    if (a.scratch_f64) return;
    const unsigned ri = a.rec_brick ? rec_brick_index(a.g, v[0], v[1], v[2]) : site;
    ((unsigned*)a.bs_scratch)[(size_t)ri * 4 + 3] = TAG_FLUID;
}

// Contact-grid cell of a centre coordinate. FP32 is enough: the cell only selects which
// pairs are tested (the tests themselves are FP64), and cells are at least 2 r_max + gap + 4
// wide, two sites more than the widest reach of a pair within one step, which absorbs the
// FP32 rounding of the coordinate by orders of magnitude (GB300's FP64 pipe is narrow, and
// the FP64 divisions here dominated the kernel).
__device__ inline int cell_coord(const ParticleArgs& a, int k, double x)
{
    const int n = axis_len(a.g, k);
    const int D = a.lattice == 0 ? 2 : 3;
    if (k >= D) return 0;
    float v;
    const float xf = (float)x;
    if (a.g.wall[k]) {
        v = xf + 0.5f;
    } else {
        v = xf - (float)n * floorf(xf / (float)n);
    }
    int c = (int)floorf(v / (float)a.cg.size[k]);
    if (c < 0) c = 0;
    if (c >= a.cg.n[k]) c = a.cg.n[k] - 1;
    return c;
}

// Eqs. 10-11 (+ external increment), force/torque output, cell of the current centre.
template <bool B>
__global__ void k_accel(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    // every load before the first store (see k_move)
    const PConst pc = a.pc[p];
    PKern& k = a.pk[p];
    double d[6], u[3], om[3], x[3];
#pragma unroll
    for (int q = 0; q < 6; ++q) d[q] = a.acc[(size_t)p * 6 + q];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        u[q] = k.u[q];
        om[q] = k.om[q];
        x[q] = a.x[(size_t)p * 3 + q];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        a.acc[(size_t)p * 6 + q] = 0.0;
        a.force[(size_t)p * 6 + q] = -d[q];
    }
    float xp[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double un = (u[q] - d[q] * pc.inv_m) + pc.ext[q];
        a.un[(size_t)p * 3 + q] = un;
        k.om[q] = om[q] - d[3 + q] * pc.inv_I;
        xp[q] = (float)(x[q] + un);
    }
    a.xpf[p] = make_float4(xp[0], xp[1], xp[2], (float)pc.r);
    const int c0 = cell_coord(a, 0, x[0]);
    const int c1 = cell_coord(a, 1, x[1]);
    const int c2 = cell_coord(a, 2, x[2]);
    const int c = (c2 * a.cg.n[1] + c1) * a.cg.n[0] + c0;
    a.cell_of[p] = c;
    atomicAdd(&a.cell_count[c], 1);
}

// Exclusive scan of the cell counts (one block of 1024 threads). The counts go through shared
// memory in tiles of 8192: one coalesced load per tile, each thread scans 8 consecutive counts,
// the threads' totals are scanned with warp shuffles, and the starts are written back
// coalesced, with a carry from tile to tile (few dependent global-memory round trips, where a
// thread walking a chunk of the counts serially would pay one per count).
constexpr int SCAN_T = 1024, SCAN_E = 8, SCAN_TILE = SCAN_T * SCAN_E;
template <bool B>
__global__ void __launch_bounds__(SCAN_T) k_cell_scan(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    __shared__ int tile[SCAN_TILE];
    __shared__ int wsum[SCAN_T / 32];
    __shared__ int carry_s;
    const int n = a.cg.total;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < n; base += SCAN_TILE) {
        for (int i = t; i < SCAN_TILE; i += SCAN_T) tile[i] = base + i < n ? a.cell_count[base + i] : 0;
        __syncthreads();
        int v[SCAN_E], sum = 0;
#pragma unroll
        for (int k = 0; k < SCAN_E; ++k) {
            v[k] = tile[t * SCAN_E + k];
            sum += v[k];
        }
        // inclusive scan of the thread sums: within the warp, then across warps
        int incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int carry = carry_s;
        int run = carry + (warp > 0 ? wsum[warp - 1] : 0) + incl - sum;
#pragma unroll
        for (int k = 0; k < SCAN_E; ++k) {
            tile[t * SCAN_E + k] = run;
            run += v[k];
        }
        __syncthreads();
        for (int i = t; i < SCAN_TILE && base + i < n; i += SCAN_T) a.cell_start[base + i] = tile[i];
        if (t == SCAN_T - 1) carry_s = carry + wsum[31];
        __syncthreads();
    }
    if (t == 0) a.cell_start[n] = carry_s;
}

template <bool B>
__global__ void k_cell_fill(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const int c = a.cell_of[p];
    a.cell_items[a.cell_start[c] + atomicAdd(&a.cell_cursor[c], 1)] = p;
}

// Distinct neighbouring cell coordinates along one axis (1 to 3 of them).
__device__ inline int nbr_cells(const ParticleArgs& a, int k, int c, int out[3])
{
    const int n = a.cg.n[k];
    if (n == 1) { out[0] = 0; return 1; }
    if (n == 2) { out[0] = 0; out[1] = 1; return 2; }
    int m = 0;
    for (int d = -1; d <= 1; ++d) {
        int v = c + d;
        if (v < 0 || v >= n) {
            if (a.g.wall[k]) continue;
            v = (v + n) % n;
        }
        out[m++] = v;
    }
    return m;
}

// Candidate pairs (i < j) whose predicted centres overlap: |(x_i+u_i')-(x_j+u_j')| < r_i+r_j+gap.
// One thread per (particle, neighbouring cell): up to 27 threads per particle.
template <bool B>
__global__ void k_pairs(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / 27, cn = t % 27;
    if (i >= a.np) return;
    const int D = a.lattice == 0 ? 2 : 3;
    const int c = a.cell_of[i];
    const int cc[3] = {c % a.cg.n[0], (c / a.cg.n[0]) % a.cg.n[1], c / (a.cg.n[0] * a.cg.n[1])};
    int lx[3], ly[3], lz[3];
    const int nxc = nbr_cells(a, 0, cc[0], lx), nyc = nbr_cells(a, 1, cc[1], ly),
              nzc = nbr_cells(a, 2, cc[2], lz);
    const int xx = cn % 3, yy = (cn / 3) % 3, zz = cn / 9;
    if (xx >= nxc || yy >= nyc || zz >= nzc) return;
    const int cell = (lz[zz] * a.cg.n[1] + ly[yy]) * a.cg.n[0] + lx[xx];
    if (!LBM_DCHECK(a.status, cell >= 0 && cell < a.cg.total)) return;
    const int s0 = a.cell_start[cell], s1 = a.cell_start[cell + 1];
    if (s0 == s1) return;
    const double ri = a.pc[i].r;
    double xi[3], ui[3];
    for (int k = 0; k < 3; ++k) {
        xi[k] = a.x[(size_t)i * 3 + k];
        ui[k] = a.un[(size_t)i * 3 + k];
    }
    const float4 fi = a.xpf[i];
    for (int s = s0; s < s1; ++s) {
        const int j = a.cell_items[s];
        if (!LBM_DCHECK(a.status, j >= 0 && j < a.np)) continue;
        if (j <= i) continue;
        // FP32 pre-test on the predicted centres: pairs clearly apart skip the FP64 test (GB300's
        // FP64 pipe is narrow). The margin, half a site plus 1e-6 of the coordinates, is far
        // above the FP32 rounding of the coordinates (6e-8 of them).
        {
            const float4 fj = a.xpf[j];
            const float dd[3] = {fj.x - fi.x, fj.y - fi.y, fj.z - fi.z};
            float d2f = 0.0f;
            for (int k = 0; k < 3; ++k) {
                float v = dd[k];
                if (periodic_axis(a.g, k, D)) {
                    const float n = (float)axis_len(a.g, k);
                    v -= n * rintf(v / n);
                }
                d2f += v * v;
            }
            const float big = fmaxf(fmaxf(fmaxf(fabsf(fi.x), fabsf(fi.y)), fabsf(fi.z)),
                                    fmaxf(fmaxf(fabsf(fj.x), fabsf(fj.y)), fabsf(fj.z)));
            const float mg = 0.5f + 1e-6f * big;
            const float Rf = fi.w + fj.w + (float)a.gap + mg;
            if (d2f > Rf * Rf) continue;
        }
        double d2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            double pd = (a.x[(size_t)j * 3 + k] + a.un[(size_t)j * 3 + k]) - (xi[k] + ui[k]);
            pd = min_image(pd, axis_len(a.g, k), periodic_axis(a.g, k, D));
            d2 += pd * pd;
        }
        const double R = ri + a.pc[j].r + a.gap;
        if (d2 < R * R) {
            const int slot = atomicAdd(&a.cnt->npairs, 1);
            if (slot < a.pair_cap)
                a.pairs[slot] = ((unsigned long long)i << 32) | (unsigned long long)j;
            else
                set_status(a.status, ERR_CAPACITY);
        }
    }
}

// One block: sort the candidate pairs and resolve them serially in (i, j) order.
template <bool B>
__global__ void k_resolve(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    extern __shared__ unsigned long long keys[];
    const int D = a.lattice == 0 ? 2 : 3;
    const int T = blockDim.x;
    int n = a.cnt->npairs;
    if (n > a.pair_cap) n = 0;  // over capacity: status already set, contacts skipped
    int m = 1;
    while (m < n) m <<= 1;
    for (int t = threadIdx.x; t < m; t += T) keys[t] = t < n ? a.pairs[t] : ~0ull;
    __syncthreads();
    // bitonic sort of m keys
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < m; t += T) {
                const int u = t ^ stride;
                if (u > t) {
                    const bool up = (t & size) == 0;
                    const unsigned long long kt = keys[t], ku = keys[u];
                    if ((kt > ku) == up) {
                        keys[t] = ku;
                        keys[u] = kt;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < n; ++q) {
            const int i = (int)(keys[q] >> 32), j = (int)(keys[q] & 0xffffffffu);
            if (!LBM_DCHECK(a.status, i >= 0 && i < a.np && j >= 0 && j < a.np)) continue;
            const double ai = a.pc[i].inv_m, aj = a.pc[j].inv_m;
            const double den = ai + aj;
            if (den == 0.0) continue;
            double d[3], nn[3];
            for (int k = 0; k < 3; ++k)
                d[k] = min_image(a.x[(size_t)j * 3 + k] - a.x[(size_t)i * 3 + k], axis_len(a.g, k),
                                 periodic_axis(a.g, k, D));
            const double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (dn == 0.0) continue;
            for (int k = 0; k < 3; ++k) nn[k] = d[k] / dn;
            double* ui = &a.un[(size_t)i * 3];
            double* uj = &a.un[(size_t)j * 3];
            const double w = (uj[0] - ui[0]) * nn[0] + (uj[1] - ui[1]) * nn[1] + (uj[2] - ui[2]) * nn[2];
            if (!(w < 0.0)) continue;
            const double ci = 2.0 * ai * w / den;
            const double cj = 2.0 * aj * w / den;
            for (int k = 0; k < 3; ++k) {
                ui[k] = ui[k] + ci * nn[k];
                uj[k] = uj[k] - cj * nn[k];
            }
        }
    }
}

// Orientation of a particle after one step (the rigid-body integration of Sec. 2.2, beside
// Eq. 13 for the position): the unit quaternion q = (w, x, y, z) turned by theta = |omega|
// about omega / |omega| (space frame), omega the angular velocity after this step's
// acceleration (Eq. 11) held over dt = 1: q' = dq q, dq = (cos(theta/2), sin(theta/2)
// omega/|omega|), then divided by its norm. FP64, evaluated as written (-fmad=false).
__device__ __forceinline__ void rotate_orientation(double* q, const double om[3])
{
    const double t2 = om[0] * om[0] + om[1] * om[1] + om[2] * om[2];  // theta^2
    if (t2 == 0.0) return;
    double c, sn;  // cos(theta / 2) and sin(theta / 2) / theta
    if (t2 < 1e-4) {
        // below theta = 0.01 (every suspension here turns by far less per step) their Taylor
        // series in theta^2 to the third order; the first term left out is below 1e-23, and GB300's
        // narrow FP64 pipe spends most of this kernel on cos, sin and the division otherwise
        c = 1.0 + t2 * (-1.0 / 8.0 + t2 * (1.0 / 384.0 + t2 * (-1.0 / 46080.0)));
        sn = 0.5 + t2 * (-1.0 / 48.0 + t2 * (1.0 / 3840.0 + t2 * (-1.0 / 645120.0)));
    } else {
        const double th = sqrt(t2);
        c = cos(0.5 * th);
        sn = sin(0.5 * th) / th;
    }
    const double d[4] = {c, sn * om[0], sn * om[1], sn * om[2]};
    const double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    double r[4];
    r[0] = d[0] * q0 - (d[1] * q1 + d[2] * q2 + d[3] * q3);
    r[1] = d[0] * q1 + q0 * d[1] + (d[2] * q3 - d[3] * q2);
    r[2] = d[0] * q2 + q0 * d[2] + (d[3] * q1 - d[1] * q3);
    r[3] = d[0] * q3 + q0 * d[3] + (d[1] * q2 - d[2] * q1);
    const double nrm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int k = 0; k < 4; ++k) q[k] = r[k] / nrm;
}

// Walls, position update (Eq. 13), new shifts (Eqs. 14-15) and the list of particles whose
// shift changed; one thread per particle.
template <bool B>
__global__ void k_move(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int D = a.lattice == 0 ? 2 : 3;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) *a.pending = 1;
    if (p < a.np) {
        // Every load first: the stores below may alias them as far as the compiler knows,
        // and interleaved they would wait for one memory round trip each.
        const PConst pc = a.pc[p];
        PKern& k = a.pk[p];
        double* ug = &a.un[(size_t)p * 3];
        double* xg = &a.x[(size_t)p * 3];
        double* qg = &a.q[(size_t)p * 4];
        double u[3] = {ug[0], ug[1], ug[2]};
        double x[3] = {xg[0], xg[1], xg[2]};
        const double om[3] = {k.om[0], k.om[1], k.om[2]};
        const int K0[3] = {k.K[0], k.K[1], k.K[2]};
        int K[3] = {K0[0], K0[1], K0[2]};
        int Kw[3] = {k.Kw[0], k.Kw[1], k.Kw[2]};
        double qv[4] = {qg[0], qg[1], qg[2], qg[3]};
        if (pc.inv_m != 0.0) {
            const double R = pc.r + a.gap;
            for (int d = 0; d < D; ++d) {
                if (!a.g.wall[d]) continue;
                const double xp = x[d] + u[d];
                const double lo = xp + 0.5;
                const double hi = ((double)axis_len(a.g, d) - 0.5) - xp;
                if (lo < R && u[d] < 0.0)
                    u[d] = -u[d];
                else if (hi < R && u[d] > 0.0)
                    u[d] = -u[d];
            }
        }
        bool changed = false;
        for (int d = 0; d < D; ++d) {
            x[d] = x[d] + u[d];
            const int s = (int)floor((x[d] - pc.x0[d]) + 0.5);
            const int Kn = pc.A[d] + s;
            const int dK = Kn - K[d];
            if (dK != 0) changed = true;
            if (dK > 1 || dK < -1) set_status(a.status, ERR_UNSTABLE);
            K[d] = Kn;
            const int n = axis_len(a.g, d);
            Kw[d] = a.g.wall[d] ? Kn : ((Kn % n) + n) % n;
        }
        rotate_orientation(qv, om);
        for (int d = 0; d < 3; ++d) {
            ug[d] = u[d];
            xg[d] = x[d];
            k.u[d] = u[d];
            a.Kold[(size_t)p * 3 + d] = K0[d];
            k.K[d] = K[d];
            k.Kw[d] = Kw[d];
        }
        for (int c = 0; c < 4; ++c) qg[c] = qv[c];
        PKernF& kf = a.pkf[p];
        for (int d = 0; d < 3; ++d) {
            kf.u[d] = (float)u[d];
            kf.om[d] = (float)om[d];
            kf.Kw[d] = Kw[d];
        }
        if (changed) a.changed[atomicAdd(&a.cnt->nchanged, 1)] = p;
    }
}

__device__ inline void add_restamp(const ParticleArgs& a, int q)
{
    if (atomicExch(&a.restamp_flag[q], 1) == 0) a.restamp[atomicAdd(&a.cnt->nrestamp, 1)] = q;
}

// Particles whose site sets may meet the old or new set of a moved particle.
template <bool B>
__global__ void k_mark_neighbours(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.cnt->nchanged) return;
    const int D = a.lattice == 0 ? 2 : 3;
    const int p = a.changed[t];
    add_restamp(a, p);
    const int c = a.cell_of[p];
    const int cc[3] = {c % a.cg.n[0], (c / a.cg.n[0]) % a.cg.n[1], c / (a.cg.n[0] * a.cg.n[1])};
    int lx[3], ly[3], lz[3];
    const int nxc = nbr_cells(a, 0, cc[0], lx), nyc = nbr_cells(a, 1, cc[1], ly),
              nzc = nbr_cells(a, 2, cc[2], lz);
    const double rp = a.pc[p].r;
    double cold[3], cnew[3];
    for (int k = 0; k < 3; ++k) {
        cold[k] = (double)a.Kold[(size_t)p * 3 + k] + a.pk[p].phi[k];
        cnew[k] = (double)a.pk[p].K[k] + a.pk[p].phi[k];
    }
    for (int zz = 0; zz < nzc; ++zz)
        for (int yy = 0; yy < nyc; ++yy)
            for (int xx = 0; xx < nxc; ++xx) {
                const int cell = (lz[zz] * a.cg.n[1] + ly[yy]) * a.cg.n[0] + lx[xx];
                for (int s = a.cell_start[cell]; s < a.cell_start[cell + 1]; ++s) {
                    const int q = a.cell_items[s];
                    if (!LBM_DCHECK(a.status, q >= 0 && q < a.np)) continue;
                    if (q == p) continue;
                    const double R = rp + a.pc[q].r + 1.0;
                    double d2o = 0.0, d2n = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        const double cq = (double)a.pk[q].K[k] + a.pk[q].phi[k];
                        const double dd0 = min_image(cold[k] - cq, axis_len(a.g, k), periodic_axis(a.g, k, D));
                        const double dd1 = min_image(cnew[k] - cq, axis_len(a.g, k), periodic_axis(a.g, k, D));
                        d2o += dd0 * dd0;
                        d2n += dd1 * dd1;
                    }
                    if (d2o <= R * R || d2n <= R * R) add_restamp(a, q);
                }
            }
}

// Releases the sites a moved particle owned at its old anchor.
template <bool B>
__global__ void k_mark_clear(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int nlist = a.cnt->nchanged;
    for (int b = blockIdx.x; b < nlist; b += gridDim.x) {
        const int p = a.changed[b];
        const PConst pc = a.pc[p];
        const int K[3] = {a.Kold[(size_t)p * 3], a.Kold[(size_t)p * 3 + 1], a.Kold[(size_t)p * 3 + 2]};
        int Kw[3];
        wrap_anchor(a.g, K, Kw);
        for (int e = threadIdx.x; e < pc.tmpl_n; e += blockDim.x) {
            const int ent = a.tmpl[pc.tmpl_off + e];
            unsigned site;
            int v[3];
            if (!site_fast_xyz(a.g, Kw, tmpl_ox(ent), tmpl_oy(ent), tmpl_oz(ent), site, v)) continue;
            const unsigned t = a.tag[site];
            if (t != TAG_FLUID && (t & PID_MASK) == (unsigned)p) {
                a.tag[site] = TAG_FLUID;
                if ((t >> 30) == CLS_BS) drop_record(a, site, v);
            }
        }
    }
}

// Claims the sites of a particle at its current anchor; the lowest code wins.
__device__ inline void stamp_particle(const ParticleArgs& a, int p)
{
    const PConst pc = a.pc[p];
    const int Kw[3] = {a.pk[p].Kw[0], a.pk[p].Kw[1], a.pk[p].Kw[2]};
    for (int e = threadIdx.x; e < pc.tmpl_n; e += blockDim.x) {
        const int ent = a.tmpl[pc.tmpl_off + e];
        unsigned site;
        int v[3];
        if (!site_fast_xyz(a.g, Kw, tmpl_ox(ent), tmpl_oy(ent), tmpl_oz(ent), site, v)) continue;
        const unsigned code = (tmpl_cls(ent) << 30) | (unsigned)p;
        const unsigned old = atomicMin(&a.tag[site], code);
        // a BS site taken over by a lower code is no longer its particle's BS site
        if (code < old && (old >> 30) == CLS_BS) drop_record(a, site, v);
    }
}

template <bool B>
__global__ void k_mark_stamp(const ParticleArgs a0, const ParticleArgs* __restrict__ cells)
{
    const ParticleArgs a = cell_args<B>(a0, cells);
    if (a.np == 0) return;  // a cell of a batch without particles
    const int nlist = a.cnt->nrestamp;
    for (int b = blockIdx.x; b < nlist; b += gridDim.x) stamp_particle(a, a.restamp[b]);
}

__global__ void k_stamp_all(const ParticleArgs a)
{
    for (int b = blockIdx.x; b < a.np; b += gridDim.x) stamp_particle(a, b);
}

int mark_grid() { return 304; }

// x, u, omega, -dP, -dL of every particle as five [np][3] blocks of out, then the device
// status word (as a double) in out[15 np].
__global__ void k_pack_particles(const ParticleArgs a, double* out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t np = (size_t)a.np;
    if (p == 0) out[15 * np] = (double)*a.status;
    if (p >= a.np) return;
    for (int k = 0; k < 3; ++k) {
        out[0 * 3 * np + (size_t)p * 3 + k] = a.x[(size_t)p * 3 + k];
        out[1 * 3 * np + (size_t)p * 3 + k] = a.pk[p].u[k];
        out[2 * 3 * np + (size_t)p * 3 + k] = a.pk[p].om[k];
        out[3 * 3 * np + (size_t)p * 3 + k] = a.force[(size_t)p * 6 + k];
        out[4 * 3 * np + (size_t)p * 3 + k] = a.force[(size_t)p * 6 + 3 + k];
    }
}

template <bool B>
int particle_phase_a(const ParticleArgs& a0, const ParticleArgs* cells, const PhaseShape& sh, cudaStream_t s)
{
    const int nc = sh.ncells;
    const dim3 gp((sh.max_np + PT - 1) / PT, nc);
    k_phase_clear<B><<<dim3(std::max(1, std::min(64, (std::max(sh.max_np, sh.max_cells) + 255) / 256)), nc), 256, 0, s>>>(
        a0, cells);
    if (sh.scratch_f64)
        k_reduce_ordered<B><<<gp, PT, 0, s>>>(a0, cells);
    else
        k_reduce_block<B><<<dim3(sh.max_np, nc), RT, 0, s>>>(a0, cells);
    k_accel<B><<<gp, PT, 0, s>>>(a0, cells);
    k_cell_scan<B><<<dim3(1, nc), SCAN_T, 0, s>>>(a0, cells);
    k_cell_fill<B><<<gp, PT, 0, s>>>(a0, cells);
    k_pairs<B><<<dim3((sh.max_np * 27 + PT - 1) / PT, nc), PT, 0, s>>>(a0, cells);
    const size_t smem = sizeof(unsigned long long) * (size_t)sh.pair_cap;
    const int rthreads = std::min(1024, std::max(32, (sh.pair_cap + 31) / 32 * 32));
    k_resolve<B><<<dim3(1, nc), rthreads, smem, s>>>(a0, cells);
    k_move<B><<<gp, PT, 0, s>>>(a0, cells);
    k_mark_neighbours<B><<<gp, PT, 0, s>>>(a0, cells);
    return 9;
}

template <bool B>
int particle_phase_b(const ParticleArgs& a0, const ParticleArgs* cells, const PhaseShape& sh, cudaStream_t s)
{
    const int nc = sh.ncells;
    const int per_cell = std::max(2, mark_grid() / nc);
    k_mark_clear<B><<<dim3(per_cell, nc), 256, 0, s>>>(a0, cells);
    k_mark_stamp<B><<<dim3(per_cell, nc), 256, 0, s>>>(a0, cells);
    return 2;
}

PhaseShape single_shape(const ParticleArgs& a)
{
    PhaseShape sh{};
    sh.ncells = 1;
    sh.max_np = a.np;
    sh.max_cells = a.cg.total;
    sh.pair_cap = a.pair_cap;
    sh.scratch_f64 = a.scratch_f64;
    return sh;
}

}  // namespace

int launch_particle_phase_a(const ParticleArgs& a, cudaStream_t s)
{
    return particle_phase_a<false>(a, nullptr, single_shape(a), s);
}

int launch_particle_phase_b(const ParticleArgs& a, cudaStream_t s)
{
    return particle_phase_b<false>(a, nullptr, single_shape(a), s);
}

int launch_particle_phase_batch_a(const ParticleArgs* cells, const PhaseShape& sh, cudaStream_t s)
{
    return particle_phase_a<true>(ParticleArgs{}, cells, sh, s);
}

int launch_particle_phase_batch_b(const ParticleArgs* cells, const PhaseShape& sh, cudaStream_t s)
{
    return particle_phase_b<true>(ParticleArgs{}, cells, sh, s);
}

void launch_pack_particles(const ParticleArgs& a, double* out, cudaStream_t s)
{
    k_pack_particles<<<(a.np + PT - 1) / PT, PT, 0, s>>>(a, out);
}

__global__ void k_wall_advance(WallVel* wv, int* pending)
{
    const int t = threadIdx.x;
    if (t < 18) {
        wv[0].u[t / 3][t % 3] = wv[1].u[t / 3][t % 3];
        wv[0].uf[t / 3][t % 3] = wv[1].uf[t / 3][t % 3];
    }
    if (t == 0) *pending = 1;
}

void launch_wall_advance(WallVel* wv, int* pending, cudaStream_t s)
{
    k_wall_advance<<<1, 32, 0, s>>>(wv, pending);
}

void launch_stamp_all(const ParticleArgs& a, cudaStream_t s)
{
    k_stamp_all<<<mark_grid(), 256, 0, s>>>(a);
}

cudaError_t prepare_particle_kernels(int pair_cap)
{
    const int bytes = (int)(sizeof(unsigned long long) * (size_t)pair_cap);
    cudaError_t e = cudaFuncSetAttribute(k_resolve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_resolve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace lbmp
