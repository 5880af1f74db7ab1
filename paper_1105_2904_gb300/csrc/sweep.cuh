// The fused lattice sweep and its companions, templated on the lattice and the storage
// format. Included by sweep_f64.cu (built with -fmad=false) and sweep_lp.cu.
//
// Pull scheme: buffer `fin` holds the post-collision populations of the previous step at
// the sites where they were computed, so site x gathers f_i(x) = fin_i(x - c_i), or
// fin_opp(i)(x) when x - c_i lies beyond a solid wall (halfway bounce-back, Sec. 3.1).
//
// The IS imposition of the previous step (Eq. 12, "velocity of the internal sites") is
// applied as populations are pulled: a value pulled from a site tagged IS of particle p is
// replaced by f^eq_d(rho_I, u_p + omega_p x r), with rho_I the post-collision density of
// that site, saved by the previous sweep (the "stash"). Only sites inside a particle can
// pull from an IS site (every neighbour of an IS site lies in the particle), so fluid sites
// never look. This removes a separate scattered pass over the IS shell.
#pragma once

#include <type_traits>
#include <utility>

#include "kernels.h"

namespace lbmp {

constexpr int SWEEP_THREADS = 128;

template <int I, int N, class F>
__device__ __forceinline__ void sfor(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, N>(f);
    }
}

// Lever arm r = (x_site - x_p) of site (sx, sy, sz) owned by particle k (Eqs. 5, 7, 12):
// the integer offset from the anchor (minimum image on periodic axes) minus phi.
template <typename C>
__device__ __forceinline__ void lever_arm(const Geom& g, const PKern& k, int sx, int sy, int sz,
                                          C r[3])
{
    const int o0 = wrap_offset(sx - k.K[0], g.nx, !g.wall[0]);
    const int o1 = wrap_offset(sy - k.K[1], g.ny, !g.wall[1]);
    const int o2 = wrap_offset(sz - k.K[2], g.nz, !g.wall[2]);
    r[0] = (C)o0 - (C)k.phi[0];
    r[1] = (C)o1 - (C)k.phi[1];
    r[2] = (C)o2 - (C)k.phi[2];
}

// Rigid-body velocity u_p + omega_p x r (Eq. 5 / Eq. 12, read as a rigid-body motion).
template <typename C>
__device__ __forceinline__ void rigid_velocity(const PKern& k, const C r[3], C out[3])
{
    const C om0 = (C)k.om[0], om1 = (C)k.om[1], om2 = (C)k.om[2];
    out[0] = (C)k.u[0] + (om1 * r[2] - om2 * r[1]);
    out[1] = (C)k.u[1] + (om2 * r[0] - om0 * r[2]);
    out[2] = (C)k.u[2] + (om0 * r[1] - om1 * r[0]);
}

// Equilibrium of direction i, or of opp(i) when sgn < 0 (c_opp = -c_i), at density rho
// (plain form, FP64) or density deviation drho (deviation form, returns f^eq - w).
template <class L, int i>
__device__ __forceinline__ double feq_plain(double sgn, double rho, const double u[3])
{
    double cu = (double)L::c(i, 0) * u[0] + (double)L::c(i, 1) * u[1] + (double)L::c(i, 2) * u[2];
    if (sgn < 0.0) cu = -cu;
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L::w(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

template <class L, int i>
__device__ __forceinline__ float geq_dev(float sgn, float drho, const float u[3])
{
    float cu = (float)L::c(i, 0) * u[0] + (float)L::c(i, 1) * u[1] + (float)L::c(i, 2) * u[2];
    cu *= sgn;
    const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float rho = 1.0f + drho;
    return (float)L::w(i) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

// BGK collision with Guo forcing (Eq. 3), plain FP64 form. The expression order matches a
// direct transcription of the equations so that results are reproducible bit for bit.
template <class L>
__device__ __forceinline__ void collide_plain(double f[], const SweepArgs& a)
{
    constexpr int Q = L::Q;
    double rho = 0.0;
    sfor<0, Q>([&](auto ic) { rho += f[decltype(ic)::value]; });
    double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 3; ++k)
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            j[k] += f[i] * (double)L::c(i, k);
        });
    double u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = (j[k] + 0.5 * a.F[k]) / rho;
    const double pre = a.pre, omega = a.omega;
    const double uF = u[0] * a.F[0] + u[1] * a.F[1] + u[2] * a.F[2];
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const double cu = (double)L::c(i, 0) * u[0] + (double)L::c(i, 1) * u[1] + (double)L::c(i, 2) * u[2];
        const double cF =
            (double)L::c(i, 0) * a.F[0] + (double)L::c(i, 1) * a.F[1] + (double)L::c(i, 2) * a.F[2];
        const double Si = pre * L::w(i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
        f[i] = f[i] - omega * (f[i] - feq_plain<L, i>(1.0, rho, u)) + Si;
    });
}

// BGK collision with Guo forcing on deviations g = f - w (FP32).
template <class L>
__device__ __forceinline__ void collide_dev(float g[], const SweepArgs& a)
{
    constexpr int Q = L::Q;
    float drho = 0.0f, j0 = 0.0f, j1 = 0.0f, j2 = 0.0f;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        drho += g[i];
        if constexpr (L::c(i, 0) != 0) j0 += (float)L::c(i, 0) * g[i];
        if constexpr (L::c(i, 1) != 0) j1 += (float)L::c(i, 1) * g[i];
        if constexpr (L::c(i, 2) != 0) j2 += (float)L::c(i, 2) * g[i];
    });
    const float F0 = (float)a.F[0], F1 = (float)a.F[1], F2 = (float)a.F[2];
    const float rho = 1.0f + drho;
    const float inv = 1.0f / rho;
    const float u[3] = {(j0 + 0.5f * F0) * inv, (j1 + 0.5f * F1) * inv, (j2 + 0.5f * F2) * inv};
    const float omega = (float)a.omega, pre = (float)a.pre;
    const float uF = u[0] * F0 + u[1] * F1 + u[2] * F2;
    const float usq15 = 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float cu = (float)L::c(i, 0) * u[0] + (float)L::c(i, 1) * u[1] + (float)L::c(i, 2) * u[2];
        const float cF = (float)L::c(i, 0) * F0 + (float)L::c(i, 1) * F1 + (float)L::c(i, 2) * F2;
        const float w = (float)L::w(i);
        const float geq = w * (drho + rho * (3.0f * cu + 4.5f * cu * cu - usq15));
        const float Si = pre * w * (3.0f * (cF - uF) + 9.0f * cu * cF);
        g[i] = g[i] - omega * (g[i] - geq) + Si;
    });
}

// Neighbour coordinates of a site along each axis with periodic wrap, and whether the step
// leaves the domain through a wall.
struct Nbr {
    int xm, xp, ym, yp, zm, zp;
    bool bxm, bxp, bym, byp, bzm, bzp;
};

template <bool WALLS>
__device__ __forceinline__ Nbr neighbours(const Geom& g, int x, int y, int z)
{
    Nbr n;
    n.xm = x - 1; n.xp = x + 1; n.ym = y - 1; n.yp = y + 1; n.zm = z - 1; n.zp = z + 1;
    n.bxm = n.bxp = n.bym = n.byp = n.bzm = n.bzp = false;
    if (n.xm < 0) { n.xm += g.nx; if (WALLS) n.bxm = g.wall[0]; }
    if (n.xp >= g.nx) { n.xp -= g.nx; if (WALLS) n.bxp = g.wall[0]; }
    if (n.ym < 0) { n.ym += g.ny; if (WALLS) n.bym = g.wall[1]; }
    if (n.yp >= g.ny) { n.yp -= g.ny; if (WALLS) n.byp = g.wall[1]; }
    if (n.zm < 0) { n.zm += g.nz; if (WALLS) n.bzm = g.wall[2]; }
    if (n.zp >= g.nz) { n.zp -= g.nz; if (WALLS) n.bzp = g.wall[2]; }
    return n;
}

// Source of the population pulled in direction i: site (sx, sy, sz) / index, and whether it
// bounces (then the source is the site itself, direction opp(i)).
template <class L, int i, bool WALLS>
__device__ __forceinline__ void pull_source(const Geom& g, const Nbr& n, int x, int y, int z,
                                            unsigned idx, int& sx, int& sy, int& sz,
                                            unsigned& sidx, bool& bounce)
{
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    sx = cx > 0 ? n.xm : (cx < 0 ? n.xp : x);
    sy = cy > 0 ? n.ym : (cy < 0 ? n.yp : y);
    sz = cz > 0 ? n.zm : (cz < 0 ? n.zp : z);
    bounce = false;
    if constexpr (WALLS)
        bounce = (cx > 0 && n.bxm) || (cx < 0 && n.bxp) || (cy > 0 && n.bym) || (cy < 0 && n.byp) ||
                 (cz > 0 && n.bzm) || (cz < 0 && n.bzp);
    if (bounce) {
        sx = x; sy = y; sz = z;
        sidx = idx;
    } else {
        sidx = ((unsigned)sz * (unsigned)g.ny + (unsigned)sy) * (unsigned)g.nx + (unsigned)sx;
    }
}

// Gathers f_i(x) for all i (pull propagation with bounce-back).
template <class L, typename S, bool WALLS>
__device__ __forceinline__ void pull(const S* __restrict__ fin, const Geom& g, const Nbr& n, int x,
                                     int y, int z, unsigned idx, typename Store<S>::C f[])
{
    using C = typename Store<S>::C;
    const size_t N = g.N;
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        int sx, sy, sz;
        unsigned sidx;
        bool bounce;
        pull_source<L, i, WALLS>(g, n, x, y, z, idx, sx, sy, sz, sidx, bounce);
        const S* p = bounce ? fin + (size_t)L::opp(i) * N + idx : fin + (size_t)i * N + sidx;
        f[i] = Store<S>::load(*p, (C)L::w(i));
    });
}

// Applies the pending IS imposition to the pulled values of a site inside a particle.
template <class L, typename S, bool WALLS>
__device__ __forceinline__ void substitute_is(const Geom& g, const Nbr& n, int x, int y, int z,
                                              unsigned idx, const PartView& pv,
                                              const typename Store<S>::C* __restrict__ stash,
                                              typename Store<S>::C f[])
{
    using C = typename Store<S>::C;
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        int sx, sy, sz;
        unsigned sidx;
        bool bounce;
        pull_source<L, i, WALLS>(g, n, x, y, z, idx, sx, sy, sz, sidx, bounce);
        const unsigned t = pv.tag[sidx];
        if ((t >> 30) == CLS_IS) {
            const PKern& k = pv.pk[t & PID_MASK];
            C r[3], uI[3];
            lever_arm<C>(g, k, sx, sy, sz, r);
            rigid_velocity<C>(k, r, uI);
            const C sgn = bounce ? (C)-1 : (C)1;
            if constexpr (Store<S>::deviation)
                f[i] = geq_dev<L, i>(sgn, stash[sidx], uI);
            else
                f[i] = feq_plain<L, i>(sgn, stash[sidx], uI);
        }
    });
}

template <class L, typename S, bool WALLS, bool PART>
__global__ void __launch_bounds__(SWEEP_THREADS) k_sweep(const SweepArgs a)
{
    using St = Store<S>;
    using C = typename St::C;
    constexpr int Q = L::Q;
    const Geom& g = a.g;
    const int xr = blockIdx.x * SWEEP_THREADS + threadIdx.x;
    const bool valid = xr < g.nx;
    const int x = valid ? xr : g.nx - 1;
    const int y = blockIdx.y, z = blockIdx.z;
    const unsigned idx = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx + (unsigned)x;
    const size_t N = g.N;
    const Nbr n = neighbours<WALLS>(g, x, y, z);

    C f[Q];
    pull<L, S, WALLS>((const S*)a.fin, g, n, x, y, z, idx, f);

    unsigned tagx = TAG_FLUID;
    if constexpr (PART) {
        tagx = a.pv.tag[idx];
        if (tagx != TAG_FLUID && *a.pv.pending)
            substitute_is<L, S, WALLS>(g, n, x, y, z, idx, a.pv, (const C*)a.stash_in, f);
    }

    if constexpr (St::deviation)
        collide_dev<L>(f, a);
    else
        collide_plain<L>(f, a);

    if constexpr (PART) {
        const unsigned cls = tagx >> 30;
        // Particle-fluid momentum transfer at BS sites (Eqs. 5-7).
        C dv[6] = {0, 0, 0, 0, 0, 0};
        const bool isbs = valid && cls == CLS_BS;
        if (isbs) {
            const PKern& k = a.pv.pk[tagx & PID_MASK];
            C r[3], ub[3], ubp[3], du[3];
            lever_arm<C>(g, k, x, y, z, r);
            rigid_velocity<C>(k, r, ubp);
            if constexpr (St::deviation) {
                float drho = 0.0f, j0 = 0.0f, j1 = 0.0f, j2 = 0.0f;
                sfor<0, Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    drho += f[i];
                    if constexpr (L::c(i, 0) != 0) j0 += (float)L::c(i, 0) * f[i];
                    if constexpr (L::c(i, 1) != 0) j1 += (float)L::c(i, 1) * f[i];
                    if constexpr (L::c(i, 2) != 0) j2 += (float)L::c(i, 2) * f[i];
                });
                const float rho = 1.0f + drho;
                ub[0] = j0 / rho; ub[1] = j1 / rho; ub[2] = j2 / rho;
                sfor<0, Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    f[i] = geq_dev<L, i>(1.0f, drho, ubp);
                });
#pragma unroll
                for (int q = 0; q < 3; ++q) du[q] = ubp[q] - ub[q];
                dv[0] = rho * du[0]; dv[1] = rho * du[1]; dv[2] = rho * du[2];
                dv[3] = rho * (r[1] * du[2] - r[2] * du[1]);
                dv[4] = rho * (r[2] * du[0] - r[0] * du[2]);
                dv[5] = rho * (r[0] * du[1] - r[1] * du[0]);
            } else {
                double rhoB = 0.0;
                sfor<0, Q>([&](auto ic) { rhoB += f[decltype(ic)::value]; });
                double jB[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    sfor<0, Q>([&](auto ic) {
                        constexpr int i = decltype(ic)::value;
                        jB[q] += f[i] * (double)L::c(i, q);
                    });
#pragma unroll
                for (int q = 0; q < 3; ++q) ub[q] = jB[q] / rhoB;
                sfor<0, Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    f[i] = feq_plain<L, i>(1.0, rhoB, ubp);
                });
#pragma unroll
                for (int q = 0; q < 3; ++q) du[q] = ubp[q] - ub[q];
                double cr[3];
                cr[0] = r[1] * du[2] - r[2] * du[1];
                cr[1] = r[2] * du[0] - r[0] * du[2];
                cr[2] = r[0] * du[1] - r[1] * du[0];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    dv[q] = rhoB * du[q];
                    dv[3 + q] = rhoB * cr[q];
                }
            }
        }
        // Per-particle sums (Eqs. 8-9).
        if constexpr (St::deviation) {
            // Warp-aggregated: one FP64 atomic per (warp, particle, component).
            const unsigned lane = threadIdx.x & 31u;
            const unsigned pid = tagx & PID_MASK;
            unsigned m = __ballot_sync(0xffffffffu, isbs);
            while (m) {
                const int leader = __ffs(m) - 1;
                const unsigned lp = __shfl_sync(0xffffffffu, pid, leader);
                const bool mine = isbs && pid == lp;
                float v[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    v[q] = mine ? (float)dv[q] : 0.0f;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
                }
                if ((int)lane == leader) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) atomicAdd(&a.acc[(size_t)lp * 6 + q], (double)v[q]);
                }
                m &= ~__ballot_sync(0xffffffffu, mine);
            }
        } else {
            if (isbs) {
#pragma unroll
                for (int q = 0; q < 6; ++q) a.bs_scratch[(size_t)idx * 6 + q] = (double)dv[q];
            }
        }
    }

    if (!valid) return;
    S* __restrict__ fout = (S*)a.fout;
    C dens = (C)0;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const S s = St::save(f[i], (C)L::w(i));
        fout[(size_t)i * N + idx] = s;
        if constexpr (PART) dens += St::load(s, (C)L::w(i));
    });
    if constexpr (PART) {
        // Post-collision density of IS sites, for the IS imposition pulled next step.
        if ((tagx >> 30) == CLS_IS) ((C*)a.stash_out)[idx] = dens;
    }
}

template <class L, typename S, bool WALLS>
__global__ void k_materialize(const MaterializeArgs a)
{
    using St = Store<S>;
    using C = typename St::C;
    constexpr int Q = L::Q;
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.count) return;
    const Geom& g = a.g;
    const unsigned idx = a.s0 + t;
    const int x = (int)(idx % (unsigned)g.nx);
    const int y = (int)((idx / (unsigned)g.nx) % (unsigned)g.ny);
    const int z = (int)(idx / ((unsigned)g.nx * (unsigned)g.ny));
    const Nbr n = neighbours<WALLS>(g, x, y, z);
    C f[Q];
    pull<L, S, WALLS>((const S*)a.fin, g, n, x, y, z, idx, f);
    if (a.pv.tag != nullptr && a.pv.tag[idx] != TAG_FLUID && *a.pv.pending)
        substitute_is<L, S, WALLS>(g, n, x, y, z, idx, a.pv, (const C*)a.stash_in, f);
    double fd[Q];
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        fd[i] = St::deviation ? (double)f[i] + L::w(i) : (double)f[i];
    });
    if (a.mode == 1) {
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            a.out0[(size_t)i * a.count + t] = fd[i];
        });
        return;
    }
    // rho = sum f (Eq. 1); rho u = sum f c + F/2 (Eq. 2 with the Guo half-force).
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    if constexpr (St::deviation) {
        double drho = 0.0;
        sfor<0, Q>([&](auto ic) { drho += (double)f[decltype(ic)::value]; });
        rho = 1.0 + drho;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            sfor<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                j[k] += (double)f[i] * (double)L::c(i, k);
            });
    } else {
        sfor<0, Q>([&](auto ic) { rho += fd[decltype(ic)::value]; });
#pragma unroll
        for (int k = 0; k < 3; ++k)
            sfor<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                j[k] += fd[i] * (double)L::c(i, k);
            });
    }
    a.out0[t] = rho;
#pragma unroll
    for (int k = 0; k < 3; ++k) a.out1[(size_t)t * 3 + k] = (j[k] + 0.5 * a.F[k]) / rho;
}

template <class L, typename S>
__global__ void k_convert_in(const ConvertArgs a)
{
    using St = Store<S>;
    using C = typename St::C;
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.count) return;
    const size_t N = a.g.N;
    S* dst = (S*)a.dst;
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const double v = a.f[(size_t)i * a.count + t];
        if constexpr (St::deviation)
            dst[(size_t)i * N + a.s0 + t] = St::save((C)(v - L::w(i)), (C)L::w(i));
        else
            dst[(size_t)i * N + a.s0 + t] = St::save((C)v, (C)L::w(i));
    });
}

// dst_j(s) = src_j(s + c_j), or src_opp(j)(s) when s + c_j lies beyond a wall: pulling
// from dst then returns exactly the populations held in src.
template <class L, typename S>
__global__ void k_unstream(const UnstreamArgs a)
{
    const Geom& g = a.g;
    const size_t N = g.N;
    const S* src = (const S*)a.src;
    S* dst = (S*)a.dst;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += gridDim.x * blockDim.x) {
        const int x = (int)(idx % (unsigned)g.nx);
        const int y = (int)((idx / (unsigned)g.nx) % (unsigned)g.ny);
        const int z = (int)(idx / ((unsigned)g.nx * (unsigned)g.ny));
        sfor<0, L::Q>([&](auto ic) {
            constexpr int j = decltype(ic)::value;
            int t[3] = {x + L::c(j, 0), y + L::c(j, 1), z + L::c(j, 2)};
            const int nn[3] = {g.nx, g.ny, g.nz};
            bool out = false;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (t[k] < 0 || t[k] >= nn[k]) {
                    if (g.wall[k]) out = true;
                    t[k] = (t[k] + nn[k]) % nn[k];
                }
            }
            const unsigned tidx = ((unsigned)t[2] * (unsigned)g.ny + (unsigned)t[1]) * (unsigned)g.nx + (unsigned)t[0];
            dst[(size_t)j * N + idx] = out ? src[(size_t)L::opp(j) * N + idx] : src[(size_t)j * N + tidx];
        });
    }
}

template <class L, typename S>
__global__ void k_fill_rest(S* dst, unsigned N)
{
    using St = Store<S>;
    using C = typename St::C;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        sfor<0, L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            dst[(size_t)i * N + idx] = St::save(St::deviation ? (C)0 : (C)L::w(i), (C)L::w(i));
        });
    }
}

// Post-collision density at the new IS sites of particles whose shift changed (their IS
// sites may not have been IS, hence not saved, during the sweep).
template <class L, typename S>
__global__ void k_stash_fix(const StashFixArgs a)
{
    using St = Store<S>;
    using C = typename St::C;
    const int nlist = a.cnt->nchanged;
    const size_t N = a.g.N;
    const S* fout = (const S*)a.fout;
    C* stash = (C*)a.stash_out;
    for (int b = blockIdx.x; b < nlist; b += gridDim.x) {
        const int p = a.list[b];
        const PConst pc = a.pc[p];
        const PKern& k = a.pk[p];
        for (int e = threadIdx.x; e < pc.tmpl_n; e += blockDim.x) {
            const int ent = a.tmpl[pc.tmpl_off + e];
            if (tmpl_cls(ent) != CLS_IS) continue;
            unsigned site;
            if (!site_of(a.g, k.K, tmpl_ox(ent), tmpl_oy(ent), tmpl_oz(ent), site)) continue;
            C s = (C)0;
            sfor<0, L::Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                s += St::load(fout[(size_t)i * N + site], (C)L::w(i));
            });
            stash[site] = s;
        }
    }
}

// ---- launchers --------------------------------------------------------------------------
template <class L, typename S>
void launch_sweep_l(const SweepArgs& a, cudaStream_t s)
{
    const dim3 grid((a.g.nx + SWEEP_THREADS - 1) / SWEEP_THREADS, a.g.ny, a.g.nz);
    const bool walls = a.g.wall[0] || a.g.wall[1] || a.g.wall[2];
    const bool part = a.pv.tag != nullptr;
    if (walls && part) k_sweep<L, S, true, true><<<grid, SWEEP_THREADS, 0, s>>>(a);
    else if (walls) k_sweep<L, S, true, false><<<grid, SWEEP_THREADS, 0, s>>>(a);
    else if (part) k_sweep<L, S, false, true><<<grid, SWEEP_THREADS, 0, s>>>(a);
    else k_sweep<L, S, false, false><<<grid, SWEEP_THREADS, 0, s>>>(a);
}

template <typename S>
void launch_sweep(const SweepArgs& a, cudaStream_t s)
{
    if (a.lattice == 0) launch_sweep_l<D2Q9, S>(a, s);
    else launch_sweep_l<D3Q19, S>(a, s);
}

template <typename S>
void launch_materialize(const MaterializeArgs& a, cudaStream_t s)
{
    const unsigned blocks = (a.count + 255) / 256;
    const bool walls = a.g.wall[0] || a.g.wall[1] || a.g.wall[2];
    if (a.lattice == 0) {
        if (walls) k_materialize<D2Q9, S, true><<<blocks, 256, 0, s>>>(a);
        else k_materialize<D2Q9, S, false><<<blocks, 256, 0, s>>>(a);
    } else {
        if (walls) k_materialize<D3Q19, S, true><<<blocks, 256, 0, s>>>(a);
        else k_materialize<D3Q19, S, false><<<blocks, 256, 0, s>>>(a);
    }
}

template <typename S>
void launch_convert_in(const ConvertArgs& a, cudaStream_t s)
{
    const unsigned blocks = (a.count + 255) / 256;
    if (a.lattice == 0) k_convert_in<D2Q9, S><<<blocks, 256, 0, s>>>(a);
    else k_convert_in<D3Q19, S><<<blocks, 256, 0, s>>>(a);
}

template <typename S>
void launch_unstream(const UnstreamArgs& a, cudaStream_t s)
{
    const unsigned blocks = (unsigned)(((size_t)a.g.N + 255) / 256 < 65536 ? ((size_t)a.g.N + 255) / 256 : 65536);
    if (a.lattice == 0) k_unstream<D2Q9, S><<<blocks, 256, 0, s>>>(a);
    else k_unstream<D3Q19, S><<<blocks, 256, 0, s>>>(a);
}

template <typename S>
void launch_fill_rest(int lattice, void* dst, unsigned N, cudaStream_t s)
{
    const unsigned blocks = (unsigned)(((size_t)N + 255) / 256 < 65536 ? ((size_t)N + 255) / 256 : 65536);
    if (lattice == 0) k_fill_rest<D2Q9, S><<<blocks, 256, 0, s>>>((S*)dst, N);
    else k_fill_rest<D3Q19, S><<<blocks, 256, 0, s>>>((S*)dst, N);
}

template <typename S>
void launch_stash_fix(const StashFixArgs& a, cudaStream_t s)
{
    if (a.lattice == 0) k_stash_fix<D2Q9, S><<<256, 128, 0, s>>>(a);
    else k_stash_fix<D3Q19, S><<<256, 128, 0, s>>>(a);
}

template <typename S>
const KernelTable* make_table()
{
    static const KernelTable t = {launch_sweep<S>,     launch_materialize<S>, launch_convert_in<S>,
                                  launch_unstream<S>,  launch_fill_rest<S>,   launch_stash_fix<S>,
                                  (int)sizeof(S),      (int)sizeof(typename Store<S>::C)};
    return &t;
}

}  // namespace lbmp
