// The fused lattice sweep and its companions, templated on the lattice and the storage
// format. Included by sweep_f64.cu (built with -fmad=false) and sweep_f32.cu, sweep_f16.cu,
// sweep_bf16.cu.
//
// Pull scheme: buffer `fin` holds the post-collision populations of the previous step at
// the sites where they were computed, so site x gathers f_i(x) = fin_i(x - c_i), or
// fin_opp(i)(x) when x - c_i lies beyond a solid wall (halfway bounce-back, Sec. 3.1).
//
// The IS imposition of the previous step (Eq. 12, "velocity of the internal sites") is
// applied as populations are pulled: a value pulled from a site tagged IS of particle p is
// replaced by f^eq_d(rho_I, u_p + omega_p x r), with rho_I the post-collision density of
// that site. Only sites inside a particle can pull from an IS site (every neighbour of an IS
// site lies in the particle), so fluid sites never look. This removes a separate scattered
// pass over the IS shell.
//
// Density carry: since no pull uses the populations of an IS site raw, the sweep stores an
// IS site's post-collision density rho_I in all Q of its slots instead. The value a site
// pulls from an IS source is then rho_I itself: the imposition needs no second, dependent
// load. The particle phase keeps this true when site sets move (k_is_density, k_is_restore,
// k_is_fix).
//
// In-place streaming (SweepArgs::aa, one buffer): two kinds of step alternate. From the
// natural layout (slot i of x holds f*_i(x)) the neighbour phase pulls as above and writes
// f*_i(x) into slot opp(i) of x + c_i (into slot i of x itself where x + c_i lies beyond a
// wall, which is the slot the bounced pull of the next step reads); the local phase then
// finds the pulled f_i(x) in slot opp(i) of x and writes f*_i(x) back into slot i. A site
// reads and writes the same Q locations in both phases, so no two sites touch one. The
// sweep's input is gone once it ran, so the density carry (which needs it to restore sites
// that stop being IS) gives way to a density array: IS sites keep their populations and
// store rho_I beside them (k_inplace_fix refreshes it for sites that become IS).
#pragma once

#include <type_traits>
#include <utility>

#include <algorithm>

#include "kernels.h"

namespace lbmp {

constexpr int SWEEP_THREADS = 128;

// Arguments of the simulation a block works on: the kernel parameter for a single context,
// entry blockIdx.y of a device array for a batch of cells.
template <bool B, class A>
__device__ __forceinline__ A pick_args(const A& a0, const A* __restrict__ cells)
{
    if constexpr (B)
        return cells[blockIdx.y];
    else
        return a0;
}

template <int I, int N, class F>
__device__ __forceinline__ void sfor(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, N>(f);
    }
}

// Lever arm r = (x_site - x_p) of site (sx, sy, sz) owned by a particle (Eqs. 5, 7, 12):
// the integer offset from the particle's anchor (minimum image on periodic axes) minus phi.
template <typename K, typename C>
__device__ __forceinline__ void lever_arm(const Geom& g, const K& k, int sx, int sy, int sz, C r[3])
{
    const int o0 = offset_from_wrapped(sx, k.Kw[0], g.nx, !g.wall[0]);
    const int o1 = offset_from_wrapped(sy, k.Kw[1], g.ny, !g.wall[1]);
    const int o2 = offset_from_wrapped(sz, k.Kw[2], g.nz, !g.wall[2]);
    r[0] = (C)o0 - k.phi[0];
    r[1] = (C)o1 - k.phi[1];
    r[2] = (C)o2 - k.phi[2];
}

// Rigid-body velocity u_p + omega_p x r (Eq. 5 / Eq. 12, read as a rigid-body motion).
template <typename K, typename C>
__device__ __forceinline__ void rigid_velocity(const K& k, const C r[3], C out[3])
{
    out[0] = k.u[0] + (k.om[1] * r[2] - k.om[2] * r[1]);
    out[1] = k.u[1] + (k.om[2] * r[0] - k.om[0] * r[2]);
    out[2] = k.u[2] + (k.om[0] * r[1] - k.om[1] * r[0]);
}

// Compile-time masks of the directions whose component k equals v.
template <class L>
__host__ __device__ constexpr unsigned dir_mask(int k, int v)
{
    unsigned m = 0;
    for (int i = 0; i < L::Q; ++i)
        if (L::c(i, k) == v) m |= 1u << i;
    return m;
}
template <class L>
__device__ __forceinline__ int c_rt(int i, int k)
{
    return (int)((dir_mask<L>(k, 1) >> i) & 1u) - (int)((dir_mask<L>(k, -1) >> i) & 1u);
}
template <class L>
__device__ __forceinline__ float w_rt(int i)
{
    constexpr unsigned axis = dir_mask<L>(0, 0) & dir_mask<L>(1, 0) & dir_mask<L>(2, 0);  // rest only
    unsigned lvl1 = 0;
    for (int j = 1; j < L::Q; ++j)
        if (L::c(j, 0) * L::c(j, 0) + L::c(j, 1) * L::c(j, 1) + L::c(j, 2) * L::c(j, 2) == 1) lvl1 |= 1u << j;
    if ((axis >> i) & 1u) return (float)L::w(0);
    return ((lvl1 >> i) & 1u) ? (float)L::w(1) : (float)L::w(L::Q - 1);
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

// BGK collision with Guo forcing on deviations g = f - w (FP32). Opposite directions i and
// opp(i) share the even part of the equilibrium and of the forcing term and differ by the
// sign of the odd part, so each pair is relaxed together:
//   g*_i = (1 - omega) g_i + A + B,  g*_opp(i) = (1 - omega) g_opp(i) + A - B,
//   A = omega w (drho + rho (4.5 (c.u)^2 - 1.5 u^2)) + pre w (9 (c.u)(c.F) - 3 u.F),
//   B = 3 omega w rho (c.u) + 3 pre w (c.F).
//
// CONSERVE (FP32 storage): the momentum the collision hands the stored populations is made
// exact. In exact arithmetic the increments g*_i - g_i carry momentum F (Eq. 3 conserves
// rho u and the Guo term adds F). In FP32 the equilibrium, evaluated at the magnitude of g,
// is off by a few units in the last place, and in a slowly changing flow those errors repeat
// step after step with the same sign: the momentum drifts (after 1000 steps of a
// body-force-driven suspension, by ~1e-4 of the velocity). Here the increments as stored are
// taken back, g*_i - g_i (exact when g*_i and g_i are within a factor of two, as they are
// near equilibrium), their momentum S = sum_i c_i (g*_i - g_i) is compared with F, and the
// axis pair of each direction k absorbs (F_k - S_k) / 2 with opposite signs. What is left is
// one rounding of that correction per axis population, which varies from step to step and
// does not accumulate.
template <class L, bool CONSERVE = false>
__device__ __forceinline__ void collide_dev(float g[], const SweepArgs& a, float& drho, float& j0, float& j1,
                                            float& j2)
{
    constexpr int Q = L::Q;
    drho = 0.0f;
    j0 = 0.0f;
    j1 = 0.0f;
    j2 = 0.0f;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        drho += g[i];
        if constexpr (L::c(i, 0) != 0) j0 += (float)L::c(i, 0) * g[i];
        if constexpr (L::c(i, 1) != 0) j1 += (float)L::c(i, 1) * g[i];
        if constexpr (L::c(i, 2) != 0) j2 += (float)L::c(i, 2) * g[i];
    });
    const float F0 = a.F_f[0], F1 = a.F_f[1], F2 = a.F_f[2];
    const float rho = 1.0f + drho;
    const float inv = 1.0f / rho;
    const float u[3] = {(j0 + 0.5f * F0) * inv, (j1 + 0.5f * F1) * inv, (j2 + 0.5f * F2) * inv};
    const float omega = a.omega_f, pre = a.pre_f, om1 = 1.0f - omega;
    const float uF3 = 3.0f * (u[0] * F0 + u[1] * F1 + u[2] * F2);
    const float usq15 = 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if constexpr (!CONSERVE) {
        {   // rest direction
            const float w = (float)L::w(0);
            g[0] = om1 * g[0] + omega * w * (drho - rho * usq15) - pre * w * uF3;
        }
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int j = L::opp(i);
            if constexpr (j > i) {
                const float cu = (float)L::c(i, 0) * u[0] + (float)L::c(i, 1) * u[1] + (float)L::c(i, 2) * u[2];
                const float cF = (float)L::c(i, 0) * F0 + (float)L::c(i, 1) * F1 + (float)L::c(i, 2) * F2;
                const float w = (float)L::w(i);
                const float ow = omega * w, pw = pre * w;
                const float A = ow * (drho + rho * (4.5f * cu * cu - usq15)) + pw * (9.0f * cu * cF - uF3);
                const float B = 3.0f * (ow * rho * cu + pw * cF);
                g[i] = om1 * g[i] + (A + B);
                g[j] = om1 * g[j] + (A - B);
            }
        });
    } else {
        {   // rest direction (no momentum)
            const float w = (float)L::w(0);
            g[0] = om1 * g[0] + omega * w * (drho - rho * usq15) - pre * w * uF3;
        }
        float S[3] = {0.0f, 0.0f, 0.0f};  // momentum of the stored increments
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int j = L::opp(i);
            if constexpr (j > i) {
                constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
                const float cu = (float)cx * u[0] + (float)cy * u[1] + (float)cz * u[2];
                const float cF = (float)cx * F0 + (float)cy * F1 + (float)cz * F2;
                const float w = (float)L::w(i);
                const float ow = omega * w, pw = pre * w;
                const float A = ow * (drho + rho * (4.5f * cu * cu - usq15)) + pw * (9.0f * cu * cF - uF3);
                const float B = 3.0f * (ow * rho * cu + pw * cF);
                const float gi = om1 * g[i] + (A + B);
                const float gj = om1 * g[j] + (A - B);
                const float d = (gi - g[i]) - (gj - g[j]);  // c_j = -c_i
                if constexpr (cx != 0) S[0] += (float)cx * d;
                if constexpr (cy != 0) S[1] += (float)cy * d;
                if constexpr (cz != 0) S[2] += (float)cz * d;
                g[i] = gi;
                g[j] = gj;
            }
        });
        const float Fk[3] = {F0, F1, F2};
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
            if constexpr (cx * cx + cy * cy + cz * cz == 1) {
                constexpr int axis = cx != 0 ? 0 : (cy != 0 ? 1 : 2);
                const float half = 0.5f * (Fk[axis] - S[axis]);
                g[i] = (cx + cy + cz) > 0 ? g[i] + half : g[i] - half;
            }
        });
    }
}

// All equilibrium deviations g^eq_i(drho, u) (FP32), by opposite pairs.
template <class L>
__device__ __forceinline__ void equilibrium_dev(float drho, const float u[3], float g[])
{
    constexpr int Q = L::Q;
    const float rho = 1.0f + drho;
    const float usq15 = 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    g[0] = (float)L::w(0) * (drho - rho * usq15);
    sfor<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int j = L::opp(i);
        if constexpr (j > i) {
            const float cu = (float)L::c(i, 0) * u[0] + (float)L::c(i, 1) * u[1] + (float)L::c(i, 2) * u[2];
            const float w = (float)L::w(i);
            const float even = w * (drho + rho * (4.5f * cu * cu - usq15));
            const float odd = 3.0f * w * rho * cu;
            g[i] = even + odd;
            g[j] = even - odd;
        }
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

// Face crossed by the move x + c_d (lowest axis first), or -1 if it stays in the domain.
template <class L, int d>
__device__ __forceinline__ int out_face(const Nbr& n)
{
    constexpr int cx = L::c(d, 0), cy = L::c(d, 1), cz = L::c(d, 2);
    if (cx > 0 && n.bxp) return 1;
    if (cx < 0 && n.bxm) return 0;
    if (cy > 0 && n.byp) return 3;
    if (cy < 0 && n.bym) return 2;
    if (cz > 0 && n.bzp) return 5;
    if (cz < 0 && n.bzm) return 4;
    return -1;
}

// Momentum of a moving wall given to a bounced population (halfway bounce-back at a wall
// moving with u_w, reference density 1): the population pulled in direction i left x in
// direction d = opp(i) and returns as f*_d - 6 w_d (c_d . u_w). The same term applies to
// the deviation g = f - w, since w_i = w_d.
template <class L, typename C, bool WALLS>
__device__ __forceinline__ void wall_momentum(const Nbr& n, int eqface, const C (*__restrict__ uw)[3], C f[])
{
    if constexpr (WALLS) {
        sfor<0, L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int d = L::opp(i);
            const int face = out_face<L, d>(n);
            if (face >= 0 && !((eqface >> face) & 1)) {  // equilibrium faces carry no wall term
                const C cuw = (C)L::c(d, 0) * uw[face][0] + (C)L::c(d, 1) * uw[face][1] +
                              (C)L::c(d, 2) * uw[face][2];
                f[i] = f[i] - (C)6 * (C)L::w(d) * cuw;
            }
        });
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

// Applies the pending IS imposition (Eq. 12) to the values a site inside a particle pulls:
// a value pulled from an IS site s in direction i becomes f^eq(rho_I(s), u_p + omega_p x r(s))
// of the stored direction, where the pulled value itself is rho_I(s) (density carry). `m` is
// the site's IS-source mask (bit i: the source of direction i is an IS site of the site's
// own owner; MASK_OTHER: some source belongs to another particle).
//
// FP64 form: every substituted value is recomputed from its own lever arm, exactly as a
// direct implementation of Eq. 12 does.
template <class L, bool WALLS>
__device__ __forceinline__ void substitute_is_plain(const Geom& g, const Nbr& n, int x, int y, int z,
                                                    unsigned idx, unsigned m, const PartView& pv, double f[])
{
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if ((m & (MASK_OTHER | (1u << i))) == 0) return;
        int sx, sy, sz;
        unsigned sidx;
        bool bounce;
        pull_source<L, i, WALLS>(g, n, x, y, z, idx, sx, sy, sz, sidx, bounce);
        const unsigned t = pv.tag[sidx];
        if ((t >> 30) == CLS_IS && LBM_DCHECK(pv.status, (t & PID_MASK) < (unsigned)pv.np)) {
            const PKern& k = pv.pk[t & PID_MASK];
            double r[3], uI[3];
            lever_arm(g, k, sx, sy, sz, r);
            rigid_velocity(k, r, uI);
            f[i] = feq_plain<L, i>(bounce ? -1.0 : 1.0, f[i], uI);
        }
    });
}

// Whether the pull of direction i leaves the domain through a wall (then its source is the
// site itself, stored direction opp(i)).
template <class L, int i, bool WALLS>
__device__ __forceinline__ bool pull_bounces(const Nbr& n)
{
    if constexpr (!WALLS) {
        return false;
    } else {
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        return (cx > 0 && n.bxm) || (cx < 0 && n.bxp) || (cy > 0 && n.bym) || (cy < 0 && n.byp) ||
               (cz > 0 && n.bzm) || (cz < 0 && n.bzp);
    }
}

template <class L, bool WALLS>
__device__ __forceinline__ void substitute_is_other_dev(const Geom& g, const Nbr& n, int x, int y, int z, unsigned owner,
                                                     const PartView& pv, float f[]);

// FP32 form. With u(s) = u(x) - omega x c_i for the source s = x - c_i of a rigid motion:
// c_i.u(s) = c_i.u(x) (c_i.(omega x c_i) = 0) and
// |u(s)|^2 = |u(x)|^2 - 2 c_i.(u(x) x omega) + |omega|^2 |c_i|^2 - (omega.c_i)^2,
// so one rigid velocity per site serves all of its sources. The work is warp-uniform: the
// directions some lane of the warp needs are evaluated by every lane and kept where the
// lane's own mask asks for them (no per-lane branches, no loads beyond the owner's record).
// Every lane of the warp that is converged here calls it; m = 0 for sites with nothing to do.
template <class L, bool WALLS>
__device__ __forceinline__ void substitute_is_dev(const Geom& g, const Nbr& n, int x, int y, int z,
                                                  unsigned m, unsigned owner, const PartView& pv, float f[])
{
    constexpr int Q = L::Q;
    const unsigned mm = m & ~MASK_OTHER;
    const unsigned wm = __reduce_or_sync(__activemask(), mm);
    if (wm) {
        unsigned ow = mm ? owner : 0u;
        if (!LBM_DCHECK(pv.status, ow < (unsigned)pv.np)) ow = 0u;
        const PKernF k = pv.pkf[ow];
        float r[3], ux[3];
        lever_arm(g, k, x, y, z, r);
        rigid_velocity(k, r, ux);
        // b = u(x) + u(x) x omega
        const float b0 = ux[0] + (ux[1] * k.om[2] - ux[2] * k.om[1]);
        const float b1 = ux[1] + (ux[2] * k.om[0] - ux[0] * k.om[2]);
        const float b2 = ux[2] + (ux[0] * k.om[1] - ux[1] * k.om[0]);
        const float usq = ux[0] * ux[0] + ux[1] * ux[1] + ux[2] * ux[2];
        const float w2 = k.om[0] * k.om[0] + k.om[1] * k.om[1] + k.om[2] * k.om[2];
        // -1.5 (|u(x)|^2 + |omega|^2 |c|^2) for |c|^2 = 1 and 2
        const float B1 = -1.5f * (usq + w2), B2 = -1.5f * (usq + 2.0f * w2);
        // rest direction: only an IS site pulls its own rest population, f^eq_0 at u(x)
        if (wm & 1u) {
            const float E = -1.5f * usq;
            const float val = (float)L::w(0) * (E + f[0] * (1.0f + E));
            if (mm & 1u) f[0] = val;
        }
        // Opposite pair (i, j = opp(i)): with cu = c_i.u(x), cb = c_i.b = cu + c_i.(u(x) x omega)
        // and cw = c_i.omega, the sources x - c_i and x - c_j give
        // E = 4.5 cu^2 - 1.5 (|u(x)|^2 + |omega|^2 |c_i|^2 - cw^2) +- 3 cb and f = w (E + drho (1 + E)).
        // A bounced pull (source x itself, stored direction opp) has E = -+3 cu + 4.5 cu^2 - 1.5 |u|^2.
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int j = L::opp(i);
            if constexpr (j > i) {
                constexpr unsigned pair = (1u << i) | (1u << j);
                if (wm & pair) {
                    constexpr float cx = (float)L::c(i, 0), cy = (float)L::c(i, 1), cz = (float)L::c(i, 2);
                    constexpr float c2 = cx * cx + cy * cy + cz * cz;
                    constexpr float w = (float)L::w(i);
                    const float cu = cx * ux[0] + cy * ux[1] + cz * ux[2];
                    const float cb = cx * b0 + cy * b1 + cz * b2;
                    const float cw = cx * k.om[0] + cy * k.om[1] + cz * k.om[2];
                    const float S = cu * (4.5f * cu) + (cw * (1.5f * cw) + (c2 == 1.0f ? B1 : B2));
                    float Ei = S + 3.0f * cb, Ej = S - 3.0f * cb;
                    if constexpr (WALLS) {
                        const float Sb = 4.5f * cu * cu - 1.5f * usq;
                        if (pull_bounces<L, i, WALLS>(n)) Ei = Sb - 3.0f * cu;
                        if (pull_bounces<L, j, WALLS>(n)) Ej = Sb + 3.0f * cu;
                    }
                    const float vi = w * (Ei + f[i] * (1.0f + Ei));
                    const float vj = w * (Ej + f[j] * (1.0f + Ej));
                    if (mm & (1u << i)) f[i] = vi;
                    if (mm & (1u << j)) f[j] = vj;
                }
            }
        });
    }
    if (m & MASK_OTHER) substitute_is_other_dev<L, WALLS>(g, n, x, y, z, owner, pv, f);
}

// Sources owned by another particle than the site's own (site sets of close particles
// meet): rare, one direction at a time.
template <class L, bool WALLS>
__device__ __forceinline__ void substitute_is_other_dev(const Geom& g, const Nbr& n, int x, int y, int z, unsigned owner,
                                                     const PartView& pv, float f[])
{
    constexpr int Q = L::Q;
    {
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
            const int cx = c_rt<L>(i, 0), cy = c_rt<L>(i, 1), cz = c_rt<L>(i, 2);
            int sx = cx > 0 ? n.xm : (cx < 0 ? n.xp : x);
            int sy = cy > 0 ? n.ym : (cy < 0 ? n.yp : y);
            int sz = cz > 0 ? n.zm : (cz < 0 ? n.zp : z);
            bool bounce = false;
            if (WALLS)
                bounce = (cx > 0 && n.bxm) || (cx < 0 && n.bxp) || (cy > 0 && n.bym) || (cy < 0 && n.byp) ||
                         (cz > 0 && n.bzm) || (cz < 0 && n.bzp);
            if (bounce) { sx = x; sy = y; sz = z; }
            const unsigned sidx = ((unsigned)sz * (unsigned)g.ny + (unsigned)sy) * (unsigned)g.nx + (unsigned)sx;
            const unsigned t = pv.tag[sidx];
            if ((t >> 30) != CLS_IS || (t & PID_MASK) == owner) continue;
            if (!LBM_DCHECK(pv.status, (t & PID_MASK) < (unsigned)pv.np)) continue;
            const PKernF k = pv.pkf[t & PID_MASK];
            float r[3], us[3];
            lever_arm(g, k, sx, sy, sz, r);
            rigid_velocity(k, r, us);
            const float sgn = bounce ? -1.0f : 1.0f;
            const float cu = sgn * ((float)cx * us[0] + (float)cy * us[1] + (float)cz * us[2]);
            const float usq = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
            sfor<0, Q>([&](auto jc) {
                constexpr int jj = decltype(jc)::value;
                if (i == jj) {
                    const float drho = f[jj];
                    f[jj] = w_rt<L>(i) * (drho + (1.0f + drho) * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
                }
            });
        }
    }
}

// In-place streaming: the value pulled in each direction the imposition substitutes (mask
// bit i, or a source tagged IS of another particle) is replaced by the source's density
// from the array the previous sweep wrote; the substitution then reads it exactly as it
// reads a carried density in the pull scheme. Sites with m = 0 have nothing to do.
template <class L, typename C, bool WALLS>
__device__ __forceinline__ void is_density_from_array(const Geom& g, const Nbr& n, int x, int y, int z,
                                                      unsigned idx, unsigned m, const PartView& pv,
                                                      const C* __restrict__ rho, C f[])
{
    if (m == 0) return;
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        int sx, sy, sz;
        unsigned sidx;
        bool bounce;
        pull_source<L, i, WALLS>(g, n, x, y, z, idx, sx, sy, sz, sidx, bounce);
        bool take = ((m >> i) & 1u) != 0;
        if (!take && (m & MASK_OTHER)) take = (pv.tag[sidx] >> 30) == CLS_IS;
        if (take) f[i] = rho[sidx];
    });
}

// The same in the sweep, where every lane of the warp calls it: a direction some lane needs
// is loaded by every lane (a lane without it loads its own site's entry) and kept by a select,
// so the warp takes no per-lane branches; sources of another particle (rare) take the plain
// form.
template <class L, typename C, bool WALLS>
__device__ __forceinline__ void is_density_from_array_warp(const Geom& g, const Nbr& n, int x, int y, int z,
                                                           unsigned idx, unsigned m, const PartView& pv,
                                                           const C* __restrict__ rho, C f[])
{
    const unsigned mm = m & ~MASK_OTHER;
    const unsigned wm = __reduce_or_sync(__activemask(), mm);
    if (wm) {
        sfor<0, L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            if (wm & (1u << i)) {
                int sx, sy, sz;
                unsigned sidx;
                bool bounce;
                pull_source<L, i, WALLS>(g, n, x, y, z, idx, sx, sy, sz, sidx, bounce);
                const bool mine = ((mm >> i) & 1u) != 0;
                const C v = rho[mine ? sidx : idx];
                f[i] = mine ? v : f[i];
            }
        });
    }
    if (m & MASK_OTHER) is_density_from_array<L, C, WALLS>(g, n, x, y, z, idx, MASK_OTHER, pv, rho, f);
}

// Rebuilds the IS-source masks at the sites of the listed particles (their site sets hold
// every site whose mask can be non-zero or can have changed).
template <class L, bool B>
__global__ void k_update_masks(const MaskArgs a0, const MaskArgs* __restrict__ cells)
{
    const MaskArgs a = pick_args<B>(a0, cells);
    if (a.np == 0 || (a.list && !a.cnt)) return;
    const int count = a.list ? a.cnt->nrestamp : a.np;
    const Geom& g = a.g;
    for (int b = blockIdx.x; b < count; b += gridDim.x) {
        const int p = a.list ? a.list[b] : b;
        const PConst pc = a.pc[p];
        const int Kw[3] = {a.pk[p].Kw[0], a.pk[p].Kw[1], a.pk[p].Kw[2]};
        for (int e = threadIdx.x; e < pc.tmpl_n; e += blockDim.x) {
            const int ent = a.tmpl[pc.tmpl_off + e];
            unsigned idx;
            int v[3];
            if (!site_fast_xyz(g, Kw, tmpl_ox(ent), tmpl_oy(ent), tmpl_oz(ent), idx, v)) continue;
            const unsigned t0 = a.tag[idx];
            const unsigned owner = t0 & PID_MASK;
            const int x = v[0], y = v[1], z = v[2];
            const Nbr n = neighbours<true>(g, x, y, z);
            unsigned m = 0;
            sfor<0, L::Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                int sx, sy, sz;
                unsigned sidx;
                bool bounce;
                pull_source<L, i, true>(g, n, x, y, z, idx, sx, sy, sz, sidx, bounce);
                const unsigned t = a.tag[sidx];
                if ((t >> 30) == CLS_IS) m |= ((t & PID_MASK) == owner) ? (1u << i) : MASK_OTHER;
            });
            a.ismask[idx] = m;
        }
    }
}

// The equilibrium face site (x, y, z) lies on (the first of -x, +x, -y, +y, -z, +z), or -1.
__device__ __forceinline__ int eq_face_of(const Geom& g, int x, int y, int z)
{
    const int m = g.eqface;
    if ((m & 1) && x == 0) return 0;
    if ((m & 2) && x == g.nx - 1) return 1;
    if ((m & 4) && y == 0) return 2;
    if ((m & 8) && y == g.ny - 1) return 3;
    if ((m & 16) && z == 0) return 4;
    if ((m & 32) && z == g.nz - 1) return 5;
    return -1;
}

// BS transfer of one site in the deviation form (Eqs. 5-7): the forced collision keeps the
// density and adds F to the momentum, so the post-collision rho_B and rho_B u_B are rho and
// j + F of the pulled values (mrho, mj). The site takes f^eq(rho_B, u_p + omega_p x r) and
// its record (dp = rho_B (u_B' - u_B) = rho_B u_B' - (j + F) and the owner's tag: 16 bytes
// at the site's index, or its brick index with BRICK: rec_brick_index) feeds the per-particle
// sums (Eqs. 8-9) that the particle phase takes afterwards in a fixed order, forming
// dl = r x dp there from the site's template offset.
template <class L, bool BRICK>
__device__ __forceinline__ void bs_transfer_dev(const SweepArgs& a, int x, int y, int z, unsigned idx, unsigned tagx,
                                                float mrho, float mj0, float mj1, float mj2, float f[])
{
    unsigned pid = tagx & PID_MASK;
    if (!LBM_DCHECK(a.pv.status, pid < (unsigned)a.pv.np)) pid = 0u;
    const PKernF k = a.pv.pkf[pid];
    float r[3], ubp[3], dv[3];
    lever_arm(a.g, k, x, y, z, r);
    rigid_velocity(k, r, ubp);
    const float rho = 1.0f + mrho;
    const float pB[3] = {mj0 + a.F_f[0], mj1 + a.F_f[1], mj2 + a.F_f[2]};
    equilibrium_dev<L>(mrho, ubp, f);
#pragma unroll
    for (int q = 0; q < 3; ++q) dv[q] = rho * ubp[q] - pB[q];
    const unsigned ri = BRICK ? rec_brick_index(a.g, x, y, z) : idx;
    ((float4*)a.bs_scratch)[ri] = make_float4(dv[0], dv[1], dv[2], __uint_as_float(tagx));
}

// Everything a site does after its populations are pulled: the pending IS imposition,
// the collision, the BS transfer and its per-site record, and the stores (IS sites store
// their density in every slot). RESTORE: store an IS site's populations instead (the
// particle phase recomputing a site that stops being IS); the caller may be divergent.
// Otherwise every lane of the warp calls it (tail lanes with valid = false). AA: the phase
// of in-place streaming (SweepArgs::aa), whose stores replace the pull scheme's.
template <class L, typename S, bool WALLS, bool PART, bool RESTORE = false, int AA = 0>
__device__ __forceinline__ void sweep_site(const SweepArgs& a, int x, int y, int z, unsigned idx, bool valid,
                                           const Nbr& n, typename Store<S>::C f[], unsigned tagx, unsigned mask)
{
    using St = Store<S>;
    using C = typename St::C;
    constexpr int Q = L::Q;
    const Geom& g = a.g;
    if constexpr (PART) {
        if (*a.pv.pending) {
            const unsigned m = tagx != TAG_FLUID ? mask : 0u;
            if constexpr (AA != 0)
                is_density_from_array_warp<L, C, WALLS>(g, n, x, y, z, idx, m, a.pv, (const C*)a.is_rho_in, f);
            if constexpr (St::deviation)
                substitute_is_dev<L, WALLS>(g, n, x, y, z, m, tagx & PID_MASK, a.pv, f);
            else if (m)
                substitute_is_plain<L, WALLS>(g, n, x, y, z, idx, m, a.pv, f);
        }
    }
    // A moving wall acts on the bounced value after the IS imposition it may have received.
    if constexpr (WALLS) {
        if (a.moving_walls && *a.pv.pending) {
            if constexpr (St::deviation)
                wall_momentum<L, C, WALLS>(n, g.eqface, a.uw->uf, f);
            else
                wall_momentum<L, C, WALLS>(n, g.eqface, a.uw->u, f);
        }
    }

    float mrho = 0.f, mj0 = 0.f, mj1 = 0.f, mj2 = 0.f;  // pre-collision moments (FP32 path)
    if constexpr (St::deviation)
        collide_dev<L, std::is_same<S, float>::value>(f, a, mrho, mj0, mj1, mj2);
    else
        collide_plain<L>(f, a);

    if constexpr (PART) {
        // Particle-fluid momentum transfer at BS sites (Eqs. 5-7).
        const bool isbs = valid && (tagx >> 30) == CLS_BS;
        if constexpr (St::deviation) {
            if (isbs)
                bs_transfer_dev<L, std::is_same<S, float>::value>(a, x, y, z, idx, tagx, mrho, mj0, mj1, mj2, f);
        } else if (isbs && LBM_DCHECK(a.pv.status, (tagx & PID_MASK) < (unsigned)a.pv.np)) {
            C r[3], ub[3], ubp[3], du[3];
            const PKern& k = a.pv.pk[tagx & PID_MASK];
            lever_arm(g, k, x, y, z, r);
            rigid_velocity(k, r, ubp);
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
            // Per-site contributions; the per-particle sums (Eqs. 8-9) are taken afterwards
            // in a fixed order by the particle phase.
            C* sc = (C*)a.bs_scratch + (size_t)idx * 6;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                sc[q] = rhoB * du[q];
                sc[3 + q] = rhoB * cr[q];
            }
        }
    }

    // Equilibrium faces: a fluid site on one takes f^eq(rho, u_face) of the current face
    // velocities, rho its post-collision density (the pre-collision one in the deviation
    // form, equal in exact arithmetic).
    if constexpr (WALLS) {
        if (g.eqface) {
            const int face = eq_face_of(g, x, y, z);
            if (face >= 0 && (!PART || tagx == TAG_FLUID)) {
                if constexpr (St::deviation) {
                    equilibrium_dev<L>(mrho, a.uw[1].uf[face], f);
                } else {
                    double rho = 0.0;
                    sfor<0, Q>([&](auto ic) { rho += f[decltype(ic)::value]; });
                    sfor<0, Q>([&](auto ic) {
                        constexpr int i = decltype(ic)::value;
                        f[i] = feq_plain<L, i>(1.0, rho, a.uw[1].u[face]);
                    });
                }
            }
        }
    }

    const size_t N = g.N;
    if constexpr (AA != 0) {
        // In-place streaming: populations to the phase's slots; an IS site's density (the sum
        // of the values as stored, in slot order) to the density array.
        S* out = (S*)a.fout;
        if constexpr (PART) {
            const bool isis = valid && (tagx >> 30) == CLS_IS;
            if (__any_sync(__activemask(), isis)) {  // warp-uniform
                C dens = (C)0;
                sfor<0, Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    dens += St::load(St::save(f[i], (C)L::w(i)), (C)L::w(i));
                });
                if (isis) ((C*)a.is_rho_out)[idx] = dens;
            }
        }
        if (!valid) return;
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            size_t at = (size_t)i * N + idx;
            if constexpr (AA == 1) {
                int tx, ty, tz;
                unsigned tidx;
                bool beyond;
                pull_source<L, L::opp(i), WALLS>(g, n, x, y, z, idx, tx, ty, tz, tidx, beyond);
                if (!beyond) at = (size_t)L::opp(i) * N + tidx;
            }
            out[at] = St::save(f[i], (C)L::w(i));
        });
        return;
    }
    S* __restrict__ fout = (S*)a.fout;
    // IS sites store their post-collision density, the sum of the values as stored, in
    // every slot (density carry); the check is warp-uniform.
    const bool isis = PART && !RESTORE && (tagx >> 30) == CLS_IS;
    bool any_is = false;
    if constexpr (PART && !RESTORE) any_is = __any_sync(__activemask(), isis);
    if (!valid) return;
    if (any_is) {
        S s[Q];
        C dens = (C)0;
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            s[i] = St::save(f[i], (C)L::w(i));
            dens += St::load(s[i], (C)L::w(i));
        });
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            fout[(size_t)i * N + idx] = isis ? St::save(dens, (C)L::w(i)) : s[i];
        });
    } else {
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            fout[(size_t)i * N + idx] = St::save(f[i], (C)L::w(i));
        });
    }
}


// Deviation storages without walls are held to nine blocks per SM (56 registers, no spills).
template <class L, typename S, bool WALLS, bool PART>
__global__ void __launch_bounds__(SWEEP_THREADS, (Store<S>::deviation && !WALLS) ? 9 : 1) k_sweep(const SweepArgs a)
{
    using C = typename Store<S>::C;
    constexpr int Q = L::Q;
    const Geom& g = a.g;
    const int y = blockIdx.y, z = blockIdx.z;
    const unsigned row = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx;
    const int xr = blockIdx.x * SWEEP_THREADS + threadIdx.x;
    const bool valid = xr < g.nx;
    const int x = valid ? xr : g.nx - 1;
    const unsigned idx = row + (unsigned)x;
    const Nbr n = neighbours<WALLS>(g, x, y, z);
    // Owner tag and IS-source mask are loaded with the populations (no dependent round trip).
    unsigned tagx = TAG_FLUID, mask = 0;
    if constexpr (PART) {
        tagx = a.pv.tag[idx];
        mask = a.pv.ismask[idx];
    }
    C f[Q];
    pull<L, S, WALLS>((const S*)a.fin, g, n, x, y, z, idx, f);
    sweep_site<L, S, WALLS, PART>(a, x, y, z, idx, valid, n, f, tagx, mask);
}

// In-place streaming, one phase (PHASE = SweepArgs::aa): the per-site step of k_sweep with
// the phase's loads and stores on the one buffer (fin == fout). Deviation storages: at most
// 56 registers (nine blocks per SM), measured 3 % faster than the unconstrained allocation at
// the 512^3 suspension (FP32); FP64 keeps its registers.
template <class L, typename S, bool WALLS, bool PART, int PHASE>
__global__ void __launch_bounds__(SWEEP_THREADS, Store<S>::deviation ? 9 : 1) k_sweep_inplace(const SweepArgs a)
{
    using C = typename Store<S>::C;
    constexpr int Q = L::Q;
    const Geom& g = a.g;
    const int y = blockIdx.y, z = blockIdx.z;
    const unsigned row = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx;
    const int xr = blockIdx.x * SWEEP_THREADS + threadIdx.x;
    const bool valid = xr < g.nx;
    const int x = valid ? xr : g.nx - 1;
    const unsigned idx = row + (unsigned)x;
    const Nbr n = neighbours<WALLS>(g, x, y, z);
    unsigned tagx = TAG_FLUID, mask = 0;
    if constexpr (PART) {
        tagx = a.pv.tag[idx];
        mask = a.pv.ismask[idx];
    }
    C f[Q];
    if constexpr (PHASE == 1) {
        pull<L, S, WALLS>((const S*)a.fin, g, n, x, y, z, idx, f);
    } else {
        const S* fin = (const S*)a.fin;
        const size_t N = g.N;
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            f[i] = Store<S>::load(fin[(size_t)L::opp(i) * N + idx], (C)L::w(i));
        });
    }
    sweep_site<L, S, WALLS, PART, false, PHASE>(a, x, y, z, idx, valid, n, f, tagx, mask);
}

// One launch over a batch of cells: each block takes tiles of the schedule table (one, or a
// stride of them in the persistent form) and runs the same per-site step as k_sweep with the
// arguments of the tile's cell. Deviation storages without walls are held to nine blocks per SM
// (56 registers, a few bytes of spills): the 64-cell ensemble's sweep 1.098 -> 1.065 ms.
template <class L, typename S, bool WALLS, bool PART>
__global__ void __launch_bounds__(SWEEP_THREADS, (Store<S>::deviation && !WALLS) ? 9 : 1)
    k_sweep_batch(const BatchSweepArgs b)
{
    using C = typename Store<S>::C;
    constexpr int Q = L::Q;
    // The tile's cell arguments (~190 bytes) are staged in shared memory by the block and
    // reloaded only when the cell changes, instead of every thread loading them per tile.
    __shared__ __align__(16) SweepArgs sa;
    int cur = -1;
    for (int e = blockIdx.x; e < b.ntiles; e += gridDim.x) {
        const int4 t = b.table[e];
        if (t.x != cur) {  // block-uniform: one table entry per block and tile
            __syncthreads();
            const int* src = reinterpret_cast<const int*>(&b.cells[t.x]);
            int* dst = reinterpret_cast<int*>(&sa);
            for (int w = threadIdx.x; w < (int)(sizeof(SweepArgs) / 4); w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            cur = t.x;
        }
        const SweepArgs& a = sa;
        const Geom& g = a.g;
        const int lw = t.z >> 16;
        const int xr = t.y + (int)(threadIdx.x & ((1u << lw) - 1u));
        const int yr = (t.z & 0xFFFF) + (int)(threadIdx.x >> lw);
        const bool valid = xr < g.nx && yr < g.ny;
        const int x = min(xr, g.nx - 1), y = min(yr, g.ny - 1), z = t.w;
        const unsigned idx = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx + (unsigned)x;
        const Nbr n = neighbours<WALLS>(g, x, y, z);
        unsigned tagx = TAG_FLUID, mask = 0;
        if constexpr (PART) {
            if (a.pv.tag != nullptr) {
                tagx = a.pv.tag[idx];
                mask = a.pv.ismask[idx];
            }
        }
        C f[Q];
        pull<L, S, WALLS>((const S*)a.fin, g, n, x, y, z, idx, f);
        sweep_site<L, S, WALLS, PART>(a, x, y, z, idx, valid, n, f, tagx, mask);
    }
}

// Populations of site idx at a step boundary (streamed, pending IS imposition and wall
// momentum applied), in the storage's compute form: f, or g = f - w for deviation storage.
template <class L, typename S, bool WALLS>
__device__ __forceinline__ void site_pull(const MaterializeArgs& a, unsigned idx, typename Store<S>::C f[])
{
    using St = Store<S>;
    using C = typename St::C;
    const Geom& g = a.g;
    const int x = (int)(idx % (unsigned)g.nx);
    const int y = (int)((idx / (unsigned)g.nx) % (unsigned)g.ny);
    const int z = (int)(idx / ((unsigned)g.nx * (unsigned)g.ny));
    const Nbr n = neighbours<WALLS>(g, x, y, z);
    if (a.aa == 1) {
        const S* fin = (const S*)a.fin;
        sfor<0, L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            f[i] = St::load(fin[(size_t)L::opp(i) * g.N + idx], (C)L::w(i));
        });
    } else {
        pull<L, S, WALLS>((const S*)a.fin, g, n, x, y, z, idx, f);
    }
    if (a.pv.tag != nullptr && a.pv.tag[idx] != TAG_FLUID && *a.pv.pending) {
        const unsigned m = a.pv.ismask[idx];
        if (m) {
            if (a.is_rho) is_density_from_array<L, C, WALLS>(g, n, x, y, z, idx, m, a.pv, (const C*)a.is_rho, f);
            if constexpr (St::deviation)
                substitute_is_dev<L, WALLS>(g, n, x, y, z, m, a.pv.tag[idx] & PID_MASK, a.pv, f);
            else
                substitute_is_plain<L, WALLS>(g, n, x, y, z, idx, m, a.pv, f);
        }
    }
    if constexpr (WALLS) {
        if (a.moving_walls && *a.pv.pending) {
            if constexpr (St::deviation)
                wall_momentum<L, C, WALLS>(n, g.eqface, a.uw->uf, f);
            else
                wall_momentum<L, C, WALLS>(n, g.eqface, a.uw->u, f);
        }
    }
}

// rho = sum f (Eq. 1) and u = (sum f c + F/2) / rho (Eq. 2 with the Guo half-force) of site
// idx; deviation storage sums the deviations (rho = 1 + sum g).
template <class L, typename S, bool WALLS>
__device__ __forceinline__ void site_moments(const MaterializeArgs& a, unsigned idx, double& rho, double u[3])
{
    using C = typename Store<S>::C;
    constexpr int Q = L::Q;
    C f[Q];
    site_pull<L, S, WALLS>(a, idx, f);
    double j[3] = {0.0, 0.0, 0.0};
    rho = 0.0;
    sfor<0, Q>([&](auto ic) { rho += (double)f[decltype(ic)::value]; });
    if constexpr (Store<S>::deviation) rho = 1.0 + rho;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            j[k] += (double)f[i] * (double)L::c(i, k);
        });
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = (j[k] + 0.5 * a.F[k]) / rho;
}

template <class L, typename S, bool WALLS>
__global__ void k_materialize(const MaterializeArgs a)
{
    constexpr int Q = L::Q;
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.count) return;
    const unsigned idx = a.s0 + t;
    if (a.mode == 1) {
        typename Store<S>::C f[Q];
        site_pull<L, S, WALLS>(a, idx, f);
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            a.out0[(size_t)i * a.count + t] = Store<S>::deviation ? (double)f[i] + L::w(i) : (double)f[i];
        });
        return;
    }
    double rho, u[3];
    site_moments<L, S, WALLS>(a, idx, rho, u);
    a.out0[t] = rho;
#pragma unroll
    for (int k = 0; k < 3; ++k) a.out1[(size_t)t * 3 + k] = u[k];
}

// Closure inputs: for particle p (blockIdx.x) and stencil node q (thread), the moments
// (rho - 1, u - u_p) / u_ref trilinearly interpolated at x_p + h (i - (n-1)/2, j - ..,
// k - ..), q = (k n + j) n + i, from the 8 surrounding sites (periodic axes wrap, walled
// axes clamp to the domain), out[p][q][4]; then the fractional offset phi of the particle's
// reference centre, out[p][4 n^3 + 0..2].
template <class L, typename S, bool WALLS>
__global__ void k_features(const FeatureArgs f)
{
    const int p = blockIdx.x;
    const int nn = f.n_side * f.n_side * f.n_side;
    const int D = f.m.lattice == 0 ? 2 : 3;
    const size_t stride = (size_t)nn * 4 + 3;
    if (threadIdx.x < 3) f.out[(size_t)p * stride + (size_t)nn * 4 + threadIdx.x] = (float)f.pk[p].phi[threadIdx.x];
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const int ii[3] = {q % f.n_side, (q / f.n_side) % f.n_side, q / (f.n_side * f.n_side)};
        const Geom& g = f.m.g;
        const int nax[3] = {g.nx, g.ny, g.nz};
        int lo[3], hi[3];
        double w1[3];
        for (int k = 0; k < 3; ++k) {
            if (k >= D) {
                lo[k] = hi[k] = 0;
                w1[k] = 0.0;
                continue;
            }
            const double pos = f.x[(size_t)p * 3 + k] + f.h * ((double)ii[k] - 0.5 * (double)(f.n_side - 1));
            const double fl = floor(pos);
            w1[k] = pos - fl;
            int a0 = (int)fl, a1 = a0 + 1;
            if (g.wall[k]) {
                a0 = min(max(a0, 0), nax[k] - 1);
                a1 = min(max(a1, 0), nax[k] - 1);
            } else {
                a0 = ((a0 % nax[k]) + nax[k]) % nax[k];
                a1 = ((a1 % nax[k]) + nax[k]) % nax[k];
            }
            lo[k] = a0;
            hi[k] = a1;
        }
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < (D == 3 ? 8 : 4); ++c) {
            const int sx = (c & 1) ? hi[0] : lo[0], sy = (c & 2) ? hi[1] : lo[1], sz = (c & 4) ? hi[2] : lo[2];
            const double w = ((c & 1) ? w1[0] : 1.0 - w1[0]) * ((c & 2) ? w1[1] : 1.0 - w1[1]) *
                             (D == 3 ? ((c & 4) ? w1[2] : 1.0 - w1[2]) : 1.0);
            const unsigned idx = ((unsigned)sz * (unsigned)g.ny + (unsigned)sy) * (unsigned)g.nx + (unsigned)sx;
            double rho, u[3];
            site_moments<L, S, WALLS>(f.m, idx, rho, u);
            acc[0] += w * (rho - 1.0);
            for (int k = 0; k < 3; ++k) acc[1 + k] += w * u[k];
        }
        float* o = f.out + (size_t)p * stride + (size_t)q * 4;
        o[0] = (float)(acc[0] / f.u_ref);
        for (int k = 0; k < 3; ++k) o[1 + k] = (float)((acc[1 + k] - f.pk[p].u[k]) / f.u_ref);
    }
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
        const size_t at = (size_t)(a.opp ? L::opp(i) : i) * N + a.s0 + t;
        if constexpr (St::deviation)
            dst[at] = St::save((C)(v - L::w(i)), (C)L::w(i));
        else
            dst[at] = St::save((C)v, (C)L::w(i));
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

// ---- IS-site bookkeeping when a particle's shift changes -------------------------------
// Density carry keeps rho_I in every slot of the sites the sweep saw tagged IS. After the
// move, the sites of a particle whose shift changed may stop or start being IS; these three
// kernels (one block per such particle, threads over its IS template entries at the anchor
// the sweep used and at the new one) restore the invariant for the new owner map.

// Site of IS template entry e of particle p at anchor K (false if it leaves a walled domain).
__device__ __forceinline__ bool is_entry_site(const ISFixArgs& a, const int K[3], int e, unsigned& site)
{
    int Kw[3];
    wrap_anchor(a.s.g, K, Kw);
    const int ent = a.tmpl[e];
    return site_fast(a.s.g, Kw, tmpl_ox(ent), tmpl_oy(ent), tmpl_oz(ent), site);
}

// (1) Before the owner map changes: the density of every visited site, read from the
// sweep's output (one slot of a site the sweep saw as IS, else the sum of its populations in
// slot order, the sum the sweep takes).
template <class L, typename S, bool B>
__global__ void k_is_density(const ISFixArgs a0, const ISFixArgs* __restrict__ cells)
{
    using St = Store<S>;
    using C = typename St::C;
    const ISFixArgs a = pick_args<B>(a0, cells);
    if (!a.cnt) return;
    const int nlist = a.cnt->nchanged;
    const size_t N = a.s.g.N;
    const S* fo = (const S*)a.s.fout;
    C* dens = (C*)a.dens;
    for (int b = blockIdx.x; b < nlist; b += gridDim.x) {
        const int p = a.list[b];
        const PConst pc = a.pc[p];
        const int Ko[3] = {a.Kold[(size_t)p * 3], a.Kold[(size_t)p * 3 + 1], a.Kold[(size_t)p * 3 + 2]};
        const int Kn[3] = {a.pk[p].K[0], a.pk[p].K[1], a.pk[p].K[2]};
        for (int e = threadIdx.x; e < 2 * pc.n_is; e += blockDim.x) {
            unsigned site;
            if (!is_entry_site(a, e < pc.n_is ? Ko : Kn, pc.tmpl_off + pc.n_bs + e % pc.n_is, site)) continue;
            C d = (C)0;
            if ((a.s.pv.tag[site] >> 30) == CLS_IS) {
                d = St::load(fo[site], (C)L::w(0));
            } else {
                sfor<0, L::Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    d += St::load(fo[(size_t)i * N + site], (C)L::w(i));
                });
            }
            dens[site] = d;
        }
    }
}

// (2) Still before the owner map changes: the sites the sweep saw as IS of a particle whose
// shift changed get the populations the sweep computed for them (recomputed from the
// sweep's input with the sweep's particle view; same code, same result bit for bit).
template <class L, typename S, bool WALLS, bool B>
__global__ void k_is_restore(const ISFixArgs a0, const ISFixArgs* __restrict__ cells)
{
    using C = typename Store<S>::C;
    const ISFixArgs a = pick_args<B>(a0, cells);
    if (!a.cnt) return;
    const int nlist = a.cnt->nchanged;
    const Geom& g = a.s.g;
    for (int b = blockIdx.x; b < nlist; b += gridDim.x) {
        const int p = a.list[b];
        const PConst pc = a.pc[p];
        const int Ko[3] = {a.Kold[(size_t)p * 3], a.Kold[(size_t)p * 3 + 1], a.Kold[(size_t)p * 3 + 2]};
        for (int e = threadIdx.x; e < pc.n_is; e += blockDim.x) {
            unsigned site;
            if (!is_entry_site(a, Ko, pc.tmpl_off + pc.n_bs + e, site)) continue;
            const unsigned t = a.s.pv.tag[site];
            if (t != ((CLS_IS << 30) | (unsigned)p)) continue;
            const int x = (int)(site % (unsigned)g.nx);
            const int y = (int)((site / (unsigned)g.nx) % (unsigned)g.ny);
            const int z = (int)(site / ((unsigned)g.nx * (unsigned)g.ny));
            const Nbr n = neighbours<WALLS>(g, x, y, z);
            C f[L::Q];
            pull<L, S, WALLS>((const S*)a.s.fin, g, n, x, y, z, site, f);
            sweep_site<L, S, WALLS, true, true>(a.s, x, y, z, site, true, n, f, t, a.s.pv.ismask[site]);
        }
    }
}

// (3) After re-marking: every visited site that is now IS holds its density in every slot.
template <class L, typename S, bool B>
__global__ void k_is_fix(const ISFixArgs a0, const ISFixArgs* __restrict__ cells)
{
    using St = Store<S>;
    using C = typename St::C;
    const ISFixArgs a = pick_args<B>(a0, cells);
    if (!a.cnt) return;
    const int nlist = a.cnt->nchanged;
    const size_t N = a.s.g.N;
    S* fo = (S*)a.s.fout;
    const C* dens = (const C*)a.dens;
    for (int b = blockIdx.x; b < nlist; b += gridDim.x) {
        const int p = a.list[b];
        const PConst pc = a.pc[p];
        const int Ko[3] = {a.Kold[(size_t)p * 3], a.Kold[(size_t)p * 3 + 1], a.Kold[(size_t)p * 3 + 2]};
        const int Kn[3] = {a.pk[p].K[0], a.pk[p].K[1], a.pk[p].K[2]};
        for (int e = threadIdx.x; e < 2 * pc.n_is; e += blockDim.x) {
            unsigned site;
            if (!is_entry_site(a, e < pc.n_is ? Ko : Kn, pc.tmpl_off + pc.n_bs + e % pc.n_is, site)) continue;
            if ((a.s.pv.tag[site] >> 30) != CLS_IS) continue;
            const C d = dens[site];
            sfor<0, L::Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                fo[(size_t)i * N + site] = St::save(d, (C)L::w(i));
            });
        }
    }
}

// In-place streaming, after re-marking: every visited site that is now IS gets its density
// in the array the next sweep reads: the sum of its post-collision populations in slot order
// (the sum the sweep takes), found where the sweep's phase left them (s.aa: 2 = slot i of x;
// 1 = slot opp(i) of x + c_i, or slot i of x where x + c_i lies beyond a wall).
template <class L, typename S, bool WALLS>
__global__ void k_inplace_fix(const ISFixArgs a)
{
    using St = Store<S>;
    using C = typename St::C;
    if (!a.cnt) return;
    const int nlist = a.cnt->nchanged;
    const Geom& g = a.s.g;
    const size_t N = g.N;
    const S* fo = (const S*)a.s.fout;
    C* dens = (C*)a.dens;
    for (int b = blockIdx.x; b < nlist; b += gridDim.x) {
        const int p = a.list[b];
        const PConst pc = a.pc[p];
        const int Ko[3] = {a.Kold[(size_t)p * 3], a.Kold[(size_t)p * 3 + 1], a.Kold[(size_t)p * 3 + 2]};
        const int Kn[3] = {a.pk[p].K[0], a.pk[p].K[1], a.pk[p].K[2]};
        for (int e = threadIdx.x; e < 2 * pc.n_is; e += blockDim.x) {
            unsigned site;
            if (!is_entry_site(a, e < pc.n_is ? Ko : Kn, pc.tmpl_off + pc.n_bs + e % pc.n_is, site)) continue;
            if ((a.s.pv.tag[site] >> 30) != CLS_IS) continue;
            C d = (C)0;
            if (a.s.aa == 2) {
                sfor<0, L::Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    d += St::load(fo[(size_t)i * N + site], (C)L::w(i));
                });
            } else {
                const int x = (int)(site % (unsigned)g.nx);
                const int y = (int)((site / (unsigned)g.nx) % (unsigned)g.ny);
                const int z = (int)(site / ((unsigned)g.nx * (unsigned)g.ny));
                const Nbr n = neighbours<WALLS>(g, x, y, z);
                sfor<0, L::Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    int tx, ty, tz;
                    unsigned tidx;
                    bool beyond;
                    pull_source<L, L::opp(i), WALLS>(g, n, x, y, z, site, tx, ty, tz, tidx, beyond);
                    const size_t at = beyond ? (size_t)i * N + site : (size_t)L::opp(i) * N + tidx;
                    d += St::load(fo[at], (C)L::w(i));
                });
            }
            dens[site] = d;
        }
    }
}

}  // namespace lbmp

#include "sweep2.cuh"

namespace lbmp {

// ---- launchers --------------------------------------------------------------------------
// Deviation storages with an even nx take the two-site kernel (a.pair_bx threads along x),
// everything else the one-site kernel.
template <class L, typename S, bool WALLS, bool PART>
void launch_sweep_v(const SweepArgs& a, cudaStream_t s)
{
    if constexpr (Store<S>::deviation) {
        if (a.pair_bx > 0 && a.g.nx % 2 == 0) {
            launch_sweep2_v<L, S, WALLS, PART>(a, a.pair_bx, s);
            return;
        }
    }
    const dim3 grid((a.g.nx + SWEEP_THREADS - 1) / SWEEP_THREADS, a.g.ny, a.g.nz);
    k_sweep<L, S, WALLS, PART><<<grid, SWEEP_THREADS, 0, s>>>(a);
}

template <class L, typename S, bool WALLS, bool PART>
void launch_inplace_v(const SweepArgs& a, cudaStream_t s)
{
    const dim3 grid((a.g.nx + SWEEP_THREADS - 1) / SWEEP_THREADS, a.g.ny, a.g.nz);
    if (a.aa == 1) k_sweep_inplace<L, S, WALLS, PART, 1><<<grid, SWEEP_THREADS, 0, s>>>(a);
    else k_sweep_inplace<L, S, WALLS, PART, 2><<<grid, SWEEP_THREADS, 0, s>>>(a);
}

template <class L, typename S>
void launch_sweep_l(const SweepArgs& a, cudaStream_t s)
{
    const bool walls = a.g.wall[0] || a.g.wall[1] || a.g.wall[2];
    const bool part = a.pv.tag != nullptr;
    if (a.aa) {
        if (walls && part) launch_inplace_v<L, S, true, true>(a, s);
        else if (walls) launch_inplace_v<L, S, true, false>(a, s);
        else if (part) launch_inplace_v<L, S, false, true>(a, s);
        else launch_inplace_v<L, S, false, false>(a, s);
        return;
    }
    if (walls && part) launch_sweep_v<L, S, true, true>(a, s);
    else if (walls) launch_sweep_v<L, S, true, false>(a, s);
    else if (part) launch_sweep_v<L, S, false, true>(a, s);
    else launch_sweep_v<L, S, false, false>(a, s);
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
void launch_features(const FeatureArgs& f, cudaStream_t s)
{
    if (f.np == 0) return;
    const bool walls = f.m.g.wall[0] || f.m.g.wall[1] || f.m.g.wall[2];
    if (f.m.lattice == 0) {
        if (walls) k_features<D2Q9, S, true><<<f.np, 64, 0, s>>>(f);
        else k_features<D2Q9, S, false><<<f.np, 64, 0, s>>>(f);
    } else {
        if (walls) k_features<D3Q19, S, true><<<f.np, 64, 0, s>>>(f);
        else k_features<D3Q19, S, false><<<f.np, 64, 0, s>>>(f);
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

template <class L, typename S, bool B>
void launch_is_save_l(const ISFixArgs& a, const ISFixArgs* cells, dim3 grid, bool walls, cudaStream_t s)
{
    k_is_density<L, S, B><<<grid, 128, 0, s>>>(a, cells);
    if (walls) k_is_restore<L, S, true, B><<<grid, 128, 0, s>>>(a, cells);
    else k_is_restore<L, S, false, B><<<grid, 128, 0, s>>>(a, cells);
}

template <typename S>
void launch_is_save(const ISFixArgs& a, cudaStream_t s)
{
    const bool walls = a.s.g.wall[0] || a.s.g.wall[1] || a.s.g.wall[2];
    if (a.s.lattice == 0) launch_is_save_l<D2Q9, S, false>(a, nullptr, dim3(256), walls, s);
    else launch_is_save_l<D3Q19, S, false>(a, nullptr, dim3(256), walls, s);
}

template <typename S>
void launch_is_fix(const ISFixArgs& a, cudaStream_t s)
{
    if (a.s.lattice == 0) k_is_fix<D2Q9, S, false><<<256, 128, 0, s>>>(a, nullptr);
    else k_is_fix<D3Q19, S, false><<<256, 128, 0, s>>>(a, nullptr);
}

template <typename S>
void launch_inplace_fix(const ISFixArgs& a, cudaStream_t s)
{
    const bool walls = a.s.g.wall[0] || a.s.g.wall[1] || a.s.g.wall[2];
    if (a.s.lattice == 0) {
        if (walls) k_inplace_fix<D2Q9, S, true><<<256, 128, 0, s>>>(a);
        else k_inplace_fix<D2Q9, S, false><<<256, 128, 0, s>>>(a);
    } else {
        if (walls) k_inplace_fix<D3Q19, S, true><<<256, 128, 0, s>>>(a);
        else k_inplace_fix<D3Q19, S, false><<<256, 128, 0, s>>>(a);
    }
}

template <typename S>
void launch_update_masks(const MaskArgs& a, cudaStream_t s)
{
    if (a.lattice == 0) k_update_masks<D2Q9, false><<<304, 128, 0, s>>>(a, nullptr);
    else k_update_masks<D3Q19, false><<<304, 128, 0, s>>>(a, nullptr);
}

// Batched forms (one lattice for every cell of a batch; walls: some cell has them).
template <typename S>
void launch_is_save_batch(int lattice, const ISFixArgs* cells, int nc, cudaStream_t s)
{
    const dim3 grid(std::max(2, 256 / nc), nc);
    if (lattice == 0) launch_is_save_l<D2Q9, S, true>(ISFixArgs{}, cells, grid, true, s);
    else launch_is_save_l<D3Q19, S, true>(ISFixArgs{}, cells, grid, true, s);
}

template <typename S>
void launch_is_fix_batch(int lattice, const ISFixArgs* cells, int nc, cudaStream_t s)
{
    const dim3 grid(std::max(2, 256 / nc), nc);
    if (lattice == 0) k_is_fix<D2Q9, S, true><<<grid, 128, 0, s>>>(ISFixArgs{}, cells);
    else k_is_fix<D3Q19, S, true><<<grid, 128, 0, s>>>(ISFixArgs{}, cells);
}

template <typename S>
void launch_update_masks_batch(int lattice, const MaskArgs* cells, int nc, cudaStream_t s)
{
    const dim3 grid(std::max(2, 304 / nc), nc);
    if (lattice == 0) k_update_masks<D2Q9, true><<<grid, 128, 0, s>>>(MaskArgs{}, cells);
    else k_update_masks<D3Q19, true><<<grid, 128, 0, s>>>(MaskArgs{}, cells);
}

template <class L, typename S, bool WALLS, bool PART>
void launch_sweep_batch_v(const BatchSweepArgs& b, cudaStream_t s)
{
    const unsigned grid = b.grid > 0 ? (unsigned)b.grid : (unsigned)b.ntiles;
    k_sweep_batch<L, S, WALLS, PART><<<grid, SWEEP_THREADS, 0, s>>>(b);
}

template <class L, typename S>
void launch_sweep_batch_l(const BatchSweepArgs& b, cudaStream_t s)
{
    if (b.walls && b.part) launch_sweep_batch_v<L, S, true, true>(b, s);
    else if (b.walls) launch_sweep_batch_v<L, S, true, false>(b, s);
    else if (b.part) launch_sweep_batch_v<L, S, false, true>(b, s);
    else launch_sweep_batch_v<L, S, false, false>(b, s);
}

template <typename S>
void launch_sweep_batch(const BatchSweepArgs& b, cudaStream_t s)
{
    if (b.ntiles == 0) return;
    if (b.lattice == 0) launch_sweep_batch_l<D2Q9, S>(b, s);
    else launch_sweep_batch_l<D3Q19, S>(b, s);
}

template <typename S>
const KernelTable* make_table()
{
    static const KernelTable t = {launch_sweep<S>,
                                  launch_update_masks<S>,
                                  launch_materialize<S>,
                                  launch_convert_in<S>,
                                  launch_unstream<S>,
                                  launch_fill_rest<S>,
                                  launch_is_save<S>,
                                  launch_is_fix<S>,
                                  launch_sweep_batch<S>,
                                  launch_is_save_batch<S>,
                                  launch_is_fix_batch<S>,
                                  launch_update_masks_batch<S>,
                                  launch_features<S>,
                                  launch_inplace_fix<S>,
                                  (int)sizeof(S),
                                  (int)sizeof(typename Store<S>::C)};
    return &t;
}

}  // namespace lbmp
