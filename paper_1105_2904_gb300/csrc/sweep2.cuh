// Two-site form of the fused sweep for the deviation storages (FP32, FP16, BF16): each thread
// owns a pair of x-neighbouring sites (x0, x0 + 1), x0 even. Populations move as aligned
// pairs (8-byte float2 or 4-byte half2 / bfloat162 accesses) wherever the pull source is the
// same pair of another row, and the collision runs on both sites at once with the packed
// FP32 pair instructions of sm_100+ (FFMA2 / FADD2 / FMUL2). Sites inside particles take the
// same per-site steps as the one-site kernel (IS imposition, BS transfer, density carry),
// applied to each half of the pair. Requires an even nx.
#pragma once

#include "sweep.cuh"

namespace lbmp {

// ---- packed FP32 pairs ---------------------------------------------------------------------
__device__ __forceinline__ float2 p2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, p2(-1.0f), a); }

// ---- storage pairs -------------------------------------------------------------------------
// Aligned loads and stores of two consecutive elements: FP32 storage in its compute form, the
// deviation g = f - w (as Store<float>); the 16-bit storages in their stored units.
template <typename S> struct Pair;
template <> struct Pair<float> {
    __device__ static float2 load(const float* p, float) { return *reinterpret_cast<const float2*>(p); }
    __device__ static void store(float* p, float2 g, float) { *reinterpret_cast<float2*>(p) = g; }
    __device__ static float2 round(float2 g, float) { return g; }
};
// The 16-bit storages: the two-site sweep computes in their stored units h = (f - w) / w.
template <> struct Pair<__half> {
    __device__ static float2 loadh(const __half* p) { return __half22float2(*reinterpret_cast<const __half2*>(p)); }
    __device__ static float loadh1(const __half* p) { return __half2float(*p); }
    __device__ static void storeh(__half* p, float2 h) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(h); }
    __device__ static float2 roundh(float2 h) { return __half22float2(__float22half2_rn(h)); }
};
template <> struct Pair<__nv_bfloat16> {
    __device__ static float2 loadh(const __nv_bfloat16* p)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
    __device__ static float loadh1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static void storeh(__nv_bfloat16* p, float2 h)
    {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(h);
    }
    __device__ static float2 roundh(float2 h) { return __bfloat1622float2(__float22bfloat162_rn(h)); }
};

// Component h (0: site x0, 1: site x0 + 1) of a pair.
template <int H> __device__ __forceinline__ float& half_of(float2& v) { if constexpr (H == 0) return v.x; else return v.y; }

// Neighbours of the pair: n0 for site x0 (x0 + 1 never wraps), n1 for site x0 + 1.
template <bool WALLS>
__device__ __forceinline__ void pair_neighbours(const Geom& g, int x0, int y, int z, Nbr& n0, Nbr& n1)
{
    n0 = neighbours<WALLS>(g, x0, y, z);
    n1 = n0;
    n1.xm = x0;
    n1.bxm = false;
    n1.xp = x0 + 2;
    n1.bxp = false;
    if (n1.xp >= g.nx) {
        n1.xp -= g.nx;
        if (WALLS) n1.bxp = g.wall[0];
    }
}

// Gathers the populations of both sites (pull propagation with bounce-back): a pair load
// when both sources are the same pair of another row (c_x = 0), two loads otherwise. FP32:
// deviations g = f - w; 16-bit storages: their stored units h = (f - w) / w, unconverted.
template <class L, typename S, bool WALLS>
__device__ __forceinline__ void pull2(const S* __restrict__ fin, const Geom& g, const Nbr& n0, const Nbr& n1,
                                      int x0, int y, int z, unsigned idx, float2 f[])
{
    using St = Store<S>;
    const size_t N = g.N;
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        constexpr float w = (float)L::w(i);
        const int sy = cy > 0 ? n0.ym : (cy < 0 ? n0.yp : y);
        const int sz = cz > 0 ? n0.zm : (cz < 0 ? n0.zp : z);
        bool brow = false;
        if constexpr (WALLS)
            brow = (cy > 0 && n0.bym) || (cy < 0 && n0.byp) || (cz > 0 && n0.bzm) || (cz < 0 && n0.bzp);
        const unsigned row = ((unsigned)sz * (unsigned)g.ny + (unsigned)sy) * (unsigned)g.nx;
        const S* own = fin + (size_t)L::opp(i) * N + idx;  // bounced: the site itself, opp(i)
        if constexpr (cx == 0) {
            const S* src = brow ? own : fin + (size_t)i * N + row + (unsigned)x0;
            if constexpr (sizeof(S) == 2) f[i] = Pair<S>::loadh(src);
            else f[i] = Pair<S>::load(src, w);
        } else {
            // source x - c_x of each site; a wall on x bounces only the site beside it
            const int sx0 = cx > 0 ? n0.xm : x0 + 1;
            const int sx1 = cx > 0 ? x0 : n1.xp;
            bool b0 = brow, b1 = brow;
            if constexpr (WALLS) {
                b0 = b0 || (cx > 0 && n0.bxm);
                b1 = b1 || (cx < 0 && n1.bxp);
            }
            const S* p0 = b0 ? own : fin + (size_t)i * N + row + (unsigned)sx0;
            const S* p1 = b1 ? own + 1 : fin + (size_t)i * N + row + (unsigned)sx1;
            if constexpr (sizeof(S) == 2) f[i] = make_float2(Pair<S>::loadh1(p0), Pair<S>::loadh1(p1));
            else f[i] = make_float2(St::load(*p0, w), St::load(*p1, w));
        }
    });
}

// BGK collision with Guo forcing (Eq. 3) of both sites on packed pairs; the same expression
// as collide_dev, one instruction for two sites (CONSERVE: the stored increments' momentum is
// made exact, as collide_dev<L, true> describes).
// HS: g holds the scaled deviations h_i = g_i / w_i of the 16-bit storages (their stored units):
// the moments weigh them by w_i and the update drops the w_i of the equilibrium and forcing
// terms, which are w_i times an expression in c_i, u and F (the same arithmetic, per unit).
template <class L, bool CONSERVE = false, bool HS = false>
__device__ __forceinline__ void collide_dev2(float2 g[], const SweepArgs& a, float2& drho, float2& j0, float2& j1,
                                             float2& j2)
{
    constexpr int Q = L::Q;
    if constexpr (HS) {
        drho = mul2(p2((float)L::w(0)), g[0]);
        j0 = j1 = j2 = p2(0.0f);
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr float w = (float)L::w(i);
            drho = fma2(p2(w), g[i], drho);
            if constexpr (L::c(i, 0) != 0) j0 = fma2(p2(L::c(i, 0) * w), g[i], j0);
            if constexpr (L::c(i, 1) != 0) j1 = fma2(p2(L::c(i, 1) * w), g[i], j1);
            if constexpr (L::c(i, 2) != 0) j2 = fma2(p2(L::c(i, 2) * w), g[i], j2);
        });
    } else {
        drho = g[0];
        j0 = j1 = j2 = p2(0.0f);
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            drho = add2(drho, g[i]);
            if constexpr (L::c(i, 0) > 0) j0 = add2(j0, g[i]);
            if constexpr (L::c(i, 0) < 0) j0 = sub2(j0, g[i]);
            if constexpr (L::c(i, 1) > 0) j1 = add2(j1, g[i]);
            if constexpr (L::c(i, 1) < 0) j1 = sub2(j1, g[i]);
            if constexpr (L::c(i, 2) > 0) j2 = add2(j2, g[i]);
            if constexpr (L::c(i, 2) < 0) j2 = sub2(j2, g[i]);
        });
    }
    const float F0 = a.F_f[0], F1 = a.F_f[1], F2 = a.F_f[2];
    const float2 rho = add2(drho, p2(1.0f));
    const float2 inv = make_float2(1.0f / rho.x, 1.0f / rho.y);
    const float2 u0 = mul2(add2(j0, p2(0.5f * F0)), inv);
    const float2 u1 = mul2(add2(j1, p2(0.5f * F1)), inv);
    const float2 u2 = mul2(add2(j2, p2(0.5f * F2)), inv);
    const float omega = a.omega_f, pre = a.pre_f, om1 = 1.0f - omega;
    const float2 uF3 = mul2(p2(3.0f), fma2(u2, p2(F2), fma2(u1, p2(F1), mul2(u0, p2(F0)))));
    const float2 usq15 = mul2(p2(1.5f), fma2(u2, u2, fma2(u1, u1, mul2(u0, u0))));
    float2 S[3] = {p2(0.0f), p2(0.0f), p2(0.0f)};  // CONSERVE: momentum of the stored increments
    {   // rest direction
        const float w = HS ? 1.0f : (float)L::w(0);
        const float2 e = fma2(rho, mul2(usq15, p2(-1.0f)), drho);  // drho - rho usq15
        g[0] = fma2(p2(om1), g[0], fma2(p2(omega * w), e, mul2(p2(-pre * w), uF3)));
    }
    sfor<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int j = L::opp(i);
        if constexpr (j > i) {
            constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
            float2 cu = p2(0.0f);
            bool first = true;
            auto acc = [&](int c, float2 v) {
                if (c == 0) return;
                if (first) {
                    cu = c > 0 ? v : mul2(v, p2(-1.0f));
                    first = false;
                } else {
                    cu = c > 0 ? add2(cu, v) : sub2(cu, v);
                }
            };
            acc(cx, u0);
            acc(cy, u1);
            acc(cz, u2);
            const float cF = (float)cx * F0 + (float)cy * F1 + (float)cz * F2;
            const float w = HS ? 1.0f : (float)L::w(i);
            const float ow = omega * w, pw = pre * w;
            // A = ow (drho + rho (4.5 cu^2 - 1.5 u^2)) + pw (9 cu cF - 3 u.F)
            const float2 q = fma2(mul2(cu, cu), p2(4.5f), mul2(usq15, p2(-1.0f)));
            const float2 A = fma2(p2(ow), fma2(rho, q, drho), mul2(p2(pw), fma2(cu, p2(9.0f * cF), mul2(uF3, p2(-1.0f)))));
            // B = 3 (ow rho cu + pw cF)
            const float2 B = mul2(p2(3.0f), fma2(mul2(p2(ow), rho), cu, p2(pw * cF)));
            const float2 gi = fma2(p2(om1), g[i], add2(A, B));
            const float2 gj = fma2(p2(om1), g[j], sub2(A, B));
            if constexpr (CONSERVE) {
                const float2 d = sub2(sub2(gi, g[i]), sub2(gj, g[j]));  // c_j = -c_i
                if constexpr (cx > 0) S[0] = add2(S[0], d);
                if constexpr (cx < 0) S[0] = sub2(S[0], d);
                if constexpr (cy > 0) S[1] = add2(S[1], d);
                if constexpr (cy < 0) S[1] = sub2(S[1], d);
                if constexpr (cz > 0) S[2] = add2(S[2], d);
                if constexpr (cz < 0) S[2] = sub2(S[2], d);
            }
            g[i] = gi;
            g[j] = gj;
        }
    });
    if constexpr (CONSERVE) {
        const float Fk[3] = {F0, F1, F2};
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
            if constexpr (cx * cx + cy * cy + cz * cz == 1) {
                constexpr int axis = cx != 0 ? 0 : (cy != 0 ? 1 : 2);
                const float2 half = mul2(p2(0.5f), sub2(p2(Fk[axis]), S[axis]));
                g[i] = (cx + cy + cz) > 0 ? add2(g[i], half) : sub2(g[i], half);
            }
        });
    }
}

// Lever arms of both sites (each from its own owner's record) as pairs.
template <typename K>
__device__ __forceinline__ void lever_arm2(const Geom& g, const K& k0, const K& k1, int x0, int y, int z, float2 r[3])
{
    float r0[3], r1[3];
    lever_arm(g, k0, x0, y, z, r0);
    lever_arm(g, k1, x0 + 1, y, z, r1);
#pragma unroll
    for (int q = 0; q < 3; ++q) r[q] = make_float2(r0[q], r1[q]);
}

// u_p + omega_p x r (Eqs. 5, 12) for both sites.
__device__ __forceinline__ void rigid_velocity2(const float2 u[3], const float2 om[3], const float2 r[3], float2 out[3])
{
    out[0] = fma2(om[1], r[2], sub2(u[0], mul2(om[2], r[1])));
    out[1] = fma2(om[2], r[0], sub2(u[1], mul2(om[0], r[2])));
    out[2] = fma2(om[0], r[1], sub2(u[2], mul2(om[1], r[0])));
}

__device__ __forceinline__ void kin2(const PKernF& k0, const PKernF& k1, float2 u[3], float2 om[3])
{
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        u[q] = make_float2(k0.u[q], k1.u[q]);
        om[q] = make_float2(k0.om[q], k1.om[q]);
    }
}

// c_i . v of a lattice direction on pairs (components 0 or +-1: adds only).
template <class L, int i>
__device__ __forceinline__ float2 cdot2(const float2 v[3])
{
    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
    float2 r = p2(0.0f);
    bool first = true;
    auto acc = [&](int c, float2 w) {
        if (c == 0) return;
        if (first) {
            r = c > 0 ? w : mul2(w, p2(-1.0f));
            first = false;
        } else {
            r = c > 0 ? add2(r, w) : sub2(r, w);
        }
    };
    acc(cx, v[0]);
    acc(cy, v[1]);
    acc(cz, v[2]);
    return r;
}

// The pending IS imposition (Eq. 12) for both sites of the pair, on packed pairs: the same
// expression as substitute_is_dev (density carry: the pulled value is rho_I of its source),
// each site with its own owner and IS-source mask. Warp-uniform; every lane calls it.
// One site of the pair in the deviation units g of the scalar (one-site) code paths, and back:
// HS pairs hold h = g / w (a value the scalar path leaves unchanged comes back within an FP32
// rounding, far below the 16-bit storage's).
template <class L, bool HS, int H>
__device__ __forceinline__ void to_g_half(const float2 f[], float fs[])
{
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float v = half_of<H>(const_cast<float2&>(f[i]));
        fs[i] = HS ? v * (float)L::w(i) : v;
    });
}
template <class L, bool HS, int H>
__device__ __forceinline__ void from_g_half(const float fs[], float2 f[])
{
    sfor<0, L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        half_of<H>(f[i]) = HS ? fs[i] * (1.0f / (float)L::w(i)) : fs[i];
    });
}

template <class L, bool WALLS, bool HS = false>
__device__ __forceinline__ void substitute_is_dev2(const Geom& g, const Nbr& n0, const Nbr& n1, int x0, int y, int z,
                                                   uint2 m, uint2 tags, const PartView& pv, float2 f[])
{
    constexpr int Q = L::Q;
    const unsigned mm0 = m.x & ~MASK_OTHER, mm1 = m.y & ~MASK_OTHER;
    const unsigned wm = __reduce_or_sync(__activemask(), mm0 | mm1);
    if (wm) {
        unsigned w0 = mm0 ? (tags.x & PID_MASK) : 0u, w1 = mm1 ? (tags.y & PID_MASK) : 0u;
        if (!LBM_DCHECK(pv.status, w0 < (unsigned)pv.np)) w0 = 0u;
        if (!LBM_DCHECK(pv.status, w1 < (unsigned)pv.np)) w1 = 0u;
        const PKernF k0 = pv.pkf[w0];
        const PKernF k1 = pv.pkf[w1];
        float2 r[3], u[3], om[3], ux[3];
        lever_arm2(g, k0, k1, x0, y, z, r);
        kin2(k0, k1, u, om);
        rigid_velocity2(u, om, r, ux);
        float2 b[3];  // u(x) + u(x) x omega
        b[0] = add2(ux[0], sub2(mul2(ux[1], om[2]), mul2(ux[2], om[1])));
        b[1] = add2(ux[1], sub2(mul2(ux[2], om[0]), mul2(ux[0], om[2])));
        b[2] = add2(ux[2], sub2(mul2(ux[0], om[1]), mul2(ux[1], om[0])));
        const float2 usq = fma2(ux[2], ux[2], fma2(ux[1], ux[1], mul2(ux[0], ux[0])));
        const float2 w2 = fma2(om[2], om[2], fma2(om[1], om[1], mul2(om[0], om[0])));
        // -1.5 (|u(x)|^2 + |omega|^2 |c|^2) for |c|^2 = 1 and 2
        const float2 usq15 = mul2(p2(-1.5f), usq);
        const float2 B1 = fma2(p2(-1.5f), w2, usq15), B2 = fma2(p2(-3.0f), w2, usq15);
        if (wm & 1u) {
            const float2 E = mul2(p2(-1.5f), usq);
            // HS: the IS slot holds its density deviation over w_0; the result is in h units
            const float2 v = HS ? fma2(mul2(p2((float)L::w(0)), f[0]), add2(E, p2(1.0f)), E)
                                : mul2(p2((float)L::w(0)), fma2(f[0], add2(E, p2(1.0f)), E));
            if (mm0 & 1u) f[0].x = v.x;
            if (mm1 & 1u) f[0].y = v.y;
        }
        sfor<1, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int j = L::opp(i);
            if constexpr (j > i) {
                constexpr unsigned pair = (1u << i) | (1u << j);
                if (wm & pair) {
                    constexpr float c2 = (float)(L::c(i, 0) * L::c(i, 0) + L::c(i, 1) * L::c(i, 1) + L::c(i, 2) * L::c(i, 2));
                    constexpr float w = (float)L::w(i);
                    const float2 cu = cdot2<L, i>(ux);
                    const float2 cb = cdot2<L, i>(b);
                    const float2 cw = cdot2<L, i>(om);
                    // E = 4.5 cu^2 + 1.5 cw^2 - 1.5 (|u|^2 + |omega|^2 |c|^2) +- 3 cb
                    const float2 S = fma2(cu, mul2(p2(4.5f), cu), fma2(cw, mul2(p2(1.5f), cw), c2 == 1.0f ? B1 : B2));
                    float2 Ei = fma2(cb, p2(3.0f), S), Ej = fma2(cb, p2(-3.0f), S);
                    if constexpr (WALLS) {
                        const float2 Sb = fma2(mul2(cu, cu), p2(4.5f), mul2(usq, p2(-1.5f)));
                        const float2 cu3 = mul2(p2(3.0f), cu);
                        if (pull_bounces<L, i, WALLS>(n0)) Ei.x = Sb.x - cu3.x;
                        if (pull_bounces<L, i, WALLS>(n1)) Ei.y = Sb.y - cu3.y;
                        if (pull_bounces<L, j, WALLS>(n0)) Ej.x = Sb.x + cu3.x;
                        if (pull_bounces<L, j, WALLS>(n1)) Ej.y = Sb.y + cu3.y;
                    }
                    const float2 vi = HS ? fma2(mul2(p2(w), f[i]), add2(Ei, p2(1.0f)), Ei)
                                         : mul2(p2(w), fma2(f[i], add2(Ei, p2(1.0f)), Ei));
                    const float2 vj = HS ? fma2(mul2(p2(w), f[j]), add2(Ej, p2(1.0f)), Ej)
                                         : mul2(p2(w), fma2(f[j], add2(Ej, p2(1.0f)), Ej));
                    if (mm0 & (1u << i)) f[i].x = vi.x;
                    if (mm1 & (1u << i)) f[i].y = vi.y;
                    if (mm0 & (1u << j)) f[j].x = vj.x;
                    if (mm1 & (1u << j)) f[j].y = vj.y;
                }
            }
        });
    }
    if ((m.x | m.y) & MASK_OTHER) {
        float fs[Q];
        if (m.x & MASK_OTHER) {
            to_g_half<L, HS, 0>(f, fs);
            substitute_is_other_dev<L, WALLS>(g, n0, x0, y, z, tags.x & PID_MASK, pv, fs);
            from_g_half<L, HS, 0>(fs, f);
        }
        if (m.y & MASK_OTHER) {
            to_g_half<L, HS, 1>(f, fs);
            substitute_is_other_dev<L, WALLS>(g, n1, x0 + 1, y, z, tags.y & PID_MASK, pv, fs);
            from_g_half<L, HS, 1>(fs, f);
        }
    }
}

// Moving-wall momentum of the bounced values of one site of the pair.
template <class L, bool WALLS, int H, bool HS = false>
__device__ __forceinline__ void wall_momentum_half(const SweepArgs& a, const Nbr& n, float2 f[])
{
    constexpr int Q = L::Q;
    float fs[Q];
    to_g_half<L, HS, H>(f, fs);
    wall_momentum<L, float, WALLS>(n, a.g.eqface, a.uw->uf, fs);
    from_g_half<L, HS, H>(fs, f);
}

// Equilibrium-face value f^eq(rho, u) of one site of the pair (deviation form).
template <class L, int H, bool HS = false>
__device__ __forceinline__ void eq_face_half(const float u[3], float drho, float2 f[])
{
    constexpr int Q = L::Q;
    float fs[Q];
    equilibrium_dev<L>(drho, u, fs);
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        half_of<H>(f[i]) = HS ? fs[i] * (1.0f / (float)L::w(i)) : fs[i];
    });
}

// BS transfer (Eqs. 5-7) of the BS sites of the pair on packed pairs: the same expression
// as bs_transfer_dev; each BS site takes f^eq(rho_B, u_p + omega_p x r) and writes its
// per-site record.
template <class L, bool BRICK, bool HS = false>
__device__ __forceinline__ void bs_transfer_dev2(const SweepArgs& a, int x0, int y, int z, unsigned idx, uint2 tags,
                                                 bool bs0, bool bs1, float2 mrho, float2 mj0, float2 mj1, float2 mj2,
                                                 float2 f[])
{
    constexpr int Q = L::Q;
    unsigned p0 = tags.x & PID_MASK, p1 = tags.y & PID_MASK;
    if (!LBM_DCHECK(a.pv.status, !bs0 || p0 < (unsigned)a.pv.np)) p0 = 0u;
    if (!LBM_DCHECK(a.pv.status, !bs1 || p1 < (unsigned)a.pv.np)) p1 = 0u;
    const PKernF k0 = a.pv.pkf[bs0 ? p0 : p1];
    const PKernF k1 = a.pv.pkf[bs1 ? p1 : p0];
    float2 r[3], u[3], om[3], ub[3];
    lever_arm2(a.g, k0, k1, x0, y, z, r);
    kin2(k0, k1, u, om);
    rigid_velocity2(u, om, r, ub);
    const float2 rho = add2(mrho, p2(1.0f));
    const float2 usq15 = mul2(p2(1.5f), fma2(ub[2], ub[2], fma2(ub[1], ub[1], mul2(ub[0], ub[0]))));
    {   // (HS: in h units, without the w_i factor)
        const float2 e = mul2(p2(HS ? 1.0f : (float)L::w(0)), fma2(rho, mul2(usq15, p2(-1.0f)), mrho));
        if (bs0) f[0].x = e.x;
        if (bs1) f[0].y = e.y;
    }
    sfor<1, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int j = L::opp(i);
        if constexpr (j > i) {
            constexpr float w = HS ? 1.0f : (float)L::w(i);
            const float2 cu = cdot2<L, i>(ub);
            const float2 even = mul2(p2(w), fma2(rho, fma2(mul2(cu, cu), p2(4.5f), mul2(usq15, p2(-1.0f))), mrho));
            const float2 odd = mul2(p2(3.0f * w), mul2(rho, cu));
            const float2 gi = add2(even, odd), gj = sub2(even, odd);
            if (bs0) {
                f[i].x = gi.x;
                f[j].x = gj.x;
            }
            if (bs1) {
                f[i].y = gi.y;
                f[j].y = gj.y;
            }
        }
    });
    // dp = rho_B u_B' - (j + F) (Eq. 6); the torque is formed in the particle phase
    float2 dv[3];
    dv[0] = sub2(mul2(rho, ub[0]), add2(mj0, p2(a.F_f[0])));
    dv[1] = sub2(mul2(rho, ub[1]), add2(mj1, p2(a.F_f[1])));
    dv[2] = sub2(mul2(rho, ub[2]), add2(mj2, p2(a.F_f[2])));
    // (x0 is even: the pair's two records are adjacent in either layout)
    float4* sc = (float4*)a.bs_scratch + (BRICK ? rec_brick_index(a.g, x0, y, z) : idx);
    if (bs0) sc[0] = make_float4(dv[0].x, dv[1].x, dv[2].x, __uint_as_float(tags.x));
    if (bs1) sc[1] = make_float4(dv[0].y, dv[1].y, dv[2].y, __uint_as_float(tags.y));
}

// One block: BX threads along x (2 BX sites) times 128 / BX rows of one z-plane, five blocks per
// SM (96 registers, no spills). The 16-bit storages compute in their stored units
// h = (f - w) / w, which saves the scaling of every load and store (FP16 sweep 3.350 -> 3.324 ms
// at the 512^3 suspension); with that and the IS-source masks loaded only at solid pairs they
// run best at five blocks as well (3.225 ms at six blocks and 80 registers, with spills; seven
// blocks spill far more), as FP32 always did (six blocks measured slower).
template <class L, typename S, bool WALLS, bool PART, int BX>
__global__ void __launch_bounds__(SWEEP_THREADS, 5) k_sweep2(const SweepArgs a)
{
    constexpr int Q = L::Q;
    constexpr int BY = SWEEP_THREADS / BX;
    const Geom& g = a.g;
    const int tx = (int)threadIdx.x % BX, ty = (int)threadIdx.x / BX;
    const int xr = (int)blockIdx.x * (2 * BX) + 2 * tx;
    const int yr = (int)blockIdx.y * BY + ty;
    const int z = (int)blockIdx.z;
    const bool valid = xr < g.nx && yr < g.ny;
    const int x0 = min(xr, g.nx - 2), y = min(yr, g.ny - 1);
    const unsigned idx = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx + (unsigned)x0;
    Nbr n0, n1;
    pair_neighbours<WALLS>(g, x0, y, z, n0, n1);
    // 16-bit storages: the pair values stay in the stored units h = (f - w) / w throughout
    constexpr bool HS = sizeof(S) == 2;
    uint2 tg = make_uint2(TAG_FLUID, TAG_FLUID), mk = make_uint2(0u, 0u);
    if constexpr (PART) {
        tg = *reinterpret_cast<const uint2*>(a.pv.tag + idx);
        if constexpr (!HS) mk = *reinterpret_cast<const uint2*>(a.pv.ismask + idx);
    }
    float2 f[Q];
    pull2<L, S, WALLS>((const S*)a.fin, g, n0, n1, x0, y, z, idx, f);
    // 16-bit storages: the IS-source masks only where a site of the pair is solid (fluid sites
    // never pull from an IS site), after the pulls so that the wait for the owner tags delays none
    // of them (FP16 sweep 3.335 -> 3.231 ms at the 512^3 suspension; the same in FP32, bound by
    // memory rather than issue, measured 3.573 -> 3.784 ms, so FP32 loads them with the tags)
    if constexpr (PART && HS)
        if (tg.x != TAG_FLUID || tg.y != TAG_FLUID) mk = *reinterpret_cast<const uint2*>(a.pv.ismask + idx);
    if constexpr (PART) {
        if (*a.pv.pending) {
            const uint2 m = make_uint2(tg.x != TAG_FLUID ? mk.x : 0u, tg.y != TAG_FLUID ? mk.y : 0u);
            substitute_is_dev2<L, WALLS, HS>(g, n0, n1, x0, y, z, m, tg, a.pv, f);
        }
    }
    // A moving wall acts on the bounced value after the IS imposition it may have received.
    if constexpr (WALLS) {
        if (a.moving_walls && *a.pv.pending) {
            wall_momentum_half<L, WALLS, 0, HS>(a, n0, f);
            wall_momentum_half<L, WALLS, 1, HS>(a, n1, f);
        }
    }
    float2 mrho, mj0, mj1, mj2;
    collide_dev2<L, std::is_same<S, float>::value, HS>(f, a, mrho, mj0, mj1, mj2);
    bool any_is = false;
    bool is0 = false, is1 = false;
    if constexpr (PART) {
        const bool bs0 = valid && (tg.x >> 30) == CLS_BS, bs1 = valid && (tg.y >> 30) == CLS_BS;
        if (bs0 || bs1)
            bs_transfer_dev2<L, std::is_same<S, float>::value, HS>(a, x0, y, z, idx, tg, bs0, bs1, mrho, mj0, mj1,
                                                                  mj2, f);
        is0 = (tg.x >> 30) == CLS_IS;
        is1 = (tg.y >> 30) == CLS_IS;
        any_is = __any_sync(0xFFFFFFFFu, is0 || is1);
    }
    // Equilibrium faces: fluid sites on one take f^eq(rho, u_face) (as the one-site kernel).
    if constexpr (WALLS) {
        if (g.eqface) {
            const int f0 = eq_face_of(g, x0, y, z), f1 = eq_face_of(g, x0 + 1, y, z);
            if (f0 >= 0 && tg.x == TAG_FLUID) eq_face_half<L, 0, HS>(a.uw[1].uf[f0], mrho.x, f);
            if (f1 >= 0 && tg.y == TAG_FLUID) eq_face_half<L, 1, HS>(a.uw[1].uf[f1], mrho.y, f);
        }
    }
    if (!valid) return;
    S* __restrict__ fout = (S*)a.fout;
    const size_t N = g.N;
    if (any_is) {
        // density carry: an IS site stores its post-collision density (the sum of its values
        // as stored) in every slot
        float2 dens = p2(0.0f);
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            if constexpr (HS) dens = fma2(p2((float)L::w(i)), Pair<S>::roundh(f[i]), dens);
            else dens = add2(dens, Pair<S>::round(f[i], (float)L::w(i)));
        });
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            float2 v = f[i];
            if constexpr (HS) {
                const float2 dh = mul2(dens, p2(1.0f / (float)L::w(i)));
                if (is0) v.x = dh.x;
                if (is1) v.y = dh.y;
                Pair<S>::storeh(fout + (size_t)i * N + idx, v);
            } else {
                if (is0) v.x = dens.x;
                if (is1) v.y = dens.y;
                Pair<S>::store(fout + (size_t)i * N + idx, v, (float)L::w(i));
            }
        });
    } else {
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            if constexpr (HS) Pair<S>::storeh(fout + (size_t)i * N + idx, f[i]);
            else Pair<S>::store(fout + (size_t)i * N + idx, f[i], (float)L::w(i));
        });
    }
}

template <class L, typename S, bool WALLS, bool PART>
void launch_sweep2_v(const SweepArgs& a, int bx, cudaStream_t s)
{
    const int by = SWEEP_THREADS / bx;
    const dim3 grid((a.g.nx + 2 * bx - 1) / (2 * bx), (a.g.ny + by - 1) / by, a.g.nz);
    switch (bx) {
    case 16: k_sweep2<L, S, WALLS, PART, 16><<<grid, SWEEP_THREADS, 0, s>>>(a); break;
    case 32: k_sweep2<L, S, WALLS, PART, 32><<<grid, SWEEP_THREADS, 0, s>>>(a); break;
    case 64: k_sweep2<L, S, WALLS, PART, 64><<<grid, SWEEP_THREADS, 0, s>>>(a); break;
    default: k_sweep2<L, S, WALLS, PART, 128><<<grid, SWEEP_THREADS, 0, s>>>(a); break;
    }
}

}  // namespace lbmp
