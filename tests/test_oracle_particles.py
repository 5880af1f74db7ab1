"""Pins of the oracle's particle coupling (Sec. 2.2-2.3, Eqs. 5-19).

Classification is checked against a brute-force classifier written here from the
definitions (every grid site tested directly, no template); the momentum transfer and the
internal-site imposition against first-step closed forms; the coupling against exact momentum and mass budgets; the
rotation sign against spin-down; the hard-core collisions against the conservation laws.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1105_2904_gb300 import workloads as W

FLUID = 0xFFFFFFFF


def brute_force_tags(lattice, shape, walls, particles):
    """Owner map computed site by site from the definitions.

    particles: list of (x0 (3,), r, s (3,)) with s the integer shift of the site set.
    S = sites y with |(y - s) - x0|^2 <= r^2 (minimum image on periodic axes, evaluated as
    an integer offset from floor(x0) minus the fractional part); BS = sites of S with a
    lattice neighbour outside S; IS = other sites of S with a neighbour in BS; IN = rest.
    Ties in ownership go to IS, then BS, then IN, then the lowest particle id.
    """
    c, _ = O.lattice_tables(lattice)
    nz, ny, nx = shape
    dims = (nx, ny, nz)
    pad = [2 if walls[k] else 0 for k in range(3)]
    ext = [dims[k] + 2 * pad[k] for k in range(3)]
    zz, yy, xx = np.meshgrid(np.arange(ext[2]) - pad[2], np.arange(ext[1]) - pad[1],
                             np.arange(ext[0]) - pad[0], indexing="ij")
    coords = [xx, yy, zz]
    tags = np.full(tuple(ext[::-1]), FLUID, dtype=np.uint64)
    D = 2 if lattice == O.D2Q9 else 3
    for pid, (x0, r, s) in enumerate(particles):
        A = np.floor(x0).astype(np.int64)
        phi = x0 - A
        d2 = np.zeros(tags.shape)
        for k in range(3):
            o = coords[k] - A[k] - int(s[k])
            if not walls[k] and k < D:
                o = (o + dims[k] // 2) % dims[k] - dims[k] // 2
            if k >= D:
                o = np.zeros_like(o)
            dk = o.astype(np.float64) - phi[k]
            d2 = d2 + dk * dk
        inS = d2 <= r * r

        def nb(a, ci):
            # a at y + c_i, periodic axes wrap (np.roll), padded wall axes never reach S
            return np.roll(a, shift=(-ci[2], -ci[1], -ci[0]), axis=(0, 1, 2))

        bs = np.zeros_like(inS)
        for ci in c[1:]:
            bs |= inS & ~nb(inS, ci)
        is_ = np.zeros_like(inS)
        for ci in c[1:]:
            is_ |= inS & ~bs & nb(bs, ci)
        cls = np.where(is_, 0, np.where(bs, 1, 2))
        code = (cls.astype(np.uint64) << np.uint64(30)) | np.uint64(pid)
        tags = np.where(inS, np.minimum(tags, code), tags)
    sl = tuple(slice(pad[k], pad[k] + dims[k]) for k in (2, 1, 0))
    return tags[sl].astype(np.uint32)


def _sim(lattice, shape, tau=0.8, walls=(0, 0, 0), **kw):
    nz, ny, nx = shape
    return O.OracleSim(lattice, nx, ny, nz, tau, walls=walls, **kw)


CASES_2D = [(O.D2Q9, (1, 40, 36))]
CASES_3D = [(O.D3Q19, (24, 24, 24))]


@pytest.mark.parametrize("lattice,shape", CASES_2D + CASES_3D)
def test_classification_matches_brute_force(lattice, shape):
    g = W.rng(101 + lattice)
    D = 2 if lattice == O.D2Q9 else 3
    nz, ny, nx = shape
    for trial in range(60):
        r = g.uniform(1.5, 9.9 if D == 2 else 9.5)
        x0 = np.zeros(3)
        x0[:D] = g.uniform(0.0, 1.0, size=D) * np.array([nx, ny, nz])[:D]
        if trial % 5 == 0:            # integer centres: points exactly on the sphere
            x0[:D] = np.round(x0[:D])
            r = float(round(r))
        if trial % 7 == 1:            # half-integer fractional parts
            x0[:D] = np.floor(x0[:D]) + 0.5
        s = _sim(lattice, shape)
        s.add_particles(x0[None], [r], [1.3])
        expect = brute_force_tags(lattice, shape, (0, 0, 0), [(x0, r, np.zeros(3))])
        np.testing.assert_array_equal(s.get_tags(), expect)


@pytest.mark.parametrize("lattice,shape", CASES_2D + CASES_3D)
def test_classification_after_shifts(lattice, shape):
    # A very heavy particle keeps its velocity; its site set must be the initial set
    # translated by floor(x - x0 + 1/2) (Eqs. 14-15), wrapped periodically.
    D = 2 if lattice == O.D2Q9 else 3
    g = W.rng(202 + lattice)
    for trial in range(4):
        r = g.uniform(3.0, 6.0)
        x0 = np.zeros(3)
        x0[:D] = g.uniform(0, 1, size=D) * np.array(shape[::-1])[:D]
        v = np.zeros(3)
        v[:D] = g.uniform(-0.35, 0.35, size=D)
        s = _sim(lattice, shape)
        s.add_particles(x0[None], [r], [1e12], velocities=v[None])
        for _ in range(7):
            s.step(1)
            x = s.get_particles()["x"][0]
            shift = np.floor((x - x0) + 0.5)
            shift[D:] = 0
            expect = brute_force_tags(lattice, shape, (0, 0, 0), [(x0, r, shift)])
            np.testing.assert_array_equal(s.get_tags(), expect)


def test_classification_with_walls_and_conflicts():
    # Several close particles in a walled 2D box: ownership follows IS > BS > IN > lowest id.
    lattice, shape, walls = O.D2Q9, (1, 48, 50), (1, 1, 0)
    centers = np.array([[10.3, 10.9, 0], [20.9, 11.2, 0], [15.5, 20.2, 0], [30.0, 30.0, 0],
                        [39.7, 38.6, 0]])
    radii = np.array([5.1, 5.2, 4.4, 6.0, 5.5])
    s = _sim(lattice, shape, walls=walls)
    s.add_particles(centers, radii, np.full(5, 1.5))
    expect = brute_force_tags(lattice, shape, walls,
                              [(centers[i], radii[i], np.zeros(3)) for i in range(5)])
    got = s.get_tags()
    np.testing.assert_array_equal(got, expect)
    # the two first disks are 0.29 apart: their discrete sets do meet
    owners = got[got != FLUID] & ((1 << 30) - 1)
    assert {0, 1, 2, 3, 4} <= set(np.unique(owners).tolist())


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_template_invariants(lattice):
    c, _ = O.lattice_tables(lattice)
    D = 2 if lattice == O.D2Q9 else 3
    shape = (1, 40, 40) if D == 2 else (24, 24, 24)
    g = W.rng(303)
    for _ in range(20):
        r = g.uniform(1.5, 8.0)
        x0 = np.zeros(3)
        x0[:D] = g.uniform(8, 16, size=D)
        s = _sim(lattice, shape)
        s.add_particles(x0[None], [r], [2.0])
        t = s.get_template(0)
        cls = {tuple(e[:3]): e[3] for e in t}
        # z, y, x lexicographic order of offsets
        keys = [(e[2], e[1], e[0]) for e in t]
        assert keys == sorted(keys)
        for o, k in cls.items():
            nbrs = [tuple(np.array(o) + ci) for ci in c[1:]]
            if k == 1:          # BS: some neighbour outside S
                assert any(n not in cls for n in nbrs)
            else:               # IS/IN: all neighbours in S
                assert all(n in cls for n in nbrs)
            if k == 2:          # IN: no neighbour in BS
                assert all(cls[n] != 1 for n in nbrs)
            if k == 0:
                assert any(cls[n] == 1 for n in nbrs)


@pytest.mark.parametrize("D,r,count", [(2, 2.0, 13), (2, 5.0, 81), (2, 10.0, 317), (3, 2.0, 33),
                                       (3, 8.0, 2109)])
def test_solid_site_counts_of_integer_centres(D, r, count):
    # Lattice points with |y|^2 <= r^2: 2D counts 13, 81, 317 (Gauss circle problem) and 3D
    # counts 33, 2109; the brute-force count is re-checked here.
    rng_ = np.arange(-int(r) - 1, int(r) + 2)
    grids = np.meshgrid(*([rng_] * D), indexing="ij")
    assert int((sum(g_ * g_ for g_ in grids) <= r * r).sum()) == count
    lattice = O.D2Q9 if D == 2 else O.D3Q19
    shape = (1, 32, 32) if D == 2 else (24, 24, 24)
    x0 = np.array([12.0, 12.0, 12.0 if D == 3 else 0.0])
    s = _sim(lattice, shape)
    s.add_particles(x0[None], [r], [2.0])
    assert len(s.get_template(0)) == count


def _bs_lever_arms(s, x0):
    t = s.get_template(0)
    phi = x0 - np.floor(x0)
    bs = t[t[:, 3] == 1][:, :3].astype(np.float64)
    return bs - phi


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_first_step_translation_closed_form(lattice):
    # Fluid at rest (f = w_i, rho = 1), a particle moving at U: every BS site receives
    # dp = rho_B (U - 0) = U (Eq. 6), so dP_B = N_BS U (Eq. 8), u' = U - N_BS U / m (Eq. 10),
    # and dL_B = (sum of lever arms) x U (Eqs. 7, 9).
    D = 2 if lattice == O.D2Q9 else 3
    shape = (1, 40, 40) if D == 2 else (24, 24, 24)
    x0 = np.array([19.37, 20.81, 11.6 if D == 3 else 0.0])
    U = np.array([0.01, -0.004, 0.003 if D == 3 else 0.0])
    r, rho_p = 6.3, 1.7
    s = _sim(lattice, shape)
    s.add_particles(x0[None], [r], [rho_p], velocities=U[None])
    s.step(1)
    arms = _bs_lever_arms(s, x0)
    nbs = len(arms)
    expect_brute = brute_force_tags(lattice, shape, (0, 0, 0), [(x0, r, np.zeros(3))])
    assert nbs == int(((expect_brute >> 30) == 1).sum())
    m = rho_p * ((4.0 / 3.0) * math.pi * r ** 3 if D == 3 else math.pi * r ** 2)
    p = s.get_particles()
    # (rho_B = sum of the rest weights is 1 up to round-off; hence relative 1e-13)
    np.testing.assert_allclose(p["force"][0], -nbs * U, rtol=1e-13, atol=1e-18)
    # the lever arms nearly cancel: bound the error by the size of the summed terms
    scale = np.abs(arms).sum() * np.abs(U).max()
    np.testing.assert_allclose(p["torque"][0], -np.cross(arms.sum(0), U), rtol=0, atol=1e-14 * scale)
    expect_u = U - nbs * U / m
    # the particle then moves by u' (Eq. 13)
    np.testing.assert_allclose(p["u"][0], expect_u, rtol=1e-13, atol=1e-18)
    np.testing.assert_allclose(p["x"][0], x0 + expect_u, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_first_step_rotation_closed_form_spins_down(lattice):
    # Fluid at rest, a particle spinning at omega: BS sites get u' = omega x r (Eq. 5 read as
    # a rigid-body velocity), dl = r x (omega x r), so dL_B = sum(|r|^2 omega - (r.omega) r),
    # a positive-definite map of omega: Eq. 11 then reduces |omega| (spin-down).
    D = 2 if lattice == O.D2Q9 else 3
    shape = (1, 40, 40) if D == 2 else (24, 24, 24)
    x0 = np.array([19.6, 20.2, 12.3 if D == 3 else 0.0])
    om = np.array([0.0, 0.0, 0.004]) if D == 2 else np.array([0.002, -0.001, 0.003])
    r, rho_p = 6.7, 1.2
    s = _sim(lattice, shape)
    s.add_particles(x0[None], [r], [rho_p], omegas=om[None])
    s.step(1)
    arms = _bs_lever_arms(s, x0)
    dL = np.zeros(3)
    for a in arms:
        dL += np.cross(a, np.cross(om, a))
    p = s.get_particles()
    np.testing.assert_allclose(p["torque"][0], -dL, rtol=1e-13, atol=1e-17)
    m = rho_p * ((4.0 / 3.0) * math.pi * r ** 3 if D == 3 else math.pi * r ** 2)
    I = (0.4 if D == 3 else 0.5) * m * r * r
    np.testing.assert_allclose(p["omega"][0], om - dL / I, rtol=1e-13, atol=1e-18)
    assert np.linalg.norm(p["omega"][0]) < np.linalg.norm(om)
    assert np.dot(p["omega"][0], om) > 0


def test_spin_down():
    # Integer centre: the discrete sphere has cubic symmetry, so omega keeps its axis. At
    # density ratio 3 the decay is monotone. At ratio 1.1 the explicit one-step exchange
    # (Eqs. 5-11) first overshoots (the BS shell holds about as much angular momentum as
    # the particle) but the spin never exceeds its initial value and decays overall.
    shape = (24, 24, 24)
    s = _sim(O.D3Q19, shape, tau=0.7)
    s.add_particles([[12.0, 12.0, 12.0]], [5.5], [3.0], omegas=[[0.0, 0.0, 0.01]])
    prev = 0.01
    for _ in range(60):
        s.step(1)
        w = s.get_particles()["omega"][0]
        assert abs(w[0]) < 1e-15 and abs(w[1]) < 1e-15
        assert 0.0 < w[2] < prev
        prev = w[2]
    s = _sim(O.D3Q19, shape, tau=0.7)
    s.add_particles([[12.2, 11.9, 12.4]], [5.5], [1.1], omegas=[[0.004, 0.0, 0.01]])
    n0 = np.linalg.norm([0.004, 0.0, 0.01])
    norms = []
    for _ in range(80):
        s.step(1)
        norms.append(np.linalg.norm(s.get_particles()["omega"][0]))
    assert max(norms) < n0 and norms[-1] < 0.2 * n0
    assert np.all(np.diff(norms[10:]) < 0)


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_momentum_budget_and_mass_with_particles(lattice):
    # Periodic box: the fluid momentum changes by exactly F N (forcing) + dP_B (boundary
    # sites) + dP_IS (internal sites) each step, and the mass is conserved.
    c, w = O.lattice_tables(lattice)
    D = 2 if lattice == O.D2Q9 else 3
    shape = (1, 48, 44) if D == 2 else (20, 22, 24)
    F = np.array([1e-5, 0.0, 0.0])
    s = _sim(lattice, shape, tau=0.75, body_force=F)
    dims = shape[::-1][:D]
    cen, rad = W.rsa_centers(dims, 3, 4.5, seed=5, min_gap=2.0)
    vel = W.gaussian_velocities(3, 0.01, seed=6, dims=D)
    om = np.zeros((3, 3))
    om[:, 2] = [0.003, -0.002, 0.001]
    s.add_particles(cen, rad, [1.3, 0.9, 2.5], velocities=vel, omegas=om)
    N = int(np.prod(shape))
    f = s.get_f()
    m0 = f.sum()
    P = np.einsum("iabc,ik->k", f, c)
    for _ in range(30):
        s.step(1)
        f = s.get_f()
        Pn = np.einsum("iabc,ik->k", f, c)
        dg = s.get_diagnostics()
        resid = Pn - P - (F * N + dg["dP_B"] + dg["dP_IS"])
        # bound: round-off of sums whose terms total sum_x sum_i f_i |c_i|
        scale = np.einsum("iabc,i->", f, np.abs(c).sum(1).astype(float))
        assert np.max(np.abs(resid)) < 1e-13 * scale
        assert abs(f.sum() - m0) / m0 < 1e-13
        P = Pn


def test_mass_conserved_with_walls_and_sedimenting_disks():
    lattice, shape, walls = O.D2Q9, (1, 64, 48), (1, 1, 0)
    s = _sim(lattice, shape, tau=0.7, walls=walls, gravity=(0.0, -2e-4, 0.0))
    cen, rad = W.rsa_centers((48, 64), 4, 5.0, seed=8, min_gap=2.0, walls=(1, 1, 0))
    s.add_particles(cen, rad, np.full(4, 1.5))
    m0 = s.get_f().sum()
    for _ in range(40):
        s.step(1)
    assert abs(s.get_f().sum() - m0) / m0 < 1e-13
    assert np.all(s.get_particles()["u"][:, 1] < 0)   # all settling


def test_particles_moving_with_uniform_flow_change_nothing():
    # Fluid at f^eq(1, U) and particles translating at U (omega = 0): the transfer gives
    # dp = 0 at every BS site, IS sites get the value they already hold, so the state is a
    # fixed point and the particles keep U.
    lattice, shape = O.D3Q19, (20, 20, 20)
    c, _ = O.lattice_tables(lattice)
    U = np.array([0.02, -0.01, 0.015])
    s1 = _sim(lattice, shape, tau=1.0)
    base = np.full(19, 1.0 / 19)
    for k in range(3):
        base[2 * k + 1] += U[k] / 2
        base[2 * k + 2] -= U[k] / 2
    feq = s1.collide_site(base)
    f = np.broadcast_to(feq[:, None, None, None], (19,) + shape).copy()
    s = _sim(lattice, shape, tau=0.8)
    s.set_f(f)
    cen, rad = W.rsa_centers((20, 20, 20), 2, 4.0, seed=12, min_gap=2.0)
    s.add_particles(cen, rad, [1.5, 0.8], velocities=np.tile(U, (2, 1)))
    s.step(8)
    np.testing.assert_allclose(s.get_f(), f, rtol=0, atol=1e-15)
    p = s.get_particles()
    np.testing.assert_allclose(p["u"], np.tile(U, (2, 1)), rtol=0, atol=1e-15)
    # a sum of ~200 site round-offs of order 1e-17 each
    np.testing.assert_allclose(p["force"], 0.0, atol=1e-13)


# ---- hard-core contacts (Sec. 2.3) ---------------------------------------------------

def _contact_sim(centers, radii, dens, walls=(0, 0, 0), shape=(60, 30, 30), gap=0.0):
    s = _sim(O.D3Q19, shape, walls=walls, gap=gap)
    s.add_particles(np.asarray(centers, float), radii, dens)
    return s


def test_head_on_equal_masses_swap_normal_velocities():
    s = _contact_sim([[15, 15, 20], [15, 15, 30.5]], [5.0, 5.0], [1.0, 1.0])
    u = np.array([[0.01, 0.002, 0.4], [-0.003, 0.0, -0.3]])   # predicted gap -0.2
    out = s.resolve_contacts(u)
    # normal = z: the z components swap, the tangential ones stay
    np.testing.assert_allclose(out[0], [0.01, 0.002, -0.3], atol=1e-15)
    np.testing.assert_allclose(out[1], [-0.003, 0.0, 0.4], atol=1e-15)


def test_oblique_unequal_masses_conserve_momentum_and_energy():
    cen = np.array([[15.0, 15.0, 20.0], [18.0, 14.0, 29.0]])
    s = _contact_sim(cen, [5.0, 4.0], [1.0, 3.0])
    u = np.array([[0.05, 0.0, 0.4], [-0.1, 0.02, -0.3]])
    out = s.resolve_contacts(u)
    m = np.array([1.0 * 4 / 3 * math.pi * 125, 3.0 * 4 / 3 * math.pi * 64])
    np.testing.assert_allclose((m[:, None] * out).sum(0), (m[:, None] * u).sum(0), rtol=1e-14)
    e0 = (m * (u * u).sum(1)).sum()
    e1 = (m * (out * out).sum(1)).sum()
    assert abs(e1 - e0) / e0 < 1e-14
    n = (cen[1] - cen[0]) / np.linalg.norm(cen[1] - cen[0])
    # relative normal velocity reverses, tangential parts of each particle unchanged
    assert abs(np.dot(out[1] - out[0], n) + np.dot(u[1] - u[0], n)) < 1e-15
    for k in range(2):
        np.testing.assert_allclose(out[k] - np.dot(out[k], n) * n, u[k] - np.dot(u[k], n) * n,
                                   atol=1e-15)


def test_separating_or_distant_pairs_are_untouched():
    s = _contact_sim([[15, 15, 20], [15, 15, 30.5]], [5.0, 5.0], [1.0, 1.0])
    u = np.array([[0.0, 0.0, -0.3], [0.0, 0.0, 0.2]])    # separating
    np.testing.assert_array_equal(s.resolve_contacts(u), u)
    u = np.array([[0.0, 0.0, 0.1], [0.0, 0.0, -0.1]])    # approaching but no predicted overlap
    s2 = _contact_sim([[15, 15, 10], [15, 15, 40]], [5.0, 5.0], [1.0, 1.0])
    np.testing.assert_array_equal(s2.resolve_contacts(u), u)


def test_fixed_partner_reflects_the_mobile_particle():
    s = _contact_sim([[15, 15, 20], [15, 15, 30.5]], [5.0, 5.0], [1.0, math.inf])
    u = np.array([[0.01, 0.0, 0.7], [0.0, 0.0, 0.0]])
    out = s.resolve_contacts(u)
    np.testing.assert_allclose(out, [[0.01, 0.0, -0.7], [0.0, 0.0, 0.0]], atol=1e-15)


def test_wall_reflects_the_normal_component():
    # walls at z = -1/2 and z = 59.5; predicted distances 4.8 and 4.9 < r = 5
    s = _contact_sim([[15, 15, 5.0]], [5.0], [1.0], walls=(0, 0, 1))
    u = np.array([[0.02, -0.01, -0.7]])
    out = s.resolve_contacts(u)
    np.testing.assert_allclose(out, [[0.02, -0.01, 0.7]], atol=1e-15)
    s2 = _contact_sim([[15, 15, 54.2]], [5.0], [1.0], walls=(0, 0, 1))
    u2 = np.array([[0.0, 0.0, 0.4]])
    np.testing.assert_allclose(s2.resolve_contacts(u2), [[0.0, 0.0, -0.4]], atol=1e-15)


def test_rejects_invalid_particles():
    with pytest.raises(ValueError):   # overlap
        _contact_sim([[15, 15, 20], [15, 15, 28]], [5.0, 5.0], [1.0, 1.0])
    with pytest.raises(ValueError):   # crosses a wall
        _contact_sim([[15, 15, 3.0]], [5.0], [1.0], walls=(0, 0, 1))
    with pytest.raises(ValueError):   # too small
        _contact_sim([[15, 15, 20]], [1.2], [1.0])
    with pytest.raises(ValueError):   # too large for the periodic box
        _contact_sim([[15, 15, 20]], [13.5], [1.0])


def _feq_np(w, c, rho, u):
    """Second-order equilibrium of every direction for velocities u[..., 3] (R1)."""
    cu = np.tensordot(u, c.T.astype(np.float64), axes=([-1], [0]))      # [..., Q]
    usq = (u * u).sum(-1)[..., None]
    return w * rho[..., None] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq)


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_first_step_internal_site_imposition_closed_form(lattice):
    # Fluid at rest (f = w_i), one particle translating fast enough that its first move
    # crosses a shift boundary on two axes (s' = (+1, -1, 0)) and spinning. Everything the
    # step does is then fixed by closed forms, and the whole state after one step is
    # predicted site by site:
    #   - collision leaves f* = w_i everywhere (rest state, no force);
    #   - old BS sites y (shift 0) take f^eq(rho_B, U + omega x (y - x0)) (Eqs. 5-7);
    #   - u' = U - dP/m, omega' = omega - dL/I (Eqs. 8-11), x' = x0 + u' (Eq. 13);
    #   - IS sites of the *shifted* set take f^eq(rho_I, u' + omega' x (y - c')) with
    #     c' = x0 + s' and rho_I the site's own post-collision density (Eq. 12, R3-R5);
    #     every other site keeps its post-collision value;
    #   - propagation moves f*_i(y) to y + c_i.
    # A mistake in the imposition (the velocities before the acceleration, the site set
    # before the move, the lever arm on the wrong side of the cross product) changes the
    # predicted populations by O(1e-2) at hundreds of sites.
    c, w = O.lattice_tables(lattice)
    D = 2 if lattice == O.D2Q9 else 3
    shape = (1, 36, 40) if D == 2 else (22, 24, 26)
    nz, ny, nx = shape
    x0 = np.array([19.37, 17.71, 10.58 if D == 3 else 0.0])
    r, rho_p = 4.6, 3.0
    U = np.array([0.78, -0.8, 0.05 if D == 3 else 0.0])
    om = np.array([0.0, 0.0, 0.03]) if D == 2 else np.array([0.012, -0.02, 0.017])
    s = _sim(lattice, shape, tau=0.8)
    s.add_particles(x0[None], [r], [rho_p], velocities=U[None], omegas=om[None])
    s.step(1)

    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    Y = np.stack([xx, yy, zz], axis=-1).astype(np.float64)      # site coordinates [z,y,x,3]
    # post-collision state: the rest weights (summed in the oracle's order for rho)
    fstar = np.broadcast_to(w, shape + (len(w),)).copy()
    old = brute_force_tags(lattice, shape, (0, 0, 0), [(x0, r, np.zeros(3))])
    bs_old = (old >> 30) == 1
    rho_rest = 0.0
    for wi in w:
        rho_rest += wi
    arms = Y[bs_old] - x0
    arms[:, D:] = 0.0
    uB = U + np.cross(om, arms)
    fstar[bs_old] = _feq_np(w, c, np.full(len(arms), rho_rest), uB)
    dP = (rho_rest * uB).sum(0)
    dL = np.cross(arms, rho_rest * uB).sum(0)
    m = rho_p * ((4.0 / 3.0) * math.pi * r ** 3 if D == 3 else math.pi * r ** 2)
    I = (0.4 if D == 3 else 0.5) * m * r * r
    u1 = U - dP / m
    om1 = om - dL / I
    if D == 2:
        om1[:2] = 0.0
        u1[2] = 0.0
    x1 = x0 + u1
    shift = np.floor(x1 - x0 + 0.5)
    shift[D:] = 0
    assert shift.tolist()[:2] == [1.0, -1.0]                    # the move crosses two boundaries

    p = s.get_particles()
    np.testing.assert_allclose(p["u"][0], u1, rtol=0, atol=1e-14)
    np.testing.assert_allclose(p["omega"][0], om1, rtol=0, atol=1e-14)
    np.testing.assert_allclose(p["x"][0], x1, rtol=0, atol=1e-13)
    new = brute_force_tags(lattice, shape, (0, 0, 0), [(x0, r, shift)])
    np.testing.assert_array_equal(s.get_tags(), new)
    is_new = (new >> 30) == 0
    left = ((old >> 30) == 0) & ~is_new
    assert is_new.sum() > 20 and left.sum() > 5 and (bs_old & is_new).sum() > 5

    rho_I = fstar[is_new].sum(-1)
    arms1 = Y[is_new] - (x0 + shift)
    arms1[:, D:] = 0.0
    fstar[is_new] = _feq_np(w, c, rho_I, u1 + np.cross(om1, arms1))
    expect = np.empty((len(w),) + shape)
    for i, ci in enumerate(c):
        expect[i] = np.roll(fstar[..., i], shift=(ci[2], ci[1], ci[0]), axis=(0, 1, 2))
    got = s.get_f()
    np.testing.assert_allclose(got, expect, rtol=0, atol=2e-15)
    # the IS sites the particle left keep their collided (rest) populations, w_i up to the
    # collision's round-off
    for i, ci in enumerate(c):
        moved = np.roll(left, shift=(ci[2], ci[1], ci[0]), axis=(0, 1, 2))
        np.testing.assert_allclose(got[i][moved], w[i], rtol=0, atol=2e-16)


# ---- orientation (rigid-body rotation integrated with the position) -------------------

def _quat_matrix(q):
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _rodrigues(om):
    """Rotation by |om| about om / |om| (Rodrigues' formula)."""
    th = np.linalg.norm(om)
    if th == 0.0:
        return np.eye(3)
    k = om / th
    K = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(th) * K + (1.0 - math.cos(th)) * (K @ K)


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_orientation_of_a_steadily_turning_particle(lattice):
    # A fixed particle (infinite density: its velocities never change) turning at omega:
    # after n steps its orientation is the rotation by n |omega| about omega, i.e. the
    # quaternion (cos(n th / 2), sin(n th / 2) omega / th), and stays of unit norm.
    D = 2 if lattice == O.D2Q9 else 3
    shape = (1, 32, 32) if D == 2 else (20, 20, 20)
    om = np.array([0.0, 0.0, 0.0371]) if D == 2 else np.array([0.021, -0.013, 0.0298])
    s = _sim(lattice, shape)
    s.add_particles([[10.3, 11.6, 9.2 if D == 3 else 0.0]], [4.2], [math.inf], omegas=om[None])
    np.testing.assert_array_equal(s.get_orientations(), [[1.0, 0.0, 0.0, 0.0]])
    th = np.linalg.norm(om)
    done = 0
    for n in (1, 7, 60):
        s.step(n - done)
        done = n
        q = s.get_orientations()[0]
        expect = np.concatenate([[math.cos(0.5 * n * th)], math.sin(0.5 * n * th) * om / th])
        np.testing.assert_allclose(q, expect, rtol=0, atol=2e-15 * n)
        assert abs(np.dot(q, q) - 1.0) < 1e-15


def test_orientation_turns_in_the_space_frame_each_step():
    # A light particle that moves and spins in still fluid: the fluid torque turns its
    # angular velocity away from its initial axis. Each step the orientation must advance by
    # the rotation through |omega'| about omega', the angular velocity after that step's
    # acceleration (Eq. 11), applied in the space frame: R(q_n+1) = Rot(omega') R(q_n).
    shape = (24, 24, 24)
    s = _sim(O.D3Q19, shape, tau=0.7)
    s.add_particles([[11.3, 12.6, 11.8]], [5.2], [0.6], velocities=[[0.02, -0.01, 0.015]],
                    omegas=[[0.01, 0.04, -0.02]])
    R = _quat_matrix(s.get_orientations()[0])
    om_first = None
    for n in range(40):
        s.step(1)
        om = s.get_particles()["omega"][0]
        om_first = om if om_first is None else om_first
        Rn = _quat_matrix(s.get_orientations()[0])
        np.testing.assert_allclose(Rn @ R.T, _rodrigues(om), rtol=0, atol=1e-14)
        R = Rn
    # the axis did turn, so the order of the rotations matters in this test
    cosang = np.dot(om, om_first) / (np.linalg.norm(om) * np.linalg.norm(om_first))
    assert cosang < 0.99

