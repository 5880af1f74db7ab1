"""Pins of the oracle's fluid core (Sec. 2.1, Eqs. 1-4) to closed forms and invariants.

None of these compare the oracle with itself: each checks a property the mathematics or
the paper fixes (exact Poiseuille flow, exact moment identities of the equilibrium and of
the forcing, exact conservation, the viscosity the paper prints for tau = 0.6).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1105_2904_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def _channel(lattice, tau, F, ny, steps):
    """Force-driven channel: walls on y, periodic x (and z); returns u_x(y)."""
    nz = 1
    s = O.OracleSim(lattice, 1, ny, nz, tau, body_force=(F, 0.0, 0.0), walls=(0, 1, 0))
    s.step(steps)
    rho, u = s.get_fields()
    return rho[0, :, 0], u[0, :, 0, 0]


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_poiseuille_curvature_is_exact(lattice, tau):
    # Steady force-driven channel flow: u'' = -F/(rho nu) with nu = c_s^2 (tau - 1/2) (Eq. 4).
    F, ny = 1e-6, 16
    rho, ux = _channel(lattice, tau, F, ny, 40000)
    nu = (tau - 0.5) / 3.0
    d2 = ux[2:] - 2.0 * ux[1:-1] + ux[:-2]
    # mass drifts only by round-off over 4e4 steps, and uniformly
    assert np.max(np.abs(rho - 1.0)) < 1e-10 and np.ptp(rho) < 1e-13
    assert np.max(np.abs(d2 + F / nu)) / (F / nu) < 1e-9


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_poiseuille_profile_exact_at_zero_slip_tau(lattice):
    # With halfway bounce-back the parabola is exact, walls at -1/2 and ny-1/2, when
    # (tau-1/2)^2 = 3/16 (tau = 1/2 + sqrt(3)/4).
    tau = 0.5 + math.sqrt(3.0) / 4.0
    F, ny = 1e-6, 16
    _, ux = _channel(lattice, tau, F, ny, 40000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny)
    exact = F / (2.0 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.max(np.abs(ux - exact)) / exact.max() < 1e-9


def test_poiseuille_off_magic_tau_has_slip():
    # Sensitivity check: away from tau*, the wall slip is visible (so the exact-profile
    # test above does discriminate).
    F, ny, tau = 1e-6, 16, 0.8
    _, ux = _channel(O.D2Q9, tau, F, ny, 40000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny)
    exact = F / (2.0 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.max(np.abs(ux - exact)) / exact.max() > 1e-4


def test_golden_viscosity_of_tau_0_6():
    # Sec. 3.2 prints: tau = 0.6 gives nu = 1/30 in lattice units.
    g = json.load(open(GOLDEN))["tau_to_nu"]
    F, ny = 1e-6, 16
    _, ux = _channel(O.D2Q9, g["tau"], F, ny, 40000)
    curv = np.mean(ux[2:] - 2.0 * ux[1:-1] + ux[:-2])
    nu_measured = -F / curv
    assert abs(nu_measured - g["nu"]) / g["nu"] < 1e-9


def test_golden_504_disk_case_reads_as_a_2_cm_box():
    # Sec. 3.4 prints 512 x 512 sites, tau = 0.9915, a 0.00025 s time step and nu = 1e-6 m^2/s.
    # Through nu_phys = nu_lattice dx^2 / dt with the oracle's measured lattice viscosity at that
    # tau they fix dx = 39.06 um: the 512 sites span 2 cm, not the printed 1e-2 m (reading R17).
    # The printed diameter 0.625 cm would then be 160 sites and 504 such disks would cover the
    # box 38 times over; 0.0625 cm = 16 sites covers 39 % of it.
    g = json.load(open(GOLDEN))["sedimentation_504"]
    F, ny = 1e-6, 16
    _, ux = _channel(O.D2Q9, g["tau"], F, ny, 40000)
    nu_l = -F / np.mean(ux[2:] - 2.0 * ux[1:-1] + ux[:-2])
    dx = math.sqrt(g["nu_m2_s"] * g["dt_s"] / nu_l)
    assert abs(g["sites"] * dx - 0.02) / 0.02 < 2e-3
    assert abs(g["sites"] * dx - g["box_printed_m"]) / g["box_printed_m"] > 0.9
    area = g["sites"] ** 2

    def cover(d_sites):
        return g["n"] * math.pi * (0.5 * d_sites) ** 2 / area

    d_printed = g["diameter_printed_cm"] * 1e-2 / dx
    d_read = 0.1 * g["diameter_printed_cm"] * 1e-2 / dx
    assert abs(d_printed - 160.0) < 0.5 and cover(d_printed) > 30.0
    assert abs(d_read - 16.0) < 0.05 and 0.35 < cover(d_read) < math.pi / (2.0 * math.sqrt(3.0))


def test_golden_table1_gives_one_grid_spacing():
    # Table 1: with the oracle's measured lattice viscosity at each tau, the four
    # (rho_f, mu_f, tau, dt) rows all map to the same grid spacing, 1 mm (D = 15 mm is
    # then 15 lattice units), through nu_phys = nu_lattice dx^2 / dt.
    t = json.load(open(GOLDEN))["table1"]
    F, ny = 1e-6, 16
    nu_l = {}
    for tau in sorted({r["tau"] for r in t["rows"]}):
        _, ux = _channel(O.D2Q9, tau, F, ny, 40000)
        nu_l[tau] = -F / np.mean(ux[2:] - 2.0 * ux[1:-1] + ux[:-2])
    dxs = []
    for r in t["rows"]:
        nu_phys = r["mu_f_1e3"] * 1e-3 / r["rho_f"]
        dt = r["dt_1e3"] * 1e-3
        dxs.append(math.sqrt(nu_phys * dt / nu_l[r["tau"]]) * 1e3)
    assert max(abs(d - 1.0) for d in dxs) < 2e-3, dxs


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_equilibrium_moments(lattice):
    # tau = 1, F = 0: the collision returns f^eq(rho, u) of the input. The second-order
    # equilibrium has rho, rho u and rho (c_s^2 I + u u) as its first three moments.
    c, _ = O.lattice_tables(lattice)
    Q = len(c)
    s = O.OracleSim(lattice, 4, 4, 1 if lattice == O.D2Q9 else 4, 1.0)
    g = W.rng(7)
    for _ in range(20):
        fin = g.uniform(0.01, 0.2, size=Q)
        feq = s.collide_site(fin)
        rho = fin.sum()
        u = (fin[:, None] * c).sum(0) / rho
        assert abs(feq.sum() - rho) < 1e-14
        assert np.max(np.abs((feq[:, None] * c).sum(0) - rho * u)) < 1e-14
        Pi = np.einsum("i,ia,ib->ab", feq, c, c)
        D = 2 if lattice == O.D2Q9 else 3
        expect = rho * (np.eye(3) / 3.0 + np.outer(u, u))
        expect[D:, :] = 0.0
        expect[:, D:] = 0.0
        assert np.max(np.abs(Pi - expect)) < 1e-14


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_bgk_relaxes_stress_by_one_over_tau(lattice):
    # Eq. 3: the non-equilibrium part of every moment is scaled by (1 - 1/tau).
    c, _ = O.lattice_tables(lattice)
    Q = len(c)
    tau = 0.63
    s1 = O.OracleSim(lattice, 4, 4, 1 if lattice == O.D2Q9 else 4, 1.0)
    st = O.OracleSim(lattice, 4, 4, 1 if lattice == O.D2Q9 else 4, tau)
    g = W.rng(8)
    fin = g.uniform(0.01, 0.2, size=Q)
    feq = s1.collide_site(fin)
    fout = st.collide_site(fin)
    Pin = np.einsum("i,ia,ib->ab", fin, c, c)
    Peq = np.einsum("i,ia,ib->ab", feq, c, c)
    Pout = np.einsum("i,ia,ib->ab", fout, c, c)
    assert np.max(np.abs(Pout - (Peq + (1.0 - 1.0 / tau) * (Pin - Peq)))) < 1e-14


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
def test_guo_forcing_adds_exactly_F(lattice):
    # The forced collision keeps the mass and adds exactly F to the site momentum.
    c, _ = O.lattice_tables(lattice)
    Q = len(c)
    F = np.array([3e-4, -2e-4, 1e-4 if lattice == O.D3Q19 else 0.0])
    s = O.OracleSim(lattice, 4, 4, 1 if lattice == O.D2Q9 else 4, 0.7, body_force=F)
    g = W.rng(9)
    for _ in range(10):
        fin = g.uniform(0.01, 0.2, size=Q)
        fout = s.collide_site(fin)
        assert abs(fout.sum() - fin.sum()) < 1e-15
        dj = (fout[:, None] * c).sum(0) - (fin[:, None] * c).sum(0)
        assert np.max(np.abs(dj - F)) < 1e-15


@pytest.mark.parametrize("lattice,shape", [(O.D2Q9, (1, 24, 20)), (O.D3Q19, (10, 12, 8))])
def test_periodic_conservation(lattice, shape):
    # Periodic box without particles: mass is constant and the total momentum grows by
    # exactly F per site and step (streaming and collision conserve; the forcing adds F).
    c, w = O.lattice_tables(lattice)
    nz, ny, nx = shape
    F = np.array([2e-5, 1e-5, -1e-5 if lattice == O.D3Q19 else 0.0])
    s = O.OracleSim(lattice, nx, ny, nz, 0.7, body_force=F)
    xi = W.perturbation(len(c), shape, seed=11)
    f0 = w[:, None, None, None] * (1.0 + 0.05 * xi)
    s.set_f(f0)
    N = nx * ny * nz
    m0 = s.get_f().sum()
    P = np.einsum("iabc,ik->k", s.get_f(), c)
    for _ in range(25):
        s.step(1)
        f = s.get_f()
        Pn = np.einsum("iabc,ik->k", f, c)
        assert abs(f.sum() - m0) / m0 < 1e-13
        assert np.max(np.abs(Pn - P - F * N)) < 1e-10 * np.abs(F * N).max()
        P = Pn


@pytest.mark.parametrize("lattice,shape", [(O.D2Q9, (1, 16, 16)), (O.D3Q19, (8, 8, 8))])
def test_uniform_flow_is_a_fixed_point(lattice, shape):
    # A uniform equilibrium state at velocity U is invariant (no force, periodic).
    c, _ = O.lattice_tables(lattice)
    Q = len(c)
    nz, ny, nx = shape
    U = np.array([0.03, -0.02, 0.01 if lattice == O.D3Q19 else 0.0])
    s1 = O.OracleSim(lattice, nx, ny, nz, 1.0)
    # build f^eq(1, U) as the tau = 1 collision of any state with rho = 1, momentum U
    c_f = c.astype(np.float64)
    base = np.full(Q, 1.0 / Q)
    # adjust the momentum with the axis populations, keeping the mass at 1
    for k in range(3 if lattice == O.D3Q19 else 2):
        ip = [i for i in range(Q) if c[i, k] == 1 and (c[i] != 0).sum() == 1][0]
        im = [i for i in range(Q) if c[i, k] == -1 and (c[i] != 0).sum() == 1][0]
        base[ip] += U[k] / 2.0
        base[im] -= U[k] / 2.0
    assert np.allclose((base[:, None] * c_f).sum(0), U)
    feq = s1.collide_site(base)
    f = np.broadcast_to(feq[:, None, None, None], (Q,) + shape).copy()
    s = O.OracleSim(lattice, nx, ny, nz, 0.8)
    s.set_f(f)
    s.step(10)
    assert np.max(np.abs(s.get_f() - f)) < 1e-15


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q19])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.3])
def test_couette_profile_is_exact(lattice, tau):
    # Walls at y = -1/2 and ny - 1/2 moving at -U and +U (velocity-imposed boundaries of
    # Secs. 3.1-3.2): the steady profile is exactly linear at any tau.
    ny, U = 16, 0.02
    s = O.OracleSim(lattice, 1, ny, 1, tau, walls=(0, 1, 0), wall_velocity={2: (-U, 0, 0), 3: (U, 0, 0)})
    s.step(20000)
    rho, u = s.get_fields()
    y = np.arange(ny)
    exact = -U + 2.0 * U * (y + 0.5) / ny
    assert np.max(np.abs(u[0, :, 0, 0] - exact)) / U < 1e-10
    assert np.max(np.abs(u[0, :, 0, 1:])) < 1e-13
    assert np.max(np.abs(rho - 1.0)) < 1e-10


def test_wall_velocity_must_be_tangential_and_on_a_wall():
    with pytest.raises(ValueError):
        O.OracleSim(O.D2Q9, 8, 8, 1, 0.8, walls=(0, 1, 0), wall_velocity={3: (0.0, 0.01, 0.0)})
    with pytest.raises(ValueError):
        O.OracleSim(O.D2Q9, 8, 8, 1, 0.8, walls=(0, 1, 0), wall_velocity={0: (0.0, 0.01, 0.0)})


# ---- Equilibrium faces (reading R16) ------------------------------------------------------
# A face that imposes a velocity the way the method imposes one at a particle's sites: after
# the collision its fluid sites take f^eq(rho, u_face); moves out through it bounce back.


@pytest.mark.parametrize("lattice,dims", [(O.D2Q9, (6, 20, 1)), (O.D3Q19, (6, 14, 5))])
def test_equilibrium_faces_keep_a_uniform_tangential_flow(lattice, dims):
    # f^eq(1, U) with U along the faces: interior sites stay exactly at f^eq(1, U); the face
    # sites' pre-collision state holds bounced values but is steady.
    U = 0.02
    c, w = O.lattice_tables(lattice)
    nx, ny, nz = dims
    s = O.OracleSim(lattice, *dims, 0.8, walls=(0, 1, 0), equilibrium_faces={2: (U, 0, 0), 3: (U, 0, 0)})
    cu = c[:, 0] * U
    feq = w * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * U * U)
    f0 = np.broadcast_to(feq[:, None, None, None], (len(w), nz, ny, nx)).copy()
    s.set_f(f0)
    s.step(30)
    f30 = s.get_f()
    s.step(30)
    f60 = s.get_f()
    assert np.max(np.abs(f60 - f30)) <= 1e-15                               # a few ulps
    assert np.max(np.abs(f60[:, :, 1:-1, :] - f0[:, :, 1:-1, :])) <= 1e-15


@pytest.mark.parametrize("lattice,tau", [(O.D2Q9, 0.6), (O.D2Q9, 0.8), (O.D2Q9, 1.3), (O.D3Q19, 0.9)])
def test_equilibrium_face_couette_profile_closed_form(lattice, tau):
    # Faces y = 0 and y = ny - 1 at -U and +U. In the steady state the interior profile is
    # exactly linear. The momentum the first interior site receives from a face site (a pure
    # equilibrium at -U) equals what a bulk site would send, f^eq(u(0)) minus its post-collision
    # non-equilibrium part 3 w c_x c_y (tau - 1) du/dy, when u(0) = -U + (tau - 1) du/dy; with
    # antisymmetry the slope is du/dy = 2U / (ny - 3 + 2 tau) and u(y) = du/dy (y - (ny-1)/2).
    ny, U = 24, 0.01
    dims = (4, ny, 1) if lattice == O.D2Q9 else (4, ny, 4)
    s = O.OracleSim(lattice, *dims, tau, walls=(0, 1, 0), equilibrium_faces={2: (-U, 0, 0), 3: (U, 0, 0)})
    for _ in range(80):
        s.step(1000)
    rho, u = s.get_fields()
    ux = u[0, :, 0, 0]
    slope = 2.0 * U / (ny - 3 + 2.0 * tau)
    y = np.arange(1, ny - 1)
    want = slope * (y - 0.5 * (ny - 1))
    assert np.max(np.abs(ux[1:-1] - want)) <= 1e-10 * U


def test_openmp_build_gives_identical_results():
    # The OpenMP build of the oracle only splits the per-site loops between threads: a moving,
    # colliding suspension between walls (one moving) evolves bit for bit as in the
    # single-threaded build.
    os.environ.setdefault("OMP_NUM_THREADS", "4")
    dims = (26, 22, 18)
    cen, rad = W.rsa_centers(dims, 4, 4.0, seed=31, min_gap=1.0, walls=(0, 0, 1))
    vel = W.gaussian_velocities(4, 0.03, seed=32)
    om = W.gaussian_velocities(4, 0.004, seed=33)
    sims = []
    for omp in (False, True):
        s = O.OracleSim(O.D3Q19, *dims, 0.7, body_force=(2e-6, 0.0, 0.0), walls=(0, 0, 1), gap=0.5,
                        wall_velocity={5: (0.01, 0.0, 0.0)}, openmp=omp)
        s.add_particles(cen, rad, [1.3, 2.0, 0.9, 1.6], velocities=vel, omegas=om)
        s.step(25)
        sims.append(s)
    a, b = sims
    np.testing.assert_array_equal(a.get_f(), b.get_f())
    np.testing.assert_array_equal(a.get_tags(), b.get_tags())
    pa, pb = a.get_particles(), b.get_particles()
    for k in pa:
        np.testing.assert_array_equal(pa[k], pb[k])
