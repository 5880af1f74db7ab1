"""CUDA path vs the FP64 oracle, element by element, on identical seeded inputs.

FP64 storage: the CUDA path evaluates the same IEEE operations in the same order as the
oracle (fixed-order reductions, no FMA contraction), so results must agree to 1e-12
relative (in practice exactly). FP32 storage: velocity within 1e-5 of max|u|, particle
forces within 1e-4 of max|F|. Masks (owner maps) are compared bit for bit.
Sizes span several 128-site tiles with a ragged tail."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()
    O.build()


def make_pair(lattice, dims, tau, precision, F=(0.0, 0.0, 0.0), walls=(0, 0, 0), gravity=(0, 0, 0),
              gap=0.0, bfp=False, particles=None, f0=None):
    nx, ny, nz = dims
    g = lbmp.Simulation(lattice, nx, ny, nz, tau, body_force=F, precision=precision, walls=walls,
                        gravity=gravity, gap=gap, body_force_on_particles=bfp)
    r = O.OracleSim(lattice, nx, ny, nz, tau, body_force=F, walls=walls, gravity=gravity, gap=gap,
                    body_force_on_particles=bfp)
    if f0 is not None:
        g.set_f(f0)
        r.set_f(f0)
    if particles is not None:
        c, rad, d, v, om = particles
        g.add_particles(c, rad, d, v, om)
        r.add_particles(c, rad, d, v, om)
    return g, r


def perturbed(lattice, dims, seed, amp=0.02):
    c, w = O.lattice_tables(lattice)
    nx, ny, nz = dims
    xi = W.perturbation(len(w), (nz, ny, nx), seed)
    return w[:, None, None, None] * (1.0 + amp * xi)


def rel(a, b, scale=None):
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


FLUID_CASES = [
    ("d2q9_periodic_ragged", O.D2Q9, (150, 40, 1), (0, 0, 0), (3e-6, -1e-6, 0.0)),
    ("d2q9_box_walls", O.D2Q9, (133, 37, 1), (1, 1, 0), (2e-6, 0.0, 0.0)),
    ("d3q19_periodic_ragged", O.D3Q19, (150, 12, 10), (0, 0, 0), (1e-6, 2e-6, -1e-6)),
    ("d3q19_channel_walls_yz", O.D3Q19, (70, 11, 9), (0, 1, 1), (2e-6, 0.0, 0.0)),
]


@pytest.mark.parametrize("name,lattice,dims,walls,F", FLUID_CASES, ids=[c[0] for c in FLUID_CASES])
def test_fluid_fp64_matches_oracle_exactly(name, lattice, dims, walls, F):
    f0 = perturbed(lattice, dims, seed=31)
    g, r = make_pair(lattice, dims, 0.73, "fp64", F=F, walls=walls, f0=f0)
    g.step(60)
    r.step(60)
    fg, fr = g.get_f(), r.get_f()
    assert rel(fg, fr) <= 1e-12
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-12 and rel(rg, rr) <= 1e-12


@pytest.mark.parametrize("name,lattice,dims,walls,F", FLUID_CASES, ids=[c[0] for c in FLUID_CASES])
def test_fluid_fp32_within_tolerance(name, lattice, dims, walls, F):
    f0 = perturbed(lattice, dims, seed=32)
    g, r = make_pair(lattice, dims, 0.73, "fp32", F=F, walls=walls, f0=f0)
    g.step(60)
    r.step(60)
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-5
    assert rel(rg, rr, np.max(np.abs(rr - 1.0))) <= 1e-5


def particle_cases():
    cases = []
    # Config-1 shape: fixed disk r = 8 in a 128x64 periodic channel (shortened run).
    cases.append(dict(name="d2q9_fixed_disk_channel", lattice=O.D2Q9, dims=(128, 64, 1), tau=0.8,
                      F=(1e-6, 0, 0), walls=(0, 0, 0), gravity=(0, 0, 0), gap=0.0, bfp=False, steps=300,
                      particles=(np.array([[64.0, 32.0, 0.0]]), [8.0], [math.inf], None, None)))
    # Moving, spinning spheres crossing shift boundaries in a periodic box with a body force.
    dims = (41, 36, 30)
    c, rad = W.rsa_centers(dims, 4, 5.0, seed=41, min_gap=2.0)
    v = W.gaussian_velocities(4, 0.03, seed=42)
    om = W.gaussian_velocities(4, 0.004, seed=43)
    cases.append(dict(name="d3q19_moving_spheres", lattice=O.D3Q19, dims=dims, tau=0.7, F=(2e-6, 0, 0),
                      walls=(0, 0, 0), gravity=(0, 0, 0), gap=0.0, bfp=True, steps=150,
                      particles=(c, rad, np.array([1.2, 2.5, 0.9, 1.5]), v, om)))
    # Settling disks in a closed box: wall and particle contacts.
    dims2 = (60, 90, 1)
    c2, r2 = W.rsa_centers((60, 90), 6, 5.0, seed=44, min_gap=1.0, walls=(1, 1, 0))
    cases.append(dict(name="d2q9_settling_box", lattice=O.D2Q9, dims=dims2, tau=0.7, F=(0, 0, 0),
                      walls=(1, 1, 0), gravity=(0.0, -2e-3, 0.0), gap=0.5, bfp=False, steps=300,
                      particles=(c2, r2, np.full(6, 2.0), None, None)))
    # Head-on collision of two spheres in a channel with walls on z.
    cases.append(dict(name="d3q19_head_on_walls", lattice=O.D3Q19, dims=(48, 20, 22), tau=0.8,
                      F=(0, 0, 0), walls=(0, 0, 1), gravity=(0, 0, 0), gap=0.5, bfp=False, steps=120,
                      particles=(np.array([[16.3, 10.1, 10.6], [29.7, 9.8, 10.4]]), [5.0, 5.5], [10.0, 15.0],
                                 np.array([[0.08, 0.0, 0.0], [-0.07, 0.0, 0.0]]), None)))
    return cases


PCASES = particle_cases()


def _run_case(case, precision):
    g, r = make_pair(case["lattice"], case["dims"], case["tau"], precision, F=case["F"], walls=case["walls"],
                     gravity=case["gravity"], gap=case["gap"], bfp=case["bfp"], particles=case["particles"])
    for _ in range(case["steps"] // 10):
        g.step(10)
        r.step(10)
    return g, r


@pytest.mark.parametrize("case", PCASES, ids=[c["name"] for c in PCASES])
def test_suspension_fp64_matches_oracle_exactly(case):
    g, r = _run_case(case, "fp64")
    np.testing.assert_array_equal(g.get_tags(), r.get_tags())
    pg, pr = g.get_particles(), r.get_particles()
    for k in ("x", "u", "omega", "force", "torque"):
        assert rel(pg[k], pr[k], max(np.max(np.abs(pr[k])), 1e-300)) <= 1e-12, k
    assert rel(g.get_f(), r.get_f()) <= 1e-12
    # orientations: FP64 quaternion integration on both sides (cos / sin of the two math
    # libraries may differ in the last place)
    qg, qr = g.get_orientations(), r.get_orientations()
    assert np.max(np.abs(qg - qr)) <= 1e-13
    np.testing.assert_allclose((qg * qg).sum(1), 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("case", PCASES, ids=[c["name"] for c in PCASES])
def test_suspension_fp32_within_tolerance(case):
    g, r = _run_case(case, "fp32")
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-5
    pg, pr = g.get_particles(), r.get_particles()
    assert rel(pg["force"], pr["force"]) <= 1e-4
    # torque relative to its natural scale |F| r (the exact torque can vanish by symmetry)
    rad = np.asarray(case["particles"][1], dtype=float)
    tscale = max(np.max(np.abs(pr["torque"])), np.max(np.abs(pr["force"])) * rad.max())
    assert rel(pg["torque"], pr["torque"], tscale) <= 1e-4
    # trajectories: relative to the particle radius; orientations: the angle between them
    assert np.max(np.abs(pg["x"] - pr["x"]) / rad[:, None]) <= 1e-5
    # (the angle between the two attitudes, against the angle |omega| sweeps over the run)
    qg, qr = g.get_orientations(), r.get_orientations()
    angle = 2.0 * np.arccos(np.clip(np.abs((qg * qr).sum(1)), 0.0, 1.0))
    sweep = case["steps"] * np.max(np.linalg.norm(pr["omega"], axis=1))
    assert np.max(angle) <= 1e-4 * sweep + 1e-7


def test_contacts_happen_in_the_collision_cases():
    # The collision cases must actually exercise the contact step.
    case = [c for c in PCASES if c["name"] == "d3q19_head_on_walls"][0]
    g, r = _run_case(case, "fp64")
    pr = r.get_particles()
    assert pr["u"][0, 0] < 0.0 < pr["u"][1, 0]   # the spheres bounced apart
