"""Full-size workloads in the benchmark's launch configuration, checked on sampled particles.

The 512^3 D3Q19 suspension (16000 spheres, FP32 storage) and the 1024x2048 D2Q9 settling box
(500 disks, walls, gravity) are too large for the oracle to run whole. After one step from
rest, though, each particle's force, torque, velocity, position and site ownership depend only
on the particle and its near neighbours (the fluid is at rest, so a boundary site pulls rest
populations; at the seeded gaps no contact is predicted). For a seeded sample of particles the
oracle recomputes that step in a walled sub-box holding the particle and every particle whose
sites can meet its sites, built from the seeded inputs alone; the CUDA path runs the whole box.
The 512^3 suspension is checked in both streaming schemes; over 20 steps, the in-place scheme
must also give every particle the forces, velocities and positions of the pull scheme.
"""
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


def _sub_box_oracle(wl, c, r, d, v, p, D):
    """Oracle run of one step for particle p and its neighbours in a walled box."""
    dims = np.array(wl.dims[:D], dtype=float)
    per = np.array([not wl.walls[k] for k in range(D)])
    dx = c[:, :D] - c[p, :D]
    dx = np.where(per, dx - dims * np.floor(dx / dims + 0.5), dx)
    dist = np.sqrt((dx * dx).sum(1))
    near = np.nonzero(dist < r[p] + r + 4.0)[0]
    near = np.concatenate([[p], near[near != p]])
    pos = c[p, :D] + dx[near]                       # unwrapped around p
    lo = np.floor((pos - r[near, None]).min(0)) - 3
    hi = np.ceil((pos + r[near, None]).max(0)) + 3
    size = (hi - lo + 1).astype(int)
    shift = lo                                       # integer: fractional parts are kept
    local = np.zeros((len(near), 3))
    local[:, :D] = pos - shift
    nx, ny = int(size[0]), int(size[1])
    nz = int(size[2]) if D == 3 else 1
    walls = (1, 1, 1 if D == 3 else 0)
    sim = O.OracleSim(O.D3Q19 if D == 3 else O.D2Q9, nx, ny, nz, wl.tau, body_force=wl.body_force, walls=walls,
                      gravity=wl.gravity, gap=0.0, body_force_on_particles=wl.body_force_on_particles)
    sim.add_particles(local, r[near], d[near], v[near])
    tags0 = sim.get_tags()
    sim.step(1)
    out = sim.get_particles()
    return near, shift, tags0, sim.get_tags(), out


def _compare_tags(sub_tags, near, shift, centre, radius, gpu_tags, wl, D):
    """Owner map of the sub-box (local ids mapped to global ids) against the full map, on every
    site within radius + 1.5 of the sampled particle's centre: only particles of the sub-box
    can claim those sites."""
    nz, ny, nx = sub_tags.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    loc = [xx, yy, zz]
    d2 = sum((loc[k] - centre[k]) ** 2 for k in range(D))
    sel = d2 <= (radius + 1.5) ** 2
    t = sub_tags[sel]
    fluid = t == np.uint32(0xFFFFFFFF)
    mapped = (t & np.uint32(0xC0000000)) | near[(t & np.uint32(0x3FFFFFFF)).astype(np.int64) % len(near)].astype(np.uint32)
    mapped = np.where(fluid, t, mapped)
    gl = [loc[k][sel] + int(shift[k]) for k in range(D)]
    for k in range(D):
        gl[k] = np.mod(gl[k], wl.dims[k])
    zi = gl[2] if D == 3 else np.zeros_like(gl[0])
    np.testing.assert_array_equal(gpu_tags[zi, gl[1], gl[0]], mapped)


@pytest.mark.parametrize("name,streaming", [("d3q19_512", "pull"), ("d3q19_512", "inplace"),
                                            ("d2q9_sedimentation", "pull")])
def test_full_size_first_step_on_sampled_particles(name, streaming):
    wl = W.suspension_3d() if name == "d3q19_512" else W.sedimentation_2d()
    D = 3 if wl.lattice == "D3Q19" else 2
    c, r, d, v = wl.particles()
    if not np.any(v):
        # the settling box starts at rest; seeded velocities make the first-step exchange non-zero
        v = W.gaussian_velocities(len(r), 1e-3, seed=wl.seed + 7, dims=D)
    nx, ny, nz = wl.dims
    sim = lbmp.Simulation(1 if D == 3 else 0, nx, ny, nz, wl.tau, body_force=wl.body_force, precision="fp32",
                          walls=wl.walls, gravity=wl.gravity, gap=0.0,
                          body_force_on_particles=wl.body_force_on_particles, streaming=streaming)
    sim.add_particles(c, r, d, v)
    tags_before = sim.get_tags()
    sim.step(1)
    got = sim.get_particles()
    tags_after = sim.get_tags()
    sim.close()
    sample = W.rng(1234).choice(len(r), size=12, replace=False)
    for p in sample:
        near, shift, t0, t1, ref = _sub_box_oracle(wl, c, r, d, v, p, D)
        centre0 = c[p, :D] - shift
        _compare_tags(t0, near, shift, centre0, r[p], tags_before, wl, D)
        _compare_tags(t1, near, shift, ref["x"][0, :D], r[p], tags_after, wl, D)
        F, T = ref["force"][0], ref["torque"][0]
        fs = max(np.max(np.abs(F)), 1e-300)
        assert np.max(np.abs(got["force"][p] - F)) <= 1e-4 * fs, p
        assert np.max(np.abs(got["torque"][p] - T)) <= 1e-4 * max(np.max(np.abs(T)), fs * r[p]), p
        assert np.max(np.abs(got["u"][p] - ref["u"][0])) <= 1e-4 * max(np.max(np.abs(ref["u"][0])), 1e-12), p
        x_ref = ref["x"][0, :D] + shift
        dxp = got["x"][p, :D] - x_ref
        assert np.max(np.abs(dxp)) <= 1e-5 * r[p], p


def test_full_size_inplace_streaming_matches_pull():
    wl = W.suspension_3d()
    c, r, d, v = wl.particles()
    nx, ny, nz = wl.dims
    out = {}
    for streaming in ("pull", "inplace"):
        sim = lbmp.Simulation(1, nx, ny, nz, wl.tau, body_force=wl.body_force, precision="fp32", walls=wl.walls,
                              gravity=wl.gravity, gap=0.0, body_force_on_particles=wl.body_force_on_particles,
                              streaming=streaming)
        sim.add_particles(c, r, d, v)
        sim.step(20)
        out[streaming] = (sim.get_particles(), sim.get_tags())
        sim.close()
    (pp, tp), (pi, ti) = out["pull"], out["inplace"]
    np.testing.assert_array_equal(ti, tp)
    for k, tol in (("force", 1e-4), ("torque", 1e-4), ("u", 1e-5)):
        scale = max(float(np.max(np.abs(pp[k]))), 1e-300)
        assert float(np.max(np.abs(pi[k] - pp[k]))) <= tol * scale, k
    assert float(np.max(np.abs(pi["x"] - pp["x"]))) <= 1e-6
