"""In-place (two-phase, one buffer) streaming against the pull scheme and the oracle.

The scheme is an implementation choice with no counterpart in the paper (Eq. 4 only moves
f*_i(x) to x + c_i), so its results must be those of the pull scheme: bit for bit in FP64
storage (which also equals the oracle), within storage rounding otherwise. The cases run
an odd and an even number of steps (the two layouts the buffer alternates between) and
cover moving, spinning spheres that cross shift boundaries (sites entering and leaving the
IS set), walls with a moving face, equilibrium faces, the getters and the closure inputs at
both layouts, distributions set between steps, checkpoints taken at both layouts, and the
memory the scheme saves.
"""
import numpy as np
import pytest

import oracle as O
from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DIMS3 = (36, 30, 26)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()
    O.build()


def suspension(streaming, precision, walls=(0, 0, 1), moving=True):
    c, rad = W.rsa_centers(DIMS3, 4, 4.5, seed=71, min_gap=2.0, walls=walls)
    v = W.gaussian_velocities(4, 0.04, seed=72)
    om = W.gaussian_velocities(4, 0.004, seed=73)
    g = lbmp.Simulation(1, *DIMS3, 0.7, body_force=(2e-6, 0.0, 0.0), precision=precision, walls=walls, gap=0.5,
                        body_force_on_particles=True, streaming=streaming)
    if moving and walls[2]:
        g.set_wall_velocity(5, (0.01, 0.0, 0.0))
    g.add_particles(c, rad, np.array([1.3, 2.0, 0.9, 1.6]), v, om)
    return g


def oracle_suspension(walls=(0, 0, 1)):
    c, rad = W.rsa_centers(DIMS3, 4, 4.5, seed=71, min_gap=2.0, walls=walls)
    v = W.gaussian_velocities(4, 0.04, seed=72)
    om = W.gaussian_velocities(4, 0.004, seed=73)
    r = O.OracleSim(1, *DIMS3, 0.7, body_force=(2e-6, 0.0, 0.0), walls=walls, gap=0.5,
                    body_force_on_particles=True, wall_velocity={5: (0.01, 0.0, 0.0)})
    r.add_particles(c, rad, np.array([1.3, 2.0, 0.9, 1.6]), v, om)
    return r


def state(g):
    p = g.get_particles()
    rho, u = g.get_fields()
    return [g.get_f(), rho, u, g.get_tags()] + [p[k].copy() for k in ("x", "u", "omega", "force", "torque")]


def assert_same(a, b):
    for k, (x, y) in enumerate(zip(a, b)):
        np.testing.assert_array_equal(x, y, err_msg="state item %d" % k)


@pytest.mark.parametrize("steps", [1, 2, 45, 70])
def test_fp64_equals_pull_bit_for_bit(steps):
    a = suspension("inplace", "fp64")
    b = suspension("pull", "fp64")
    x0 = a.get_particles()["x"].copy()
    a.step(steps)
    b.step(steps)
    sa, sb = state(a), state(b)
    assert_same(sa, sb)
    if steps == 70:  # the spheres crossed a shift boundary: sites entered and left the IS set
        assert np.max(np.abs(np.floor(sa[4] + 0.5) - np.floor(x0 + 0.5))) >= 1
    a.close()
    b.close()


def test_fp64_matches_oracle():
    a = suspension("inplace", "fp64")
    r = oracle_suspension()
    a.step(45)
    r.step(45)
    assert float(np.max(np.abs(a.get_f() - r.get_f()))) <= 1e-12
    pa, pr = a.get_particles(), r.get_particles()
    for k in ("x", "u", "omega", "force", "torque"):
        assert float(np.max(np.abs(pa[k] - pr[k]))) <= 1e-12, k
    np.testing.assert_array_equal(a.get_tags(), r.get_tags())
    a.close()


@pytest.mark.parametrize("steps", [41, 60])
def test_fp32_matches_pull_and_oracle(steps):
    a = suspension("inplace", "fp32")
    b = suspension("pull", "fp32")
    r = oracle_suspension()
    for s in (a, b, r):
        s.step(steps)
    _, ua = a.get_fields()
    _, ub = b.get_fields()
    _, ur = r.get_fields()
    umax = float(np.max(np.abs(ur)))
    assert float(np.max(np.abs(ua - ur))) / umax <= 1e-5
    assert float(np.max(np.abs(ua - ub))) / umax <= 1e-5
    fa, fr = a.get_particles()["force"], r.get_particles()["force"]
    assert float(np.max(np.abs(fa - fr))) / float(np.max(np.abs(fr))) <= 1e-4
    np.testing.assert_array_equal(a.get_tags(), r.get_tags())
    a.close()
    b.close()


def test_fp16_within_storage_bound():
    a = suspension("inplace", "fp16")
    r = oracle_suspension()
    a.step(41)
    r.step(41)
    _, ua = a.get_fields()
    _, ur = r.get_fields()
    assert float(np.max(np.abs(ua - ur)) / np.max(np.abs(ur))) <= 2e-3
    a.close()


def test_d2q9_equilibrium_faces_and_particles_bit_for_bit():
    dims = (64, 40, 1)

    def make(streaming):
        g = lbmp.Simulation(0, *dims, 0.8, body_force=(0.0, 0.0, 0.0), precision="fp64",
                            equilibrium_faces={2: (0.0, 0.0, 0.0), 3: (0.04, 0.0, 0.0)}, streaming=streaming)
        g.add_particles(np.array([[20.3, 18.6, 0.0], [44.7, 22.2, 0.0]]), np.array([5.0, 4.0]),
                        np.array([1.5, 1.2]), np.array([[0.01, 0.0, 0.0], [-0.01, 0.005, 0.0]]))
        return g

    a, b = make("inplace"), make("pull")
    for n in (1, 30, 29):  # layouts: after a neighbour phase, after a local phase, then again
        a.step(n)
        b.step(n)
        assert_same(state(a), state(b))
    a.close()
    b.close()


def test_closure_inputs_at_both_layouts():
    a = suspension("inplace", "fp64")
    b = suspension("pull", "fp64")
    for n in (7, 8):
        a.step(n)
        b.step(n)
        fa = a.closure_features(4, 2.0, 0.01).cpu().numpy()
        fb = b.closure_features(4, 2.0, 0.01).cpu().numpy()
        np.testing.assert_array_equal(fa, fb)
    a.close()
    b.close()


@pytest.mark.parametrize("first", [13, 14])
def test_set_distributions_between_steps(first):
    a = suspension("inplace", "fp64")
    b = suspension("pull", "fp64")
    a.step(first)
    b.step(first)
    f = b.get_f()
    gen = np.random.Generator(np.random.PCG64(3))
    f = f * (1.0 + 1e-3 * gen.standard_normal(f.shape))
    a.set_f(f)
    b.set_f(f)
    np.testing.assert_array_equal(a.get_f(), f)
    a.step(21)
    b.step(21)
    assert_same(state(a), state(b))
    a.close()
    b.close()


@pytest.mark.parametrize("split", [35, 36])
def test_checkpoint_resume_at_both_layouts(split, tmp_path):
    ref = suspension("inplace", "fp32")
    ref.step(70)
    want = state(ref)
    ref.close()
    a = suspension("inplace", "fp32")
    a.step(split)
    path = tmp_path / "s.ckpt"
    a.save(str(path))
    a.close()
    c = suspension("inplace", "fp32")
    c.load(str(path))
    c.step(70 - split)
    assert_same(state(c), want)
    # a checkpoint of one scheme does not load into a context of the other
    d = suspension("pull", "fp32")
    with pytest.raises(lbmp.LbmError):
        d.load(str(path))
    d.close()
    c.close()


def test_memory_and_restrictions():
    a = suspension("inplace", "fp32", walls=(0, 0, 0), moving=False)
    b = suspension("pull", "fp32", walls=(0, 0, 0), moving=False)
    ia, ib = a.info(), b.info()
    N = DIMS3[0] * DIMS3[1] * DIMS3[2]
    assert ia["bytes_per_site"] == 19 * 4 + 2 * 4 and ib["bytes_per_site"] == 2 * 19 * 4
    # one distribution buffer and the carry's density array fewer, two density arrays more
    assert ib["device_bytes"] - ia["device_bytes"] == 19 * 4 * N + 4 * N - 2 * 4 * N
    # the scheme is chosen before the buffers exist
    with pytest.raises(lbmp.LbmError):
        lbmp.lbm_set_streaming(a.h, lbmp.LBM_STREAM_PULL)
    a.close()
    b.close()
    # a batch refuses a cell switched to in-place streaming
    bt = lbmp.Batch(1, [(16, 16, 16), (16, 16, 16)], [0.7, 0.7])
    lbmp.lbm_set_streaming(lbmp.lbm_batch_cell(bt.h, 0), lbmp.LBM_STREAM_INPLACE)
    with pytest.raises(lbmp.LbmError):
        bt.step(1)
    bt.close()


@pytest.mark.parametrize("lattice,dims", [(0, (61, 47, 1)), (1, (29, 23, 21))], ids=["d2q9_cavity", "d3q19_box"])
def test_walls_on_every_axis_bit_for_bit(lattice, dims):
    """Closed box: walls on every axis (at edges a move crosses two walls), a moving
    lid, a body force and settling particles near the walls."""
    D = 2 if lattice == 0 else 3
    walls = (1, 1, 1 if D == 3 else 0)

    def make(streaming):
        g = lbmp.Simulation(lattice, *dims, 0.75, body_force=(1e-6, 0.0, 0.0), precision="fp64", walls=walls,
                            gravity=(0.0, -2e-5, 0.0), gap=0.5, streaming=streaming,
                            wall_velocity={3: (0.02, 0.0, 0.0)})
        c, rad = W.rsa_centers(dims if D == 3 else dims[:2], 3, 4.0, seed=17, min_gap=1.5, walls=walls)
        v = W.gaussian_velocities(3, 0.01, seed=18, dims=D)
        g.add_particles(c, rad, np.array([1.5, 2.0, 1.2]), v)
        return g

    a, b = make("inplace"), make("pull")
    for n in (1, 24, 25):
        a.step(n)
        b.step(n)
        assert_same(state(a), state(b))
    a.close()
    b.close()
