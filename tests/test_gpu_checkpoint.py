"""Checkpoint and resume: a run split by a checkpoint continues bit for bit.

Moving, spinning spheres that cross shift boundaries (so the IS-site bookkeeping runs on both
sides of the checkpoint), a moving wall, a body force; FP64 and FP32 storage. The resumed
context is a fresh one set up by the same calls. Also: rolling back the same context, and a
checkpoint refused by a context set up differently."""
import numpy as np
import pytest

from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DIMS = (36, 30, 26)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()


def _setup(precision, radius=4.5):
    c, rad = W.rsa_centers(DIMS, 4, radius, seed=71, min_gap=2.0, walls=(0, 0, 1))
    v = W.gaussian_velocities(4, 0.04, seed=72)
    om = W.gaussian_velocities(4, 0.004, seed=73)
    g = lbmp.Simulation(1, *DIMS, 0.7, body_force=(2e-6, 0.0, 0.0), precision=precision, walls=(0, 0, 1),
                        gap=0.5, body_force_on_particles=True)
    g.set_wall_velocity(5, (0.01, 0.0, 0.0))
    g.add_particles(c, rad, np.array([1.3, 2.0, 0.9, 1.6]), v, om)
    return g


def _state(g):
    p = g.get_particles()
    d = {k: p[k].copy() for k in ("x", "u", "omega", "force", "torque")}
    d["orientation"] = g.get_orientations()
    return g.get_f(), g.get_tags(), d


def _same(a, b):
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    for k in a[2]:
        np.testing.assert_array_equal(a[2][k], b[2][k], err_msg=k)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resume_is_bit_for_bit(precision, tmp_path):
    a = _setup(precision)
    x0 = a.get_particles()["x"].copy()
    a.step(70)
    ref = _state(a)
    # the spheres must have crossed a shift boundary during the run
    assert np.max(np.abs(np.floor(ref[2]["x"] + 0.5) - np.floor(x0 + 0.5))) >= 1
    a.close()

    b = _setup(precision)
    b.step(35)
    path = tmp_path / "state.ckpt"
    b.save(str(path))
    b.close()

    c = _setup(precision)
    c.load(str(path))
    assert c.info()["steps"] == 35
    c.step(35)
    _same(_state(c), ref)
    c.close()


def test_rollback_in_the_same_context():
    g = _setup("fp32")
    g.step(20)
    ck = g.checkpoint()
    g.step(30)
    first = _state(g)
    g.restore(ck)
    g.step(30)
    _same(_state(g), first)
    g.close()


def test_checkpoint_of_a_different_setup_is_refused():
    g = _setup("fp32")
    g.step(5)
    ck = g.checkpoint()
    other = _setup("fp32", radius=4.0)   # different particles: different fingerprint
    with pytest.raises(lbmp.LbmError):
        other.restore(ck)
    with pytest.raises(lbmp.LbmError):
        g.restore(ck[:100])                # truncated
    other.close()
    g.close()


def test_checkpoint_with_other_face_kinds_is_refused():
    # Equilibrium faces and no-slip faces on the same axis are both walls; a checkpoint of one
    # must not load into the other (the saved face velocities drive different rules).
    def make(eq):
        faces = {4: (0.0, 0.0, 0.0), 5: (0.01, 0.0, 0.0)} if eq else None
        g = lbmp.Simulation(1, *DIMS, 0.7, precision="fp32", walls=(0, 0, 1), equilibrium_faces=faces)
        if not eq:
            g.set_wall_velocity(5, (0.01, 0.0, 0.0))
        return g
    a, b = make(True), make(False)
    a.step(3)
    b.step(3)
    ca, cb = a.checkpoint(), b.checkpoint()
    with pytest.raises(lbmp.LbmError):
        b.restore(ca)
    with pytest.raises(lbmp.LbmError):
        a.restore(cb)
    a.restore(ca)
    b.restore(cb)
    a.close()
    b.close()
