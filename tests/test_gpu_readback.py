"""Asynchronous particle read-back (lbm_get_particles_async / lbm_wait_particles): the same
values as the synchronous lbm_get_particles, step after step, with read-backs in flight while
later steps run; the ticket rules. Also the device bytes lbm_get_info reports when particles
are added in several calls (the arrays of the earlier calls are freed)."""
import numpy as np
import pytest

from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()


def _sim():
    dims = (40, 34, 30)
    c, rad = W.rsa_centers(dims, 5, 4.0, seed=91, min_gap=2.0)
    v = W.gaussian_velocities(5, 0.02, seed=92)
    g = lbmp.Simulation(1, *dims, 0.7, body_force=(1e-6, 0, 0), precision="fp32", body_force_on_particles=True)
    g.add_particles(c, rad, np.full(5, 1.5), v)
    return g


def test_async_read_back_equals_the_synchronous_one():
    # a: every step enqueues a read-back and waits for the one two steps back; b: the
    # synchronous getter after every step. Same inputs, same kernels: identical values.
    a, b = _sim(), _sim()
    n = a.np
    bufs = [torch.empty(15 * n + 1, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    want, tickets = [], []
    for k in range(12):
        a.step(1)
        tickets.append(a.get_particles_async(bufs[k % 3]))
        b.step(1)
        want.append(b.get_particles())
        if k >= 2:
            j = k - 2
            a.wait_particles(tickets[j])
            have = lbmp.unpack_particles(bufs[j % 3].numpy(), n)
            for key in want[j]:
                np.testing.assert_array_equal(have[key], want[j][key], err_msg=key)
    for t in tickets[-2:]:
        a.wait_particles(t)
    a.close()
    b.close()


def test_ticket_rules():
    g = _sim()
    n = g.np
    bufs = [torch.empty(15 * n + 1, dtype=torch.float64, pin_memory=True) for _ in range(9)]
    ts = [g.get_particles_async(bufs[i]) for i in range(8)]
    with pytest.raises(lbmp.LbmError):
        g.get_particles_async(bufs[8])          # 8 outstanding
    g.wait_particles(ts[0])
    with pytest.raises(lbmp.LbmError):
        g.wait_particles(ts[0])                 # already waited
    t = g.get_particles_async(bufs[8])          # a slot is free again
    for x in ts[1:] + [t]:
        g.wait_particles(x)
    g.close()


def test_device_bytes_after_particles_added_in_two_calls():
    dims = (40, 34, 30)
    c, rad = W.rsa_centers(dims, 5, 4.0, seed=91, min_gap=2.0)
    v = W.gaussian_velocities(5, 0.02, seed=92)
    one = lbmp.Simulation(1, *dims, 0.7, precision="fp32")
    one.add_particles(c, rad, np.full(5, 1.5), v)
    two = lbmp.Simulation(1, *dims, 0.7, precision="fp32")
    two.add_particles(c[:2], rad[:2], np.full(2, 1.5), v[:2])
    two.add_particles(c[2:], rad[2:], np.full(3, 1.5), v[2:])
    assert two.info()["device_bytes"] == one.info()["device_bytes"]
    one.step(3)
    two.step(3)
    np.testing.assert_array_equal(two.get_particles()["force"], one.get_particles()["force"])
    one.close()
    two.close()
