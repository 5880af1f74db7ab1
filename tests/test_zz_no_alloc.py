"""The allocation-free boundary-site exchange agrees with the step a context takes.

lbm_bs_exchange_noalloc serves callers that cannot allocate device memory (memory owned by
their own pool, allocation forbidden while recording work or inside a real-time loop): they
pass all buffers and the library only uses a fixed device array of its own. Here the force
and torque it returns for a state are checked against what lbm_step + lbm_get_particles
report for one step from the same state, with the FP32 tolerances of the parity tests, on
two calls in a row (the second call must not see the first call's sums): for the state the
particles were added in, and for a state reached after the particles have moved by
fractions of a site and some have changed their whole-site shift, where the centres passed
are those of the site sets, x_p0 + floor(x_p - x_p0 + 1/2), not the positions x_p."""
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


def _case(lattice):
    if lattice == lbmp.LBM_D3Q19:
        dims, walls, F = (41, 36, 30), (0, 0, 0), (2e-6, -1e-6, 0.0)
        c, r = W.rsa_centers(dims, 5, 5.0, seed=71, min_gap=1.0)
        v = W.gaussian_velocities(5, 0.02, seed=72)
        om = W.gaussian_velocities(5, 0.003, seed=73)
        dens = np.array([1.2, 2.0, 0.9, 1.5, 3.0])
    else:
        dims, walls, F = (60, 90, 1), (1, 1, 0), (1e-6, 0.0, 0.0)
        c, r = W.rsa_centers((60, 90), 6, 5.0, seed=74, min_gap=1.0, walls=(1, 1, 0))
        v = W.gaussian_velocities(6, 0.02, seed=75, dims=2)
        om = np.zeros((6, 3))
        om[:, 2] = W.rng(76).normal(0.0, 0.003, 6)
        dens = np.full(6, 1.5)
    return dims, walls, F, c, r, v, om, dens


@pytest.mark.parametrize("steps_before", [0, 90], ids=["at_start", "moved"])
@pytest.mark.parametrize("lattice", [lbmp.LBM_D3Q19, lbmp.LBM_D2Q9], ids=["d3q19", "d2q9"])
def test_noalloc_exchange_matches_the_context_step(lattice, steps_before):
    import torch

    dims, walls, F, c, r, v, om, dens = _case(lattice)
    nx, ny, nz = dims
    D = 3 if lattice == lbmp.LBM_D3Q19 else 2
    _, w = O.lattice_tables(lattice)
    Q, N = len(w), nx * ny * nz
    xi = W.perturbation(Q, (nz, ny, nx), seed=77)
    f0 = w[:, None, None, None] * (1.0 + 0.02 * xi)

    sim = lbmp.Simulation(lattice, nx, ny, nz, 0.7, body_force=F, precision="fp32", walls=walls)
    sim.set_f(f0)
    sim.add_particles(c, r, dens, v, om)
    sim.step(steps_before)
    f_start = sim.get_f()
    tags = sim.get_tags()
    p = sim.get_particles()
    # centre of each particle's site set: the initial centre moved by whole sites (Eqs. 14-15)
    centre = np.array(c, dtype=np.float64).copy()
    centre[:, :D] += np.floor((p["x"][:, :D] - centre[:, :D]) + 0.5)
    if steps_before:
        frac = np.abs(p["x"][:, :D] - centre[:, :D])
        assert np.any(centre[:, :D] != np.asarray(c)[:, :D])      # some shift changed
        assert np.any((frac > 0.05) & (frac < 0.45))             # away from the site-set centre
    sim.step(1)
    ref = sim.get_particles()
    sim.close()

    dev = "cuda"
    g = torch.tensor((f_start - w[:, None, None, None]).reshape(Q, N), dtype=torch.float32, device=dev)
    t = torch.from_numpy(np.ascontiguousarray(tags.reshape(-1)).view(np.int32)).to(dev)
    cen = torch.tensor(centre, dtype=torch.float64, device=dev)
    vel = torch.tensor(p["u"], dtype=torch.float64, device=dev)
    omg = torch.tensor(p["omega"], dtype=torch.float64, device=dev)
    n = len(r)
    force = torch.empty((n, 3), dtype=torch.float64, device=dev)
    torque = torch.empty((n, 3), dtype=torch.float64, device=dev)
    fscale = np.max(np.abs(ref["force"]))
    tscale = max(np.max(np.abs(ref["torque"])), fscale * float(np.max(r)))
    for call in range(2):
        force.fill_(math.nan)
        torque.fill_(math.nan)
        lbmp.lbm_bs_exchange_noalloc(lattice, nx, ny, nz, walls, F, g.data_ptr(), t.data_ptr(), n,
                                     cen.data_ptr(), vel.data_ptr(), omg.data_ptr(), force.data_ptr(),
                                     torque.data_ptr(), None)
        torch.cuda.synchronize()
        fo, to = force.cpu().numpy(), torque.cpu().numpy()
        assert np.max(np.abs(fo - ref["force"])) / fscale <= 1e-4, call
        assert np.max(np.abs(to - ref["torque"])) / tscale <= 1e-4, call


def test_noalloc_rejects_too_many_particles():
    with pytest.raises(lbmp.LbmError):
        lbmp.lbm_bs_exchange_noalloc(1, 8, 8, 8, None, None, 1, 1, 65537, 1, 1, 1, 1, 1, None)
