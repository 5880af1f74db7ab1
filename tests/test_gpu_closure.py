"""Closure inputs on the GPU (lbm_closure_features) against the oracle's stencil moments
computed from the oracle's own fields after the same steps (FP64 storage, so the two
states agree to round-off and the features to FP32 rounding)."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp_oracle as M
from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()
    O.build()


@pytest.mark.parametrize("walls", [(0, 0, 0), (0, 1, 1)])
def test_features_match_oracle_stencil_moments(walls):
    dims = (30, 26, 28)
    c = np.array([[8.3, 9.1, 10.4], [20.6, 15.2, 17.7], [14.0, 19.5, 7.1]])
    r = np.array([3.0, 3.5, 2.5])
    d = np.array([1.5, np.inf, 2.0])
    v = W.gaussian_velocities(3, 5e-3, seed=4)
    F = (2e-5, -1e-5, 0.0)
    g = lbmp.Simulation(1, *dims, 0.8, body_force=F, precision="fp64", walls=walls, gap=0.5)
    o = O.OracleSim(1, *dims, 0.8, body_force=F, walls=walls, gap=0.5)
    g.add_particles(c, r, d, v)
    o.add_particles(c, r, d, v)
    g.step(40)
    o.step(40)
    U = 3e-3
    got = g.closure_features(4, 4.0, U).cpu().double().numpy()
    rho, u = o.get_fields()
    p = o.get_particles()
    want = M.stencil_features(rho, u, p["x"], p["u"], 4, 4.0, U, walls)
    assert got.shape == (3, 4 * 64 + 3)
    assert np.max(np.abs(got[:, :256] - want)) <= 1e-6 * np.max(np.abs(want))
    # the fractional offset of each reference centre, as added
    assert np.max(np.abs(got[:, 256:] - (c - np.floor(c)))) <= 1e-6
    g.close()


def test_trained_closure_beats_the_coarse_method_on_held_out_seeds():
    # Paired coarse (r = 3) / fine (r = 12) runs of the same seeded cells; the network is
    # trained on the GPU on one set of seeds and judged on another. The plain coarse method
    # misses the fine drag by ~2.4 % on average; trained on 2048 samples the closure must
    # remove at least 40 % of that error (measured ~1.0 %; the bench's 3072 samples reach 0.9 %).
    from paper_1105_2904_gb300 import closure as CL
    spec = CL.PairSpec()
    Xtr, Ttr, ctr, ftr, str_ = CL.generate(spec, 256, seed=1)
    Xte, Tte, cte, fte, ste = CL.generate(spec, 32, seed=2)
    assert Xtr.shape == (256 * spec.n_spheres, CL.SIZES[0])
    cl = CL.Closure(seed=0)
    losses = cl.fit(Xtr, Ttr)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0]
    e_coarse = CL.drag_errors(cte, fte).mean()
    e_closure = CL.drag_errors(cl.corrected(Xte, cte, ste), fte).mean()
    print("held-out mean drag error vs fine: coarse %.4f, coarse + closure %.4f" % (e_coarse, e_closure))
    assert e_closure <= 0.6 * e_coarse
    cl.close()
