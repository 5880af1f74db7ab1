"""Every sweep kernel shape against the FP64 oracle on the same seeded suspensions.

The two-site kernel (threads_x = 16, 32, 64, 128) and the one-site kernel (0) run moving,
spinning spheres that cross shift boundaries, in boxes whose nx and ny leave ragged tails
for every block shape, with walls on x (bounce-back inside the paired loads) or fully
periodic. Bars as for the one-site kernel: FP32 storage within 1e-5 of max|u| and 1e-4 of
max|F|, owner maps bit for bit; FP16 / BF16 storage within the storage-precision bounds
of the long parity test."""
import numpy as np
import pytest

import oracle as O
from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [0, 16, 32, 64, 128]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()
    O.build()


def rel(a, b, scale=None):
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


CASES = {
    # nx = 70: 35 pairs, ragged for every threads_x; ny = 21: ragged for 2, 4 and 8 rows
    "periodic": dict(dims=(70, 21, 18), walls=(0, 0, 0), F=(2e-6, 0.0, 0.0), n=4, seed=61),
    "walls_x": dict(dims=(66, 19, 20), walls=(1, 0, 0), F=(0.0, 1e-6, 0.0), n=4, seed=62),
}


def _setup(case, precision, steps):
    dims, walls = case["dims"], case["walls"]
    c, rad = W.rsa_centers(dims, case["n"], 4.5, seed=case["seed"], min_gap=2.0, walls=walls)
    v = W.gaussian_velocities(case["n"], 0.03, seed=case["seed"] + 1)
    om = W.gaussian_velocities(case["n"], 0.004, seed=case["seed"] + 2)
    d = np.array([1.3, 2.0, 0.9, 1.6])[: case["n"]]
    r = O.OracleSim(1, *dims, 0.7, body_force=case["F"], walls=walls, gap=0.5, body_force_on_particles=True)
    r.add_particles(c, rad, d, v, om)
    r.step(steps)
    return (dims, walls, c, rad, d, v, om), r


@pytest.fixture(scope="module")
def oracle_runs():
    return {name: _setup(case, "fp32", 120) for name, case in CASES.items()}


def _gpu(case, setup, precision, shape, steps):
    dims, walls, c, rad, d, v, om = setup
    g = lbmp.Simulation(1, *dims, 0.7, body_force=case["F"], precision=precision, walls=walls, gap=0.5,
                        body_force_on_particles=True)
    g.set_sweep_shape(shape)
    g.add_particles(c, rad, d, v, om)
    g.step(steps)
    return g


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("name", list(CASES))
def test_fp32_shapes_match_oracle(name, shape, oracle_runs):
    setup, r = oracle_runs[name]
    g = _gpu(CASES[name], setup, "fp32", shape, 120)
    np.testing.assert_array_equal(g.get_tags(), r.get_tags())
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-5
    pg, pr = g.get_particles(), r.get_particles()
    assert rel(pg["force"], pr["force"]) <= 1e-4
    rad = setup[3]
    assert np.max(np.abs(pg["x"] - pr["x"]) / np.asarray(rad)[:, None]) <= 1e-5
    g.close()


@pytest.mark.parametrize("precision,bound", [("fp16", 2e-3), ("bf16", 2e-2)])
@pytest.mark.parametrize("shape", [0, 32])
def test_reduced_storage_shapes_within_bounds(precision, bound, shape, oracle_runs):
    setup, r = oracle_runs["periodic"]
    g = _gpu(CASES["periodic"], setup, precision, shape, 120)
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    pg, pr = g.get_particles(), r.get_particles()
    assert rel(ug, ur) <= bound
    assert rel(pg["force"], pr["force"]) <= bound
    g.close()


def test_invalid_shape_is_rejected():
    g = lbmp.Simulation(1, 8, 8, 8, 0.7, precision="fp32")
    with pytest.raises(lbmp.LbmError):
        g.set_sweep_shape(48)
    g.close()


# D2Q9: settling disks in a closed box (walls on x and y; bounce-back of both sites of a pair at
# the x walls), the shape of the 1024 x 2048 sedimentation workload at a small size.
D2_DIMS = (62, 90, 1)


@pytest.fixture(scope="module")
def oracle_2d():
    c, rad = W.rsa_centers((62, 90), 6, 5.0, seed=81, min_gap=1.0, walls=(1, 1, 0))
    d = np.full(6, 1.5)
    r = O.OracleSim(0, *D2_DIMS, 0.7, walls=(1, 1, 0), gravity=(0.0, -2e-3, 0.0), gap=0.5)
    r.add_particles(c, rad, d)
    r.step(200)
    return (c, rad, d), r


def _gpu2d(setup, precision, shape):
    c, rad, d = setup
    g = lbmp.Simulation(0, *D2_DIMS, 0.7, precision=precision, walls=(1, 1, 0), gravity=(0.0, -2e-3, 0.0), gap=0.5)
    g.set_sweep_shape(shape)
    g.add_particles(c, rad, d)
    g.step(200)
    return g


@pytest.mark.parametrize("shape", [0, 16, 32, 128])
def test_d2q9_walled_settling_fp32_shapes(shape, oracle_2d):
    setup, r = oracle_2d
    g = _gpu2d(setup, "fp32", shape)
    np.testing.assert_array_equal(g.get_tags(), r.get_tags())
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    assert rel(ug, ur) <= 1e-5
    pg, pr = g.get_particles(), r.get_particles()
    assert rel(pg["force"], pr["force"]) <= 1e-4
    assert np.max(np.abs(pg["x"] - pr["x"]) / np.asarray(setup[1])[:, None]) <= 1e-5
    g.close()


@pytest.mark.parametrize("precision,bound", [("fp16", 2e-3), ("bf16", 2e-2)])
def test_d2q9_walled_settling_reduced_storage_default_shape(precision, bound, oracle_2d):
    setup, r = oracle_2d
    g = _gpu2d(setup, precision, -1)
    rg, ug = g.get_fields()
    rr, ur = r.get_fields()
    pg, pr = g.get_particles(), r.get_particles()
    assert rel(ug, ur) <= bound
    assert rel(pg["force"], pr["force"]) <= bound
    g.close()
