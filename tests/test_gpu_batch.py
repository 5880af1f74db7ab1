"""Batched ensembles on the CUDA path.

- FP64 storage: each cell of a batch matches its own FP64 oracle run to 1e-12 relative
  (fields, particle trajectories, force and torque) and bit for bit on the owner map.
- FP32 / FP16 storage: each cell of a batch is bit for bit the same as the same cell stepped
  alone as a single context with the one-site sweep kernel, under every launch tuning (tile
  widths, schedule orders, persistent grids, multi-step graphs): the batch changes how the
  work is launched, not what is computed.
- Cells without particles, walls, and the buffer-parity rule.
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


def rel(a, b, scale=None):
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / max(s, 1e-300))


def small_ensemble(n_cells, seed, edge=(20, 44), spheres=(0, 3), radius=(3.0, 5.0)):
    return W.ensemble_cells(n_cells=n_cells, seed=seed, edge=edge, spheres=spheres, radius=radius,
                            velocity_sigma=5e-3)


def make_batch(e, precision, walls=(0, 0, 0), gravity=(0, 0, 0), gap=0.5):
    F = [e.body_force] * len(e.dims)
    b = lbmp.Batch(O.D3Q19, e.dims, e.taus, F, precision=precision, walls=walls, gravity=gravity, gap=gap,
                   body_force_on_particles=e.body_force_on_particles)
    for k in range(len(e.dims)):
        if len(e.radii[k]):
            b.add_particles(k, e.centers[k], e.radii[k], e.densities[k], e.velocities[k])
    return b


def test_batch_fp64_matches_oracle_per_cell():
    e = small_ensemble(5, 21)
    assert any(len(r) == 0 for r in e.radii) and any(len(r) > 1 for r in e.radii)
    b = make_batch(e, "fp64")
    b.set_tuning(tile_width=[32, 64, 128, 32, 64], order=1, steps_per_graph=5)
    b.step(120)
    for k in range(len(e.dims)):
        nx, ny, nz = e.dims[k]
        r = O.OracleSim(O.D3Q19, nx, ny, nz, e.taus[k], body_force=e.body_force, gap=0.5,
                        body_force_on_particles=e.body_force_on_particles)
        if len(e.radii[k]):
            r.add_particles(e.centers[k], e.radii[k], e.densities[k], e.velocities[k])
        r.step(120)
        g = b.cell(k)
        rg, ug = g.get_fields()
        rr, ur = r.get_fields()
        assert rel(ug, ur) <= 1e-12 and rel(rg, rr, np.max(np.abs(rr - 1.0))) <= 1e-12, k
        if len(e.radii[k]):
            assert np.array_equal(g.get_tags(), r.get_tags()), k
            pg, pr = g.get_particles(), r.get_particles()
            for key in ("x", "u", "omega", "force", "torque"):
                assert rel(pg[key], pr[key]) <= 1e-12, (k, key)
    b.close()


def _separate(e, precision, steps, walls=(0, 0, 0), gravity=(0, 0, 0)):
    out = []
    for k in range(len(e.dims)):
        nx, ny, nz = e.dims[k]
        s = lbmp.Simulation(O.D3Q19, nx, ny, nz, e.taus[k], body_force=e.body_force, precision=precision,
                            walls=walls, gravity=gravity, gap=0.5, body_force_on_particles=e.body_force_on_particles)
        s.set_sweep_shape(0)   # the batch runs the one-site sweep of every cell
        if len(e.radii[k]):
            s.add_particles(e.centers[k], e.radii[k], e.densities[k], e.velocities[k])
        s.step(steps)
        out.append((s.get_f(), s.get_particles() if len(e.radii[k]) else None, s.get_tags()))
        s.close()
    return out


def _same_bits(b, ref, e):
    for k in range(len(e.dims)):
        c = b.cell(k)
        f, p, t = ref[k]
        assert np.array_equal(c.get_f(), f), k
        assert np.array_equal(c.get_tags(), t), k
        if p is not None:
            q = c.get_particles()
            for key in ("x", "u", "omega", "force", "torque"):
                assert np.array_equal(q[key], p[key]), (k, key)


TUNINGS = [
    dict(tile_width=None, order=0, grid=0, steps_per_graph=1),
    dict(tile_width="random", order=1, grid=0, steps_per_graph=7),
    dict(tile_width="random", order=2, grid=304, steps_per_graph=4),
    dict(tile_width=32, order=0, grid=152, steps_per_graph=1),
]


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("ti", range(len(TUNINGS)))
def test_batch_is_bitwise_the_cells_stepped_alone(precision, ti):
    e = small_ensemble(6, 31 + ti)
    ref = _separate(e, precision, 60)
    b = make_batch(e, precision)
    t = dict(TUNINGS[ti])
    if t["tile_width"] == "random":
        t["tile_width"] = [int(w) for w in W.rng(ti).choice([32, 64, 128], size=len(e.dims))]
    elif isinstance(t["tile_width"], int):
        t["tile_width"] = [t["tile_width"]] * len(e.dims)
    b.set_tuning(**t)
    b.step(60)
    _same_bits(b, ref, e)
    b.close()


def test_batch_with_walls_and_gravity_is_bitwise_the_cells_stepped_alone():
    e = small_ensemble(4, 41, spheres=(1, 3))
    walls, grav = (0, 1, 1), (0.0, -2e-4, 0.0)
    # spheres must clear the walls: keep only those inside
    for k, (nx, ny, nz) in enumerate(e.dims):
        keep = [i for i in range(len(e.radii[k]))
                if e.centers[k][i, 1] - e.radii[k][i] > 0.5 and e.centers[k][i, 1] + e.radii[k][i] < ny - 1.5
                and e.centers[k][i, 2] - e.radii[k][i] > 0.5 and e.centers[k][i, 2] + e.radii[k][i] < nz - 1.5]
        e.centers[k], e.radii[k] = e.centers[k][keep], e.radii[k][keep]
        e.densities[k], e.velocities[k] = e.densities[k][keep], e.velocities[k][keep]
    ref = _separate(e, "fp32", 50, walls, grav)
    b = make_batch(e, "fp32", walls=walls, gravity=grav)
    b.set_tuning(order=2, steps_per_graph=5)
    b.step(50)
    _same_bits(b, ref, e)
    b.close()


def test_cells_must_share_their_parity():
    e = small_ensemble(2, 51)
    b = make_batch(e, "fp32")
    b.step(2)
    b.cell(0).step(1)
    with pytest.raises(lbmp.LbmError):
        b.step(1)
    b.cell(1).step(1)
    b.step(1)
    b.synchronize()
    b.close()
