"""Host-side logic of the batched ensemble (no GPU): the sweep schedule covers every site of
every cell exactly once in each order and tile width, and the ensemble generator honours its
recipe (sizes, counts, radii, non-overlap under the minimum image, determinism)."""
import numpy as np
import pytest

from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()


def _covered(dims, table):
    seen = [np.zeros((d[2], d[1], d[0]), dtype=np.int64) for d in dims]
    for cell, x0, yw, z in table:
        lw = yw >> 16
        y0 = yw & 0xFFFF
        w = 1 << lw
        h = 128 // w
        nx, ny, nz = dims[cell]
        assert 0 <= z < nz and 0 <= x0 < nx and 0 <= y0 < ny
        xs = np.arange(x0, min(x0 + w, nx))
        ys = np.arange(y0, min(y0 + h, ny))
        seen[cell][z][np.ix_(ys, xs)] += 1
    return seen


@pytest.mark.parametrize("order", [0, 1, 2])
def test_schedule_covers_every_site_once(order):
    g = W.rng(5)
    dims = [tuple(int(v) for v in g.integers(1, 70, size=3)) for _ in range(7)]
    widths = [int(w) for w in g.choice([32, 64, 128], size=7)]
    table = lbmp.lbm_schedule_tiles(dims, widths, order)
    for s in _covered(dims, table):
        assert np.all(s == 1)
    expect = sum(-(-d[0] // w) * -(-d[1] // (128 // w)) * d[2] for d, w in zip(dims, widths))
    assert len(table) == expect


def test_schedule_orders():
    dims = [(40, 3, 2), (200, 5, 3), (10, 1, 1)]
    t0 = lbmp.lbm_schedule_tiles(dims, None, 0)
    t1 = lbmp.lbm_schedule_tiles(dims, None, 1)
    t2 = lbmp.lbm_schedule_tiles(dims, None, 2)
    # cell-major: cells in index order
    assert list(t0[:, 0]) == sorted(t0[:, 0])
    # round robin: the first tiles are one per cell
    assert list(t1[:3, 0]) == [0, 1, 2]
    # largest first: cell 1 (3000 sites) leads, then 0, then 2
    firsts = [int(c) for i, c in enumerate(t2[:, 0]) if i == 0 or t2[i - 1, 0] != c]
    assert firsts == [1, 0, 2]
    # the same tiles in every order
    key = lambda t: sorted(map(tuple, t.tolist()))
    assert key(t0) == key(t1) == key(t2)


def test_schedule_rejects_bad_arguments():
    with pytest.raises(ValueError):
        lbmp.lbm_schedule_tiles([(8, 8, 8)], [48], 0)
    with pytest.raises(ValueError):
        lbmp.lbm_schedule_tiles([(8, 8, 8)], None, 3)
    with pytest.raises(ValueError):
        lbmp.lbm_schedule_tiles([(0, 8, 8)], None, 0)


def test_ensemble_recipe():
    e = W.ensemble_cells(n_cells=16, seed=9)
    assert len(e.dims) == 16
    for (nx, ny, nz), tau, c, r, d, v in zip(e.dims, e.taus, e.centers, e.radii, e.densities, e.velocities):
        assert all(32 <= a <= 128 for a in (nx, ny, nz))
        assert 0.55 <= tau <= 1.0
        assert 0 <= len(r) <= 8 and c.shape == (len(r), 3) and v.shape == (len(r), 3)
        assert np.all((r >= 4.0) & (r <= 10.0)) and np.all(d == 1.2)
        L = np.array([nx, ny, nz], dtype=float)
        assert np.all((c >= 0) & (c < L))
        for i in range(len(r)):
            for j in range(i):
                dd = c[i] - c[j]
                dd -= L * np.floor(dd / L + 0.5)
                assert np.sqrt((dd * dd).sum()) >= r[i] + r[j] + 1.0 - 1e-12
    e2 = W.ensemble_cells(n_cells=16, seed=9)
    assert e2.dims == e.dims and all(np.array_equal(a, b) for a, b in zip(e.centers, e2.centers))


def test_crowded_cells_drop_spheres_and_count_them():
    # 8 spheres of radius 10 cannot all fit a 32^3 periodic cell
    c, r, dropped = W._place_spheres((32, 32, 32), np.full(8, 10.0), W.rng(1))
    assert dropped > 0 and len(r) + dropped == 8


class _FakeBatch:
    """Stands in for a Batch: records the tuning and reports a synthetic sweep time."""

    def __init__(self, dims, cost):
        self.dims = dims
        self.cost = cost
        self.tuning = None
        self.closed = False

    def set_tuning(self, **t):
        self.tuning = t

    def close(self):
        self.closed = True


def test_min_waste_width():
    from paper_1105_2904_gb300 import autotune as AT
    assert AT.min_waste_width(128, 64) == 128
    assert AT.min_waste_width(33, 100) == 64 and AT.padded_sites(33, 100, 64) == 64 * 100  # tie: wider
    assert AT.min_waste_width(70, 7) == 32   # 3 x 32 wide, 2 x 4 rows
    for nx, ny in [(32, 32), (45, 77), (128, 1), (1, 128)]:
        w = AT.min_waste_width(nx, ny)
        assert all(AT.padded_sites(nx, ny, w) <= AT.padded_sites(nx, ny, v) for v in AT.WIDTHS)


def test_tune_picks_fastest_and_caches(tmp_path):
    from paper_1105_2904_gb300 import autotune as AT
    dims = [(40, 50, 60), (100, 33, 70)]

    def cost(t):
        return 1.0 + 0.1 * t["order"] + (0.5 if t["grid"] else 0.0) + (0.0 if all(w == 64 for w in t["tile_width"]) else 0.3)

    b = _FakeBatch(dims, cost)
    timer = lambda bb, n: cost(bb.tuning)
    cache = str(tmp_path / "tune.json")
    key = AT.shape_key("D3Q19", "fp32", dims, 9)
    best, res = AT.tune(b, timer=timer, cache=cache, key=key, steps_per_graph=10)
    assert best["order"] == 0 and best["grid"] == 0 and best["tile_width"] == [64, 64]
    assert len(res) == 4 * 3 * 2 and b.tuning["steps_per_graph"] == 10
    # the second call reads the cache and times nothing
    b2 = _FakeBatch(dims, cost)
    best2, res2 = AT.tune(b2, timer=lambda *a: 1 / 0, cache=cache, key=key)
    assert res2 == [] and best2["tile_width"] == [64, 64] and b2.tuning["order"] == 0


def test_choose_precision_respects_the_error_bound():
    from paper_1105_2904_gb300 import autotune as AT
    dims = [(64, 64, 64)]
    speed = {"fp32": 2.0, "fp16": 1.2, "bf16": 1.1}
    made = []

    def make(p):
        b = _FakeBatch(dims, None)
        b.p = p
        made.append(b)
        return b

    timer = lambda b, n: speed[b.p]
    p, table = AT.choose_precision(make, 1e-5, timer=timer)
    assert p == "fp32" and set(table) == {"fp32"}
    p, table = AT.choose_precision(make, 1e-3, timer=timer)
    assert p == "fp16" and set(table) == {"fp32", "fp16"}
    p, table = AT.choose_precision(make, 1e-2, timer=timer)
    assert p == "bf16"
    assert all(b.closed for b in made)
    with pytest.raises(ValueError):
        AT.choose_precision(make, 1e-9, timer=timer)
