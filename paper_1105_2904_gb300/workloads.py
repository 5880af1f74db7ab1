"""Seeded synthetic inputs: particle placements, velocities and distribution perturbations.

This module holds no arithmetic of the method itself. It only draws inputs (positions,
radii, velocities, random perturbation fields) from seeded generators, so that the CUDA
path and the FP64 oracle can be fed identical data. The workloads mirror the shapes of
the paper's experiments (Sec. 3): a fixed disk in a periodic channel (Sec. 3.1), hundreds
of disks sedimenting in a closed box (Sec. 3.4) and dense 3D suspensions of spheres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def perturbation(q: int, shape, seed: int) -> np.ndarray:
    """Uniform(-1, 1) field of shape (q,) + shape, used to perturb rest distributions."""
    return rng(seed).uniform(-1.0, 1.0, size=(q,) + tuple(shape))


def rsa_centers(dims, n, radii, seed, min_gap=1.0, walls=(0, 0, 0), wall_clearance=None,
                batch=4096, max_batches=100_000):
    """Random sequential addition of ``n`` non-overlapping spheres (disks when dims has two
    entries, or nz == 1) in a box of size ``dims`` = (nx, ny[, nz]).

    ``radii`` is a scalar or an array of n radii (sphere k gets radii[k]). Spheres keep a
    surface gap >= min_gap; along axes with walls[k] = 1 the centre stays wall_clearance
    (default r + min_gap) away from the wall planes at -1/2 and n - 1/2; other axes are
    periodic (minimum image). Proposals are drawn in batches; proposal j of a batch is kept
    when it clears every sphere placed before the batch and every earlier kept proposal of
    the same batch, so the result depends only on the seed. Returns (centers (n,3), radii).
    """
    dims = tuple(int(d) for d in dims)
    if len(dims) == 2:
        dims = dims + (1,)
    D = 2 if dims[2] == 1 else 3
    r_all = np.broadcast_to(np.asarray(radii, dtype=np.float64), (n,)).copy()
    g = rng(seed)
    rmax = float(r_all.max()) if n else 1.0
    h = 2.0 * rmax + min_gap
    ncell = np.array([max(1, int(dims[k] // h)) if k < D else 1 for k in range(3)])
    csize = np.array([dims[k] / ncell[k] for k in range(3)])
    rmin = float(r_all.min()) if n else 1.0
    cap = int(math.ceil((h / (2.0 * rmin + min_gap) + 1.0) ** D))
    members = -np.ones((int(np.prod(ncell)), cap), dtype=np.int64)
    counts = np.zeros(int(np.prod(ncell)), dtype=np.int64)
    centers = np.zeros((n, 3))
    dimsf = np.array(dims, dtype=np.float64)
    per = np.array([(not walls[k]) and k < D for k in range(3)])
    offs = np.array([(dx, dy, dz) for dz in ((-1, 0, 1) if D == 3 else (0,))
                     for dy in (-1, 0, 1) for dx in (-1, 0, 1)], dtype=np.int64)
    placed = 0

    def cell_ids(c):
        key = np.minimum((c // csize).astype(np.int64), ncell - 1)
        key = np.maximum(key, 0)
        return key

    def in_grid(cells):
        """Wraps periodic cell coordinates; returns (flat ids, valid mask)."""
        cells = cells.copy()
        valid = np.ones(cells.shape[:-1], dtype=bool)
        for k in range(3):
            out = (cells[..., k] < 0) | (cells[..., k] >= ncell[k])
            if walls[k] or k >= D:
                valid &= ~out
            cells[..., k] %= ncell[k]
        return (cells[..., 2] * ncell[1] + cells[..., 1]) * ncell[0] + cells[..., 0], valid

    def clashes(c, rc, ids):
        """True per row of ``ids`` where sphere (c[row], rc[row]) overlaps one of the
        spheres listed in that row (-1 = empty slot)."""
        rows, cols = np.nonzero(ids >= 0)
        m = ids[rows, cols]
        d = c[rows] - centers[m]
        d = np.where(per, d - dimsf * np.floor(d / dimsf + 0.5), d)
        rr = rc[rows] + r_all[m] + min_gap
        hit = (d * d).sum(-1) < rr * rr
        out = np.zeros(ids.shape[0], dtype=bool)
        out[rows[hit]] = True
        return out

    for _ in range(max_batches):
        if placed >= n:
            break
        ri = r_all[placed]
        lo = np.zeros(3)
        hi = np.zeros(3)
        for k in range(D):
            if walls[k]:
                cl = ri + min_gap if wall_clearance is None else wall_clearance
                lo[k], hi[k] = -0.5 + cl, dims[k] - 0.5 - cl
            else:
                lo[k], hi[k] = 0.0, float(dims[k])
        prop = g.uniform(lo, hi, size=(batch, 3))
        prop[:, D:] = 0.0
        key = cell_ids(prop)
        flat, valid = in_grid(key[:, None, :] + offs[None, :, :])
        cand = np.where(valid[:, :, None], members[flat], -1).reshape(batch, -1)
        survivors = np.nonzero(~clashes(prop, np.full(batch, ri), cand))[0]
        run = 1
        while placed + run < n and r_all[placed + run] == ri:
            run += 1
        survivors = survivors[: 4 * run + 64]
        sp = prop[survivors]
        d2 = np.zeros((len(sp), len(sp)))
        for k in range(D):
            dk = sp[:, None, k] - sp[None, :, k]
            if per[k]:
                dk = dk - dimsf[k] * np.floor(dk / dimsf[k] + 0.5)
            d2 += dk * dk
        conflict = np.triu(d2 < (2.0 * ri + min_gap) ** 2, k=1)   # conflict[a, b], a < b
        kept = np.zeros(len(sp), dtype=bool)
        for j in range(len(sp)):
            if kept.sum() >= run:
                break
            if conflict[:j, j][kept[:j]].any():
                continue
            kept[j] = True
        for j in survivors[kept]:
            fid = (key[j][2] * ncell[1] + key[j][1]) * ncell[0] + key[j][0]
            if counts[fid] >= cap:
                raise RuntimeError("rsa_centers: cell capacity exceeded")
            members[fid, counts[fid]] = placed
            counts[fid] += 1
            centers[placed] = prop[j]
            placed += 1
    if placed < n:
        raise RuntimeError("rsa_centers: could not place %d spheres (placed %d)" % (n, placed))
    return centers, r_all


def gaussian_velocities(n, sigma, seed, dims=3):
    v = rng(seed).normal(0.0, sigma, size=(n, 3))
    if dims == 2:
        v[:, 2] = 0.0
    return v


@dataclass
class Workload:
    """A named synthetic workload (sizes in lattice units)."""

    name: str
    lattice: str                 # "D2Q9" or "D3Q19"
    dims: tuple                  # (nx, ny, nz)
    tau: float
    body_force: tuple = (0.0, 0.0, 0.0)
    walls: tuple = (0, 0, 0)
    gravity: tuple = (0.0, 0.0, 0.0)
    n_particles: int = 0
    radius: float = 0.0
    density_ratio: float = 1.0
    velocity_sigma: float = 0.0
    seed: int = 0
    min_gap: float = 1.0
    steps: int = 1
    precision: str = "fp32"
    body_force_on_particles: bool = False
    fixed_centers: list = field(default_factory=list)

    @property
    def sites(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    def particles(self):
        """(centers, radii, densities, velocities) drawn from the workload's seed."""
        if self.fixed_centers:
            c = np.asarray(self.fixed_centers, dtype=np.float64).reshape(-1, 3)
            n = c.shape[0]
            r = np.full(n, float(self.radius))
            d = np.full(n, float(self.density_ratio))
            v = np.zeros((n, 3))
            return c, r, d, v
        if self.n_particles == 0:
            z = np.zeros((0, 3))
            return z, np.zeros(0), np.zeros(0), z
        two_d = self.lattice == "D2Q9"
        dims = self.dims[:2] if two_d else self.dims
        c, r = rsa_centers(dims, self.n_particles, self.radius, self.seed, self.min_gap, self.walls)
        d = np.full(self.n_particles, float(self.density_ratio))
        v = gaussian_velocities(self.n_particles, self.velocity_sigma, self.seed + 1,
                                2 if two_d else 3)
        return c, r, d, v


def channel_disk_2d() -> Workload:
    """D2Q9 128x64 periodic channel, body force 1e-6, tau 0.8, one fixed disk r = 8 at the
    centre, FP64, 2000 steps (flow past a massive particle, Sec. 3.1)."""
    return Workload("d2q9_channel_disk_128x64", "D2Q9", (128, 64, 1), 0.8, body_force=(1e-6, 0, 0),
                    radius=8.0, density_ratio=math.inf, fixed_centers=[[64.0, 32.0, 0.0]],
                    steps=2000, precision="fp64")


def sedimentation_2d() -> Workload:
    """D2Q9 1024x2048 closed box, 500 disks r = 10, density ratio 1.5, gravity 1e-5,
    tau 0.7, FP32, 20000 steps (many disks settling in an enclosure, Sec. 3.4)."""
    return Workload("d2q9_sedimentation_1024x2048_500disks", "D2Q9", (1024, 2048, 1), 0.7,
                    walls=(1, 1, 0), gravity=(0.0, -1e-5, 0.0), n_particles=500, radius=10.0,
                    density_ratio=1.5, seed=2, min_gap=2.0, steps=20000, precision="fp32")


def suspension_3d(n=512, n_particles=16000, radius=8.0, seed=3) -> Workload:
    """D3Q19 n^3 periodic box with spheres r = 8 at about 25 % solid fraction (16000 spheres
    at 512^3), velocities N(0, 1e-3), density ratio 1.2, tau 0.6, body force 1e-6, 1000 steps."""
    return Workload("d3q19_suspension_%d^3_%dspheres_r%g" % (n, n_particles, radius), "D3Q19",
                    (n, n, n), 0.6, body_force=(1e-6, 0.0, 0.0), n_particles=n_particles,
                    radius=radius, density_ratio=1.2, velocity_sigma=1e-3, seed=seed, min_gap=1.0,
                    steps=1000, precision="fp32", body_force_on_particles=True)


def suspension_3d_scaled(n: int, seed=3) -> Workload:
    """The 512^3 suspension scaled to n^3 with the same solid fraction and sphere size."""
    n_particles = max(1, int(round(16000 * (n / 512.0) ** 3)))
    return suspension_3d(n, n_particles, 8.0, seed)


@dataclass
class Ensemble:
    """Independent periodic D3Q19 cells of uneven sizes, each with a few spheres."""

    name: str
    dims: list                   # [(nx, ny, nz)] per cell
    taus: list
    centers: list                # per cell: [n_k, 3]
    radii: list                  # per cell: [n_k]
    densities: list
    velocities: list
    dropped: list                # spheres of the draw that did not fit, per cell
    body_force: tuple = (1e-6, 0.0, 0.0)
    body_force_on_particles: bool = True
    steps: int = 500
    precision: str = "fp32"

    @property
    def sites(self) -> int:
        return int(sum(int(a) * int(b) * int(c) for a, b, c in self.dims))

    @property
    def n_particles(self) -> int:
        return int(sum(len(r) for r in self.radii))


def _place_spheres(dims, radii, g, min_gap=1.0, attempts=10_000):
    """Random sequential addition in a periodic box: each sphere takes the first of
    `attempts` uniform candidate centres that keeps a surface gap >= min_gap to the spheres
    already placed (minimum image); a sphere with no such candidate is dropped."""
    L = np.asarray(dims, dtype=np.float64)
    placed_c, placed_r, dropped = [], [], 0
    for r in radii:
        cand = g.uniform(0.0, 1.0, size=(attempts, 3)) * L
        ok = np.ones(attempts, dtype=bool)
        for c, rr in zip(placed_c, placed_r):
            d = cand - c
            d -= L * np.floor(d / L + 0.5)
            ok &= (d * d).sum(1) >= (r + rr + min_gap) ** 2
        idx = np.flatnonzero(ok)
        if idx.size == 0:
            dropped += 1
            continue
        placed_c.append(cand[idx[0]])
        placed_r.append(float(r))
    c = np.asarray(placed_c, dtype=np.float64).reshape(-1, 3)
    return c, np.asarray(placed_r, dtype=np.float64), dropped


def ensemble_cells(n_cells=64, seed=4, edge=(32, 128), spheres=(1, 8), radius=(4.0, 10.0),
                   tau=(0.55, 1.0), density_ratio=1.2, velocity_sigma=1e-3) -> Ensemble:
    """Batched-ensemble workload: n_cells periodic cells, each edge drawn independently and
    uniformly from the integers edge[0]..edge[1], a uniform integer number of spheres in
    spheres[0]..spheres[1] with radii uniform in radius (placed by random sequential
    addition, min gap 1; spheres that do not fit after 10^4 attempts are dropped and
    counted), tau uniform in the given range, velocities N(0, velocity_sigma^2), density
    ratio 1.2, body force 1e-6 along x on fluid and particles, FP32, 500 steps."""
    g = rng(seed)
    dims = [tuple(int(v) for v in g.integers(edge[0], edge[1] + 1, size=3)) for _ in range(n_cells)]
    taus = [float(v) for v in g.uniform(tau[0], tau[1], size=n_cells)]
    cs, rs, ds, vs, drop = [], [], [], [], []
    for k in range(n_cells):
        gk = rng(seed * 1000 + 17 + k)
        n = int(gk.integers(spheres[0], spheres[1] + 1))
        r = gk.uniform(radius[0], radius[1], size=n)
        c, rr, dropped = _place_spheres(dims[k], r, gk)
        cs.append(c)
        rs.append(rr)
        ds.append(np.full(len(rr), float(density_ratio)))
        vs.append(gk.normal(0.0, velocity_sigma, size=(len(rr), 3)))
        drop.append(dropped)
    return Ensemble("d3q19_ensemble_%dcells_edge%d-%d" % (n_cells, edge[0], edge[1]), dims, taus, cs, rs, ds, vs, drop)
