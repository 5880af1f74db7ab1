"""Learned drag / torque closure for coarse-resolution particles (not in the paper).

A coarse run resolves each sphere with radius r_c = 3 lattice units; a fine run of the same
configuration uses radius 12 (a factor f = 4 finer lattice). With the same relaxation time in
both, diffusive scaling makes them the same physical problem: the fine run takes f^2 steps
per coarse step, its body-force acceleration is f^-3 of the coarse one, and forces in lattice
units agree while torques carry a factor f (force unit rho dx^4 / dt^2, torque unit
rho dx^5 / dt^2). A network trained on pairs of such runs predicts, from moments of the
coarse flow around a sphere, the difference between the fine and the coarse force and
torque. The coarse method without the network stays the fallback, and the fine method the
judge of the error.

The inputs are the stencil moments (rho - 1, u - u_p) / U on an n_side^3 stencil around the
particle and the fractional lattice offset of its reference centre, which together with the
radius fixes the particle's discrete site set (a radius-3 sphere's site count and shape vary
strongly with it). Inputs are centred on the training set's means and scaled by one common
spread for all moments (stencil nodes inside the sphere vary little; scaling each to unit
spread would amplify their noise) and by their own spread for the three offsets; targets
are standardised per output.

Everything here is orchestration over the C-ABI: the runs, the inputs
(lbm_closure_features), the training and the inference (lbm_mlp_*) run in the library's
kernels; torch only holds device memory.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import lbmp
from . import workloads as W

N_SIDE = 4
SIZES = [4 * N_SIDE ** 3 + 3, 128, 128, 6]


@dataclass
class PairSpec:
    """Coarse periodic cells of edge L with n fixed spheres of radius r driven by a body
    force along x, observed after `steps` coarse steps; the fine twin is `factor` times
    finer."""

    L: int = 32
    n_spheres: int = 8
    r: float = 3.0
    tau: float = 1.0
    accel: float = 1e-5
    steps: int = 200
    factor: int = 4
    min_gap: float = 2.0
    n_side: int = N_SIDE
    spacing: float = 4.0     # stencil node spacing (coarse lattice units)
    precision: str = "fp32"


def place(spec: PairSpec, n_cells: int, seed: int):
    """Seeded sphere centres (random sequential addition, periodic, surface gap >= min_gap)."""
    out = []
    for k in range(n_cells):
        g = W.rng(seed * 7919 + k)
        c, r, dropped = W._place_spheres((spec.L,) * 3, np.full(spec.n_spheres, spec.r), g, spec.min_gap)
        out.append(c)
    return out


def _run(spec: PairSpec, centers, fine: bool):
    f = spec.factor if fine else 1
    L = spec.L * f
    n = len(centers)
    b = lbmp.Batch(1, [(L, L, L)] * n, [spec.tau] * n, [(spec.accel / f ** 3, 0.0, 0.0)] * n,
                   precision=spec.precision)
    for k, c in enumerate(centers):
        cc = c * f + 0.5 * (f - 1) if fine else c
        b.add_particles(k, cc, np.full(len(c), spec.r * f), np.full(len(c), np.inf))
    b.set_tuning(steps_per_graph=50)
    b.step(spec.steps * f * f)
    b.synchronize()
    return b


def generate(spec: PairSpec, n_cells: int, seed: int, max_sites: int = 600_000_000):
    """One set of coarse / fine pairs. Returns (inputs [N, 4 n_side^3 + 3] CUDA tensor,
    targets [N, 6], coarse [N, 6], fine [N, 6], scale [N, 2]) with N = spheres of all cells;
    force rows are (Fx, Fy, Fz, Tx, Ty, Tz), the fine torque already scaled to coarse units;
    targets are (fine - coarse) divided by the Stokes scales 6 pi nu r U and 6 pi nu r^2 U,
    U the cell's mean fluid velocity along x (scale holds both). The runs go in batches of at
    most max_sites lattice sites (a 512^3 fine cell holds ~26 GB)."""
    import torch

    centers = place(spec, n_cells, seed)
    nu = (spec.tau - 0.5) / 3.0

    def chunks(fine):
        per = max(1, int(max_sites // (spec.L * (spec.factor if fine else 1)) ** 3))
        return [list(range(i, min(n_cells, i + per))) for i in range(0, n_cells, per)]

    feats, coarse, scales = [], [], []
    for ks in chunks(False):
        bc = _run(spec, [centers[k] for k in ks], fine=False)
        for j, k in enumerate(ks):
            cell = bc.cell(j)
            rho, u = cell.get_fields()
            tags = cell.get_tags()
            U = float(u[..., 0][tags == 0xFFFFFFFF].mean())
            feats.append(cell.closure_features(spec.n_side, spec.spacing, U))
            p = cell.get_particles()
            coarse.append(np.concatenate([p["force"], p["torque"]], axis=1))
            s_f = 6.0 * math.pi * nu * spec.r * U
            scales.append(np.tile([s_f, s_f * spec.r], (len(centers[k]), 1)))
        bc.close()
    fine = []
    for ks in chunks(True):
        bf = _run(spec, [centers[k] for k in ks], fine=True)
        for j, k in enumerate(ks):
            p = bf.cell(j).get_particles()
            fine.append(np.concatenate([p["force"], p["torque"] / spec.factor], axis=1))
        bf.close()
    X = torch.cat(feats, 0)
    coarse = np.concatenate(coarse, 0)
    fine = np.concatenate(fine, 0)
    scale = np.concatenate(scales, 0)
    S = np.repeat(scale, 3, axis=1)
    T = (fine - coarse) / S
    return X, T, coarse, fine, scale


class Closure:
    """The trained network with its output normalisation."""

    def __init__(self, sizes=SIZES, seed=0):
        self.sizes = list(sizes)
        self.net = lbmp.MLP(self.sizes)
        self.net.set_params(_he_init(self.sizes, seed))
        self.mu = np.zeros(self.sizes[-1])
        self.sd = np.ones(self.sizes[-1])

    def close(self):
        self.net.close()

    def fit(self, X, T, epochs=200, batch=128, lr=5e-4, seed=0):
        """Trains on inputs X (CUDA tensor) and targets T (numpy [N, 6]), scaled with the
        training set's statistics (module docstring). Returns the per-epoch losses."""
        import torch

        Xh = X.double().cpu().numpy()
        nm = Xh.shape[1] - 3
        spread = np.empty(Xh.shape[1])
        spread[:nm] = Xh[:, :nm].std()
        spread[nm:] = Xh[:, nm:].std(0)
        self.net.set_input_scaling(Xh.mean(0), 1.0 / np.where(spread > 0, spread, 1.0))
        self.mu = T.mean(0)
        self.sd = T.std(0) + 1e-12
        Tn = torch.tensor((T - self.mu) / self.sd, dtype=torch.float32, device=X.device)
        return self.net.train(X, Tn, batch=batch, epochs=epochs, lr=lr, seed=seed)

    def predict(self, X):
        """Predicted targets (denormalised), numpy [N, 6]."""
        return self.net.forward(X).cpu().double().numpy() * self.sd + self.mu

    def corrected(self, X, coarse, scale):
        """Coarse force and torque plus the predicted correction."""
        return coarse + self.predict(X) * np.repeat(scale, 3, axis=1)


def _he_init(sizes, seed):
    g = W.rng(seed)
    out = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        bound = math.sqrt(6.0 / a)
        out.append([g.uniform(-bound, bound, size=(b, a)), np.zeros(b)])
    return out


def drag_errors(pred, fine):
    """Relative error of the drag (x force) against the fine method."""
    return np.abs(pred[:, 0] - fine[:, 0]) / np.abs(fine[:, 0])
