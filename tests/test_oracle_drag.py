"""Steady Stokes drag on a square array of cylinders against Hasimoto's closed form.

A fixed disk of radius r in a periodic L x L cell (L = 8 r, solid fraction pi/64) under a
body force F on the fluid; at steady state the whole injected momentum F L^2 per step leaves
through the disk. Hasimoto (1959), square array of cylinders, small solid fraction c:
drag per unit length = 4 pi mu U / K(c), K(c) = -1/2 ln c - 0.738 + c - 0.887 c^2 + O(c^3),
U the mean velocity over the cell (superficial). Inverting K for the measured U gives the
effective hydrodynamic radius a_eff of the discrete disk; the pin is that the offset
delta = r - a_eff is the same at every resolution (within +-0.15, a lattice-boundary offset),
so the drag converges to the closed form as r grows.

The force the method itself reports for the disk (Eqs. 8-9: the momentum exchanged at the BS
sites) is systematically lower than F L^2: the IS imposition (Eq. 12) also removes the
momentum that streams from the BS layer into the IS layer, and the paper's force does not
count it. Its ratio to F L^2 is pinned here as measured (0.74-0.78), in line with the paper's
remark that its drags come out systematically lower than reference values (Sec. 3.1)."""
import math

import numpy as np
import pytest

import oracle as O


def _K(c):
    return -0.5 * math.log(c) - 0.738 + c - 0.887 * c * c


def _c_of(k):
    lo, hi = 1e-8, 0.3
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _K(mid) > k:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def steady_cylinder(make, r, tau=1.0, F=1e-6):
    """Runs a cell of edge 8 r to steady state; returns (delta, reported force / (F L^2))."""
    L = int(8 * r)
    nu = (tau - 0.5) / 3.0
    s = make(L, tau, F)
    s.add_particles(np.array([[L / 2 - 0.5, L / 2 - 0.5, 0.0]]), [r], [math.inf])
    prev = None
    for _ in range(1000):
        s.step(500)
        Fr = s.get_particles()["force"][0, 0]
        if prev is not None and abs(Fr - prev) < 1e-7 * abs(Fr):
            break
        prev = Fr
    rho, u = s.get_fields()
    fluid = s.get_tags() == 0xFFFFFFFF
    U = u[..., 0][fluid].sum() / (L * L)
    Ft = F * L * L
    a_eff = L * math.sqrt(_c_of(4.0 * math.pi * nu * U / Ft) / math.pi)
    return r - a_eff, Fr / Ft


def test_closed_form_inversion_round_trips():
    for c in (0.01, math.pi / 64, 0.1):
        assert abs(_c_of(_K(c)) - c) <= 1e-12 * max(c, 1.0)


def test_hasimoto_offset_is_resolution_independent():
    O.build()
    make = lambda L, tau, F: O.OracleSim(0, L, L, 1, tau, body_force=(F, 0.0, 0.0))
    res = [steady_cylinder(make, r) for r in (4.0, 6.0, 8.0)]
    deltas = np.array([d for d, _ in res])
    ratios = np.array([q for _, q in res])
    print("delta", deltas, "reported / total", ratios)
    assert np.all((deltas > 0.0) & (deltas < 1.0))          # a_eff within one site below r
    assert deltas.max() - deltas.min() <= 0.3                # stable within +-0.15
    assert np.all((ratios > 0.70) & (ratios < 0.80))         # systematically lower (Sec. 3.1)
