"""Addressing rules of in-place (two-phase) streaming, checked on index maps on the CPU.

The rules (stated with lbm_set_streaming in include/lbmp.h and implemented by the sweep's
in-place phases): the neighbour phase reads slot i of x - c_i (slot opp(i) of x where
x - c_i lies beyond a wall) and writes f*_i(x) into slot opp(i) of x + c_i (slot i of x where
x + c_i lies beyond a wall); the local phase reads slot opp(i) of x and writes slot i of x.
Checked here for D2Q9 and D3Q19 with periodic and walled axes:
  - every site writes exactly the locations it read (no location is written by one site and
    read by another in the same phase, so the sweep needs no second buffer);
  - the read sets of all sites partition the buffer;
  - a neighbour phase then a local phase, with an arbitrary per-site collision, give the
    populations of two pull steps with halfway bounce-back, and the layout between them
    holds the pulled values of the second pull step.
"""
import itertools

import numpy as np
import pytest

D2Q9_C = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
D3Q19_C = [(0, 0, 0)] + [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(abs(t) for t in v) in (1, 2)]


def opp_of(c):
    return [c.index(tuple(-t for t in v)) for v in c]


def shift(dims, walls, x, v, sign):
    """x + sign v with periodic wrap; None where it leaves through a wall."""
    out = []
    for k in range(3):
        t = x[k] + sign * v[k]
        if t < 0 or t >= dims[k]:
            if walls[k]:
                return None
            t %= dims[k]
        out.append(t)
    return tuple(out)


def maps(dims, walls, c):
    opp = opp_of(c)
    sites = list(itertools.product(*[range(n) for n in dims]))
    R1, W1, R2, W2 = {}, {}, {}, {}
    for x in sites:
        for i, v in enumerate(c):
            src = shift(dims, walls, x, v, -1)
            R1[x, i] = (src, i) if src is not None else (x, opp[i])
            dst = shift(dims, walls, x, v, +1)
            W1[x, i] = (dst, opp[i]) if dst is not None else (x, i)
            R2[x, i] = (x, opp[i])
            W2[x, i] = (x, i)
    return sites, opp, R1, W1, R2, W2


CASES = [
    ("d2q9_periodic", (5, 4, 1), (0, 0, 0), D2Q9_C),
    ("d2q9_walls", (5, 4, 1), (1, 1, 0), D2Q9_C),
    ("d3q19_periodic", (4, 3, 5), (0, 0, 0), D3Q19_C),
    ("d3q19_zwalls", (4, 3, 5), (0, 0, 1), D3Q19_C),
    ("d3q19_box", (4, 3, 5), (1, 1, 1), D3Q19_C),
]


@pytest.mark.parametrize("name,dims,walls,c", CASES, ids=[k[0] for k in CASES])
def test_each_site_writes_what_it_read(name, dims, walls, c):
    sites, opp, R1, W1, R2, W2 = maps(dims, walls, c)
    Q = len(c)
    everything = {(x, i) for x in sites for i in range(Q)}
    for R, W in ((R1, W1), (R2, W2)):
        for x in sites:
            reads = {R[x, i] for i in range(Q)}
            writes = {W[x, i] for i in range(Q)}
            assert len(reads) == Q and reads == writes
        assert set(R.values()) == everything and len(set(R.values())) == len(R)


@pytest.mark.parametrize("name,dims,walls,c", CASES, ids=[k[0] for k in CASES])
def test_two_phases_equal_two_pull_steps(name, dims, walls, c):
    sites, opp, R1, W1, R2, W2 = maps(dims, walls, c)
    Q = len(c)
    gen = np.random.Generator(np.random.PCG64(11))
    M = gen.standard_normal((Q, Q))

    def collide(f):  # any per-site map will do: the layout must not depend on it
        return np.tanh(M @ f) + 0.1 * f

    P0 = {x: gen.standard_normal(Q) for x in sites}        # post-collision state, natural slots

    def pull_step(P):
        pulled, out = {}, {}
        for x in sites:
            f = np.empty(Q)
            for i, v in enumerate(c):
                src = shift(dims, walls, x, v, -1)
                f[i] = P[src][i] if src is not None else P[x][opp[i]]
            pulled[x] = f
            out[x] = collide(f)
        return pulled, out

    _, P1 = pull_step(P0)
    pulled2, P2 = pull_step(P1)

    buf = {(x, i): P0[x][i] for x in sites for i in range(Q)}  # the one buffer

    def phase(R, W):
        new = {}
        for x in sites:
            f = np.array([buf[R[x, i]] for i in range(Q)])
            fs = collide(f)
            for i in range(Q):
                new[W[x, i]] = fs[i]
        assert len(new) == len(buf)
        buf.update(new)

    phase(R1, W1)
    for x in sites:  # between the phases: slot opp(i) of x holds the pulled f_i(x)
        np.testing.assert_array_equal([buf[x, opp[i]] for i in range(Q)], pulled2[x])
    phase(R2, W2)
    for x in sites:  # after the local phase: the natural layout of two pull steps
        np.testing.assert_array_equal([buf[x, i] for i in range(Q)], P2[x])
