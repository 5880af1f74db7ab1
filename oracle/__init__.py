"""FP64 CPU oracle of the site-based particle-suspension LBM (arXiv:1105.2904).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow reference the CUDA path is
checked against. Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference legs may import it; the product package never does.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only builds it with gcc and marshals numpy arrays.
The step it implements, and the readings of the paper it takes, are listed at the top
of ``lbm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_SO_OMP = os.path.join(_BUILD, "liblbm_oracle_omp.so")
_LOCK = threading.Lock()
_LIB = None
_LIB_OMP = None

D2Q9 = 0
D3Q19 = 1

CLS_IS, CLS_BS, CLS_IN = 0, 1, 2
TAG_FLUID = 0xFFFFFFFF


def build(force: bool = False, openmp: bool = False) -> str:
    """Compiles the oracle into ``oracle/_build/liblbm_oracle.so`` (gcc, FP64, one thread).

    openmp=True builds ``liblbm_oracle_omp.so`` from the same source with ``-fopenmp``: the
    collision and propagation loops are split between threads, each site's arithmetic is
    unchanged, so the results are identical to the single-threaded build (a CPU test checks
    that). It serves the timed all-core CPU baseline and long parity runs on large boxes.
    """
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_OMP if openmp else _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h"))
    ):
        return so
    tmp = so + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-Wall",
           "-shared", "-fPIC"] + (["-fopenmp"] if openmp else ["-Wno-unknown-pragmas"]) + [_SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def _lib(openmp: bool = False):
    global _LIB, _LIB_OMP
    with _LOCK:
        if (_LIB_OMP if openmp else _LIB) is None:
            lib = ctypes.CDLL(build(openmp=openmp))
            P = ctypes.c_void_p
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            U = ctypes.POINTER(ctypes.c_uint)
            lib.osim_create.restype = P
            lib.osim_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, D]
            lib.osim_destroy.argtypes = [P]
            lib.osim_set_walls.argtypes = [P, I]
            lib.osim_set_particle_options.argtypes = [P, D, ctypes.c_double, ctypes.c_int]
            lib.osim_set_wall_velocity.argtypes = [P, ctypes.c_int, D]
            lib.osim_set_equilibrium_face.argtypes = [P, ctypes.c_int, D]
            lib.osim_add_particles.argtypes = [P, ctypes.c_int, D, D, D, D, D]
            lib.osim_step.argtypes = [P, ctypes.c_int]
            lib.osim_get_f.argtypes = [P, D]
            lib.osim_set_f.argtypes = [P, D]
            lib.osim_get_fields.argtypes = [P, D, D]
            lib.osim_get_particles.argtypes = [P, D, D, D, D, D]
            lib.osim_get_tags.argtypes = [P, U]
            lib.osim_get_orientations.argtypes = [P, D]
            lib.osim_get_diagnostics.argtypes = [P, D]
            lib.osim_num_particles.argtypes = [P]
            lib.osim_get_template.argtypes = [P, ctypes.c_int, I]
            lib.osim_resolve_contacts.argtypes = [P, D]
            lib.osim_collide_site.argtypes = [P, D, D]
            if openmp:
                _LIB_OMP = lib
            else:
                _LIB = lib
    return _LIB_OMP if openmp else _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleSim:
    """One FP64 CPU simulation (lattice 0 = D2Q9 with nz = 1, 1 = D3Q19)."""

    def __init__(self, lattice, nx, ny, nz, tau, body_force=(0.0, 0.0, 0.0),
                 walls=(0, 0, 0), gravity=(0.0, 0.0, 0.0), gap=0.0, body_force_on_particles=False,
                 wall_velocity=None, equilibrium_faces=None, openmp=False):
        """openmp: use the OpenMP build (same arithmetic, identical results, all cores;
        thread count from OMP_NUM_THREADS)."""
        self.lib = _lib(openmp)
        self.lattice = lattice
        self.Q = 9 if lattice == D2Q9 else 19
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        F = _f64(body_force, (3,))
        self.h = self.lib.osim_create(lattice, nx, ny, nz, float(tau), _dp(F))
        if not self.h:
            raise ValueError("oracle: invalid lattice arguments")
        w = np.ascontiguousarray(walls, dtype=np.int32)
        if self.lib.osim_set_walls(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int))) != 0:
            raise ValueError("oracle: walls must be set before particles")
        g = _f64(gravity, (3,))
        self.lib.osim_set_particle_options(self.h, _dp(g), float(gap), int(bool(body_force_on_particles)))
        for face, u in (equilibrium_faces or {}).items():
            uu = _f64(u, (3,))
            if self.lib.osim_set_equilibrium_face(self.h, int(face), _dp(uu)) != 0:
                raise ValueError("oracle: face %d is not on a walled axis" % face)
        for face, u in (wall_velocity or {}).items():
            self.set_wall_velocity(face, u)

    def set_wall_velocity(self, face, u):
        uu = _f64(u, (3,))
        if self.lib.osim_set_wall_velocity(self.h, int(face), _dp(uu)) != 0:
            raise ValueError("oracle: face %d is not a wall, or the velocity is not tangential" % face)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.osim_destroy(h)
            self.h = None

    def add_particles(self, centers, radii, densities, velocities=None, omegas=None):
        c = _f64(centers).reshape(-1, 3)
        n = c.shape[0]
        r = _f64(radii, (n,))
        d = _f64(densities, (n,))
        v = None if velocities is None else _f64(velocities).reshape(n, 3)
        o = None if omegas is None else _f64(omegas).reshape(n, 3)
        rc = self.lib.osim_add_particles(self.h, n, _dp(c), _dp(r), _dp(d),
                                         None if v is None else _dp(v),
                                         None if o is None else _dp(o))
        if rc != 0:
            raise ValueError("oracle: add_particles rejected the input (code %d)" % rc)

    def step(self, n=1):
        self.lib.osim_step(self.h, int(n))

    def get_f(self):
        f = np.empty((self.Q,) + self.shape, dtype=np.float64)
        self.lib.osim_get_f(self.h, _dp(f))
        return f

    def set_f(self, f):
        f = _f64(f, (self.Q,) + self.shape)
        self.lib.osim_set_f(self.h, _dp(f))

    def get_fields(self):
        rho = np.empty(self.shape, dtype=np.float64)
        u = np.empty(self.shape + (3,), dtype=np.float64)
        self.lib.osim_get_fields(self.h, _dp(rho), _dp(u))
        return rho, u

    @property
    def num_particles(self):
        return self.lib.osim_num_particles(self.h)

    def get_particles(self):
        n = self.num_particles
        out = [np.zeros((n, 3), dtype=np.float64) for _ in range(5)]
        self.lib.osim_get_particles(self.h, *[_dp(a) for a in out])
        return dict(zip(("x", "u", "omega", "force", "torque"), out))

    def get_orientations(self):
        q = np.zeros((self.num_particles, 4), dtype=np.float64)
        if len(q):
            self.lib.osim_get_orientations(self.h, _dp(q))
        return q

    def get_tags(self):
        t = np.empty(self.shape, dtype=np.uint32)
        self.lib.osim_get_tags(self.h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)))
        return t

    def get_diagnostics(self):
        d = np.zeros(6, dtype=np.float64)
        self.lib.osim_get_diagnostics(self.h, _dp(d))
        return {"dP_B": d[:3].copy(), "dP_IS": d[3:].copy()}

    def get_template(self, p):
        n = self.lib.osim_get_template(self.h, int(p), None)
        if n < 0:
            raise IndexError(p)
        t = np.zeros((max(n, 1), 4), dtype=np.int32)
        self.lib.osim_get_template(self.h, int(p), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return t[:n]

    def resolve_contacts(self, u):
        u = _f64(u).reshape(-1, 3).copy()
        self.lib.osim_resolve_contacts(self.h, _dp(u))
        return u

    def collide_site(self, fin):
        fin = _f64(fin, (self.Q,))
        fout = np.empty(self.Q, dtype=np.float64)
        self.lib.osim_collide_site(self.h, _dp(fin), _dp(fout))
        return fout


def lattice_tables(lattice):
    """Velocity set and weights in the order the oracle and the C-ABI use (D2Q9 per Fig. 1)."""
    if lattice == D2Q9:
        c = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0],
                      [1, 1, 0], [-1, 1, 0], [-1, -1, 0], [1, -1, 0]], dtype=np.int64)
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    else:
        c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                      [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
                      [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.int64)
        w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    return c, w
