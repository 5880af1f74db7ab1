"""Thin ctypes binding of the C-ABI in ``include/lbmp.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls. ``Simulation`` bundles a
context handle with numpy-returning getters; it adds no arithmetic of its own. The
library must have been built (``paper_1105_2904_gb300.build.build()``); loading fails
loudly otherwise, and every call raises ``LbmError`` on a non-OK status.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBMP_DEBUG=1 selects the bounds-checked build (build.build(debug=True)).
LIB_PATH = os.path.join(_PKG, "_lib_debug" if os.environ.get("LBMP_DEBUG") == "1" else "_lib", "liblbmp.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", 1: "LBM_E_INVALID", 2: "LBM_E_OOM", 3: "LBM_E_CUDA", 4: "LBM_E_OVERLAP",
          5: "LBM_E_TIMEOUT", 6: "LBM_E_STATE", 7: "LBM_E_NAN", 8: "LBM_E_CAPACITY", 9: "LBM_E_UNSTABLE",
          10: "LBM_E_BOUNDS"}
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16DEV, LBM_BF16DEV = 0, 1, 2, 3
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP16DEV, "bf16": LBM_BF16DEV}
LBM_PERIODIC, LBM_NOSLIP, LBM_EQUILIBRIUM = 0, 1, 2
LBM_STREAM_PULL, LBM_STREAM_INPLACE = 0, 1
STREAMING = {"pull": LBM_STREAM_PULL, "inplace": LBM_STREAM_INPLACE}

EXPORTED = ("lbm_create", "lbm_configure", "lbm_set_wall_velocity", "lbm_add_particles", "lbm_step", "lbm_synchronize",
            "lbm_get_fields", "lbm_get_particles", "lbm_get_orientations", "lbm_get_distributions",
            "lbm_set_distributions",
            "lbm_get_masks", "lbm_get_info", "lbm_profile_steps", "lbm_set_sweep_shape", "lbm_set_streaming", "lbm_diagnostics",
            "lbm_bs_exchange_noalloc",
            "lbm_checkpoint_size", "lbm_checkpoint_save", "lbm_checkpoint_load", "lbm_get_particles_async",
            "lbm_wait_particles",
            "lbm_last_error", "lbm_destroy",
            "lbm_batch_create", "lbm_batch_add_particles", "lbm_batch_cell", "lbm_batch_set_tuning",
            "lbm_batch_step", "lbm_batch_synchronize", "lbm_batch_profile_steps", "lbm_batch_get_info",
            "lbm_batch_stream", "lbm_schedule_tiles", "lbm_batch_last_error", "lbm_batch_destroy",
            "lbm_closure_features",
            "lbm_mlp_create", "lbm_mlp_num_params", "lbm_mlp_set_params", "lbm_mlp_set_input_scaling",
            "lbm_mlp_get_params", "lbm_mlp_forward",
            "lbm_mlp_loss_grad", "lbm_mlp_adam_step", "lbm_mlp_train", "lbm_mlp_last_error", "lbm_mlp_destroy")
# entry points whose return value is not an lbm_status
_NOT_STATUS = ("lbm_last_error", "lbm_destroy", "lbm_batch_cell", "lbm_batch_stream", "lbm_schedule_tiles",
               "lbm_batch_last_error", "lbm_batch_destroy", "lbm_mlp_num_params", "lbm_mlp_last_error",
               "lbm_mlp_destroy")


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))


_lib = None


def load(path: str = LIB_PATH):
    """Loads liblbmp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblbmp.so not found at %s: build it with paper_1105_2904_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    i32 = ctypes.c_int
    lib.lbm_create.argtypes = [ctypes.POINTER(P), i32, i32, i32, i32, ctypes.c_double, D]
    lib.lbm_configure.argtypes = [P, i32, I, D, ctypes.c_double, i32, P]
    lib.lbm_set_wall_velocity.argtypes = [P, i32, D]
    lib.lbm_add_particles.argtypes = [P, i32, D, D, D, D, D, I]
    lib.lbm_step.argtypes = [P, i32]
    lib.lbm_synchronize.argtypes = [P]
    lib.lbm_get_fields.argtypes = [P, D, D]
    lib.lbm_get_particles.argtypes = [P, D, D, D, D, D]
    lib.lbm_get_orientations.argtypes = [P, D]
    lib.lbm_get_distributions.argtypes = [P, D]
    lib.lbm_set_distributions.argtypes = [P, D]
    lib.lbm_get_masks.argtypes = [P, ctypes.POINTER(ctypes.c_uint)]
    lib.lbm_get_info.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.lbm_profile_steps.argtypes = [P, i32, D]
    lib.lbm_set_sweep_shape.argtypes = [P, i32]
    lib.lbm_set_streaming.argtypes = [P, i32]
    lib.lbm_diagnostics.argtypes = [P, D]
    lib.lbm_get_particles_async.argtypes = [P, P, ctypes.POINTER(ctypes.c_longlong)]
    lib.lbm_wait_particles.argtypes = [P, ctypes.c_longlong]
    lib.lbm_checkpoint_size.argtypes = [P, ctypes.POINTER(ctypes.c_ulonglong)]
    lib.lbm_checkpoint_save.argtypes = [P, P, ctypes.c_ulonglong]
    lib.lbm_checkpoint_load.argtypes = [P, P, ctypes.c_ulonglong]
    lib.lbm_bs_exchange_noalloc.argtypes = [i32, i32, i32, i32, I, D, P, P, i32, P, P, P, P, P, P]
    lib.lbm_last_error.argtypes = [P]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_destroy.argtypes = [P]
    lib.lbm_batch_create.argtypes = [ctypes.POINTER(P), i32, i32, I, D, D, i32, I, D, ctypes.c_double, i32]
    lib.lbm_batch_add_particles.argtypes = [P, i32, i32, D, D, D, D, D]
    lib.lbm_batch_cell.argtypes = [P, i32]
    lib.lbm_batch_cell.restype = P
    lib.lbm_batch_set_tuning.argtypes = [P, I, i32, i32, i32]
    lib.lbm_batch_step.argtypes = [P, i32]
    lib.lbm_batch_synchronize.argtypes = [P]
    lib.lbm_batch_profile_steps.argtypes = [P, i32, D]
    lib.lbm_batch_get_info.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.lbm_batch_stream.argtypes = [P]
    lib.lbm_batch_stream.restype = P
    lib.lbm_schedule_tiles.argtypes = [i32, I, I, i32, I]
    lib.lbm_schedule_tiles.restype = ctypes.c_longlong
    lib.lbm_batch_last_error.argtypes = [P]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    lib.lbm_batch_destroy.argtypes = [P]
    lib.lbm_batch_destroy.restype = None
    lib.lbm_closure_features.argtypes = [P, i32, ctypes.c_double, ctypes.c_double, P]
    lib.lbm_mlp_create.argtypes = [ctypes.POINTER(P), i32, I, P]
    lib.lbm_mlp_num_params.argtypes = [P]
    lib.lbm_mlp_num_params.restype = ctypes.c_longlong
    lib.lbm_mlp_set_params.argtypes = [P, D]
    lib.lbm_mlp_get_params.argtypes = [P, D, D]
    lib.lbm_mlp_set_input_scaling.argtypes = [P, D, D]
    lib.lbm_mlp_forward.argtypes = [P, P, i32, P]
    lib.lbm_mlp_loss_grad.argtypes = [P, P, P, i32, D]
    lib.lbm_mlp_adam_step.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.lbm_mlp_train.argtypes = [P, P, P, i32, i32, i32, ctypes.c_double, ctypes.c_uint, D]
    lib.lbm_mlp_last_error.argtypes = [P]
    lib.lbm_mlp_last_error.restype = ctypes.c_char_p
    lib.lbm_mlp_destroy.argtypes = [P]
    lib.lbm_mlp_destroy.restype = None
    for name in EXPORTED:
        if name not in _NOT_STATUS:
            getattr(lib, name).restype = ctypes.c_int
    lib.lbm_destroy.restype = None
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if n is None else a.reshape(n)


def _check(h, status):
    if status != LBM_OK:
        msg = load().lbm_last_error(h) if h else b"(no context)"
        raise LbmError(status, msg.decode(errors="replace") if msg else "")


# ---- same-name wrappers ------------------------------------------------------------------

def lbm_create(lattice, nx, ny, nz, tau, body_force=None):
    lib = load()
    h = ctypes.c_void_p()
    F = _f64(body_force, 3)
    st = lib.lbm_create(ctypes.byref(h), int(lattice), int(nx), int(ny), int(nz), float(tau), _dp(F))
    if st != LBM_OK:
        raise LbmError(st, "lbm_create(%d, %d, %d, %d, %g)" % (lattice, nx, ny, nz, tau))
    return h


def lbm_configure(h, precision, faces=None, particle_gravity=None, contact_gap=0.0,
                  body_force_on_particles=False, cuda_stream=None):
    lib = load()
    fa = None if faces is None else np.ascontiguousarray(faces, dtype=np.int32).reshape(6)
    g = _f64(particle_gravity, 3)
    _check(h, lib.lbm_configure(h, int(precision),
                                None if fa is None else fa.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                _dp(g), float(contact_gap), int(bool(body_force_on_particles)),
                                ctypes.c_void_p(cuda_stream) if cuda_stream else None))


def lbm_set_wall_velocity(h, face, u):
    u = _f64(u, 3)
    _check(h, load().lbm_set_wall_velocity(h, int(face), _dp(u)))


def lbm_add_particles(h, centers, radii, densities, velocities=None, omegas=None):
    lib = load()
    c = _f64(centers).reshape(-1, 3)
    n = c.shape[0]
    r = _f64(radii, n)
    d = _f64(densities, n)
    v = None if velocities is None else _f64(velocities).reshape(n, 3)
    o = None if omegas is None else _f64(omegas).reshape(n, 3)
    first = ctypes.c_int(-1)
    _check(h, lib.lbm_add_particles(h, n, _dp(c), _dp(r), _dp(d), _dp(v), _dp(o), ctypes.byref(first)))
    return first.value


def lbm_step(h, n=1):
    _check(h, load().lbm_step(h, int(n)))


def lbm_synchronize(h):
    _check(h, load().lbm_synchronize(h))


def lbm_get_fields(h, N, rho=None, u=None):
    rho = np.empty(N) if rho is None else rho
    u = np.empty((N, 3)) if u is None else u
    _check(h, load().lbm_get_fields(h, _dp(rho), _dp(u)))
    return rho, u


def lbm_get_particles(h, n, out=None):
    out = out or {k: np.empty((n, 3)) for k in ("x", "u", "omega", "force", "torque")}
    _check(h, load().lbm_get_particles(h, _dp(out["x"]), _dp(out["u"]), _dp(out["omega"]),
                                       _dp(out["force"]), _dp(out["torque"])))
    return out


def lbm_get_orientations(h, n, out=None):
    out = np.empty((n, 4)) if out is None else out
    _check(h, load().lbm_get_orientations(h, _dp(out)))
    return out


def lbm_get_particles_async(h, dst_ptr):
    """Enqueues a read-back of the particle state into page-locked host memory at dst_ptr
    (15 np + 1 doubles); returns its ticket."""
    t = ctypes.c_longlong()
    _check(h, load().lbm_get_particles_async(h, ctypes.c_void_p(dst_ptr), ctypes.byref(t)))
    return t.value


def lbm_wait_particles(h, ticket):
    _check(h, load().lbm_wait_particles(h, int(ticket)))


def unpack_particles(buf, n):
    """Views of a read-back buffer (numpy float64, 15 n + 1 values) as the five [n][3] arrays."""
    keys = ("x", "u", "omega", "force", "torque")
    return {k: buf[3 * n * i:3 * n * (i + 1)].reshape(n, 3) for i, k in enumerate(keys)}


def lbm_get_distributions(h, Q, N, f=None):
    f = np.empty((Q, N)) if f is None else f
    _check(h, load().lbm_get_distributions(h, _dp(f)))
    return f


def lbm_set_distributions(h, f):
    f = _f64(f)
    _check(h, load().lbm_set_distributions(h, _dp(f)))


def lbm_get_masks(h, N):
    t = np.empty(N, dtype=np.uint32)
    _check(h, load().lbm_get_masks(h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint))))
    return t


def lbm_get_info(h):
    out = (ctypes.c_longlong * 6)()
    _check(h, load().lbm_get_info(h, out))
    keys = ("particles", "steps", "launches_per_step", "device_bytes", "bytes_per_site", "precision")
    return dict(zip(keys, list(out)))


def lbm_profile_steps(h, n):
    out = np.zeros(3)
    _check(h, load().lbm_profile_steps(h, int(n), _dp(out)))
    return {"sweep_ms": float(out[0]), "particle_ms": float(out[1]), "step_ms": float(out[2])}


def lbm_checkpoint_save(h):
    """The context's state at the current step boundary as a numpy uint8 array."""
    n = ctypes.c_ulonglong()
    _check(h, load().lbm_checkpoint_size(h, ctypes.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(h, load().lbm_checkpoint_save(h, buf.ctypes.data_as(ctypes.c_void_p), n.value))
    return buf


def lbm_checkpoint_load(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(h, load().lbm_checkpoint_load(h, buf.ctypes.data_as(ctypes.c_void_p), buf.size))


def lbm_set_sweep_shape(h, threads_x):
    _check(h, load().lbm_set_sweep_shape(h, int(threads_x)))


def lbm_set_streaming(h, mode):
    _check(h, load().lbm_set_streaming(h, int(mode)))


def lbm_diagnostics(h):
    """Totals and extremes of the state (lbm_diagnostics); raises LbmError(LBM_E_NAN) when some
    site's moments are not finite, with the values in the exception's ``diagnostics``."""
    out = np.zeros(7)
    st = load().lbm_diagnostics(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    d = {"mass": out[0], "momentum": out[1:4].copy(), "max_speed": out[4], "mach": out[5],
         "nonfinite_sites": int(out[6])}
    try:
        _check(h, st)
    except LbmError as e:
        e.diagnostics = d
        raise
    return d


def lbm_bs_exchange_noalloc(lattice, nx, ny, nz, walls, body_force, g_ptr, tags_ptr, n, centers_ptr,
                            velocities_ptr, omegas_ptr, force_ptr, torque_ptr, cuda_stream=None):
    """Allocation-free boundary-site momentum exchange on caller-owned device buffers
    (integer device addresses, e.g. torch ``data_ptr()``); see include/lbmp.h."""
    wa = None if walls is None else np.ascontiguousarray(walls, dtype=np.int32).reshape(3)
    F = _f64(body_force, 3)
    st = load().lbm_bs_exchange_noalloc(
        int(lattice), int(nx), int(ny), int(nz),
        None if wa is None else wa.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(F),
        ctypes.c_void_p(g_ptr), ctypes.c_void_p(tags_ptr), int(n), ctypes.c_void_p(centers_ptr),
        ctypes.c_void_p(velocities_ptr), ctypes.c_void_p(omegas_ptr), ctypes.c_void_p(force_ptr),
        ctypes.c_void_p(torque_ptr), ctypes.c_void_p(cuda_stream) if cuda_stream else None)
    if st != LBM_OK:
        raise LbmError(st, "lbm_bs_exchange_noalloc(n=%d)" % n)


def lbm_last_error(h):
    m = load().lbm_last_error(h)
    return m.decode(errors="replace") if m else ""


def lbm_destroy(h):
    if h:
        load().lbm_destroy(h)


def _ip(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _bcheck(b, status):
    if status != LBM_OK:
        msg = load().lbm_batch_last_error(b) if b else b"(no batch)"
        raise LbmError(status, msg.decode(errors="replace") if msg else "")


def lbm_batch_create(lattice, dims, taus, body_forces=None, precision=LBM_FP32, faces=None, particle_gravity=None,
                     contact_gap=0.0, body_force_on_particles=False):
    lib = load()
    d = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
    n = d.shape[0]
    t = _f64(taus, n)
    F = None if body_forces is None else _f64(body_forces).reshape(n, 3)
    fa = None if faces is None else np.ascontiguousarray(faces, dtype=np.int32).reshape(6)
    g = _f64(particle_gravity, 3)
    h = ctypes.c_void_p()
    st = lib.lbm_batch_create(ctypes.byref(h), int(lattice), n, _ip(d), _dp(t), _dp(F), int(precision), _ip(fa), _dp(g),
                              float(contact_gap), int(bool(body_force_on_particles)))
    if st != LBM_OK:
        raise LbmError(st, "lbm_batch_create(%d cells)" % n)
    return h


def lbm_batch_add_particles(b, cell, centers, radii, densities, velocities=None, omegas=None):
    c = _f64(centers).reshape(-1, 3)
    n = c.shape[0]
    r = _f64(radii, n)
    d = _f64(densities, n)
    v = None if velocities is None else _f64(velocities).reshape(n, 3)
    o = None if omegas is None else _f64(omegas).reshape(n, 3)
    _bcheck(b, load().lbm_batch_add_particles(b, int(cell), n, _dp(c), _dp(r), _dp(d), _dp(v), _dp(o)))


def lbm_batch_cell(b, cell):
    h = load().lbm_batch_cell(b, int(cell))
    if not h:
        raise IndexError(cell)
    return ctypes.c_void_p(h)


def lbm_batch_set_tuning(b, tile_width=None, order=0, grid=0, steps_per_graph=1):
    tw = None if tile_width is None else np.ascontiguousarray(tile_width, dtype=np.int32)
    _bcheck(b, load().lbm_batch_set_tuning(b, _ip(tw), int(order), int(grid), int(steps_per_graph)))


def lbm_batch_step(b, n=1):
    _bcheck(b, load().lbm_batch_step(b, int(n)))


def lbm_batch_synchronize(b):
    _bcheck(b, load().lbm_batch_synchronize(b))


def lbm_batch_profile_steps(b, n):
    out = np.zeros(3)
    _bcheck(b, load().lbm_batch_profile_steps(b, int(n), _dp(out)))
    return {"sweep_ms": float(out[0]), "particle_ms": float(out[1]), "step_ms": float(out[2])}


def lbm_batch_get_info(b):
    out = (ctypes.c_longlong * 5)()
    _bcheck(b, load().lbm_batch_get_info(b, out))
    return dict(zip(("cells", "sites", "particles", "tiles", "launches_per_step"), list(out)))


def lbm_batch_stream(b):
    return load().lbm_batch_stream(b)


def lbm_schedule_tiles(dims, tile_width=None, order=0):
    """Sweep schedule of a batch (host-only): int32 array [tiles, 4] of (cell, x0,
    y0 | log2(width) << 16, z) in launch order."""
    d = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
    tw = None if tile_width is None else np.ascontiguousarray(tile_width, dtype=np.int32)
    lib = load()
    n = lib.lbm_schedule_tiles(d.shape[0], _ip(d), _ip(tw), int(order), None)
    if n < 0:
        raise ValueError("lbm_schedule_tiles: bad argument")
    out = np.zeros((n, 4), dtype=np.int32)
    lib.lbm_schedule_tiles(d.shape[0], _ip(d), _ip(tw), int(order), _ip(out))
    return out


def lbm_batch_last_error(b):
    m = load().lbm_batch_last_error(b)
    return m.decode(errors="replace") if m else ""


def lbm_batch_destroy(b):
    if b:
        load().lbm_batch_destroy(b)


class Simulation:
    """A context handle plus numpy-shaped getters (lattice 0 = D2Q9, 1 = D3Q19)."""

    @classmethod
    def borrowed(cls, handle, lattice, nx, ny, nz, np_):
        """A view of a context owned elsewhere (a cell of a Batch): never destroyed here."""
        s = cls.__new__(cls)
        s.lattice = lattice
        s.Q = 9 if lattice == LBM_D2Q9 else 19
        s.shape = (nz, ny, nx)
        s.N = nx * ny * nz
        s.h = handle
        s.np = np_
        s._owned = False
        return s

    def __init__(self, lattice, nx, ny, nz, tau, body_force=(0.0, 0.0, 0.0), precision="fp32",
                 walls=(0, 0, 0), gravity=(0.0, 0.0, 0.0), gap=0.0, body_force_on_particles=False,
                 cuda_stream=None, wall_velocity=None, equilibrium_faces=None, streaming="pull"):
        """walls[k]: no-slip walls at both ends of axis k; equilibrium_faces: {face: velocity}
        for faces (0..5 = -x,+x,-y,+y,-z,+z) that impose their velocity by equilibrium
        (LBM_EQUILIBRIUM; their axis is walled); wall_velocity: {face: velocity} of no-slip
        faces moving in their plane; streaming: "pull" (two buffers) or "inplace" (one
        buffer, lbm_set_streaming)."""
        if isinstance(precision, str) and precision not in PRECISIONS:
            raise ValueError("precision must be one of %s, not %r" % (sorted(PRECISIONS), precision))
        if isinstance(streaming, str) and streaming not in STREAMING:
            raise ValueError("streaming must be one of %s, not %r" % (sorted(STREAMING), streaming))
        self.lattice = lattice
        self.Q = 9 if lattice == LBM_D2Q9 else 19
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.h = lbm_create(lattice, nx, ny, nz, tau, body_force)
        eq = equilibrium_faces or {}
        faces = []
        for f in range(6):
            walled = walls[f // 2] or (2 * (f // 2)) in eq or (2 * (f // 2) + 1) in eq
            faces.append(LBM_EQUILIBRIUM if f in eq else (LBM_NOSLIP if walled else LBM_PERIODIC))
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        try:
            lbm_configure(self.h, prec, faces, gravity, gap, body_force_on_particles, cuda_stream)
            lbm_set_streaming(self.h, STREAMING[streaming] if isinstance(streaming, str) else int(streaming))
            for face, u in eq.items():
                lbm_set_wall_velocity(self.h, face, u)
            for face, u in (wall_velocity or {}).items():
                lbm_set_wall_velocity(self.h, face, u)
        except Exception:
            lbm_destroy(self.h)
            self.h = None
            raise
        self.np = 0
        self._owned = True

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_wall_velocity(self, face, u):
        lbm_set_wall_velocity(self.h, face, u)

    def add_particles(self, centers, radii, densities, velocities=None, omegas=None):
        first = lbm_add_particles(self.h, centers, radii, densities, velocities, omegas)
        self.np = lbm_get_info(self.h)["particles"]
        return first

    def step(self, n=1):
        lbm_step(self.h, n)

    def synchronize(self):
        lbm_synchronize(self.h)

    def get_fields(self):
        rho, u = lbm_get_fields(self.h, self.N)
        return rho.reshape(self.shape), u.reshape(self.shape + (3,))

    def get_particles(self):
        return lbm_get_particles(self.h, self.np)

    def get_orientations(self):
        """[np][4] unit quaternions (w, x, y, z) of the particles' attitudes (lbm_get_orientations)."""
        return lbm_get_orientations(self.h, self.np)

    def get_particles_async(self, pinned):
        """Enqueues a read-back into `pinned` (a page-locked float64 torch tensor of 15 np + 1
        values); returns a ticket for wait_particles."""
        if not (pinned.is_pinned() and str(pinned.dtype) == "torch.float64" and pinned.numel() >= 15 * self.np + 1):
            raise ValueError("expected a pinned float64 tensor of at least 15 np + 1 values")
        return lbm_get_particles_async(self.h, pinned.data_ptr())

    def wait_particles(self, ticket):
        lbm_wait_particles(self.h, ticket)

    def get_f(self):
        return lbm_get_distributions(self.h, self.Q, self.N).reshape((self.Q,) + self.shape)

    def set_f(self, f):
        lbm_set_distributions(self.h, np.ascontiguousarray(f, dtype=np.float64).reshape(self.Q, self.N))

    def get_tags(self):
        return lbm_get_masks(self.h, self.N).reshape(self.shape)

    def info(self):
        return lbm_get_info(self.h)

    def profile(self, n):
        return lbm_profile_steps(self.h, n)

    def diagnostics(self):
        """Total mass and momentum, max |u|, Mach number, non-finite sites (lbm_diagnostics)."""
        return lbm_diagnostics(self.h)

    def run(self, steps, log=None, every=1):
        """Advances `steps` steps. With `log` (a path, opened for appending, or a text file),
        writes one JSON line after every `every` steps and after the last: the step count,
        total mass and fluid momentum, max |u| and Mach number, non-finite sites
        (lbm_diagnostics), and with particles the summed force and torque on them (-dP_B and
        -dL_B of Eqs. 8-9, lbm_get_particles). When the state turns non-finite the line is
        written with "error": "LBM_E_NAN" before the LbmError propagates."""
        if log is None:
            self.step(steps)
            return
        if every < 1:
            raise ValueError("every must be at least 1")
        own = isinstance(log, (str, os.PathLike))
        f = open(log, "a") if own else log
        try:
            done = 0
            while done < steps:
                n = min(every, steps - done)
                self.step(n)
                done += n
                rec, err = self._log_record()
                f.write(json.dumps(rec) + "\n")
                f.flush()
                if err is not None:
                    raise err
        finally:
            if own:
                f.close()

    def _log_record(self):
        """The JSON record of the current step boundary and the LbmError to raise once it is
        written (None when the state is finite)."""
        rec = {"step": int(self.info()["steps"])}
        err = None
        try:
            d = self.diagnostics()
        except LbmError as e:
            d = getattr(e, "diagnostics", None)
            if d is None:
                raise
            rec["error"] = STATUS.get(e.status, str(e.status))
            err = e
        rec["mass"] = float(d["mass"])
        rec["momentum"] = [float(v) for v in d["momentum"]]
        rec["max_speed"] = float(d["max_speed"])
        rec["mach"] = float(d["mach"])
        rec["nonfinite_sites"] = int(d["nonfinite_sites"])
        if err is None and self.np > 0:
            p = self.get_particles()
            rec["force_sum"] = [float(v) for v in np.sum(p["force"], axis=0)]
            rec["torque_sum"] = [float(v) for v in np.sum(p["torque"], axis=0)]
        return rec, err

    def checkpoint(self):
        """State at the current step boundary (lbm_checkpoint_save) as a numpy uint8 array."""
        return lbm_checkpoint_save(self.h)

    def restore(self, buf):
        """Continues from a checkpoint of a context set up by the same calls."""
        lbm_checkpoint_load(self.h, buf)

    def save(self, path):
        self.checkpoint().tofile(path)

    def load(self, path):
        self.restore(np.fromfile(path, dtype=np.uint8))

    def set_sweep_shape(self, threads_x):
        """Sweep kernel shape (lbm_set_sweep_shape): 16, 32, 64, 128 threads along x for the
        two-site kernel, 0 for the one-site kernel, -1 automatic."""
        lbm_set_sweep_shape(self.h, threads_x)

    def closure_features(self, n_side, spacing, u_ref):
        """Closure inputs of every particle as a CUDA float32 tensor [np, 4 n_side^3 + 3]: the
        stencil moments, then the fractional offset of the reference centre."""
        import torch
        out = torch.empty((self.np, 4 * n_side ** 3 + 3), dtype=torch.float32, device="cuda")
        lbm_closure_features(self.h, n_side, spacing, u_ref, out.data_ptr())
        self.synchronize()
        return out


class Batch:
    """An ensemble of independent cells stepped together (lbm_batch_*)."""

    def __init__(self, lattice, dims, taus, body_forces=None, precision="fp32", walls=(0, 0, 0),
                 gravity=(0.0, 0.0, 0.0), gap=0.0, body_force_on_particles=False):
        self.lattice = lattice
        self.dims = [tuple(int(v) for v in d) for d in np.asarray(dims).reshape(-1, 3)]
        faces = [LBM_NOSLIP if walls[k // 2] else LBM_PERIODIC for k in range(6)]
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.h = lbm_batch_create(lattice, self.dims, taus, body_forces, prec, faces, gravity, gap,
                                  body_force_on_particles)
        self.np = [0] * len(self.dims)

    def __len__(self):
        return len(self.dims)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def add_particles(self, cell, centers, radii, densities, velocities=None, omegas=None):
        lbm_batch_add_particles(self.h, cell, centers, radii, densities, velocities, omegas)
        self.np[cell] = lbm_get_info(lbm_batch_cell(self.h, cell))["particles"]

    def cell(self, i):
        nx, ny, nz = self.dims[i]
        return Simulation.borrowed(lbm_batch_cell(self.h, i), self.lattice, nx, ny, nz, self.np[i])

    def set_tuning(self, tile_width=None, order=0, grid=0, steps_per_graph=1):
        lbm_batch_set_tuning(self.h, tile_width, order, grid, steps_per_graph)

    def step(self, n=1):
        lbm_batch_step(self.h, n)

    def synchronize(self):
        lbm_batch_synchronize(self.h)

    def profile(self, n):
        return lbm_batch_profile_steps(self.h, n)

    def info(self):
        return lbm_batch_get_info(self.h)

    @property
    def stream(self):
        return lbm_batch_stream(self.h)


def lbm_closure_features(h, n_side, spacing, u_ref, out_ptr):
    _check(h, load().lbm_closure_features(h, int(n_side), float(spacing), float(u_ref), ctypes.c_void_p(out_ptr)))


def _mcheck(h, status):
    if status != LBM_OK:
        msg = load().lbm_mlp_last_error(h) if h else b"(no network)"
        raise LbmError(status, msg.decode(errors="replace") if msg else "")


def lbm_mlp_create(sizes, cuda_stream=None):
    sz = np.ascontiguousarray(sizes, dtype=np.int32)
    h = ctypes.c_void_p()
    st = load().lbm_mlp_create(ctypes.byref(h), len(sz) - 1, _ip(sz), ctypes.c_void_p(cuda_stream) if cuda_stream else None)
    if st != LBM_OK:
        raise LbmError(st, "lbm_mlp_create(%s)" % list(sizes))
    return h


def lbm_mlp_num_params(h):
    return int(load().lbm_mlp_num_params(h))


def lbm_mlp_set_params(h, flat):
    flat = _f64(flat)
    _mcheck(h, load().lbm_mlp_set_params(h, _dp(flat)))


def lbm_mlp_set_input_scaling(h, shift, scale):
    if shift is None:
        _mcheck(h, load().lbm_mlp_set_input_scaling(h, None, None))
        return
    shift = np.ascontiguousarray(shift, dtype=np.float64)
    scale = np.ascontiguousarray(scale, dtype=np.float64)
    _mcheck(h, load().lbm_mlp_set_input_scaling(h, _dp(shift), _dp(scale)))


def lbm_mlp_get_params(h, params=True, grads=False):
    n = lbm_mlp_num_params(h)
    p = np.empty(n) if params else None
    g = np.empty(n) if grads else None
    _mcheck(h, load().lbm_mlp_get_params(h, _dp(p), _dp(g)))
    return p, g


def lbm_mlp_forward(h, x_ptr, rows, y_ptr):
    _mcheck(h, load().lbm_mlp_forward(h, ctypes.c_void_p(x_ptr), int(rows), ctypes.c_void_p(y_ptr)))


def lbm_mlp_loss_grad(h, x_ptr, t_ptr, rows, want_loss=True):
    loss = ctypes.c_double(0.0)
    _mcheck(h, load().lbm_mlp_loss_grad(h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(rows),
                                        ctypes.byref(loss) if want_loss else None))
    return loss.value


def lbm_mlp_adam_step(h, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _mcheck(h, load().lbm_mlp_adam_step(h, float(lr), float(beta1), float(beta2), float(eps)))


def lbm_mlp_train(h, x_ptr, t_ptr, n, batch, epochs, lr, seed=0):
    out = np.zeros(epochs)
    _mcheck(h, load().lbm_mlp_train(h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(n), int(batch), int(epochs),
                                    float(lr), int(seed), _dp(out)))
    return out


def lbm_mlp_last_error(h):
    m = load().lbm_mlp_last_error(h)
    return m.decode(errors="replace") if m else ""


def lbm_mlp_destroy(h):
    if h:
        load().lbm_mlp_destroy(h)


def pack_params(layers):
    """[[W, b], ...] (W: out x in) -> the flat layer-major vector of the C-ABI."""
    return np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in layers])


def unpack_params(flat, sizes):
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = np.asarray(flat[o:o + a * b]).reshape(b, a)
        o += a * b
        out.append([W, np.asarray(flat[o:o + b])])
        o += b
    return out


class MLP:
    """The closure network on the GPU. Data arguments are torch CUDA tensors (FP32,
    contiguous, row-major); torch only provides their memory."""

    def __init__(self, sizes, cuda_stream=None):
        self.sizes = list(sizes)
        self.h = lbm_mlp_create(sizes, cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            lbm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_params(self, layers):
        lbm_mlp_set_params(self.h, pack_params(layers))

    def set_input_scaling(self, shift, scale):
        """Inputs enter the network as (x - shift) * scale (lbm_mlp_set_input_scaling)."""
        lbm_mlp_set_input_scaling(self.h, shift, scale)

    def params(self):
        p, _ = lbm_mlp_get_params(self.h)
        return unpack_params(p, self.sizes)

    def grads(self):
        _, g = lbm_mlp_get_params(self.h, params=False, grads=True)
        return unpack_params(g, self.sizes)

    @staticmethod
    def _check(t, cols):
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32" and t.dim() == 2 and t.shape[1] == cols):
            raise ValueError("expected a contiguous CUDA float32 tensor with %d columns" % cols)

    def forward(self, x):
        import torch
        self._check(x, self.sizes[0])
        y = torch.empty((x.shape[0], self.sizes[-1]), dtype=torch.float32, device=x.device)
        lbm_mlp_forward(self.h, x.data_ptr(), x.shape[0], y.data_ptr())
        return y

    def loss_grad(self, x, t):
        self._check(x, self.sizes[0])
        self._check(t, self.sizes[-1])
        return lbm_mlp_loss_grad(self.h, x.data_ptr(), t.data_ptr(), x.shape[0])

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        lbm_mlp_adam_step(self.h, lr, beta1, beta2, eps)

    def train(self, x, t, batch, epochs, lr, seed=0):
        self._check(x, self.sizes[0])
        self._check(t, self.sizes[-1])
        return lbm_mlp_train(self.h, x.data_ptr(), t.data_ptr(), x.shape[0], batch, epochs, lr, seed)
