"""The bounds-checked build (LBM_DEBUG) runs the parity cases without a fault and gives the
same bits as the normal build.

The bounds-checked build checks particle ids read from the owner map, BS record slots and
contact-list indices in the kernels; an index out of range records LBM_E_BOUNDS in the device
status word and the access is skipped. Its checks must never fire on valid states, and since
they only guard accesses the arithmetic is the same: the two builds, each loaded in its own
process, must produce identical distributions, particle states and owner maps."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, %(root)r)
import numpy as np
from paper_1105_2904_gb300 import build as B
B.build()
from paper_1105_2904_gb300 import lbmp
from paper_1105_2904_gb300 import workloads as W
out = {}
dims = (42, 36, 30)
c, rad = W.rsa_centers(dims, 5, 5.0, seed=61, min_gap=1.0, walls=(0, 0, 1))
v = W.gaussian_velocities(5, 0.04, seed=62)
om = W.gaussian_velocities(5, 0.004, seed=63)
d = np.array([1.2, 2.0, 0.9, 1.5, 3.0])
for prec, shape in (("fp64", -1), ("fp32", 16), ("fp32", 0), ("fp16", 16)):
    g = lbmp.Simulation(1, *dims, 0.7, body_force=(2e-6, 0.0, 0.0), precision=prec, walls=(0, 0, 1),
                        gap=0.5, body_force_on_particles=True, wall_velocity={5: (0.01, 0.0, 0.0)})
    g.set_sweep_shape(shape)
    g.add_particles(c, rad, d, v, om)
    g.step(60)
    st = g.synchronize()
    p = g.get_particles()
    key = "%%s_%%d" %% (prec, shape)
    out[key + "_f"] = g.get_f()
    out[key + "_tags"] = g.get_tags()
    for k in ("x", "u", "omega", "force", "torque"):
        out[key + "_" + k] = p[k]
    g.close()
np.savez(sys.argv[1], **out)
'''


def _run(debug, path):
    env = dict(os.environ)
    env["LBMP_DEBUG"] = "1" if debug else "0"
    code = SCRIPT % {"root": ROOT}
    r = subprocess.run([sys.executable, "-c", code, path], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    return np.load(path)


def test_bounds_checked_build_matches_the_normal_build(tmp_path):
    a = _run(False, str(tmp_path / "normal.npz"))
    b = _run(True, str(tmp_path / "checked.npz"))   # a recorded LBM_E_BOUNDS raises in the run
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
