"""GB300-native (sm_103a) site-based particle-suspension lattice Boltzmann.

The compute path is a CUDA shared library (``liblbmp.so``, C-ABI declared in
``include/lbmp.h``); ``paper_1105_2904_gb300.lbmp`` is its thin ctypes binding and
``paper_1105_2904_gb300.workloads`` draws seeded synthetic inputs. Importing this package
loads nothing; the binding loads the library on first use and raises if it is missing.
"""

__all__ = ["lbmp", "workloads"]
