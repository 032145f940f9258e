"""GB300-native multidirect-forcing immersed-boundary library.

Implements the data-parallel hot path of the particle-resolved method of
Zeng et al. (arXiv 2408.14140): Algorithm 1 (multidirect forcing) with the
regularised delta kernel, the PVF volume integrals (Sec. 4.1), the marker
force/torque reductions and the repulsive-potential collision + Newton-Euler
update (Secs. 3.2.2, 4.6).  All arithmetic runs in hand-written CUDA kernels
for sm_103a behind the C ABI declared in ``include/gbib.h``; this package is
the thin ctypes binding (``api``) plus the seeded input generators
(``synth``).  Importing the package does not load the CUDA library; the first
call into ``api`` does, and raises if it is missing.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "api"]


def __getattr__(name):
    if name == "api":
        import importlib
        return importlib.import_module(__name__ + ".api")
    raise AttributeError(name)
