"""FP64 CPU oracle for the multidirect-forcing IB step (arXiv 2408.14140).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_2408_14140_gb300``) never imports it, and it imports nothing
from the product: the two share no code.

The arithmetic lives in ``ib_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that x86 and Arm hosts round identically); this
module only builds it with gcc and marshals numpy arrays through ctypes.
Every function cites the passage of the paper it follows in the C source.

The fluid step around the forcing (Sec. 3.1 Steps 1 and 3, one periodic
level) is in ``fluid.py``, in numpy, with numpy's FFT as its only library
step.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
against values the paper prints (PVF tables, Sec. 4.1), closed forms and
brute force, and the fluid step by ``tests/test_oracle_fluid.py`` (closed-form
gradient and solves, adjointness, divergence-free and idempotent projection,
Taylor-Green convergence); see the test modules for which pin covers which
function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ib_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ROMA3 = 0
PESKIN4 = 1
SEQUENTIAL = 0
SIMULTANEOUS = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile ``ib_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
    lib.or_phi.restype = d
    lib.or_phi.argtypes = [i, d]
    lib.or_interpolate.restype = None
    lib.or_interpolate.argtypes = [p, d, p, p, l, p, i, p]
    lib.or_spread.restype = None
    lib.or_spread.argtypes = [p, d, p, l, p, p, p, i, p]
    lib.or_multidirect.restype = i
    lib.or_multidirect.argtypes = [p, d, p, p, i, p, p, p, p, p, p, i, d, i, i,
                                   p, p]
    lib.or_pvf_ellipsoid_volume.restype = d
    lib.or_pvf_ellipsoid_volume.argtypes = [p, d, p, p, p]
    lib.or_volume_integrals.restype = None
    lib.or_volume_integrals.argtypes = [p, d, p, p, i, p, p, p, p, p]
    lib.or_volume_integrals_ellipsoid.restype = None
    lib.or_volume_integrals_ellipsoid.argtypes = [p, d, p, p, i, p, p, p, p, p]
    lib.or_drag_force.restype = None
    lib.or_drag_force.argtypes = [i, p, p, p, d, d, p]
    lib.or_force_torque.restype = None
    lib.or_force_torque.argtypes = [i, p, p, p, p, d, p, p]
    lib.or_collide_update.restype = None
    lib.or_collide_update.argtypes = [i, p, p, p, p, p, p, d, p, d, p, p, p, p,
                                      p, p, p]
    lib.or_num_threads.restype = i
    lib.or_num_threads.argtypes = []
    lib.or_set_num_threads.restype = None
    lib.or_set_num_threads.argtypes = [i]
    _lib = lib
    return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _grid(n, org):
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int32).reshape(3))
    org = _f64(org, (3,))
    return n, org


def phi(kernel: int, r: float) -> float:
    """1-D kernel value phi(r), r in cell units."""
    return _load().or_phi(int(kernel), float(r))


def num_threads() -> int:
    return _load().or_num_threads()


def set_num_threads(t: int) -> None:
    _load().or_set_num_threads(int(t))


def interpolate(n, h, org, u, X, kernel=ROMA3):
    """U[M,3] = J u at positions X[M,3]; u is [3, n2, n1, n0] float64."""
    n, org = _grid(n, org)
    u = _f64(u)
    X = _f64(X).reshape(-1, 3)
    U = np.zeros_like(X)
    _load().or_interpolate(_ptr(n), float(h), _ptr(org), _ptr(u), X.shape[0],
                           _ptr(X), int(kernel), _ptr(U))
    return U


def spread(n, h, org, X, F, dV, kernel=ROMA3, f=None):
    """f += S F (returns f, a new zero field when ``f`` is None)."""
    n, org = _grid(n, org)
    X = _f64(X).reshape(-1, 3)
    F = _f64(F).reshape(-1, 3)
    dV = _f64(dV).reshape(-1)
    if f is None:
        f = np.zeros((3, int(n[2]), int(n[1]), int(n[0])))
    assert f.dtype == np.float64 and f.flags.c_contiguous
    _load().or_spread(_ptr(n), float(h), _ptr(org), X.shape[0], _ptr(X),
                      _ptr(F), _ptr(dV), int(kernel), _ptr(f))
    return f


def multidirect(n, h, org, u, Xr, Ur, Wr, moff, R, dV, Ns, dt,
                kernel=ROMA3, order=SEQUENTIAL, want_f=False):
    """Algorithm 1 over all particles.  Returns (u_new, F[M,3], f or None).

    ``u`` is not modified; ``moff`` is the CSR offset array [P+1] of the
    markers of each particle; ``R`` are marker offsets X_l - X_r.
    """
    n, org = _grid(n, org)
    u = _f64(u).copy()
    Xr = _f64(Xr).reshape(-1, 3)
    Ur = _f64(Ur).reshape(-1, 3)
    Wr = _f64(Wr).reshape(-1, 3)
    moff = np.ascontiguousarray(np.asarray(moff, dtype=np.int64))
    R = _f64(R).reshape(-1, 3)
    dV = _f64(dV).reshape(-1)
    P = Xr.shape[0]
    M = int(moff[-1])
    assert R.shape[0] == M and dV.shape[0] == M and moff.shape[0] == P + 1
    F = np.zeros((M, 3))
    f = np.zeros_like(u) if want_f else None
    rc = _load().or_multidirect(_ptr(n), float(h), _ptr(org), _ptr(u), P,
                                _ptr(Xr), _ptr(Ur), _ptr(Wr), _ptr(moff),
                                _ptr(R), _ptr(dV), int(Ns), float(dt),
                                int(kernel), int(order), _ptr(F), _ptr(f))
    if rc != 0:
        raise MemoryError("oracle multidirect: allocation failed")
    return u, F, f


def pvf_ellipsoid_volume(n, h, org, centre, axes) -> float:
    """sum alpha h^3 of an ellipsoid on a box of n cells (Sec. 4.1 tables)."""
    n, org = _grid(n, org)
    c = _f64(centre, (3,))
    ax = _f64(axes, (3,))
    return _load().or_pvf_ellipsoid_volume(_ptr(n), float(h), _ptr(org),
                                           _ptr(c), _ptr(ax))


def volume_integrals(n, h, org, u, Xr, radius):
    """(Iu[P,3], Irxu[P,3], vol[P]) of each sphere through its PVF."""
    n, org = _grid(n, org)
    u = _f64(u)
    Xr = _f64(Xr).reshape(-1, 3)
    radius = _f64(radius).reshape(-1)
    P = Xr.shape[0]
    Iu = np.zeros((P, 3))
    Irxu = np.zeros((P, 3))
    vol = np.zeros(P)
    _load().or_volume_integrals(_ptr(n), float(h), _ptr(org), _ptr(u), P,
                                _ptr(Xr), _ptr(radius), _ptr(Iu), _ptr(Irxu),
                                _ptr(vol))
    return Iu, Irxu, vol


def volume_integrals_ellipsoid(n, h, org, u, Xr, axes):
    """(Iu[P,3], Irxu[P,3], vol[P]) of axis-aligned ellipsoids of semi-axes
    axes[P,3] through their PVF (the sphere is a = b = c = R)."""
    n, org = _grid(n, org)
    u = _f64(u)
    Xr = _f64(Xr).reshape(-1, 3)
    axes = _f64(axes).reshape(-1, 3)
    P = Xr.shape[0]
    Iu = np.zeros((P, 3))
    Irxu = np.zeros((P, 3))
    vol = np.zeros(P)
    _load().or_volume_integrals_ellipsoid(_ptr(n), float(h), _ptr(org), _ptr(u), P,
                                          _ptr(Xr), _ptr(axes), _ptr(Iu), _ptr(Irxu),
                                          _ptr(vol))
    return Iu, Irxu, vol


def drag_force(F_ib, Iu_new, Iu_old, rho_f, dt):
    """F_D[P,3] of Eq. FD: F_ib + rho_f (Iu^{n+1} - Iu^n) / dt."""
    F_ib = _f64(F_ib).reshape(-1, 3)
    Iu_new = _f64(Iu_new).reshape(-1, 3)
    Iu_old = _f64(Iu_old).reshape(-1, 3)
    P = F_ib.shape[0]
    FD = np.zeros((P, 3))
    _load().or_drag_force(P, _ptr(F_ib), _ptr(Iu_new), _ptr(Iu_old), float(rho_f), float(dt),
                          _ptr(FD))
    return FD


def force_torque(moff, R, dV, F, rho_f):
    """(F_ib[P,3], T_ib[P,3]) = (-rho_f sum F dV, -rho_f sum R x F dV)."""
    moff = np.ascontiguousarray(np.asarray(moff, dtype=np.int64))
    R = _f64(R).reshape(-1, 3)
    dV = _f64(dV).reshape(-1)
    F = _f64(F).reshape(-1, 3)
    P = moff.shape[0] - 1
    Fib = np.zeros((P, 3))
    Tib = np.zeros((P, 3))
    _load().or_force_torque(P, _ptr(moff), _ptr(R), _ptr(dV), _ptr(F),
                            float(rho_f), _ptr(Fib), _ptr(Tib))
    return Fib, Tib


def collide_update(Xr, Ur, Wr, radius, rho_p, n, h, phys, dt, Fib, Tib,
                   Iu_new, Iu_old, Irxu_new, Irxu_old):
    """Collision force + Newton-Euler + centroid update.

    ``phys`` = (rho_f, gx, gy, gz, g_coll, eps_c, d_c).  Returns new copies
    (Xr, Ur, Wr, Fc).
    """
    Xr = _f64(Xr).reshape(-1, 3).copy()
    Ur = _f64(Ur).reshape(-1, 3).copy()
    Wr = _f64(Wr).reshape(-1, 3).copy()
    P = Xr.shape[0]
    radius = _f64(radius).reshape(-1)
    rho_p = _f64(rho_p).reshape(-1)
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int32).reshape(3))
    phys = _f64(phys, (7,))
    Fc = np.zeros((P, 3))
    args = [_f64(a).reshape(-1, 3) for a in (Fib, Tib, Iu_new, Iu_old,
                                             Irxu_new, Irxu_old)]
    _load().or_collide_update(P, _ptr(Xr), _ptr(Ur), _ptr(Wr), _ptr(radius),
                              _ptr(rho_p), _ptr(n), float(h), _ptr(phys),
                              float(dt), *[_ptr(a) for a in args], _ptr(Fc))
    return Xr, Ur, Wr, Fc
