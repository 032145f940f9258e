"""ctypes binding of ``libgbib.so`` (C ABI in ``include/gbib.h``).

Argument marshalling only: PyTorch tensors supply device memory and the
current CUDA stream; every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback -- loading fails loudly when the library
is missing.

Entry points mirror the C ABI names:
  ib_interpolate, ib_spread, ib_multidirect_forcing,
  particle_volume_integrals, particle_force_torque, particle_collide_update,
  ib_batch_multidirect_forcing, ib_batch_volume_integrals, ib_batch_collide_update
as methods of :class:`Context`.  :func:`pack_batch` lays several cases'
particles and markers out as one flat set for the batch entry points.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbib.so")

IB_OK = 0
IB_ERR_INVALID = -1
IB_ERR_OOM = -2
IB_ERR_CUDA = -3
IB_ERR_TIMEOUT = -4
IB_ERR_NONFINITE = -5
IB_ERR_UNSUPPORTED = -6

IB_F64 = 0
IB_F32 = 1
ROMA3 = 0
PESKIN4 = 1
SEQUENTIAL = 0
SIMULTANEOUS = 1
PASSES = {"auto": 0, "wavefront": 1, "resident": 2, "groups": 3}

SPREAD_MODES = {"gather": 0, "atomic": 1}

PHASES = {"mdf_prep": 0, "mdf_passes": 1, "spread": 2, "interp": 3, "volume": 4,
          "force": 5, "collide": 6, "mdf_interp": 7, "mdf_gather": 8, "fluid_predictor": 9,
          "fluid_projection": 10}

EXPORTS = ["ib_ctx_create", "ib_ctx_reserve", "ib_ctx_destroy", "ib_ctx_status",
           "ib_last_error", "ib_workspace_needed", "ib_ctx_sm_count",
           "ib_ctx_set_timing", "ib_ctx_read_timing", "ib_ctx_set_pass_kernels", "ib_ctx_set_volume_split",
           "ib_ctx_set_field_wait", "ib_selftest_wait_timeout",
           "ib_interpolate", "ib_spread", "ib_multidirect_forcing",
           "particle_volume_integrals", "particle_force_torque",
           "particle_collide_update", "particle_volume_integrals_static",
           "ib_batch_multidirect_forcing", "ib_batch_volume_integrals", "ib_batch_collide_update",
           "particle_volume_integrals_ellipsoid", "particle_drag_force",
           "ib_batch_table_create", "ib_batch_table_destroy", "ib_batch_table_multidirect_forcing",
           "ib_batch_table_volume_integrals", "ib_batch_table_collide_update", "ib_ctx_set_spread_mode",
           "ib_ctx_set_gather", "fluid_predictor", "level_projection", "ib_batch_table_update",
           "ib_pvf_plan_create", "ib_pvf_plan_destroy", "particle_volume_integrals_keep",
           "particle_volume_integrals_plan"]


class IBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gbib error %d: %s" % (code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("origin", ctypes.c_double * 3), ("prec", ctypes.c_int)]


class Particles(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("Xr", ctypes.c_void_p), ("Ur", ctypes.c_void_p),
                ("Wr", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("rho_p", ctypes.c_void_p), ("marker_offset", ctypes.c_void_p)]


class Markers(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("R", ctypes.c_void_p), ("dV", ctypes.c_void_p)]


class Case(ctypes.Structure):
    _fields_ = [("grid", Grid), ("u", ctypes.c_void_p), ("f_out", ctypes.c_void_p),
                ("p_begin", ctypes.c_int), ("p_end", ctypes.c_int)]


class Phys(ctypes.Structure):
    _fields_ = [("rho_f", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("g_coll", ctypes.c_double), ("eps_c", ctypes.c_double),
                ("d_c", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libgbib.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    i, p, d, sz = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_size_t
    sig = {
        "ib_ctx_create": (i, [ctypes.POINTER(p), sz]),
        "ib_ctx_reserve": (i, [p, sz]),
        "ib_ctx_destroy": (i, [p]),
        "ib_ctx_status": (i, [p, p]),
        "ib_last_error": (ctypes.c_char_p, []),
        "ib_workspace_needed": (sz, []),
        "ib_ctx_sm_count": (i, [p]),
        "ib_ctx_set_timing": (i, [p, i]),
        "ib_ctx_read_timing": (i, [p, i, ctypes.POINTER(d), ctypes.POINTER(i)]),
        "ib_ctx_set_pass_kernels": (i, [p, i]),
        "ib_ctx_set_volume_split": (i, [p, i]),
        "ib_ctx_set_field_wait": (i, [p, p]),
        "ib_selftest_wait_timeout": (i, [p, ctypes.c_longlong, p]),
        "ib_interpolate": (i, [p, p, p, i, p, i, p, p]),
        "ib_spread": (i, [p, p, i, p, p, p, i, p, p]),
        "ib_multidirect_forcing": (i, [p, p, p, p, p, i, d, i, i, p, p, p]),
        "particle_volume_integrals": (i, [p, p, p, p, p, p, p, p]),
        "particle_volume_integrals_static": (i, [p, p, p, p, p, p, p]),
        "particle_force_torque": (i, [p, p, p, p, d, p, p, p]),
        "particle_collide_update": (i, [p, p, p, p, d, p, p, p, p, p, p, p, p]),
        "ib_batch_multidirect_forcing": (i, [p, i, p, p, p, i, d, i, i, p, p]),
        "particle_volume_integrals_ellipsoid": (i, [p, p, p, i, p, p, p, p, p, p]),
        "particle_drag_force": (i, [p, i, p, p, p, d, d, p, p]),
        "ib_batch_volume_integrals": (i, [p, i, p, p, p, p, p, p]),
        "ib_batch_collide_update": (i, [p, i, p, p, p, d, p, p, p, p, p, p, p, p]),
        "ib_ctx_set_spread_mode": (i, [p, i]),
        "ib_ctx_set_gather": (i, [p, i, i]),
        "fluid_predictor": (i, [p, p, p, p, d, d, ctypes.POINTER(d), d, p, p]),
        "level_projection": (i, [p, p, p, p, d, d, p]),
        "ib_batch_table_create": (i, [p, i, p, i, p, ctypes.POINTER(p)]),
        "ib_batch_table_destroy": (i, [p]),
        "ib_batch_table_update": (i, [p, i, p, i, p, p]),
        "ib_batch_table_multidirect_forcing": (i, [p, p, p, p, i, d, i, i, p, p]),
        "ib_batch_table_volume_integrals": (i, [p, p, p, p, p, p, p]),
        "ib_batch_table_collide_update": (i, [p, p, p, d, p, p, p, p, p, p, p, p]),
        "ib_pvf_plan_create": (i, [p, i, i, ctypes.POINTER(p)]),
        "ib_pvf_plan_destroy": (i, [p]),
        "particle_volume_integrals_keep": (i, [p, p, p, p, p, p, p, p, p]),
        "particle_volume_integrals_plan": (i, [p, p, p, p, p, p, p, p, p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t


def field_dtype(prec):
    return torch.float64 if prec == IB_F64 else torch.float32


def make_grid(n, h, origin=(0.0, 0.0, 0.0), prec=IB_F64) -> Grid:
    g = Grid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.origin[a] = float(origin[a])
    g.h = float(h)
    g.prec = int(prec)
    return g


class Context:
    """Owns one ``ib_ctx`` (device workspace + error latch)."""

    def __init__(self, workspace_bytes: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        self._check(self.lib.ib_ctx_create(ctypes.byref(h), int(workspace_bytes)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.ib_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != IB_OK:
            raise IBError(rc, self.lib.ib_last_error().decode())

    def _call(self, fn, *args):
        """Call an entry point; on IB_ERR_OOM grow the workspace to what the
        call reported and retry (a call can stop at an earlier allocation, so
        the need may grow over a few retries)."""
        rc = fn(*args)
        for _ in range(4):
            if rc != IB_ERR_OOM:
                break
            need = self.lib.ib_workspace_needed()
            if not need:
                break
            self._check(self.lib.ib_ctx_reserve(self.handle, int(need * 5 // 4) + (1 << 20)))
            rc = fn(*args)
        self._check(rc)

    @property
    def sm_count(self):
        return self.lib.ib_ctx_sm_count(self.handle)

    def reserve(self, nbytes: int):
        self._check(self.lib.ib_ctx_reserve(self.handle, int(nbytes)))

    def set_timing(self, enable: bool):
        """Record CUDA events around the library's kernels (see gbib.h)."""
        self._check(self.lib.ib_ctx_set_timing(self.handle, 1 if enable else 0))

    def set_pass_kernels(self, which: str):
        """Kernels of the sequential-order passes: "auto", "wavefront",
        "resident" or "groups" (see gbib.h; every choice gives bitwise the
        same result)."""
        self._check(self.lib.ib_ctx_set_pass_kernels(self.handle, PASSES[which]))

    def set_spread_mode(self, mode: str):
        """Spreading form: "gather" (deterministic, the default) or "atomic"
        (warp-aggregated atomic additions; see gbib.h)."""
        self._check(self.lib.ib_ctx_set_spread_mode(self.handle, SPREAD_MODES[mode]))

    def set_gather(self, ctas_per_sm: int = 0, stage: int = 0):
        """Wavefront gather layout: resident CTAs per SM and staged candidates
        per tile (0: the defaults; see gbib.h).  Results do not change."""
        self._check(self.lib.ib_ctx_set_gather(self.handle, int(ctas_per_sm), int(stage)))

    def fluid_predictor(self, u, p, h, rho_f, mu, g, dt, u_star=None, origin=(0.0, 0.0, 0.0), stream=None):
        """Step 1 (Eq. 31): u~* from u^n [3, n2, n1, n0] and p^{n-1/2} [n2, n1, n0]
        (nodes) on a periodic power-of-two grid; returns u_star."""
        prec = IB_F64 if u.dtype == torch.float64 else IB_F32
        n = (u.shape[3], u.shape[2], u.shape[1])
        _need(u, "u", u.dtype, (3, n[2], n[1], n[0]))
        _need(p, "p", u.dtype, (n[2], n[1], n[0]))
        if u_star is None:
            u_star = torch.empty_like(u)
        _need(u_star, "u_star", u.dtype, tuple(u.shape))
        gr = make_grid(n, h, origin, prec)
        gv = (ctypes.c_double * 3)(*[float(x) for x in g])
        self._call(self.lib.fluid_predictor, self.handle, ctypes.byref(gr), _ptr(u), _ptr(p), float(rho_f),
                   float(mu), gv, float(dt), _ptr(u_star), _stream(stream))
        return u_star

    def level_projection(self, u, p, h, rho_f, dt, origin=(0.0, 0.0, 0.0), stream=None):
        """Step 3 (Eqs. ns_lp1-3) in place: u* -> u^{n+1}, p^{n-1/2} -> p^{n+1/2}."""
        prec = IB_F64 if u.dtype == torch.float64 else IB_F32
        n = (u.shape[3], u.shape[2], u.shape[1])
        _need(u, "u", u.dtype, (3, n[2], n[1], n[0]))
        _need(p, "p", u.dtype, (n[2], n[1], n[0]))
        gr = make_grid(n, h, origin, prec)
        self._call(self.lib.level_projection, self.handle, ctypes.byref(gr), _ptr(u), _ptr(p), float(rho_f),
                   float(dt), _stream(stream))
        return u, p

    def set_field_wait(self, event):
        """Make the forcing calls on this context wait for a torch.cuda.Event
        (None clears it) after their preparation, before they touch the field
        (see gbib.h).  The caller keeps the event alive."""
        self._field_wait = event
        handle = None if event is None else ctypes.c_void_p(event.cuda_event)
        self._check(self.lib.ib_ctx_set_field_wait(self.handle, handle))

    def selftest_wait_timeout(self, cycles: int = 1_000_000, stream=None):
        """Enqueue a bounded wait that runs out (a device word nothing sets):
        the next :meth:`status` raises IB_ERR_TIMEOUT and clears it."""
        self._check(self.lib.ib_selftest_wait_timeout(self.handle, int(cycles), _stream(stream)))

    def set_volume_split(self, ctas_per_particle: int):
        """CTAs per particle of the volume integrals, 0 = automatic (see gbib.h)."""
        self._check(self.lib.ib_ctx_set_volume_split(self.handle, int(ctas_per_particle)))

    def read_timing(self, phase: str):
        """(total ms, launches) of one phase since the last read; resets it."""
        ms = ctypes.c_double()
        n = ctypes.c_int()
        self._check(self.lib.ib_ctx_read_timing(self.handle, PHASES[phase], ctypes.byref(ms),
                                                ctypes.byref(n)))
        return ms.value, n.value

    def status(self, stream=None):
        """Synchronise the stream and raise the first device-side error."""
        self._check(self.lib.ib_ctx_status(self.handle, _stream(stream)))

    # -- operators -------------------------------------------------------
    @staticmethod
    def _grid_of(u, n, h, origin):
        prec = IB_F64 if u.dtype == torch.float64 else IB_F32
        return make_grid(n, h, origin, prec)

    def ib_interpolate(self, u, X, h, origin=(0.0, 0.0, 0.0), delta=ROMA3, U=None, stream=None):
        """U[M,3] (float64) = J u at positions X[M,3]; u is [3, n2, n1, n0]."""
        if u.dtype not in (torch.float64, torch.float32):
            raise TypeError("u must be float64 or float32")
        n = (u.shape[3], u.shape[2], u.shape[1])
        _need(u, "u", u.dtype, (3, n[2], n[1], n[0]))
        M = X.shape[0]
        _need(X, "X", torch.float64, (M, 3))
        if U is None:
            U = torch.empty((M, 3), dtype=torch.float64, device=X.device)
        _need(U, "U", torch.float64, (M, 3))
        g = self._grid_of(u, n, h, origin)
        self._call(self.lib.ib_interpolate, self.handle, ctypes.byref(g), _ptr(u), M, _ptr(X),
                   int(delta), _ptr(U), _stream(stream))
        return U

    def ib_spread(self, f, X, F, dV, h, origin=(0.0, 0.0, 0.0), delta=ROMA3, stream=None):
        """f += S F (deterministic gather); f is [3, n2, n1, n0]."""
        n = (f.shape[3], f.shape[2], f.shape[1])
        _need(f, "f", f.dtype, (3, n[2], n[1], n[0]))
        M = X.shape[0]
        _need(X, "X", torch.float64, (M, 3))
        _need(F, "F", torch.float64, (M, 3))
        _need(dV, "dV", torch.float64, (M,))
        g = self._grid_of(f, n, h, origin)
        self._call(self.lib.ib_spread, self.handle, ctypes.byref(g), M, _ptr(X), _ptr(F), _ptr(dV),
                   int(delta), _ptr(f), _stream(stream))
        return f

    @staticmethod
    def particles_struct(Xr, Ur, Wr, radius, rho_p, moff):
        P = Xr.shape[0]
        for t, nm in ((Xr, "Xr"), (Ur, "Ur"), (Wr, "Wr")):
            _need(t, nm, torch.float64, (P, 3))
        _need(radius, "radius", torch.float64, (P,))
        _need(rho_p, "rho_p", torch.float64, (P,))
        _need(moff, "marker_offset", torch.int32, (P + 1,))
        s = Particles()
        s.P = P
        s.Xr, s.Ur, s.Wr = Xr.data_ptr(), Ur.data_ptr(), Wr.data_ptr()
        s.radius, s.rho_p, s.marker_offset = radius.data_ptr(), rho_p.data_ptr(), moff.data_ptr()
        return s

    @staticmethod
    def markers_struct(R, dV):
        M = R.shape[0]
        _need(R, "R", torch.float64, (M, 3))
        _need(dV, "dV", torch.float64, (M,))
        s = Markers()
        s.M = M
        s.R, s.dV = R.data_ptr(), dV.data_ptr()
        return s

    def ib_multidirect_forcing(self, u, h, parts, marks, Ns, dt, origin=(0.0, 0.0, 0.0),
                               delta=ROMA3, order=SEQUENTIAL, F_out=None, f_out=None,
                               stream=None):
        """Algorithm 1 in place on u; returns F_out[M,3] (float64).

        ``parts`` = dict(Xr, Ur, Wr, radius, rho_p, moff); ``marks`` = dict(R, dV).
        """
        n = (u.shape[3], u.shape[2], u.shape[1])
        _need(u, "u", u.dtype, (3, n[2], n[1], n[0]))
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        ms = self.markers_struct(marks["R"], marks["dV"])
        if F_out is None:
            F_out = torch.empty((ms.M, 3), dtype=torch.float64, device=u.device)
        _need(F_out, "F_out", torch.float64, (ms.M, 3))
        if f_out is not None:
            _need(f_out, "f_out", u.dtype, tuple(u.shape))
        g = self._grid_of(u, n, h, origin)
        self._call(self.lib.ib_multidirect_forcing, self.handle, ctypes.byref(g), _ptr(u),
                   ctypes.byref(ps), ctypes.byref(ms), int(Ns), float(dt), int(delta), int(order),
                   _ptr(F_out), _ptr(f_out), _stream(stream))
        return F_out

    def particle_volume_integrals(self, u, h, parts, origin=(0.0, 0.0, 0.0), out=None, stream=None):
        """(Iu[P,3], Irxu[P,3], vol[P]) through the PVF of each sphere."""
        n = (u.shape[3], u.shape[2], u.shape[1])
        _need(u, "u", u.dtype, (3, n[2], n[1], n[0]))
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        P = ps.P
        if out is None:
            out = (torch.empty((P, 3), dtype=torch.float64, device=u.device),
                   torch.empty((P, 3), dtype=torch.float64, device=u.device),
                   torch.empty((P,), dtype=torch.float64, device=u.device))
        Iu, Irxu, vol = out
        _need(Iu, "Iu", torch.float64, (P, 3))
        _need(Irxu, "Irxu", torch.float64, (P, 3))
        _need(vol, "vol", torch.float64, (P,))
        g = self._grid_of(u, n, h, origin)
        self._call(self.lib.particle_volume_integrals, self.handle, ctypes.byref(g), _ptr(u),
                   ctypes.byref(ps), _ptr(Iu), _ptr(Irxu), _ptr(vol), _stream(stream))
        return Iu, Irxu, vol

    def _volume_call(self, fn, u, h, parts, plan, origin, out, stream):
        n = (u.shape[3], u.shape[2], u.shape[1])
        _need(u, "u", u.dtype, (3, n[2], n[1], n[0]))
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        P = ps.P
        if out is None:
            out = (torch.empty((P, 3), dtype=torch.float64, device=u.device),
                   torch.empty((P, 3), dtype=torch.float64, device=u.device),
                   torch.empty((P,), dtype=torch.float64, device=u.device))
        Iu, Irxu, vol = out
        _need(Iu, "Iu", torch.float64, (P, 3))
        _need(Irxu, "Irxu", torch.float64, (P, 3))
        _need(vol, "vol", torch.float64, (P,))
        g = self._grid_of(u, n, h, origin)
        self._call(fn, self.handle, ctypes.byref(g), _ptr(u), ctypes.byref(ps), plan.handle, _ptr(Iu), _ptr(Irxu),
                   _ptr(vol), _stream(stream))
        return Iu, Irxu, vol

    def particle_volume_integrals_keep(self, u, h, parts, plan, origin=(0.0, 0.0, 0.0), out=None, stream=None):
        """particle_volume_integrals, keeping the visited cells and their alpha
        in ``plan`` (a :class:`PvfPlan`)."""
        return self._volume_call(self.lib.particle_volume_integrals_keep, u, h, parts, plan, origin, out, stream)

    def particle_volume_integrals_plan(self, u, h, parts, plan, origin=(0.0, 0.0, 0.0), out=None, stream=None):
        """The volume integrals of another field at the particle positions the
        plan was kept for, from the kept cells and alpha."""
        return self._volume_call(self.lib.particle_volume_integrals_plan, u, h, parts, plan, origin, out, stream)

    def particle_volume_integrals_ellipsoid(self, u, h, Xr, axes, origin=(0.0, 0.0, 0.0), out=None,
                                            stream=None):
        """(Iu[P,3], Irxu[P,3], vol[P]) through the PVF of axis-aligned
        ellipsoids (semi-axes axes[P,3])."""
        n = (u.shape[3], u.shape[2], u.shape[1])
        _need(u, "u", u.dtype, (3, n[2], n[1], n[0]))
        P = Xr.shape[0]
        _need(Xr, "Xr", torch.float64, (P, 3))
        _need(axes, "axes", torch.float64, (P, 3))
        if out is None:
            out = (torch.empty((P, 3), dtype=torch.float64, device=u.device),
                   torch.empty((P, 3), dtype=torch.float64, device=u.device),
                   torch.empty((P,), dtype=torch.float64, device=u.device))
        Iu, Irxu, vol = out
        _need(Iu, "Iu", torch.float64, (P, 3))
        _need(Irxu, "Irxu", torch.float64, (P, 3))
        _need(vol, "vol", torch.float64, (P,))
        g = self._grid_of(u, n, h, origin)
        self._call(self.lib.particle_volume_integrals_ellipsoid, self.handle, ctypes.byref(g), _ptr(u), P,
                   _ptr(Xr), _ptr(axes), _ptr(Iu), _ptr(Irxu), _ptr(vol), _stream(stream))
        return Iu, Irxu, vol

    def particle_drag_force(self, F_ib, Iu_new, Iu_old, rho_f, dt, out=None, stream=None):
        """F_D[P,3] of Eq. FD = F_ib + rho_f (Iu_new - Iu_old) / dt."""
        P = F_ib.shape[0]
        for t, nm in ((F_ib, "F_ib"), (Iu_new, "Iu_new"), (Iu_old, "Iu_old")):
            _need(t, nm, torch.float64, (P, 3))
        if out is None:
            out = torch.empty((P, 3), dtype=torch.float64, device=F_ib.device)
        _need(out, "F_D", torch.float64, (P, 3))
        self._call(self.lib.particle_drag_force, self.handle, P, _ptr(F_ib), _ptr(Iu_new), _ptr(Iu_old),
                   float(rho_f), float(dt), _ptr(out), _stream(stream))
        return out

    def particle_force_torque(self, parts, marks, F, rho_f, out=None, stream=None):
        """(F_ib[P,3], T_ib[P,3]) = (-rho_f sum F dV, -rho_f sum R x F dV)."""
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        ms = self.markers_struct(marks["R"], marks["dV"])
        _need(F, "F", torch.float64, (ms.M, 3))
        P = ps.P
        if out is None:
            out = (torch.empty((P, 3), dtype=torch.float64, device=F.device),
                   torch.empty((P, 3), dtype=torch.float64, device=F.device))
        Fib, Tib = out
        _need(Fib, "F_ib", torch.float64, (P, 3))
        _need(Tib, "T_ib", torch.float64, (P, 3))
        self._call(self.lib.particle_force_torque, self.handle, ctypes.byref(ps), ctypes.byref(ms),
                   _ptr(F), float(rho_f), _ptr(Fib), _ptr(Tib), _stream(stream))
        return Fib, Tib

    def particle_collide_update(self, parts, n, h, phys, dt, F_ib, T_ib, Iu_new, Iu_old,
                                Irxu_new, Irxu_old, Fc_out=None, origin=(0.0, 0.0, 0.0),
                                stream=None):
        """Collision + Newton-Euler + centroid update, in place on parts['Xr','Ur','Wr'].

        ``phys`` = (rho_f, gx, gy, gz, g_coll, eps_c, d_c).
        """
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        P = ps.P
        for t, nm in ((F_ib, "F_ib"), (T_ib, "T_ib"), (Iu_new, "Iu_new"), (Iu_old, "Iu_old"),
                      (Irxu_new, "Irxu_new"), (Irxu_old, "Irxu_old")):
            _need(t, nm, torch.float64, (P, 3))
        if Fc_out is not None:
            _need(Fc_out, "Fc_out", torch.float64, (P, 3))
        ph = _phys_struct(phys)
        g = make_grid(n, h, origin, IB_F64)
        self._call(self.lib.particle_collide_update, self.handle, ctypes.byref(ps), ctypes.byref(g),
                   ctypes.byref(ph), float(dt), _ptr(F_ib), _ptr(T_ib), _ptr(Iu_new), _ptr(Iu_old),
                   _ptr(Irxu_new), _ptr(Irxu_old), _ptr(Fc_out), _stream(stream))
        return Fc_out

    def ib_batch_multidirect_forcing(self, fields, hs, parts, marks, ranges, Ns, dt, origins=None,
                                     delta=ROMA3, order=SEQUENTIAL, F_out=None, f_outs=None,
                                     stream=None):
        """Algorithm 1 on every case of a batch, in place on ``fields``.

        ``parts``/``marks`` are the flat particle and marker sets of the
        batch (see :func:`pack_batch`); ``ranges[c]`` = (p_begin, p_end).
        Returns F_out[M,3] over the flat markers.
        """
        cases = case_array(fields, hs, ranges, origins, f_outs)
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        ms = self.markers_struct(marks["R"], marks["dV"])
        if F_out is None:
            F_out = torch.empty((ms.M, 3), dtype=torch.float64, device=parts["Xr"].device)
        _need(F_out, "F_out", torch.float64, (ms.M, 3))
        self._call(self.lib.ib_batch_multidirect_forcing, self.handle, len(cases), cases,
                   ctypes.byref(ps), ctypes.byref(ms), int(Ns), float(dt), int(delta), int(order),
                   _ptr(F_out), _stream(stream))
        return F_out

    def ib_batch_volume_integrals(self, fields, hs, parts, ranges, origins=None, out=None,
                                  stream=None):
        """(Iu, Irxu, vol) of every particle of a batch in its case's field."""
        cases = case_array(fields, hs, ranges, origins)
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        P = ps.P
        dev = parts["Xr"].device
        if out is None:
            out = (torch.empty((P, 3), dtype=torch.float64, device=dev),
                   torch.empty((P, 3), dtype=torch.float64, device=dev),
                   torch.empty((P,), dtype=torch.float64, device=dev))
        Iu, Irxu, vol = out
        _need(Iu, "Iu", torch.float64, (P, 3))
        _need(Irxu, "Irxu", torch.float64, (P, 3))
        _need(vol, "vol", torch.float64, (P,))
        self._call(self.lib.ib_batch_volume_integrals, self.handle, len(cases), cases, ctypes.byref(ps),
                   _ptr(Iu), _ptr(Irxu), _ptr(vol), _stream(stream))
        return Iu, Irxu, vol

    def ib_batch_collide_update(self, parts, shapes, hs, ranges, phys, dt, F_ib, T_ib, Iu_new,
                                Iu_old, Irxu_new, Irxu_old, Fc_out=None, origins=None, stream=None):
        """Collision within each case + Newton-Euler, in place on the flat set.

        ``shapes[c]`` = (n0, n1, n2) of case c's periodic box; ``phys`` is one
        (rho_f, gx, gy, gz, g_coll, eps_c, d_c) per case, or one for all.
        """
        cases = case_array(None, hs, ranges, origins, shapes=shapes)
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        P = ps.P
        for t, nm in ((F_ib, "F_ib"), (T_ib, "T_ib"), (Iu_new, "Iu_new"), (Iu_old, "Iu_old"),
                      (Irxu_new, "Irxu_new"), (Irxu_old, "Irxu_old")):
            _need(t, nm, torch.float64, (P, 3))
        if Fc_out is not None:
            _need(Fc_out, "Fc_out", torch.float64, (P, 3))
        per_case = phys if len(phys) == len(cases) and not isinstance(phys[0], (int, float)) else \
            [phys] * len(cases)
        ph = (Phys * len(cases))(*[_phys_struct(x) for x in per_case])
        self._call(self.lib.ib_batch_collide_update, self.handle, len(cases), cases, ctypes.byref(ps),
                   ph, float(dt), _ptr(F_ib), _ptr(T_ib), _ptr(Iu_new), _ptr(Iu_old),
                   _ptr(Irxu_new), _ptr(Irxu_old), _ptr(Fc_out), _stream(stream))
        return Fc_out

    def ib_batch_table_multidirect_forcing(self, table, parts, marks, Ns, dt, delta=ROMA3,
                                           order=SEQUENTIAL, F_out=None, stream=None):
        """Algorithm 1 on every case of a prepared batch (see :class:`BatchTable`)."""
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        ms = self.markers_struct(marks["R"], marks["dV"])
        if F_out is None:
            F_out = torch.empty((ms.M, 3), dtype=torch.float64, device=parts["Xr"].device)
        _need(F_out, "F_out", torch.float64, (ms.M, 3))
        self._call(self.lib.ib_batch_table_multidirect_forcing, self.handle, table.handle, ctypes.byref(ps),
                   ctypes.byref(ms), int(Ns), float(dt), int(delta), int(order), _ptr(F_out), _stream(stream))
        return F_out

    def ib_batch_table_volume_integrals(self, table, parts, out=None, stream=None):
        """(Iu, Irxu, vol) of every particle of a prepared batch."""
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        P, dev = ps.P, parts["Xr"].device
        if out is None:
            out = (torch.empty((P, 3), dtype=torch.float64, device=dev),
                   torch.empty((P, 3), dtype=torch.float64, device=dev),
                   torch.empty((P,), dtype=torch.float64, device=dev))
        Iu, Irxu, vol = out
        _need(Iu, "Iu", torch.float64, (P, 3))
        _need(Irxu, "Irxu", torch.float64, (P, 3))
        _need(vol, "vol", torch.float64, (P,))
        self._call(self.lib.ib_batch_table_volume_integrals, self.handle, table.handle, ctypes.byref(ps),
                   _ptr(Iu), _ptr(Irxu), _ptr(vol), _stream(stream))
        return Iu, Irxu, vol

    def ib_batch_table_collide_update(self, table, parts, dt, F_ib, T_ib, Iu_new, Iu_old, Irxu_new,
                                      Irxu_old, Fc_out=None, stream=None):
        """Collision within each case + Newton-Euler on a prepared batch."""
        ps = self.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                   parts["rho_p"], parts["moff"])
        P = ps.P
        for t, nm in ((F_ib, "F_ib"), (T_ib, "T_ib"), (Iu_new, "Iu_new"), (Iu_old, "Iu_old"),
                      (Irxu_new, "Irxu_new"), (Irxu_old, "Irxu_old")):
            _need(t, nm, torch.float64, (P, 3))
        if Fc_out is not None:
            _need(Fc_out, "Fc_out", torch.float64, (P, 3))
        self._call(self.lib.ib_batch_table_collide_update, self.handle, table.handle, ctypes.byref(ps),
                   float(dt), _ptr(F_ib), _ptr(T_ib), _ptr(Iu_new), _ptr(Iu_old), _ptr(Irxu_new),
                   _ptr(Irxu_old), _ptr(Fc_out), _stream(stream))
        return Fc_out


class PvfPlan:
    """Device lists of a kept volume plan (``ib_pvf_plan_create``): up to P
    particles whose stencil boxes have at most ``max_box_cells`` cells."""

    def __init__(self, ctx, P, max_box_cells):
        self.lib = ctx.lib
        h = ctypes.c_void_p()
        rc = self.lib.ib_pvf_plan_create(ctx.handle, int(P), int(max_box_cells), ctypes.byref(h))
        if rc != IB_OK:
            raise IBError(rc, self.lib.ib_last_error().decode())
        self.handle = h
        self.P = int(P)

    def close(self):
        if self.handle:
            self.lib.ib_pvf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchTable:
    """A batch's case table uploaded once (``ib_batch_table_create``): the
    ``ib_batch_table_*`` calls that take it stage nothing on the host, so they
    can be captured into a CUDA graph.  It serves exactly the given fields
    and particle ranges; ``fields`` are kept referenced while it lives.
    ``phys`` (one tuple per case, or one for all) is needed only by the
    collision update."""

    def __init__(self, ctx, fields, hs, ranges, P, phys=None, origins=None, f_outs=None):
        self.lib = ctx.lib
        self._keep = (list(fields), list(f_outs) if f_outs is not None else None)
        cases = case_array(fields, hs, ranges, origins, f_outs)
        ph = None
        if phys is not None:
            per_case = phys if len(phys) == len(cases) and not isinstance(phys[0], (int, float)) else \
                [phys] * len(cases)
            ph = (Phys * len(cases))(*[_phys_struct(x) for x in per_case])
        h = ctypes.c_void_p()
        rc = self.lib.ib_batch_table_create(ctx.handle, len(cases), cases, int(P), ph, ctypes.byref(h))
        if rc != IB_OK:
            raise IBError(rc, self.lib.ib_last_error().decode())
        self.handle = h
        self.P = int(P)
        self.ncases = len(cases)

    def update(self, fields, hs, ranges, P, phys=None, origins=None, f_outs=None, stream=None):
        """Point the table at another batch: an asynchronous upload on
        ``stream`` (see ``ib_batch_table_update``)."""
        cases = case_array(fields, hs, ranges, origins, f_outs)
        ph = None
        if phys is not None:
            per_case = phys if len(phys) == len(cases) and not isinstance(phys[0], (int, float)) else \
                [phys] * len(cases)
            ph = (Phys * len(cases))(*[_phys_struct(x) for x in per_case])
        rc = self.lib.ib_batch_table_update(self.handle, len(cases), cases, int(P), ph, _stream(stream))
        if rc != IB_OK:
            raise IBError(rc, self.lib.ib_last_error().decode())
        self._keep = (list(fields), list(f_outs) if f_outs is not None else None)
        self.P = int(P)
        self.ncases = len(cases)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.ib_batch_table_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _phys_struct(phys):
    ph = Phys()
    ph.rho_f = float(phys[0])
    for a in range(3):
        ph.g[a] = float(phys[1 + a])
    ph.g_coll, ph.eps_c, ph.d_c = float(phys[4]), float(phys[5]), float(phys[6])
    return ph


def case_array(fields, hs, ranges, origins=None, f_outs=None, shapes=None):
    """ctypes ``ib_case[]`` of a batch.

    ``fields[c]`` is case c's field [3, n2, n1, n0] (or None with ``shapes[c]``
    = (n0, n1, n2) where no field is read), ``hs[c]`` its spacing and
    ``ranges[c]`` = (p_begin, p_end) its particles in the flat set.
    """
    nc = len(ranges)
    arr = (Case * nc)()
    for c in range(nc):
        u = fields[c] if fields is not None else None
        if u is not None:
            n = (u.shape[3], u.shape[2], u.shape[1])
            _need(u, "fields[%d]" % c, u.dtype, (3, n[2], n[1], n[0]))
            prec = IB_F64 if u.dtype == torch.float64 else IB_F32
        else:
            n, prec = shapes[c], IB_F64
        f = f_outs[c] if f_outs is not None else None
        if f is not None:
            _need(f, "f_outs[%d]" % c, u.dtype, tuple(u.shape))
        arr[c].grid = make_grid(n, hs[c], origins[c] if origins is not None else (0.0, 0.0, 0.0), prec)
        arr[c].u = u.data_ptr() if u is not None else None
        arr[c].f_out = f.data_ptr() if f is not None else None
        arr[c].p_begin, arr[c].p_end = int(ranges[c][0]), int(ranges[c][1])
    return arr


def pack_batch(parts_list, marks_list):
    """Concatenate per-case particle/marker dicts into one flat set.

    Returns (parts, marks, ranges, mranges): marker offsets are shifted to
    index the flat marker arrays; ``ranges[c]`` / ``mranges[c]`` are case c's
    particle and marker index ranges.
    """
    keys = ("Xr", "Ur", "Wr", "radius", "rho_p")
    parts = {k: torch.cat([p[k] for p in parts_list]).contiguous() for k in keys}
    offs, ranges, mranges = [], [], []
    pb = mb = 0
    for p, m in zip(parts_list, marks_list):
        P, M = p["Xr"].shape[0], m["R"].shape[0]
        offs.append(p["moff"][:P] + mb)
        ranges.append((pb, pb + P))
        mranges.append((mb, mb + M))
        pb += P
        mb += M
    dev = parts_list[0]["Xr"].device
    offs.append(torch.tensor([mb], dtype=torch.int32, device=dev))
    parts["moff"] = torch.cat(offs).to(torch.int32).contiguous()
    marks = {k: torch.cat([m[k] for m in marks_list]).contiguous() for k in ("R", "dV")}
    return parts, marks, ranges, mranges


def device_case(case, prec=IB_F64, device="cuda"):
    """Copy a :class:`synth.Case` to the device: returns (u, parts, marks).

    ``u`` has the field dtype of ``prec``; particle and marker arrays are
    float64 (offsets int32), as the C ABI expects.
    """
    dt = field_dtype(prec)

    def t(a, dtype=torch.float64):
        return torch.as_tensor(a).to(device=device, dtype=dtype).contiguous()

    u = t(case.u, dt)
    parts = dict(Xr=t(case.Xr), Ur=t(case.Ur), Wr=t(case.Wr), radius=t(case.radius),
                 rho_p=t(case.rho_p), moff=t(case.moff, torch.int32))
    marks = dict(R=t(case.R), dV=t(case.dV))
    return u, parts, marks
