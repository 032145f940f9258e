"""The allocation-free volume-integral entry point against the regular one.

particle_volume_integrals_static serves callers that cannot allocate device
memory (stream capture, latency-critical loops, hosts whose device memory
belongs to another allocator): it keeps its scratch in a fixed array inside
the library instead of a context workspace.  This file is named to be
collected last so that a run stopping at its first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2408_14140_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2408_14140_gb300 import api as a
    from paper_2408_14140_gb300 import build
    build.build()
    a.load()
    return a


def static_call(api, u, h, parts, out):
    lib = api.load()
    n = (u.shape[3], u.shape[2], u.shape[1])
    g = api.make_grid(n, h, (0.0, 0.0, 0.0), api.IB_F64 if u.dtype == torch.float64 else api.IB_F32)
    ps = api.Context.particles_struct(parts["Xr"], parts["Ur"], parts["Wr"], parts["radius"],
                                      parts["rho_p"], parts["moff"])
    Iu, Irxu, vol = out
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.particle_volume_integrals_static(ctypes.byref(g), ctypes.c_void_p(u.data_ptr()),
                                                ctypes.byref(ps), ctypes.c_void_p(Iu.data_ptr()),
                                                ctypes.c_void_p(Irxu.data_ptr()),
                                                ctypes.c_void_p(vol.data_ptr()), stream)


def nerr(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", [0, 1])
def test_static_matches_context_version_twice(api, prec):
    ctx = api.Context()
    cases = [synth.cluster_case(N=64, P=10, D_cells=12, phi=0.2, K=5, Ns=3, seed=31),
             synth.cluster_case(N=48, P=3, D_cells=9, phi=0.1, K=3, Ns=3, seed=32)]
    for case in cases:  # two calls in a row, different sizes: no stale scratch
        u, parts, _ = api.device_case(case, prec)
        ref = ctx.particle_volume_integrals(u, case.h, parts)
        out = tuple(torch.full_like(t, float("nan")) for t in ref)
        rc = static_call(api, u, case.h, parts, out)
        assert rc == api.IB_OK, api.load().ib_last_error()
        torch.cuda.synchronize()
        for a, b in zip(out, ref):
            assert nerr(a, b) <= 1e-12
        # the static call's slab split is fixed at 8 CTAs per particle: a
        # context call with the same split runs the same sums bit for bit
        ctx.set_volume_split(8)
        ref8 = ctx.particle_volume_integrals(u, case.h, parts)
        ctx.set_volume_split(0)
        out8 = tuple(torch.full_like(t, float("nan")) for t in ref)
        assert static_call(api, u, case.h, parts, out8) == api.IB_OK
        torch.cuda.synchronize()
        for a, b in zip(out8, ref8):
            assert torch.equal(a, b)
    ctx.close()


def test_static_rejects_too_many_particles(api):
    P = 2049  # IB_STATIC_VOLUME_MAX_P + 1
    u = torch.zeros((3, 16, 16, 16), device="cuda", dtype=torch.float64)
    z3 = torch.zeros((P, 3), device="cuda", dtype=torch.float64)
    parts = dict(Xr=z3, Ur=z3, Wr=z3, radius=torch.full((P,), 0.1, device="cuda", dtype=torch.float64),
                 rho_p=torch.ones(P, device="cuda", dtype=torch.float64),
                 moff=torch.zeros(P + 1, device="cuda", dtype=torch.int32))
    out = (z3.clone(), z3.clone(), torch.zeros(P, device="cuda", dtype=torch.float64))
    rc = static_call(api, u, 1 / 16, parts, out)
    assert rc == api.IB_ERR_INVALID
    assert b"exceeds the fixed maximum 2048" in api.load().ib_last_error()
