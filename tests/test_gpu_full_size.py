"""Full-size GPU parity against the FP64 oracle.

* The benchmark's workload (256^3 periodic grid, 64 spheres of D = 24 cells,
  115,840 markers, Ns = 5, sequential order) in FP64 and FP32 fields, through
  each way the library can run the forcing passes: the particle-resident
  kernel eagerly and as a CUDA-graph replay, and the wavefront form's first
  call on a context (persistent kernel), a later call (per-wavefront
  kernels) and a CUDA-graph replay of the later call (the form bench.py
  times).
* The dense 384^3 case (512 spheres of D = 16 at volume fraction 0.3, Ns = 3,
  FP32 fields) with active collisions, through a whole hot-path step.

Every output array is compared element by element; gates 1e-12 (FP64) and
2e-5 (FP32) normwise, as in the other parity tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_14140_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = {0: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def api():
    from paper_2408_14140_gb300 import api as a
    from paper_2408_14140_gb300 import build
    build.build()
    return a


def nerr(g, o):
    g = g.detach().double().cpu().numpy() if isinstance(g, torch.Tensor) else np.asarray(g)
    o = np.asarray(o)
    return float(np.max(np.abs(g - o)) / max(np.max(np.abs(o)), 1e-300))


def host_field(case, prec):
    u = synth.fourier_eval_torch(case.n, case.meta["modes"], case.h, case.org, device="cuda")
    if prec == 1:
        u = u.float().double()
    return u.cpu().numpy()


@pytest.fixture(scope="module")
def cluster256():
    case = synth.cluster_case(N=256, P=64, D_cells=24, phi=0.2, K=32, Ns=5, seed=0, build_field=False)
    return case


@pytest.mark.parametrize("prec", [0, 1])
def test_mdf_bench_workload_all_paths(api, cluster256, prec):
    case = cluster256
    u_host = host_field(case, prec)
    un, Fo, _ = oracle.multidirect(case.n, case.h, case.org, u_host, case.Xr, case.Ur, case.Wr,
                                   case.moff, case.R, case.dV, case.Ns, case.dt)
    ctx = api.Context()
    dt = api.field_dtype(prec)
    u0 = torch.tensor(u_host, device="cuda", dtype=dt)
    _, parts, marks = api.device_case(case.__class__(**{**case.__dict__, "u": np.zeros((3, 1, 1, 1))}),
                                      prec)
    F = torch.zeros((case.M, 3), dtype=torch.float64, device="cuda")
    results = []
    u = u0.clone()

    def call(name):
        u.copy_(u0)
        ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt, F_out=F)
        ctx.status()
        results.append((name, u.clone(), F.clone()))

    def graph_replay(name):
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            u.copy_(u0)
            ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt, F_out=F)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt, F_out=F)
        u.copy_(u0)
        g.replay()
        torch.cuda.synchronize()
        ctx.status()
        results.append((name, u.clone(), F.clone()))

    ctx.set_pass_kernels("resident")
    call("resident")
    graph_replay("resident, graph replay")
    ctx.set_pass_kernels("groups")
    call("groups")
    graph_replay("groups, graph replay")
    ctx.set_pass_kernels("wavefront")
    call("persistent")          # first wavefront-form call: all wavefronts in the persistent kernel
    call("wavefront kernels")   # later call: the wavefronts as separate kernels
    graph_replay("wavefront kernels, graph replay")
    for name, ug, Fg in results:
        assert nerr(ug, un) <= TOL[prec], name
        assert nerr(Fg, Fo) <= TOL[prec], name
    # every path agrees bitwise
    for name, ug, Fg in results[1:]:
        assert torch.equal(ug, results[0][1]) and torch.equal(Fg, results[0][2]), name
    ctx.close()


def test_full_step_dense_cluster_384(api):
    """384^3, 512 spheres of D = 16 at phi = 0.3 (gaps below h: collisions
    active), Ns = 3, FP32 fields: the whole hot-path step against the oracle."""
    case = synth.cluster_case(N=384, P=512, D_cells=16, phi=0.3, K=16, Ns=3, seed=1,
                              min_gap_cells=0.25, build_field=False)
    u_host = host_field(case, 1)
    ctx = api.Context()
    u = torch.tensor(u_host, device="cuda", dtype=torch.float32)
    _, parts, marks = api.device_case(case.__class__(**{**case.__dict__, "u": np.zeros((3, 1, 1, 1))}), 1)
    I0 = ctx.particle_volume_integrals(u, case.h, parts)
    F = ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt)
    Fib, Tib = ctx.particle_force_torque(parts, marks, F, case.rho_f)
    I1 = ctx.particle_volume_integrals(u, case.h, parts)
    Fc = torch.zeros((case.P, 3), dtype=torch.float64, device="cuda")
    ctx.particle_collide_update(parts, case.n, case.h, case.phys(), case.dt, Fib, Tib, I1[0], I0[0],
                                I1[1], I0[1], Fc_out=Fc)
    ctx.status()

    a0 = oracle.volume_integrals(case.n, case.h, case.org, u_host, case.Xr, case.radius)
    un, Fo, _ = oracle.multidirect(case.n, case.h, case.org, u_host, case.Xr, case.Ur, case.Wr,
                                   case.moff, case.R, case.dV, case.Ns, case.dt)
    fo, to = oracle.force_torque(case.moff, case.R, case.dV, Fo, case.rho_f)
    a1 = oracle.volume_integrals(case.n, case.h, case.org, un, case.Xr, case.radius)
    X, U, W, Fco = oracle.collide_update(case.Xr, case.Ur, case.Wr, case.radius, case.rho_p, case.n,
                                         case.h, case.phys(), case.dt, fo, to, a1[0], a0[0], a1[1],
                                         a0[1])
    assert np.count_nonzero(np.any(Fco != 0, axis=1)) > 10  # collisions are active
    assert nerr(u, un) <= 2e-5
    assert nerr(F, Fo) <= 2e-5
    assert nerr(I0[0], a0[0]) <= 1e-12 and nerr(I0[1], a0[1]) <= 1e-12 and nerr(I0[2], a0[2]) <= 1e-12
    assert nerr(I1[0], a1[0]) <= 2e-5 and nerr(I1[2], a1[2]) <= 1e-12
    assert nerr(Fib, fo) <= 2e-5 and nerr(Tib, to) <= 2e-5
    assert nerr(Fc, Fco) <= 1e-12
    # X^{n+1} = X^n + dt/2 (U^{n+1} + U^n): an FP32-level error in U^{n+1} moves
    # X by at most dt/2 times that error
    tol_x = 2e-5 * 0.5 * case.dt * np.max(np.abs(U)) / np.max(np.abs(X)) + 1e-14
    assert nerr(parts["Xr"], X) <= tol_x
    assert nerr(parts["Ur"], U) <= 2e-5
    assert nerr(parts["Wr"], W) <= 2e-5
    ctx.close()
