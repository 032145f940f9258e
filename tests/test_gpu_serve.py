"""The request loop on the device: every request completes, each result is
the same alone and in the mix, and a served request matches the oracle's
time steps.

A short Poisson trace of small uneven cases (FP32 and FP64 fields mixed)
runs through the continuous-batching server; requests arrive while others
are on the device and share its batch launches.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_14140_gb300 import api, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 2], ids=["eager", "graph-replay"])
def served(request):
    """The trace served with eager launches, and with each precision's step
    replayed from a CUDA graph once its active set held for two steps."""
    from paper_2408_14140_gb300 import build
    build.build()
    cfg = serve.ServeConfig(rate=150.0, seconds=0.25, grids=(48, 64), P_max=6, D_lo=8.0, D_hi=14.0,
                            steps=4, fp64_fraction=0.3, budget_bytes=8 << 30, max_active=16, seed=5,
                            graph_after=request.param)
    trace = serve.make_trace(cfg)
    srv = serve.Server(cfg)
    srv.run(trace)
    srv.close()
    return cfg, trace, srv


def test_every_request_completes(served):
    cfg, trace, srv = served
    assert len(trace) > 10
    assert all(r.latency is not None and r.latency > 0 for r in trace)
    assert srv.active_peak > 1  # requests overlapped on the device
    assert srv.used == 0
    s = serve.summarize(trace, cfg, max(r.done_time for r in trace))
    assert s["completed"] == len(trace) and s["p99_ms"] >= s["p50_ms"] > 0


def test_result_alone_equals_result_in_the_mix(served):
    cfg, trace, _ = served
    picks = [r for r in trace if r.prec == api.IB_F64][:1] + [r for r in trace if r.prec == api.IB_F32][:2]
    assert len(picks) == 3
    for r in picks:
        alone = serve.serve_alone(cfg, serve.Request(r.rid, r.arrival, r.case, r.prec))
        for k in ("Xr", "Ur", "Wr"):
            assert torch.equal(alone[k], r.host[k]), (r.rid, k)


def test_served_request_matches_oracle_steps(served):
    cfg, trace, _ = served
    for prec in (api.IB_F64, api.IB_F32):
        r = [r for r in trace if r.prec == prec][0]
        c = r.case
        ubg = synth.taylor_green_field(c.n, cfg.U0, c.h)
        if prec == api.IB_F32:
            ubg = ubg.astype(np.float32).astype(np.float64)
        X, U, W = c.Xr.copy(), c.Ur.copy(), c.Wr.copy()
        phys = c.phys()
        for _ in range(cfg.steps):
            a0 = oracle.volume_integrals(c.n, c.h, c.org, ubg, X, c.radius)
            un, Fo, _ = oracle.multidirect(c.n, c.h, c.org, ubg, X, U, W, c.moff, c.R, c.dV, cfg.Ns, cfg.dt)
            fo, to = oracle.force_torque(c.moff, c.R, c.dV, Fo, phys[0])
            a1 = oracle.volume_integrals(c.n, c.h, c.org, un, X, c.radius)
            X, U, W, _ = oracle.collide_update(X, U, W, c.radius, c.rho_p, c.n, c.h, phys, cfg.dt, fo, to,
                                               a1[0], a0[0], a1[1], a0[1])
        tol = 1e-12 if prec == api.IB_F64 else 2e-5
        for k, o in (("Ur", U), ("Wr", W)):
            g = r.host[k].numpy()
            assert np.max(np.abs(g - o)) / np.max(np.abs(o)) <= tol, (prec, k)
        # positions move by dt/2 (U^{n+1} + U^n) per step: their error is dt times the velocities'
        g = r.host["Xr"].numpy()
        tol_x = tol * cfg.steps * cfg.dt * np.max(np.abs(U)) / np.max(np.abs(X)) + 1e-14
        assert np.max(np.abs(g - X)) / np.max(np.abs(X)) <= tol_x, prec
