"""GPU parity of the fluid step around the forcing (Sec. 3.1 Steps 1 and 3)
against the FP64 oracle (oracle/fluid.py), and a full single-level step --
predictor, multidirect forcing, projection -- against the oracle's chain.

Gates: normwise max|gpu - oracle| / max|oracle| <= 1e-12 with FP64 fields and
<= 2e-5 with FP32 fields (the oracle then takes the FP32-rounded inputs)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fluid
from paper_2408_14140_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def api():
    from paper_2408_14140_gb300 import api as a
    from paper_2408_14140_gb300 import build
    build.build()
    return a


def nerr(g, o):
    g = g.detach().double().cpu().numpy() if isinstance(g, torch.Tensor) else np.asarray(g)
    return float(np.max(np.abs(g - o)) / max(np.max(np.abs(o)), 1e-300))


def inputs(n, prec, seed):
    """A Fourier-mode velocity (cells) and a smooth nodal pressure, rounded to
    the field precision; returned as FP64 numpy arrays of those values."""
    rng = synth.SplitMix64(seed)
    h = 1.0 / n[0]
    u = synth.fourier_field(n, 6, rng, h)
    p = 0.3 * synth.fourier_field(n, 4, rng, h)[0]
    if prec == 1:
        u = u.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    return h, u, p


@pytest.mark.parametrize("prec", [0, 1])
def test_predictor_matches_oracle(api, prec):
    n = (32, 16, 64)  # ragged powers of two
    h, u, p = inputs(n, prec, 3)
    rho, mu, g, dt = 1.2, 0.03, (0.0, -1.0, -9.81), 2e-3
    ref = fluid.predictor(u, p, rho, mu, g, dt, h)
    dtype = api.field_dtype(prec)
    ctx = api.Context()
    us = ctx.fluid_predictor(torch.tensor(u, device="cuda", dtype=dtype), torch.tensor(p, device="cuda", dtype=dtype),
                             h, rho, mu, g, dt)
    ctx.status()
    assert nerr(us, ref) <= TOL[prec]
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_projection_matches_oracle_and_is_divergence_free(api, prec):
    n = (16, 32, 32)
    h, u, p = inputs(n, prec, 4)
    rho, dt = 0.9, 1e-3
    u_ref, p_ref = fluid.projection(u, p, rho, dt, h)
    dtype = api.field_dtype(prec)
    ctx = api.Context()
    ug = torch.tensor(u, device="cuda", dtype=dtype)
    pg = torch.tensor(p, device="cuda", dtype=dtype)
    ctx.level_projection(ug, pg, h, rho, dt)
    ctx.status()
    assert nerr(ug, u_ref) <= TOL[prec]
    # the pressure is defined up to its mean (and the null modes, zero in both)
    pn, pr = pg.double().cpu().numpy(), p_ref
    assert nerr(pn - pn.mean(), pr - pr.mean()) <= TOL[prec]
    # D u^{n+1} = 0 up to the rounding of the stored u: each of D's three
    # terms is (1/4h) times four differences, so |D e| <= 6 max|e| / h, and
    # the stored u carries a few units of rounding of max|u| (a factor 4 here)
    eps = np.finfo(np.float64 if prec == 0 else np.float32).eps
    div = fluid.div_cell_to_node(ug.double().cpu().numpy(), h)
    assert np.max(np.abs(div)) <= 6 * 4 * eps * np.max(np.abs(u_ref)) / h
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_full_single_level_step_matches_oracle(api, prec):
    """u^n -> predictor (Step 1) -> multidirect forcing (Step 2) -> projection
    (Step 3), one sphere of D = 10 cells in a 32^3 periodic box."""
    case = synth.cluster_case(N=32, P=2, D_cells=10, phi=0.05, K=5, Ns=2, seed=9)
    n, h = case.n, case.h
    u = case.u if prec == 0 else case.u.astype(np.float32).astype(np.float64)
    p = np.zeros((n[2], n[1], n[0]))
    rho, mu, g, dt = 1.0, 0.01, (0.0, 0.0, 0.0), case.dt
    # oracle chain
    us = fluid.predictor(u, p, rho, mu, g, dt, h)
    if prec == 1:
        us = us.astype(np.float32).astype(np.float64)
    un, Fo, _ = oracle.multidirect(n, h, case.org, us, case.Xr, case.Ur, case.Wr, case.moff, case.R, case.dV,
                                   case.Ns, dt)
    u1, p1 = fluid.projection(un, p, rho, dt, h)
    # GPU chain
    dtype = api.field_dtype(prec)
    ctx = api.Context()
    ug = torch.tensor(u, device="cuda", dtype=dtype)
    pg = torch.zeros((n[2], n[1], n[0]), device="cuda", dtype=dtype)
    usg = ctx.fluid_predictor(ug, pg, h, rho, mu, g, dt)
    _, parts, marks = api.device_case(case.__class__(**{**case.__dict__, "u": np.zeros((3, 1, 1, 1))}), prec)
    F = ctx.ib_multidirect_forcing(usg, h, parts, marks, case.Ns, dt)
    ctx.level_projection(usg, pg, h, rho, dt)
    ctx.status()
    assert nerr(F, Fo) <= TOL[prec]
    assert nerr(usg, u1) <= TOL[prec]
    ctx.close()


def test_fluid_step_rejects_other_grid_sizes(api):
    ctx = api.Context()
    u = torch.zeros((3, 24, 32, 32), device="cuda", dtype=torch.float64)  # n2 = 24
    p = torch.zeros((24, 32, 32), device="cuda", dtype=torch.float64)
    with pytest.raises(api.IBError) as e:
        ctx.level_projection(u, p, 1 / 32, 1.0, 1e-3)
    assert e.value.code == api.IB_ERR_UNSUPPORTED
    ctx.close()
