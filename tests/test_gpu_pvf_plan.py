"""Volume integrals twice at the same particle positions: the keeping call
equals particle_volume_integrals bit for bit; the plan call on another field
sums the kept cells in another order, so it agrees with
particle_volume_integrals on that field to rounding (at the keeping call's
split or another), matches the oracle at the library's gates and is
deterministic, both precisions, under CUDA-graph capture too; and the plan
refuses particles or grids other than its own and boxes beyond its capacity."""
import numpy as np
import pytest
import torch

import oracle
from paper_2408_14140_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2408_14140_gb300 import api as a
    from paper_2408_14140_gb300 import build
    build.build()
    return a


CASES = {
    "cluster": lambda: synth.cluster_case(N=48, P=6, D_cells=10, phi=0.2, K=6, Ns=3, seed=3),
    "dense": lambda: synth.cluster_case(N=64, P=24, D_cells=12, phi=0.25, K=6, Ns=3, seed=6, min_gap_cells=0.25),
    "seam": lambda: synth.single_sphere_case(N=48, D_cells=12, K=5, Ns=2, seed=4, centre=[0.01, 0.995, 0.5 / 48]),
}


def cap_of(case):
    return int(2 * np.max(case.radius) / case.h + 4) ** 3


def equal(a, b):
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def close(a, b, tol):
    """Every output array of a within tol (relative to the array's largest
    magnitude) of b's."""
    for x, y in zip(a, b):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.max(np.abs(x - y)) <= tol * max(np.max(np.abs(y)), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_plan_matches_plain_calls(api, name, prec):
    case = CASES[name]()
    u0, parts, marks = api.device_case(case, prec)
    ctx = api.Context()
    ctx.set_volume_split(3)
    plan = api.PvfPlan(ctx, case.P, cap_of(case))
    kept = ctx.particle_volume_integrals_keep(u0, case.h, parts, plan)
    plain0 = ctx.particle_volume_integrals(u0, case.h, parts)
    # another field at the same positions: the forced field
    u1 = u0.clone()
    ctx.ib_multidirect_forcing(u1, case.h, parts, marks, case.Ns, case.dt)
    planned = ctx.particle_volume_integrals_plan(u1, case.h, parts, plan)
    again = ctx.particle_volume_integrals_plan(u1, case.h, parts, plan)
    plain1 = ctx.particle_volume_integrals(u1, case.h, parts)
    # the plan call at another split than the keeping call's, and automatic
    ctx.set_volume_split(5)
    planned5 = ctx.particle_volume_integrals_plan(u1, case.h, parts, plan)
    ctx.set_volume_split(0)
    planned_auto = ctx.particle_volume_integrals_plan(u1, case.h, parts, plan)
    ctx.set_volume_split(3)
    ctx.status()
    equal(kept, plain0)
    equal(planned, again)
    # the same cells, alpha and per-cell double-float arithmetic in another
    # summation order: rounding-level differences only
    for pl in (planned, planned5, planned_auto):
        close(pl, plain1, 1e-12)
    # and the oracle's integrals of the forced field
    o = oracle.volume_integrals(case.n, case.h, case.org, u1.double().cpu().numpy(), case.Xr, case.radius)
    tol = 1e-12 if prec == 0 else 2e-5
    for pl in (planned, planned5, planned_auto):
        for g, ov in zip(pl, o):
            ov = np.asarray(ov)
            assert np.max(np.abs(g.cpu().numpy() - ov)) <= tol * max(np.max(np.abs(ov)), 1e-300)
    # both calls captured into a CUDA graph and replayed
    outs = [tuple(torch.empty_like(t) for t in kept), tuple(torch.empty_like(t) for t in planned)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ctx.particle_volume_integrals_keep(u0, case.h, parts, plan, out=outs[0])
        ctx.particle_volume_integrals_plan(u1, case.h, parts, plan, out=outs[1])
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.particle_volume_integrals_keep(u0, case.h, parts, plan, out=outs[0])
        ctx.particle_volume_integrals_plan(u1, case.h, parts, plan, out=outs[1])
    for o2 in outs:
        for t in o2:
            t.zero_()
    g.replay()
    torch.cuda.synchronize()
    ctx.status()
    equal(outs[0], plain0)
    equal(outs[1], planned)
    plan.close()
    ctx.close()


def test_plan_refuses_other_particles_grids_and_boxes(api):
    case = CASES["cluster"]()
    u0, parts, _ = api.device_case(case, 0)
    ctx = api.Context()
    plan = api.PvfPlan(ctx, case.P, cap_of(case))
    ctx.particle_volume_integrals_keep(u0, case.h, parts, plan)
    ctx.status()
    moved = dict(parts)
    moved["Xr"] = parts["Xr"] + 1e-3
    ctx.particle_volume_integrals_plan(u0, case.h, moved, plan)
    with pytest.raises(api.IBError) as e:
        ctx.status()
    assert e.value.code == api.IB_ERR_INVALID
    with pytest.raises(api.IBError) as e:
        ctx.particle_volume_integrals_plan(u0, case.h * 1.01, parts, plan)
    assert e.value.code == api.IB_ERR_INVALID
    small = api.PvfPlan(ctx, case.P, 8)
    ctx.particle_volume_integrals_keep(u0, case.h, parts, small)
    with pytest.raises(api.IBError) as e:
        ctx.status()
    assert e.value.code == api.IB_ERR_UNSUPPORTED
    small.close()
    plan.close()
    ctx.close()
