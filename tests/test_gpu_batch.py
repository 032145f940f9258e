"""Batches of independent cases through the ib_batch_* entry points.

A batch runs uneven cases -- different grid sizes, particle counts, sphere
diameters, a case with no particles -- through the same launches.  Each
case's outputs must be bitwise those of the single-case entry point on that
case alone (same kernels, same summation orders), and within the FP64 / FP32
gates of the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
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
    o = np.asarray(o)
    return float(np.max(np.abs(g - o)) / max(np.max(np.abs(o)), 1e-300))


def uneven_cases(seed, Ns=3):
    """Grids from {32, 48, 64}, 1-4 spheres of D 8-16 cells each."""
    rng = synth.SplitMix64(seed)
    shapes = [(48, 3), (32, 1), (64, 4), (48, 2), (32, 2)]
    return [synth.random_case(N, P, 8.0, 16.0 if N > 32 else 12.0, 6, Ns, rng) for N, P in shapes]


def empty_case_field(N, prec, seed):
    rng = synth.SplitMix64(seed)
    u = synth.fourier_field((N, N, N), 4, rng, 1.0 / N)
    return torch.tensor(u, device="cuda", dtype=torch.float64 if prec == 0 else torch.float32)


def batch_inputs(api, cases, prec, empty_at=2):
    """Device inputs of the cases, plus a particle-free case inserted at
    ``empty_at`` (its field must come back unchanged)."""
    us, parts_l, marks_l = [], [], []
    for c in cases:
        u, p, m = api.device_case(c, prec)
        us.append(u)
        parts_l.append(p)
        marks_l.append(m)
    parts, marks, ranges, mranges = api.pack_batch(parts_l, marks_l)
    hs = [c.h for c in cases]
    ue = empty_case_field(40, prec, 99)
    b = ranges[empty_at - 1][1] if empty_at > 0 else 0
    us.insert(empty_at, ue)
    hs.insert(empty_at, 1.0 / 40)
    ranges.insert(empty_at, (b, b))
    return us, parts_l, marks_l, parts, marks, ranges, mranges, hs


@pytest.mark.parametrize("prec,order,delta", [(1, 0, 0), (0, 0, 0), (1, 1, 0), (1, 0, 1)])
def test_batch_mdf_equals_each_case_alone(api, prec, order, delta):
    cases = uneven_cases(7 + 10 * prec + order + 3 * delta)
    ctx = api.Context()
    us, parts_l, marks_l, parts, marks, ranges, mranges, hs = batch_inputs(api, cases, prec)
    real = [i for i in range(len(us)) if ranges[i][1] > ranges[i][0]]
    # each case alone
    alone = {}
    for k, i in enumerate(real):
        u = us[i].clone()
        f = torch.zeros_like(u)
        F = ctx.ib_multidirect_forcing(u, hs[i], parts_l[k], marks_l[k], cases[k].Ns, cases[k].dt,
                                       delta=delta, order=order, f_out=f)
        alone[i] = (u, F, f)
    ctx.status()
    # the batch, twice (first call: persistent kernel; second: wavefront kernels)
    for rep in range(2):
        ub = [u.clone() for u in us]
        fb = [torch.zeros_like(u) for u in us]
        Fb = ctx.ib_batch_multidirect_forcing(ub, hs, parts, marks, ranges, cases[0].Ns, cases[0].dt,
                                              delta=delta, order=order, f_outs=fb)
        ctx.status()
        for k, i in enumerate(real):
            u, F, f = alone[i]
            m0, m1 = mranges[k]
            assert torch.equal(ub[i], u), (rep, i)
            assert torch.equal(Fb[m0:m1], F), (rep, i)
            assert torch.equal(fb[i], f), (rep, i)
        e = [i for i in range(len(us)) if i not in real][0]
        assert torch.equal(ub[e], us[e]) and not torch.any(fb[e])
    # and each against the oracle
    for k, i in enumerate(real):
        c = cases[k]
        u_host = us[i].double().cpu().numpy()
        un, Fo, fo = oracle.multidirect(c.n, c.h, c.org, u_host, c.Xr, c.Ur, c.Wr, c.moff, c.R, c.dV,
                                        c.Ns, c.dt, kernel=delta, order=order, want_f=True)
        u, F, f = alone[i]
        assert nerr(u, un) <= TOL[prec]
        assert nerr(F, Fo) <= TOL[prec]
        assert nerr(f, fo) <= TOL[prec]
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_volume_and_collide_equal_each_case_alone(api, prec):
    cases = uneven_cases(41 + prec)
    ctx = api.Context()
    us, parts_l, marks_l, parts, marks, ranges, mranges, hs = batch_inputs(api, cases, prec)
    real = [i for i in range(len(us)) if ranges[i][1] > ranges[i][0]]
    Ib = ctx.ib_batch_volume_integrals(us, hs, parts, ranges)
    ctx.status()
    shapes = [(u.shape[3], u.shape[2], u.shape[1]) for u in us]
    P = parts["Xr"].shape[0]
    g = torch.Generator(device="cpu").manual_seed(5)
    Fib, Tib = (torch.randn((P, 3), generator=g, dtype=torch.float64).cuda() for _ in range(2))
    I0 = tuple(t.clone() for t in Ib[:2])
    I1 = tuple(t * 1.01 for t in Ib[:2])
    # per-case physics: d_c is each case's own h (the particle-free case too)
    phys = [c.phys() for c in cases]
    phys.insert(2, cases[0].phys()[:6] + (1.0 / 40,))
    pb = {k: v.clone() for k, v in parts.items()}
    Fcb = torch.zeros((P, 3), dtype=torch.float64, device="cuda")
    ctx.ib_batch_collide_update(pb, shapes, hs, ranges, phys, cases[0].dt, Fib, Tib, I1[0], I0[0], I1[1],
                                I0[1], Fc_out=Fcb)
    ctx.status()
    for k, i in enumerate(real):
        p0, p1 = ranges[i]
        c = cases[k]
        Ia = ctx.particle_volume_integrals(us[i], hs[i], parts_l[k])
        for a, b in zip(Ia, Ib):
            assert torch.equal(a, b[p0:p1])
        pa = {kk: v.clone() for kk, v in parts_l[k].items()}
        Fca = torch.zeros((p1 - p0, 3), dtype=torch.float64, device="cuda")
        ctx.particle_collide_update(pa, c.n, c.h, c.phys(), c.dt, Fib[p0:p1].contiguous(),
                                    Tib[p0:p1].contiguous(), I1[0][p0:p1].contiguous(),
                                    I0[0][p0:p1].contiguous(), I1[1][p0:p1].contiguous(),
                                    I0[1][p0:p1].contiguous(), Fc_out=Fca)
        ctx.status()
        assert torch.equal(Fca, Fcb[p0:p1])
        for key in ("Xr", "Ur", "Wr"):
            assert torch.equal(pa[key], pb[key][p0:p1]), key
        a = oracle.volume_integrals(c.n, c.h, c.org, us[i].double().cpu().numpy(), c.Xr, c.radius)
        assert nerr(Ia[0], a[0]) <= 1e-12 and nerr(Ia[2], a[2]) <= 1e-12
    ctx.close()


def test_batch_collisions_stay_within_a_case(api):
    """Two cases whose spheres occupy the same coordinates: in one batch they
    must not push each other (pairs are taken within a case only)."""
    c = synth.cluster_case(N=48, P=6, D_cells=10, phi=0.2, K=4, Ns=2, seed=3, min_gap_cells=0.3)
    ctx = api.Context()
    _, p, m = api.device_case(c, 0)
    q = {k: v.clone() for k, v in p.items()}
    q["Xr"] += 0.5 * c.h  # would be overlapping pairs across cases
    parts, marks, ranges, _ = api.pack_batch([p, q], [m, m])
    P = parts["Xr"].shape[0]
    z = torch.zeros((P, 3), dtype=torch.float64, device="cuda")
    Fc = torch.zeros_like(z)
    phys = c.phys()
    ctx.ib_batch_collide_update(parts, [c.n, c.n], [c.h, c.h], ranges, phys, c.dt, z, z, z, z, z, z,
                                Fc_out=Fc)
    ctx.status()
    X, U, W, Fco = oracle.collide_update(c.Xr, c.Ur, c.Wr, c.radius, c.rho_p, c.n, c.h, phys, c.dt,
                                         np.zeros((6, 3)), np.zeros((6, 3)), np.zeros((6, 3)),
                                         np.zeros((6, 3)), np.zeros((6, 3)), np.zeros((6, 3)))
    assert np.any(Fco)  # gaps below d_c = h: collisions are active within the case
    assert nerr(Fc[:6], Fco) <= 1e-12
    assert nerr(parts["Ur"][:6], U) <= 1e-12
    ctx.close()


def test_batch_rejects_bad_ranges_and_mixed_precision(api):
    c = synth.cluster_case(N=32, P=2, D_cells=8, phi=0.1, K=3, Ns=2, seed=4)
    ctx = api.Context()
    u, p, m = api.device_case(c, 0)
    parts, marks, ranges, _ = api.pack_batch([p, p], [m, m])
    u2 = u.clone()
    with pytest.raises(api.IBError) as e:
        ctx.ib_batch_multidirect_forcing([u, u2], [c.h, c.h], parts, marks, [(0, 2), (1, 4)], 2, c.dt)
    assert e.value.code == api.IB_ERR_INVALID and "partition" in str(e.value)
    with pytest.raises(api.IBError) as e:
        ctx.ib_batch_volume_integrals([u, u2], [c.h, c.h], parts, [(0, 2), (2, 3)])
    assert e.value.code == api.IB_ERR_INVALID
    with pytest.raises(api.IBError) as e:
        ctx.ib_batch_multidirect_forcing([u, u2.float()], [c.h, c.h], parts, marks, ranges, 2, c.dt)
    assert e.value.code == api.IB_ERR_INVALID and "mixed" in str(e.value)
    # nothing was written
    assert torch.equal(u, u2)
    ctx.close()


def test_autotune_on_a_batch_keeps_results(api):
    """The tuner times every launch choice on a real batch step and leaves the
    fastest set; the forcing results do not depend on the choice."""
    from paper_2408_14140_gb300 import autotune
    cases = uneven_cases(71)
    ctx = api.Context()
    us, parts_l, marks_l, parts, marks, ranges, mranges, hs = batch_inputs(api, cases, 1)
    base = [u.clone() for u in us]
    outs = {}

    def step():
        for u, b in zip(us, base):
            u.copy_(b)
        ctx.ib_batch_volume_integrals(us, hs, parts, ranges)
        F = ctx.ib_batch_multidirect_forcing(us, hs, parts, marks, ranges, cases[0].Ns, cases[0].dt)
        outs[autotune_key[0]] = ([u.clone() for u in us], F.clone())

    autotune_key = [None]
    for form in ("wavefront", "groups"):
        ctx.set_pass_kernels(form)
        autotune_key[0] = form
        step()
    ctx.status()
    for a, b in zip(outs["wavefront"][0], outs["groups"][0]):
        assert torch.equal(a, b)
    assert torch.equal(outs["wavefront"][1], outs["groups"][1])
    autotune_key[0] = "tuned"
    res = autotune.tune([ctx], step, warmup=1, reps=2, steps_per_rep=1)
    step()  # once more with the tuned choice set
    ctx.status()
    for k, v in res["choice"].items():
        assert v in autotune.SPACE[k]
    assert len(res["table"]) >= 1 + sum(len(v) - 1 for v in autotune.SPACE.values())
    assert all(ms > 0 for _, ms in res["table"])
    for a, b in zip(outs["tuned"][0], outs["wavefront"][0]):
        assert torch.equal(a, b)
    assert torch.equal(outs["tuned"][1], outs["wavefront"][1])
    ctx.close()
