"""Prepared batches: the case table uploaded once (ib_batch_table_create).

The ib_batch_table_* calls must compute exactly what the ib_batch_* calls
compute (same kernels: bitwise equal), and because they stage nothing on
the host, a whole batched step of them captured into a CUDA graph must
replay to the same bits as the eager calls.
"""
import pytest
import torch

from paper_2408_14140_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2408_14140_gb300 import api as a
    from paper_2408_14140_gb300 import build
    build.build()
    return a


def uneven_cases(seed, Ns=3):
    rng = synth.SplitMix64(seed)
    shapes = [(48, 3), (32, 1), (64, 4), (48, 2)]
    return [synth.random_case(N, P, 8.0, 16.0 if N > 32 else 12.0, 6, Ns, rng) for N, P in shapes]


class Batch:
    """Device state of one batch: fields, flat particles and markers, outputs."""

    def __init__(self, api, cases, prec):
        self.cases = cases
        us, pl, ml = [], [], []
        for c in cases:
            u, p, m = api.device_case(c, prec)
            us.append(u)
            pl.append(p)
            ml.append(m)
        self.fields = us
        self.parts, self.marks, self.ranges, _ = api.pack_batch(pl, ml)
        self.hs = [c.h for c in cases]
        self.shapes = [c.n for c in cases]
        self.phys = [c.phys() for c in cases]
        P, M = self.parts["Xr"].shape[0], self.marks["R"].shape[0]
        z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")  # noqa: E731
        self.F = z(M, 3)
        self.I0 = (z(P, 3), z(P, 3), z(P))
        self.I1 = (z(P, 3), z(P, 3), z(P))
        self.Fib, self.Tib, self.Fc = z(P, 3), z(P, 3), z(P, 3)
        self.P = P

    def state(self):
        return [t.clone() for t in self.fields] + [self.parts[k].clone() for k in ("Xr", "Ur", "Wr")] + \
            [self.F.clone(), self.Fc.clone()] + [t.clone() for t in self.I0 + self.I1]


def staged_step(ctx, b):
    c0 = b.cases[0]
    ctx.ib_batch_volume_integrals(b.fields, b.hs, b.parts, b.ranges, out=b.I0)
    ctx.ib_batch_multidirect_forcing(b.fields, b.hs, b.parts, b.marks, b.ranges, c0.Ns, c0.dt, F_out=b.F)
    ctx.particle_force_torque(b.parts, b.marks, b.F, 1.0, out=(b.Fib, b.Tib))
    ctx.ib_batch_volume_integrals(b.fields, b.hs, b.parts, b.ranges, out=b.I1)
    ctx.ib_batch_collide_update(b.parts, b.shapes, b.hs, b.ranges, b.phys, c0.dt, b.Fib, b.Tib, b.I1[0],
                                b.I0[0], b.I1[1], b.I0[1], Fc_out=b.Fc)


def table_step(ctx, b, table):
    c0 = b.cases[0]
    ctx.ib_batch_table_volume_integrals(table, b.parts, out=b.I0)
    ctx.ib_batch_table_multidirect_forcing(table, b.parts, b.marks, c0.Ns, c0.dt, F_out=b.F)
    ctx.particle_force_torque(b.parts, b.marks, b.F, 1.0, out=(b.Fib, b.Tib))
    ctx.ib_batch_table_volume_integrals(table, b.parts, out=b.I1)
    ctx.ib_batch_table_collide_update(table, b.parts, c0.dt, b.Fib, b.Tib, b.I1[0], b.I0[0], b.I1[1],
                                      b.I0[1], Fc_out=b.Fc)


@pytest.mark.parametrize("prec", [0, 1])
def test_table_calls_equal_staged_calls_and_replay(api, prec):
    cases = uneven_cases(41 + prec)
    ctx = api.Context()
    staged, eager, graph = Batch(api, cases, prec), Batch(api, cases, prec), Batch(api, cases, prec)
    # two steps each: the second starts from the first one's particle state
    for _ in range(2):
        staged_step(ctx, staged)
    table = api.BatchTable(ctx, eager.fields, eager.hs, eager.ranges, eager.P, phys=eager.phys)
    for _ in range(2):
        table_step(ctx, eager, table)
    ctx.status()
    for a, b in zip(staged.state(), eager.state()):
        assert torch.equal(a, b)
    # the same two steps captured once and replayed twice
    gtable = api.BatchTable(ctx, graph.fields, graph.hs, graph.ranges, graph.P, phys=graph.phys)
    init = graph.state()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        table_step(ctx, graph, gtable)  # sizes the workspace outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for t, v in zip(graph.fields + [graph.parts[k] for k in ("Xr", "Ur", "Wr")], init):
        t.copy_(v)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        table_step(ctx, graph, gtable)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    ctx.status()
    for a, b in zip(eager.state(), graph.state()):
        assert torch.equal(a, b)
    table.close()
    gtable.close()
    ctx.close()


def test_table_rejects_mismatches(api):
    cases = uneven_cases(43)
    ctx = api.Context()
    b = Batch(api, cases, 1)
    table = api.BatchTable(ctx, b.fields, b.hs, b.ranges, b.P)  # no physical parameters
    with pytest.raises(api.IBError) as e:
        ctx.ib_batch_table_collide_update(table, b.parts, 1e-3, b.Fib, b.Tib, b.I1[0], b.I0[0], b.I1[1],
                                          b.I0[1])
    assert e.value.code == api.IB_ERR_INVALID
    fewer = {k: v[:-1] for k, v in b.parts.items()}  # P - 1 particles
    with pytest.raises(api.IBError) as e:
        ctx.ib_batch_table_volume_integrals(table, fewer)
    assert e.value.code == api.IB_ERR_INVALID
    with pytest.raises(api.IBError):
        api.BatchTable(ctx, b.fields, b.hs, b.ranges, b.P + 1)  # ranges must end at P
    table.close()
    ctx.close()


def test_table_update_equals_a_fresh_table(api):
    """A table re-pointed at another batch (asynchronous upload on the stream)
    computes exactly what a table created for that batch computes."""
    ctx = api.Context()
    a = Batch(api, uneven_cases(51), 1)
    b1, b2 = Batch(api, uneven_cases(52), 1), Batch(api, uneven_cases(52), 1)
    table = api.BatchTable(ctx, a.fields, a.hs, a.ranges, a.P, phys=a.phys)
    table_step(ctx, a, table)
    table.update(b1.fields, b1.hs, b1.ranges, b1.P, phys=b1.phys)  # on the current stream
    table_step(ctx, b1, table)
    fresh = api.BatchTable(ctx, b2.fields, b2.hs, b2.ranges, b2.P, phys=b2.phys)
    table_step(ctx, b2, fresh)
    ctx.status()
    for x, y in zip(b1.state(), b2.state()):
        assert torch.equal(x, y)
    table.close()
    fresh.close()
    ctx.close()
