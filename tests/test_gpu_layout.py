"""Layout choices leave results unchanged: the wavefront gather's CTAs per SM
and its per-tile staging capacity (ib_ctx_set_gather) change which CTA sums
which tile and whether its candidates come from shared memory, never a sum."""
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


@pytest.mark.parametrize("prec", [0, 1])
def test_gather_layout_keeps_results_bitwise(api, prec):
    # dense small spheres: tiles with more candidates than the small capacities
    case = synth.cluster_case(N=64, P=24, D_cells=10, phi=0.3, K=6, Ns=3, seed=12, min_gap_cells=0.25)
    outs = []
    for ctas, stage in ((0, 0), (2, 64), (1, 32), (4, 128)):
        ctx = api.Context()
        ctx.set_gather(ctas, stage)
        for _ in range(2):  # the second call runs the wavefront gather kernels
            u, parts, marks = api.device_case(case, prec)
            f = torch.zeros_like(u)
            F = ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt, f_out=f)
        ctx.status()
        outs.append((u, F, f))
        ctx.close()
    for out in outs[1:]:
        for a, b in zip(out, outs[0]):
            assert torch.equal(a, b)


def test_gather_layout_rejects_bad_values(api):
    ctx = api.Context()
    for ctas, stage in ((-1, 0), (0, 48), (0, 512), (33, 0)):
        with pytest.raises(api.IBError) as e:
            ctx.set_gather(ctas, stage)
        assert e.value.code == api.IB_ERR_INVALID
    ctx.close()
