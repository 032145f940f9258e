"""Failure detection without a GPU fault: a bounded device-side wait that runs
out (on a device word nothing sets) raises IB_ERR_TIMEOUT in the context's
status latch; the host reads it once, the latch clears, and the same context
then runs the method and matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_2408_14140_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2408_14140_gb300 import api as a
    from paper_2408_14140_gb300 import build
    build.build()
    return a


def test_wait_times_out_and_context_survives(api):
    ctx = api.Context()
    ctx.selftest_wait_timeout(1_000_000)  # about half a millisecond
    with pytest.raises(api.IBError) as e:
        ctx.status()
    assert e.value.code == api.IB_ERR_TIMEOUT
    ctx.status()  # read once, then clear
    case = synth.single_sphere_case(N=32, D_cells=8, K=4, Ns=2, seed=6)
    u, parts, marks = api.device_case(case, api.IB_F64)
    F = ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt)
    ctx.status()
    un, Fo, _ = oracle.multidirect(case.n, case.h, case.org, case.u, case.Xr, case.Ur, case.Wr,
                                   case.moff, case.R, case.dV, case.Ns, case.dt)
    assert np.max(np.abs(u.cpu().numpy() - un)) / np.max(np.abs(un)) <= 1e-12
    assert np.max(np.abs(F.cpu().numpy() - Fo)) / np.max(np.abs(Fo)) <= 1e-12
    ctx.close()


def test_selftest_rejects_bad_budgets(api):
    ctx = api.Context()
    for cycles in (0, -5, 5_000_000_000):
        with pytest.raises(api.IBError) as e:
            ctx.selftest_wait_timeout(cycles)
        assert e.value.code == api.IB_ERR_INVALID
    ctx.status()
    ctx.close()
