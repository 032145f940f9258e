"""Dense small spheres whose conflict lists overflow (more than 48 earlier
conflicting particles): the wavefront levels then come from the ordered
sweep over full lists instead of the parallel relaxation.  The forcing still
matches the oracle's sequential order, and every pass form agrees bit for bit."""
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


def overflow_case():
    return synth.cluster_case(N=32, P=560, D_cells=3.0, phi=0.3, K=4, Ns=2, seed=11)


def earlier_conflicts(case, kernel_width=3):
    """Conflicts of each particle with earlier ones (the library's test)."""
    rho = np.array([np.max(np.linalg.norm(case.R[case.moff[p]:case.moff[p + 1]], axis=1)) for p in range(case.P)])
    L = np.asarray(case.n) * case.h
    out = []
    for p in range(case.P):
        d = case.Xr[:p] - case.Xr[p]
        d -= L * np.rint(d / L)
        lim = rho[:p] + rho[p] + np.sqrt(3) * kernel_width * case.h + case.h / 16
        out.append(int(np.sum(np.sqrt(np.sum(d * d, axis=1)) < lim)))
    return np.array(out)


def test_case_overflows_the_lists():
    assert np.sum(earlier_conflicts(overflow_case()) > 48) >= 5


def test_overflowing_lists_match_oracle_and_forms(api):
    case = overflow_case()
    u0, parts, marks = api.device_case(case, 0)
    un, Fo, _ = oracle.multidirect(case.n, case.h, case.org, case.u, case.Xr, case.Ur, case.Wr, case.moff,
                                   case.R, case.dV, case.Ns, case.dt)
    out = {}
    for form in ("wavefront", "groups", "resident"):
        ctx = api.Context()
        ctx.set_pass_kernels(form)
        for rep in range(2):  # first call: persistent remainder; second: level kernels
            u = u0.clone()
            F = ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt)
            ctx.status()
            out[(form, rep)] = (u, F)
        ctx.close()
    u, F = out[("wavefront", 1)]
    scale = max(np.max(np.abs(un)), 1e-300)
    assert np.max(np.abs(u.cpu().numpy() - un)) / scale <= 1e-12
    assert np.max(np.abs(F.cpu().numpy() - Fo)) / np.max(np.abs(Fo)) <= 1e-12
    for key, (uu, FF) in out.items():
        assert torch.equal(uu, u), key
        assert torch.equal(FF, F), key
