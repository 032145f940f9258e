"""The forms of the sequential-order passes give bitwise the same result.

The particle-resident kernel (one thread-block cluster per particle, band in
shared memory), the particle-group kernel (a group of CTAs per particle in a
persistent launch) and the wavefront kernels (per wavefront and pass through
global memory) sum every cell and marker in the same order, so u, F and f
agree bit for bit; all stay within the oracle's gates.  Cases cover the
resident fast path, the slow path of particles too large for the cluster's
shared memory, and conflicts between the two.
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
    g = g.detach().double().cpu().numpy()
    o = np.asarray(o)
    return float(np.max(np.abs(g - o)) / max(np.max(np.abs(o)), 1e-300))


def big_and_small(N=96, seed=11):
    """One sphere of D = 44 cells (stencil box beyond the cluster's capacity)
    with small spheres packed around it (their bands overlap its band)."""
    rng = synth.SplitMix64(seed)
    c = np.array([N / 2.0, N / 2.0, N / 2.0])
    cent, radii = [c], [22.0]
    for k in range(6):
        d = np.zeros(3)
        d[k // 2] = (1 if k % 2 == 0 else -1) * (22.0 + 5.0 + 0.6)
        cent.append(c + d)
        radii.append(5.0)
    h = 1.0 / N
    u = synth.fourier_field((N, N, N), 6, rng, h)
    return synth._assemble((N, N, N), h, u, np.array(cent) * h, np.array(radii) * h, rng, 3, 1e-3,
                           meta={"workload": "big+small"})


CASES = {
    "cluster": lambda: synth.cluster_case(N=48, P=6, D_cells=10, phi=0.2, K=6, Ns=3, seed=3),
    "seam": lambda: synth.single_sphere_case(N=48, D_cells=12, K=5, Ns=3, seed=4,
                                             centre=[0.01, 0.995, 0.5 / 48]),
    "dense": lambda: synth.cluster_case(N=64, P=24, D_cells=12, phi=0.25, K=6, Ns=3, seed=6,
                                        min_gap_cells=0.25),
    "big_and_small": big_and_small,
}


def run(api, ctx, case, prec, kernel, u0):
    _, parts, marks = api.device_case(case.__class__(**{**case.__dict__, "u": np.zeros((3, 1, 1, 1))}),
                                      prec)
    u = u0.clone()
    f = torch.zeros_like(u)
    F = ctx.ib_multidirect_forcing(u, case.h, parts, marks, case.Ns, case.dt, delta=kernel,
                                   order=0, f_out=f)
    ctx.status()
    return u, F, f


@pytest.mark.parametrize("form", ["resident", "groups"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,kernel", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_resident_equals_wavefront_and_oracle(api, form, name, prec, kernel):
    case = CASES[name]()
    u0 = torch.tensor(case.u, device="cuda", dtype=api.field_dtype(prec))
    ctx = api.Context()
    ctx.set_pass_kernels(form)
    res = [run(api, ctx, case, prec, kernel, u0) for _ in range(2)]
    ctx.set_pass_kernels("wavefront")
    wav = [run(api, ctx, case, prec, kernel, u0) for _ in range(2)]  # persistent, then per wavefront
    ctx.set_pass_kernels(form)
    res.append(run(api, ctx, case, prec, kernel, u0))
    ref = res[0]
    for out in res[1:] + wav:
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
    un, Fo, fo = oracle.multidirect(case.n, case.h, case.org, u0.double().cpu().numpy(), case.Xr,
                                    case.Ur, case.Wr, case.moff, case.R, case.dV, case.Ns, case.dt,
                                    kernel, 0, want_f=True)
    u, F, f = ref
    assert nerr(u, un) <= TOL[prec]
    assert nerr(F, Fo) <= TOL[prec]
    assert nerr(f, fo) <= TOL[prec]
    ctx.close()
