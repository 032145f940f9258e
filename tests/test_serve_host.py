"""Host logic of the request loop: the arrival trace and the admission rule."""
import numpy as np

from paper_2408_14140_gb300 import api, serve


def test_trace_is_seeded_poisson():
    cfg = serve.ServeConfig(rate=200.0, seconds=1.5, P_max=4, grids=(48, 64), seed=3)
    a = serve.make_trace(cfg)
    b = serve.make_trace(cfg)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert [r.case.P for r in a] == [r.case.P for r in b]
    # count over 1.5 s at 200/s: 300 +- 3 sigma (sqrt(300) ~ 17)
    assert 250 < len(a) < 350
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 200.0) < 0.2 / 200.0
    assert all(r.case.n[0] in (48, 64) and 1 <= r.case.P <= 4 for r in a)
    assert all(r.prec == api.IB_F32 for r in a)


def test_trace_precision_mix():
    cfg = serve.ServeConfig(rate=400.0, seconds=1.0, P_max=2, grids=(48,), fp64_fraction=0.5, seed=1)
    t = serve.make_trace(cfg)
    f64 = sum(r.prec == api.IB_F64 for r in t) / len(t)
    assert 0.4 < f64 < 0.6


def test_admission_by_budget_and_slots_fifo():
    assert serve.admit_count([10, 10, 10], used=0, budget=25, n_active=0, max_active=8) == 2
    assert serve.admit_count([10, 10, 10], used=0, budget=100, n_active=6, max_active=8) == 2
    # a head that does not fit blocks smaller requests behind it
    assert serve.admit_count([50, 1, 1], used=60, budget=100, n_active=0, max_active=8) == 0
    assert serve.admit_count([], used=0, budget=100, n_active=0, max_active=8) == 0


def test_request_bytes_grows_with_grid_and_precision():
    cfg = serve.ServeConfig(rate=50.0, seconds=0.5, P_max=2, grids=(48, 192), seed=2)
    t = serve.make_trace(cfg)
    small = [r for r in t if r.case.n[0] == 48][0]
    big = [r for r in t if r.case.n[0] == 192][0]
    assert serve.request_bytes(big.case, api.IB_F32) > serve.request_bytes(small.case, api.IB_F32)
    assert serve.request_bytes(small.case, api.IB_F64) > serve.request_bytes(small.case, api.IB_F32)
    # fields dominate: 2 copies x 3 components x 192^3 x 4 bytes
    assert serve.request_bytes(big.case, api.IB_F32) >= 2 * 3 * 192 ** 3 * 4
