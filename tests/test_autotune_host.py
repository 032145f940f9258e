"""Host logic of the autotuner, with a fake context and step."""
from paper_2408_14140_gb300 import autotune


class FakeCtx:
    def __init__(self):
        self.calls = []
        self.gather = (0, 0)

    def set_pass_kernels(self, which):
        self.calls.append(("pass", which))
        self.pass_kernels = which

    def set_volume_split(self, n):
        self.calls.append(("split", n))
        self.volume_split = n

    def set_gather(self, ctas, stage):
        self.calls.append(("gather", ctas, stage))
        self.gather = (ctas, stage)


SPACE2 = {"pass_kernels": ("wavefront", "groups"), "volume_split": (0, 4, 8, 16)}


def test_tune_picks_the_fastest_and_leaves_it_set(monkeypatch):
    ctxs = [FakeCtx(), FakeCtx()]
    cost = {("wavefront", 0): 2.2, ("wavefront", 4): 3.0, ("wavefront", 8): 2.0, ("wavefront", 16): 2.5,
            ("groups", 0): 1.7, ("groups", 4): 4.0, ("groups", 8): 1.5, ("groups", 16): 5.0}
    monkeypatch.setattr(autotune, "time_step",
                        lambda step, **kw: cost[(ctxs[0].pass_kernels, ctxs[0].volume_split)])
    out = autotune.tune(ctxs, step=lambda: None, space=SPACE2)
    assert out["choice"] == {"pass_kernels": "groups", "volume_split": 8}
    assert out["ms"] == 1.5
    # coordinate descent: the start, then each choice in turn (distinct combinations only)
    assert len(out["table"]) == 6
    for c in ctxs:  # every context carries the winner at the end
        assert (c.pass_kernels, c.volume_split) == ("groups", 8)


def test_tune_default_space_covers_the_gather_layout(monkeypatch):
    ctx = FakeCtx()

    def cost(step, **kw):
        ctas, stage = ctx.gather
        return 1.0 + (0.0 if ctas == 3 else 0.5) + (0.0 if stage == 128 else 0.25) + \
            (0.0 if ctx.volume_split == 4 else 0.1)

    monkeypatch.setattr(autotune, "time_step", cost)
    out = autotune.tune([ctx], step=lambda: None)
    assert set(out["choice"]) == set(autotune.SPACE)
    assert out["choice"]["gather_ctas"] == 3 and out["choice"]["gather_stage"] == 128
    assert out["choice"]["volume_split"] == 4
    assert ctx.gather == (3, 128)


def test_tune_custom_space(monkeypatch):
    ctx = FakeCtx()
    monkeypatch.setattr(autotune, "time_step", lambda step, **kw: {4: 2.0, 32: 1.0}[ctx.volume_split])
    out = autotune.tune([ctx], step=lambda: None, space={"volume_split": (4, 32)})
    assert out["choice"] == {"volume_split": 32}
    assert ctx.calls[-1] == ("split", 32)


def test_tune_cached_reuses_the_stored_choice(monkeypatch, tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = FakeCtx()
    timed = []

    def cost(step, **kw):
        timed.append(1)
        return {4: 2.0, 32: 1.0}[ctx.volume_split]

    monkeypatch.setattr(autotune, "time_step", cost)
    space = {"volume_split": (4, 32)}
    first = autotune.tune_cached("dev|f32|D8-24|N128", [ctx], lambda: None, path=path, space=space)
    assert not first["cached"] and first["choice"] == {"volume_split": 32}
    n = len(timed)
    ctx2 = FakeCtx()
    again = autotune.tune_cached("dev|f32|D8-24|N128", [ctx2], lambda: None, path=path, space=space)
    assert again["cached"] and again["choice"] == {"volume_split": 32}
    assert len(timed) == n  # nothing timed the second time
    assert ctx2.volume_split == 32
    other = autotune.tune_cached("dev|f64|D8-24|N128", [FakeCtx()], lambda: None, path=path, space=space)
    assert not other["cached"]
