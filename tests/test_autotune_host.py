"""Host logic of the autotuner, with a fake context and step."""
import pytest

from paper_2408_14140_gb300 import autotune


class FakeCtx:
    def __init__(self):
        self.calls = []

    def set_pass_kernels(self, which):
        self.calls.append(("pass", which))
        self.pass_kernels = which

    def set_volume_split(self, n):
        self.calls.append(("split", n))
        self.volume_split = n


def test_tune_picks_the_fastest_and_leaves_it_set(monkeypatch):
    ctxs = [FakeCtx(), FakeCtx()]
    cost = {("wavefront", 0): 2.2, ("wavefront", 4): 3.0, ("wavefront", 8): 2.0, ("wavefront", 16): 2.5,
            ("groups", 0): 1.7, ("groups", 4): 4.0, ("groups", 8): 1.5, ("groups", 16): 5.0}
    monkeypatch.setattr(autotune, "time_step",
                        lambda step, **kw: cost[(ctxs[0].pass_kernels, ctxs[0].volume_split)])
    out = autotune.tune(ctxs, step=lambda: None)
    assert out["choice"] == {"pass_kernels": "groups", "volume_split": 8}
    assert out["ms"] == 1.5
    assert len(out["table"]) == 8
    for c in ctxs:  # every context carries the winner at the end
        assert (c.pass_kernels, c.volume_split) == ("groups", 8)


def test_tune_custom_space(monkeypatch):
    ctx = FakeCtx()
    monkeypatch.setattr(autotune, "time_step", lambda step, **kw: {4: 2.0, 32: 1.0}[ctx.volume_split])
    out = autotune.tune([ctx], step=lambda: None, space={"volume_split": (4, 32)})
    assert out["choice"] == {"volume_split": 32}
    assert ctx.calls[-1] == ("split", 32)
