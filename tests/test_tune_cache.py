"""The tuning cache (paper_2001_08289_gb300.tune) on the CPU: the measurement is
replaced by a fake, so only the keying, storing and reuse are checked."""
import json

from paper_2001_08289_gb300 import tune


class FakeGrid:
    def __init__(self, n, d=2):
        self.n, self.d, self.handle = n, d, 1
        self.split = None

    def set_column_split(self, split):
        self.split = split


def test_tuned_options_are_measured_once_and_cached(tmp_path, monkeypatch):
    calls = []

    def fake_autotune(handle, sigma1, e, opts, iters=32):
        calls.append((opts.scheme, opts.precision, iters))
        return {"check_every": 16, "column_split": 0, "ms_per_iter": 0.5, "candidates": 10}

    monkeypatch.setattr(tune, "lsfft_autotune", fake_autotune)
    path = str(tmp_path / "tune.json")
    g = FakeGrid((8192, 8192))
    kw = tune.tuned(g, 10.0, [1.0, 0.0], path=path, scheme="em_sub", precision="fp32", alpha=0.25, beta=4.0)
    assert kw["check_every"] == 16 and kw["alpha"] == 0.25 and g.split is False
    data = json.load(open(path))
    assert list(data) == ["8192x8192|d2|em_sub|fp32"]
    # the same shape, scheme and precision: no new measurement
    g2 = FakeGrid((8192, 8192))
    kw2 = tune.tuned(g2, 3.0, [0.0, 1.0], path=path, scheme="em_sub", precision="fp32")
    assert kw2["check_every"] == 16 and g2.split is False and len(calls) == 1
    # another scheme or shape is measured and stored beside it
    tune.tuned(FakeGrid((256, 256)), 10.0, [1.0, 0.0], path=path, scheme="ms", precision="fp64")
    assert len(calls) == 2
    assert sorted(json.load(open(path))) == ["256x256|d2|ms|fp64", "8192x8192|d2|em_sub|fp32"]
