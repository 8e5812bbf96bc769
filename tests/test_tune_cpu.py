"""The autotuner's search on the host: a fake trainer whose forward +
backward 'takes' a time that depends on the launch choice in its layout,
and fake CUDA events that read a clock the fake trainer advances.  Checks
that every stage of the staged search (blend choices, the backward's own
pair, the forward's pair again, the sort digit widths, the duplication
order) finds its fastest option, that the result is written into the
layout, and that the cache returns it without timing again.  No GPU."""
import types

import pytest

from paper_2602_09999_gb300 import binding as B
from paper_2602_09999_gb300 import build_lib, scenes, tune


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return B.lib()


class _Clock:
    now = 0.0


class _Event:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = _Clock.now

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


def _cost(t):
    """A separable time model with one best value per field."""
    fwd = {(4, 64): 1.0}.get((t.blend_pixels_per_thread, t.blend_batch), 2.0)
    sched = 0.0 if t.blend_schedule == B.FGS_SCHEDULE_QUEUE else 0.5
    bwd_pair = (t.backward_pixels_per_thread, t.backward_batch)
    bwd = 0.25 if bwd_pair == (2, 128) else 1.0
    sort = 0.0 if (t.depth_sort_digit_bits, t.tile_sort_digit_bits) == (11, 8) else 0.1
    dup = 0.0 if t.duplicate_order == B.FGS_DUPLICATE_SPLIT else 0.05
    return fwd + sched + bwd + sort + dup


def _fake_trainer():
    cam = B.camera_array([scenes.tiny_camera(100, 70)])
    layout = B.fgs_workspace_size(1000, cam, 1, 64_000)
    tr = types.SimpleNamespace(rast=types.SimpleNamespace(layout=layout), calls=0)

    def forward_backward():
        tr.calls += 1
        _Clock.now += _cost(layout.tuning)

    tr.forward_backward = forward_backward
    return tr


def test_staged_search_finds_each_stage_optimum(lib, tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tuning.json"))
    monkeypatch.setattr(tune, "_key", lambda trainer: "fake-gpu/shape")
    monkeypatch.setattr(tune.torch.cuda, "Event", _Event)
    monkeypatch.setattr(tune.torch.cuda, "current_stream", lambda: None)
    tr = _fake_trainer()
    choice, ms = tune.autotune(tr, reps=2)
    assert tuple(choice) == (4, 64, B.FGS_SCHEDULE_QUEUE, 2, 128, 11, 8, B.FGS_DUPLICATE_SPLIT)
    t = tr.rast.layout.tuning
    assert (t.blend_pixels_per_thread, t.blend_batch, t.blend_schedule) == (4, 64, B.FGS_SCHEDULE_QUEUE)
    assert (t.backward_pixels_per_thread, t.backward_batch) == (2, 128)
    assert (t.depth_sort_digit_bits, t.tile_sort_digit_bits, t.duplicate_order) == (11, 8, 1)
    # 12 blend choices, 5 backward pairs, 5 forward pairs, 3 digit widths, 1 duplication order;
    # each timed once as a warm-up and `reps` times
    stages = len(B.BLEND_CONFIGS) * len(B.BLEND_SCHEDULES) + 2 * (len(B.BLEND_CONFIGS) - 1) + 3 + 1
    assert len(ms) == stages and tr.calls == stages * 3
    assert ms[tune.label(choice)] == pytest.approx(_cost(t))
    # the cache answers the same shape without timing
    again, _ = tune.autotune(_fake_trainer(), reps=2)
    assert tuple(again) == tuple(choice)
    fresh = _fake_trainer()
    tune.autotune(fresh, reps=2)
    assert fresh.calls == 0 and fresh.rast.layout.tuning.duplicate_order == B.FGS_DUPLICATE_SPLIT
