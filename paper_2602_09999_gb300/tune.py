"""Autotuner for the launch choices of the blend kernels.

The choices (pixels per blend thread, list entries per shared-memory batch,
and the tile schedule -- a work queue in longest-list-first order or one CTA
per tile; see fgs_tuning in include/fastergs.h) change speed only: every
choice gives bit-identical images and the same gradients up to atomic-add
order.  The tuner times forward + loss + backward of the caller's own batch
shape for each supported choice with CUDA events, keeps the fastest, then
times the per-pixel backward with each other (pixels, batch) pair of its own
with that choice fixed (the backward's best pair can differ from the
forward's: it sums each entry's gradients over the warp once per entry, so
more pixels per thread spread that cost over more pixels), then the
forward's other pairs with the backward's fixed, then the radix digit width
(8 or 11 bits) of the depth sort and of the tile sort, then the duplication
order (strided or split), keeps the fastest, and caches it in a JSON file keyed by GPU name, Gaussian count and pixel count
(rounded to powers of two), view count, backward order and storage types,
so later runs of the same shape skip the search.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")


def _key(trainer) -> str:
    """Cache key of a trainer's shape: GPU, Gaussian and pixel counts (as
    powers of two), the number of views, the blend backward's order and the
    SH parameter and Adam moment storage types."""
    name = torch.cuda.get_device_name().replace(" ", "_")
    n, pixels = trainer.n, trainer.views.total_pixels
    order = "pg" if trainer.rast.layout.tuning.blend_backward == B.FGS_BACKWARD_PER_GAUSSIAN else "pp"
    sh = str(trainer.params["sh_rest"].dtype).replace("torch.", "")
    mom = str(trainer.exp_avg["means"].dtype).replace("torch.", "")
    return (f"{name}/n2^{round(math.log2(max(n, 1)))}/px2^{round(math.log2(max(pixels, 1)))}"
            f"/v{trainer.views.n}/{order}/sh-{sh}/m-{mom}")


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(table):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


CHOICE_FIELDS = 8


def apply(layout, choice):
    """choice = (pixels per thread, batch[, schedule[, backward pixels per
    thread, backward batch[, depth-sort digit bits, tile-sort digit
    bits[, duplication order]]]]); a backward pair of (0, 0) or none means
    the forward's pair, digit bits of 0 or none mean 8, no duplication order
    means the strided one.  The layout's sorted_in_alt follows the tile
    sort's pass count."""
    layout.tuning.blend_pixels_per_thread = int(choice[0])
    layout.tuning.blend_batch = int(choice[1])
    layout.tuning.blend_schedule = int(choice[2]) if len(choice) > 2 else B.FGS_SCHEDULE_QUEUE
    bwd = tuple(choice[3:5]) if len(choice) > 4 else (0, 0)
    layout.tuning.backward_pixels_per_thread = int(bwd[0])
    layout.tuning.backward_batch = int(bwd[1])
    digits = tuple(choice[5:7]) if len(choice) > 6 else (0, 0)
    layout.tuning.depth_sort_digit_bits = int(digits[0])
    layout.tuning.tile_sort_digit_bits = int(digits[1])
    rb = int(digits[1]) or 8
    layout.sorted_in_alt = ((int(layout.sort_bits) + rb - 1) // rb) & 1
    layout.tuning.duplicate_order = int(choice[7]) if len(choice) > 7 else B.FGS_DUPLICATE_STRIDED


def label(choice) -> str:
    sched = "grid" if len(choice) > 2 and choice[2] == B.FGS_SCHEDULE_GRID else "queue"
    text = f"{choice[0]}x{choice[1]}/{sched}"
    if len(choice) > 4 and choice[3]:
        text += f"+bwd{choice[3]}x{choice[4]}"
    if len(choice) > 6 and (choice[5] or choice[6]):
        text += f"+sort{choice[5] or 8}/{choice[6] or 8}"
    if len(choice) > 7 and choice[7] == B.FGS_DUPLICATE_SPLIT:
        text += "+dupsplit"
    return text


def all_choices():
    return [(p, b, s) for s in B.BLEND_SCHEDULES for (p, b) in B.BLEND_CONFIGS]


def autotune(trainer, reps: int = 3, use_cache: bool = True, configs=None):
    """Picks the fastest blend configuration for `trainer`'s batch shape and
    writes it into its workspace layout.  Runs forward, loss and backward
    only (the parameters are not updated).  Returns (choice, timings_ms)."""
    configs = all_choices() if configs is None else [
        (tuple(c) + (B.FGS_SCHEDULE_QUEUE,))[:3] for c in configs]
    key = _key(trainer)
    table = _load() if use_cache else {}
    if key in table and len(table[key].get("choice", [])) == CHOICE_FIELDS:
        choice = tuple(table[key]["choice"])
        apply(trainer.rast.layout, choice)
        return choice, table[key].get("ms", {})
    timings = {}
    stream = torch.cuda.current_stream()

    def time_choice(cfg):
        apply(trainer.rast.layout, cfg)
        trainer.forward_backward()        # warm-up of this configuration
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            trainer.forward_backward()
        t1.record(stream)
        t1.synchronize()
        timings[label(cfg)] = t0.elapsed_time(t1) / reps

    for cfg in configs:
        time_choice(cfg)
    best = min(configs, key=lambda c: timings[label(c)])
    best = tuple(best[:3]) + (0, 0)
    # then the per-pixel backward's own pair, the forward's choice fixed
    if trainer.rast.layout.tuning.blend_backward == B.FGS_BACKWARD_PER_PIXEL:
        own = [best[:3] + tuple(pb) for pb in B.BLEND_CONFIGS if tuple(pb) != tuple(best[:2])]
        for cfg in own:
            time_choice(cfg)
        best = min([best] + own, key=lambda c: timings[label(c)])
        # and the forward's pair once more, the backward's pair fixed
        bwd = tuple(best[3:5]) if best[3] else tuple(best[:2])
        fwd = [tuple(pb) + (best[2],) + bwd for pb in B.BLEND_CONFIGS if tuple(pb) != tuple(best[:2])]
        for cfg in fwd:
            time_choice(cfg)
        best = min([best] + fwd, key=lambda c: timings[label(c)])
    # then the radix digit width of each sort, the blend choice fixed
    best = tuple(best[:5]) + (0, 0)
    sorts = [tuple(best[:5]) + (d, t) for d in B.SORT_DIGIT_BITS for t in B.SORT_DIGIT_BITS
             if (d, t) != (8, 8)]
    for cfg in sorts:
        time_choice(cfg)
    best = min([best] + sorts, key=lambda c: timings[label(c)])
    # then the duplication order, everything else fixed
    best = tuple(best[:7]) + (B.FGS_DUPLICATE_STRIDED,)
    split = tuple(best[:7]) + (B.FGS_DUPLICATE_SPLIT,)
    time_choice(split)
    best = min([best, split], key=lambda c: timings[label(c)])
    apply(trainer.rast.layout, best)
    if use_cache:
        table[key] = {"choice": list(best), "ms": timings}
        _store(table)
    return best, timings
