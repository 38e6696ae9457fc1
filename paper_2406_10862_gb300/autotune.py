"""Launch-shape autotuning with a JSON cache.

``ocp_batch_tune`` times every linearisation stage (cell, face, assembly)
over tile sizes and persistent-grid sizes on the device and keeps the fastest;
results do not depend on the shape, only the speed does.  This module keys
the chosen shape by device, block size and problem size (cells and models,
rounded to powers of two) and keeps it in ``_build/launch_shapes.json`` so a
later run reuses it instead of tuning again.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import build as _build

CACHE = os.path.join(_build.BUILD, "launch_shapes.json")


def _key(batch):
    g0 = batch.grids[0]
    ncell = sum(g.N for g in batch.grids)
    name = torch.cuda.get_device_name(g0.device).replace(" ", "_")
    # "ordered|cluster": the tuner also times the ordered (persistent) and one-cluster launches
    return "%s|nb%d|cells2^%d|models2^%d|ordered|cluster" % (name, g0.nb, int(round(math.log2(max(ncell, 1)))),
                                                   int(round(math.log2(len(batch.grids)))))


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tuned_shape(batch, dt, reps=3, retune=False):
    """Apply (and return) the cached or freshly tuned launch shape of a batch."""
    cache = _load()
    key = _key(batch)
    if key in cache and not retune:
        batch.set_shape(cache[key])
        return cache[key], True
    shape = batch.tune(dt, reps=reps)
    cache[key] = shape
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)
    return shape, False
