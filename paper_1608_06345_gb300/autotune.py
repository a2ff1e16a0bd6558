"""Autotuner front end: pick the fastest compiled step shape for an instance
(lbm_autotune times every candidate on the instance's own buffers) and keep
the winner in a JSON cache keyed by lattice, precision, grid and SM count,
so later instances of the same kind skip the timing."""
from __future__ import annotations

import json
import os

from . import lbm

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1608_06345_gb300", "autotune.json")


def _key(solver):
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return (f"lat{solver.lattice}-prec{solver.prec}-{'x'.join(map(str, solver.shape))}-"
            f"sm{props.multi_processor_count}")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(solver, reps=5, cache_path=DEFAULT_CACHE, refresh=False):
    """Select the fastest shape for `solver` (an lbm.Solver).  Returns a dict
    with the chosen index, its (stage, block) and the time per step."""
    key = _key(solver)
    cache = _load(cache_path) if cache_path else {}
    if not refresh and key in cache:
        lbm.lbm_set_shape(solver.h, cache[key]["index"])
        return dict(cache[key], cached=True)
    index, us = lbm.lbm_autotune(solver.h, reps)
    stage, block = lbm.lbm_shape_info(solver.lattice, solver.prec, index)
    rec = {"index": index, "stage": stage, "block": block, "us_per_step": us}
    if cache_path:
        cache[key] = rec
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(rec, cached=False)
