"""Tile-shape and CSR row-group autotuning with a persistent cache.

The library's tuners (eb_autotune, amg_autotune, batch_autotune,
amg_tune_csr) time the candidates on the GPU and keep the fastest.  This
module remembers the winner per (GPU, operation, problem) in a JSON file so
that later runs apply it directly (eb_retile, amg_set_csr_epl) instead of
timing again.  The cache file is
``$EB_TUNE_CACHE`` if set, else ``~/.cache/paper_2204_06083_gb300/tiles.json``.
"""
from __future__ import annotations

import json
import os
from typing import Optional

from . import AMG, EB, EB_F64, EB_TUNE_APPLY, Batch, TuneResult


def cache_path() -> str:
    p = os.environ.get("EB_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2204_06083_gb300", "tiles.json")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, key, shape, res: TuneResult):
    d = _load(path)
    d[key] = {"tile": list(shape), "us": dict((f"{a}x{b}x{c}", u) for (a, b, c), u in zip(res.shapes, res.us))}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _device():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _grid_key(eb: EB):
    g = eb.grid
    return f"{g.dim}D {'x'.join(str(int(v)) for v in g.n[:g.dim])} cp={eb.info.num_cp}"


def tune_eb(eb: EB, prec=EB_F64, reps=20, op=EB_TUNE_APPLY, path: Optional[str] = None, retune=False):
    """Tile shape for the apply (op EB_TUNE_APPLY) or the leapfrog step
    (EB_TUNE_LEAPFROG) on this grid."""
    path = path or cache_path()
    key = f"{_device()} | {'apply' if op == EB_TUNE_APPLY else 'leapfrog'} prec={prec} | {_grid_key(eb)}"
    hit = None if retune else _load(path).get(key)
    if hit:
        eb.retile(hit["tile"])
        return tuple(hit["tile"]), None
    res = eb.autotune(prec, reps, op)
    _store(path, key, res.shape, res)
    return res.shape, res


def tune_amg(amg: AMG, reps=20, path: Optional[str] = None, retune=False):
    """Tile shape for the solves of this hierarchy (timed on its V-cycle)."""
    path = path or cache_path()
    key = f"{_device()} | vcycle prec={amg.vcycle_prec} | {_grid_key(amg.eb)}"
    hit = None if retune else _load(path).get(key)
    if hit:
        amg.eb.retile(hit["tile"])
        return tuple(hit["tile"]), None
    res = amg.autotune(reps)
    _store(path, key, res.shape, res)
    return res.shape, res


def tune_batch(batch: Batch, reps=10, path: Optional[str] = None, retune=False):
    """Tile shape of a batch after heat_setup (timed on its V-cycle).  The
    winner is cached, but a batch is always re-timed: retiling it needs the
    same tile rebuild as timing the shape."""
    path = path or cache_path()
    key = f"{_device()} | batch vcycle | count={batch.count} cp={batch.num_cp} nodes={batch.num_nodes}"
    res = batch.autotune(reps)
    _store(path, key, res.shape, res)
    return res.shape, res


def tune_csr(amg: AMG, reps=10, path: Optional[str] = None, retune=False):
    """Entries per lane of the CSR kernels of this hierarchy (amg_tune_csr);
    returns (entries per lane, {entries per lane: microseconds per V-cycle} or
    None when taken from the cache)."""
    path = path or cache_path()
    key = f"{_device()} | csr vcycle prec={amg.vcycle_prec} | {_grid_key(amg.eb)}"
    hit = None if retune else _load(path).get(key)
    if hit:
        amg.set_csr_epl(hit["epl"])
        return int(hit["epl"]), None
    epl, us = amg.tune_csr(reps)
    d = _load(path)
    d[key] = {"epl": epl, "us": {str(k): v for k, v in us.items()}}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return epl, us
