"""Launch-shape autotuner for the batched persistent curvature kernel.

The shape (threads per block, interface cells claimed per work-queue ticket,
resident blocks per SM, lanes per interface cell: one thread per cell or
eight cooperating lanes) is chosen by timing every candidate on the actual
fields with CUDA events and keeping the fastest.  Results are cached in a JSON
file keyed by GPU name, kernel (method + flags) and a shape class of the
workload (number of fields and total interface cells, both rounded to powers
of two), so a workload of the same class reuses the choice without timing.

The cache lives next to the built library (``_build/autotune.json``) unless
``PLIC_AUTOTUNE_CACHE`` names another file.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import build as _build
from . import plic

CANDIDATES = ([(128, ch, bps, 1) for ch in (32, 64, 128, 256, 1024) for bps in (0, 2, 3, 4)] +
              [(128, ch, bps, 8) for ch in (32, 64, 128, 256) for bps in (0, 2, 3)])
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("PLIC_AUTOTUNE_CACHE", os.path.join(_build.BUILD, "autotune.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def shape_class(fields) -> str:
    nf = len(fields)
    tot = sum(int(f[2]) for f in fields)
    return "f%d-k%d" % (1 << max(0, math.ceil(math.log2(max(nf, 1)))),
                        1 << max(0, math.ceil(math.log2(max(tot, 1)))))


def key(fields, method, flags) -> str:
    dev = torch.cuda.get_device_name(fields[0][0].device)
    return "%s|batched-v2|%s|%d|%s" % (dev, method, flags, shape_class(fields))


def tune(fields, method="sz_opt", flags=0, reps=5, candidates=None, force=False):
    """Best (block_threads, cells_per_chunk, blocks_per_sm, lanes_per_cell) for these fields;
    returns (shape, timings) where timings maps str(shape) -> ms (empty when
    the cache answered)."""
    flist = fields.fields if isinstance(fields, plic.BatchedFields) else fields
    k = key(flist, method, flags)
    with _lock:
        cache = _load()
        if not force and k in cache:
            return tuple(cache[k]["shape"]), {}
    batch = fields if isinstance(fields, plic.BatchedFields) else plic.BatchedFields(fields)
    times = {}
    s = torch.cuda.current_stream()
    for cand in (candidates or CANDIDATES):
        plic.curvature_batched(batch, method=method, flags=flags, tuning=cand)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            plic.curvature_batched(batch, method=method, flags=flags, tuning=cand)
        b.record(s)
        torch.cuda.synchronize()
        times[str(cand)] = a.elapsed_time(b) / reps
    best = min(times, key=times.get)
    shape = tuple(int(v) for v in best.strip("()").split(","))
    with _lock:
        cache = _load()
        cache[k] = {"shape": list(shape), "ms": times[best]}
        _save(cache)
    return shape, times
