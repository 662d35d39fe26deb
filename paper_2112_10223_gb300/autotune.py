"""Autotuner for the library's work-class thresholds and accumulator layout.

The paper tunes its sliding hash to the memory hierarchy: the part size of
Alg. 7/8 comes from the cache size, and Sec. IV-D measures the best hash-table
size against the L1 and L3 capacities.  The knobs that play that role here are
the options that split columns into work classes and size the thread-block
tables:

    warp_max          largest s_j = sum_i nnz(A_i(:,j)) run by one warp
                      (32 threads per column)
    cta_max           largest s_j run by one thread block (256 threads);
                      larger columns are cut into row windows
    window_max        rows per numeric window (Alg. 7/8's part size)
    block_accumulator thread-block table layout (0 automatic, 1 flat row
                      bitmap, 2 compact word table)

``Autotuner.tune`` times a workload under candidate options (one coordinate
sweep from the defaults: each knob in turn over its values, the others held
at the best so far) and keeps the fastest; results are cached in a JSON file
keyed by the device (name, SM count), the CUDA runtime and library versions
and a coarse description of the workload, so a later run with the same key
reuses them without timing anything.

The cache path is ``$SPKADD_AUTOTUNE_CACHE`` if set, else
``~/.cache/spkadd/autotune.json``.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
import time

SPACE = {
    "warp_max": [512, 256, 128],
    "cta_max": [4096, 2048, 1024],
    "window_max": [4096, 2048],
    "block_accumulator": [0, 1, 2],
}
DEFAULTS = {"warp_max": 512, "cta_max": 4096, "window_max": 4096, "block_accumulator": 0}


def default_cache_path() -> str:
    env = os.environ.get("SPKADD_AUTOTUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "spkadd", "autotune.json")


def device_key(device=None) -> dict:
    """Device name, SM count, CUDA runtime and library versions of `device` (default: current)."""
    import torch

    from . import library

    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    p = torch.cuda.get_device_properties(dev)
    return {"device": p.name, "sms": int(p.multi_processor_count), "cuda": str(torch.version.cuda),
            "library": int(library().spkadd_version())}


def _bucket(x: float) -> int:
    return int(math.floor(math.log2(max(x, 1.0))))


def workload_key(ks, ns, nnzs, dtypes) -> dict:
    """A coarse description of a set of problems: value types, log2 ranges of k
    and n, and log2 of the mean summed input count per column."""
    cols = sum(int(n) for n in ns)
    mean_s = sum(int(z) for z in nnzs) / max(cols, 1)
    return {"dtypes": sorted({str(d).replace("torch.", "") for d in dtypes}),
            "k": [_bucket(min(ks)), _bucket(max(ks))], "n": [_bucket(min(ns)), _bucket(max(ns))],
            "s_mean": _bucket(mean_s), "problems": _bucket(len(ks))}


def _key_string(dev: dict, work: dict) -> str:
    return json.dumps({"dev": dev, "work": work}, sort_keys=True)


class Autotuner:
    """Chooses options by timing; remembers the choice per (device, workload) key."""

    def __init__(self, cache_path: str | None = None, space: dict | None = None):
        self.cache_path = cache_path or default_cache_path()
        self.space = dict(space or SPACE)
        self._cache = None
        self.last = None  # the cache record of the last tune() call

    # -- cache ---------------------------------------------------------------
    def _load(self) -> dict:
        if self._cache is None:
            try:
                with open(self.cache_path) as f:
                    self._cache = json.load(f)
            except (OSError, ValueError):
                self._cache = {}
        return self._cache

    def _store(self) -> None:
        d = os.path.dirname(self.cache_path)
        if d:
            os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d or ".", suffix=".tmp")
        with os.fdopen(fd, "w") as f:
            json.dump(self._cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def lookup(self, dev: dict, work: dict) -> dict | None:
        e = self._load().get(_key_string(dev, work))
        return dict(e["options"]) if e else None

    # -- search --------------------------------------------------------------
    def tune(self, run, dev: dict, work: dict, repeats: int = 2, timer=None, force: bool = False,
             margin: float = 0.03) -> dict:
        """Best option values for the workload that ``run(values)`` executes.

        ``run`` takes a dict of option values, runs the workload once and
        returns when its work is done (synchronised).  ``timer(run, values)``
        may replace the default wall-clock timing (a warm-up run, then the
        mean of `repeats` runs).  A candidate replaces the best so far only
        when it is faster by more than the fraction `margin`, so timing noise
        does not move the choice away from the defaults.  The result is cached
        under (dev, work); a cached result is returned without running
        anything unless `force`.
        """
        if not force:
            hit = self.lookup(dev, work)
            if hit is not None:
                self.last = dict(self._load()[_key_string(dev, work)], cached=True)
                return hit
        if timer is None:
            def timer(fn, values):
                fn(values)
                t0 = time.perf_counter()
                for _ in range(repeats):
                    fn(values)
                return (time.perf_counter() - t0) / repeats

        seen = {}

        def cost(values):
            key = tuple(sorted(values.items()))
            if key not in seen:
                seen[key] = timer(run, dict(values))
            return seen[key]

        best = {k: DEFAULTS[k] for k in self.space}
        best_t = cost(best)
        for knob, choices in self.space.items():
            for v in choices:
                cand = dict(best, **{knob: v})
                if not valid(cand):
                    continue
                t = cost(cand)
                if t < best_t * (1.0 - margin):
                    best, best_t = cand, t
        rec = {"options": best, "seconds": best_t, "timed": len(seen),
               "candidates": [dict(dict(k), seconds=t) for k, t in seen.items()]}
        self._load()[_key_string(dev, work)] = rec
        self._store()
        self.last = dict(rec, cached=False)
        return best


def valid(values: dict) -> bool:
    """The library's own range rules (spkadd_options): warp_max <= cta_max."""
    return values.get("warp_max", 512) <= values.get("cta_max", 4096)


def tune_batch(desc: dict, device=None, tuner: Autotuner | None = None, repeats: int = 2, force: bool = False):
    """Options for a batch given as flat descriptors (keys k, m, n, nnz, cp,
    ri, va, dtypes: as for spkadd_batch_plan_raw), tuned on that batch.
    Returns an Options struct."""
    import numpy as np
    import torch

    from . import (default_options, spkadd_batch_numeric_raw, spkadd_batch_plan_raw, spkadd_batch_symbolic,
                   spkadd_destroy)

    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    ks = [int(x) for x in desc["k"]]
    starts = np.concatenate([[0], np.cumsum(ks)])
    nnzs = [int(np.sum(desc["nnz"][starts[q]:starts[q + 1]])) for q in range(len(ks))]
    work = workload_key(ks, [int(x) for x in desc["n"]], nnzs, desc["dtypes"])
    tuner = tuner or Autotuner()

    def run(values):
        opt = default_options(**values)
        h = spkadd_batch_plan_raw(desc["k"], desc["m"], desc["n"], desc["nnz"], desc["cp"], desc["ri"], desc["va"],
                                  desc["dtypes"], options=opt, device=dev)
        nnz = np.asarray(spkadd_batch_symbolic(h), dtype=np.int64)
        n1 = np.asarray(desc["n"], dtype=np.int64) + 1
        is64 = np.asarray([d == torch.float64 for d in desc["dtypes"]])
        cp = torch.empty(int(n1.sum()), dtype=torch.int64, device=dev)
        ri = torch.empty(max(int(nnz.sum()), 1), dtype=torch.int32, device=dev)
        v64 = torch.empty(max(int(nnz[is64].sum()), 1), dtype=torch.float64, device=dev)
        v32 = torch.empty(max(int(nnz[~is64].sum()), 1), dtype=torch.float32, device=dev)

        def offs(sizes):
            o = np.zeros(sizes.size, dtype=np.uint64)
            o[1:] = np.cumsum(sizes[:-1]).astype(np.uint64)
            return o

        a_va = np.zeros(nnz.size, dtype=np.uint64)
        a_va[is64] = np.uint64(v64.data_ptr()) + offs(nnz[is64]) * np.uint64(8)
        a_va[~is64] = np.uint64(v32.data_ptr()) + offs(nnz[~is64]) * np.uint64(4)
        spkadd_batch_numeric_raw(h, np.uint64(cp.data_ptr()) + offs(n1) * np.uint64(8),
                                 np.uint64(ri.data_ptr()) + offs(nnz) * np.uint64(4), a_va)
        spkadd_destroy(h)
        torch.cuda.synchronize(dev)

    best = tuner.tune(run, device_key(dev), work, repeats=repeats, force=force)
    return default_options(**best)
