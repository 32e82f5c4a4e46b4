"""Persistent cache of tuned launch shapes.

``gmres_autotune`` (native) times GMRES-IR cycles of one handle under a grid of launch shapes;
this module keys its choice by what decides it -- the GPU, the size bucket (log2 n), nonzeros per
row, the basis precision, the restart length and the polynomial degree -- and keeps the choices
in a JSON file so later handles of the same class skip the timing.  ``gmres_batch_autotune``
does the same for the batched solver (chunk size and sweep pipeline), keyed by the GPU, the
number of systems, the size bucket of the padded total and the restart length.
"""
from __future__ import annotations

import json
import math
import os

SCHEMA = 1


def default_path() -> str:
    return os.environ.get("GMRESB3_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gmresb3", "tuning.json"))


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def key(gpu: str, n: int, nnz: int, basis: str, m: int, degree: int) -> str:
    """Cache key: sizes are bucketed (log2 n rounded, nonzeros per row rounded to an integer)."""
    nb = int(round(math.log2(max(n, 1))))
    w = int(round(nnz / max(n, 1)))
    return f"{gpu}|n2^{nb}|w{w}|{basis}|m{m}|d{degree}"


class TuningCache:
    def __init__(self, path: str | None = None):
        self.path = path or default_path()
        self.entries = {}
        if os.path.exists(self.path):
            with open(self.path) as f:
                data = json.load(f)
            if data.get("schema") == SCHEMA:
                self.entries = data.get("entries", {})

    def get(self, k):
        return self.entries.get(k)

    def put(self, k, shapes: dict, s_per_iter: float, default_s_per_iter: float):
        self.entries[k] = dict(shapes=shapes, s_per_iter=s_per_iter,
                               default_s_per_iter=default_s_per_iter)
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"schema": SCHEMA, "entries": self.entries}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tune(solver, b, nnz: int, basis: str, degree: int, cache: TuningCache | None = None,
         cycles: int = 2) -> dict:
    """Apply the cached shapes for this solver's class, or time them (and cache the result)."""
    cache = cache or TuningCache()
    k = key(gpu_name(), solver.n, nnz, basis, solver.params.m or solver.m, degree)
    hit = cache.get(k)
    if hit is not None:
        solver.set_tuning(**hit["shapes"])
        return dict(hit, key=k, cached=True)
    shapes, t_best, t_def = solver.autotune(b, cycles)
    cache.put(k, shapes, t_best, t_def)
    return dict(shapes=shapes, s_per_iter=t_best, default_s_per_iter=t_def, key=k, cached=False)


def batch_key(gpu: str, nsys: int, total_n: int, nnz: int, m: int) -> str:
    """Cache key of a batch: system count, log2 of the total rows, nonzeros per row, m."""
    nb = int(round(math.log2(max(total_n, 1))))
    w = int(round(nnz / max(total_n, 1)))
    return f"{gpu}|batch|s{nsys}|n2^{nb}|w{w}|m{m}"


def tune_batch(solver, B, nnz: int, m: int, tol: float = 1e-10, max_cycles: int = 1000,
               cache: TuningCache | None = None) -> dict:
    """Apply the cached shapes for this batch's class, or time them (and cache the result).
    The costs stored for a batch are whole-solve seconds."""
    cache = cache or TuningCache()
    k = batch_key(gpu_name(), len(solver.sizes), sum(solver.sizes), nnz, m)
    hit = cache.get(k)
    if hit is not None:
        solver.set_tuning(**hit["shapes"])
        return dict(hit, key=k, cached=True)
    shapes, t_best, t_def = solver.autotune(B, tol, max_cycles)
    cache.put(k, shapes, t_best, t_def)
    return dict(shapes=shapes, s_per_iter=t_best, default_s_per_iter=t_def, key=k, cached=False)
