"""Autotuner of the mapping iteration's tile and launch shapes.

The batched iteration (`pipeline.MappingStep`) has shapes whose best values
depend on the keyframe batch -- its resolutions, how its splats crowd into
a few tiles near the vanishing points, the partition mix -- and on the
device:

  chunk             splats per compositing work item (the list of a tile
                    is cut into chunks of this many splats)
  fwd_ctas_per_sm   CTAs per SM of the persistent forward compositing kernels
  bwd_ctas_per_sm   CTAs per SM of the persistent reverse compositing kernel
  sort_ctas_per_sm  CTAs per SM of the radix-sort and compaction passes
  emit_ctas_per_sm  CTAs per SM of the pair emission

(0 is the library's own choice for the last four; see gs_set_tuning).  `tune`
measures candidates on the actual batch: each candidate iteration is captured
into a CUDA graph exactly as MappingStep runs it and replayed `reps` times
with CUDA events on its stream; the median is its time.  The search is
coordinate descent from the defaults, one knob at a time, for `rounds`
rounds.  The best configuration is cached per (device name, workload
signature) in a JSON file, so a later call on the same device and workload
returns it without measuring.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import time

import numpy as np

from . import _lib as L
from . import api

KNOBS = ("chunk",) + api.TUNING_FIELDS
DEFAULTS = {"chunk": 0, "fwd_ctas_per_sm": 0, "bwd_ctas_per_sm": 0, "sort_ctas_per_sm": 0, "emit_ctas_per_sm": 0}
SPACE = {
    "chunk": (0, 256, 512, 768, 1024),
    "bwd_ctas_per_sm": (0, 4, 6, 8),
    "fwd_ctas_per_sm": (0, 4, 6, 8),
    "sort_ctas_per_sm": (0, 2, 3),
    "emit_ctas_per_sm": (0, 2, 6, 8),
}


def signature(views: api.Views, anchors: api.Anchors, precision: int, loss: str = "l1") -> str:
    """Workload key: view resolutions, anchor count and decoder shape, the
    partition sizes, precision and loss.  Two batches with the same key have
    the same buffers and launch grids (their data may differ)."""
    wh = np.asarray(views.wh, np.int64).reshape(-1, 2)
    part = anchors.part.detach().cpu().numpy() if hasattr(anchors.part, "detach") else np.asarray(anchors.part)
    sizes = np.bincount(part.astype(np.int64), minlength=anchors.M) if part.size else np.zeros(anchors.M, np.int64)
    h = hashlib.sha256()
    h.update(wh.tobytes())
    h.update(sizes.astype(np.int64).tobytes())
    h.update(json.dumps([anchors.N, anchors.F, anchors.k, anchors.hidden, anchors.M, int(precision), loss]).encode())
    return f"V{views.V}-N{anchors.N}-M{anchors.M}-p{int(precision)}-{loss}-{h.hexdigest()[:16]}"


class TuneCache:
    """JSON file of tuned configurations keyed by device name and workload
    signature.  Writes go through a temporary file and a rename."""

    def __init__(self, path: str):
        self.path = path

    def _load(self) -> dict:
        if not os.path.exists(self.path):
            return {}
        with open(self.path) as f:
            return json.load(f)

    @staticmethod
    def key(device: str, sig: str) -> str:
        return f"{device}|{sig}"

    def get(self, device: str, sig: str):
        e = self._load().get(self.key(device, sig))
        return None if e is None else {k: int(e["config"].get(k, 0)) for k in KNOBS}

    def entry(self, device: str, sig: str):
        return self._load().get(self.key(device, sig))

    def put(self, device: str, sig: str, config: dict, ms: float, default_ms: float):
        data = self._load()
        data[self.key(device, sig)] = {"config": {k: int(config.get(k, 0)) for k in KNOBS}, "ms": float(ms),
                                       "default_ms": float(default_ms), "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def coordinate_descent(measure, space=SPACE, start=None, rounds=2, min_gain=0.01):
    """Minimises measure(config) one knob at a time (host logic, no GPU):
    a value replaces the current one only if it is faster by more than
    min_gain.  Returns (best config, its time, {config key: time})."""
    best = dict(DEFAULTS if start is None else start)
    seen = {}

    def timed(cfg):
        key = json.dumps(cfg, sort_keys=True)
        if key not in seen:
            seen[key] = float(measure(cfg))
        return seen[key]

    best_ms = timed(best)
    for _ in range(rounds):
        changed = False
        for knob, values in space.items():
            for v in values:
                if v == best[knob]:
                    continue
                cand = dict(best, **{knob: v})
                ms = timed(cand)
                if ms < best_ms * (1.0 - min_gain):
                    best, best_ms, changed = cand, ms, True
        if not changed:
            break
    return best, best_ms, seen


def time_config(views, anchors, target, precision, loss, cfg, reps=10, steps_cache=None, cap_rows=None,
                cap_pairs=None):
    """Median device time (ms) of the captured mapping iteration with the
    given shapes.  steps_cache keeps the last candidate's buffers (one chunk
    length at a time, so that large batches do not hold several copies)."""
    import torch

    from . import pipeline
    chunk = int(cfg.get("chunk", 0))
    steps_cache = {} if steps_cache is None else steps_cache
    prev = api.get_tuning()
    api.set_tuning({k: cfg.get(k, 0) for k in api.TUNING_FIELDS})
    try:
        ms = steps_cache.get(chunk)
        if ms is None:
            steps_cache.clear()
            torch.cuda.empty_cache()
            ms = pipeline.MappingStep(views, anchors, precision=precision, chunk=chunk, loss=loss, cap_rows=cap_rows)
            if cap_pairs is not None and cap_pairs > ms.rp.cap_pairs:
                ms.rp.cap_pairs = int(cap_pairs)
                ms.rp._alloc()
            ms.prepare(target)
            steps_cache[chunk] = ms
        else:
            ms.recapture()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = []
        for it in range(reps + 2):
            with torch.cuda.stream(ms.stream):
                e0.record()
                ms.graph.replay()
                e1.record()
            ms.stream.synchronize()
            if it >= 2:
                out.append(e0.elapsed_time(e1))
        code = api.read_status(ms.rp.status)[0]
        if code != L.GS_OK:
            raise L.GsError("autotune candidate", code)
        return statistics.median(out)
    finally:
        api.set_tuning(prev)


def tune(views, anchors, target, precision=L.GS_PREC_BF16, loss="l1", cache_path=None, reps=10, rounds=2,
         space=SPACE, log=None, cap_rows=None, cap_pairs=None):
    """The best shapes for this batch on the current device (measured, or
    from the cache).  Returns (config, info) with info = {"ms", "default_ms",
    "evaluated", "cached", "signature", "device"}."""
    import torch
    device = torch.cuda.get_device_name()
    sig = signature(views, anchors, precision, loss)
    cache = TuneCache(cache_path) if cache_path else None
    if cache is not None:
        e = cache.entry(device, sig)
        if e is not None:
            cfg = cache.get(device, sig)
            return cfg, {"ms": e["ms"], "default_ms": e["default_ms"], "evaluated": 0, "cached": True,
                         "signature": sig, "device": device}
    steps = {}

    def measure(cfg):
        t = time_config(views, anchors, target, precision, loss, cfg, reps, steps, cap_rows, cap_pairs)
        if log:
            log(f"autotune {cfg}: {t:.3f} ms")
        return t

    best, best_ms, seen = coordinate_descent(measure, space, rounds=rounds)
    default_ms = seen[json.dumps(dict(DEFAULTS), sort_keys=True)]
    del steps
    torch.cuda.empty_cache()
    if cache is not None:
        cache.put(device, sig, best, best_ms, default_ms)
    return best, {"ms": best_ms, "default_ms": default_ms, "evaluated": len(seen), "cached": False,
                  "signature": sig, "device": device}
