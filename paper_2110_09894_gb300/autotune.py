"""Autotuner for group launches: picks the persistent grid (CTAs per SM) by timing.

Each candidate builds the group, captures one run in a CUDA graph and times
graph replays with CUDA events; the fastest setting is cached in a JSON file
keyed by the members' plans, so later runs reuse it without timing.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import qx

CACHE = os.environ.get("QX_AUTOTUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))


def group_key(members, d_bits):
    h = hashlib.sha256()
    for m, b in zip(members, d_bits):
        h.update(f"{m.n_qubits}:{m.n_open}:{m.n_slices}:{m.peak_entries}:{b.shape[0]};".encode())
    return h.hexdigest()[:24]


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def tuned_group(members, d_bits, candidates=(1, 2, 3), reps=3):
    """Return (Group, ctas_per_sm, timings_ms) with the fastest cached or measured setting."""
    import torch
    key = group_key(members, d_bits)
    cache = _load()
    if key in cache:
        best = int(cache[key]["ctas_per_sm"])
        return qx.Group(members, d_bits, best), best, cache[key].get("ms", {})
    stream = members[0].stream
    times = {}
    for c in candidates:
        g = qx.Group(members, d_bits, c)
        g.capture()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g.replay()
        ev0.record(stream)
        for _ in range(reps):
            g.replay()
        ev1.record(stream)
        ev1.synchronize()
        times[c] = ev0.elapsed_time(ev1) / reps
        g.close()
    best = min(times, key=times.get)
    cache[key] = {"ctas_per_sm": best, "ms": {str(k): v for k, v in times.items()}}
    _store(cache)
    return qx.Group(members, d_bits, best), best, times
