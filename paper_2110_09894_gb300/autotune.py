"""Autotuner for batches of uneven circuits.

* tuned_group: the persistent grid (CTAs per SM) of a group launch;
* tuned_uneven: for an uneven batch, the tile family (GEMM threshold) and the
  slice-batch size of each heavy member, and the persistent grid of the light
  members' launch.

Each candidate is built, captured in a CUDA graph and timed over graph
replays with CUDA events; the fastest setting is cached in a JSON file keyed
by the members' plans, so later runs reuse it without timing.
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


# --------------------------------------------------------------------------------------------------
# Uneven batches (light members in the persistent launch, heavy ones on the batched executor)
# --------------------------------------------------------------------------------------------------
# Settings tried for a heavy member: the plan compiler's GEMM threshold (steps with k, m, n >= this
# many bits run as GEMM tiles, smaller ones as gathers against a shared-memory operand: the tile
# family of every step) and the slice-batch size (pairs per launch: all that fit, or a cap).
HEAVY_SETTINGS = ({}, {"gemm_min_bits": 4}, {"gemm_min_bits": 6}, {"max_items": 4096}, {"max_items": 512})


def uneven_key(workloads, precision):
    h = hashlib.sha256()
    for w in workloads:
        h.update(repr((w.n_qubits, list(w.sliced), [tuple(p) for p in w.order], int(len(w.bitstrings)))).encode())
    h.update(str(precision).encode())
    return h.hexdigest()[:24]


def _time_member(w, precision, s, dev, stream, reps):
    import torch
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings), device=dev.index,
                      precision=precision, max_items=s.get("max_items", 0), gemm_min_bits=s.get("gemm_min_bits", 0),
                      stream=stream, executor=qx.EXEC_BATCHED)
    try:
        with torch.cuda.stream(stream):  # the copy is ordered before the contraction's launches
            d_bits = torch.from_numpy(w.bitstrings).to(dev)
        out = c.contract_device(d_bits)
        c.contract_device(d_bits, out)  # eager, then the captured graph
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            c.contract_device(d_bits, out)
        ev1.record(stream)
        ev1.synchronize()
        qx.qx_device_status(c.h)
        return ev0.elapsed_time(ev1) / reps
    finally:
        c.close()
        del c


def tuned_uneven(workloads, precision=qx.QX_PREC_3XTF32, ctas_candidates=(1, 2, 3), heavy_settings=HEAVY_SETTINGS,
                 reps=2, min_share=0.02, device=0):
    """Return (UnevenBatch, choice, timings) with the fastest cached or measured settings.

    Each heavy member that takes at least min_share of the heavy members' time under the default
    setting is timed alone under every setting of heavy_settings (CUDA events over graph replays);
    the persistent grid of the light members' launch is timed over ctas_candidates.  The choice is
    cached by the members' plans."""
    import torch
    from .batch import LIGHT_MAX_PEAK, UnevenBatch
    key = "uneven:" + uneven_key(workloads, precision)
    cache = _load()
    if key in cache:
        ch = cache[key]
        settings = {int(i): s for i, s in ch["settings"].items()}
        return UnevenBatch(workloads, precision=precision, ctas_per_sm=ch["ctas_per_sm"], settings=settings,
                           device=device), ch, ch.get("ms", {})
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    heavy = [i for i, w in enumerate(workloads) if w.peak_rank > LIGHT_MAX_PEAK]
    light = [i for i, w in enumerate(workloads) if w.peak_rank <= LIGHT_MAX_PEAK]
    base = {i: _time_member(workloads[i], precision, {}, dev, stream, reps) for i in heavy}
    total = sum(base.values())
    settings, times = {}, {"heavy_default": base}
    for i in heavy:
        if base[i] < min_share * total:
            continue
        t = {0: base[i]}
        for k, s in enumerate(heavy_settings[1:], 1):
            t[k] = _time_member(workloads[i], precision, s, dev, stream, reps)
        best = min(t, key=t.get)
        if best:
            settings[i] = dict(heavy_settings[best])
        times[f"heavy{i}"] = t
    ctas = 2
    if light:
        lw = [workloads[i] for i in light]
        tl = {}
        for cps in ctas_candidates:
            b = UnevenBatch(lw, precision=precision, ctas_per_sm=cps, device=device)
            b.capture()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b.replay()
            ev0.record(b.stream)
            for _ in range(reps):
                b.replay()
            ev1.record(b.stream)
            ev1.synchronize()
            tl[cps] = ev0.elapsed_time(ev1) / reps
            b.close()
        ctas = min(tl, key=tl.get)
        times["light_ctas_per_sm"] = tl
    ch = {"ctas_per_sm": ctas, "settings": {str(i): s for i, s in settings.items()},
          "ms": {k: ({str(a): b for a, b in v.items()} if isinstance(v, dict) else v) for k, v in times.items()}}
    cache[key] = ch
    _store(cache)
    return UnevenBatch(workloads, precision=precision, ctas_per_sm=ctas, settings=settings, device=device), ch, \
        ch["ms"]
