"""Autotuner for the compile pipeline's launch shapes.

The tunables are those of ``gp_tuning``: threads and resident blocks per SM
for the stage-1 walk and whether its emitters deal wide steps out lane by
lane, threads and blocks per SM for the grid-stride stage-2 kernels, and how
the observable walk is split (observable word columns, and the most time
segments of one observable walk).  The tuner times candidate shapes on the
caller's own workload (device-resident inputs, CUDA events on the compile
stream, median of a few compiles after a warm-up) by coordinate search:
stage 1 first with the rest fixed, then stage 2, then the observable split,
each with the choices made before it.  Results are cached per
workload signature.  Tuning changes only speed: the compile's outputs are
identical under every shape (classes are numbered by their smallest member
and class sums are exact integers).
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import native

STAGE1 = [(256, 0), (512, 0), (1024, 0), (512, 1), (256, 1)]
STAGE2 = [(256, 8), (128, 16), (512, 4), (256, 4), (256, 16), (512, 8)]
# (observable word columns, most time segments of one observable walk)
OBS_SPLIT = [(4, 3), (1, 3), (2, 3), (8, 3), (4, 2), (4, 1)]
FIELDS = ("stage1_threads", "stage1_blocks_per_sm", "stage2_threads", "stage2_blocks_per_sm", "obs_words",
          "obs_segments", "stage1_wide_emit")

_cache: dict = {}


def signature(circuits, level) -> str:
    cl = circuits if isinstance(circuits, (list, tuple)) else [circuits]
    qubits = max(c.n_qubits for c in cl)
    rows = sum(c.n_ops for c in cl)
    return f"B{len(cl)}-q{qubits}-r{rows >> 12}-{level}"


def _time(driver, circuits, noise, level, repeats: int) -> float:
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    driver.compile(circuits, noise, level)          # warm-up (also re-captures the graph)
    times = []
    for _ in range(repeats):
        t0.record(stream)
        driver.compile(circuits, noise, level)
        t1.record(stream)
        t1.synchronize()
        times.append(t0.elapsed_time(t1))
    return statistics.median(times)


def autotune(driver, circuits, noise, level="L2", repeats: int = 5, cache_file: str | None = None,
             verbose: bool = False) -> dict:
    """Pick and apply the fastest launch shape for this workload; returns it
    with the measured milliseconds per compile."""
    key = signature(circuits, level)
    if cache_file and os.path.exists(cache_file):
        try:
            _cache.update(json.load(open(cache_file)))
        except (OSError, ValueError):
            pass
    if key in _cache:
        t = _cache[key]
        driver.set_tuning(**{f: t[f] for f in FIELDS if f in t})
        return dict(t)
    best = driver.get_tuning()
    best_ms = float("inf")
    trials = []
    n_obs = max(c.n_observables for c in (circuits if isinstance(circuits, (list, tuple)) else [circuits]))

    def trial(**change):
        nonlocal best, best_ms
        shape = dict(best, **change)
        try:
            driver.set_tuning(**shape)
            ms = _time(driver, circuits, noise, level, repeats)
        except native.GpError:
            return
        trials.append((tuple(shape[f] for f in FIELDS), ms))
        if ms < best_ms:
            best_ms, best = ms, driver.get_tuning()

    for s1t, s1b in STAGE1:
        trial(stage1_threads=s1t, stage1_blocks_per_sm=s1b)
    trial(stage1_wide_emit=1 - best["stage1_wide_emit"])
    for s2t, s2b in STAGE2:
        trial(stage2_threads=s2t, stage2_blocks_per_sm=s2b)
    if n_obs:
        for ow, osg in OBS_SPLIT:
            if ow <= max(n_obs, 1):
                trial(obs_words=ow, obs_segments=osg)
    driver.set_tuning(**best)
    if verbose:
        for shape, ms in trials:
            print(f"  tune {shape}: {ms:.3f} ms")
    result = dict(best, ms=best_ms)
    _cache[key] = result
    if cache_file:
        try:
            json.dump(_cache, open(cache_file, "w"), indent=1)
        except OSError:
            pass
    return dict(result)
