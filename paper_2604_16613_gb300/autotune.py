"""Autotuner for the compile pipeline's launch shapes.

The tunables are those of ``gp_tuning``: threads and resident blocks per SM
for the stage-1 walk, and threads and blocks per SM for the grid-stride
stage-2 kernels.  The tuner times candidate shapes on the caller's own
workload (device-resident inputs, CUDA events on the compile stream, median
of a few compiles after a warm-up) by coordinate search: stage 1 first with
stage 2 fixed, then stage 2 with the chosen stage 1.  Results are cached per
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
        driver.set_tuning(t["stage1_threads"], t["stage1_blocks_per_sm"], t["stage2_threads"],
                          t["stage2_blocks_per_sm"])
        return dict(t)
    best = driver.get_tuning()
    best_ms = float("inf")
    trials = []
    for s1t, s1b in STAGE1:
        try:
            driver.set_tuning(s1t, s1b, best["stage2_threads"], best["stage2_blocks_per_sm"])
            ms = _time(driver, circuits, noise, level, repeats)
        except native.GpError:
            continue
        trials.append(((s1t, s1b, best["stage2_threads"], best["stage2_blocks_per_sm"]), ms))
        if ms < best_ms:
            best_ms, best = ms, driver.get_tuning()
    for s2t, s2b in STAGE2:
        try:
            driver.set_tuning(best["stage1_threads"], best["stage1_blocks_per_sm"], s2t, s2b)
            ms = _time(driver, circuits, noise, level, repeats)
        except native.GpError:
            continue
        trials.append(((best["stage1_threads"], best["stage1_blocks_per_sm"], s2t, s2b), ms))
        if ms < best_ms:
            best_ms, best = ms, driver.get_tuning()
    driver.set_tuning(best["stage1_threads"], best["stage1_blocks_per_sm"], best["stage2_threads"],
                      best["stage2_blocks_per_sm"])
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
