"""Serving semantics on the oracle (no GPU): streaming a circuit cycle by
cycle through windows of 3H + K cycles and sealing the classes whose
smallest detector lies H cycles back gives exactly the classes of the
full-circuit compile (reading C17 of the scope table)."""
import numpy as np
import pytest

import oracle
from paper_2604_16613_gb300 import circuits as C

from serve_reference import HorizonError, serve


def full(circ, level="L2"):
    dem = oracle.analyze_circuit(circ, level=level)
    return {k: p for k, (p, w) in dem.edges().items()}


def check(circ, H, K, level="L2"):
    got, per_request = serve(circ, H, K, level)
    ref = full(circ, level)
    assert set(got) == set(ref)
    for k, p in ref.items():
        assert got[k] == pytest.approx(p, rel=1e-12, abs=0.0)
    return per_request


@pytest.mark.parametrize("K", [1, 2, 3])
def test_surface_stream_equals_full_compile(K):
    circ = C.rotated_surface_code_memory(3, 6, C.NoiseModel.uniform(1e-3))
    per_request = check(circ, H=1, K=K)
    # every request past the horizon seals something
    assert all(n > 0 for n in per_request[1:])


def test_surface_d5_log_uniform_noise():
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    circ._p = [C.log_uniform_noise(circ.n_locations, seed=11)]
    circ._frozen = None
    check(circ, H=1, K=1)


def test_levels():
    circ = C.rotated_surface_code_memory(3, 5, C.NoiseModel.uniform(2e-3))
    for level in ("L0", "L1"):
        check(circ, H=1, K=2, level=level)


def test_bb_stream():
    circ = C.bb_memory(4, C.NoiseModel.uniform(1e-3), seed=3)
    check(circ, H=1, K=2)


def test_adaptive_concatenated_stream():
    # outer checks may skip up to gamma = d/2 cycles, so H = gamma
    circ = C.concatenated_adaptive_branch(4, 7, seed=5, noise=C.NoiseModel.uniform(1e-3),
                                          layout=C.ConcatenatedLayout(4))
    check(circ, H=2, K=1)
    check(circ, H=3, K=2)


def delay_line(cycles: int, p: float = 1e-2):
    """A deterministic toy whose records reach one cycle back but whose
    errors surface later: a bucket brigade d -> b1 -> b2 moves one hop per
    cycle (each source is reset after handing its value on), ancilla a reads
    b2 every cycle, each detector compares consecutive readings.  An X error
    on d in cycle c flips the detectors of cycles c + 2 and c + 3, so the
    horizon must be 3."""
    c = C.Circuit(4)
    d, b1, b2, a = 0, 1, 2, 3
    c.gate1(C.R, [d, b1, b2, a])
    c.tick()
    prev = None
    for t in range(cycles):
        c.gate2(C.CX, [(b2, a)])
        c.tick()
        m = c.measure(C.M, [a])[0]
        c.detectors([[m] if prev is None else [m, prev]])
        prev = m
        c.tick()
        c.gate1(C.R, [a, b2])
        c.tick()
        c.gate2(C.CX, [(b1, b2)])
        c.tick()
        c.gate1(C.R, [b1])
        c.noise(C.X_ERROR, [d], p)
        c.tick()
        c.gate2(C.CX, [(d, b1)])
        c.tick()
        c.gate1(C.R, [d])
        c.tick()
        if t < cycles - 1:
            c.mark_cycle()
    md = c.measure(C.M, [d])[0]
    c.observable(0, [md])
    c.logicals = [np.array([d])]
    return c


def test_delay_line_needs_three_cycles():
    circ = delay_line(10)
    with pytest.raises(HorizonError):
        serve(circ, H=1, K=1)
    with pytest.raises(HorizonError):
        serve(circ, H=2, K=1)
    check(circ, H=3, K=1)


def test_short_horizon_is_detected():
    # H = 0 leaves no records-only cycles and nothing to detect with; the
    # adaptive code's outer detectors reach two cycles back, past H = 1
    circ = C.concatenated_adaptive_branch(4, 8, seed=5, noise=C.NoiseModel.uniform(1e-3),
                                          layout=C.ConcatenatedLayout(4))
    with pytest.raises((HorizonError, oracle.OracleError)):
        serve(circ, H=1, K=1)
