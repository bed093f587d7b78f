"""The plain-text model writer and reader (CPU: the oracle's models)."""
import pytest

import oracle
from paper_2604_16613_gb300 import circuits as C
from paper_2604_16613_gb300.demtext import read_dem, write_dem


@pytest.mark.parametrize("make", [lambda: C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3)),
                                  lambda: C.bb_memory(1, C.NoiseModel.uniform(1e-3), seed=3)])
def test_round_trip_exact(make):
    circ = make()
    edges = oracle.analyze_circuit(circ).edges()
    text = write_dem(edges, circ.n_detectors, circ.n_observables)
    back, n_det, n_obs = read_dem(text)
    assert n_det == circ.n_detectors and n_obs == circ.n_observables
    assert back == {k: p for k, (p, _) in edges.items()}        # repr round-trips exactly


def test_reader_semantics():
    text = """
    # comment line
    error(0.1) D0 D1 L0
    error(0.2) D1 D0 L0          # same mechanism set: merged
    error(0.05) D0 ^ D0 D2       # decomposition: flips D2 only
    error(0.3) D3 ^ D3           # flips nothing: dropped
    detector(1, 2, 0) D7
    logical_observable L2
    """
    edges, n_det, n_obs = read_dem(text)
    assert edges[((0, 1), 1)] == pytest.approx(0.1 + 0.2 - 2 * 0.1 * 0.2)
    assert edges[((2,), 0)] == pytest.approx(0.05)
    assert len(edges) == 2
    assert (n_det, n_obs) == (8, 3)


@pytest.mark.parametrize("bad", ["repeat 3 {", "shift_detectors 2", "error(0.1) X3", "error(1.5) D0", "error 0.1 D0"])
def test_reader_rejects(bad):
    with pytest.raises(ValueError):
        read_dem(bad)
