"""The Pauli-frame sampler against the oracle's model (CPU).

The sampler simulates the channels from their definitions and shares nothing
with the error analysis, so agreement pins both: sampled single-detector
rates and XOR rates of detector pairs must match 1/2 (1 - prod (1 - 2 P_e))
over the oracle's hyperedges (Eq. pmerge) within sampling error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2604_16613_gb300 import circuits as C
from paper_2604_16613_gb300.calibrate import DetectorStatistics
from paper_2604_16613_gb300.sampler import sample


def oracle_csr(dem):
    edges = sorted(dem.edges().items())
    off, idx, prob = [0], [], []
    for (dets, _obs), (p, _w) in edges:
        idx.extend(dets)
        off.append(len(idx))
        prob.append(p)
    return np.array(off), np.array(idx, np.int64), np.array(prob)


def test_noiseless_circuit_never_fires():
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    d, o = sample(circ, np.zeros(circ.n_locations), 2048, seed=1)
    assert not d.any() and not o.any()


@pytest.mark.parametrize("make", [lambda: C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(3e-3)),
                                  lambda: C.bb_memory(1, C.NoiseModel.uniform(2e-3), seed=3)])
def test_sampled_statistics_match_oracle_model(make):
    circ = make()
    noise = np.asarray(circ.default_noise, np.float64)
    shots = 1 << 16
    det, _ = sample(circ, noise, shots, seed=7)
    off, idx, prob = oracle_csr(oracle.analyze_circuit(circ, noise))
    stats = DetectorStatistics(off, idx, circ.n_detectors, device="cpu")
    r_model, x_model = (t.numpy() for t in stats.model(torch.tensor(prob)))
    r_emp, x_emp = stats.empirical(det)
    for model, emp in ((r_model, r_emp), (x_model, x_emp)):
        z = (emp - model) / np.sqrt(np.maximum(model * (1 - model), 1e-9) / shots)
        assert np.abs(z).max() < 5.0
