"""Noise recalibration with the adjoint: fit channel parameters to
detection-event statistics.

A compiled model gives every hyperedge e a probability P_e (Eq. pmerge) as a
differentiable function of the noise vector (forward and adjoint kernels,
``DemFunction``).  Its detector statistics follow in closed form: the
hyperedges fire independently, so a detector (or the XOR of two) fires with
probability 1/2 (1 - prod (1 - 2 P_e)) over the hyperedges that flip it an
odd number of times.  ``fit_groups`` matches the single-detector rates and
the XOR rates of detector pairs that share a hyperedge against sampled ones,
with the noise vector tied to a few group parameters (one per channel
class), by quasi-Newton steps on gradients through the adjoint.
"""
from __future__ import annotations

import numpy as np
import torch

from .dem import DemFunction, DeviceCircuit


class DetectorStatistics:
    """Model rates of one circuit's hypergraph: det_offsets / det_idx are the
    compile's CSR (host arrays), fixed while every noise value stays > 0."""

    def __init__(self, det_offsets, det_idx, n_detectors: int, device="cuda"):
        off = np.asarray(det_offsets, np.int64)
        idx = np.asarray(det_idx, np.int64)
        counts = np.diff(off)
        self.n_detectors = int(n_detectors)
        pair_of: dict = {}
        pair_edge, pair_slot = [], []
        for e in np.flatnonzero(counts >= 2):
            ds = idx[off[e]:off[e + 1]]
            for i in range(ds.size):
                for j in range(i + 1, ds.size):
                    slot = pair_of.setdefault((int(ds[i]), int(ds[j])), len(pair_of))
                    pair_edge.append(e)
                    pair_slot.append(slot)
        self.pairs = np.array(sorted(pair_of, key=pair_of.get), np.int64).reshape(-1, 2)
        t = lambda a: torch.as_tensor(np.asarray(a, np.int64), device=device)
        self._entry_edge = t(np.repeat(np.arange(counts.size), counts))
        self._det = t(idx)
        self._pair_edge = t(pair_edge)
        self._pair_slot = t(pair_slot)
        self._pi, self._pj = t(self.pairs[:, 0]), t(self.pairs[:, 1])

    def model(self, prob: torch.Tensor):
        """(detector rates, pair XOR rates) for hyperedge probabilities."""
        logt = torch.log1p(-2.0 * prob.double().clamp(max=0.499999))
        s = torch.zeros(self.n_detectors, dtype=torch.float64, device=prob.device)
        s = s.index_add(0, self._det, logt[self._entry_edge])
        both = torch.zeros(self.pairs.shape[0], dtype=torch.float64, device=prob.device)
        both = both.index_add(0, self._pair_slot, logt[self._pair_edge])
        rates = 0.5 * (1.0 - torch.exp(s))
        xor = 0.5 * (1.0 - torch.exp(s[self._pi] + s[self._pj] - 2.0 * both))
        return rates, xor

    def empirical(self, detections: np.ndarray):
        """The same statistics from sampled detection events (shots, n)."""
        d = np.asarray(detections, bool)
        rates = d.mean(axis=0)
        xor = (d[:, self.pairs[:, 0]] ^ d[:, self.pairs[:, 1]]).mean(axis=0)
        return rates, xor


def location_kinds(circuit) -> np.ndarray:
    """Channel kind of every noise location (X_ERROR, Z_ERROR, DEPOLARIZE1,
    DEPOLARIZE2), read from the circuit's noise rows."""
    ops = circuit.ops
    rows = ops[(ops[:, 0] >= 32) & (ops[:, 0] <= 35)]
    kinds = np.zeros(circuit.n_locations, np.int64)
    kinds[rows[:, 3].astype(np.int64)] = rows[:, 0]
    return kinds


def fit_groups(driver, circuit, groups, detections, p0, steps: int = 100, level: str = "L2"):
    """Fit one noise parameter per group to sampled detection events.

    groups: group id of every noise location (length n_locations); p0:
    starting parameters; detections: (shots, n_detectors) bool.  The
    parameters are fitted in log space by L-BFGS with a strong-Wolfe line
    search (a few parameters, an ill-conditioned valley where groups trade
    off: first-order steps stall there); ``steps`` bounds the loss
    evaluations, each one compile and one adjoint.  Returns the fitted
    parameters and the loss of every evaluation."""
    dc = circuit if isinstance(circuit, DeviceCircuit) else DeviceCircuit(circuit)
    g = torch.as_tensor(np.asarray(groups, np.int64), device="cuda")
    theta = torch.log(torch.as_tensor(np.asarray(p0, np.float64), device="cuda")).requires_grad_(True)
    host = driver.compile(dc, torch.exp(theta.detach())[g].float(), level).to_host()
    stats = DetectorStatistics(host["det_offsets"], host["det_idx"], detections.shape[1])
    r_obs, x_obs = stats.empirical(detections)
    shots = detections.shape[0]
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    r_obs, x_obs = dev(r_obs), dev(x_obs)
    # inverse binomial variances (floored for rare events)
    wr = shots / torch.clamp(r_obs * (1 - r_obs), min=1.0 / shots)
    wx = shots / torch.clamp(x_obs * (1 - x_obs), min=1.0 / shots)
    opt = torch.optim.LBFGS([theta], lr=1.0, max_iter=steps, max_eval=steps, line_search_fn="strong_wolfe",
                            tolerance_grad=1e-9, tolerance_change=1e-12)
    history = []

    def closure():
        opt.zero_grad()
        noise = torch.exp(theta)[g].float()
        prob, _ = DemFunction.apply(noise, driver, dc, level)
        rates, xor = stats.model(prob)
        loss = ((rates - r_obs) ** 2 * wr).sum() + ((xor - x_obs) ** 2 * wx).sum()
        loss.backward()
        history.append(float(loss.detach()))
        return loss

    opt.step(closure)
    return torch.exp(theta.detach()).cpu().numpy(), history
