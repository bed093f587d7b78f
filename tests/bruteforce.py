"""Brute-force forward tracking (Sec. 2.1.5, "forward tracking") for tests.

Every error mechanism is injected on its own into a Pauli frame at its
space-time point and pushed forward through the rest of the circuit; the
measurements it flips give the detectors and observables it flips.  All
mechanisms are simulated at once, one frame column each (numpy bool arrays).

Random gauges: after every Z-basis reset or measurement the frame's Z part on
that qubit is re-randomised (an eigenstate of Z absorbs a Z error), likewise
X for X-basis operations, and the initial |0> state starts with a random Z
frame.  A deterministic detector cannot see these gauges, so (i) with no
injected errors every detector must read 0 on every shot, and (ii) the flips
caused by an injected error do not depend on the gauge draw.

This module is independent of both the oracle and the CUDA library; its
Pauli-component tables are written out here from Table tab:correlation-level.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from paper_2604_16613_gb300 import circuits as C

# one-qubit Pauli as (x, z)
_P = {"I": (0, 0), "X": (1, 0), "Z": (0, 1), "Y": (1, 1)}
# components per channel and level (order irrelevant here: keyed by name)
DEP1_BY_LEVEL = {0: ["X", "Z"], 1: ["X", "Z", "Y"], 2: ["X", "Z", "Y"]}
_L0 = ["IX", "IZ", "XI", "XX", "ZI", "ZZ"]
_L1 = _L0 + ["IY", "XZ", "YI", "ZX"]
_L2 = _L1 + ["XY", "YX", "YY", "YZ", "ZY"]
DEP2_BY_LEVEL = {0: _L0, 1: _L1, 2: _L2}


def components(kind: int, level: int) -> list[str]:
    if kind == C.X_ERROR:
        return ["X"]
    if kind == C.Z_ERROR:
        return ["Z"]
    if kind == C.DEPOLARIZE1:
        return DEP1_BY_LEVEL[level]
    if kind == C.DEPOLARIZE2:
        return DEP2_BY_LEVEL[level]
    raise ValueError(kind)


def _records(circuit):
    """(measurement index per row, detector list, observable lists)."""
    ops, recs = circuit.ops, circuit.recs
    meas_of_row = -np.ones(ops.shape[0], dtype=np.int64)
    dets, obs = [], {}
    nm = 0
    for i, (k, a, b, c) in enumerate(ops.tolist()):
        if k in C.MEASURE_KINDS:
            meas_of_row[i] = nm
            nm += 1
        elif k == C.DETECTOR:
            dets.append([nm - int(x) for x in recs[a:a + b]])
        elif k == C.OBSERVABLE_INCLUDE:
            obs.setdefault(c, []).extend(nm - int(x) for x in recs[a:a + b])
    n_obs = (max(obs) + 1) if obs else 0
    obs_lists = [obs.get(k, []) for k in range(n_obs)]
    return meas_of_row, nm, dets, obs_lists


def simulate(circuit, inject, n_cols, rng):
    """Forward frame simulation.

    inject: dict row -> list of (column, x_a, z_a, x_b, z_b) applied when the
    noise row is reached.  Returns (detector flips [D, n_cols], observable
    flips [O, n_cols]).
    """
    ops = circuit.ops
    n = circuit.n_qubits
    meas_of_row, nm, dets, obs_lists = _records(circuit)
    X = np.zeros((n, n_cols), dtype=bool)
    Z = rng.random((n, n_cols)) < 0.5          # gauge of |0>
    flips = np.zeros((max(nm, 1), n_cols), dtype=bool)
    for i, (k, a, b, c) in enumerate(ops.tolist()):
        if k == C.H:
            X[a], Z[a] = Z[a].copy(), X[a].copy()
        elif k == C.S:
            Z[a] ^= X[a]
        elif k == C.CX:
            X[b] ^= X[a]
            Z[a] ^= Z[b]
        elif k == C.CZ:
            Z[a] ^= X[b]
            Z[b] ^= X[a]
        elif k in (C.M, C.MR):
            flips[meas_of_row[i]] = X[a]
            Z[a] = rng.random(n_cols) < 0.5
            if k == C.MR:
                X[a] = False
        elif k == C.R:
            X[a] = False
            Z[a] = rng.random(n_cols) < 0.5
        elif k in (C.MX, C.MRX):
            flips[meas_of_row[i]] = Z[a]
            X[a] = rng.random(n_cols) < 0.5
            if k == C.MRX:
                Z[a] = False
        elif k == C.RX:
            Z[a] = False
            X[a] = rng.random(n_cols) < 0.5
        elif k in C.NOISE_KINDS and i in inject:
            for col, xa, za, xb, zb in inject[i]:
                X[a, col] ^= bool(xa)
                Z[a, col] ^= bool(za)
                if k == C.DEPOLARIZE2:
                    X[b, col] ^= bool(xb)
                    Z[b, col] ^= bool(zb)
    D = np.zeros((len(dets), n_cols), dtype=bool)
    for j, ms in enumerate(dets):
        for m in ms:
            D[j] ^= flips[m]
    O = np.zeros((len(obs_lists), n_cols), dtype=bool)
    for j, ms in enumerate(obs_lists):
        for m in ms:
            O[j] ^= flips[m]
    return D, O


def mechanism_masks(circuit, noise, level: int, seed: int = 0):
    """{(row, component name): (detector tuple, observable mask)} for every
    mechanism with probability > 0 whose flip set is non-empty."""
    ops = circuit.ops
    keys, inject = [], {}
    for i, (k, a, b, c) in enumerate(ops.tolist()):
        if k not in C.NOISE_KINDS or not noise[c] > 0:
            continue
        for name in components(k, level):
            if k == C.DEPOLARIZE2:
                xa, za = _P[name[0]]
                xb, zb = _P[name[1]]
            elif k == C.X_ERROR:
                xa, za, xb, zb = 1, 0, 0, 0
            elif k == C.Z_ERROR:
                xa, za, xb, zb = 0, 1, 0, 0
            else:
                xa, za = _P[name]
                xb = zb = 0
            inject.setdefault(i, []).append((len(keys), xa, za, xb, zb))
            keys.append((i, name))
    rng = np.random.default_rng(seed)
    D, O = simulate(circuit, inject, max(len(keys), 1), rng)
    out = {}
    for col, key in enumerate(keys):
        dets = tuple(int(j) for j in np.flatnonzero(D[:, col]))
        obs = 0
        for j in np.flatnonzero(O[:, col]):
            obs |= 1 << int(j)
        if dets or obs:
            out[key] = (dets, obs)
    return out


def noiseless_flips(circuit, shots: int = 256, seed: int = 1):
    """Detector and observable flips of the noiseless circuit under random gauges."""
    rng = np.random.default_rng(seed)
    return simulate(circuit, {}, shots, rng)


# ---- probabilities from the plain definitions -------------------------------

def boxplus(a, b):
    """Eq. pmerge: a [+] b = a(1-b) + b(1-a)."""
    return a * (1 - b) + b * (1 - a)


def component_probability(kind: int, p: float) -> float:
    """Probability of each independent component, derived here from the
    requirement that the components reproduce the channel (each non-identity
    Pauli of DEPOLARIZE1 with p/3, of DEPOLARIZE2 with p/15): the identity
    has probability (1 + 3(1-2q)^2)/4 resp. (1 + 15(1-2q)^8)/16, which must
    equal 1 - p."""
    if kind in (C.X_ERROR, C.Z_ERROR):
        return p
    if kind == C.DEPOLARIZE1:
        return 0.5 - 0.5 * math.sqrt((4 * (1 - p) - 1) / 3)
    if kind == C.DEPOLARIZE2:
        return 0.5 - 0.5 * ((16 * (1 - p) - 1) / 15) ** 0.125
    raise ValueError(kind)


def dem_from_masks(masks: dict, circuit, noise) -> dict:
    """Group brute-force masks and combine with iterated [+] in exact rationals
    of the floating component probabilities; returns {edge: P (float)}."""
    ops = circuit.ops
    groups: dict = {}
    for (row, name), edge in masks.items():
        k, a, b, c = ops[row].tolist()
        q = Fraction(component_probability(k, float(noise[c])))
        groups.setdefault(edge, []).append(q)
    out = {}
    for edge, qs in groups.items():
        acc = Fraction(0)
        for q in qs:
            acc = boxplus(acc, q)
        out[edge] = float(acc)
    return out
