"""Pauli-frame sampler: synthetic detection events of a noisy circuit.

Input generation, independent of the error analysis: every shot carries an
X/Z Pauli frame (the error accumulated so far relative to the noiseless
run), bit-packed 64 shots per word.  Gates conjugate the frame, noise
channels draw their Paulis from their definitions (X_ERROR / Z_ERROR: the
Pauli with probability p; DEPOLARIZE1: one of X, Y, Z with p/3 each;
DEPOLARIZE2: one of the 15 non-identity two-qubit Paulis with p/15 each), a
Z-basis measurement reads the frame's X bit (X-basis: the Z bit), and a
detector or observable is the XOR of the records it names.  After every
reset or measurement the frame part an eigenstate absorbs is redrawn at
random, so a deterministic detector is blind to it.
"""
from __future__ import annotations

import numpy as np

from . import circuits as C


class _Bits:
    def __init__(self, shots: int, rng):
        self.shots = shots
        self.words = (shots + 63) // 64
        self.rng = rng
        self.tail = np.uint64((1 << (shots % 64)) - 1) if shots % 64 else np.uint64(0xFFFFFFFFFFFFFFFF)

    def zeros(self):
        return np.zeros(self.words, np.uint64)

    def random(self):
        b = self.rng.integers(0, 1 << 63, size=self.words, dtype=np.uint64) << np.uint64(1)
        b ^= self.rng.integers(0, 2, size=self.words, dtype=np.uint64)
        b[-1] &= self.tail
        return b

    def hits(self, p: float):
        """Shot indices hit by an event of probability p."""
        k = self.rng.binomial(self.shots, p)
        return self.rng.choice(self.shots, size=k, replace=False) if k else np.zeros(0, np.int64)

    @staticmethod
    def flip(arr, shots):
        np.bitwise_xor.at(arr, shots >> 6, np.left_shift(np.uint64(1), (shots & 63).astype(np.uint64)))


def sample(circuit: C.Circuit, noise: np.ndarray, shots: int, seed: int = 0):
    """Detection events and observable flips of ``shots`` runs.

    Returns (detectors, observables) as bool arrays of shape (shots, n) --
    the noise vector gives each location's channel parameter."""
    rng = np.random.default_rng(seed)
    bits = _Bits(shots, rng)
    nq = circuit.n_qubits
    X = np.zeros((nq, bits.words), np.uint64)
    Z = np.zeros((nq, bits.words), np.uint64)
    for q in range(nq):                      # |0>: Z part absorbed
        Z[q] = bits.random()
    ops, recs = circuit.ops, circuit.recs
    p = np.asarray(noise, dtype=np.float64)
    meas = []
    dets = np.zeros((circuit.n_detectors, bits.words), np.uint64)
    obs = np.zeros((max(circuit.n_observables, 1), bits.words), np.uint64)
    n_det = 0
    for row in ops:
        k, a, b, c = (int(x) for x in row)
        if k == C.TICK:
            continue
        if k in (C.R, C.M, C.MR):
            if k != C.R:
                meas.append(X[a].copy())
            if k != C.M:
                X[a] = 0
            Z[a] = bits.random()
        elif k in (C.RX, C.MX, C.MRX):
            if k != C.RX:
                meas.append(Z[a].copy())
            if k != C.MX:
                Z[a] = 0
            X[a] = bits.random()
        elif k == C.H:
            X[a], Z[a] = Z[a].copy(), X[a].copy()
        elif k == C.S:
            Z[a] ^= X[a]
        elif k == C.CX:
            X[b] ^= X[a]
            Z[a] ^= Z[b]
        elif k == C.CZ:
            Z[a] ^= X[b]
            Z[b] ^= X[a]
        elif k == C.X_ERROR:
            bits.flip(X[a], bits.hits(p[c]))
        elif k == C.Z_ERROR:
            bits.flip(Z[a], bits.hits(p[c]))
        elif k == C.DEPOLARIZE1:
            h = bits.hits(p[c])
            which = rng.integers(1, 4, size=h.size)          # 1 X, 2 Z, 3 Y
            bits.flip(X[a], h[(which & 1) == 1])
            bits.flip(Z[a], h[(which & 2) == 2])
        elif k == C.DEPOLARIZE2:
            h = bits.hits(p[c])
            which = rng.integers(1, 16, size=h.size)         # 4 bits: xa za xb zb
            bits.flip(X[a], h[(which & 1) == 1])
            bits.flip(Z[a], h[(which & 2) == 2])
            bits.flip(X[b], h[(which & 4) == 4])
            bits.flip(Z[b], h[(which & 8) == 8])
        elif k in (C.DETECTOR, C.OBSERVABLE_INCLUDE):
            acc = bits.zeros()
            for j in range(b):
                acc ^= meas[len(meas) - int(recs[a + j])]
            if k == C.DETECTOR:
                dets[n_det] = acc
                n_det += 1
            else:
                obs[c] ^= acc
        else:
            raise ValueError(f"unknown row kind {k}")

    def unpack(words):
        by = words.view(np.uint8).reshape(words.shape[0], -1)
        return np.unpackbits(by, axis=1, bitorder="little")[:, :shots].T.astype(bool)
    return unpack(dets), unpack(obs[:circuit.n_observables])
