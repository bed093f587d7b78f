"""Circuit IR and seeded synthetic workload generators.

This module only BUILDS inputs: realised, fully unrolled, noisy Clifford
syndrome-measurement circuits (Sec. 2.1.2-2.1.3) and per-location noise
vectors.  It holds none of the error-analysis arithmetic (no sensitivity
propagation, no mechanism probabilities, no grouping): both the CUDA path and
the CPU oracle consume what it produces, and neither is imported here.

Flat circuit format (shared interface, parsed independently by each side)
-------------------------------------------------------------------------
``ops``  uint32 array of shape (n_ops, 4): rows ``(kind, a, b, c)`` in time order.

====================  =====================================================
kind                  operands
====================  =====================================================
TICK (0)              layer boundary
R/M/MR (1/2/3)        a = qubit (Z basis reset / measure / measure+reset)
RX/MX/MRX (4/5/6)     a = qubit (X basis variants)
H/S (8/9)             a = qubit
CX (10)               a = control, b = target
CZ (11)               a, b = qubits
DETECTOR (16)         a = offset into ``recs``, b = number of records
OBSERVABLE_INCLUDE    a = offset into ``recs``, b = number of records,
(17)                  c = observable index
X_ERROR/Z_ERROR (32/33) a = qubit, c = noise location
DEPOLARIZE1 (34)      a = qubit, c = noise location
DEPOLARIZE2 (35)      a, b = qubits, c = noise location
====================  =====================================================

``recs`` uint32 array of measurement-record lookbacks: ``k`` names the k-th
most recent measurement before the annotation (``rec[-k]``, k >= 1).
Detectors and observables are numbered in declaration order.

Layer rule: between two TICKs every qubit takes part in at most one gate; a
noise op on a qubit that still has a gate later in the same layer acts before
that gate, otherwise after the layer's gate on it.
"""
from __future__ import annotations

import math
import re
from dataclasses import dataclass, field

import numpy as np

TICK = 0
R, M, MR, RX, MX, MRX = 1, 2, 3, 4, 5, 6
H, S = 8, 9
CX, CZ = 10, 11
DETECTOR, OBSERVABLE_INCLUDE = 16, 17
X_ERROR, Z_ERROR, DEPOLARIZE1, DEPOLARIZE2 = 32, 33, 34, 35

MEASURE_KINDS = (M, MR, MX, MRX)
RESET_KINDS = (R, MR, RX, MRX)
NOISE_KINDS = (X_ERROR, Z_ERROR, DEPOLARIZE1, DEPOLARIZE2)
ONE_QUBIT_GATES = (R, M, MR, RX, MX, MRX, H, S)
TWO_QUBIT_GATES = (CX, CZ)

_NAMES = {
    "TICK": TICK, "R": R, "M": M, "MR": MR, "RX": RX, "MX": MX, "MRX": MRX,
    "H": H, "S": S, "CX": CX, "CNOT": CX, "CZ": CZ, "DETECTOR": DETECTOR,
    "OBSERVABLE_INCLUDE": OBSERVABLE_INCLUDE, "X_ERROR": X_ERROR,
    "Z_ERROR": Z_ERROR, "DEPOLARIZE1": DEPOLARIZE1, "DEPOLARIZE2": DEPOLARIZE2,
}
KIND_NAMES = {v: k for k, v in _NAMES.items() if k != "CNOT"}


class Circuit:
    """Incremental builder for the flat format above.

    Noise methods allocate consecutive location indices and remember the
    channel parameter given at build time as the default noise vector.
    """

    def __init__(self, n_qubits: int):
        self.n_qubits = int(n_qubits)
        self._ops: list[np.ndarray] = []
        self._recs: list[np.ndarray] = []
        self._n_recs = 0
        self._p: list[np.ndarray] = []
        self.n_locations = 0
        self.n_measurements = 0
        self.n_detectors = 0
        self.n_observables = 0
        self.n_ticks = 0
        self._frozen: tuple | None = None
        # cycle boundaries for serving: (rows, recs, locations, measurements,
        # detectors) counted at the end of every cycle but the last
        self.cycle_marks: list[tuple] = []
        # declared logical operators: per observable, the qubits whose Z
        # measurement defines it at a cycle boundary
        self.logicals: list[np.ndarray] = []

    # -- raw appends -------------------------------------------------------
    def _append(self, rows: np.ndarray) -> None:
        self._frozen = None
        self._ops.append(np.ascontiguousarray(rows, dtype=np.uint32))

    def tick(self) -> None:
        self._append(np.array([[TICK, 0, 0, 0]]))
        self.n_ticks += 1

    def gate1(self, kind: int, qubits) -> None:
        q = np.asarray(qubits, dtype=np.int64).reshape(-1)
        if q.size == 0:
            return
        assert kind in ONE_QUBIT_GATES
        assert q.min() >= 0 and q.max() < self.n_qubits
        rows = np.zeros((q.size, 4), dtype=np.uint32)
        rows[:, 0] = kind
        rows[:, 1] = q
        self._append(rows)

    def measure(self, kind: int, qubits) -> np.ndarray:
        """Append measurements; returns their absolute record indices."""
        assert kind in MEASURE_KINDS
        q = np.asarray(qubits, dtype=np.int64).reshape(-1)
        self.gate1(kind, q)
        idx = np.arange(self.n_measurements, self.n_measurements + q.size, dtype=np.int64)
        self.n_measurements += q.size
        return idx

    def gate2(self, kind: int, pairs) -> None:
        p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
        if p.shape[0] == 0:
            return
        assert kind in TWO_QUBIT_GATES
        assert p.min() >= 0 and p.max() < self.n_qubits
        assert np.all(p[:, 0] != p[:, 1])
        rows = np.zeros((p.shape[0], 4), dtype=np.uint32)
        rows[:, 0] = kind
        rows[:, 1:3] = p
        self._append(rows)

    def _rec_block(self, kind: int, groups, extra: int = 0) -> None:
        rows = []
        for g in groups:
            g = np.asarray(g, dtype=np.int64).reshape(-1)
            assert g.size == 0 or (g.min() >= 0 and g.max() < self.n_measurements), \
                "annotation refers to a future measurement"
            look = (self.n_measurements - g).astype(np.uint32)
            rows.append((kind, self._n_recs, look.size, extra))
            self._recs.append(look)
            self._n_recs += look.size
        if rows:
            self._append(np.array(rows, dtype=np.uint32))

    def detector(self, records) -> int:
        """One DETECTOR over absolute record indices; returns its index."""
        self._rec_block(DETECTOR, [records])
        self.n_detectors += 1
        return self.n_detectors - 1

    def detectors(self, groups) -> None:
        groups = list(groups)
        self._rec_block(DETECTOR, groups)
        self.n_detectors += len(groups)

    def observable(self, index: int, records) -> None:
        self._rec_block(OBSERVABLE_INCLUDE, [records], extra=int(index))
        self.n_observables = max(self.n_observables, int(index) + 1)

    def noise(self, kind: int, targets, p) -> np.ndarray:
        """Append one noise site per qubit (or pair); returns their locations."""
        assert kind in NOISE_KINDS
        width = 2 if kind == DEPOLARIZE2 else 1
        t = np.asarray(targets, dtype=np.int64).reshape(-1, width)
        k = t.shape[0]
        if k == 0:
            return np.zeros(0, dtype=np.int64)
        assert t.min() >= 0 and t.max() < self.n_qubits
        locs = np.arange(self.n_locations, self.n_locations + k, dtype=np.int64)
        rows = np.zeros((k, 4), dtype=np.uint32)
        rows[:, 0] = kind
        rows[:, 1] = t[:, 0]
        if width == 2:
            rows[:, 2] = t[:, 1]
        rows[:, 3] = locs
        self._append(rows)
        self._p.append(np.broadcast_to(np.asarray(p, dtype=np.float64), (k,)).copy())
        self.n_locations += k
        return locs

    def noise_at(self, kind: int, targets, location: int) -> None:
        """Append noise sites that all read the given existing location."""
        width = 2 if kind == DEPOLARIZE2 else 1
        t = np.asarray(targets, dtype=np.int64).reshape(-1, width)
        if t.shape[0] == 0:
            return
        assert 0 <= location < self.n_locations
        rows = np.zeros((t.shape[0], 4), dtype=np.uint32)
        rows[:, 0] = kind
        rows[:, 1] = t[:, 0]
        if width == 2:
            rows[:, 2] = t[:, 1]
        rows[:, 3] = location
        self._append(rows)

    def mark_cycle(self) -> None:
        """End the current cycle here (the serving stream cuts the circuit
        at these marks)."""
        self.cycle_marks.append((self.n_ops, self._n_recs, self.n_locations, self.n_measurements,
                                 self.n_detectors))

    def cycle_blocks(self) -> list[dict]:
        """The circuit cut at its cycle marks, each piece self-contained:
        detector and observable rows index the piece's own record array and
        noise rows its own locations (record lookbacks stay relative and may
        reach into earlier pieces).  Concatenating the pieces, with those
        offsets added back, gives the circuit."""
        ops, recs, p = self._freeze()
        ends = list(self.cycle_marks) + [(ops.shape[0], recs.size, self.n_locations, self.n_measurements,
                                          self.n_detectors)]
        out, start = [], (0, 0, 0, 0, 0)
        for i, end in enumerate(ends):
            r0, c0, l0, m0, d0 = start
            r1, c1, l1, m1, d1 = end
            o = ops[r0:r1].copy()
            k = o[:, 0]
            ann = (k == DETECTOR) | (k == OBSERVABLE_INCLUDE)
            o[ann, 1] -= np.uint32(c0)
            nz = np.isin(k, NOISE_KINDS)
            o[nz, 3] -= np.uint32(l0)
            out.append(dict(ops=o, recs=recs[c0:c1].copy(), noise=p[l0:l1].copy(), n_detectors=d1 - d0,
                            n_measurements=m1 - m0, n_locations=l1 - l0, n_ticks=int((k == TICK).sum()),
                            final=i == len(ends) - 1))
            start = end
        return out

    # -- views -------------------------------------------------------------
    def _freeze(self):
        if self._frozen is None:
            ops = (np.concatenate(self._ops) if self._ops else np.zeros((0, 4), np.uint32))
            recs = (np.concatenate(self._recs).astype(np.uint32) if self._recs
                    else np.zeros(0, np.uint32))
            p = (np.concatenate(self._p) if self._p else np.zeros(0, np.float64))
            self._ops = [ops] if ops.shape[0] else []
            self._recs = [recs] if recs.size else []
            self._p = [p] if p.size else []
            self._frozen = (ops, recs, p)
        return self._frozen

    @property
    def ops(self) -> np.ndarray:
        return self._freeze()[0]

    @property
    def recs(self) -> np.ndarray:
        return self._freeze()[1]

    @property
    def default_noise(self) -> np.ndarray:
        return self._freeze()[2].copy()

    @property
    def n_ops(self) -> int:
        return int(self.ops.shape[0])

    @property
    def n_layers(self) -> int:
        return self.n_ticks + 1

    def n_sites(self) -> int:
        ops = self.ops
        return int(np.isin(ops[:, 0], NOISE_KINDS).sum())

    # -- text form (Stim-like subset) ---------------------------------------
    @staticmethod
    def from_text(text: str) -> "Circuit":
        """Parse a small Stim-like text form (one instruction per line)."""
        lines = []
        nq = 0
        for raw in text.splitlines():
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            m = re.match(r"^([A-Z_0-9]+)(?:\(([^)]*)\))?\s*(.*)$", line)
            if not m:
                raise ValueError(f"cannot parse line: {raw!r}")
            name, arg, rest = m.group(1), m.group(2), m.group(3).split()
            if name not in _NAMES:
                raise ValueError(f"unknown instruction {name}")
            lines.append((name, arg, rest))
            if _NAMES[name] not in (DETECTOR, OBSERVABLE_INCLUDE, TICK):
                for tok in rest:
                    nq = max(nq, int(tok) + 1)
        c = Circuit(nq)
        for name, arg, rest in lines:
            kind = _NAMES[name]
            if kind == TICK:
                c.tick()
            elif kind in (DETECTOR, OBSERVABLE_INCLUDE):
                recs = []
                for tok in rest:
                    mm = re.match(r"^rec\[-(\d+)\]$", tok)
                    if not mm:
                        raise ValueError(f"bad record target {tok}")
                    recs.append(c.n_measurements - int(mm.group(1)))
                if kind == DETECTOR:
                    c.detector(recs)
                else:
                    c.observable(int(float(arg)), recs)
            elif kind in NOISE_KINDS:
                width = 2 if kind == DEPOLARIZE2 else 1
                t = np.array([int(x) for x in rest]).reshape(-1, width)
                c.noise(kind, t, float(arg))
            elif kind in MEASURE_KINDS:
                c.measure(kind, [int(x) for x in rest])
            elif kind in TWO_QUBIT_GATES:
                c.gate2(kind, np.array([int(x) for x in rest]).reshape(-1, 2))
            else:
                c.gate1(kind, [int(x) for x in rest])
        return c

    def to_text(self, noise=None) -> str:
        noise = self.default_noise if noise is None else np.asarray(noise)
        out = []
        recs = self.recs
        for kind, a, b, cc in self.ops.tolist():
            name = KIND_NAMES[kind]
            if kind == TICK:
                out.append("TICK")
            elif kind == DETECTOR:
                out.append("DETECTOR " + " ".join(f"rec[-{k}]" for k in recs[a:a + b]))
            elif kind == OBSERVABLE_INCLUDE:
                out.append(f"OBSERVABLE_INCLUDE({cc}) " +
                           " ".join(f"rec[-{k}]" for k in recs[a:a + b]))
            elif kind == DEPOLARIZE2:
                out.append(f"{name}({float(noise[cc])!r}) {a} {b}")
            elif kind in NOISE_KINDS:
                out.append(f"{name}({float(noise[cc])!r}) {a}")
            elif kind in TWO_QUBIT_GATES:
                out.append(f"{name} {a} {b}")
            else:
                out.append(f"{name} {a}")
        return "\n".join(out) + "\n"


# ---------------------------------------------------------------------------
# Noise vectors
# ---------------------------------------------------------------------------

def splitmix64(seed: int) -> int:
    """One step of the published splitmix64 generator (Steele et al. 2014)."""
    z = (seed + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """numpy generator whose seed is derived from (seed, stream) by splitmix64."""
    return np.random.default_rng(splitmix64((int(seed) << 16) ^ int(stream)))


def log_uniform_noise(n_locations: int, seed: int, lo: float = 1e-4, hi: float = 3e-3) -> np.ndarray:
    """Per-location probabilities exp(U[ln lo, ln hi]) (workload recipe of config 2)."""
    r = rng_for(seed, 2)
    return np.exp(r.uniform(math.log(lo), math.log(hi), size=n_locations))


# ---------------------------------------------------------------------------
# Noise model helper: circuit-level noise after every gate layer (Sec. 2.1.3)
# ---------------------------------------------------------------------------

@dataclass
class NoiseModel:
    """Circuit-level noise parameters (Sec. 2.1.3).

    p1: after single-qubit Clifford gates (DEPOLARIZE1)
    p2: after two-qubit gates (DEPOLARIZE2)
    pm: measurement flips (X_ERROR / Z_ERROR before the measurement)
    pr: reset failures (X_ERROR / Z_ERROR after the reset)
    pi: idle qubits in a layer (DEPOLARIZE1)
    """
    p1: float = 1e-3
    p2: float = 1e-3
    pm: float = 1e-3
    pr: float = 1e-3
    pi: float = 1e-3

    @staticmethod
    def uniform(p: float) -> "NoiseModel":
        return NoiseModel(p, p, p, p, p)

    @staticmethod
    def hardware_inspired(p: float) -> "NoiseModel":
        """p1 = pi = p/10 and p2 = pr = pm = p (Sec. 4)."""
        return NoiseModel(p / 10, p, p, p, p / 10)


class _Layer:
    """One TICK layer under construction, with idle bookkeeping."""

    def __init__(self, c: Circuit, nm: NoiseModel | None, qubits):
        self.c, self.nm = c, nm
        self.all = np.asarray(qubits, dtype=np.int64)
        self.busy = np.zeros(c.n_qubits, dtype=bool)
        self.pending_after: list[tuple[int, np.ndarray, float]] = []

    def reset(self, qubits, basis="Z"):
        q = np.asarray(qubits, dtype=np.int64)
        if q.size == 0:
            return
        self.busy[q] = True
        self.c.gate1(R if basis == "Z" else RX, q)
        if self.nm:
            self.pending_after.append((X_ERROR if basis == "Z" else Z_ERROR, q, self.nm.pr))

    def measure(self, qubits, basis="Z", reset=False) -> np.ndarray:
        q = np.asarray(qubits, dtype=np.int64)
        if q.size == 0:
            return np.zeros(0, dtype=np.int64)
        self.busy[q] = True
        if self.nm:
            self.c.noise(X_ERROR if basis == "Z" else Z_ERROR, q, self.nm.pm)
        kind = {("Z", False): M, ("Z", True): MR, ("X", False): MX, ("X", True): MRX}[(basis, reset)]
        rec = self.c.measure(kind, q)
        if reset and self.nm:
            self.pending_after.append((X_ERROR if basis == "Z" else Z_ERROR, q, self.nm.pr))
        return rec

    def single(self, kind, qubits):
        q = np.asarray(qubits, dtype=np.int64)
        if q.size == 0:
            return
        self.busy[q] = True
        self.c.gate1(kind, q)
        if self.nm:
            self.pending_after.append((DEPOLARIZE1, q, self.nm.p1))

    def two(self, kind, pairs):
        p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
        if p.shape[0] == 0:
            return
        assert not self.busy[p.reshape(-1)].any(), "qubit used twice in one layer"
        assert len(np.unique(p.reshape(-1))) == p.size, "qubit used twice in one layer"
        self.busy[p.reshape(-1)] = True
        self.c.gate2(kind, p)
        if self.nm:
            self.pending_after.append((DEPOLARIZE2, p, self.nm.p2))

    def close(self, tick=True):
        if self.nm:
            for kind, t, p in self.pending_after:
                self.c.noise(kind, t, p)
            idle = self.all[~self.busy[self.all]]
            if idle.size:
                self.c.noise(DEPOLARIZE1, idle, self.nm.pi)
        if tick:
            self.c.tick()


# ---------------------------------------------------------------------------
# Repetition / bit-flip code (Fig. 1)
# ---------------------------------------------------------------------------

def repetition_code_memory(d: int, rounds: int, noise: NoiseModel | None = None,
                           final_data: bool = True) -> Circuit:
    """Bit-flip repetition code on a line: data 0,2,..,2d-2, ancillas between.

    Each round: reset ancillas, CX layer {data 2i -> anc 2i+1}, CX layer
    {data 2i+2 -> anc 2i+1}, measure ancillas.  Round 1 detectors are the
    single ancilla outcomes, later rounds compare with the previous round;
    with ``final_data`` the data are measured and a last detector layer and
    observable (data qubit 0) are added.
    """
    n = 2 * d - 1
    c = Circuit(n)
    data = np.arange(0, n, 2)
    anc = np.arange(1, n, 2)
    allq = np.arange(n)
    prev = None
    L = _Layer(c, noise, allq)
    L.reset(allq)
    L.close()
    for r in range(rounds):
        if r > 0:
            L = _Layer(c, noise, allq)
            L.reset(anc)
            L.close()
        L = _Layer(c, noise, allq)
        L.two(CX, np.stack([data[:-1], anc], axis=1))
        L.close()
        L = _Layer(c, noise, allq)
        L.two(CX, np.stack([data[1:], anc], axis=1))
        L.close()
        L = _Layer(c, noise, allq)
        rec = L.measure(anc)
        L.close(tick=False)
        if prev is None:
            c.detectors([[m] for m in rec])
        else:
            c.detectors([[m, pm] for m, pm in zip(rec, prev)])
        prev = rec
        c.tick()
    if final_data:
        L = _Layer(c, noise, allq)
        drec = L.measure(data)
        L.close(tick=False)
        c.detectors([[drec[i], drec[i + 1], prev[i]] for i in range(d - 1)])
        c.observable(0, [drec[0]])
    return c


def fig1_bitflip_circuit() -> Circuit:
    """Noiseless d = 3 bit-flip code, two rounds, as drawn in Fig. 1(a).

    Data qubits 0, 2, 4; ancillas 1, 3.  CNOT layers {0->1, 2->3} and
    {2->1, 4->3} per round.  Detectors in declaration order: orange (first
    outcome of ancilla 1), green (first outcome of ancilla 3), blue (parity of
    the two outcomes of ancilla 1), yellow (same for ancilla 3).  A single
    X_ERROR site on data qubit 2 right after the second CNOT layer is E12.
    """
    c = Circuit(5)
    c.gate1(R, range(5))
    c.tick()
    c.gate2(CX, [(0, 1), (2, 3)])
    c.tick()
    c.gate2(CX, [(2, 1), (4, 3)])
    c.noise(X_ERROR, [2], 0.01)          # E12
    c.tick()
    r1 = c.measure(MR, [1, 3])
    c.detector([r1[0]])                  # orange
    c.detector([r1[1]])                  # green
    c.tick()
    c.gate2(CX, [(0, 1), (2, 3)])
    c.tick()
    c.gate2(CX, [(2, 1), (4, 3)])
    c.tick()
    r2 = c.measure(M, [1, 3])
    c.detector([r1[0], r2[0]])           # blue
    c.detector([r1[1], r2[1]])           # yellow
    return c


# ---------------------------------------------------------------------------
# Rotated surface code, Z-basis memory
# ---------------------------------------------------------------------------

@dataclass
class SurfaceLayout:
    d: int
    data_xy: np.ndarray               # (d*d, 2) coordinates of data qubits
    x_checks: list = field(default_factory=list)   # list of (qubit, [data per CX step or -1])
    z_checks: list = field(default_factory=list)
    n_qubits: int = 0
    data: np.ndarray | None = None
    xanc: np.ndarray | None = None
    zanc: np.ndarray | None = None
    z_logical: np.ndarray | None = None   # data qubit ids of Z_L (one row)
    x_logical: np.ndarray | None = None


# CX visiting orders (dx, dy) for the two plaquette types.  X checks finish on
# one row so their hook X errors lie along Z_L's direction (horizontal); Z
# checks finish on one column.  Interleaved in the same four layers, each X/Z
# pair that shares two data qubits meets them in the same relative order, so
# the two measurement circuits commute.
_X_ORDER = [(-1, -1), (1, -1), (-1, 1), (1, 1)]
_Z_ORDER = [(-1, -1), (-1, 1), (1, -1), (1, 1)]


def rotated_surface_layout(d: int) -> SurfaceLayout:
    """Rotated surface code of distance d (odd or even).

    Data qubits sit at odd coordinates (x, y) in [1, 2d-1]; measure qubits at
    even coordinates; a plaquette at (x, y) is X-type when (x + y)/2 is even.
    Weight-2 X plaquettes lie on the top/bottom edges, weight-2 Z plaquettes
    on the left/right edges.  Z_L is Z on the data row y = 1.
    """
    coords = [(x, y) for y in range(1, 2 * d, 2) for x in range(1, 2 * d, 2)]
    data_index = {xy: i for i, xy in enumerate(coords)}
    n_data = len(coords)
    xs, zs = [], []
    for y in range(0, 2 * d + 1, 2):
        for x in range(0, 2 * d + 1, 2):
            is_x = ((x + y) // 2) % 2 == 0
            interior = 0 < x < 2 * d and 0 < y < 2 * d
            if not interior:
                top_bottom = (y == 0 or y == 2 * d) and 0 < x < 2 * d
                left_right = (x == 0 or x == 2 * d) and 0 < y < 2 * d
                if not ((top_bottom and is_x) or (left_right and not is_x)):
                    continue
            order = _X_ORDER if is_x else _Z_ORDER
            nb = [data_index.get((x + dx, y + dy), -1) for dx, dy in order]
            (xs if is_x else zs).append(((x, y), nb))
    lay = SurfaceLayout(d=d, data_xy=np.array(coords))
    q = n_data
    for lst, out in ((xs, lay.x_checks), (zs, lay.z_checks)):
        for _, nb in lst:
            out.append((q, nb))
            q += 1
    lay.n_qubits = q
    lay.data = np.arange(n_data)
    lay.xanc = np.array([a for a, _ in lay.x_checks], dtype=np.int64)
    lay.zanc = np.array([a for a, _ in lay.z_checks], dtype=np.int64)
    lay.z_logical = np.array([data_index[(x, 1)] for x in range(1, 2 * d, 2)])
    lay.x_logical = np.array([data_index[(1, y)] for y in range(1, 2 * d, 2)])
    return lay


def rotated_surface_code_memory(d: int, rounds: int | None = None,
                                noise: NoiseModel | None = None, z_detectors_only: bool = False) -> Circuit:
    """Z-basis memory experiment on the rotated surface code (Sec. 4).

    Per round, TICK layers: reset ancillas (data too in round 1), H on X
    ancillas, four CX layers, H on X ancillas, measure ancillas.  Noise after
    every gate layer (Sec. 2.1.3): X_ERROR after resets and before
    measurements, DEPOLARIZE1 after single-qubit gates and on idle qubits,
    DEPOLARIZE2 after CX.  Round 1 has Z-check detectors only; later rounds
    compare each check with its previous outcome; the final data measurement
    closes every Z check and defines observable 0 = Z_L.
    Detector count: d (d^2 - 1).  With ``z_detectors_only`` the X checks are
    still measured but declare no detectors, (d^2 - 1)/2 (rounds + 1) in all:
    the detector set the configurable-correlation-level section pairs with
    level L0 in a Z-basis experiment.
    """
    rounds = d if rounds is None else rounds
    lay = rotated_surface_layout(d)
    c = Circuit(lay.n_qubits)
    c.layout = lay
    allq = np.arange(lay.n_qubits)
    anc = np.concatenate([lay.xanc, lay.zanc])
    checks = lay.x_checks + lay.z_checks
    n_x = len(lay.x_checks)
    prev = None
    for r in range(rounds):
        L = _Layer(c, noise, allq)
        L.reset(allq if r == 0 else anc)
        L.close()
        L = _Layer(c, noise, allq)
        L.single(H, lay.xanc)
        L.close()
        for k in range(4):
            L = _Layer(c, noise, allq)
            pairs = []
            for i, (a, nb) in enumerate(checks):
                dq = nb[k]
                if dq < 0:
                    continue
                pairs.append((a, dq) if i < n_x else (dq, a))
            L.two(CX, pairs)
            L.close()
        L = _Layer(c, noise, allq)
        L.single(H, lay.xanc)
        L.close()
        L = _Layer(c, noise, allq)
        rec = L.measure(anc)
        L.close(tick=False)
        if prev is None:
            c.detectors([[rec[n_x + i]] for i in range(len(lay.z_checks))])
        elif z_detectors_only:
            c.detectors([[rec[n_x + i], prev[n_x + i]] for i in range(len(lay.z_checks))])
        else:
            c.detectors([[m, pm] for m, pm in zip(rec, prev)])
        prev = rec
        c.tick()
        if r < rounds - 1:
            c.mark_cycle()
    L = _Layer(c, noise, allq)
    drec = L.measure(lay.data)
    L.close(tick=False)
    groups = []
    for i, (a, nb) in enumerate(lay.z_checks):
        groups.append([drec[q] for q in nb if q >= 0] + [prev[n_x + i]])
    c.detectors(groups)
    c.observable(0, [drec[q] for q in lay.z_logical])
    c.logicals = [np.asarray(lay.z_logical, dtype=np.int64)]
    return c


# ---------------------------------------------------------------------------
# Tiny random deterministic circuits (for brute-force pins)
# ---------------------------------------------------------------------------

def random_circuit(seed: int, n_qubits: int | None = None, n_blocks: int | None = None,
                   p_range=(1e-3, 5e-2)) -> Circuit:
    """A small random circuit whose detectors are deterministic by construction.

    Qubits are prepared in the Z or X basis, then blocks of random layers of
    H / S / CX / CZ are applied and undone in reverse order (S is its own
    inverse up to a Pauli, which leaves every basis measurement
    deterministic), after which a random subset of qubits is measured in its
    preparation basis.  Detectors are parities of one to three deterministic
    records; observables likewise.  Noise of every kind is sprinkled before and
    after gates.  Determinism is checked independently by the tests.
    """
    rng = rng_for(seed, 7)
    n = int(n_qubits or rng.integers(2, 7))
    blocks = int(n_blocks or rng.integers(1, 4))
    c = Circuit(n)
    basis = np.where(rng.random(n) < 0.35, 1, 0)       # 0 = Z, 1 = X
    pool: list[int] = []

    def p():
        return float(np.exp(rng.uniform(np.log(p_range[0]), np.log(p_range[1]))))

    def sprinkle(qubits_busy, before=None):
        # noise after this layer's gates (or on idle qubits)
        for q in range(n):
            if rng.random() < 0.45:
                kind = [X_ERROR, Z_ERROR, DEPOLARIZE1][rng.integers(0, 3)]
                c.noise(kind, [q], p())
        if n >= 2 and rng.random() < 0.6:
            a, b = rng.choice(n, size=2, replace=False)
            c.noise(DEPOLARIZE2, [(a, b)], p())

    # preparation
    c.gate1(R, np.flatnonzero(basis == 0))
    c.gate1(RX, np.flatnonzero(basis == 1))
    sprinkle(None)
    c.tick()
    for _ in range(blocks):
        layers = []
        for _ in range(int(rng.integers(1, 4))):
            perm = rng.permutation(n)
            ops = []
            i = 0
            while i < n:
                choice = rng.integers(0, 5)
                if choice >= 3 and i + 1 < n:
                    ops.append((CX if choice == 3 else CZ, int(perm[i]), int(perm[i + 1])))
                    i += 2
                else:
                    if choice < 2:
                        ops.append((H if choice == 0 else S, int(perm[i]), -1))
                    i += 1
            layers.append(ops)
        for ops in layers + layers[::-1]:
            # occasional noise placed before a gate in the same layer
            for kind, a, b in ops:
                if rng.random() < 0.2:
                    c.noise(DEPOLARIZE1, [a], p())
            for kind, a, b in ops:
                if b < 0:
                    c.gate1(kind, [a])
                else:
                    c.gate2(kind, [(a, b)])
            sprinkle(None)
            c.tick()
        # measurement layer on a random non-empty subset, each in its basis
        sub = np.flatnonzero(rng.random(n) < 0.7)
        if sub.size == 0:
            sub = np.array([int(rng.integers(0, n))])
        for q in sub:
            if rng.random() < 0.5:
                c.noise(X_ERROR if basis[q] == 0 else Z_ERROR, [q], p())
        recs = []
        for q in sub:
            reset = rng.random() < 0.4
            kind = (MR if reset else M) if basis[q] == 0 else (MRX if reset else MX)
            recs.append(int(c.measure(kind, [q])[0]))
        pool.extend(recs)
        for r in recs:
            k = int(rng.integers(0, 3))
            cand = [x for x in pool if x != r]
            others = list(rng.choice(cand, size=min(k, len(cand)), replace=False)) if cand else []
            c.detector([r] + [int(o) for o in others])
        sprinkle(None)
        c.tick()
        # re-prepare a few qubits, possibly in the other basis
        flip = np.flatnonzero(rng.random(n) < 0.25)
        if flip.size:
            newb = 1 - basis[flip]
            c.gate1(R, flip[newb == 0])
            c.gate1(RX, flip[newb == 1])
            basis[flip] = newb
            sprinkle(None)
            c.tick()
    for k in range(int(rng.integers(1, 3))):
        if pool:
            sel = rng.choice(pool, size=min(len(pool), int(rng.integers(1, 4))), replace=False)
            c.observable(k, [int(x) for x in sel])
    return c


# ---------------------------------------------------------------------------
# GF(2) helpers for code construction (inputs only)
# ---------------------------------------------------------------------------

def _gf2_rank_basis(rows: np.ndarray):
    """Row-echelon form over GF(2); returns (echelon rows, pivot columns)."""
    m = rows.copy().astype(np.uint8) & 1
    piv = []
    r = 0
    for c in range(m.shape[1]):
        if r >= m.shape[0]:
            break
        nz = np.flatnonzero(m[r:, c])
        if nz.size == 0:
            continue
        p = r + nz[0]
        if p != r:
            m[[r, p]] = m[[p, r]]
        others = np.flatnonzero(m[:, c])
        others = others[others != r]
        m[others] ^= m[r]
        piv.append(c)
        r += 1
    return m[:r], piv


def _gf2_kernel(h: np.ndarray) -> np.ndarray:
    """Basis of {v : h v = 0} over GF(2) (rows of the result)."""
    ech, piv = _gf2_rank_basis(h)
    n = h.shape[1]
    free = [c for c in range(n) if c not in set(piv)]
    basis = []
    for f in free:
        v = np.zeros(n, dtype=np.uint8)
        v[f] = 1
        for i, pc in enumerate(piv):
            if ech[i, f]:
                v[pc] = 1
        basis.append(v)
    return np.array(basis, dtype=np.uint8).reshape(-1, n)


def _greedy_colouring(edges, rng) -> list:
    """Greedy proper edge colouring of a bipartite multigraph given as (u, v)
    pairs in a seeded random order; returns one list of edges per colour."""
    order = rng.permutation(len(edges))
    used_u: dict = {}
    used_v: dict = {}
    colours: list = []
    for i in order:
        u, v = edges[i]
        cu, cv = used_u.setdefault(u, set()), used_v.setdefault(v, set())
        c = 0
        while c in cu or c in cv:
            c += 1
        cu.add(c)
        cv.add(c)
        while len(colours) <= c:
            colours.append([])
        colours[c].append((u, v))
    return colours


# ---------------------------------------------------------------------------
# Bivariate bicycle code [[144, 12, 12]] (Sec. 4), Z-basis memory
# ---------------------------------------------------------------------------

def bb_check_matrices(l: int = 12, m: int = 6):
    """H_X = [A | B], H_Z = [B^T | A^T] with A = x^3 + y + y^2 and
    B = y^3 + x + x^2, x = S_l (x) I_m and y = I_l (x) S_m (cyclic shifts)."""
    Sl = np.roll(np.eye(l, dtype=np.uint8), 1, axis=1)
    Sm = np.roll(np.eye(m, dtype=np.uint8), 1, axis=1)
    x = np.kron(Sl, np.eye(m, dtype=np.uint8))
    y = np.kron(np.eye(l, dtype=np.uint8), Sm)
    mp = np.linalg.matrix_power
    A = (mp(x, 3) + y + mp(y, 2)) % 2
    B = (mp(y, 3) + x + mp(x, 2)) % 2
    hx = np.concatenate([A, B], axis=1).astype(np.uint8)
    hz = np.concatenate([B.T, A.T], axis=1).astype(np.uint8)
    return hx, hz


def z_logicals(hx: np.ndarray, hz: np.ndarray) -> np.ndarray:
    """A basis of Z-type logical operators: kernel of H_X modulo the row space
    of H_Z (rows of the result)."""
    ker = _gf2_kernel(hx)
    ech, _ = _gf2_rank_basis(hz)
    rank = ech.shape[0]
    out = []
    cur = ech
    for v in ker:
        trial, _ = _gf2_rank_basis(np.vstack([cur, v[None, :]]))
        if trial.shape[0] > rank:
            out.append(v)
            cur, rank = trial, trial.shape[0]
    return np.array(out, dtype=np.uint8)


def css_memory_circuit(hx, hz, zlog, rounds: int, noise: NoiseModel | None, seed: int,
                       data_qubits=None) -> Circuit:
    """Z-basis memory of a CSS code with a seeded syndrome circuit.

    Per round: reset ancillas (data too in round 1), H on X ancillas, all
    Z-check CX layers (data -> ancilla), then all X-check CX layers
    (ancilla -> data), each block scheduled by a greedy edge colouring of its
    Tanner graph; H on X ancillas; measure ancillas.  Running the Z checks
    and X checks as separate blocks keeps the two measurement circuits
    commuting.  Detectors: Z checks in round 1, every check against its
    previous outcome afterwards, Z checks closed by the final data
    measurement; one observable per row of zlog.
    """
    n = hx.shape[1]
    nx, nz = hx.shape[0], hz.shape[0]
    data = np.arange(n)
    xanc = np.arange(n, n + nx)
    zanc = np.arange(n + nx, n + nx + nz)
    c = Circuit(n + nx + nz)
    allq = np.arange(c.n_qubits)
    rng = rng_for(seed, 3)
    z_edges = [(int(zanc[i]), int(j)) for i in range(nz) for j in np.flatnonzero(hz[i])]
    x_edges = [(int(xanc[i]), int(j)) for i in range(nx) for j in np.flatnonzero(hx[i])]
    z_layers = _greedy_colouring(z_edges, rng)
    x_layers = _greedy_colouring(x_edges, rng)
    anc = np.concatenate([xanc, zanc])
    prev = None
    for r in range(rounds):
        L = _Layer(c, noise, allq)
        L.reset(allq if r == 0 else anc)
        L.close()
        L = _Layer(c, noise, allq)
        L.single(H, xanc)
        L.close()
        for layer in z_layers:
            L = _Layer(c, noise, allq)
            L.two(CX, [(d_, a) for a, d_ in layer])
            L.close()
        for layer in x_layers:
            L = _Layer(c, noise, allq)
            L.two(CX, [(a, d_) for a, d_ in layer])
            L.close()
        L = _Layer(c, noise, allq)
        L.single(H, xanc)
        L.close()
        L = _Layer(c, noise, allq)
        rec = L.measure(anc)
        L.close(tick=False)
        if prev is None:
            c.detectors([[rec[nx + i]] for i in range(nz)])
        else:
            c.detectors([[m_, pm] for m_, pm in zip(rec, prev)])
        prev = rec
        c.tick()
        if r < rounds - 1:
            c.mark_cycle()
    L = _Layer(c, noise, allq)
    drec = L.measure(data)
    L.close(tick=False)
    c.detectors([[drec[j] for j in np.flatnonzero(hz[i])] + [prev[nx + i]] for i in range(nz)])
    for k, lg in enumerate(zlog):
        c.observable(k, [drec[j] for j in np.flatnonzero(lg)])
    c.logicals = [np.flatnonzero(lg).astype(np.int64) for lg in zlog]
    return c


def bb_memory(rounds: int = 12, noise: NoiseModel | None = None, seed: int = 3) -> Circuit:
    """[[144,12,12]] bivariate bicycle Z-memory (workload of config 3)."""
    hx, hz = bb_check_matrices(12, 6)
    zl = z_logicals(hx, hz)
    return css_memory_circuit(hx, hz, zl, rounds, noise, seed)


# ---------------------------------------------------------------------------
# Adaptive [[4,2,2]]-concatenated rotated surface code (Sec. 5)
# ---------------------------------------------------------------------------

def iceberg_pairs(d: int) -> list:
    """Pairs of outer data qubits sharing one [[4,2,2]] block.

    Eq. iceberg-mapping sends (r, c) to (d-1-r, (c+2) mod d).  That map is an
    involution only when d is a multiple of 4, so the pairs are taken along
    its orbits (each orbit has even length because the row flips at every
    step): consecutive orbit elements are paired, starting from the smallest
    row-major index.  Qubit index = r * d + c.
    """
    seen = set()
    pairs = []
    for start in range(d * d):
        if start in seen:
            continue
        orbit = []
        q = start
        while q not in orbit:
            orbit.append(q)
            r, cc = divmod(q, d)
            q = (d - 1 - r) * d + (cc + 2) % d
        assert len(orbit) % 2 == 0
        for i in range(0, len(orbit), 2):
            pairs.append((orbit[i], orbit[i + 1]))
        seen.update(orbit)
    return pairs


class ConcatenatedLayout:
    """Physical layout of the [[4,2,2]]-concatenated rotated surface code.

    Each block holds physical qubits p0..p3 with stabilisers XXXX and ZZZZ and
    two logical qubits: logical 1 has X1 = X p0 p1, Z1 = Z p0 p2; logical 2
    has X2 = X p0 p2, Z2 = Z p0 p1.  Outer data qubit q is logical j of block
    b; an outer check is the product of the matching logical operators.
    """

    def __init__(self, d: int):
        self.d = d
        self.surface = rotated_surface_layout(d)
        pairs = iceberg_pairs(d)
        self.n_blocks = len(pairs)
        self.block_of = {}
        for b, (q1, q2) in enumerate(pairs):
            self.block_of[q1] = (b, 1)
            self.block_of[q2] = (b, 2)
        # outer data index in the surface layout: coordinates -> r*d + c
        coords = self.surface.data_xy
        self.outer_id = {i: ((int(y) - 1) // 2) * d + (int(x) - 1) // 2 for i, (x, y) in enumerate(coords.tolist())}
        nb = self.n_blocks
        self.phys = np.arange(4 * nb).reshape(nb, 4)
        self.inner_x = np.arange(4 * nb, 5 * nb)
        self.inner_z = np.arange(5 * nb, 6 * nb)
        base = 6 * nb
        self.outer_checks = []            # (ancilla, is_x, physical support, outer qubits)
        for is_x, checks in ((True, self.surface.x_checks), (False, self.surface.z_checks)):
            for _, nb_list in checks:
                outer = [self.outer_id[q] for q in nb_list if q >= 0]
                blocks = [self.block_of[o][0] for o in outer]
                assert len(set(blocks)) == len(blocks), "two qubits of one block in a check"
                sup = set()
                for o in outer:
                    b, j = self.block_of[o]
                    p = self.phys[b]
                    if is_x:
                        op = (p[0], p[1]) if j == 1 else (p[0], p[2])
                    else:
                        op = (p[0], p[2]) if j == 1 else (p[0], p[1])
                    sup ^= set(int(v) for v in op)
                self.outer_checks.append((base, is_x, sorted(sup), outer))
                base += 1
        self.n_qubits = base
        # Z_L of the outer code on the data row y = 1 -> physical support
        zl = set()
        for i in self.surface.z_logical:
            b, j = self.block_of[self.outer_id[int(i)]]
            p = self.phys[b]
            zl ^= set(int(v) for v in ((p[0], p[2]) if j == 1 else (p[0], p[1])))
        self.z_logical = sorted(zl)


def concatenated_adaptive_branch(d: int = 10, cycles: int = 20, seed: int = 0, fire_rate: float = 0.05,
                                 noise: NoiseModel | None = None, layout: ConcatenatedLayout | None = None
                                 ) -> Circuit:
    """One realised branch of the adaptive [[4,2,2]]-concatenated surface-code
    memory (Sec. 5.1-5.2; workload of config 4).

    Every cycle measures all inner checks (ZZZZ block, then XXXX block).  The
    outer checks run in the first and last cycle and every gamma = d/2 cycles
    (Sec. 5.2.3); in other cycles only the outer checks touching a block whose
    inner syndrome fired run, a block firing with seeded Bernoulli(fire_rate)
    per cycle.  Detectors are instantiated dynamically (Sec. 5.2.4): a check
    gets a detector when it runs and has a previous outcome; Z-type checks
    also on their first run (deterministic from |0>).  The final cycle
    measures the physical data: inner ZZZZ and outer Z checks are closed and
    the outer Z_L is observable 0.
    """
    lay = layout or ConcatenatedLayout(d)
    rng = rng_for(seed, 4)
    gamma = max(1, d // 2)
    c = Circuit(lay.n_qubits)
    allq = np.arange(lay.n_qubits)
    phys = lay.phys.reshape(-1)
    last = {}                        # check id -> last measurement record

    def run_checks(checks):
        """checks: list of (id, ancilla, is_x, physical support)."""
        if not checks:
            return
        anc = np.array([a for _, a, _, _ in checks])
        xanc = np.array([a for _, a, ix, _ in checks if ix], dtype=np.int64)
        L = _Layer(c, noise, allq)
        L.reset(anc)
        L.close()
        L = _Layer(c, noise, allq)
        L.single(H, xanc)
        L.close()
        for want_x in (False, True):
            edges = [(a, q) for _, a, ix, sup in checks if ix == want_x for q in sup]
            for layer in _greedy_colouring(edges, rng):
                L = _Layer(c, noise, allq)
                L.two(CX, [(a, q) if want_x else (q, a) for a, q in layer])
                L.close()
        L = _Layer(c, noise, allq)
        L.single(H, xanc)
        L.close()
        L = _Layer(c, noise, allq)
        rec = L.measure(anc)
        L.close(tick=False)
        groups = []
        for (cid, a, ix, sup), m_ in zip(checks, rec):
            if cid in last:
                groups.append([m_, last[cid]])
            elif not ix:
                groups.append([m_])
            last[cid] = m_
        c.detectors(groups)
        c.tick()

    L = _Layer(c, noise, allq)
    L.reset(phys)
    L.close()
    inner = []
    for b in range(lay.n_blocks):
        inner.append((("iz", b), int(lay.inner_z[b]), False, [int(v) for v in lay.phys[b]]))
        inner.append((("ix", b), int(lay.inner_x[b]), True, [int(v) for v in lay.phys[b]]))
    outer = [(("o", i), a, ix, sup) for i, (a, ix, sup, _) in enumerate(lay.outer_checks)]
    touches = [set(lay.block_of[o][0] for o in og) for (_, _, _, og) in lay.outer_checks]
    for t in range(cycles):
        run_checks(inner)
        if t == 0 or t == cycles - 1 or t % gamma == 0:
            active = outer
        else:
            fired = set(np.flatnonzero(rng.random(lay.n_blocks) < fire_rate).tolist())
            active = [oc for oc, tb in zip(outer, touches) if tb & fired]
        run_checks(active)
        if t < cycles - 1:
            c.mark_cycle()
    L = _Layer(c, noise, allq)
    drec = L.measure(phys)
    L.close(tick=False)
    pos = {int(q): i for i, q in enumerate(phys)}
    groups = []
    for b in range(lay.n_blocks):
        groups.append([drec[pos[int(q)]] for q in lay.phys[b]] + [last[("iz", b)]])
    for i, (a, ix, sup, _) in enumerate(lay.outer_checks):
        if not ix:
            groups.append([drec[pos[q]] for q in sup] + [last[("o", i)]])
    c.detectors(groups)
    c.observable(0, [drec[pos[q]] for q in lay.z_logical])
    c.logicals = [np.asarray(lay.z_logical, dtype=np.int64)]
    c.n_cycles = cycles
    return c


def adaptive_branches(n: int = 256, d: int = 10, lo: int = 10, hi: int = 30, seed: int = 4,
                      noise: NoiseModel | None = None) -> list:
    """n realised branches with cycle counts U{lo..hi} (config 4)."""
    lay = ConcatenatedLayout(d)
    r = rng_for(seed, 5)
    lengths = r.integers(lo, hi + 1, size=n)
    nm = noise or NoiseModel.uniform(1e-3)
    return [concatenated_adaptive_branch(d, int(lengths[i]), seed=seed * 100003 + i, noise=nm, layout=lay)
            for i in range(n)]
