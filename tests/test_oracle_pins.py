"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the worked
example of Fig. fig:error-analysis, brute-force forward tracking of every
single error, invariants of repetition and surface codes, exact rational
evaluations of Eq. pmerge and of the channel decompositions, and finite
differences of the gradient.
"""
import itertools
import math
import os
from collections import deque
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as BF
import oracle
from paper_2604_16613_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def oracle_masks(dem, circuit, level):
    """{(row, component name): edge} from the oracle's mechanism list."""
    out = {}
    ops = circuit.ops
    for i in range(dem.n_mechanisms):
        row = int(dem.mech_op[i])
        kind = int(ops[row, 0])
        comp = int(dem.mech_comp[i])
        if kind == C.X_ERROR:
            name = "X"
        elif kind == C.Z_ERROR:
            name = "Z"
        elif kind == C.DEPOLARIZE1:
            name = ["X", "Z", "Y"][comp]
        else:
            name = BF.DEP2_BY_LEVEL[2][comp]
        out[(row, name)] = dem.split_ids(dem.mech_ids(i))
    return out


# --------------------------------------------------------------------------
# (ii) Fig. 1 worked example
# --------------------------------------------------------------------------

def test_fig1_worked_example():
    text = open(os.path.join(GOLDEN, "fig1_bitflip.txt")).read()
    expect = [l for l in text.splitlines() if l.startswith("# EXPECT")][0]
    fields = dict(kv.split("=") for kv in expect.split()[2:])
    want_dets = tuple(int(x) for x in fields["detectors"].split(",") if x)
    circ = C.Circuit.from_text(text)
    dem = oracle.analyze_circuit(circ)
    assert dem.n_detectors == 4
    assert dem.n_mechanisms == 1
    assert dem.split_ids(dem.mech_ids(0)) == (want_dets, 0)
    # the builder's version of the same circuit agrees
    dem2 = oracle.analyze_circuit(C.fig1_bitflip_circuit())
    assert dem2.split_ids(dem2.mech_ids(0)) == (want_dets, 0)
    # merging at the third CNOT layer: the same error one layer later (after
    # CNOT layer 3) is seen by the yellow detector only (data 2 -> ancilla 1
    # is the fourth layer), one layer earlier (before layer 2) it also meets
    # ancilla 1 in round 1.
    assert want_dets == (2, 3)


# --------------------------------------------------------------------------
# (i) brute force: every single error forward-tracked
# --------------------------------------------------------------------------

SMALL = [
    ("rep3", lambda: C.repetition_code_memory(3, 3, C.NoiseModel.uniform(2e-3))),
    ("rep5", lambda: C.repetition_code_memory(5, 4, C.NoiseModel.hardware_inspired(1e-2))),
    ("fig1-noisy", lambda: C.repetition_code_memory(3, 2, C.NoiseModel.uniform(1e-3), final_data=False)),
    ("surf3", lambda: C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))),
    ("surf4", lambda: C.rotated_surface_code_memory(4, 2, C.NoiseModel.hardware_inspired(1e-3))),
]


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
@pytest.mark.parametrize("level", [0, 1, 2])
def test_bruteforce_masks_codes(name, make, level):
    circ = make()
    noise = circ.default_noise
    dem = oracle.analyze_circuit(circ, noise, level)
    bf = BF.mechanism_masks(circ, noise, level, seed=level)
    assert oracle_masks(dem, circ, level) == bf
    # a second gauge draw gives the same flips (deterministic detectors)
    assert BF.mechanism_masks(circ, noise, level, seed=99) == bf


def test_bruteforce_random_circuits():
    n_checked = 0
    for seed in range(520):
        circ = C.random_circuit(seed)
        noise = circ.default_noise
        D, O = BF.noiseless_flips(circ, shots=64, seed=seed)
        assert not D.any() and not O.any(), f"seed {seed}: generator made a random detector"
        level = seed % 3
        dem = oracle.analyze_circuit(circ, noise, level)
        bf = BF.mechanism_masks(circ, noise, level, seed=seed)
        assert oracle_masks(dem, circ, level) == bf, f"seed {seed}"
        # classes and probabilities from the plain definition
        ref = BF.dem_from_masks(bf, circ, noise)
        got = dem.edges()
        assert set(got) == set(ref), f"seed {seed}"
        for e, P in ref.items():
            assert got[e][0] == pytest.approx(P, rel=1e-12, abs=0), f"seed {seed}"
        n_checked += len(bf)
    assert n_checked > 10000


# --------------------------------------------------------------------------
# (iii) invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [3, 5, 7])
def test_noiseless_surface_deterministic_and_counts(d):
    circ = C.rotated_surface_code_memory(d, d, C.NoiseModel.uniform(1e-3))
    assert circ.n_detectors == d * (d * d - 1)
    D, O = BF.noiseless_flips(circ, shots=128, seed=d)
    assert not D.any() and not O.any()
    dem = oracle.analyze_circuit(circ)          # raises if non-deterministic
    assert dem.n_detectors == d * (d * d - 1)
    assert dem.n_observables == 1


def _bulk_sites(circ, lay, rounds):
    """DEPOLARIZE1 idle sites on interior data qubits in the H layers of
    interior rounds (between two complete syndrome rounds)."""
    d = lay.d
    interior = {i for i, (x, y) in enumerate(lay.data_xy.tolist())
                if 1 < x < 2 * d - 1 and 1 < y < 2 * d - 1}
    ops = circ.ops
    tick = 0
    out = []
    layers_per_round = 8
    for i, (k, a, b, c) in enumerate(ops.tolist()):
        if k == C.TICK:
            tick += 1
            continue
        rnd, lay_in_round = divmod(tick, layers_per_round)
        if (k == C.DEPOLARIZE1 and a in interior and 1 <= rnd <= rounds - 2
                and lay_in_round == 1):
            out.append(i)
    return out


@pytest.mark.parametrize("d", [5, 7])
def test_bulk_data_errors_flip_two_detectors(d):
    circ = C.rotated_surface_code_memory(d, d, C.NoiseModel.uniform(1e-3))
    dem = oracle.analyze_circuit(circ)
    masks = oracle_masks(dem, circ, 2)
    rows = _bulk_sites(circ, circ.layout, d)
    assert len(rows) > 0
    for r in rows:
        assert len(masks[(r, "X")][0]) == 2 and masks[(r, "X")][1] == 0
        assert len(masks[(r, "Z")][0]) == 2
        assert len(masks[(r, "Y")][0]) == 4


def test_bulk_repetition_errors_flip_two():
    d, rounds = 7, 6
    circ = C.repetition_code_memory(d, rounds, C.NoiseModel.uniform(1e-3))
    dem = oracle.analyze_circuit(circ)
    masks = oracle_masks(dem, circ, 2)
    # idle DEPOLARIZE1 on interior data during the ancilla-reset layers of
    # interior rounds: X flips the two neighbouring checks, Z flips nothing
    tick, seen = 0, 0
    for i, (k, a, b, c) in enumerate(circ.ops.tolist()):
        if k == C.TICK:
            tick += 1
            continue
        rnd, li = divmod(tick - 1, 4)
        if k == C.DEPOLARIZE1 and a % 2 == 0 and 0 < a < 2 * d - 2 and li == 3 and 1 <= rnd <= rounds - 2:
            assert len(masks[(i, "X")][0]) == 2
            assert (i, "Z") not in masks
            seen += 1
    assert seen > 0


def _bell_probe():
    """Two Bell pairs (a, a') (b, b'), one DEPOLARIZE2 on (a, b), then undo:
    each of X_a, Z_a, X_b, Z_b flips its own measurement, so all fifteen
    components have distinct non-empty flip sets."""
    c = C.Circuit(4)
    c.gate1(C.R, range(4)); c.tick()
    c.gate1(C.H, [0, 2]); c.tick()
    c.gate2(C.CX, [(0, 1), (2, 3)]); c.tick()
    c.noise(C.DEPOLARIZE2, [(0, 2)], 0.01); c.tick()
    c.gate2(C.CX, [(0, 1), (2, 3)]); c.tick()
    c.gate1(C.H, [0, 2]); c.tick()
    rec = c.measure(C.M, range(4))
    c.detectors([[r] for r in rec])
    return c


def test_level_component_counts_and_alpha():
    circ = _bell_probe()
    counts = {}
    for level in (0, 1, 2):
        dem = oracle.analyze_circuit(circ, level=level)
        counts[level] = dem.n_mechanisms
        assert len(set(map(tuple, (dem.mech_ids(i) for i in range(dem.n_mechanisms))))) == dem.n_mechanisms
    assert counts == {0: 6, 1: 10, 2: 15}
    # alpha = ceil(|set| / 2) (Table tab:correlation-level): 3, 5, 8
    assert [math.ceil(counts[l] / 2) for l in (0, 1, 2)] == [3, 5, 8]
    # level 0 keeps only pure X and pure Z products
    dem0 = oracle.analyze_circuit(circ, level=0)
    names = {BF.DEP2_BY_LEVEL[2][int(c)] for c in dem0.mech_comp}
    assert names == set(BF.DEP2_BY_LEVEL[0])
    assert all(("Y" not in n) and not ({"X", "Z"} <= set(n)) for n in names)


def test_linearity_of_masks():
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    dem = oracle.analyze_circuit(circ)
    masks = oracle_masks(dem, circ, 2)

    def ids(row, name):
        e = masks.get((row, name), ((), 0))
        return set(e[0]), e[1]

    def xor(u, v):
        return (u[0] ^ v[0], u[1] ^ v[1])

    checked = 0
    for i, (k, a, b, c) in enumerate(circ.ops.tolist()):
        if k == C.DEPOLARIZE1:
            assert ids(i, "Y") == xor(ids(i, "X"), ids(i, "Z"))
            checked += 1
        elif k == C.DEPOLARIZE2:
            for name in BF.DEP2_BY_LEVEL[2]:
                pa, pb = name
                if pa != "I" and pb != "I":
                    assert ids(i, name) == xor(ids(i, pa + "I"), ids(i, "I" + pb))
            assert ids(i, "YI") == xor(ids(i, "XI"), ids(i, "ZI"))
            assert ids(i, "IY") == xor(ids(i, "IX"), ids(i, "IZ"))
            checked += 1
    assert checked > 100


# --------------------------------------------------------------------------
# (iv)-(vi) probabilities
# --------------------------------------------------------------------------

def test_boxplus_closed_form_exact():
    rng = np.random.default_rng(5)
    for _ in range(200):
        qs = [Fraction(int(rng.integers(1, 500)), int(rng.integers(1001, 5000)))
              for _ in range(int(rng.integers(1, 12)))]
        acc = Fraction(0)
        for q in qs:
            acc = BF.boxplus(acc, q)
        prod = Fraction(1)
        for q in qs:
            prod *= 1 - 2 * q
        assert acc == (1 - prod) / 2


def test_oracle_class_probability_matches_exact_rationals():
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=11)
    dem = oracle.analyze_circuit(circ, noise)
    for cl in range(dem.n_classes):
        members = np.flatnonzero(dem.mech_class == cl)
        acc = Fraction(0)
        for i in members:
            acc = BF.boxplus(acc, Fraction(float(dem.mech_q[i])))
        assert dem.class_p[cl] == pytest.approx(float(acc), rel=1e-13)
        assert dem.class_p_iter[cl] == pytest.approx(float(acc), rel=1e-13)
        P = float(acc)
        assert dem.class_w[cl] == pytest.approx(math.log((1 - P) / P), rel=1e-12)


def _enumerate_channel(q: Fraction, comps):
    """Exact distribution of the product of independent components."""
    dist = {}
    for bits in itertools.product((0, 1), repeat=len(comps)):
        pr = Fraction(1)
        x = z = 0
        for bit, (cx, cz) in zip(bits, comps):
            pr *= q if bit else 1 - q
            if bit:
                x ^= cx
                z ^= cz
        dist[(x, z)] = dist.get((x, z), Fraction(0)) + pr
    return dist


def test_channel_decomposition_exact():
    # one qubit: X, Z, Y as (x, z) bit patterns
    q = Fraction(1, 37)
    p1 = 1 - (1 + 3 * (1 - 2 * q) ** 2) / 4
    dist = _enumerate_channel(q, [(1, 0), (0, 1), (1, 1)])
    assert dist[(0, 0)] == 1 - p1
    for key in [(1, 0), (0, 1), (1, 1)]:
        assert dist[key] == p1 / 3
    # two qubits: 15 components as 4-bit patterns (xa, za, xb, zb)
    comps = [v for v in itertools.product((0, 1), repeat=4) if any(v)]
    q2 = Fraction(1, 53)
    p2 = Fraction(15, 16) * (1 - (1 - 2 * q2) ** 8)
    dist2 = {}
    for bits in itertools.product((0, 1), repeat=15):
        pr = Fraction(1)
        acc = (0, 0, 0, 0)
        for bit, v in zip(bits, comps):
            if bit:
                pr *= q2
                acc = tuple(a ^ b for a, b in zip(acc, v))
            else:
                pr *= 1 - q2
        dist2[acc] = dist2.get(acc, Fraction(0)) + pr
    assert dist2[(0, 0, 0, 0)] == 1 - p2
    for v in comps:
        assert dist2[v] == p2 / 15
    # the oracle inverts the same relation: q from p
    circ = _bell_probe()
    for p, qq in ((float(p2), float(q2)),):
        noise = np.array([p])
        dem = oracle.analyze_circuit(circ, noise, level=2)
        assert np.allclose(dem.mech_q, qq, rtol=1e-12, atol=0)
        # (vi) singleton classes: P = q
        assert dem.n_classes == 15
        assert np.allclose(dem.class_p, qq, rtol=1e-13, atol=0)


def test_depolarize1_q_single_qubit():
    c = C.Circuit(2)
    c.gate1(C.R, [0, 1]); c.tick()
    c.gate1(C.H, [0]); c.tick()
    c.gate2(C.CX, [(0, 1)]); c.tick()
    q = Fraction(1, 29)
    p1 = 1 - (1 + 3 * (1 - 2 * q) ** 2) / 4
    c.noise(C.DEPOLARIZE1, [0], float(p1)); c.tick()
    c.gate2(C.CX, [(0, 1)]); c.tick()
    c.gate1(C.H, [0]); c.tick()
    rec = c.measure(C.M, [0, 1])
    c.detectors([[r] for r in rec])
    dem = oracle.analyze_circuit(c)
    assert dem.n_mechanisms == 3 and dem.n_classes == 3
    assert np.allclose(dem.mech_q, float(q), rtol=1e-13)
    dem0 = oracle.analyze_circuit(c, level=0)
    assert dem0.n_mechanisms == 2        # Y dropped at level 0


# --------------------------------------------------------------------------
# (vii) gradient
# --------------------------------------------------------------------------

def _loss(dem, gP, gW):
    return sum(gP[e] * P + gW[e] * w for e, (P, w) in dem.edges().items())


def test_gradient_exact_rational_xerror_circuit():
    # X_ERROR only: q = p, so P and w are rational in p and the gradient is
    # available in exact arithmetic.
    c = C.repetition_code_memory(3, 2, None)
    # add independent X_ERROR sites on data and ancillas between layers
    circ = C.Circuit(c.n_qubits)
    rng = np.random.default_rng(3)
    for k, a, b, cc in c.ops.tolist():
        if k == C.TICK:
            for q in range(c.n_qubits):
                if rng.random() < 0.6:
                    circ.noise(C.X_ERROR, [q], float(rng.uniform(1e-3, 2e-2)))
            circ.tick()
        elif k in C.MEASURE_KINDS:
            circ.measure(k, [a])
        elif k in C.TWO_QUBIT_GATES:
            circ.gate2(k, [(a, b)])
        elif k == C.DETECTOR:
            circ._rec_block(C.DETECTOR, [[circ.n_measurements - int(x) for x in c.recs[a:a + b]]])
            circ.n_detectors += 1
        elif k == C.OBSERVABLE_INCLUDE:
            circ.observable(cc, [circ.n_measurements - int(x) for x in c.recs[a:a + b]])
        else:
            circ.gate1(k, [a])
    noise = circ.default_noise
    dem = oracle.analyze_circuit(circ, noise)
    edges = list(dem.edges())
    rng = np.random.default_rng(4)
    gPv = rng.normal(size=len(edges))
    gWv = rng.normal(size=len(edges))
    g = dem.gradient(gPv, gWv, circ.n_locations)
    # exact: classes from the oracle's masks, members' p as Fractions
    exact = [Fraction(0)] * circ.n_locations
    for cl in range(dem.n_classes):
        members = np.flatnonzero(dem.mech_class == cl)
        ps = [Fraction(float(noise[dem.mech_loc[i]])) for i in members]
        prod = Fraction(1)
        for p in ps:
            prod *= 1 - 2 * p
        P = (1 - prod) / 2
        gbar = Fraction(float(gPv[cl])) - Fraction(float(gWv[cl])) / (P * (1 - P))
        for j, i in enumerate(members):
            others = Fraction(1)
            for k2, p in enumerate(ps):
                if k2 != j:
                    others *= 1 - 2 * p
            exact[int(dem.mech_loc[i])] += gbar * others
    assert np.allclose(g, [float(x) for x in exact], rtol=1e-11, atol=1e-13)


def test_gradient_central_differences():
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=2)
    dem = oracle.analyze_circuit(circ, noise)
    edges = sorted(dem.edges())
    rng = np.random.default_rng(8)
    gP = {e: float(x) for e, x in zip(edges, rng.normal(size=len(edges)))}
    gW = {e: float(x) * 1e-3 for e, x in zip(edges, rng.normal(size=len(edges)))}
    order = [dem.split_ids(dem.class_ids(c)) for c in range(dem.n_classes)]
    g = dem.gradient(np.array([gP[e] for e in order]), np.array([gW[e] for e in order]),
                     circ.n_locations)
    h = 1e-7
    locs = rng.choice(circ.n_locations, size=64, replace=False)
    for loc in locs:
        up, dn = noise.copy(), noise.copy()
        up[loc] += h
        dn[loc] -= h
        fd = (_loss(oracle.analyze_circuit(circ, up), gP, gW) -
              _loss(oracle.analyze_circuit(circ, dn), gP, gW)) / (2 * h)
        assert g[loc] == pytest.approx(fd, rel=2e-5, abs=1e-6 * max(1.0, abs(fd)))


# --------------------------------------------------------------------------
# non-determinism and malformed input
# --------------------------------------------------------------------------

def test_nondeterministic_detector_rejected():
    c = C.Circuit(1)
    c.gate1(C.RX, [0]); c.tick()
    rec = c.measure(C.M, [0])
    c.detector([rec[0]])
    D, _ = BF.noiseless_flips(c, shots=64)
    assert D.any()
    with pytest.raises(oracle.OracleError) as e:
        oracle.analyze_circuit(c, np.zeros(0))
    assert e.value.code == oracle.NONDETERMINISTIC


def test_invalid_inputs_rejected():
    c = C.Circuit(2)
    c.gate1(C.R, [0, 1])
    ops = c.ops.copy()
    ops[0, 1] = 7                       # qubit out of range
    with pytest.raises(oracle.OracleError) as e:
        oracle.analyze(ops, c.recs, 2, np.zeros(0))
    assert e.value.code == oracle.INVALID
    ops = np.array([[C.DETECTOR, 0, 1, 0]], dtype=np.uint32)
    with pytest.raises(oracle.OracleError):
        oracle.analyze(ops, np.array([1], np.uint32), 1, np.zeros(0))
    c2 = C.Circuit(1)
    c2.gate1(C.R, [0])
    c2.noise(C.DEPOLARIZE1, [0], 0.9)   # above 3/4
    with pytest.raises(oracle.OracleError):
        oracle.analyze_circuit(c2)


# --------------------------------------------------------------------------
# circuit distance of the generated surface code (graph-like L0 classes)
# --------------------------------------------------------------------------

def _graphlike_distance(dem):
    D = dem.n_detectors
    B = D                      # boundary node
    adj = [[] for _ in range(D + 1)]
    for cl in range(dem.n_classes):
        dets, obs = dem.split_ids(dem.class_ids(cl))
        if len(dets) == 1:
            u, v = dets[0], B
        elif len(dets) == 2:
            u, v = dets
        else:
            continue
        adj[u].append((v, obs & 1))
        adj[v].append((u, obs & 1))
    dist = {(B, 0): 0}
    dq = deque([(B, 0)])
    while dq:
        node, par = dq.popleft()
        for nb, o in adj[node]:
            st = (nb, par ^ o)
            if st not in dist:
                dist[st] = dist[(node, par)] + 1
                dq.append(st)
    return dist.get((B, 1))


@pytest.mark.parametrize("d", [3, 5])
def test_surface_circuit_distance(d):
    circ = C.rotated_surface_code_memory(d, d, C.NoiseModel.uniform(1e-3))
    dem = oracle.analyze_circuit(circ, level=0)
    assert _graphlike_distance(dem) == d


@pytest.mark.parametrize("d", [3, 5])
def test_z_only_detectors_equal_restricted_full_model(d):
    """Dropping the X-check detectors of a Z-basis memory experiment (the
    configurable-correlation-level section pairs level L0 with such a
    detector set) must give the full model restricted to the Z-check
    detectors: each class's mask loses
    its X detectors, classes whose restricted masks coincide merge with
    P = 1/2 (1 - prod (1 - 2 P_c)) (Eq. pmerge), and classes left with an
    empty mask disappear.  Built here from the full model, independently of
    the oracle's own grouping."""
    noise = C.NoiseModel.uniform(1e-3)
    full = C.rotated_surface_code_memory(d, d, noise)
    zonly = C.rotated_surface_code_memory(d, d, noise, z_detectors_only=True)
    n_z = (d * d - 1) // 2
    n_x = n_z
    assert zonly.n_detectors == n_z * (d + 1)
    assert full.n_detectors == d * (d * d - 1)
    # detector numbering: round 1 has Z checks only; later rounds list the X
    # checks, then the Z checks; the final data measurement closes Z checks
    remap, k, z = {}, 0, 0
    blocks = [(0, n_z)] + [(n_x, n_z)] * (d - 1) + [(0, n_z)]
    for nx, nz in blocks:
        k += nx
        for _ in range(nz):
            remap[k] = z
            k += 1
            z += 1
    assert k == full.n_detectors and z == zonly.n_detectors
    expected: dict = {}
    for (dets, obs), (p, _) in oracle.analyze_circuit(full).edges().items():
        key = (tuple(remap[x] for x in dets if x in remap), obs)
        if not key[0] and not key[1]:
            continue
        expected[key] = expected.get(key, 1.0) * (1.0 - 2.0 * p)
    expected = {k: 0.5 * (1.0 - v) for k, v in expected.items()}
    got = {k: p for k, (p, _) in oracle.analyze_circuit(zonly).edges().items()}
    assert set(got) == set(expected)
    for k, p in expected.items():
        assert got[k] == pytest.approx(p, rel=1e-12), k
