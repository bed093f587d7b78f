"""Planted mistakes: the pins catch a wrong oracle (CPU).

Each case copies the oracle's C source with one plausible mistake planted in
it: a transposed operand, a dropped term, a wrong constant, sign or index.
It compiles the copy into the test's temporary directory and runs the pins'
checks against it: brute-force forward tracking, exact rational evaluation
of Eq. pmerge, the channel decompositions, the level table and finite
differences of the gradient.  Every planted mistake must fail at least one
check, and the unmodified oracle must pass them all.  The oracle in the
repository is never modified.
"""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as BF
import oracle
from paper_2604_16613_gb300 import circuits as C
from test_oracle_pins import SMALL, _bell_probe, _loss, oracle_masks

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))

# name -> (text in oracle.c, its replacement); each text occurs exactly once
MUTANTS = {
    # Eq. slp, CX: control and target transposed
    "cx-transposed": ("if (set_xor_inplace(&xs[a], &xs[b], &t1)) goto nomem;\n"
                      "                if (set_xor_inplace(&zs[b], &zs[a], &t1)) goto nomem;",
                      "if (set_xor_inplace(&xs[b], &xs[a], &t1)) goto nomem;\n"
                      "                if (set_xor_inplace(&zs[a], &zs[b], &t1)) goto nomem;"),
    # Eq. slp, H: the swap of the X and Z planes dropped
    "h-dropped": ("case K_H: { idset t = xs[a]; xs[a] = zs[a]; zs[a] = t; break; }", "case K_H: break;"),
    # CZ: X picks up the partner's X plane instead of its Z plane
    "cz-wrong-plane": ("if (set_xor_inplace(&xs[a], &zs[b], &t1)) goto nomem;",
                       "if (set_xor_inplace(&xs[a], &xs[b], &t1)) goto nomem;"),
    # S: the Z plane updated instead of the X plane
    "s-transposed": ("case K_S:  /* X before S is Y after */\n"
                     "                if (set_xor_inplace(&xs[a], &zs[a], &t1)) goto nomem;",
                     "case K_S:  /* X before S is Y after */\n"
                     "                if (set_xor_inplace(&zs[a], &xs[a], &t1)) goto nomem;"),
    # a reset clears the Z plane only
    "reset-keeps-x": ("xs[a].n = 0;\n                    zs[a].n = 0;", "zs[a].n = 0;"),
    # Eq. init-slp: a detector keeps only its first measurement record
    "first-record-only": ("if (set_toggle(&meas_ids[m], id)) goto nomem;",
                          "if (r == 0 && set_toggle(&meas_ids[m], id)) goto nomem;"),
    # every observable collapses onto observable 0
    "observable-index": ("(uint32_t)(n_det + o[3]);", "(uint32_t)(n_det);"),
    # Sec. 2.3.4: a Y component loses its Z part
    "y-without-z": ("static int pauli_z(int p) { return p == 2 || p == 3; }",
                    "static int pauli_z(int p) { return p == 2; }"),
    # Table tab:correlation-level: L1 keeps all fifteen two-qubit components
    "level1-count": ("case K_DEP2: return level == 0 ? 6 : (level == 1 ? 10 : 15);",
                     "case K_DEP2: return level == 0 ? 6 : 15;"),
    # reading C1: wrong DEPOLARIZE1 constant
    "dep1-q-constant": ("case K_DEP1: return 0.5 * (1.0 - sqrt(1.0 - 4.0 * p / 3.0));",
                        "case K_DEP1: return 0.5 * (1.0 - sqrt(1.0 - 2.0 * p / 3.0));"),
    # reading C1: wrong DEPOLARIZE2 root
    "dep2-q-root": ("pow(1.0 - 16.0 * p / 15.0, 0.125)", "pow(1.0 - 16.0 * p / 15.0, 0.25)"),
    # Eq. pmerge: the factor 2 dropped
    "pmerge-factor": ("s += log1p(-2.0 * q);", "s += log1p(-q);"),
    # reading C18: the weight's sign flipped
    "weight-sign": ("d->class_w[cc] = log1p(-P) - log(P);", "d->class_w[cc] = log(P) - log1p(-P);"),
    # the adjoint: wrong exponent in dq/dp of DEPOLARIZE2
    "dep2-dqdp": ("pow(1.0 - 16.0 * p / 15.0, -0.875)", "pow(1.0 - 16.0 * p / 15.0, -0.75)"),
}


def build_copy(tmp_path, name: str, old: str | None, new: str | None):
    src = open(os.path.join(ORACLE_DIR, "oracle.c")).read()
    if old is not None:
        assert src.count(old) == 1, f"{name}: the text to replace must occur once"
        src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    (d / "oracle.c").write_text(src)
    shutil.copy(os.path.join(ORACLE_DIR, "oracle.h"), d / "oracle.h")
    so = d / "liboracle.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(d / "oracle.c"), "-lm"])
    return oracle.load_library(str(so))


# ---- the checks: each returns None when it passes, else what failed --------

def check_masks_small(lib):
    for name, make in SMALL:
        circ = make()
        for level in (0, 1, 2):
            dem = oracle.analyze_circuit(circ, circ.default_noise, level, lib=lib)
            if oracle_masks(dem, circ, level) != BF.mechanism_masks(circ, circ.default_noise, level, seed=level):
                return f"masks of {name} at L{level} differ from brute force"
    return None


def check_random_circuits(lib):
    for seed in range(120):
        circ = C.random_circuit(seed)
        level = seed % 3
        dem = oracle.analyze_circuit(circ, circ.default_noise, level, lib=lib)
        bf = BF.mechanism_masks(circ, circ.default_noise, level, seed=seed)
        if oracle_masks(dem, circ, level) != bf:
            return f"random circuit {seed}: masks differ from brute force"
        ref = BF.dem_from_masks(bf, circ, circ.default_noise)
        got = dem.edges()
        if set(got) != set(ref) or any(abs(got[e][0] - P) > 1e-12 * P for e, P in ref.items()):
            return f"random circuit {seed}: classes or probabilities differ"
    return None


def check_observables(lib):
    # three observables, each on its own qubit, must stay apart: brute force
    # on bit flips read by one observable each
    circ = C.Circuit(3)
    circ.gate1(C.R, range(3)); circ.tick()
    circ.noise(C.X_ERROR, [0, 1, 2], 0.01); circ.tick()
    rec = circ.measure(C.M, range(3))
    circ.observable(0, [rec[0]])
    circ.observable(1, [rec[1]])
    circ.observable(2, [rec[2]])
    dem = oracle.analyze_circuit(circ, circ.default_noise, 2, lib=lib)
    if oracle_masks(dem, circ, 2) != BF.mechanism_masks(circ, circ.default_noise, 2, seed=1):
        return "observable masks differ from brute force"
    return None


def check_probabilities_exact(lib):
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=11)
    dem = oracle.analyze_circuit(circ, noise, lib=lib)
    kinds = circ.ops[dem.mech_op, 0]
    for i in range(dem.n_mechanisms):
        q = BF.component_probability(int(kinds[i]), float(noise[dem.mech_loc[i]]))
        if abs(dem.mech_q[i] - q) > 1e-9 * q:        # the two forms round differently for small p
            return f"mechanism {i}: q differs from the channel decomposition"
    for cl in range(dem.n_classes):
        acc = Fraction(0)
        for i in np.flatnonzero(dem.mech_class == cl):
            acc = BF.boxplus(acc, Fraction(float(dem.mech_q[i])))
        P = float(acc)
        if abs(dem.class_p[cl] - P) > 1e-13 * P:
            return f"class {cl}: P differs from iterated boxplus"
        if abs(dem.class_w[cl] - math.log((1 - P) / P)) > 1e-12 * abs(math.log((1 - P) / P)):
            return f"class {cl}: w differs from log((1 - P) / P)"
    return None


def check_level_counts(lib):
    counts = {level: oracle.analyze_circuit(_bell_probe(), level=level, lib=lib).n_mechanisms for level in (0, 1, 2)}
    return None if counts == {0: 6, 1: 10, 2: 15} else f"component counts per level {counts}"


def check_gradient(lib):
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=2)
    dem = oracle.analyze_circuit(circ, noise, lib=lib)
    edges = sorted(dem.edges())
    rng = np.random.default_rng(8)
    gP = {e: float(x) for e, x in zip(edges, rng.normal(size=len(edges)))}
    gW = {e: float(x) * 1e-3 for e, x in zip(edges, rng.normal(size=len(edges)))}
    order = [dem.split_ids(dem.class_ids(c)) for c in range(dem.n_classes)]
    g = dem.gradient(np.array([gP[e] for e in order]), np.array([gW[e] for e in order]), circ.n_locations)
    h = 1e-7
    for loc in rng.choice(circ.n_locations, size=64, replace=False):
        up, dn = noise.copy(), noise.copy()
        up[loc] += h
        dn[loc] -= h
        fd = (_loss(oracle.analyze_circuit(circ, up, lib=lib), gP, gW) -
              _loss(oracle.analyze_circuit(circ, dn, lib=lib), gP, gW)) / (2 * h)
        if abs(g[loc] - fd) > 2e-5 * abs(fd) + 1e-6 * max(1.0, abs(fd)):
            return f"location {loc}: gradient differs from central differences"
    return None


CHECKS = [check_masks_small, check_level_counts, check_observables, check_probabilities_exact,
          check_random_circuits, check_gradient]


def failures(lib, stop_at_first: bool):
    out = []
    for check in CHECKS:
        try:
            f = check(lib)
        except oracle.OracleError as e:         # e.g. a detector made non-deterministic
            f = f"{check.__name__}: oracle error {e}"
        if f:
            out.append(f)
            if stop_at_first:
                break
    return out


def test_unmodified_copy_passes_every_check(tmp_path):
    assert failures(build_copy(tmp_path, "unmodified", None, None), stop_at_first=False) == []


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    assert failures(build_copy(tmp_path, name, old, new), stop_at_first=True), \
        f"no check caught the planted mistake {name}"
