"""Plain-text detector error model.

The line format of `.dem` files, written and read here so that compiled
models can feed external decoders (the output of the compile is the
hypergraph of the DEM section):

    error(0.00123) D4 D17 L0      one hyperedge: probability, detectors,
                                  observables
    detector D15599               declares a detector (optional coordinates
                                  in parentheses are ignored when reading)
    logical_observable L0         declares an observable

Reading also accepts `^` between groups of targets (a suggested
decomposition: the error flips the symmetric difference of the groups),
merges repeated mechanisms with P = p1 + p2 - 2 p1 p2 (independent errors,
Eq. pmerge) and rejects the block instructions (`repeat`,
`shift_detectors`) rather than misread them.
"""
from __future__ import annotations

import re

_NUM = re.compile(r"^[DL](\d+)$")


def write_dem(edges: dict, n_detectors: int, n_observables: int) -> str:
    """Text of a model given as {(detector tuple, observable mask): (P, w)}
    (what ``Dem.edges`` and the oracle's ``edges`` return).  Hyperedges are
    written in sorted key order; probabilities with ``repr`` (round-trips
    exactly); every detector and observable index up to the counts given is
    declared, so unused ones still count."""
    lines = []
    for (dets, obs), val in sorted(edges.items()):
        p = val[0] if isinstance(val, tuple) else val
        targets = [f"D{int(d)}" for d in dets] + [f"L{k}" for k in range(64) if (int(obs) >> k) & 1]
        lines.append(f"error({float(p)!r}) " + " ".join(targets))
    if n_detectors:
        lines.append(f"detector D{n_detectors - 1}")
    for k in range(n_observables):
        lines.append(f"logical_observable L{k}")
    return "\n".join(lines) + "\n"


def read_dem(text: str) -> tuple[dict, int, int]:
    """({(sorted detector tuple, observable mask): P}, n_detectors,
    n_observables) from model text."""
    edges: dict = {}
    n_det = n_obs = 0
    for lineno, raw in enumerate(text.splitlines(), 1):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        head, _, rest = line.partition(" ")
        name = head.split("(", 1)[0]
        if name == "error":
            m = re.match(r"^error\(\s*([^)]+)\)\s*(.*)$", line)
            if not m:
                raise ValueError(f"line {lineno}: malformed error instruction")
            p = float(m.group(1))
            if not 0.0 <= p <= 1.0:
                raise ValueError(f"line {lineno}: probability {p} outside [0, 1]")
            dets: set = set()
            obs = 0
            for tok in m.group(2).split():
                if tok == "^":
                    continue
                num = _NUM.match(tok)
                if not num:
                    raise ValueError(f"line {lineno}: unknown target {tok!r}")
                i = int(num.group(1))
                if tok[0] == "D":
                    dets ^= {i}
                    n_det = max(n_det, i + 1)
                else:
                    obs ^= 1 << i
                    n_obs = max(n_obs, i + 1)
            key = (tuple(sorted(dets)), obs)
            if not key[0] and not key[1]:
                continue
            q = edges.get(key, 0.0)
            edges[key] = q + p - 2.0 * q * p
        elif name in ("detector", "logical_observable"):
            for tok in re.sub(r"\([^)]*\)", " ", line).split()[1:]:
                num = _NUM.match(tok)
                if not num:
                    raise ValueError(f"line {lineno}: unknown target {tok!r}")
                if tok[0] == "D":
                    n_det = max(n_det, int(num.group(1)) + 1)
                else:
                    n_obs = max(n_obs, int(num.group(1)) + 1)
        else:
            raise ValueError(f"line {lineno}: unsupported instruction {name!r}")
    return edges, n_det, n_obs
