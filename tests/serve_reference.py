"""Windowed serving semantics, restated on the oracle (test infrastructure).

A patch streams its circuit one cycle at a time.  A step takes the patch's
pending cycles t_a..t_b and compiles one window circuit made of cycles
c0..t_b, c0 = max(0, t_a - 3H):

* when c0 > 0, cycles c0 .. c0 + H - 1 only supply measurement records (a
  detector looks back at most H cycles for its records): their detectors
  are emptied, so no column starts there, and in the final window their
  noise is zeroed as well (their mechanisms, cut off from their detectors,
  must not reach the observable-only classes the final request takes);
* unless t_b is the final cycle, a TICK, one Z measurement per qubit of the
  declared logicals and one OBSERVABLE_INCLUDE per logical close the window
  (the observable frame seeded at the cycle boundary);
* a class is sealed for request t when its smallest detector lies in cycle
  t - H; the final request also takes every later class and the classes
  without detectors.

H bounds how many cycles back a detector's sensitivity reaches: no mechanism
of cycle c may flip a detector after cycle c + H.  The mechanisms of the
records-only cycles are checked against that bound in every window but the
final one (where their noise is zero); their allowed detectors all lie inside
the window, so a violation there is seen (the horizon error).

Nothing here is shared with the CUDA server: it is the same rule set written
on top of the oracle, so a test can compare the two.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2604_16613_gb300 import circuits as C


class HorizonError(RuntimeError):
    pass


def window(blocks, c0: int, c1: int, n_rec: int, logicals, final: bool):
    """Flat window circuit over cycles c0..c1 whose first n_rec cycles only
    supply records, and the window-local detector offset of every cycle
    (len c1 - c0 + 2)."""
    ops_l, recs_l, noise_l = [], [], []
    rc = lc = 0
    det_off = [0]
    for k in range(c0, c1 + 1):
        b = blocks[k]
        o = b["ops"].copy()
        kinds = o[:, 0]
        ann = (kinds == C.DETECTOR) | (kinds == C.OBSERVABLE_INCLUDE)
        o[ann, 1] += np.uint32(rc)
        nz = np.isin(kinds, C.NOISE_KINDS)
        o[nz, 3] += np.uint32(lc)
        nzv = b["noise"]
        if k < c0 + n_rec:
            o[kinds == C.DETECTOR, 2] = 0
            if final:
                nzv = np.zeros_like(nzv)
        ops_l.append(o)
        recs_l.append(b["recs"])
        noise_l.append(nzv)
        rc += b["recs"].size
        lc += b["n_locations"]
        det_off.append(det_off[-1] + b["n_detectors"])
    if not final:
        qs = sorted(set(int(q) for lg in logicals for q in lg))
        idx = {q: i for i, q in enumerate(qs)}
        extra = [[C.TICK, 0, 0, 0]] + [[C.M, q, 0, 0] for q in qs]
        ex_recs = []
        for k, lg in enumerate(logicals):
            extra.append([C.OBSERVABLE_INCLUDE, rc + len(ex_recs), len(lg), k])
            ex_recs += [len(qs) - idx[int(q)] for q in lg]
        ops_l.append(np.asarray(extra, dtype=np.uint32))
        recs_l.append(np.asarray(ex_recs, dtype=np.uint32))
    ops = np.concatenate(ops_l)
    recs = np.concatenate(recs_l) if recs_l else np.zeros(0, np.uint32)
    noise = np.concatenate(noise_l)
    return ops, recs, noise, det_off


def serve(circ, H: int, K: int = 1, level: str = "L2"):
    """Stream ``circ`` in steps of up to K cycles; return {(global dets, obs): P}
    over every sealed class and the per-request class counts."""
    blocks = circ.cycle_blocks()
    n = len(blocks)
    det_base = np.concatenate([[0], np.cumsum([b["n_detectors"] for b in blocks])])
    out, per_request = {}, [0] * n
    t_a = 0
    while t_a < n:
        t_b = min(n - 1, t_a + K - 1)
        final = t_b == n - 1
        c0 = max(0, t_a - 3 * H)
        n_rec = H if c0 > 0 else 0
        ops, recs, noise, det_off = window(blocks, c0, t_b, n_rec, circ.logicals, final)
        dem = oracle.analyze(ops, recs, circ.n_qubits, noise, level)
        loc_end = np.cumsum([blocks[k]["n_locations"] for k in range(c0, c0 + n_rec)])
        if n_rec and not final:
            rec = np.flatnonzero(dem.mech_loc < loc_end[-1])
            for m in rec:
                ids = dem.mech_ids(m)
                dets = ids[ids < dem.n_detectors]
                j = int(np.searchsorted(loc_end, dem.mech_loc[m], side="right"))   # its cycle is c0 + j
                if dets.size and dets.max() >= det_off[j + H + 1]:
                    raise HorizonError(f"a mechanism of cycle {c0 + j} flips a detector more than H cycles later")
        D = dem.n_detectors
        for c in range(dem.n_classes):
            ids = dem.class_ids(c)
            dets, obs = dem.split_ids(ids)
            if dets:
                cyc = c0 + int(np.searchsorted(det_off, dets[0], side="right")) - 1
                owner = cyc + H                     # the request that seals it
                if owner < t_a:
                    continue                        # sealed by an earlier step
                if owner > t_b:
                    if not final:
                        continue                    # not sealed yet
                    owner = t_b
            else:
                if not final:
                    continue
                owner = t_b
            key = (tuple(int(det_base[c0] + d) for d in dets), obs)
            assert key not in out, key
            out[key] = float(dem.class_p[c])
            per_request[owner] += 1
            assert D == det_off[-1]
        t_a = t_b + 1
    return out, per_request
