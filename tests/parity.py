"""Helpers comparing the GPU library with the CPU oracle."""
import numpy as np

import oracle

# Probability tolerance: |P_gpu - P_oracle| <= 1e-5 P_oracle (FP32 vs FP64).
P_RTOL = 1e-5
# Weight w = log((1-P)/P): dw = dP / (P (1-P)), so a 1e-5 relative error in P
# moves w by at most 1e-5 / (1-P) <= 2e-5, plus FP32 rounding of w itself.
W_ATOL = 2e-5
W_RTOL = 1e-6


def oracle_edges(circuit, noise32, level="L2"):
    """Oracle on the same FP32 noise values the GPU sees (widened to FP64)."""
    noise64 = np.asarray(noise32, dtype=np.float32).astype(np.float64)
    return oracle.analyze_circuit(circuit, noise64, level)


def compare_edges(got: dict, ref: dict, label=""):
    """Masks bit-exact (same key sets), P within P_RTOL, w within W_ATOL."""
    missing = set(ref) - set(got)
    extra = set(got) - set(ref)
    assert not missing and not extra, (
        f"{label}: {len(missing)} oracle hyperedges missing, {len(extra)} unexpected; "
        f"e.g. missing {sorted(missing)[:3]} extra {sorted(extra)[:3]}")
    worst_p = 0.0
    worst_w = 0.0
    for e, (P, w) in ref.items():
        gp, gw = got[e]
        rp = abs(gp - P) / P
        worst_p = max(worst_p, rp)
        dw = abs(gw - w)
        assert rp <= P_RTOL, f"{label}: edge {e}: P {gp!r} vs {P!r} (rel {rp:.3g})"
        assert dw <= W_ATOL + W_RTOL * abs(w), f"{label}: edge {e}: w {gw!r} vs {w!r}"
        worst_w = max(worst_w, dw)
    return worst_p, worst_w


def _canonical_rows(lengths, ids, obs, P, W):
    """Rows (length, sorted ids padded with -1, observable mask) in
    lexicographic order, with P and w permuted alike."""
    n = lengths.size
    width = int(lengths.max()) if n else 0
    mat = np.full((n, width + 2), -1, dtype=np.int64)
    mat[:, 0] = lengths
    if ids.size:
        row = np.repeat(np.arange(n), lengths)
        start = np.repeat(np.cumsum(lengths) - lengths, lengths)
        mat[row, 1 + np.arange(ids.size) - start] = ids
    mat[:, -1] = obs.astype(np.int64)
    order = np.lexsort(mat.T[::-1])
    return mat[order], P[order], W[order]


def compare_arrays(host: dict, circuit: int, ref, label=""):
    """The GPU model of one circuit of a compile (``Dem.to_host()`` arrays)
    against an oracle result, vectorized: the same number of hyperedges, no
    hyperedge twice, every mask identical after canonical sorting, P within
    P_RTOL and w within W_ATOL + W_RTOL |w|.  Returns the worst relative P
    error."""
    lo, hi = int(host["edge_offsets"][circuit]), int(host["edge_offsets"][circuit + 1])
    off = host["det_offsets"].astype(np.int64)
    g_len = off[lo + 1:hi + 1] - off[lo:hi]
    g_ids = host["det_idx"][off[lo]:off[hi]].astype(np.int64)
    g = _canonical_rows(g_len, g_ids, host["obs_mask"][lo:hi].astype(np.uint64),
                        host["prob"][lo:hi].astype(np.float64), host["logodds"][lo:hi].astype(np.float64))
    D = ref.n_detectors
    coff = ref.class_mask_off
    ids = ref.class_mask
    is_det = ids < D
    cls = np.repeat(np.arange(ref.n_classes), np.diff(coff))
    r_len = np.bincount(cls[is_det], minlength=ref.n_classes)
    r_obs = np.zeros(ref.n_classes, dtype=np.uint64)
    if (~is_det).any():
        np.bitwise_or.at(r_obs, cls[~is_det], (np.uint64(1) << (ids[~is_det] - D).astype(np.uint64)))
    r = _canonical_rows(r_len, ids[is_det], r_obs, ref.class_p, ref.class_w)
    assert hi - lo == ref.n_classes, f"{label}: {hi - lo} hyperedges, oracle has {ref.n_classes} classes"
    if g[0].shape[0] > 1:
        dup = np.all(g[0][1:] == g[0][:-1], axis=1)
        assert not dup.any(), f"{label}: {int(dup.sum())} hyperedges appear twice (a class was split)"
    assert g[0].shape == r[0].shape and np.array_equal(g[0], r[0]), f"{label}: hyperedge masks differ"
    rel = np.abs(g[1] - r[1]) / r[1]
    assert rel.max(initial=0.0) <= P_RTOL, f"{label}: worst relative P error {rel.max():.3g}"
    dw = np.abs(g[2] - r[2])
    assert np.all(dw <= W_ATOL + W_RTOL * np.abs(r[2])), f"{label}: log-odds differ by up to {dw.max():.3g}"
    return float(rel.max(initial=0.0))


def oracle_arrays(args):
    """One oracle run as a task of a spawn process pool: args = (ops, recs,
    n_qubits, noise (FP64), level); returns the picklable arrays that
    ``compare_arrays`` reads."""
    from types import SimpleNamespace
    ops, recs, n_qubits, noise64, level = args
    r = oracle.analyze(ops, recs, n_qubits, noise64, level)
    return SimpleNamespace(n_detectors=r.n_detectors, n_classes=r.n_classes, class_mask_off=r.class_mask_off,
                           class_mask=r.class_mask, class_p=r.class_p, class_w=r.class_w)
