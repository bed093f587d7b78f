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
