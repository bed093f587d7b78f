"""gp_pmerge_noalloc: class probabilities without any device allocation.

Callers such as a decoder host in a real-time loop with a fixed memory budget
cannot call cudaMalloc.  This entry point keeps its scratch in a built-in
device array instead; here it is checked through the C ABI against the
probabilities and weights gp_compile produces for the same classes, on two
calls in a row (the second call reuses the array the first one left behind).
The file is named to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_16613_gb300 import circuits as C
from paper_2604_16613_gb300 import native
from paper_2604_16613_gb300.dem import DeviceCircuit, Driver

from parity import P_RTOL, W_ATOL, W_RTOL

pytestmark = pytest.mark.gpu

_NCOMP = {C.X_ERROR: (1, 1, 1), C.Z_ERROR: (1, 1, 1), C.DEPOLARIZE1: (2, 3, 3), C.DEPOLARIZE2: (6, 10, 15)}


def component_q(kind, p):
    """Component probability of each independent Pauli term of a channel."""
    if kind in (C.X_ERROR, C.Z_ERROR):
        return p
    if kind == C.DEPOLARIZE1:
        return 0.5 * (1.0 - math.sqrt(1.0 - 4.0 * p / 3.0))
    return 0.5 * (1.0 - (1.0 - 16.0 * p / 15.0) ** 0.125)


def mechanism_q(circ, noise, level):
    """q of every mechanism, numbered as gpdem.h documents: noise rows in row
    order, their components in table order, at the given level."""
    out = []
    for kind, a, b, loc in circ.ops.tolist():
        if kind in _NCOMP:
            out += [component_q(kind, float(noise[loc]))] * _NCOMP[kind][level]
    return np.array(out, dtype=np.float64)


def test_noalloc_matches_compile_on_two_calls():
    lib = native.load()
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=12).astype(np.float32)
    drv = Driver.for_circuits([circ])
    dem = drv.compile(DeviceCircuit(circ), torch.tensor(noise, device="cuda"), "L2")
    n_mech, n_edges = dem.n_mechanisms, dem.n_edges
    mech_class = dem.mech_class.clone()
    ref_p = dem.prob.cpu().numpy().astype(np.float64)
    ref_w = dem.logodds.cpu().numpy().astype(np.float64)
    q = mechanism_q(circ, noise.astype(np.float64), 2)
    assert q.size == n_mech
    q_dev = torch.tensor(q, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        prob = torch.full((n_edges,), float("nan"), dtype=torch.float32, device="cuda")
        logodds = torch.full((n_edges,), float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.gp_pmerge_noalloc(ctypes.c_void_p(mech_class.data_ptr()), ctypes.c_void_p(q_dev.data_ptr()),
                                   n_mech, n_edges, ctypes.c_void_p(prob.data_ptr()),
                                   ctypes.c_void_p(logodds.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == native.GP_OK, lib.gp_last_error()
        torch.cuda.synchronize()
        p = prob.cpu().numpy().astype(np.float64)
        w = logodds.cpu().numpy().astype(np.float64)
        rel = np.abs(p - ref_p) / ref_p
        assert rel.max() <= P_RTOL, f"call {call}: worst relative P error {rel.max():.3g}"
        assert np.all(np.abs(w - ref_w) <= W_ATOL + W_RTOL * np.abs(ref_w)), f"call {call}: log-odds differ"


def test_noalloc_rejects_too_many_classes():
    lib = native.load()
    rc = lib.gp_pmerge_noalloc(None, None, 0, (1 << 19) + 1, None, None, None)
    assert rc == native.GP_ERR_CAPACITY
    assert b"524288" in lib.gp_last_error()


def test_noalloc_edge_cases_closed_form():
    """Documented edge behaviour on a hand-built case, against the closed
    form P = (1 - prod(1 - 2 q)) / 2 in FP64: class ids -1 and n_classes are
    skipped, q = 0 contributes nothing, q >= 1/2 saturates the class at 1/2,
    a class without a positive member gets P = 0, and logodds may be NULL."""
    lib = native.load()
    n_classes = 5
    mech_class = np.array([0, 0, 1, -1, 5, 2, 2, 3, 1, 0], dtype=np.int32)
    q = np.array([1e-3, 2e-2, 0.0, 0.3, 0.4, 0.5, 1e-4, 0.0, 3e-4, 0.7], dtype=np.float32)
    q[9] = 0.25          # keep class 0 below saturation; class 2 holds q = 1/2
    expect = np.zeros(n_classes)
    for c in range(n_classes):
        qs = q[mech_class == c].astype(np.float64)
        expect[c] = 0.5 * (1.0 - np.prod(1.0 - 2.0 * np.minimum(qs, 0.5)))
    sat = torch.tensor([0.7], dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    mc = torch.tensor(mech_class, device="cuda")
    qd = torch.tensor(q, device="cuda")
    for call in range(2):
        prob = torch.full((n_classes,), float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.gp_pmerge_noalloc(ctypes.c_void_p(mc.data_ptr()), ctypes.c_void_p(qd.data_ptr()), mech_class.size,
                                   n_classes, ctypes.c_void_p(prob.data_ptr()), None,
                                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == native.GP_OK, lib.gp_last_error()
        torch.cuda.synchronize()
        p = prob.cpu().numpy().astype(np.float64)
        assert p[3] == 0.0 and p[4] == 0.0                     # no positive member, or no member at all
        assert p[2] == pytest.approx(0.5, abs=1e-7)            # q = 1/2 saturates
        for c in (0, 1):
            assert abs(p[c] - expect[c]) <= P_RTOL * expect[c], (call, c, p[c], expect[c])
    # a lone member with q above 1/2 also saturates at 1/2, with log-odds 0
    one = torch.zeros(1, dtype=torch.int32, device="cuda")
    prob = torch.empty(1, dtype=torch.float32, device="cuda")
    lo = torch.empty(1, dtype=torch.float32, device="cuda")
    rc = lib.gp_pmerge_noalloc(ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(sat.data_ptr()), 1, 1,
                               ctypes.c_void_p(prob.data_ptr()), ctypes.c_void_p(lo.data_ptr()),
                               ctypes.c_void_p(stream.cuda_stream))
    assert rc == native.GP_OK, lib.gp_last_error()
    torch.cuda.synchronize()
    assert prob.item() == pytest.approx(0.5, abs=1e-7) and abs(lo.item()) < 1e-6
