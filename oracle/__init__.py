"""CPU oracle for the detector error model -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it; see ``oracle.h`` for what it computes and which
passages of the paper it follows.

The C source is compiled on demand with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

LEVELS = {"L0": 0, "L1": 1, "L2": 2, 0: 0, 1: 1, 2: 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain gcc, no tuning flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH) or
             os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str):
    """Load an oracle shared library and declare its entry points (the built
    oracle, or a copy that a test compiled from a modified source)."""
    lib = ctypes.CDLL(path)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    f64p = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    lib.orc_analyze.argtypes = [u32p, ctypes.c_uint64, u32p, ctypes.c_uint64, ctypes.c_uint32,
                                f64p, ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(vp),
                                ctypes.c_char_p, ctypes.c_int]
    lib.orc_analyze.restype = ctypes.c_int
    lib.orc_free.argtypes = [vp]
    for name, rt in [("orc_n_detectors", ctypes.c_uint32), ("orc_n_observables", ctypes.c_uint32),
                     ("orc_n_mechanisms", ctypes.c_uint64), ("orc_n_classes", ctypes.c_uint64)]:
        getattr(lib, name).argtypes = [vp]
        getattr(lib, name).restype = rt
    for name, rt in [("orc_mech_op", u64p), ("orc_mech_comp", u32p), ("orc_mech_loc", u32p),
                     ("orc_mech_q", f64p), ("orc_mech_mask_off", u64p), ("orc_mech_mask", u32p),
                     ("orc_mech_class", u64p), ("orc_class_mask_off", u64p),
                     ("orc_class_mask", u32p), ("orc_class_p", f64p), ("orc_class_p_iter", f64p),
                     ("orc_class_w", f64p), ("orc_class_size", u64p)]:
        getattr(lib, name).argtypes = [vp]
        getattr(lib, name).restype = rt
    lib.orc_gradient.argtypes = [vp, f64p, f64p, f64p]
    lib.orc_gradient.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(msg)
        self.code = code


NONDETERMINISTIC = 2
INVALID = 1


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(int(n),)).astype(dtype, copy=True)


@dataclass
class OracleDem:
    """Oracle output (copied out of the C result)."""
    n_detectors: int
    n_observables: int
    # mechanisms
    mech_op: np.ndarray
    mech_comp: np.ndarray
    mech_loc: np.ndarray
    mech_q: np.ndarray
    mech_mask_off: np.ndarray
    mech_mask: np.ndarray
    mech_class: np.ndarray
    # classes (sorted by flip set)
    class_mask_off: np.ndarray
    class_mask: np.ndarray
    class_p: np.ndarray
    class_p_iter: np.ndarray
    class_w: np.ndarray
    class_size: np.ndarray
    _handle: object = None

    @property
    def n_mechanisms(self) -> int:
        return int(self.mech_op.size)

    @property
    def n_classes(self) -> int:
        return int(self.class_p.size)

    def mech_ids(self, i: int) -> np.ndarray:
        return self.mech_mask[self.mech_mask_off[i]:self.mech_mask_off[i + 1]]

    def class_ids(self, c: int) -> np.ndarray:
        return self.class_mask[self.class_mask_off[c]:self.class_mask_off[c + 1]]

    def split_ids(self, ids: np.ndarray):
        """(detector tuple, observable bitmask) of an id list."""
        D = self.n_detectors
        dets = tuple(int(x) for x in ids if x < D)
        obs = 0
        for x in ids:
            if x >= D:
                obs |= 1 << int(x - D)
        return dets, obs

    def edges(self) -> dict:
        """{(detector tuple, observable mask): (P, w)} for every class."""
        out = {}
        for c in range(self.n_classes):
            out[self.split_ids(self.class_ids(c))] = (float(self.class_p[c]), float(self.class_w[c]))
        return out

    def gradient(self, gP: np.ndarray, gW: np.ndarray, n_locations: int) -> np.ndarray:
        """d/dp of sum_c gP[c] P_c + gW[c] w_c (classes in this object's order)."""
        lib = self._handle.lib
        gP = np.ascontiguousarray(gP, dtype=np.float64)
        gW = np.ascontiguousarray(gW, dtype=np.float64)
        g = np.zeros(max(n_locations, 1), dtype=np.float64)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.orc_gradient(self._handle.value, gP.ctypes.data_as(f64p), gW.ctypes.data_as(f64p),
                         g.ctypes.data_as(f64p))
        return g[:n_locations]


class _Handle:
    def __init__(self, lib, ptr):
        self.lib, self.value = lib, ptr

    def __del__(self):
        try:
            self.lib.orc_free(self.value)
        except Exception:
            pass


def analyze(ops: np.ndarray, recs: np.ndarray, n_qubits: int, noise: np.ndarray,
            level="L2", lib=None) -> OracleDem:
    """Run the oracle on a flat circuit (see circuits.py for the format);
    `lib` selects another loaded copy (default: the built oracle)."""
    lib = lib or _load()
    ops = np.ascontiguousarray(ops, dtype=np.uint32).reshape(-1, 4)
    recs = np.ascontiguousarray(recs, dtype=np.uint32).reshape(-1)
    noise = np.ascontiguousarray(noise, dtype=np.float64).reshape(-1)
    if recs.size == 0:
        recs = np.zeros(1, dtype=np.uint32)
        n_recs = 0
    else:
        n_recs = recs.size
    nz = noise if noise.size else np.zeros(1, dtype=np.float64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    out = ctypes.c_void_p()
    err = ctypes.create_string_buffer(512)
    rc = lib.orc_analyze(ops.ctypes.data_as(u32p), ops.shape[0], recs.ctypes.data_as(u32p), n_recs,
                         int(n_qubits), nz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         int(noise.size), LEVELS[level], ctypes.byref(out), err, 512)
    if rc != 0:
        raise OracleError(rc, err.value.decode())
    h = out.value
    nm = lib.orc_n_mechanisms(h)
    nc = lib.orc_n_classes(h)
    moff = _arr(lib.orc_mech_mask_off(h), nm + 1, np.int64)
    coff = _arr(lib.orc_class_mask_off(h), nc + 1, np.int64)
    dem = OracleDem(
        n_detectors=int(lib.orc_n_detectors(h)), n_observables=int(lib.orc_n_observables(h)),
        mech_op=_arr(lib.orc_mech_op(h), nm, np.int64), mech_comp=_arr(lib.orc_mech_comp(h), nm, np.int64),
        mech_loc=_arr(lib.orc_mech_loc(h), nm, np.int64), mech_q=_arr(lib.orc_mech_q(h), nm, np.float64),
        mech_mask_off=moff, mech_mask=_arr(lib.orc_mech_mask(h), moff[-1], np.int64),
        mech_class=_arr(lib.orc_mech_class(h), nm, np.int64),
        class_mask_off=coff, class_mask=_arr(lib.orc_class_mask(h), coff[-1], np.int64),
        class_p=_arr(lib.orc_class_p(h), nc, np.float64),
        class_p_iter=_arr(lib.orc_class_p_iter(h), nc, np.float64),
        class_w=_arr(lib.orc_class_w(h), nc, np.float64),
        class_size=_arr(lib.orc_class_size(h), nc, np.int64),
    )
    dem._handle = _Handle(lib, h)
    return dem


def analyze_circuit(circuit, noise=None, level="L2", lib=None) -> OracleDem:
    noise = circuit.default_noise if noise is None else noise
    return analyze(circuit.ops, circuit.recs, circuit.n_qubits, noise, level, lib)
