"""Python driver over the C ABI (mirrors the buffer-reuse API of Sec. 3.4).

    drv = Driver.for_circuits([max_circuit])        # buffers sized once
    dem = drv.compile(circuit, noise)               # host inputs
    dem = drv.compile(dev_circuit, noise_cuda)      # inputs already on the GPU
    edges = dem.edges()                             # {(dets, obs): (P, w)}

PyTorch supplies the device workspace, the stream and the autograd plumbing;
every step of the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import circuits as C
from . import native

_COMPONENTS_L2 = {C.X_ERROR: 1, C.Z_ERROR: 1, C.DEPOLARIZE1: 3, C.DEPOLARIZE2: 15}


def circuit_sizes(c: C.Circuit) -> dict:
    """Counts a driver must be able to hold for circuit c."""
    ops = c.ops
    kinds = ops[:, 0]
    mech = 0
    for k, n in _COMPONENTS_L2.items():
        mech += n * int((kinds == k).sum())
    return dict(ops=int(ops.shape[0]), recs=int(c.recs.size), qubits=c.n_qubits,
                layers=int((kinds == C.TICK).sum()) + 1,
                measurements=int(np.isin(kinds, C.MEASURE_KINDS).sum()),
                detectors=int((kinds == C.DETECTOR).sum()), locations=c.n_locations, mechanisms=mech)


@dataclass
class Bounds:
    max_circuits: int = 1
    max_qubits: int = 64
    max_ops: int = 1 << 16
    max_recs: int = 1 << 16
    max_layers: int = 1 << 12
    max_measurements: int = 1 << 14
    max_detectors: int = 1 << 14
    max_locations: int = 1 << 16
    max_mechanisms: int = 1 << 18
    max_mask_words: int = 16
    max_det_entries: int = 0

    def to_c(self) -> native.GpBounds:
        return native.GpBounds(**{k: int(getattr(self, k)) for k in self.__dataclass_fields__})

    @staticmethod
    def for_circuits(circuits, batch: int | None = None, slack: float = 1.0) -> "Bounds":
        """Bounds that fit a batch of ``batch`` circuits no larger than the
        largest of ``circuits`` (the "max circuit" of Sec. 3.4)."""
        circuits = list(circuits)
        sz = [circuit_sizes(c) for c in circuits]
        B = batch if batch is not None else len(circuits)
        if batch is None:
            tot = {k: sum(s[k] for s in sz) for k in sz[0]}
        else:
            tot = {k: max(s[k] for s in sz) * batch for k in sz[0]}

        def up(x):
            return int(max(16, x * slack + 16))
        return Bounds(max_circuits=B, max_qubits=max(s["qubits"] for s in sz), max_ops=up(tot["ops"]),
                      max_recs=up(tot["recs"]), max_layers=up(tot["layers"]),
                      max_measurements=up(tot["measurements"]), max_detectors=up(tot["detectors"]),
                      max_locations=up(tot["locations"]), max_mechanisms=up(tot["mechanisms"]))


class DeviceCircuit:
    """A circuit whose rows live in device memory (int32 tensors)."""

    def __init__(self, c: C.Circuit, device="cuda"):
        self.ops = torch.from_numpy(c.ops.astype(np.int32).reshape(-1, 4)).to(device)
        recs = c.recs if c.recs.size else np.zeros(1, np.uint32)
        self.recs = torch.from_numpy(recs.astype(np.int32)).to(device)
        self.n_ops = c.n_ops
        self.n_recs = int(c.recs.size)
        self.n_qubits = c.n_qubits
        self.n_detectors = c.n_detectors
        self.n_observables = c.n_observables
        self.n_locations = c.n_locations
        self.host = c

    def to_c(self) -> native.GpCircuit:
        return native.GpCircuit(self.ops.data_ptr(), self.n_ops, self.recs.data_ptr(), self.n_recs,
                                self.n_qubits, self.n_detectors, self.n_observables, self.n_locations)


def _host_c(c: C.Circuit, keep: list) -> native.GpCircuit:
    ops = np.ascontiguousarray(c.ops, dtype=np.uint32)
    recs = np.ascontiguousarray(c.recs if c.recs.size else np.zeros(1, np.uint32), dtype=np.uint32)
    keep += [ops, recs]
    return native.GpCircuit(ops.ctypes.data, c.n_ops, recs.ctypes.data, int(c.recs.size),
                            c.n_qubits, c.n_detectors, c.n_observables, c.n_locations)


class _CudaArray:
    """Zero-copy handle for torch.as_tensor (driver-owned device memory)."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr) if ptr else 0, False), "version": 3}
        self._owner = owner


def _view(ptr, n, dtype, owner) -> torch.Tensor:
    typestr = {torch.int32: "<i4", torch.float32: "<f4", torch.int64: "<i8"}[dtype]
    if n == 0:
        return torch.zeros(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, (n,), typestr, owner), device="cuda")


class Dem:
    """Result of one compile.  Tensors alias driver memory and stay valid
    until the driver compiles again (use ``clone()`` to keep them)."""

    def __init__(self, driver: "Driver", view: native.GpDemView):
        self.driver = driver
        self.generation = driver.generation
        self.n_circuits = view.n_circuits
        self.n_edges = view.n_edges
        self.n_det_entries = view.n_det_entries
        self.n_mechanisms = view.n_mechanisms
        self.edge_offsets = np.array([view.edge_offsets[i] for i in range(view.n_circuits + 1)], np.int64)
        # device pointers; the tensors over them are made on first access
        self._ptr = {"det_offsets": (view.det_offsets, self.n_edges + 1, torch.int32),
                     "det_idx": (view.det_idx, self.n_det_entries, torch.int32),
                     "obs_mask": (view.obs_mask, self.n_edges, torch.int64),
                     "prob": (view.prob, self.n_edges, torch.float32),
                     "logodds": (view.logodds, self.n_edges, torch.float32),
                     "edge_circuit": (view.edge_circuit, self.n_edges, torch.int32),
                     "mech_class": (view.mech_class, self.n_mechanisms, torch.int32)}
        self._tensors: dict = {}

    def _tensor(self, name: str) -> torch.Tensor:
        t = self._tensors.get(name)
        if t is None:
            ptr, n, dtype = self._ptr[name]
            t = self._tensors[name] = _view(ptr, n, dtype, self.driver)
        return t

    det_offsets = property(lambda self: self._tensor("det_offsets"))
    det_idx = property(lambda self: self._tensor("det_idx"))
    obs_mask = property(lambda self: self._tensor("obs_mask"))
    prob = property(lambda self: self._tensor("prob"))
    logodds = property(lambda self: self._tensor("logodds"))
    edge_circuit = property(lambda self: self._tensor("edge_circuit"))
    mech_class = property(lambda self: self._tensor("mech_class"))

    def _check(self):
        if self.driver.generation != self.generation:
            raise RuntimeError("this result was overwritten by a later compile on the same driver")

    def to_host(self) -> dict:
        self._check()
        return dict(det_offsets=self.det_offsets.cpu().numpy().astype(np.int64),
                    det_idx=self.det_idx.cpu().numpy().astype(np.int64),
                    obs_mask=self.obs_mask.cpu().numpy().view(np.uint64),
                    prob=self.prob.cpu().numpy(), logodds=self.logodds.cpu().numpy(),
                    edge_offsets=self.edge_offsets.copy())

    def copy_to_host(self, out: dict, stream=None) -> dict:
        """Copy the hyperedges into caller-owned host arrays (numpy arrays or
        CPU tensors, pinned or not): any of det_offsets (int32/uint32,
        n_edges + 1), det_idx (int32/uint32, n_det_entries), obs_mask
        (int64/uint64, n_edges), prob and logodds (float32, n_edges).
        Returns ``out``."""
        self._check()
        want = {"det_offsets": (self.n_edges + 1, 4), "det_idx": (self.n_det_entries, 4),
                "obs_mask": (self.n_edges, 8), "prob": (self.n_edges, 4), "logodds": (self.n_edges, 4)}
        ptrs = []
        for name, (n, size) in want.items():
            a = out.get(name)
            if a is None:
                ptrs.append(None)
                continue
            if isinstance(a, torch.Tensor):
                if a.is_cuda or not a.is_contiguous() or a.element_size() != size or a.numel() < n:
                    raise ValueError(f"{name}: a contiguous CPU tensor of >= {n} {size}-byte elements")
                ptrs.append(a.data_ptr())
            else:
                if not a.flags["C_CONTIGUOUS"] or a.itemsize != size or a.size < n:
                    raise ValueError(f"{name}: a contiguous array of >= {n} {size}-byte elements")
                ptrs.append(a.ctypes.data)
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        native.check(self.driver.lib.gp_result_to_host(self.driver.handle, *[ctypes.c_void_p(p) for p in ptrs], s))
        return out

    def edges(self, circuit: int = 0, host: dict | None = None) -> dict:
        """{(detector tuple, observable mask): (P, w)} for one circuit."""
        h = host or self.to_host()
        out = {}
        lo, hi = int(h["edge_offsets"][circuit]), int(h["edge_offsets"][circuit + 1])
        off, idx = h["det_offsets"], h["det_idx"]
        for e in range(lo, hi):
            key = (tuple(int(x) for x in idx[off[e]:off[e + 1]]), int(h["obs_mask"][e]))
            if key in out:
                raise ValueError(f"circuit {circuit}: hyperedge {key} appears twice (a class was split)")
            out[key] = (float(h["prob"][e]), float(h["logodds"][e]))
        return out


class Driver:
    """Compiler driver with preallocated device buffers (Sec. 3.4)."""

    def __init__(self, bounds: Bounds, device: int | None = None):
        self.lib = native.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.bounds = bounds
        cb = bounds.to_c()
        size = ctypes.c_uint64()
        native.check(self.lib.gp_workspace_size(ctypes.byref(cb), ctypes.byref(size)))
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(int(size.value) + 256, dtype=torch.uint8, device=self.device)
            base = (self.workspace.data_ptr() + 255) // 256 * 256
            h = ctypes.c_void_p()
            native.check(self.lib.gp_driver_create(ctypes.byref(cb), ctypes.c_void_p(base),
                                                   ctypes.c_uint64(size.value), ctypes.byref(h)))
        self.handle = h
        self.generation = 0
        self._last_noise = None

    @classmethod
    def for_circuits(cls, circuits, batch: int | None = None, slack: float = 1.0) -> "Driver":
        return cls(Bounds.for_circuits(circuits, batch=batch, slack=slack))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gp_driver_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- compile ---------------------------------------------------------------
    def compile(self, circuits, noise, level="L2", stream: torch.cuda.Stream | None = None) -> Dem:
        """Compile one circuit or a batch.  ``circuits``: a Circuit or
        DeviceCircuit, or a list of them (all of one kind).  ``noise``: the
        concatenated noise vectors, numpy (host circuits) or a CUDA float32
        tensor (device circuits)."""
        single = not isinstance(circuits, (list, tuple))
        cl = [circuits] if single else list(circuits)
        on_dev = isinstance(cl[0], DeviceCircuit)
        keep: list = []
        arr = (native.GpCircuit * len(cl))()
        for i, c in enumerate(cl):
            if isinstance(c, DeviceCircuit) != on_dev:
                raise TypeError("a batch must be all host circuits or all device circuits")
            arr[i] = c.to_c() if on_dev else _host_c(c, keep)
        if on_dev:
            if not (isinstance(noise, torch.Tensor) and noise.is_cuda and noise.dtype == torch.float32):
                raise TypeError("device circuits need a CUDA float32 noise tensor")
            noise = noise.contiguous()
            nptr = noise.data_ptr()
        else:
            noise = np.ascontiguousarray(np.asarray(noise, dtype=np.float32))
            keep.append(noise)
            nptr = noise.ctypes.data if noise.size else None
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        view = native.GpDemView()
        self.generation += 1
        code = self.lib.gp_compile_batch(self.handle, arr, len(cl), ctypes.c_void_p(nptr), int(on_dev),
                                         native.LEVELS[level], ctypes.c_void_p(s.cuda_stream),
                                         ctypes.byref(view))
        native.check(code)
        self._last_noise = noise if on_dev else None
        self._last_noise_len = int(sum(c.n_locations for c in cl))
        return Dem(self, view)

    def backward(self, g_prob: torch.Tensor | None, g_logodds: torch.Tensor | None,
                 stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        """d(sum g_prob*P + g_logodds*w)/d(noise) for the last compile."""
        g = torch.empty(max(self._last_noise_len, 1), dtype=torch.float32, device=self.device)
        gp = g_prob.contiguous().float() if g_prob is not None else None
        gw = g_logodds.contiguous().float() if g_logodds is not None else None
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        native.check(self.lib.gp_backward(self.handle, ctypes.c_void_p(gp.data_ptr() if gp is not None else None),
                                          ctypes.c_void_p(gw.data_ptr() if gw is not None else None),
                                          ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
        return g[:self._last_noise_len]

    # -- knobs -------------------------------------------------------------------
    def set_tuning(self, stage1_threads=512, stage1_blocks_per_sm=0, stage2_threads=512, stage2_blocks_per_sm=8,
                   obs_words=4, obs_segments=3, stage1_wide_emit=0):
        t = native.GpTuning(stage1_threads, stage1_blocks_per_sm, stage2_threads, stage2_blocks_per_sm, obs_words,
                            obs_segments, stage1_wide_emit)
        native.check(self.lib.gp_set_tuning(self.handle, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = native.GpTuning()
        native.check(self.lib.gp_get_tuning(self.handle, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in t._fields_}

    def set_host_output(self, arrays: dict | None):
        """Host arrays every later compile also fills with its hyperedges
        (gp_set_host_output): ``det_offsets`` (int32, edges_cap + 1),
        ``det_idx`` (int32), ``obs_mask`` (int64), ``prob`` and ``logodds``
        (float32, edges_cap each) -- page-locked torch tensors or, on a device
        that reads host memory coherently, numpy arrays.  None turns it off.
        The arrays are kept referenced while they are in use."""
        if arrays is None:
            native.check(self.lib.gp_set_host_output(self.handle, None))
            self._host_out = None
            return

        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        def n(a):
            return a.numel() if hasattr(a, "numel") else a.size
        o = native.GpHostOutput(ptr(arrays["det_offsets"]), ptr(arrays["det_idx"]), ptr(arrays["obs_mask"]),
                                ptr(arrays["prob"]), ptr(arrays["logodds"]),
                                min(n(arrays["det_offsets"]) - 1, n(arrays["obs_mask"]), n(arrays["prob"]),
                                    n(arrays["logodds"])), n(arrays["det_idx"]))
        native.check(self.lib.gp_set_host_output(self.handle, ctypes.byref(o)))
        self._host_out = arrays

    def set_debug(self, weak_hash: int = 0, wait_limit: int = 0, stall_windows: int = 0):
        """Test knobs of gp_set_debug: the weak grouping hashes (1: one tag for
        every mask, 2: one hash for every mask), the polls before a device
        wait gives up (0: the default), and a stage 1 that stages no window."""
        d = native.GpDebug(weak_hash, wait_limit, stall_windows, 0)
        native.check(self.lib.gp_set_debug(self.handle, ctypes.byref(d)))

    def enable_timing(self, on: bool = True):
        native.check(self.lib.gp_enable_timing(self.handle, int(on)))

    def last_timing(self) -> list[float]:
        a = (ctypes.c_float * 4)()
        native.check(self.lib.gp_last_timing(self.handle, a))
        return list(a)

    def last_launch_count(self) -> int:
        return int(self.lib.gp_last_launch_count(self.handle))


class DemFunction(torch.autograd.Function):
    """noise (CUDA float32) -> (prob, logodds) of every hyperedge, with the
    hand-written adjoint kernel as backward."""

    @staticmethod
    def forward(ctx, noise, driver, circuits, level):
        dem = driver.compile(circuits, noise.detach(), level)
        ctx.driver, ctx.circuits, ctx.level = driver, circuits, level
        ctx.generation = driver.generation
        ctx.save_for_backward(noise)
        return dem.prob.clone(), dem.logodds.clone()

    @staticmethod
    def backward(ctx, g_prob, g_logodds):
        (noise,) = ctx.saved_tensors
        drv = ctx.driver
        if drv.generation != ctx.generation:       # another compile ran since
            drv.compile(ctx.circuits, noise.detach(), ctx.level)
        g = drv.backward(g_prob, g_logodds)
        return g.to(noise.dtype), None, None, None
