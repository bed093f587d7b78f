"""Python binding of the cycle-streaming server (include/gpserve.h).

Argument marshalling only: window assembly, compilation and selection of the
sealed hyperedges run in the library.  ``Server.for_circuits`` sizes a
server from example patches; ``Server.stream`` pushes whole patches through
it (a convenience for tests and benchmarks).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native
from .circuits import DEPOLARIZE1, DEPOLARIZE2, MEASURE_KINDS, TICK, X_ERROR, Z_ERROR

# components per noise channel at L0, L1, L2
_COMP = {X_ERROR: (1, 1, 1), Z_ERROR: (1, 1, 1), DEPOLARIZE1: (2, 3, 3), DEPOLARIZE2: (6, 10, 15)}


def cycle_sizes(block: dict) -> dict:
    """Per-cycle sizes the server bounds (mechanisms at L2)."""
    k = block["ops"][:, 0]
    mech = sum(int((k == kind).sum()) * c[2] for kind, c in _COMP.items())
    return dict(ops=int(k.size), recs=int(block["recs"].size), locations=int(block["n_locations"]),
                measurements=int(np.isin(k, list(MEASURE_KINDS)).sum()), detectors=int(block["n_detectors"]),
                mechanisms=mech, layers=int((k == TICK).sum()) + 1)


class Server:
    """A cycle-streaming server on the current CUDA device."""

    def __init__(self, **cfg):
        self.lib = native.load()
        c = native.GpServerConfig()
        for name, _ in native.GpServerConfig._fields_:
            setattr(c, name, int(cfg.get(name, 0)))
        self.config = c
        h = ctypes.c_void_p()
        native.check(self.lib.gp_server_create(ctypes.byref(c), ctypes.byref(h)))
        self.handle = h
        self._patches = {}

    @classmethod
    def for_circuits(cls, circuits, max_patches=None, max_batch=None, max_cycles_per_step=1, max_horizon=1,
                     max_pending=None, slack=1.0) -> "Server":
        """Bounds from the cycles of example patches (circuits with cycle
        marks and declared logicals)."""
        circuits = list(circuits)
        agg = dict(ops=0, recs=0, locations=0, measurements=0, detectors=0, mechanisms=0, layers=0)
        for c in circuits:
            for b in c.cycle_blocks():
                for k, v in cycle_sizes(b).items():
                    agg[k] = max(agg[k], v)
        n = len(circuits)
        mp = max_patches or n
        return cls(max_patches=mp, max_batch=max_batch or mp, max_cycles_per_step=max_cycles_per_step,
                   max_horizon=max_horizon, max_pending=max_pending or 4 * mp * max(1, max_cycles_per_step),
                   max_qubits=max(c.n_qubits for c in circuits),
                   max_cycle_ops=int(agg["ops"] * slack) + 1, max_cycle_recs=int(agg["recs"] * slack) + 1,
                   max_cycle_locations=int(agg["locations"] * slack) + 1,
                   max_cycle_measurements=int(agg["measurements"] * slack) + 1,
                   max_cycle_detectors=int(agg["detectors"] * slack) + 1,
                   max_cycle_mechanisms=int(agg["mechanisms"] * slack) + 1,
                   max_cycle_layers=int(agg["layers"] * slack) + 1,
                   max_logical_qubits=max(sum(len(lg) for lg in c.logicals) for c in circuits))

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.gp_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- patches ---------------------------------------------------------------
    def open_patch(self, n_qubits: int, logicals, horizon: int = 1) -> int:
        flat = np.ascontiguousarray(np.concatenate([np.asarray(lg, np.uint32) for lg in logicals])
                                    if len(logicals) else np.zeros(1, np.uint32), dtype=np.uint32)
        off = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(lg) for lg in logicals])]), dtype=np.uint32)
        spec = native.GpPatchSpec(int(n_qubits), int(horizon), len(logicals),
                                  flat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                  off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        pid = ctypes.c_uint32()
        native.check(self.lib.gp_server_open_patch(self.handle, ctypes.byref(spec), ctypes.byref(pid)))
        self._patches[pid.value] = (int(n_qubits), len(logicals))
        return pid.value

    def open_circuit_patch(self, circuit, horizon: int = 1) -> int:
        return self.open_patch(circuit.n_qubits, circuit.logicals, horizon)

    def close_patch(self, patch: int):
        native.check(self.lib.gp_server_close_patch(self.handle, int(patch)))
        self._patches.pop(patch, None)

    # -- requests ----------------------------------------------------------------
    def submit(self, patch: int, block: dict, final: bool | None = None, t_arrival_ns: int = 0) -> int:
        n_qubits, n_obs = self._patches[patch]
        ops = np.ascontiguousarray(block["ops"], dtype=np.uint32)
        recs = np.ascontiguousarray(block["recs"], dtype=np.uint32)
        noise = np.ascontiguousarray(block["noise"], dtype=np.float32)
        g = native.GpCircuit(ops.ctypes.data if ops.size else None, ops.shape[0],
                             recs.ctypes.data if recs.size else None, recs.size, n_qubits,
                             int(block["n_detectors"]), n_obs, int(block["n_locations"]))
        fin = block.get("final", False) if final is None else final
        rid = ctypes.c_uint64()
        native.check(self.lib.gp_server_submit(self.handle, int(patch), ctypes.byref(g),
                                               noise.ctypes.data if noise.size else None, int(bool(fin)),
                                               int(t_arrival_ns), ctypes.byref(rid)))
        return rid.value

    def register_cycle(self, patch: int, block: dict) -> int:
        """Register a cycle the patch repeats; returns its id."""
        n_qubits, n_obs = self._patches[patch]
        ops = np.ascontiguousarray(block["ops"], dtype=np.uint32)
        recs = np.ascontiguousarray(block["recs"], dtype=np.uint32)
        noise = np.ascontiguousarray(block["noise"], dtype=np.float32)
        g = native.GpCircuit(ops.ctypes.data if ops.size else None, ops.shape[0],
                             recs.ctypes.data if recs.size else None, recs.size, n_qubits,
                             int(block["n_detectors"]), n_obs, int(block["n_locations"]))
        cid = ctypes.c_uint32()
        native.check(self.lib.gp_server_register_cycle(self.handle, int(patch), ctypes.byref(g),
                                                       noise.ctypes.data if noise.size else None,
                                                       ctypes.byref(cid)))
        return cid.value

    def submit_registered(self, patch: int, cycle_id: int, final: bool = False, t_arrival_ns: int = 0) -> int:
        rid = ctypes.c_uint64()
        native.check(self.lib.gp_server_submit_registered(self.handle, int(patch), int(cycle_id), int(bool(final)),
                                                          int(t_arrival_ns), ctypes.byref(rid)))
        return rid.value

    def submit_registered_many(self, patches, cycle_ids, finals=None, t_arrival_ns=None,
                               stop_when_full: bool = False) -> np.ndarray:
        """Submit many registered cycles (numpy arrays); returns the ids of
        those queued.  With ``stop_when_full`` a full queue ends the call
        early instead of raising."""
        p = np.ascontiguousarray(patches, dtype=np.uint32)
        c = np.ascontiguousarray(cycle_ids, dtype=np.uint32)
        f = None if finals is None else np.ascontiguousarray(finals, dtype=np.uint8)
        t = None if t_arrival_ns is None else np.ascontiguousarray(t_arrival_ns, dtype=np.uint64)
        ids = np.zeros(p.size, dtype=np.uint64)
        n = ctypes.c_uint32()
        code = self.lib.gp_server_submit_registered_many(
            self.handle, p.size, p.ctypes.data, c.ctypes.data, None if f is None else f.ctypes.data,
            None if t is None else t.ctypes.data, ids.ctypes.data, ctypes.byref(n))
        if not (stop_when_full and code == native.GP_ERR_CAPACITY):
            native.check(code)
        return ids[:n.value]

    def drain(self, cap: int = 65536) -> dict:
        """Finished requests (released): ids, arrival and completion times,
        hyperedges delivered, status."""
        ids = np.zeros(cap, np.uint64)
        ta = np.zeros(cap, np.uint64)
        td = np.zeros(cap, np.uint64)
        ne = np.zeros(cap, np.uint32)
        st = np.zeros(cap, np.int32)
        n = ctypes.c_uint32()
        native.check(self.lib.gp_server_drain(self.handle, cap, ids.ctypes.data, ta.ctypes.data, td.ctypes.data,
                                              ne.ctypes.data, st.ctypes.data, ctypes.byref(n)))
        k = n.value
        return dict(ids=ids[:k], t_arrival_ns=ta[:k], t_done_ns=td[:k], n_edges=ne[:k], status=st[:k])

    def step(self, level="L2", stream=None) -> int:
        n = ctypes.c_uint32()
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else None)
        native.check(self.lib.gp_server_step(self.handle, native.LEVELS[level], s, ctypes.byref(n)))
        return n.value

    def set_tuning(self, stage1_threads=512, stage1_blocks_per_sm=0, stage2_threads=512, stage2_blocks_per_sm=8,
                   obs_words=4, obs_segments=3, stage1_wide_emit=1):
        """Launch and work-split parameters of the server's compiles (as
        ``Driver.set_tuning``); results do not change."""
        t = native.GpTuning(stage1_threads, stage1_blocks_per_sm, stage2_threads, stage2_blocks_per_sm, obs_words,
                            obs_segments, stage1_wide_emit)
        native.check(self.lib.gp_server_set_tuning(self.handle, ctypes.byref(t)))

    def last_timing(self) -> list[float]:
        """Microseconds of the last step: host build, compile, select,
        hand-out, then the compile's device stages (lowering, stage 1,
        grouping, compaction)."""
        a = (ctypes.c_float * 8)()
        native.check(self.lib.gp_server_last_timing(self.handle, a))
        return list(a)

    def completed(self, cap: int = 4096) -> list[int]:
        out = []
        buf = (ctypes.c_uint64 * cap)()
        while True:
            n = ctypes.c_uint32()
            native.check(self.lib.gp_server_completed(self.handle, buf, cap, ctypes.byref(n)))
            out.extend(buf[: n.value])
            if n.value < cap:
                return out

    def result(self, request: int, raise_on_error: bool = True) -> dict:
        v = native.GpSealedView()
        native.check(self.lib.gp_server_result(self.handle, int(request), ctypes.byref(v)))
        if raise_on_error and v.status != native.GP_OK:
            raise native.GpError(v.status, f"request {request} (patch {v.patch}, cycle {v.cycle}) failed")

        def arr(ptr, n, dt):
            return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True) if n else np.zeros(0, dt)

        return dict(request=v.request, patch=v.patch, cycle=v.cycle, status=v.status,
                    det_offsets=arr(v.det_offsets, v.n_edges + 1, np.uint32),
                    det_idx=arr(v.det_idx, v.n_det_entries, np.uint32),
                    obs_mask=arr(v.obs_mask, v.n_edges, np.uint64), prob=arr(v.prob, v.n_edges, np.float32),
                    logodds=arr(v.logodds, v.n_edges, np.float32),
                    t_arrival_ns=v.t_arrival_ns, t_done_ns=v.t_done_ns)

    def release(self, request: int):
        native.check(self.lib.gp_server_release(self.handle, int(request)))

    # -- convenience ---------------------------------------------------------------
    @staticmethod
    def edges(res: dict) -> dict:
        """{(detector tuple, observable mask): (P, w)} of one request's result."""
        off, det = res["det_offsets"], res["det_idx"]
        out = {}
        for i in range(len(res["prob"])):
            key = (tuple(int(x) for x in det[off[i]:off[i + 1]]), int(res["obs_mask"][i]))
            if key in out:
                raise ValueError(f"request {res['request']}: hyperedge {key} delivered twice")
            out[key] = (float(res["prob"][i]), float(res["logodds"][i]))
        return out

    @staticmethod
    def _merge(acc: dict, part: dict, patch: int):
        """Add one request's hyperedges to a patch's union; a hyperedge
        delivered by two requests of one patch is an error."""
        dup = acc.keys() & part.keys()
        if dup:
            raise ValueError(f"patch {patch}: hyperedge {next(iter(dup))} delivered by two requests")
        acc.update(part)

    def stream(self, circuits, horizons=None, level="L2", interleave=True) -> list[dict]:
        """Open one patch per circuit, submit every cycle (round-robin over
        patches when ``interleave``), step until all are done; returns, per
        circuit, the union of its requests' hyperedges."""
        horizons = horizons or [1] * len(circuits)
        pids = [self.open_circuit_patch(c, h) for c, h in zip(circuits, horizons)]
        blocks = [c.cycle_blocks() for c in circuits]
        out = [dict() for _ in circuits]
        owner = {}
        order = []
        if interleave:
            for t in range(max(len(b) for b in blocks)):
                order += [(i, t) for i in range(len(circuits)) if t < len(blocks[i])]
        else:
            order = [(i, t) for i in range(len(circuits)) for t in range(len(blocks[i]))]
        pending = 0
        for i, t in order:
            while True:
                try:
                    rid = self.submit(pids[i], blocks[i][t])
                    break
                except native.GpError as e:
                    if e.code != native.GP_ERR_CAPACITY or pending == 0:
                        raise
                    done = self.step(level)
                    if done == 0:
                        raise RuntimeError("server made no progress")
                    pending -= done
                    for r in self.completed():
                        self._merge(out[owner[r]], self.edges(self.result(r)), owner[r])
                        self.release(r)
            owner[rid] = i
            pending += 1
        while pending:
            done = self.step(level)
            if done == 0:
                raise RuntimeError("server made no progress")
            pending -= done
            for r in self.completed():
                self._merge(out[owner[r]], self.edges(self.result(r)), owner[r])
                self.release(r)
        for p in pids:
            self.close_patch(p)
        return out
