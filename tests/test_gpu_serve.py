"""GPU checks of the cycle-streaming server: a patch streamed cycle by cycle
through the server delivers exactly the hyperedges of the full-circuit
compile (the same GPU library bit for bit; the oracle within the parity
tolerance), whatever the number of cycles merged per step and whatever
other patches share the steps; a horizon that is too short is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_16613_gb300 import circuits as C
from paper_2604_16613_gb300 import native
from paper_2604_16613_gb300.dem import Driver
from paper_2604_16613_gb300.serve import Server

from parity import compare_edges, oracle_edges
from test_serve_semantics import delay_line

pytestmark = pytest.mark.gpu


def f32(x):
    return np.asarray(x, dtype=np.float32)


def gpu_full(circ, level="L2"):
    drv = Driver.for_circuits([circ])
    return drv.compile(circ, f32(circ.default_noise), level).edges()


def log_uniform(circ, seed):
    circ._p = [C.log_uniform_noise(circ.n_locations, seed=seed)]
    circ._frozen = None
    return circ


def workloads():
    return {
        "surface3": (C.rotated_surface_code_memory(3, 6, C.NoiseModel.uniform(1e-3)), 1),
        "surface5": (log_uniform(C.rotated_surface_code_memory(5, 7, C.NoiseModel.uniform(1e-3)), 3), 1),
        "bb": (C.bb_memory(4, C.NoiseModel.uniform(1e-3), seed=3), 1),
        "adaptive": (C.concatenated_adaptive_branch(4, 9, seed=5, noise=C.NoiseModel.uniform(1e-3),
                                                    layout=C.ConcatenatedLayout(4)), 2),
        "delay": (delay_line(9), 3),
    }


@pytest.fixture(scope="module")
def wl():
    return workloads()


@pytest.mark.parametrize("name", ["surface3", "surface5", "bb", "adaptive", "delay"])
@pytest.mark.parametrize("K", [1, 3])
def test_stream_equals_full_compile(wl, name, K):
    circ, H = wl[name]
    srv = Server.for_circuits([circ], max_cycles_per_step=K, max_horizon=H)
    got = srv.stream([circ], [H])[0]
    ref = gpu_full(circ)
    orc = oracle_edges(circ, f32(circ.default_noise))
    assert len(got) == len(ref) == orc.n_classes
    assert set(got) == set(ref)
    for k, (p, w) in ref.items():
        assert got[k][0] == p and got[k][1] == w, k
    compare_edges(got, orc.edges(), f"{name} K={K}")


@pytest.mark.parametrize("name,K", [("surface5", 8), ("adaptive", 6)])
def test_many_cycles_per_step(wl, name, K):
    """Up to K cycles of a patch per step: a window's hyperedges go to up to K
    request slots in one select pass."""
    circ, H = wl[name]
    got = Server.for_circuits([circ], max_cycles_per_step=K, max_horizon=H).stream([circ], [H])[0]
    ref = gpu_full(circ)
    assert got == ref


def test_wide_windows_span_select_chunks():
    """Windows of thousands of hyperedges (several select chunks of 1,024)
    against the full compile and the oracle."""
    circ = C.rotated_surface_code_memory(11, 6, C.NoiseModel.uniform(1e-3))
    srv = Server.for_circuits([circ], max_cycles_per_step=2, max_horizon=1)
    got = srv.stream([circ], [1])[0]
    ref = gpu_full(circ)
    assert got == ref
    orc = oracle_edges(circ, f32(circ.default_noise))
    assert len(got) == orc.n_classes
    compare_edges(got, orc.edges(), "d=11 stream")


def stream_registered(srv, circ, H, mid_repeats_registered=True):
    """Stream a memory experiment whose first and repeated middle cycles are
    registered once and submitted by id (the final cycle as rows); returns
    the union of the delivered hyperedges."""
    blocks = circ.cycle_blocks()
    pid = srv.open_circuit_patch(circ, H)
    first = srv.register_cycle(pid, blocks[0])
    mid = srv.register_cycle(pid, blocks[1])
    rids = [srv.submit_registered(pid, first)]
    rids += [srv.submit_registered(pid, mid) for _ in blocks[1:-1]]
    rids.append(srv.submit(pid, blocks[-1]))
    out, done = {}, 0
    for _ in range(4 * len(rids)):          # a server that stops making progress fails, never hangs
        if done == len(rids):
            break
        srv.step()
        for r in srv.completed():
            Server._merge(out, Server.edges(srv.result(r)), 0)
            srv.release(r)
            done += 1
    assert done == len(rids)
    srv.close_patch(pid)
    return out


@pytest.mark.parametrize("name,rounds,K", [("surface", 9, 1), ("surface", 9, 2), ("bb", 7, 1)])
def test_registered_cycles_equal_full_compile(name, rounds, K):
    """Registered cycles repeated by id: the first window of each pattern
    runs the horizon test, later windows of the same registered cycles leave
    the records-only noise out.  The stream equals the full compile bit for
    bit and the oracle within tolerance, on a server reused for a second
    stream."""
    circ = (C.rotated_surface_code_memory(5, rounds, C.NoiseModel.uniform(1e-3)) if name == "surface"
            else C.bb_memory(rounds, C.NoiseModel.uniform(1e-3), seed=3))
    blocks = circ.cycle_blocks()
    for b in blocks[2:-1]:
        for k in ("ops", "recs", "noise"):
            assert np.array_equal(np.asarray(blocks[1][k]), np.asarray(b[k]))
    srv = Server.for_circuits([circ], max_cycles_per_step=K, max_horizon=1, max_pending=4 * rounds)
    ref = gpu_full(circ)
    for _ in range(2):
        got = stream_registered(srv, circ, 1)
        assert got == ref
    orc = oracle_edges(circ, f32(circ.default_noise))
    assert len(ref) == orc.n_classes
    compare_edges(got, orc.edges(), f"{name} registered K={K}")


def test_adaptive_d10_stream_equals_full_compile():
    """A realised branch of the adaptive [[4,2,2]]-concatenated code at outer
    distance 10 (the serving bench's adaptive patch), streamed cycle by cycle
    as rows with H = 5 (its outer checks run every d/2 cycles), two cycles per
    step: the delivered hyperedges equal the full compile bit for bit."""
    circ = C.concatenated_adaptive_branch(10, 14, seed=4000, noise=C.NoiseModel.uniform(1e-3))
    got = Server.for_circuits([circ], max_cycles_per_step=2, max_horizon=5).stream([circ], [5])[0]
    ref = gpu_full(circ)
    assert len(got) == len(ref)
    assert got == ref


def test_levels(wl):
    circ, H = wl["surface5"]
    srv = Server.for_circuits([circ], max_cycles_per_step=2, max_horizon=H)
    for level in ("L0", "L1"):
        got = srv.stream([circ], [H], level=level)[0]
        orc = oracle_edges(circ, f32(circ.default_noise), level)
        assert len(got) == orc.n_classes, level
        compare_edges(got, orc.edges(), level)


def test_mix_equals_alone(wl):
    """Patches sharing steps (batch smaller than the patch count, cycles
    interleaved) get the same hyperedges as each patch served alone."""
    names = ["surface3", "surface5", "bb", "adaptive", "delay", "surface3"]
    circs = [wl[n][0] for n in names]
    hs = [wl[n][1] for n in names]
    mixed = Server.for_circuits(circs, max_batch=4, max_cycles_per_step=2, max_horizon=max(hs),
                                max_pending=64).stream(circs, hs)
    for n, c, h, got in zip(names, circs, hs, mixed):
        alone = Server.for_circuits([c], max_cycles_per_step=1, max_horizon=h).stream([c], [h])[0]
        assert got == alone, n


def test_tuning_does_not_change_stream(wl):
    """The server's compile tuning (launch shapes, observable split) changes
    no delivered hyperedge."""
    names = ["surface5", "bb", "adaptive"]
    circs = [wl[n][0] for n in names]
    hs = [wl[n][1] for n in names]
    base = Server.for_circuits(circs, max_cycles_per_step=2, max_horizon=max(hs)).stream(circs, hs)
    srv = Server.for_circuits(circs, max_cycles_per_step=2, max_horizon=max(hs))
    srv.set_tuning(1024, 0, 256, 4, 1, 1, 1)
    assert srv.stream(circs, hs) == base
    with pytest.raises(native.GpError):
        srv.set_tuning(obs_words=0)


def test_record_horizon_refused_at_submit(wl):
    circ, _ = wl["adaptive"]          # outer detectors look two cycles back
    srv = Server.for_circuits([circ], max_horizon=2)
    pid = srv.open_circuit_patch(circ, horizon=1)
    blocks = circ.cycle_blocks()
    with pytest.raises(native.GpError) as e:
        for b in blocks:
            srv.submit(pid, b)
    assert e.value.code == native.GP_ERR_HORIZON


def test_reach_horizon_found_on_the_device(wl):
    """The bucket brigade's records reach one cycle back, its errors three:
    with H = 1 the submissions pass and the windows report the horizon."""
    circ, _ = wl["delay"]
    srv = Server.for_circuits([circ], max_horizon=1, max_pending=32)
    pid = srv.open_circuit_patch(circ, horizon=1)
    ids = [srv.submit(pid, b) for b in circ.cycle_blocks()]
    statuses = []
    for _ in range(4 * len(ids)):            # a server that stops making progress fails, never hangs
        if len(statuses) == len(ids):
            break
        srv.step()
        for r in srv.completed():
            statuses.append(srv.result(r, raise_on_error=False)["status"])
    assert len(statuses) == len(ids), "the server stopped completing requests"
    assert native.GP_ERR_HORIZON in statuses
    # the server stays usable
    good = Server.for_circuits([circ], max_horizon=3).stream([circ], [3])[0]
    assert set(good) == set(gpu_full(circ))


def test_api_errors(wl):
    circ, _ = wl["surface3"]
    srv = Server.for_circuits([circ], max_patches=1)
    pid = srv.open_circuit_patch(circ)
    with pytest.raises(native.GpError) as e:
        srv.open_circuit_patch(circ)
    assert e.value.code == native.GP_ERR_CAPACITY
    blocks = circ.cycle_blocks()
    with pytest.raises(native.GpError):
        srv.submit(pid, blocks[-1], final=False)      # observables only in a final cycle
    big = dict(blocks[0])
    big["ops"] = np.concatenate([blocks[0]["ops"]] * 3)
    with pytest.raises(native.GpError) as e:
        srv.submit(pid, big)
    assert e.value.code == native.GP_ERR_CAPACITY
    rid = srv.submit(pid, blocks[0])
    with pytest.raises(native.GpError):
        srv.close_patch(pid)                          # pending cycle
    with pytest.raises(native.GpError):
        srv.result(rid)                               # not finished
    assert srv.step() == 1
    assert srv.completed() == [rid]
    assert srv.result(rid)["cycle"] == 0
    srv.release(rid)
    srv.close_patch(pid)
