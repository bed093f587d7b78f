"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

Masks (hyperedge keys) must match bit-exactly; probabilities within 1e-5
relative; gradients within 1e-4 relative (or 1e-6 of the largest entry).
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_2604_16613_gb300 import circuits as C
from paper_2604_16613_gb300 import native
from paper_2604_16613_gb300.dem import Bounds, DeviceCircuit, Driver

from parity import compare_arrays, compare_edges, oracle_edges

pytestmark = pytest.mark.gpu


def f32(x):
    return np.asarray(x, dtype=np.float32)


def run(circ, noise, level="L2", device=True, drv=None):
    drv = drv or Driver.for_circuits([circ])
    if device:
        dem = drv.compile(DeviceCircuit(circ), torch.tensor(f32(noise), device="cuda"), level)
    else:
        dem = drv.compile(circ, f32(noise), level)
    return drv, dem


CODES = [
    ("fig1", lambda: C.repetition_code_memory(3, 2, C.NoiseModel.uniform(1e-3), final_data=False)),
    ("rep5", lambda: C.repetition_code_memory(5, 5, C.NoiseModel.hardware_inspired(1e-2))),
    ("surf3", lambda: C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))),
    ("surf4", lambda: C.rotated_surface_code_memory(4, 4, C.NoiseModel.uniform(2e-3))),
    ("surf5", lambda: C.rotated_surface_code_memory(5, 5, C.NoiseModel.hardware_inspired(1e-3))),
    ("surf7", lambda: C.rotated_surface_code_memory(7, 7, C.NoiseModel.uniform(1e-3))),
]


@pytest.mark.parametrize("name,make", CODES, ids=[c[0] for c in CODES])
@pytest.mark.parametrize("level", ["L0", "L1", "L2"])
def test_codes_parity(name, make, level):
    circ = make()
    noise = C.log_uniform_noise(circ.n_locations, seed=3)
    _, dem = run(circ, noise, level)
    ref = oracle_edges(circ, noise, level)
    compare_edges(dem.edges(), ref.edges(), f"{name}/{level}")
    assert dem.n_edges == ref.n_classes


def test_host_and_device_inputs_agree():
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=4)
    drv, d1 = run(circ, noise, device=True)
    h1 = d1.to_host()
    _, d2 = run(circ, noise, device=False, drv=drv)
    h2 = d2.to_host()
    for k in ("det_offsets", "det_idx", "obs_mask", "prob", "logodds"):
        assert np.array_equal(h1[k], h2[k]), k


def test_repeated_compiles_bit_identical():
    circ = C.rotated_surface_code_memory(7, 7, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=5)
    drv = Driver.for_circuits([circ])
    dc = DeviceCircuit(circ)
    nz = torch.tensor(f32(noise), device="cuda")
    outs = [drv.compile(dc, nz).to_host() for _ in range(3)]
    for o in outs[1:]:
        for k in o:
            assert np.array_equal(o[k], outs[0][k]), k


def test_random_circuits_parity():
    for seed in range(240):
        circ = C.random_circuit(seed)
        noise = circ.default_noise
        level = ["L0", "L1", "L2"][seed % 3]
        _, dem = run(circ, noise, level)
        ref = oracle_edges(circ, noise, level)
        assert dem.n_edges == ref.n_classes, f"seed {seed}"
        compare_edges(dem.edges(), ref.edges(), f"seed {seed}")


def test_batch_matches_individual_and_oracle():
    circs = [C.random_circuit(1000 + s) for s in range(40)]
    circs += [C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3)),
              C.repetition_code_memory(5, 3, C.NoiseModel.uniform(1e-3))]
    noises = [c.default_noise for c in circs]
    drv = Driver.for_circuits(circs)
    dem = drv.compile(circs, f32(np.concatenate(noises)))
    host = dem.to_host()
    assert dem.n_circuits == len(circs)
    for b, (c, nz) in enumerate(zip(circs, noises)):
        got = dem.edges(b, host)
        compare_arrays(host, b, oracle_edges(c, nz), f"batch circuit {b}")
        solo = Driver.for_circuits([c]).compile(c, f32(nz)).edges()
        assert got == solo, f"circuit {b}: result differs alone and in the batch"


@pytest.mark.parametrize("d", [11, 15])
def test_surface_parity_large(d):
    circ = C.rotated_surface_code_memory(d, d, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=2)
    _, dem = run(circ, noise)
    ref = oracle_edges(circ, noise)
    compare_arrays(dem.to_host(), 0, ref, f"d={d}")


def test_surface_d25_full_size():
    """The benchmark's workload (d = 25, 25 rounds, log-uniform noise, L2) in
    the benchmark's launch configuration, compared with the oracle on every
    hyperedge."""
    circ = C.rotated_surface_code_memory(25, 25, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=2)
    _, dem = run(circ, noise)
    ref = oracle_edges(circ, noise)
    assert dem.n_edges == ref.n_classes
    wp, _ = compare_edges(dem.edges(), ref.edges(), "d=25")
    assert wp <= 1e-5


# ---------------------------------------------------------------------------
# exact grouping under hash collisions
# ---------------------------------------------------------------------------

WEAK = [
    ("surf5-constant-hash", lambda: C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3)), 2),
    ("surf5-constant-tag", lambda: C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3)), 1),
    ("surf15-constant-tag", lambda: C.rotated_surface_code_memory(15, 15, C.NoiseModel.uniform(1e-3)), 1),
    ("bb4-constant-tag", lambda: C.bb_memory(4, C.NoiseModel.uniform(1e-3), seed=3), 1),
]


@pytest.mark.parametrize("name,make,mode", WEAK, ids=[w[0] for w in WEAK])
def test_weak_hash_grouping_stays_exact(name, make, mode):
    """The grouping table's claims are verified on whole masks (Sec. 3.2's
    aggregator only argues that hash collisions are unlikely).  With every
    mask given the same tag (mode 1) or the same hash (mode 2), every probe
    that meets another class must be told apart by the word-by-word check;
    the model must still equal the oracle's exactly, class for class."""
    circ = make()
    noise = f32(C.log_uniform_noise(circ.n_locations, seed=2))
    drv = Driver.for_circuits([circ])
    dc, nz = DeviceCircuit(circ), torch.tensor(noise, device="cuda")
    normal = drv.compile(dc, nz).to_host()
    drv.set_debug(weak_hash=mode)
    weak = drv.compile(dc, nz).to_host()
    compare_arrays(weak, 0, oracle_edges(circ, noise), name)
    for k in ("det_offsets", "det_idx", "obs_mask", "prob", "logodds"):
        assert np.array_equal(weak[k], normal[k]), k


def test_weak_hash_random_batch_stays_exact():
    """A batch of random circuits (all gate kinds, both bases) grouped with a
    single hash value for every mask."""
    circs = [C.random_circuit(3000 + s) for s in range(24)]
    noises = [f32(c.default_noise) for c in circs]
    drv = Driver.for_circuits(circs)
    drv.set_debug(weak_hash=2)
    for level in ("L0", "L2"):
        host = drv.compile(circs, np.concatenate(noises), level).to_host()
        for b, (c, nz) in enumerate(zip(circs, noises)):
            compare_arrays(host, b, oracle_edges(c, nz, level), f"weak batch {level} circuit {b}")


# ---------------------------------------------------------------------------
# bounded device waits
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("walk", ["role-split", "block-wide"])
def test_device_wait_timeout_is_reported_and_driver_recovers(walk):
    """Stage 1 with no layer window staged: the first wait of every walk can
    only run out.  With a short wait limit the compile returns
    GP_ERR_TIMEOUT quickly (no hang, no fault, nothing left running), and the
    next compile on the same driver, with the knobs back to normal, equals the
    oracle and the compile made before the timeout."""
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    noise = f32(C.log_uniform_noise(circ.n_locations, seed=8))
    bd = Bounds.for_circuits([circ])
    if walk == "block-wide":
        bd.max_qubits = 4096          # the role-split tables no longer fit
    drv = Driver(bd)
    dc, nz = DeviceCircuit(circ), torch.tensor(noise, device="cuda")
    before = drv.compile(dc, nz).to_host()
    drv.set_debug(wait_limit=256, stall_windows=1)
    t0 = time.perf_counter()
    msg = expect_error(native.GP_ERR_TIMEOUT, lambda: drv.compile(dc, nz))
    assert "timed out" in msg
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 30.0
    drv.set_debug()
    after = drv.compile(dc, nz).to_host()
    compare_arrays(after, 0, oracle_edges(circ, noise), f"{walk} after timeout")
    for k in ("det_offsets", "det_idx", "obs_mask", "prob", "logodds"):
        assert np.array_equal(after[k], before[k]), k


def test_debug_knobs_are_validated():
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    drv = Driver.for_circuits([circ])
    expect_error(native.GP_ERR_INVALID, lambda: drv.set_debug(weak_hash=3))
    expect_error(native.GP_ERR_INVALID, lambda: drv.set_debug(stall_windows=2))


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_noiseless_and_detectorless_circuits():
    c = C.rotated_surface_code_memory(3, 2, None)          # no noise rows
    _, dem = run(c, np.zeros(0))
    assert dem.n_edges == 0
    c2 = C.Circuit(2)                                        # noise, nothing to flip
    c2.gate1(C.R, [0, 1]); c2.tick()
    c2.noise(C.DEPOLARIZE1, [0, 1], 0.01)
    c2.measure(C.M, [0])
    _, dem2 = run(c2, c2.default_noise)
    assert dem2.n_edges == 0


def test_zero_probability_locations_are_dropped():
    circ = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=6)
    noise[::3] = 0.0
    _, dem = run(circ, noise)
    compare_edges(dem.edges(), oracle_edges(circ, noise).edges(), "p=0")


def test_nop_rows_equal_zero_probability_locations():
    """A NOP row is ignored: noise rows turned into NOP rows give the model of
    the same circuit with those locations at p = 0 (which contribute no
    mechanism, Sec. 2.1.4), against the oracle."""
    import copy
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    noise = C.log_uniform_noise(circ.n_locations, seed=8)
    ops = np.array(circ.ops, dtype=np.uint32).reshape(-1, 4).copy()
    rows = np.flatnonzero(ops[:, 0] >= 32)[1::3]
    zero = noise.copy()
    zero[ops[rows, 3]] = 0.0
    ops[rows] = [7, 0, 0, 0]
    nop = copy.copy(circ)
    nop._ops, nop._frozen = [ops], None
    assert np.array_equal(nop.recs, circ.recs)
    _, dem = run(nop, noise)
    compare_edges(dem.edges(), oracle_edges(circ, zero).edges(), "nop")


def test_host_output_equals_device_result():
    """Host output (gp_set_host_output): the compaction kernel also writes the
    hyperedges into caller-owned host arrays; they equal the device result
    bit for bit (page-locked tensors, and numpy arrays where the device reads
    host memory coherently); a capacity too small fails the compile; turning
    it off restores the plain compile."""
    circs = [C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3)),
             C.bb_memory(3, C.NoiseModel.uniform(1e-3), seed=3)] + [C.random_circuit(s) for s in range(4)]
    noise = np.concatenate([f32(c.default_noise) for c in circs])
    drv = Driver.for_circuits(circs)
    ref = drv.compile(circs, noise).to_host()
    ne, nd = ref["det_offsets"].size - 1, ref["det_idx"].size
    cap_e, cap_d = ne + 7, nd + 13

    def arrays(make):
        return {"det_offsets": make(cap_e + 1, np.int32), "det_idx": make(cap_d, np.int32),
                "obs_mask": make(cap_e, np.int64), "prob": make(cap_e, np.float32),
                "logodds": make(cap_e, np.float32)}

    def check(out):
        assert np.array_equal(np.asarray(out["det_offsets"])[:ne + 1], ref["det_offsets"])
        assert np.array_equal(np.asarray(out["det_idx"])[:nd], ref["det_idx"])
        assert np.array_equal(np.asarray(out["obs_mask"])[:ne].view(np.uint64), ref["obs_mask"])
        assert np.array_equal(np.asarray(out["prob"])[:ne], ref["prob"])
        assert np.array_equal(np.asarray(out["logodds"])[:ne], ref["logodds"])

    pinned = arrays(lambda n, t: torch.full((n,), -1, dtype=getattr(torch, np.dtype(t).name), pin_memory=True))
    drv.set_host_output(pinned)
    for inputs_on_device in (False, True):
        for a in pinned.values():
            a.fill_(-1)
        if inputs_on_device:
            drv.compile([DeviceCircuit(c) for c in circs], torch.tensor(noise, device="cuda"))
        else:
            drv.compile(circs, noise)
        check({k: v.numpy() for k, v in pinned.items()})
    try:
        plain = arrays(lambda n, t: np.full(n, -1, dtype=t))
        drv.set_host_output(plain)
    except native.GpError as e:
        assert e.code == native.GP_ERR_INVALID        # pageable memory on a device that cannot read it
    else:
        drv.compile(circs, noise)
        check(plain)
    small = {k: v[: (ne // 2 + 1 if k == "det_offsets" else ne // 2)] for k, v in pinned.items()}
    drv.set_host_output(small)
    with pytest.raises(native.GpError) as e:
        drv.compile(circs, noise)
    assert e.value.code == native.GP_ERR_CAPACITY
    drv.set_host_output(None)
    again = drv.compile(circs, noise).to_host()
    for k in ref:
        assert np.array_equal(ref[k], again[k]), k


def test_saturated_x_error():
    c = C.Circuit(1)
    c.gate1(C.R, [0]); c.tick()
    c.noise(C.X_ERROR, [0], 0.5)
    c.noise(C.X_ERROR, [0], 0.01)
    rec = c.measure(C.M, [0])
    c.detector([rec[0]])
    _, dem = run(c, c.default_noise)
    (e, (P, w)), = dem.edges().items()
    assert e == ((0,), 0)
    assert P == pytest.approx(0.5, abs=1e-7) and abs(w) < 1e-6


def expect_error(code, fn):
    with pytest.raises(native.GpError) as ex:
        fn()
    assert ex.value.code == code, str(ex.value)
    return str(ex.value)


def test_error_paths_and_recovery():
    good = C.rotated_surface_code_memory(3, 3, C.NoiseModel.uniform(1e-3))
    noise = good.default_noise
    drv = Driver(Bounds.for_circuits([good], slack=2.0))
    # non-deterministic detector: X-basis reset measured in Z
    nd = C.Circuit(good.n_qubits)
    nd.gate1(C.RX, [0]); nd.tick()
    r = nd.measure(C.M, [0])
    nd.detector([r[0]])
    msg = expect_error(native.GP_ERR_NONDETERMINISTIC, lambda: drv.compile(nd, np.zeros(0)))
    assert "anticommutes" in msg
    # qubit out of range
    bad = C.Circuit.from_text(good.to_text())
    ops = bad.ops.copy()
    ops[0, 1] = good.n_qubits + 5
    bad._frozen = (ops, bad.recs, bad.default_noise)
    expect_error(native.GP_ERR_INVALID, lambda: drv.compile(bad, noise))
    # two gates on one qubit in one layer
    two = C.Circuit(2)
    two.gate1(C.R, [0, 1]); two.tick()
    two.gate1(C.H, [0]); two.gate1(C.H, [0]); two.tick()
    rr = two.measure(C.M, [1])
    two.detector([rr[0]])
    two.noise(C.X_ERROR, [1], 0.01)
    expect_error(native.GP_ERR_INVALID, lambda: drv.compile(two, two.default_noise))
    # noise outside the channel's range
    nz = noise.copy()
    nz[5] = 0.9
    expect_error(native.GP_ERR_INVALID, lambda: drv.compile(good, nz))
    # detector count in the header disagrees with the rows
    wrong = C.Circuit.from_text(good.to_text())
    wrong.n_detectors += 1
    expect_error(native.GP_ERR_INVALID, lambda: drv.compile(wrong, noise))
    # mask wider than the slot bound
    wide = C.rotated_surface_code_memory(11, 2, C.NoiseModel.uniform(1e-3))
    small2 = Driver(Bounds(**{**Bounds.for_circuits([wide]).__dict__, "max_mask_words": 1}))
    expect_error(native.GP_ERR_CAPACITY, lambda: small2.compile(wide, wide.default_noise))
    # too many circuits for the bounds
    expect_error(native.GP_ERR_CAPACITY, lambda: drv.compile([good, good], np.concatenate([noise, noise])))
    # the drivers still work after every failure (a one-word bound still
    # serves circuits whose masks fit one word: no observable, 64 detectors)
    ok = drv.compile(good, f32(noise)).edges()
    compare_edges(ok, oracle_edges(good, noise).edges(), "after errors")
    narrow = C.repetition_code_memory(5, 3, C.NoiseModel.uniform(1e-3), final_data=False)
    ok2 = small2.compile(narrow, f32(narrow.default_noise)).edges()
    compare_edges(ok2, oracle_edges(narrow, narrow.default_noise).edges(), "narrow after errors")


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d", [3, 5])
def test_gradient_matches_oracle(d):
    circ = C.rotated_surface_code_memory(d, d, C.NoiseModel.uniform(1e-3))
    noise = f32(C.log_uniform_noise(circ.n_locations, seed=9))
    drv = Driver.for_circuits([circ])
    dem = drv.compile(DeviceCircuit(circ), torch.tensor(noise, device="cuda"))
    host = dem.to_host()
    ref = oracle_edges(circ, noise)
    keys_ref = [ref.split_ids(ref.class_ids(c)) for c in range(ref.n_classes)]
    rng = np.random.default_rng(d)
    gP_ref = rng.normal(size=ref.n_classes)
    gW_ref = rng.normal(size=ref.n_classes) * 1e-3
    index = {k: i for i, k in enumerate(keys_ref)}
    keys_gpu = list(dem.edges(0, host).keys())
    order = np.array([index[k] for k in keys_gpu])
    g_gpu = drv.backward(torch.tensor(gP_ref[order], dtype=torch.float32, device="cuda"),
                         torch.tensor(gW_ref[order], dtype=torch.float32, device="cuda")).cpu().numpy()
    g_ref = ref.gradient(gP_ref.astype(np.float32).astype(np.float64),
                         gW_ref.astype(np.float32).astype(np.float64), circ.n_locations)
    floor = 1e-6 * np.abs(g_ref).max()
    err = np.abs(g_gpu - g_ref)
    bad = err > 1e-4 * np.abs(g_ref) + floor
    assert not bad.any(), f"{bad.sum()} locations off; worst {err.max():.3g}"


@pytest.mark.parametrize("staged", [False, True])
def test_result_to_host_matches_to_host(staged, monkeypatch):
    """gp_result_to_host (one device pass into host memory, or per-array
    copies) delivers the same arrays as reading the device tensors."""
    if staged:
        monkeypatch.setenv("GPDEM_STAGE_HOST_INPUTS", "1")
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    drv = Driver.for_circuits([circ])
    dem = drv.compile(circ, f32(circ.default_noise))
    ref = dem.to_host()
    out = {"det_offsets": np.zeros(dem.n_edges + 1, np.int32), "det_idx": np.zeros(dem.n_det_entries, np.int32),
           "obs_mask": np.zeros(dem.n_edges, np.uint64), "prob": np.zeros(dem.n_edges, np.float32),
           "logodds": torch.zeros(dem.n_edges, dtype=torch.float32, pin_memory=True)}
    dem.copy_to_host(out)
    assert np.array_equal(out["det_offsets"], ref["det_offsets"])
    assert np.array_equal(out["det_idx"], ref["det_idx"])
    assert np.array_equal(out["obs_mask"], ref["obs_mask"])
    assert np.array_equal(out["prob"], ref["prob"])
    assert np.array_equal(out["logodds"].numpy(), ref["logodds"])
    part = {"prob": np.zeros(dem.n_edges, np.float32)}
    dem.copy_to_host(part)
    assert np.array_equal(part["prob"], ref["prob"])


@pytest.mark.parametrize("level", ["L0", "L1", "L2"])
def test_z_check_detectors_only_parity(level):
    """The Z-basis memory experiment with its X-check detectors left out (the
    detector set paired with L0) against the oracle, at every level."""
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3), z_detectors_only=True)
    nz = f32(C.log_uniform_noise(circ.n_locations, seed=11))
    got = Driver.for_circuits([circ]).compile(circ, nz, level).edges()
    compare_edges(got, oracle_edges(circ, nz, level).edges(), f"z-only {level}")


def test_dem_text_round_trip_gpu():
    """A compiled model written as text and read back is the same model (the
    FP32 probabilities survive exactly)."""
    from paper_2604_16613_gb300.demtext import read_dem, write_dem
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    got = Driver.for_circuits([circ]).compile(circ, f32(circ.default_noise)).edges()
    back, n_det, n_obs = read_dem(write_dem(got, circ.n_detectors, circ.n_observables))
    assert (n_det, n_obs) == (circ.n_detectors, circ.n_observables)
    assert back == {k: p for k, (p, _) in got.items()}
