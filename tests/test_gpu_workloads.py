"""GPU parity on the other workloads of the paper: bivariate bicycle memory
(forward and adjoint), adaptive [[4,2,2]]-concatenated branches compiled as
one batch, the autotuner and the autograd function."""
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from paper_2604_16613_gb300 import circuits as C
from paper_2604_16613_gb300.autotune import autotune
from paper_2604_16613_gb300.dem import Bounds, DemFunction, DeviceCircuit, Driver
from paper_2604_16613_gb300.native import GpError

from parity import compare_arrays, compare_edges, oracle_arrays, oracle_edges

pytestmark = pytest.mark.gpu


def f32(x):
    return np.asarray(x, dtype=np.float32)


@pytest.fixture(scope="module")
def bb():
    circ = C.bb_memory(12, C.NoiseModel.uniform(1e-3), seed=3)
    noise = f32(circ.default_noise)
    return circ, noise


def test_bb_forward_parity(bb):
    circ, noise = bb
    drv = Driver.for_circuits([circ])
    for level in ("L0", "L2"):
        dem = drv.compile(DeviceCircuit(circ), torch.tensor(noise, device="cuda"), level)
        compare_edges(dem.edges(), oracle_edges(circ, noise, level).edges(), f"bb/{level}")


def _grad_setup(circ, noise, seed):
    drv = Driver.for_circuits([circ])
    dem = drv.compile(DeviceCircuit(circ), torch.tensor(noise, device="cuda"))
    keys = list(dem.edges().keys())
    ref = oracle_edges(circ, noise)
    order = [ref.split_ids(ref.class_ids(c)) for c in range(ref.n_classes)]
    rng = np.random.default_rng(seed)
    gw = {k: float(v) for k, v in zip(order, rng.normal(size=len(order)).astype(np.float32))}
    return drv, dem, keys, ref, order, gw


def test_bb_adjoint_log_odds(bb):
    """Config 3: gradient of sum_e gW_e w_e with respect to every location,
    FP32 on the GPU against the FP64 oracle's analytic gradient (all
    locations) and against FP64 central differences (h = 1e-7) of the oracle
    on 64 seeded locations."""
    circ, noise = bb
    drv, dem, keys, ref, order, gw = _grad_setup(circ, noise, 13)
    g_gpu = drv.backward(None, torch.tensor([gw[k] for k in keys], dtype=torch.float32,
                                            device="cuda")).cpu().numpy().astype(np.float64)
    g_ref = ref.gradient(np.zeros(ref.n_classes), np.array([gw[k] for k in order]), circ.n_locations)
    floor = 1e-6 * np.abs(g_ref).max()
    err = np.abs(g_gpu - g_ref)
    assert np.all(err <= 1e-4 * np.abs(g_ref) + floor), f"worst {err.max():.3g}"
    n64 = noise.astype(np.float64)
    h = 1e-7
    rng = np.random.default_rng(21)
    for loc in rng.choice(circ.n_locations, size=64, replace=False):
        up, dn = n64.copy(), n64.copy()
        up[loc] += h
        dn[loc] -= h
        lu = sum(gw[k] * w for k, (P, w) in oracle.analyze_circuit(circ, up).edges().items())
        ld = sum(gw[k] * w for k, (P, w) in oracle.analyze_circuit(circ, dn).edges().items())
        fd = (lu - ld) / (2 * h)
        assert g_gpu[loc] == pytest.approx(fd, rel=1e-3, abs=1e-5 * np.abs(g_ref).max())


def test_dem_function_autograd():
    circ = C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))
    noise = torch.tensor(f32(C.log_uniform_noise(circ.n_locations, seed=7)), device="cuda", requires_grad=True)
    drv = Driver.for_circuits([circ])
    dc = DeviceCircuit(circ)
    prob, logodds = DemFunction.apply(noise, drv, dc, "L2")
    rng = np.random.default_rng(1)
    a = torch.tensor(rng.normal(size=prob.numel()), dtype=torch.float32, device="cuda")
    b = torch.tensor(rng.normal(size=prob.numel()) * 1e-3, dtype=torch.float32, device="cuda")
    loss = (a * prob).sum() + (b * logodds).sum()
    loss.backward()
    drv.compile(dc, noise.detach())
    g = drv.backward(a, b)
    assert torch.equal(noise.grad, g)


def test_concatenated_branches_one_batch():
    lay4 = C.ConcatenatedLayout(4)
    branches = [C.concatenated_adaptive_branch(4, n, seed=s, noise=C.NoiseModel.uniform(1e-3), layout=lay4)
                for s, n in enumerate([3, 5, 4, 6, 2, 7])]
    branches += [C.concatenated_adaptive_branch(10, 3, seed=99, noise=C.NoiseModel.uniform(1e-3))]
    noises = [f32(b.default_noise) for b in branches]
    drv = Driver.for_circuits(branches)
    dem = drv.compile([DeviceCircuit(b) for b in branches], torch.tensor(np.concatenate(noises), device="cuda"))
    host = dem.to_host()
    for i, (b, nz) in enumerate(zip(branches, noises)):
        compare_arrays(host, i, oracle_edges(b, nz), f"branch {i}")


def test_adaptive_256_branch_batch_parity():
    """The benchmark's batched workload at full size: 256 realised branches of
    the adaptive [[4,2,2]]-concatenated surface code (outer distance 10,
    10-30 cycles each, seed 4; Secs. 5.1-5.2), compiled as one batch with the
    benchmark's bounds and autotuned launch shape.  Every branch is compared
    with the oracle: same number of hyperedges, identical masks, P and w
    within tolerance.  The oracle runs first, in a spawn process pool."""
    branches = C.adaptive_branches(n=256, d=10, lo=10, hi=30, seed=4)
    noises = [f32(b.default_noise) for b in branches]
    tasks = [(b.ops, b.recs, b.n_qubits, nz.astype(np.float64), "L2") for b, nz in zip(branches, noises)]
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        refs = pool.map(oracle_arrays, tasks, chunksize=4)
    nz = torch.tensor(np.concatenate(noises), device="cuda")
    dcs = [DeviceCircuit(b) for b in branches]
    bd = Bounds.for_circuits(branches)
    bd.max_det_entries = 8 * bd.max_mechanisms
    drv = Driver(bd)
    autotune(drv, dcs, nz, repeats=2)
    dem = drv.compile(dcs, nz)
    assert dem.n_circuits == 256
    host = dem.to_host()
    for i, ref in enumerate(refs):
        compare_arrays(host, i, ref, f"branch {i}")


def test_autotune_does_not_change_results():
    circs = [C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3)),
             C.concatenated_adaptive_branch(4, 4, seed=3, noise=C.NoiseModel.uniform(1e-3))]
    noise = torch.tensor(f32(np.concatenate([c.default_noise for c in circs])), device="cuda")
    dcs = [DeviceCircuit(c) for c in circs]
    drv = Driver.for_circuits(circs)
    base = drv.compile(dcs, noise).to_host()
    best = autotune(drv, dcs, noise, repeats=2)
    assert best["ms"] > 0
    tuned = drv.compile(dcs, noise).to_host()
    for k in base:
        assert np.array_equal(base[k], tuned[k]), k
    for shape in [(256, 1, 128, 16), (1024, 0, 512, 4)]:
        drv.set_tuning(*shape)
        other = drv.compile(dcs, noise).to_host()
        for k in base:
            assert np.array_equal(base[k], other[k]), (shape, k)


def test_observable_split_does_not_change_results():
    """The observables of a circuit may be walked as 1 to 8 word columns,
    each in 1 to 3 time segments, and stage 1 may deal wide steps out lane by
    lane: the compile is the same bit for bit, and equal to the oracle.  The [[144,12,12]] code has 12 logicals (uneven
    splits at 5 and 8 columns); the random circuits have one or two."""
    circs = [C.bb_memory(3, C.NoiseModel.uniform(1e-3), seed=3),
             C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3))]
    circs += [C.random_circuit(s) for s in range(6)]
    noises = [f32(c.default_noise) for c in circs]
    noise = torch.tensor(np.concatenate(noises), device="cuda")
    dcs = [DeviceCircuit(c) for c in circs]
    drv = Driver.for_circuits(circs)
    base = drv.compile(dcs, noise).to_host()
    for i, (c, nz) in enumerate(zip(circs, noises)):
        compare_arrays(base, i, oracle_arrays((c.ops, c.recs, c.n_qubits, nz.astype(np.float64), "L2")), f"circuit {i}")
    for ow, osg, wide in [(1, 3, 0), (2, 1, 1), (5, 2, 0), (8, 3, 1), (3, 1, 0), (4, 3, 1)]:
        drv.set_tuning(obs_words=ow, obs_segments=osg, stage1_wide_emit=wide)
        got = drv.compile(dcs, noise).to_host()
        for k in base:
            assert np.array_equal(base[k], got[k]), (ow, osg, wide, k)
    for bad in [dict(obs_words=0), dict(obs_words=9), dict(obs_segments=0), dict(obs_segments=4),
                dict(stage1_wide_emit=2)]:
        with pytest.raises(GpError):
            drv.set_tuning(**bad)


def test_block_wide_walk_equals_role_split_walk():
    """Stage 1 has two walks: the role-split one (a walker warp and emitter
    warps, used when its per-qubit tables fit in shared memory) and the
    block-wide one (used above that, here forced by bounds for 4096 qubits).
    Both give the same compile bit for bit, at every launch shape."""
    circs = [C.rotated_surface_code_memory(7, 7, C.NoiseModel.uniform(1e-3)),
             C.concatenated_adaptive_branch(4, 5, seed=7, noise=C.NoiseModel.uniform(1e-3)),
             C.bb_memory(3, C.NoiseModel.uniform(1e-3), seed=3)]
    noise = torch.tensor(f32(np.concatenate([c.default_noise for c in circs])), device="cuda")
    dcs = [DeviceCircuit(c) for c in circs]
    split = Driver.for_circuits(circs).compile(dcs, noise).to_host()
    bd = Bounds.for_circuits(circs)
    bd.max_qubits = 4096
    wide = Driver(bd)
    for shape in [(512, 1, 256, 16), (256, 2, 256, 16, 1, 3, 1), (128, 1, 256, 16, 8, 2)]:
        wide.set_tuning(*shape)
        got = wide.compile(dcs, noise).to_host()
        for k in split:
            assert np.array_equal(split[k], got[k]), (shape, k)


def test_host_inputs_gathered_equal_staged(monkeypatch):
    """Host arrays reach the device either gathered by the device itself
    (coherent host memory) or through pinned staging copies; both give the
    same compile bit for bit, for one circuit and for a batch."""
    circs = [C.rotated_surface_code_memory(5, 5, C.NoiseModel.uniform(1e-3)),
             C.concatenated_adaptive_branch(4, 4, seed=3, noise=C.NoiseModel.uniform(1e-3))]
    noises = [f32(c.default_noise) for c in circs]
    gathered = Driver.for_circuits(circs)
    monkeypatch.setenv("GPDEM_STAGE_HOST_INPUTS", "1")
    staged = Driver.for_circuits(circs)
    for c, nz in zip(circs, noises):
        a, b = gathered.compile(c, nz).to_host(), staged.compile(c, nz).to_host()
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    a = gathered.compile(circs, np.concatenate(noises)).to_host()
    b = staged.compile(circs, np.concatenate(noises)).to_host()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_noise_recalibration_recovers_channel_groups():
    """Noise recalibration with the adjoint: detection events sampled with
    known per-channel parameters (two-qubit depolarising, one-qubit
    depolarising, bit flips at resets and measurements) are fitted from a
    uniform start; the fit recovers every group's parameter."""
    from paper_2604_16613_gb300.calibrate import fit_groups, location_kinds
    from paper_2604_16613_gb300.sampler import sample
    circ = C.rotated_surface_code_memory(5, 3, C.NoiseModel.uniform(1e-3))
    kinds = location_kinds(circ)
    groups = np.select([kinds == C.DEPOLARIZE2, kinds == C.DEPOLARIZE1], [0, 1], 2)
    true = np.array([3e-3, 1e-3, 2e-3])
    det, _ = sample(circ, true[groups], 1 << 17, seed=3)
    drv = Driver.for_circuits([circ])
    fitted, history = fit_groups(drv, circ, groups, det, p0=[1e-3, 1e-3, 1e-3], steps=100)
    assert min(history) < 0.01 * history[0]
    assert np.all(np.abs(fitted / true - 1.0) < 0.05), fitted
