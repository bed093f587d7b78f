// lower.cu -- device-side lowering of flat circuit rows (Sec. 2.3.1: the
// realised circuit is lowered to a layered space-time structure before the
// backward wave runs).
//
// Four launches, no device-wide waits (grid-stride loops, grids capped by the
// SM count):
//   tile_count   per tile of 512 rows: counts of TICKs, measurements,
//                detectors and mechanisms (components at the chosen level)
//   tile_scan    one block: per-circuit scan of the tile counts, circuit
//                totals and batch offsets, capacity checks
//   tile_lower   per tile: exclusive row scan, validation of every row and
//                the scatters stage 1 reads (layer starts, record layers,
//                detector rows, observable rows, per-row auxiliary index,
//                per-mechanism location/kind/component)
//   layer_index  one block per TICK layer: checks that no qubit takes part
//                in two gates, decides for every noise row whether it acts
//                before or after the layer's gate on its qubit(s), and writes
//                the layer's qubit index: each qubit's gate as seen from the
//                qubit, and per qubit the lists of packed noise rows that
//                touch it after and before the gates (CSR, a two-qubit row
//                listed under both of its qubits)
#include <algorithm>

#include "common.cuh"

namespace gpdem {

namespace {

constexpr int kRowsPerThread = kRowTile / kLowerThreads;

__device__ __forceinline__ uint4 row_counts(uint4 op, uint32_t level) {
    uint4 c = make_uint4(0, 0, 0, 0);
    const uint32_t k = op.x;
    c.x = (k == K_TICK);
    c.y = is_measure(k);
    c.z = (k == K_DET);
    c.w = is_noise(k) ? n_comp(k, level) : 0u;
    return c;
}

__device__ __forceinline__ uint4 add4(uint4 a, uint4 b) {
    return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ uint4 sub4(uint4 a, uint4 b) {
    return make_uint4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

// Tiles, layer slots and scan chunks are visited by grid-stride loops whose
// trip counts depend only on blockIdx and the compile's sizes, so every
// block-wide barrier inside them (including status_set's) is reached by the
// whole block; grids are capped by the SM count, not by the driver's bounds.
__device__ __forceinline__ void tile_count_one(const Buffers &B, const Params &P, uint32_t t, uint4 *red) {
    const uint2 tile = B.tiles[t];
    const CircuitDev &C = B.circ[tile.x];
    const uint32_t r0 = tile.y + threadIdx.x * kRowsPerThread;
    const uint32_t r1 = min(r0 + kRowsPerThread, C.n_ops);
    uint4 acc = make_uint4(0, 0, 0, 0);
    for (uint32_t r = r0; r < r1; r++) acc = add4(acc, row_counts(C.ops[r], P.level));
    // block reduction of four counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xFFFFFFFFu, acc.x, o);
        acc.y += __shfl_down_sync(0xFFFFFFFFu, acc.y, o);
        acc.z += __shfl_down_sync(0xFFFFFFFFu, acc.z, o);
        acc.w += __shfl_down_sync(0xFFFFFFFFu, acc.w, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint4 s = make_uint4(0, 0, 0, 0);
        for (int w = 0; w < kLowerThreads / 32; w++) s = add4(s, red[w]);
        B.tile_sums[t] = s;
    }
    __syncthreads();           // red is reused by the block's next tile
}

__global__ void __launch_bounds__(kLowerThreads) tile_count_kernel(Buffers B) {
    const Params &P = *B.params;
    __shared__ uint4 red[kLowerThreads / 32];
    for (uint32_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x)
        tile_count_one(B, P, t, red);
}

// block-wide exclusive scans of a uint4 (four channels at once) and of a
// 64-bit value: warp shuffles, then one exchange of the warp totals
constexpr int kLowerWarps = kLowerThreads / 32;

__device__ __forceinline__ uint4 block_scan4(uint4 v, uint4 *warp_tot, uint4 &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(0xFFFFFFFFu, x.x, o), b = __shfl_up_sync(0xFFFFFFFFu, x.y, o);
        const uint32_t c = __shfl_up_sync(0xFFFFFFFFu, x.z, o), d = __shfl_up_sync(0xFFFFFFFFu, x.w, o);
        if (lane >= o) x = add4(x, make_uint4(a, b, c, d));
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    uint4 before = make_uint4(0, 0, 0, 0), all = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int w = 0; w < kLowerWarps; w++) {
        const uint4 t = warp_tot[w];
        if (w < warp) before = add4(before, t);
        all = add4(all, t);
    }
    __syncthreads();
    total = all;
    return add4(before, sub4(x, v));
}

__device__ __forceinline__ unsigned long long block_scan64(unsigned long long v, unsigned long long *warp_tot,
                                                           unsigned long long &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    unsigned long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kLowerWarps; w++) {
        const unsigned long long t = warp_tot[w];
        if (w < warp) before += t;
        all += t;
    }
    __syncthreads();
    total = all;
    return before + x - v;
}

// One block.  An exclusive scan of the tile sums over the whole batch gives
// each tile's offset (tiles of a circuit are contiguous, so a tile's offset
// within its circuit is its offset less that of the circuit's first tile):
// each thread sums a run of consecutive tiles, one block scan, then each
// thread writes its run.  Block scans over the circuits then give the batch
// offsets.
__global__ void __launch_bounds__(kLowerThreads) tile_scan_kernel(Buffers B) {
    const Params &P = *B.params;
    __shared__ uint4 warp_tot4[kLowerWarps];
    __shared__ unsigned long long warp_tot64[kLowerWarps];
    {
        const uint32_t n = P.n_tiles;
        const uint32_t per = (n + kLowerThreads - 1) / kLowerThreads;
        const uint32_t t0 = min(n, threadIdx.x * per), t1 = min(n, t0 + per);
        uint4 acc = make_uint4(0, 0, 0, 0);
        for (uint32_t t = t0; t < t1; t++) acc = add4(acc, B.tile_sums[t]);
        uint4 tot;
        uint4 run = block_scan4(acc, warp_tot4, tot);
        for (uint32_t t = t0; t < t1; t++) {
            B.tile_off[t] = run;
            run = add4(run, B.tile_sums[t]);
        }
    }
    __syncthreads();           // every tile offset written before the circuits read them
    // running batch offsets (64-bit before the capacity checks, so no wrap)
    unsigned long long carry_layer = 0, carry_meas = 0, carry_mech = 0, carry_qidx = 0;
    for (uint32_t base = 0; base < P.n_circuits; base += kLowerThreads) {
        const uint32_t b = base + threadIdx.x;
        uint32_t layers = 0, meas = 0, mech = 0, qblocks = 0;
        if (b < P.n_circuits) {
            CircuitDev &C = B.circ[b];
            uint4 run = make_uint4(0, 0, 0, 0);
            if (C.n_tiles) {
                const uint32_t f = C.tile_first, l = f + C.n_tiles - 1u;
                run = sub4(add4(B.tile_off[l], B.tile_sums[l]), B.tile_off[f]);
            }
            if (run.z != C.n_det) report(B.status, GP_ERR_INVALID, 1u, b, run.z);
            C.n_layers = run.x + 1;
            C.n_meas = run.y;
            C.n_mech = run.w;
            layers = C.n_layers + 1;       // row offsets incl. the end sentinel
            meas = run.y;
            mech = run.w;
            // index blocks for layers 0 .. n_layers, in 16-byte units
            const unsigned long long qb = (unsigned long long)layers * (layer_geo(C.n_qubits).bytes / 16u);
            qblocks = (uint32_t)min(qb, 0xFFFFFFFFull);
            B.obs_count[b] = 0;
            B.circ_edges[b] = 0;
        }
        uint4 tot;
        const uint4 off = block_scan4(make_uint4(layers, meas, mech, 0u), warp_tot4, tot);
        unsigned long long qtot;
        const unsigned long long qoff = block_scan64(qblocks, warp_tot64, qtot);
        if (b < P.n_circuits) {
            CircuitDev &C = B.circ[b];
            C.layer_base = (uint32_t)min(carry_layer + off.x, 0xFFFFFFFFull);
            C.meas_base = (uint32_t)min(carry_meas + off.y, 0xFFFFFFFFull);
            C.mech_base = (uint32_t)min(carry_mech + off.z, 0xFFFFFFFFull);
            const unsigned long long qo = carry_qidx + qoff;
            C.qidx_off = (uint32_t)min(qo, 0xFFFFFFFFull);
            if (qo + qblocks > P.qidx_cap16) report(B.status, GP_ERR_CAPACITY, 9u, b, (uint32_t)min(qo + qblocks, 0xFFFFFFFFull));
        }
        carry_layer += tot.x;
        carry_meas += tot.y;
        carry_mech += tot.z;
        carry_qidx += qtot;
    }
    if (threadIdx.x == 0) {
        if (carry_layer > P.max_layer_slots)
            report(B.status, GP_ERR_CAPACITY, 1u, (uint32_t)min(carry_layer, 0xFFFFFFFFull), P.max_layer_slots);
        if (carry_meas > P.max_meas || carry_meas > kMaxMeasurements)
            report(B.status, GP_ERR_CAPACITY, 2u, (uint32_t)min(carry_meas, 0xFFFFFFFFull), min(P.max_meas, kMaxMeasurements));
        if (carry_mech > P.max_mech)
            report(B.status, GP_ERR_CAPACITY, 3u, (uint32_t)min(carry_mech, 0xFFFFFFFFull), P.max_mech);
        B.status->n_mech = (uint32_t)min(carry_mech, 0xFFFFFFFFull);
    }
    // layer 0 starts at row 0; the sentinel after the last layer is n_ops
    __syncthreads();
    if (B.status->code == 0) {
        for (uint32_t b = threadIdx.x; b < P.n_circuits; b += kLowerThreads) {
            const CircuitDev &C = B.circ[b];
            B.layer_start[C.layer_base] = 0;
            B.layer_start[C.layer_base + C.n_layers] = C.n_ops;
        }
    }
}

__device__ __forceinline__ void tile_lower_one(const Buffers &B, const Params &P, uint32_t t, uint32_t *warp_tmp) {
    const uint2 tile = B.tiles[t];
    const uint32_t b = tile.x;
    const CircuitDev &C = B.circ[b];
    const uint32_t r0 = tile.y + threadIdx.x * kRowsPerThread;
    const uint32_t r1 = min(r0 + kRowsPerThread, C.n_ops);
    uint4 mine = make_uint4(0, 0, 0, 0);
    for (uint32_t r = r0; r < r1; r++) mine = add4(mine, row_counts(C.ops[r], P.level));
    uint32_t tot;
    const uint4 toff = sub4(B.tile_off[t], B.tile_off[C.tile_first]);
    uint4 run;
    run.x = block_exclusive_scan<kLowerThreads>(mine.x, warp_tmp, tot) + toff.x;
    run.y = block_exclusive_scan<kLowerThreads>(mine.y, warp_tmp, tot) + toff.y;
    run.z = block_exclusive_scan<kLowerThreads>(mine.z, warp_tmp, tot) + toff.z;
    run.w = block_exclusive_scan<kLowerThreads>(mine.w, warp_tmp, tot) + toff.w;
    for (uint32_t r = r0; r < r1; r++) {
        const uint4 op = C.ops[r];
        const uint32_t k = op.x;
        const uint32_t ticks = run.x, meas = run.y, dets = run.z, mech = run.w;
        uint32_t aux = 0;
        bool bad = false;
        switch (k) {
        case K_TICK:
            B.layer_start[C.layer_base + ticks + 1] = r + 1;
            break;
        case K_NOP:
            break;
        case K_R: case K_RX: case K_H: case K_S:
            bad = op.y >= C.n_qubits;
            break;
        case K_M: case K_MR: case K_MX: case K_MRX:
            bad = op.y >= C.n_qubits;
            aux = meas;
            if (!bad) B.meas_lq[C.meas_base + meas] = make_uint2(ticks, op.y | ((k == K_MX || k == K_MRX) ? 0x80000000u : 0u));
            break;
        case K_CX: case K_CZ:
            bad = op.y >= C.n_qubits || op.z >= C.n_qubits || op.y == op.z;
            break;
        case K_DET: case K_OBS: {
            bad = (unsigned long long)op.y + op.z > C.n_recs;
            if (!bad) {
                for (uint32_t i = 0; i < op.z; i++) {
                    const uint32_t lb = C.recs[op.y + i];
                    if (lb == 0 || lb > meas) { bad = true; break; }
                }
            }
            if (k == K_OBS && op.w >= C.n_obs) bad = true;
            aux = meas;
            if (!bad) {
                if (k == K_DET) B.det_row[C.det_base + dets] = r;
                else B.obs_rows[C.op_base + atomicAdd(&B.obs_count[b], 1u)] = r;
            }
            break;
        }
        case K_XERR: case K_ZERR: case K_DEP1: case K_DEP2:
            bad = op.y >= C.n_qubits || op.w >= C.n_loc ||
                  (k == K_DEP2 && (op.z >= C.n_qubits || op.y == op.z));
            aux = mech;
            if (!bad) {
                const uint32_t nc = n_comp(k, P.level);
                for (uint32_t c = 0; c < nc; c++)
                    B.mech_info[C.mech_base + mech + c] = (unsigned long long)(C.loc_base + op.w) |
                                                          ((unsigned long long)k << 32) |
                                                          ((unsigned long long)c << 40) |
                                                          ((unsigned long long)b << 48);
            }
            break;
        default:
            bad = true;
            break;
        }
        if (bad) report(B.status, GP_ERR_INVALID, 2u, b, r);
        B.aux[C.op_base + r] = aux;
        run = add4(run, row_counts(op, P.level));
    }
}

__global__ void __launch_bounds__(kLowerThreads) tile_lower_kernel(Buffers B) {
    const Params &P = *B.params;
    __shared__ uint32_t warp_tmp[kLowerThreads / 32];
    for (uint32_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x) {
        if (status_set(B.status)) return;      // the whole block, every iteration
        tile_lower_one(B, P, t, warp_tmp);
    }
}

// One block per layer slot.  Slots are numbered across the batch; circuit b
// owns slots [layer_base, layer_base + n_layers] (the last one is the end
// sentinel, which has no rows).
//
// Shared memory: gt[q] = row of q's gate in the layer; cnt[q] = q's list
// lengths, after-gate entries in the low half and before-gate entries in
// the high half (a layer has at most kMaxLayerRows rows, so neither half
// can carry into the other), later turned into fill positions.
__device__ __forceinline__ void layer_index_one(const Buffers &B, const Params &P, uint32_t g, uint32_t *lsm,
                                                uint32_t *warp_tmp) {
    // circuit owning slot g (circuits are laid out in slot order)
    uint32_t lo = 0, hi = P.n_circuits;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (B.circ[mid].layer_base <= g) lo = mid; else hi = mid;
    }
    const uint32_t b = lo;
    const CircuitDev &C = B.circ[b];
    if (g < C.layer_base || g > C.layer_base + C.n_layers) return;
    if (g == C.layer_base + C.n_layers) {
        // end sentinel: no rows, no before-gate noise
        if (threadIdx.x == 0) B.layer_seg[g] = make_uint4(C.n_ops, 0, 0, 0);
        return;
    }
    const uint32_t L = g - C.layer_base;
    const uint32_t nq = C.n_qubits;
    const uint32_t rs = B.layer_start[g], re = B.layer_start[g + 1];
    if (re - rs > kMaxLayerRows) {
        if (threadIdx.x == 0) report(B.status, GP_ERR_CAPACITY, 10u, b, L);
        return;
    }
    uint32_t *gt = lsm, *cnt = lsm + P.max_qubits;
    for (uint32_t q = threadIdx.x; q < nq; q += kPackThreads) { gt[q] = kNone; cnt[q] = 0u; }
    __syncthreads();
    for (uint32_t r = rs + threadIdx.x; r < re; r += kPackThreads) {
        const uint4 op = C.ops[r];
        if (!is_gate(op.x)) continue;
        bool dup = atomicExch(&gt[op.y], r) != kNone;
        if (is_gate2(op.x)) dup |= atomicExch(&gt[op.z], r) != kNone;
        if (dup) report(B.status, GP_ERR_INVALID, 4u, b, r);
    }
    __syncthreads();
    // side of a noise row: 0 after the gates of its qubit(s), 1 before;
    // 2 for rows that are not noise (or a two-qubit row split across sides)
    auto side = [&](uint32_t r, const uint4 &op) -> uint32_t {
        if (!is_noise(op.x)) return 2u;
        const uint32_t ga = gt[op.y];
        const bool bef = ga != kNone && ga > r;
        if (op.x == K_DEP2) {
            const uint32_t gb = gt[op.z];
            if ((gb != kNone && gb > r) != bef) {
                report(B.status, GP_ERR_INVALID, 3u, b, r);
                return 2u;
            }
        }
        return bef ? 1u : 0u;
    };
    for (uint32_t r = rs + threadIdx.x; r < re; r += kPackThreads) {
        const uint4 op = C.ops[r];
        const uint32_t sd = side(r, op);
        if (sd == 2u) continue;
        const uint32_t inc = sd ? 0x10000u : 1u;
        atomicAdd(&cnt[op.y], inc);
        if (op.x == K_DEP2) atomicAdd(&cnt[op.z], inc);
    }
    __syncthreads();
    // exclusive scan of the packed counts: each thread a contiguous run of
    // qubits, one block scan over the runs
    const uint32_t per = (nq + kPackThreads - 1) / kPackThreads;
    const uint32_t q0 = min(threadIdx.x * per, nq), q1 = min(q0 + per, nq);
    uint32_t local = 0;
    for (uint32_t q = q0; q < q1; q++) local += cnt[q];
    uint32_t tot;
    uint32_t run = block_exclusive_scan<kPackThreads>(local, warp_tmp, tot);
    const uint32_t n_after = tot & 0xFFFFu, n_before = tot >> 16;
    const LayerGeo geo = layer_geo(nq);
    unsigned char *blk = B.qidx + (size_t)C.qidx_off * 16u + (size_t)L * geo.bytes;
    uint16_t *boff = reinterpret_cast<uint16_t *>(blk);
    uint32_t *gate = reinterpret_cast<uint32_t *>(blk + 2u * geo.qb);
    uint16_t *aoff = reinterpret_cast<uint16_t *>(blk + 2u * geo.qb + 4u * geo.nq4);
    for (uint32_t q = q0; q < q1; q++) {
        const uint32_t c = cnt[q];
        aoff[q] = (uint16_t)(run & 0xFFFFu);
        boff[q] = (uint16_t)(run >> 16);
        cnt[q] = run;
        run += c;
    }
    if (threadIdx.x == 0) {
        aoff[nq] = (uint16_t)n_after;
        boff[nq] = (uint16_t)n_before;
        B.layer_seg[g] = make_uint4(rs, n_after, n_before, 0u);
    }
    __syncthreads();
    // each qubit's gate as seen from the qubit
    for (uint32_t q = threadIdx.x; q < geo.nq4; q += kPackThreads) {
        uint32_t v = GV_NONE;
        const uint32_t r = q < nq ? gt[q] : kNone;
        if (r != kNone) {
            const uint4 op = C.ops[r];
            if (op.x == K_CX) v = (op.y == q) ? (GV_CX_C << 28) | op.z : (GV_CX_T << 28) | op.y;
            else if (op.x == K_CZ) v = (op.y == q) ? (GV_CZ_A << 28) | op.z : (GV_CZ_B << 28) | op.y;
            else v = (op.x << 28) | (is_measure(op.x) ? B.aux[C.op_base + r] : 0u);
        }
        gate[q] = v;
    }
    // fill the lists: before-gate lists start at the layer's first slot,
    // after-gate lists end at its last
    uint2 *before = B.lists + 2ull * (C.op_base + rs);
    uint2 *after = B.lists + 2ull * (C.op_base + re) - n_after;
    for (uint32_t r = rs + threadIdx.x; r < re; r += kPackThreads) {
        const uint4 op = C.ops[r];
        if (!is_noise(op.x)) continue;
        const uint32_t ga = gt[op.y];
        const bool bef = ga != kNone && ga > r;
        if (op.x == K_DEP2) {
            const uint32_t gb = gt[op.z];
            if ((gb != kNone && gb > r) != bef) continue;     // reported above
        }
        // the second qubit field is meaningful (and validated) only for
        // two-qubit noise
        const uint2 row = pack_row(op.x, op.y, op.x == K_DEP2 ? op.z : 0u, B.aux[C.op_base + r]);
        const uint32_t inc = bef ? 0x10000u : 1u;
        const uint32_t pa = atomicAdd(&cnt[op.y], inc);
        if (bef) before[pa >> 16] = row; else after[pa & 0xFFFFu] = row;
        if (op.x == K_DEP2) {
            const uint32_t pb = atomicAdd(&cnt[op.z], inc);
            if (bef) before[pb >> 16] = row; else after[pb & 0xFFFFu] = row;
        }
    }
}

__global__ void __launch_bounds__(kPackThreads) layer_index_kernel(Buffers B) {
    extern __shared__ uint32_t lsm[];
    __shared__ uint32_t warp_tmp[kPackThreads / 32];
    const Params &P = *B.params;
    // slots of the whole batch: those of the last circuit end it
    const CircuitDev &last = B.circ[P.n_circuits - 1u];
    const uint32_t n_slots = last.layer_base + last.n_layers + 1u;
    for (uint32_t g = blockIdx.x; g < n_slots; g += gridDim.x) {
        // the whole block, every iteration: the barriers also separate one
        // slot's use of the shared arrays from the next one's
        if (status_set(B.status)) return;
        layer_index_one(B, P, g, lsm, warp_tmp);
    }
}

// Host arrays gathered into device arenas by the GPU itself, through the
// coherent host memory of a Grace-Blackwell node (pageable memory is
// addressable from the device there): block (x, j) copies its share of job
// j, 16 bytes per thread when both ends are 16-byte aligned, else 4.
__global__ void __launch_bounds__(256) gather_host_kernel(const CopyJob *jobs, uint32_t n_jobs) {
    const uint32_t j = blockIdx.y;
    if (j >= n_jobs) return;
    const CopyJob job = jobs[j];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool wide = ((reinterpret_cast<uintptr_t>(job.src) | reinterpret_cast<uintptr_t>(job.dst)) & 15u) == 0u;
    uint64_t done = 0;
    if (wide) {
        // four independent 16-byte loads in flight per thread (the link's
        // latency, not its bandwidth, limits one load at a time)
        const uint64_t n16 = job.bytes / 16u;
        const uint4 *__restrict__ src = static_cast<const uint4 *>(job.src);
        uint4 *__restrict__ dst = static_cast<uint4 *>(job.dst);
        uint64_t i = tid;
        for (; i + 3u * stride < n16; i += 4u * stride) {
            const uint4 a = src[i], b = src[i + stride], c = src[i + 2u * stride], d = src[i + 3u * stride];
            dst[i] = a;
            dst[i + stride] = b;
            dst[i + 2u * stride] = c;
            dst[i + 3u * stride] = d;
        }
        for (; i < n16; i += stride) dst[i] = src[i];
        done = n16 * 16u;
    }
    const uint64_t n4 = (job.bytes - done) / 4u;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(static_cast<const unsigned char *>(job.src) + done);
    uint32_t *dst = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(job.dst) + done);
    for (uint64_t i = tid; i < n4; i += stride) dst[i] = src[i];
}

}  // namespace

void launch_gather_host(const CopyJob *jobs, uint32_t n_jobs, uint64_t max_bytes, uint32_t n_sms, cudaStream_t s) {
    if (!n_jobs) return;
    // enough blocks that the largest job is spread over the whole GPU (each
    // thread moves four 16-byte words per round)
    const uint64_t per_block = 256ull * 16u * 4u;
    uint32_t gx = (uint32_t)std::min<uint64_t>((max_bytes + per_block - 1) / per_block, 8ull * n_sms);
    if (gx == 0) gx = 1;
    gather_host_kernel<<<dim3(gx, n_jobs), 256, 0, s>>>(jobs, n_jobs);
}

void launch_lowering(const Buffers &b, uint32_t n_tiles, uint32_t layer_slots, uint32_t max_qubits, uint32_t n_sms,
                     cudaStream_t s, uint32_t *launches) {
    // grid-stride kernels: at most eight blocks per SM, fewer when the
    // bounds allow fewer tiles or layer slots
    const uint32_t cap = 8u * std::max(n_sms, 1u);
    const uint32_t grid = std::max(1u, std::min(n_tiles, cap));
    const uint32_t grid_l = std::max(1u, std::min(layer_slots, cap));
    tile_count_kernel<<<grid, kLowerThreads, 0, s>>>(b);
    tile_scan_kernel<<<1, kLowerThreads, 0, s>>>(b);
    tile_lower_kernel<<<grid, kLowerThreads, 0, s>>>(b);
    layer_index_kernel<<<grid_l, kPackThreads, 2u * max_qubits * sizeof(uint32_t), s>>>(b);
    *launches += 4;
}

cudaError_t lowering_setup(uint32_t max_qubits) {
    return cudaFuncSetAttribute(layer_index_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2u * max_qubits * sizeof(uint32_t)));
}

}  // namespace gpdem
