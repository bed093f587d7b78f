// stage1.cu -- error-equivalence-class generation (Sec. 3.1).
//
// The straight-line program of Eq. slp is linear over GF(2), so every 64
// detectors (one "word column") can be propagated on their own.  A thread
// block takes word columns from a work queue and keeps, in shared memory, two
// 64-bit bit-planes per qubit of the column:
//   xs[q] bit j = detector j flips under an X error on q at the current time
//   zs[q] bit j = the same for a Z error.
// It walks the TICK layers backward from the latest measurement of the
// column's detectors (Eq. init-slp seeds the bits there) and stops once every
// plane is zero and no earlier measurement of the column remains, so a column
// only pays for the layers its detecting regions cover.
//
// Layers arrive pre-packed by the lowering (gates | noise after the gates |
// noise before the gates, 8 bytes a row).  Each layer is staged into shared
// memory by a 1-D bulk copy (TMA) issued one layer ahead into a
// double buffer and tracked by an mbarrier; layers larger than a buffer are
// read from global memory directly.  Per layer L two barrier-separated
// phases run:
//   A  mask words of the noise rows acting after the gates of L and before
//      the gates of L+1 (the planes hold the state between the two), and the
//      termination test;
//   B  the gates of L undone backward: H swaps the planes, S: x ^= z,
//      CX(c,t): x_c ^= x_t and z_t ^= z_c, CZ(a,b): x_a ^= z_b and
//      x_b ^= z_a; measurements XOR in the column's detector bits; resets
//      clear the planes after checking that the detectors commute with them.
// A component's mask word is the XOR of the planes its Pauli names (Y = X xor
// Z, two-qubit terms combine both qubits: Sec. 2.3.4).  Non-zero words become
// 16-byte records {mechanism, column, word}; they are staged in shared memory
// during phase A and copied to the block's chunk of the global record pool
// during phase B, so the walk never waits on a global atomic.
#include "common.cuh"

namespace gpdem {

namespace {

constexpr int kRowBufs = 3;         // layer buffers: L+1 (held), L, L-1 .. L-2 in flight
constexpr int kSegCache = 256;      // layer segments cached in shared memory
constexpr int kActive = 2 * kRowBuf; // noise rows examined per emission piece

struct Smem {
    unsigned long long *xs, *zs;
    unsigned long long *ent_w;
    unsigned long long *st_word;    // staged records: word
    uint4 *segc;
    uint2 *rows[kRowBufs];
    uint32_t *ent_m;
    uint32_t *st_mech;              // staged records: mechanism
    uint16_t *act;                  // active noise rows of the current piece
};

__device__ __forceinline__ Smem carve(unsigned char *base, uint32_t maxq) {
    Smem s;
    s.xs = reinterpret_cast<unsigned long long *>(base);
    s.zs = s.xs + maxq;
    s.ent_w = s.zs + maxq;
    s.st_word = s.ent_w + kMaxEntries;
    s.segc = reinterpret_cast<uint4 *>(s.st_word + kStageRecs);
    uint2 *rw = reinterpret_cast<uint2 *>(s.segc + kSegCache);
    for (int i = 0; i < kRowBufs; i++) s.rows[i] = rw + i * (kRowBuf + 2);
    s.ent_m = reinterpret_cast<uint32_t *>(rw + kRowBufs * (kRowBuf + 2));
    s.st_mech = s.ent_m + kMaxEntries;
    s.act = reinterpret_cast<uint16_t *>(s.st_mech + kStageRecs);
    return s;
}

// XOR of the entry words recorded for measurement m (entries sorted by m)
__device__ __forceinline__ unsigned long long meas_word(const Smem &s, uint32_t n_ent, uint32_t m,
                                                        uint32_t m_lo, uint32_t m_hi) {
    if (m < m_lo || m > m_hi) return 0ull;
    uint32_t lo = 0, hi = n_ent;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.ent_m[mid] < m) lo = mid + 1; else hi = mid;
    }
    unsigned long long w = 0ull;
    for (uint32_t i = lo; i < n_ent && s.ent_m[i] == m; i++) w ^= s.ent_w[i];
    return w;
}

// rows of one layer: a base pointer (shared or global) and segment bounds
struct LayerView {
    const uint2 *rows;      // rows[0] is the layer's first packed row
    uint32_t g, a, b;       // ends of the gate, after-noise, before-noise segments
};

struct Shared {
    unsigned long long mbar[kRowBufs];
    uint32_t cnt[2];        // staged records per epoch parity (one data buffer:
                            // an epoch's records are copied out before the
                            // next epoch stages any)
    uint32_t chunk_pos, chunk_end;
    uint32_t item, bail, nent, lmax, lmin, tmo;
    uint32_t n_act;         // active rows listed for the current piece
    uint32_t next_chunk;    // record chunk requested ahead (kNone: none)
};

// The noise rows of one emission step are rows [g, a) of layer L (after its
// gates) followed by rows [a', b') of layer L+1 (before its gates), indexed
// 0 .. nA + nB - 1.
__device__ __forceinline__ uint2 emission_row(const LayerView &cur, const LayerView &nxt, uint32_t nA, uint32_t i) {
    return i < nA ? cur.rows[cur.g + i] : nxt.rows[nxt.a + (i - nA)];
}

// A1: list the rows of [p0, p1) whose planes are not all zero (warp-aggregated
// appends to the shared list).
template <int NT>
__device__ __forceinline__ void list_active(const Smem &s, Shared &sh, const LayerView &cur, const LayerView &nxt,
                                            uint32_t nA, uint32_t p0, uint32_t p1) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t base = p0; base < p1; base += NT) {
        const uint32_t i = base + threadIdx.x;
        bool active = false;
        if (i < p1) {
            const uint2 r = emission_row(cur, nxt, nA, i);
            const uint32_t a = row_a(r);
            unsigned long long v = s.xs[a] | s.zs[a];
            if (row_kind(r) == K_DEP2) {
                const uint32_t bq = row_b(r);
                v |= s.xs[bq] | s.zs[bq];
            }
            active = v != 0ull;
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, active);
        if (m == 0u) continue;
        uint32_t wbase = 0;
        if (lane == 0u) wbase = atomicAdd(&sh.n_act, (uint32_t)__popc(m));
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
        if (active) s.act[wbase + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(i - p0);
    }
}

// A2: every half-warp takes one listed row and evaluates its Pauli
// components one per lane; non-zero words are staged with one reservation per
// warp (spilling straight to the pool if the stage is full).
template <int NT>
__device__ __forceinline__ void emit_active(const Buffers &B, const Smem &s, Shared &sh, const CircuitDev &C,
                                            const LayerView &cur, const LayerView &nxt, uint32_t nA, uint32_t p0,
                                            uint32_t n_act, uint32_t col_tag, uint32_t level, uint32_t sb,
                                            uint32_t rec_cap) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t c = lane & 15u;
    const uint32_t mech_base = C.mech_base;
    for (uint32_t base = 2u * warp; base < n_act; base += 2u * (NT / 32)) {
        const uint32_t idx = base + (lane >> 4);
        unsigned long long w = 0ull;
        uint32_t mech = 0;
        if (idx < n_act) {
            const uint2 r = emission_row(cur, nxt, nA, p0 + s.act[idx]);
            const uint32_t kind = row_kind(r);
            if (c < n_comp(kind, level)) {
                const uint32_t code = comp_planes(kind, c);
                const uint32_t a = row_a(r), bq = row_b(r);
                if (code & 1u) w ^= s.xs[a];
                if (code & 2u) w ^= s.zs[a];
                if (code & 4u) w ^= s.xs[bq];
                if (code & 8u) w ^= s.zs[bq];
                mech = mech_base + r.y + c;
            }
        }
        const unsigned m = __ballot_sync(0xFFFFFFFFu, w != 0ull);
        if (m == 0u) continue;
        uint32_t wbase = 0;
        if (lane == 0u) wbase = atomicAdd(&sh.cnt[sb], (uint32_t)__popc(m));
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
        if (w != 0ull) {
            const uint32_t pos = wbase + __popc(m & ((1u << lane) - 1u));
            if (pos < (uint32_t)kStageRecs) {
                s.st_mech[pos] = mech;
                s.st_word[pos] = w;
            } else {
                const uint32_t g = atomicAdd(&B.status->rec_count, 1u);
                if (g < rec_cap) {
                    B.records[g] = make_uint4(mech, col_tag, (uint32_t)w, (uint32_t)(w >> 32));
                    atomicAdd(&B.mech_cnt[mech], 1u);
                } else {
                    report(B.status, GP_ERR_CAPACITY, 8u, g, rec_cap);
                }
            }
        }
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) stage1_kernel(Buffers B, uint32_t maxq) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Smem s = carve(smem_raw, maxq);
    __shared__ Shared sh;
    const Params &P = *B.params;
    const uint32_t level = P.level, rec_cap = P.rec_cap;
    const uint4 *layer_seg = B.layer_seg;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kRowBufs; i++) mbar_init(&sh.mbar[i], 1);
        fence_mbar_init();
        sh.cnt[0] = sh.cnt[1] = 0;
        sh.chunk_pos = sh.chunk_end = 0;
        sh.tmo = 0;
        sh.next_chunk = kNone;
        sh.n_act = 0;
    }
    __syncthreads();
    uint32_t phase_bits = 0u;         // mbarrier parity per row buffer (bit i)
    uint32_t pend_bits = 0u;          // copies issued and not yet waited for
    uint32_t epoch = 0;               // emission epochs alternate staging buffers
    bool timed_out = false;

    // thread 0, at the start of every phase A: retire the previous epoch's
    // staged records (copied during the last phase B) and make sure the
    // block's chunk can take a full staging buffer
    auto housekeeping = [&](uint32_t ep) {
        if (threadIdx.x != 0) return;
        if (ep > 0) {
            const uint32_t pb = (ep - 1u) & 1u;
            sh.chunk_pos += min(sh.cnt[pb], (uint32_t)kStageRecs);
            sh.cnt[pb] = 0;
        }
        const uint32_t room = sh.chunk_end - sh.chunk_pos;
        // ask for the next chunk while two stages still fit, so the atomic's
        // latency is hidden behind later layers
        if (room < 3u * (uint32_t)kStageRecs && sh.next_chunk == kNone)
            sh.next_chunk = atomicAdd(&B.status->rec_count, kChunkRecs);
        if (room < (uint32_t)kStageRecs) {
            const uint32_t base = sh.next_chunk;
            sh.next_chunk = kNone;
            if (base == kNone || base + kChunkRecs > rec_cap || base + kChunkRecs < base) {
                report(B.status, GP_ERR_CAPACITY, 8u, base, rec_cap);
                sh.chunk_pos = sh.chunk_end = 0;   // nothing is flushed below
            } else {
                sh.chunk_pos = base;
                sh.chunk_end = base + kChunkRecs;
            }
        }
    };
    // all threads, during phase B: copy epoch ep's staged records to the chunk
    auto flush = [&](uint32_t ep, uint32_t col_tag) {
        const uint32_t sb = ep & 1u;
        const uint32_t n = min(sh.cnt[sb], (uint32_t)kStageRecs);
        if (sh.chunk_end - sh.chunk_pos < n) return;    // capacity already reported
        for (uint32_t i = threadIdx.x; i < n; i += NT) {
            const unsigned long long w = s.st_word[i];
            const uint32_t mech = s.st_mech[i];
            B.records[sh.chunk_pos + i] = make_uint4(mech, col_tag, (uint32_t)w, (uint32_t)(w >> 32));
            atomicAdd(&B.mech_cnt[mech], 1u);
        }
    };

    for (;;) {
        if (threadIdx.x == 0) {
            sh.item = atomicAdd(&B.status->queue_head, 1u);
            sh.bail = (*(volatile uint32_t *)&B.status->code) != 0u;
            sh.nent = 0;
            sh.lmax = 0;
            sh.lmin = 0xFFFFFFFFu;
        }
        __syncthreads();
        const uint32_t item = sh.item;
        if (item >= P.n_items || sh.bail || timed_out) break;
        const uint32_t gcol = B.items[item];
        const uint32_t b = B.col_circ[gcol];
        const CircuitDev &C = B.circ[b];
        const uint32_t local = gcol - C.col_base;
        const bool is_obs = (C.n_obs > 0u) && (local == C.n_cols - 1u);
        const uint32_t col_tag = gcol | (is_obs ? kObsColFlag : 0u);
        const uint32_t nq = C.n_qubits;

        for (uint32_t q = threadIdx.x; q < nq; q += NT) {
            s.xs[q] = 0ull;
            s.zs[q] = 0ull;
        }
        // (measurement, word) entries of this column (Eq. init-slp)
        if (!is_obs) {
            const uint32_t j0 = local * 64u, j1 = min(j0 + 64u, C.n_det);
            for (uint32_t j = j0 + threadIdx.x; j < j1; j += NT) {
                const uint32_t row = B.det_row[C.det_base + j];
                const uint4 op = C.ops[row];
                const uint32_t mb = B.aux[C.op_base + row];
                for (uint32_t i = 0; i < op.z; i++) {
                    const uint32_t e = atomicAdd(&sh.nent, 1u);
                    if (e < (uint32_t)kMaxEntries) {
                        s.ent_m[e] = mb - C.recs[op.y + i];
                        s.ent_w[e] = 1ull << (j & 63u);
                    }
                }
            }
        } else {
            const uint32_t n_rows = B.obs_count[b];
            for (uint32_t i0 = threadIdx.x; i0 < n_rows; i0 += NT) {
                const uint32_t row = B.obs_rows[C.op_base + i0];
                const uint4 op = C.ops[row];
                const uint32_t mb = B.aux[C.op_base + row];
                for (uint32_t i = 0; i < op.z; i++) {
                    const uint32_t e = atomicAdd(&sh.nent, 1u);
                    if (e < (uint32_t)kMaxEntries) {
                        s.ent_m[e] = mb - C.recs[op.y + i];
                        s.ent_w[e] = 1ull << op.w;
                    }
                }
            }
        }
        __syncthreads();
        const uint32_t n_ent = sh.nent;
        if (n_ent > (uint32_t)kMaxEntries) {
            if (threadIdx.x == 0) report(B.status, GP_ERR_CAPACITY, 5u, gcol, n_ent);
            __syncthreads();
            continue;
        }
        if (n_ent == 0u) { __syncthreads(); continue; }
        // bitonic sort of the entries by measurement index
        uint32_t npow = 1;
        while (npow < n_ent) npow <<= 1;
        for (uint32_t i = n_ent + threadIdx.x; i < npow; i += NT) { s.ent_m[i] = 0xFFFFFFFFu; s.ent_w[i] = 0ull; }
        __syncthreads();
        for (uint32_t k2 = 2; k2 <= npow; k2 <<= 1) {
            for (uint32_t j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                for (uint32_t i = threadIdx.x; i < npow; i += NT) {
                    const uint32_t ixj = i ^ j2;
                    if (ixj > i) {
                        const bool asc = (i & k2) == 0u;
                        const uint32_t mi = s.ent_m[i], mj = s.ent_m[ixj];
                        if ((mi > mj) == asc) {
                            s.ent_m[i] = mj; s.ent_m[ixj] = mi;
                            const unsigned long long wi = s.ent_w[i];
                            s.ent_w[i] = s.ent_w[ixj]; s.ent_w[ixj] = wi;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < n_ent; i += NT) {
            const uint32_t L = B.meas_layer[C.meas_base + s.ent_m[i]];
            atomicMax(&sh.lmax, L);
            atomicMin(&sh.lmin, L);
        }
        __syncthreads();
        const uint32_t lmax = sh.lmax, lmin = sh.lmin;
        const uint32_t m_lo = s.ent_m[0], m_hi = s.ent_m[n_ent - 1];
        const uint4 *seg_g = layer_seg + C.layer_base;
        const uint2 *packed = B.packed + C.op_base;
        // the column's layer segments, cached once
        const uint32_t n_cache = min(lmax + 1u, (uint32_t)kSegCache);
        for (uint32_t i = threadIdx.x; i < n_cache; i += NT) s.segc[i] = seg_g[i];
        __syncthreads();
        auto segL = [&](uint32_t L) -> uint4 { return L < (uint32_t)kSegCache ? s.segc[L] : seg_g[L]; };
        auto staged = [&](const uint4 &sg) -> bool {
            const uint32_t n = sg.w - sg.x;
            return n != 0u && n <= (uint32_t)kRowBuf;
        };
        auto row_delta = [&](const uint4 &sg) -> uint32_t {
            return (uint32_t)((reinterpret_cast<uintptr_t>(packed + sg.x) & 15u) >> 3);
        };
        // stage layer L into buffer L % 3 (thread 0 issues the bulk copy)
        auto issue = [&](uint32_t L) {
            const uint4 sg = segL(L);
            if (!staged(sg)) return;
            const uint32_t bi = L % (uint32_t)kRowBufs;
            if (threadIdx.x == NT - 32) {
                const uint32_t delta = row_delta(sg);
                const uint32_t bytes = ((sg.w - sg.x + delta) * 8u + 15u) & ~15u;
                fence_proxy_async_smem();
                mbar_expect_tx(&sh.mbar[bi], bytes);
                bulk_load(s.rows[bi], packed + sg.x - delta, bytes, &sh.mbar[bi]);
            }
            pend_bits |= 1u << bi;
        };
        // every thread waits for layer L's copy itself (no block barrier)
        auto wait = [&](uint32_t L) {
            const uint32_t bi = L % (uint32_t)kRowBufs;
            if (!((pend_bits >> bi) & 1u)) return;
            if (!mbar_wait_bounded(&sh.mbar[bi], (phase_bits >> bi) & 1u)) sh.tmo = 1u;
            phase_bits ^= 1u << bi;
            pend_bits &= ~(1u << bi);
        };
        auto view = [&](uint32_t L) -> LayerView {
            const uint4 sg = segL(L);
            LayerView v;
            v.rows = staged(sg) ? s.rows[L % (uint32_t)kRowBufs] + row_delta(sg) : packed + sg.x;
            v.g = sg.y - sg.x;
            v.a = sg.z - sg.x;
            v.b = sg.w - sg.x;
            return v;
        };

        // backward wave over the layers
        uint32_t L = lmax;
        bool stopped = false;
        issue(L);
        if (L > 0u) issue(L - 1u);
        wait(L);
        LayerView vnext{};            // layer L+1 (held for its before-noise)
        for (;;) {
            const LayerView vcur = view(L);
            // phase A: noise after the gates of L and before the gates of L+1,
            // in pieces of at most kActive rows (one piece for staged layers)
            housekeeping(epoch);
            const uint32_t sb = epoch & 1u;
            const bool tmo_here = sh.tmo != 0u;
            const uint32_t nA = (L < lmax) ? vcur.a - vcur.g : 0u;
            const uint32_t total = (L < lmax && !tmo_here) ? nA + (vnext.b - vnext.a) : 0u;
            const bool check = (L < lmax) && (L + 1u <= lmin);
            int any = 1;
            for (uint32_t p0 = 0;; p0 += (uint32_t)kActive) {
                const uint32_t p1 = min(p0 + (uint32_t)kActive, total);
                if (p0 < p1) list_active<NT>(s, sh, vcur, vnext, nA, p0, p1);
                int nonzero = 0;
                if (check && p0 == 0u) {
                    for (uint32_t q = threadIdx.x; q < nq; q += NT)
                        if ((s.xs[q] | s.zs[q]) != 0ull) { nonzero = 1; break; }
                }
                const int piece_any = __syncthreads_or(nonzero);
                if (p0 == 0u) any = piece_any;
                const uint32_t n_act = sh.n_act;
                if (n_act) emit_active<NT>(B, s, sh, C, vcur, vnext, nA, p0, n_act, col_tag, level, sb, rec_cap);
                __syncthreads();
                if (threadIdx.x == 0) sh.n_act = 0;
                if (p1 >= total) break;
                __syncthreads();
            }
            if (sh.tmo) { timed_out = true; break; }
            // phase B: records of phase A flushed, the gates of L undone
            flush(epoch, col_tag);
            epoch++;
            if (check && !any) { stopped = true; break; }
            if (L >= 2u) issue(L - 2u);     // into the buffer layer L+1 held
            for (uint32_t i = threadIdx.x; i < vcur.g; i += NT) {
                const uint2 r = vcur.rows[i];
                const uint32_t k = row_kind(r), a = row_a(r);
                switch (k) {
                case K_H: { const unsigned long long t = s.xs[a]; s.xs[a] = s.zs[a]; s.zs[a] = t; break; }
                case K_S: s.xs[a] ^= s.zs[a]; break;
                case K_CX: { const uint32_t t = row_b(r); s.xs[a] ^= s.xs[t]; s.zs[t] ^= s.zs[a]; break; }
                case K_CZ: {
                    const uint32_t t = row_b(r);
                    const unsigned long long za = s.zs[a], zb = s.zs[t];
                    s.xs[a] ^= zb;
                    s.xs[t] ^= za;
                    break;
                }
                case K_R: case K_M: case K_MR: {
                    if (s.zs[a] != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, L, gcol);
                    if (k != K_M) { s.xs[a] = 0ull; s.zs[a] = 0ull; }
                    if (k != K_R) s.xs[a] ^= meas_word(s, n_ent, r.y, m_lo, m_hi);
                    break;
                }
                case K_RX: case K_MX: case K_MRX: {
                    if (s.xs[a] != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, L, gcol);
                    if (k != K_MX) { s.xs[a] = 0ull; s.zs[a] = 0ull; }
                    if (k != K_RX) s.zs[a] ^= meas_word(s, n_ent, r.y, m_lo, m_hi);
                    break;
                }
                default: break;
                }
            }
            __syncthreads();
            if (L == 0u) break;
            vnext = vcur;
            L--;
            wait(L);
        }
        if (!stopped && !timed_out) {
            // before-gate noise of layer 0, then the |0> initial state
            const LayerView v0 = view(0u);
            housekeeping(epoch);
            const uint32_t sb = epoch & 1u;
            const uint32_t total = v0.b - v0.a;
            LayerView none = v0;
            none.g = none.a;             // empty "after" part: rows [a, a)
            for (uint32_t p0 = 0;; p0 += (uint32_t)kActive) {
                const uint32_t p1 = min(p0 + (uint32_t)kActive, total);
                if (p0 < p1) list_active<NT>(s, sh, none, v0, 0u, p0, p1);
                __syncthreads();
                const uint32_t n_act = sh.n_act;
                if (n_act) emit_active<NT>(B, s, sh, C, none, v0, 0u, p0, n_act, col_tag, level, sb, rec_cap);
                __syncthreads();
                if (threadIdx.x == 0) sh.n_act = 0;
                if (p1 >= total) break;
                __syncthreads();
            }
            for (uint32_t q = threadIdx.x; q < nq; q += NT)
                if (s.zs[q] != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, 0xFFFFFFFFu, gcol);
            __syncthreads();
            flush(epoch, col_tag);
            epoch++;
        }
        // copies still in flight after an early stop land before the buffers
        // are reused
        for (uint32_t i = 0; i < (uint32_t)kRowBufs; i++) {
            if ((pend_bits >> i) & 1u) {
                if (!mbar_wait_bounded(&sh.mbar[i], (phase_bits >> i) & 1u)) sh.tmo = 1u;
                phase_bits ^= 1u << i;
                pend_bits &= ~(1u << i);
            }
        }
        __syncthreads();
        if (timed_out || sh.tmo) {
            if (threadIdx.x == 0) report(B.status, GP_ERR_TIMEOUT, 1u, gcol, L);
            break;
        }
    }
}

}  // namespace

size_t stage1_smem_bytes(uint32_t maxq) {
    return (size_t)maxq * 16 + (size_t)kMaxEntries * 12 + (size_t)kStageRecs * 12 + (size_t)kSegCache * 16 +
           (size_t)(kRowBuf + 2) * kRowBufs * 8 + (size_t)kActive * 2;
}

const void *stage1_kernel_ptr(uint32_t threads) {
    switch (threads) {
    case 128: return (const void *)stage1_kernel<128>;
    case 256: return (const void *)stage1_kernel<256>;
    case 1024: return (const void *)stage1_kernel<1024>;
    default: return (const void *)stage1_kernel<512>;
    }
}

void launch_stage1(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t maxq, cudaStream_t s,
                   uint32_t *launches) {
    const size_t smem = stage1_smem_bytes(maxq);
    switch (threads) {
    case 128: stage1_kernel<128><<<grid, 128, smem, s>>>(b, maxq); break;
    case 256: stage1_kernel<256><<<grid, 256, smem, s>>>(b, maxq); break;
    case 1024: stage1_kernel<1024><<<grid, 1024, smem, s>>>(b, maxq); break;
    default: stage1_kernel<512><<<grid, 512, smem, s>>>(b, maxq); break;
    }
    *launches += 1;
}

}  // namespace gpdem
