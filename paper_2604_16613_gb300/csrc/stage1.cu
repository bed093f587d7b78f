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
// plane is zero and no earlier measurement of the column remains.
//
// The walk is sparse: it touches only the qubits whose planes are non-zero
// (the "active" qubits, a few per detector), never the whole layer.  A
// candidate list holds every qubit whose planes may be non-zero (the active
// qubits of the last layer plus the qubits the last layer's gates and
// measurements touched); per layer L two barrier-separated phases run:
//   A  a candidate whose planes are non-zero is active (marked in a per-qubit
//      state byte); a half-warp evaluates the mask words of the noise rows
//      touching it after the gates of L and before the gates of L+1 (the
//      planes hold the state between the two), one Pauli component per lane.
//      A two-qubit row is listed under both of its qubits and evaluated from
//      the first active one.
//   B  the gates of L on active qubits are undone backward: H swaps the
//      planes, S: x ^= z, CX(c,t): x_c ^= x_t and z_t ^= z_c, CZ(a,b):
//      x_a ^= z_b and x_b ^= z_a; measurements XOR in the column's detector
//      bits; resets clear the planes after checking that the detectors
//      commute with them.  The next candidate list is built here: the active
//      qubits, the inactive partners of their two-qubit gates, and inactive
//      qubits the column measures in L.
// A component's mask word is the XOR of the planes its Pauli names (Y = X xor
// Z, two-qubit terms combine both qubits: Sec. 2.3.4).  Non-zero words become
// 16-byte records {mechanism, column, word} that every warp writes straight to
// its own chunk of the global record pool (a warp-uniform running position;
// the next chunk is requested ahead, so the walk never waits on a global
// atomic).  The last warp of the block is a producer: it stages the layer
// windows, concurrently with phase A of the other (consumer) warps, and
// publishes with each window a descriptor of where its parts are.
//
// What a step at L reads -- the gates of L as seen from each qubit, the
// after-gate list offsets of L, the before-gate list offsets of L+1 and the
// list entries between them -- is contiguous in the lowering's layer index,
// so it is staged into shared memory by two 1-D bulk copies (TMA) issued
// several layers ahead into a ring of window buffers, each tracked by an
// mbarrier.  Windows too large for a buffer are read from global memory.
#include <algorithm>

#include "common.cuh"

namespace gpdem {

namespace {

constexpr int kSegCache = 256;      // layer segments cached for the producer
constexpr uint32_t kSplitMinLayers = 64;   // observable walks this long are split in two (twice: three)
constexpr uint32_t kRankSortMax = 256;     // column entries sorted in one rank pass (else bitonic)
constexpr int kMaxBufs = 4;         // window ring slots at most

struct Smem {
    ulonglong2 *pl;                 // per qubit: {X plane, Z plane}
    unsigned long long *ent_w;      // entry words (merged per measurement)
    uint4 *segc;                    // layer segments [seg_lo, seg_lo + kSegCache)
    uint32_t *ent_m;                // entry measurement (sorted)
    uint32_t *ent_l;                // entry layer
    uint32_t *ent_q;                // entry qubit | x-basis << 31
    uint16_t *cand0, *cand1;        // candidate lists (ping-pong)
    unsigned char *bits;            // per qubit: kActive (set in phase A), kAdded
                                    // (put on the next list in phase B) or 0
    unsigned char *win;             // window buffers
};

__host__ __device__ inline uint32_t round8(uint32_t x) { return (x + 7u) & ~7u; }

// bytes of the fixed part of the layout (everything but the windows)
__host__ __device__ inline size_t smem_base_bytes(uint32_t maxq) {
    const size_t q8 = round8(maxq);
    size_t b = 16 * q8                              // xs, zs
               + 8 * (size_t)kMaxEntries            // ent_w
               + 16 * (size_t)kSegCache             // segc
               + 12 * (size_t)kMaxEntries           // ent_m, ent_l, ent_q
               + 4 * q8                             // cand0, cand1
               + q8;                                // bits
    return (b + 127) & ~(size_t)127;
}

// bytes of the index part of a window buffer
__host__ __device__ inline uint32_t window_index_bytes(uint32_t maxq) {
    const uint32_t b = layer_geo(maxq).bytes;
    return (b + 127u) & ~127u;
}

__device__ __forceinline__ Smem carve(unsigned char *base, uint32_t maxq) {
    const uint32_t q8 = round8(maxq);
    Smem s;
    s.pl = reinterpret_cast<ulonglong2 *>(base);
    s.ent_w = reinterpret_cast<unsigned long long *>(s.pl + q8);
    s.segc = reinterpret_cast<uint4 *>(s.ent_w + kMaxEntries);
    s.ent_m = reinterpret_cast<uint32_t *>(s.segc + kSegCache);
    s.ent_l = s.ent_m + kMaxEntries;
    s.ent_q = s.ent_l + kMaxEntries;
    s.cand0 = reinterpret_cast<uint16_t *>(s.ent_q + kMaxEntries);
    s.cand1 = s.cand0 + q8;
    s.bits = reinterpret_cast<unsigned char *>(s.cand1 + q8);
    s.win = base + smem_base_bytes(maxq);
    return s;
}

__device__ __forceinline__ uint16_t *cand_list(const Smem &s, uint32_t i) { return i ? s.cand1 : s.cand0; }

constexpr unsigned char kAdded = 1, kActive = 2;

// XOR of the entry words recorded for measurement m (entries sorted by m)
__device__ __forceinline__ unsigned long long meas_word(const Smem &s, uint32_t n_ent, uint32_t m) {
    uint32_t lo = 0, hi = n_ent;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.ent_m[mid] < m) lo = mid + 1; else hi = mid;
    }
    unsigned long long w = 0ull;
    for (uint32_t i = lo; i < n_ent && s.ent_m[i] == m; i++) w ^= s.ent_w[i];
    return w;
}

__device__ __forceinline__ unsigned long long meas_word_at(const uint32_t *ent_m, const unsigned long long *ent_w,
                                                         uint32_t n_ent, uint32_t m) {
    uint32_t lo = 0, hi = n_ent;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (ent_m[mid] < m) lo = mid + 1; else hi = mid;
    }
    unsigned long long w = 0ull;
    for (uint32_t i = lo; i < n_ent && ent_m[i] == m; i++) w ^= ent_w[i];
    return w;
}

// what one walk step reads (shared or global memory), published by the
// producer with the window
struct Window {
    const uint32_t *gate;       // gate of each qubit in L (step L >= 0)
    const uint16_t *aoff;       // after-gate list offsets of L
    const uint16_t *boff;       // before-gate list offsets of L + 1
    const uint2 *lists;         // after-gate lists of L, then before-gate
                                // lists of L + 1
    uint32_t n_after;           // entries of the after-gate lists
};

struct Shared {
    unsigned long long mbar[kMaxBufs];
    Window desc[kMaxBufs];
    uint32_t item, bail, nent, lmax, tmo;
    uint32_t n_cand[2];     // length of each candidate list (built in phase B)
};

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The (measurement, word) entries of one word column (Eq. init-slp): each
// measurement a detector of the column (or an observable of an observable
// word) reads, with the column bit it sets, sorted by measurement, each run merged into its first
// entry, and each entry's layer and qubit.  Every thread of the block calls
// it, with nent_sh and lmax_sh zeroed.  Returns the entry count, or 0 when
// the column has nothing to walk (no entries, every word cancelled, or over
// capacity: reported); then lmax_sh - 1 is the latest layer holding a
// non-zero word and ent_l[0] the earliest layer of an entry.
template <int NT>
__device__ uint32_t column_entries(const Buffers &B, const CircuitDev &C, uint32_t cidx, uint32_t local, bool is_obs,
                                   uint32_t gcol, uint32_t *ent_m, unsigned long long *ent_w, uint32_t *ent_l,
                                   uint32_t *ent_q, uint32_t &nent_sh, uint32_t &lmax_sh) {
    // (measurement, word) entries of this column (Eq. init-slp)
    if (!is_obs) {
        const uint32_t j0 = local * 64u, j1 = min(j0 + 64u, C.n_det);
        for (uint32_t j = j0 + threadIdx.x; j < j1; j += NT) {
            const uint32_t row = B.det_row[C.det_base + j];
            const uint4 op = C.ops[row];
            const uint32_t mb = B.aux[C.op_base + row];
            for (uint32_t i = 0; i < op.z; i++) {
                const uint32_t e = atomicAdd(&nent_sh, 1u);
                if (e < (uint32_t)kMaxEntries) {
                    ent_m[e] = mb - C.recs[op.y + i];
                    ent_w[e] = 1ull << (j & 63u);
                }
            }
        }
    } else {
        // observable word k holds observables k * obs_per .. (bit = observable)
        const uint32_t o0 = (local - (C.n_cols - C.n_ocols)) * C.obs_per, o1 = o0 + C.obs_per;
        // one warp per row, its records over the lanes (a logical reads
        // many records)
        const uint32_t n_rows = B.obs_count[cidx];
        const uint32_t lane = threadIdx.x & 31u;
        for (uint32_t i0 = threadIdx.x >> 5; i0 < n_rows; i0 += NT / 32u) {
            const uint32_t row = B.obs_rows[C.op_base + i0];
            const uint4 op = C.ops[row];
            if (op.w < o0 || op.w >= o1) continue;
            const uint32_t mb = B.aux[C.op_base + row];
            for (uint32_t i = lane; i < op.z; i += 32u) {
                const uint32_t e = atomicAdd(&nent_sh, 1u);
                if (e < (uint32_t)kMaxEntries) {
                    ent_m[e] = mb - C.recs[op.y + i];
                    ent_w[e] = 1ull << op.w;
                }
            }
        }
    }
    __syncthreads();
    const uint32_t n_ent = nent_sh;
    if (n_ent > (uint32_t)kMaxEntries) {
        if (threadIdx.x == 0) report(B.status, GP_ERR_CAPACITY, 5u, gcol, n_ent);
        return 0u;
    }
    if (n_ent == 0u) return 0u;
    if (n_ent <= kRankSortMax) {
        // few entries: each one's place is the number of entries before it
        // in (measurement, position) order -- one pass instead of the
        // bitonic network's barriers.  The sorted copies go to the layer and
        // qubit arrays (free until the merge below), then back.
        unsigned long long *sw = reinterpret_cast<unsigned long long *>(ent_l);     // n_ent words
        uint32_t *sm = ent_q + kMaxEntries / 2u;                                   // n_ent measurements
        static_assert(2 * kRankSortMax <= kMaxEntries / 2, "rank-sort scratch inside ent_l / ent_q");
        for (uint32_t i = threadIdx.x; i < n_ent; i += NT) {
            const uint32_t m = ent_m[i];
            uint32_t r = 0;
            for (uint32_t j = 0; j < n_ent; j++) {
                const uint32_t mj = ent_m[j];
                r += (mj < m || (mj == m && j < i)) ? 1u : 0u;
            }
            sm[r] = m;
            sw[r] = ent_w[i];
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n_ent; i += NT) {
            ent_m[i] = sm[i];
            ent_w[i] = sw[i];
        }
        __syncthreads();
    } else {
    // bitonic sort of the entries by measurement index
    uint32_t npow = 1;
    while (npow < n_ent) npow <<= 1;
    for (uint32_t i = n_ent + threadIdx.x; i < npow; i += NT) { ent_m[i] = 0xFFFFFFFFu; ent_w[i] = 0ull; }
    __syncthreads();
    for (uint32_t k2 = 2; k2 <= npow; k2 <<= 1) {
        for (uint32_t j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
            for (uint32_t i = threadIdx.x; i < npow; i += NT) {
                const uint32_t ixj = i ^ j2;
                if (ixj > i) {
                    const bool asc = (i & k2) == 0u;
                    const uint32_t mi = ent_m[i], mj = ent_m[ixj];
                    if ((mi > mj) == asc) {
                        ent_m[i] = mj; ent_m[ixj] = mi;
                        const unsigned long long wi = ent_w[i];
                        ent_w[i] = ent_w[ixj]; ent_w[ixj] = wi;
                    }
                }
            }
            __syncthreads();
        }
    }
    }
    // merge the entries of one measurement: the first of a run holds the
    // XOR of the run, the rest hold zero (the layer array holds the merged
    // words meanwhile)
    unsigned long long *merged = reinterpret_cast<unsigned long long *>(ent_l);
    static_assert(kMaxEntries % 2 == 0, "ent_l and ent_q hold one 64-bit word per entry");
    for (uint32_t i = threadIdx.x; i < n_ent; i += NT) {
        unsigned long long w = 0ull;
        if (i == 0u || ent_m[i] != ent_m[i - 1u]) {
            for (uint32_t j = i; j < n_ent && ent_m[j] == ent_m[i]; j++) w ^= ent_w[j];
        }
        merged[i] = w;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_ent; i += NT) {
        const unsigned long long w = merged[i];
        ent_w[i] = w;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_ent; i += NT) {
        const uint2 lq = B.meas_lq[C.meas_base + ent_m[i]];
        ent_l[i] = lq.x;
        ent_q[i] = lq.y;
        if (ent_w[i] != 0ull) atomicMax(&lmax_sh, lq.x + 1u);
    }
    __syncthreads();
    if (lmax_sh == 0u) return 0u;   // every word cancelled
    return n_ent;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) stage1_kernel(Buffers B, uint32_t maxq, uint32_t nbuf, uint32_t list_cap,
                                                       uint32_t wbytes, uint32_t wchunk) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Smem s = carve(smem_raw, maxq);
    __shared__ Shared sh;
    constexpr uint32_t NW = NT / 32;               // warps
    constexpr uint32_t NCW = NW - 1;               // consumer warps (the last one produces)
    constexpr uint32_t NCT = NCW * 32;             // consumer threads
    const Params &P = *B.params;
    const uint32_t level = P.level, rec_cap = P.rec_cap;
    const uint32_t wlim = P.wait_limit;            // polls of a bounded wait
    const bool stall = P.stall_windows != 0u;      // test knob: no window is staged
    // Pauli components a level keeps (Table tab:correlation-level)
    const uint32_t nc_dep1 = level == 0u ? 2u : 3u, nc_dep2 = level == 0u ? 6u : (level == 1u ? 10u : 15u);
    const uint32_t lane = threadIdx.x & 31u, l16 = lane & 15u, half = lane >> 4;
    const uint32_t warp = threadIdx.x >> 5;
    const bool producer = warp == NW - 1;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t windex = window_index_bytes(maxq);
    // ring of window slots: window L in slot (L + 1) mod nring; windows are
    // staged in shared memory only with nbuf >= 2 buffers
    const uint32_t nring = nbuf >= 2u ? nbuf : 2u;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kMaxBufs; i++) mbar_init(&sh.mbar[i], 1);
        fence_mbar_init();
        sh.tmo = 0;
    }
    __syncthreads();
    uint32_t phase_bits = 0u;         // mbarrier parity per ring slot (bit i)
    uint32_t post_par = 0u, posted_any = 0u;   // producer: parity of its posts per slot
    bool timed_out = false;
    // this warp's chunk of the record pool [ck_pos, ck_end) and the next one,
    // requested ahead (its base lives in lane 0 until it is taken)
    uint32_t ck_pos = 0, ck_end = 0, ck_next = 0;
    bool has_next = false;
    // producer warp: first layer held by the segment cache
    uint32_t seg_lo = 0xFFFFFFFFu;

    // positions [a, b) of the record pool (within its capacity) marked empty
    // by the warp: every position handed out is a record or empty, so the
    // scatter never reads a stale record
    auto fill_empty = [&](uint32_t a, uint32_t b) {
        b = min(b, rec_cap);
        for (uint32_t i = a + lane; i < b; i += 32u) B.records[i].x = kNone;
    };
    // at the end: the unused rest of the current chunk and the chunk
    // requested ahead (warp-uniform)
    auto flush_chunks = [&]() {
        fill_empty(ck_pos, ck_end);
        ck_pos = ck_end;
        if (has_next) {
            const uint32_t nb = __shfl_sync(0xFFFFFFFFu, ck_next, 0);
            if (nb < rec_cap) fill_empty(nb, nb + wchunk);
            has_next = false;
        }
    };
    // room for `need` more records in this warp's chunk (warp-uniform);
    // false once the pool is exhausted (reported)
    auto warp_room = [&](uint32_t need) -> bool {
        if (ck_end - ck_pos >= need) return true;
        fill_empty(ck_pos, ck_end);
        uint32_t nb = 0;
        if (has_next) {
            nb = __shfl_sync(0xFFFFFFFFu, ck_next, 0);
        } else {
            if (lane == 0u) nb = atomicAdd(&B.status->rec_count, wchunk);
            nb = __shfl_sync(0xFFFFFFFFu, nb, 0);
        }
        has_next = false;
        if (nb + wchunk > rec_cap || nb + wchunk < nb) {
            if (lane == 0u) report(B.status, GP_ERR_CAPACITY, 8u, nb, rec_cap);
            ck_pos = ck_end = 0;
            return false;
        }
        ck_pos = nb;
        ck_end = nb + wchunk;
        return true;
    };
    // once the warp holds a chunk, ask for the next one while half of it is
    // left (the atomic's result is read only when the chunk is switched)
    auto warp_prefetch = [&]() {
        if (!has_next && ck_end != 0u && ck_end - ck_pos < wchunk / 2u) {
            if (lane == 0u) ck_next = atomicAdd(&B.status->rec_count, wchunk);
            has_next = true;
        }
    };

    for (;;) {
        if (threadIdx.x == 0) {
            sh.item = atomicAdd(&B.status->queue_head, 1u);
            sh.bail = (*(volatile uint32_t *)&B.status->code) != 0u;
            sh.nent = 0;
            sh.lmax = 0;
            sh.n_cand[0] = sh.n_cand[1] = 0;
        }
        __syncthreads();
        const uint32_t item = sh.item;
        if (item >= P.n_items || sh.bail || timed_out) break;
        const uint32_t gcol = B.items[item];
        const uint32_t b = B.col_circ[gcol];
        const CircuitDev &C = B.circ[b];
        const uint32_t local = gcol - C.col_base;
        const bool is_obs = local >= C.n_cols - C.n_ocols;
        const uint32_t col_tag = gcol | (is_obs ? kObsColFlag : 0u);
        const uint32_t nq = C.n_qubits;
        const uint32_t mech_base = C.mech_base;
        seg_lo = 0xFFFFFFFFu;             // the segment cache belongs to the last column

        for (uint32_t q = threadIdx.x; q < nq; q += NT) {
            s.pl[q] = make_ulonglong2(0ull, 0ull);
            s.bits[q] = 0;
        }
        const uint32_t n_ent = column_entries<NT>(B, C, b, local, is_obs, gcol, s.ent_m, s.ent_w, s.ent_l, s.ent_q,
                                                  sh.nent, sh.lmax);
        if (n_ent == 0u) { __syncthreads(); continue; }
        const uint32_t lmax = sh.lmax - 1u;
        const uint32_t lmin = s.ent_l[0];

        // ---- layer index geometry of this circuit --------------------------
        const LayerGeo geo = layer_geo(nq);
        const unsigned char *qbase = B.qidx + (size_t)C.qidx_off * 16u;
        const uint2 *lbase = B.lists + 2ull * C.op_base;
        const uint4 *seg_g = B.layer_seg + C.layer_base;
        auto slot_of = [&](int L) -> uint32_t { return (uint32_t)(L + 1) % nring; };
        // producer warp: publish window L (L = -1: the before-gate noise of
        // layer 0) in its slot -- descriptor, then the bulk copies (or a plain
        // arrive when the window is read from global memory)
        auto post = [&](int L) {
            const uint32_t need = L > 0 ? (uint32_t)L : 0u;
            if (seg_lo == 0xFFFFFFFFu || need < seg_lo || (uint32_t)L + 1u >= seg_lo + (uint32_t)kSegCache) {
                seg_lo = (uint32_t)L + 2u > (uint32_t)kSegCache ? (uint32_t)L + 2u - (uint32_t)kSegCache : 0u;
                const uint32_t n = min((uint32_t)kSegCache, C.n_layers + 1u - seg_lo);
                __syncwarp();
                for (uint32_t i = lane; i < n; i += 32u) s.segc[i] = seg_g[seg_lo + i];
                __syncwarp();
            }
            if (lane != 0u) return;
            const uint4 s1 = s.segc[L + 1 - (int)seg_lo];
            const uint32_t n_after = L >= 0 ? s.segc[L - (int)seg_lo].y : 0u;
            const uint32_t list_start = 2u * s1.x - n_after;
            const uint32_t list_n = n_after + s1.z;
            const uint32_t slot = slot_of(L);
            Window &d = sh.desc[slot];
            d.n_after = n_after;
            if (nbuf >= 2u && list_n + 1u <= list_cap) {
                unsigned char *dst = s.win + (size_t)slot * wbytes;
                const unsigned char *qsrc = L >= 0 ? qbase + (size_t)L * geo.bytes + 2u * geo.qb : qbase;
                const uint32_t qbytes = L >= 0 ? 4u * geo.nq4 + 4u * geo.qb : 2u * geo.qb;
                const uint32_t delta = list_start & 1u;
                const uint32_t lbytes = list_n ? ((list_n + delta) * 8u + 15u) & ~15u : 0u;
                d.lists = reinterpret_cast<const uint2 *>(dst + windex) + delta;
                if (L >= 0) {
                    d.gate = reinterpret_cast<const uint32_t *>(dst);
                    d.aoff = reinterpret_cast<const uint16_t *>(dst + 4u * geo.nq4);
                    d.boff = d.aoff + geo.qb;
                } else {
                    d.gate = nullptr;
                    d.aoff = nullptr;
                    d.boff = reinterpret_cast<const uint16_t *>(dst);
                }
                mbar_expect_tx(&sh.mbar[slot], qbytes + lbytes);
                bulk_load(dst, qsrc, qbytes, &sh.mbar[slot]);
                if (lbytes) bulk_load(dst + windex, lbase + list_start - delta, lbytes, &sh.mbar[slot]);
            } else {
                d.lists = lbase + list_start;
                if (L >= 0) {
                    const unsigned char *p = qbase + (size_t)L * geo.bytes + 2u * geo.qb;
                    d.gate = reinterpret_cast<const uint32_t *>(p);
                    d.aoff = reinterpret_cast<const uint16_t *>(p + 4u * geo.nq4);
                    d.boff = d.aoff + geo.qb;
                } else {
                    d.gate = nullptr;
                    d.aoff = nullptr;
                    d.boff = reinterpret_cast<const uint16_t *>(qbase);
                }
                mbar_arrive(&sh.mbar[slot]);
            }
        };
        // every thread waits for the window of step L itself and reads its
        // descriptor
        auto wait = [&](int L) -> Window {
            const uint32_t slot = slot_of(L);
            if (!mbar_wait_bounded(&sh.mbar[slot], (phase_bits >> slot) & 1u, wlim)) sh.tmo = 1u;
            phase_bits ^= 1u << slot;
            return sh.desc[slot];
        };

        // mask word of component l16 of noise row r seen from candidate q (0
        // for an empty slot, a component the level drops, or a two-qubit row
        // whose first qubit is active: that one evaluates it)
        auto row_word = [&](uint2 r, uint32_t q) -> unsigned long long {
            const uint32_t kind = row_kind(r);
            if (kind < K_XERR) return 0ull;
            const uint32_t ra = row_a(r), rb = row_b(r);
            const bool two = kind == K_DEP2;
            const ulonglong2 pa = s.pl[ra];
            const ulonglong2 pb = two ? s.pl[rb] : make_ulonglong2(0ull, 0ull);
            if (two && q == rb && (pa.x | pa.y) != 0ull) return 0ull;
            const uint32_t nc = two ? nc_dep2 : (kind == K_DEP1 ? nc_dep1 : 1u);
            if (l16 >= nc) return 0ull;
            const unsigned long long codes = two ? 0x0EBF7D639CA25184ull : (kind == K_DEP1 ? 0x321ull : (kind == K_XERR ? 1ull : 2ull));
            const uint32_t code = (uint32_t)(codes >> (4u * l16)) & 0xFu;
            return ((code & 1u) ? pa.x : 0ull) ^ ((code & 2u) ? pa.y : 0ull) ^ ((code & 4u) ? pb.x : 0ull) ^
                   ((code & 8u) ? pb.y : 0ull);
        };
        // write the warp's non-zero words as records (warp-uniform call)
        auto emit = [&](uint2 r, unsigned long long w) {
            const unsigned m = __ballot_sync(0xFFFFFFFFu, w != 0ull);
            if (m == 0u) return;
            const uint32_t cnt = (uint32_t)__popc(m);
            if (!warp_room(cnt)) return;
            if (w != 0ull) {
                const uint32_t mech = mech_base + r.y + l16;
                B.records[ck_pos + __popc(m & lt_mask)] = make_uint4(mech, col_tag, (uint32_t)w, (uint32_t)(w >> 32));
            }
            ck_pos += cnt;
        };

        // phase A for one candidate list (consumer warps): keep the non-zero
        // candidates (appended to list `out`) and emit the mask words of their
        // noise rows; with `after` false only the before-gate lists are read
        // (step -1).  The two half-warps of a warp take two candidates in
        // lockstep, so ballots span the whole warp.
        auto phase_a = [&](const Window &v, const uint16_t *in, uint32_t n_in, bool after, bool check_initial) {
            warp_prefetch();
            for (uint32_t base = 2u * warp; base < n_in; base += 2u * NCW) {
                const uint32_t c = base + half;
                const bool valid = c < n_in;
                const uint32_t q = valid ? in[c] : 0u;
                // the planes and the list offsets load together (the offsets
                // do not wait for the activity test)
                const ulonglong2 pq = s.pl[q];
                uint32_t a0 = 0, a1 = 0;
                if (after) { a0 = v.aoff[q]; a1 = v.aoff[q + 1u]; }
                const uint32_t b0 = v.boff[q], b1 = v.boff[q + 1u];
                const bool act = valid && (pq.x | pq.y) != 0ull;
                if (valid && l16 == 0u) {
                    s.bits[q] = act ? kActive : (unsigned char)0;
                    if (check_initial && act && pq.y != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, 0xFFFFFFFFu, gcol);
                }
                const uint32_t na = act ? a1 - a0 : 0u;
                const uint32_t n = act ? na + (b1 - b0) : 0u;
                const uint32_t nmax = max(n, __shfl_xor_sync(0xFFFFFFFFu, n, 16));
                // two rows per iteration, their loads issued together
                for (uint32_t i = 0; i < nmax; i += 2u) {
                    uint2 r0 = make_uint2(0u, 0u), r1 = make_uint2(0u, 0u);
                    if (i < n) r0 = v.lists[i < na ? a0 + i : v.n_after + b0 + (i - na)];
                    if (i + 1u < n) r1 = v.lists[i + 1u < na ? a0 + i + 1u : v.n_after + b0 + (i + 1u - na)];
                    const unsigned long long w0 = row_word(r0, q), w1 = row_word(r1, q);
                    emit(r0, w0);
                    emit(r1, w1);
                }
            }
        };
        // append up to two qubits per lane to the list being built (one
        // shared atomic per warp)
        auto append2 = [&](uint16_t *list, uint32_t o, bool add_a, uint32_t qa, bool add_b, uint32_t qb) {
            const unsigned ma = __ballot_sync(0xFFFFFFFFu, add_a), mb = __ballot_sync(0xFFFFFFFFu, add_b);
            const uint32_t na = (uint32_t)__popc(ma), tot = na + (uint32_t)__popc(mb);
            if (tot == 0u) return;
            uint32_t nb = 0;
            if (lane == 0u) nb = atomicAdd(&sh.n_cand[o], tot);
            nb = __shfl_sync(0xFFFFFFFFu, nb, 0);
            if (add_a) list[nb + __popc(ma & lt_mask)] = (uint16_t)qa;
            if (add_b) list[nb + na + __popc(mb & lt_mask)] = (uint16_t)qb;
        };

        // ---- backward wave over the layers ---------------------------------
        // At the start of step L the producer refills the slot step L+1 used
        // with window L - nring + 1, so nring - 1 windows are in flight ahead.
        int L = (int)lmax;
        uint32_t p = 0;                   // list read in this step
        uint32_t n_in = 0;                // its length
        uint32_t cur = n_ent;             // entries with layer <= L
        bool stopped = false;
        int posted = L + 1;               // lowest window published so far
        // the producer's posts (a stalled producer posts nothing)
        auto post_tracked = [&](int k) {
            if (!producer || stall) return;
            post(k);
            post_par ^= 1u << slot_of(k);
            posted_any |= 1u << slot_of(k);
        };
        for (int k = L; k >= L - (int)nring + 2 && k >= -1; k--) {
            post_tracked(k);
            posted = k;
        }
        for (;;) {
            if (L - (int)nring + 1 >= -1) {
                post_tracked(L - (int)nring + 1);
                posted = L - (int)nring + 1;
            }
            const Window v = wait(L);
            // phase A
            const uint16_t *const in_list = cand_list(s, p);
            if (!producer && !sh.tmo) phase_a(v, in_list, n_in, true, false);
            __syncthreads();
            if (sh.tmo) { timed_out = true; break; }
            // phase B: the gates of L undone
            const uint32_t o = p ^ 1u;
            uint16_t *const next = cand_list(s, o);
            if (threadIdx.x == 0) sh.n_cand[p] = 0;
            if (!producer) {
                for (uint32_t base = 0; base < n_in; base += NCT) {
                    const uint32_t i = base + threadIdx.x;
                    uint32_t partner = kNone, q = 0;
                    bool keep_q = false;
                    if (i < n_in) q = in_list[i];
                    if (i < n_in && s.bits[q] == kActive) {
                        keep_q = true;
                        const uint32_t g = v.gate[q];
                        const uint32_t k = g >> 28, pay = g & 0x0FFFFFFFu;
                        switch (k) {
                        case K_H: { const ulonglong2 t = s.pl[q]; s.pl[q] = make_ulonglong2(t.y, t.x); break; }
                        case K_S: { ulonglong2 t = s.pl[q]; t.x ^= t.y; s.pl[q] = t; break; }
                        case GV_CX_C: {
                            ulonglong2 c_ = s.pl[q], t_ = s.pl[pay];
                            c_.x ^= t_.x;
                            t_.y ^= c_.y;
                            s.pl[q] = c_;
                            s.pl[pay] = t_;
                            partner = pay;
                            break;
                        }
                        case GV_CX_T: {
                            if (s.bits[pay] == kActive) break;    // undone from the active control
                            ulonglong2 c_ = s.pl[pay], t_ = s.pl[q];
                            c_.x ^= t_.x;
                            t_.y ^= c_.y;
                            s.pl[pay] = c_;
                            s.pl[q] = t_;
                            partner = pay;
                            break;
                        }
                        case GV_CZ_B:
                            if (s.bits[pay] == kActive) break;    // undone from the active first qubit
                            // fall through
                        case GV_CZ_A: {
                            ulonglong2 a_ = s.pl[q], b_ = s.pl[pay];
                            const unsigned long long za = a_.y, zb = b_.y;
                            a_.x ^= zb;
                            b_.x ^= za;
                            s.pl[q] = a_;
                            s.pl[pay] = b_;
                            partner = pay;
                            break;
                        }
                        case K_R: case K_M: case K_MR: {
                            ulonglong2 t = s.pl[q];
                            if (t.y != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, (uint32_t)L, gcol);
                            if (k != K_M) t = make_ulonglong2(0ull, 0ull);
                            if (k != K_R) t.x ^= meas_word(s, n_ent, pay);
                            s.pl[q] = t;
                            break;
                        }
                        case K_RX: case K_MX: case K_MRX: {
                            ulonglong2 t = s.pl[q];
                            if (t.x != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, (uint32_t)L, gcol);
                            if (k != K_MX) t = make_ulonglong2(0ull, 0ull);
                            if (k != K_RX) t.y ^= meas_word(s, n_ent, pay);
                            s.pl[q] = t;
                            break;
                        }
                        default: break;
                        }
                    }
                    const bool add = partner != kNone && s.bits[partner] == 0;
                    if (add) s.bits[partner] = kAdded;
                    append2(next, o, keep_q, q, add, partner);
                }
            }
            // measurements of the column at L on inactive qubits
            uint32_t lo = cur;
            if (cur > 0u && s.ent_l[cur - 1u] == (uint32_t)L) {
                uint32_t l0 = 0, h0 = cur;
                while (l0 < h0) {
                    const uint32_t mid = (l0 + h0) >> 1;
                    if (s.ent_l[mid] < (uint32_t)L) l0 = mid + 1; else h0 = mid;
                }
                lo = l0;
                if (!producer) {
                    for (uint32_t base = lo; base < cur; base += NCT) {
                        const uint32_t i = base + threadIdx.x;
                        bool add = false;
                        uint32_t q = 0;
                        if (i < cur) {
                            const unsigned long long w = s.ent_w[i];
                            const uint32_t qv = s.ent_q[i];
                            q = qv & 0x7FFFFFFFu;
                            // an active qubit had the word applied by its gate above
                            if (w != 0ull && s.bits[q] == 0) {
                                if (qv >> 31) s.pl[q].y ^= w; else s.pl[q].x ^= w;
                                s.bits[q] = kAdded;
                                add = true;
                            }
                        }
                        append2(next, o, add, q, false, 0u);
                    }
                }
            }
            cur = lo;
            __syncthreads();
            n_in = sh.n_cand[o];
            p = o;
            if (L == 0) break;
            if (n_in == 0u && (uint32_t)(L - 1) < lmin) { stopped = true; break; }
            L--;
        }
        if (!stopped && !timed_out) {
            // before-gate noise of layer 0 on the candidates, then the |0>
            // initial state
            L = -1;
            const Window v = wait(-1);
            if (!producer && !sh.tmo) phase_a(v, cand_list(s, p), n_in, false, true);
        }
        // windows published ahead of an early stop land before their slots
        // are reused
        if (!stall)
            for (int k = L - 1; k >= posted; k--) wait(k);
        __syncthreads();
        if (timed_out || sh.tmo) {
            if (threadIdx.x == 0) report(B.status, GP_ERR_TIMEOUT, 1u, gcol, (uint32_t)L);
            break;
        }
    }
    flush_chunks();
    // after a wait gave up, copies may still be in flight: the last one posted
    // to each slot lands before the block exits (full limit)
    if (producer && lane == 0u) {
        for (uint32_t i = 0; i < nring; i++)
            if ((posted_any >> i) & 1u) mbar_wait_bounded(&sh.mbar[i], ((post_par >> i) & 1u) ^ 1u);
    }
}

// ---------------------------------------------------------------------------
// Role-split walk.  The walk of a column is a chain over its layers; the
// noise rows of a layer only read the planes of that layer.  So one warp (the
// walker) advances the planes layer by layer with warp-level syncs only, and
// publishes for each step a snapshot of its active qubits' planes; the other
// warps (emitters) evaluate the noise rows of a step from that snapshot while
// the walker is already on the next one; the last warp stages the layer
// windows.  From 512 threads a second walker warp (four from 1024) waits on a
// named barrier and joins only the steps of more than 64 candidates, which
// warp 0 hands to it: the long chain of small steps (an observable's walk)
// keeps its single-warp latency, and the wide steps of detector columns are
// undone in parallel.  The snapshot tables are double-buffered by step parity and
// tagged with the step that wrote an entry (a qubit whose tag differs is not
// active in that step), so they are never cleared.  mbarriers order the
// roles: window full (producer -> walker), window free (walker, emitters ->
// producer), table full (walker -> emitters: it also carries the window,
// which the walker saw land before publishing), table free (emitters ->
// walker); every wait is bounded.
// ---------------------------------------------------------------------------
struct SplitSmem {
    ulonglong2 *pl;                 // walker: per qubit {X plane, Z plane}
    ulonglong2 *tab0, *tab1;        // snapshot planes per step parity
    uint4 *segc;                    // producer: layer segments
    unsigned long long *ent_w;      // entry words
    uint32_t *tag0, *tag1;          // step that wrote a snapshot entry
    uint32_t *ent_m, *ent_l, *ent_q;
    uint16_t *act0, *act1;          // active qubits of a step
    uint16_t *add;                  // qubits the walker adds to the next step's candidates
    unsigned char *bits;            // walker: kActive / kAdded / 0 per qubit
    unsigned char *win;             // window buffers
};

// Share r of R of [base, base + bytes) prefetched into L2 (a hint: bulk
// prefetches of up to 64 KB, which nothing waits for).  base is 16-byte aligned.
__device__ __forceinline__ void l2_prefetch_share(const void *base, size_t bytes, uint32_t r, uint32_t R) {
    const char *p = static_cast<const char *>(base);
    for (size_t off = (size_t)r * 65536u; off < bytes; off += (size_t)R * 65536u) {
        const uint32_t len = (uint32_t)(min(bytes - off, (size_t)65536u) & ~(size_t)15u);
        if (len) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + off), "r"(len) : "memory");
    }
}

// Warps of a block: the first warps walk (two from 512 threads, four from
// 1024), the last warp stages windows, the rest emit.
__host__ __device__ constexpr uint32_t split_walkers(uint32_t nt) { return nt >= 1024u ? 4u : (nt >= 512u ? 2u : 1u); }
__host__ __device__ constexpr uint32_t split_emitters(uint32_t nt) { return nt / 32u - 1u - split_walkers(nt); }

__host__ __device__ inline size_t split_base_bytes(uint32_t maxq) {
    const size_t q8 = round8(maxq);
    size_t b = 16 * q8 * 3                          // pl, tab[2]
               + 16 * (size_t)kSegCache             // segc
               + 8 * (size_t)kMaxEntries            // ent_w
               + 4 * q8 * 2                         // tag[2]
               + 12 * (size_t)kMaxEntries           // ent_m, ent_l, ent_q
               + 2 * q8 * 3                         // act[2], add
               + q8;                                // bits
    return (b + 127) & ~(size_t)127;
}

__device__ __forceinline__ SplitSmem split_carve(unsigned char *base, uint32_t maxq) {
    const uint32_t q8 = round8(maxq);
    SplitSmem s;
    s.pl = reinterpret_cast<ulonglong2 *>(base);
    s.tab0 = s.pl + q8;
    s.tab1 = s.tab0 + q8;
    s.segc = reinterpret_cast<uint4 *>(s.tab1 + q8);
    s.ent_w = reinterpret_cast<unsigned long long *>(s.segc + kSegCache);
    s.tag0 = reinterpret_cast<uint32_t *>(s.ent_w + kMaxEntries);
    s.tag1 = s.tag0 + q8;
    s.ent_m = s.tag1 + q8;
    s.ent_l = s.ent_m + kMaxEntries;
    s.ent_q = s.ent_l + kMaxEntries;
    s.act0 = reinterpret_cast<uint16_t *>(s.ent_q + kMaxEntries);
    s.act1 = s.act0 + q8;
    s.add = s.act1 + q8;
    s.bits = reinterpret_cast<unsigned char *>(s.add + q8);
    s.win = base + split_base_bytes(maxq);
    return s;
}
// the parity-b copies (selects, not an indexed array: no stack frame)
__device__ __forceinline__ ulonglong2 *tab_of(const SplitSmem &s, uint32_t b) { return b ? s.tab1 : s.tab0; }
__device__ __forceinline__ uint32_t *tag_of(const SplitSmem &s, uint32_t b) { return b ? s.tag1 : s.tag0; }
__device__ __forceinline__ uint16_t *act_of(const SplitSmem &s, uint32_t b) { return b ? s.act1 : s.act0; }

// what the walker publishes with a step's snapshot
struct StepDesc {
    int layer;          // L (-1: the before-gate noise of layer 0)
    uint32_t n_act;     // active qubits (act list of the step's parity)
    uint32_t slot;      // window slot of L
    uint32_t end;       // 1: no step; the column is done
};

// a large step of the walk, as warp 0 hands it to the helper walker warps
struct WalkStep {
    int L;
    uint32_t n_prev, n_cand, slot;
    uint16_t *ab;
    const uint16_t *prev;
    uint32_t b, snap, stamp, cmd;     // cmd 0: the walk is over
};

struct SplitShared {
    unsigned long long win_full[kMaxBufs], win_free[kMaxBufs];
    unsigned long long tab_full[2], tab_free[2];
    Window desc[kMaxBufs];
    StepDesc step[2];
    uint32_t item, bail, nent, lmax;
    uint32_t tmo;           // a wait gave up (every role leaves)
    uint32_t walk_done;     // the walker left the column (the producer stops)
    int stop_layer;         // last layer the walker stepped through
    int posted_lo;          // lowest window the producer posted
    WalkStep wstep;         // warp 0 -> helper walker warps: the large step
    uint32_t wcnt[2];       // large step: {active, added}
    uint32_t worked;        // the block took at least one work item
};

template <int NT, bool WIDE>
__global__ void __launch_bounds__(NT, 1) stage1_split_kernel(Buffers B, uint32_t maxq, uint32_t nbuf,
                                                             uint32_t list_cap, uint32_t wbytes, uint32_t wchunk) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const SplitSmem s = split_carve(smem_raw, maxq);
    __shared__ SplitShared sh;
    constexpr uint32_t NW = NT / 32;
    constexpr uint32_t WW = split_walkers(NT);      // walker warps
    constexpr uint32_t NE = split_emitters(NT);     // emitter warps
    static_assert(NE >= 1, "walkers, emitters and producer");
    const Params &P = *B.params;
    const uint32_t level = P.level, rec_cap = P.rec_cap;
    const uint32_t wlim = P.wait_limit;            // polls of a bounded wait
    const bool stall = P.stall_windows != 0u;      // test knob: no window is staged
    const uint32_t nc_dep1 = level == 0u ? 2u : 3u, nc_dep2 = level == 0u ? 6u : (level == 1u ? 10u : 15u);
    const uint32_t lane = threadIdx.x & 31u, l16 = lane & 15u, half = lane >> 4;
    const uint32_t warp = threadIdx.x >> 5;
    const bool walker = warp < WW, producer = warp == NW - 1u;
    const uint32_t ew = warp - WW;                  // emitter index
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t windex = window_index_bytes(maxq);
    const uint32_t nring = nbuf >= 2u ? nbuf : 2u;
    volatile uint32_t *const tmo_v = &sh.tmo;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kMaxBufs; i++) {
            mbar_init(&sh.win_full[i], 1);
            mbar_init(&sh.win_free[i], NE + 1u);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&sh.tab_full[i], 1);
            mbar_init(&sh.tab_free[i], NE);
        }
        fence_mbar_init();
        sh.tmo = 0;
        sh.worked = 0;
    }
    for (uint32_t q = threadIdx.x; q < round8(maxq); q += NT) s.tag0[q] = s.tag1[q] = kNone;
    __syncthreads();

    // per-thread barrier phases (bit i: slot or buffer i)
    uint32_t full_par = 0;                  // walker: window full
    uint32_t free_par = 0, free_pend = 0;   // producer: window free; slots awaiting a release
    uint32_t post_par = 0, posted_any = 0;  // producer: parity of the posts per slot
    uint32_t tfull_par = 0;                 // emitters: table full
    uint32_t tfree_par = 0, tfree_pend = 0; // walker: table free; buffers awaiting a release
    uint32_t st = 0;                        // steps taken by this block (snapshot tags)
    uint32_t ck_pos = 0, ck_end = 0, ck_next = 0;
    bool has_next = false;
    uint32_t seg_lo = 0xFFFFFFFFu;

    // bounded wait; gives up early once another role has given up
    auto wait_bar = [&](unsigned long long *bar, uint32_t parity) -> bool {
        for (uint32_t it = 0; it < wlim; it++) {
            if (mbar_try_wait(bar, parity)) return true;
            if ((it & 31u) == 31u && *tmo_v) return false;
        }
        *tmo_v = 1u;
        return false;
    };
    // the same, by every lane of a warp with one outcome for all (the loops
    // around it use warp-wide votes)
    auto wait_warp = [&](unsigned long long *bar, uint32_t parity) -> bool {
        if (__all_sync(0xFFFFFFFFu, mbar_try_wait(bar, parity))) return true;     // usually done already
        return __all_sync(0xFFFFFFFFu, wait_bar(bar, parity));
    };
    auto fill_empty = [&](uint32_t a, uint32_t b) {
        b = min(b, rec_cap);
        for (uint32_t i = a + lane; i < b; i += 32u) B.records[i].x = kNone;
    };
    auto flush_chunks = [&]() {
        fill_empty(ck_pos, ck_end);
        ck_pos = ck_end;
        if (has_next) {
            const uint32_t nb = __shfl_sync(0xFFFFFFFFu, ck_next, 0);
            if (nb < rec_cap) fill_empty(nb, nb + wchunk);
            has_next = false;
        }
    };
    auto warp_room = [&](uint32_t need) -> bool {
        if (ck_end - ck_pos >= need) return true;
        fill_empty(ck_pos, ck_end);
        uint32_t nb = 0;
        if (has_next) {
            nb = __shfl_sync(0xFFFFFFFFu, ck_next, 0);
        } else {
            if (lane == 0u) nb = atomicAdd(&B.status->rec_count, wchunk);
            nb = __shfl_sync(0xFFFFFFFFu, nb, 0);
        }
        has_next = false;
        if (nb + wchunk > rec_cap || nb + wchunk < nb) {
            if (lane == 0u) report(B.status, GP_ERR_CAPACITY, 8u, nb, rec_cap);
            ck_pos = ck_end = 0;
            return false;
        }
        ck_pos = nb;
        ck_end = nb + wchunk;
        return true;
    };
    auto warp_prefetch = [&]() {
        if (!has_next && ck_end != 0u && ck_end - ck_pos < wchunk / 2u) {
            if (lane == 0u) ck_next = atomicAdd(&B.status->rec_count, wchunk);
            has_next = true;
        }
    };

    for (;;) {
        if (threadIdx.x == 0) {
            sh.item = atomicAdd(&B.status->queue_head, 1u);
            if (sh.item < P.n_items) sh.worked = 1u;
            sh.bail = (*(volatile uint32_t *)&B.status->code) != 0u;
            sh.nent = 0;
            sh.lmax = 0;
            sh.walk_done = 0;
            sh.stop_layer = 0;
            sh.posted_lo = 0;
            sh.wcnt[0] = sh.wcnt[1] = 0;
        }
        __syncthreads();
        const uint32_t item = sh.item;
        if (item >= P.n_items || sh.bail || sh.tmo) break;
        const uint32_t item_word = B.items[item];
        const uint32_t seg = item_word >> kSegShift;      // segment of a split walk
        const uint32_t gcol = item_word & kColMask;
        const uint32_t cidx = B.col_circ[gcol];
        const CircuitDev &C = B.circ[cidx];
        const uint32_t local = gcol - C.col_base;
        const bool is_obs = local >= C.n_cols - C.n_ocols;
        const uint32_t col_tag = gcol | (is_obs ? kObsColFlag : 0u);
        const uint32_t nq = C.n_qubits;
        const uint32_t mech_base = C.mech_base;
        seg_lo = 0xFFFFFFFFu;
        for (uint32_t q = threadIdx.x; q < nq; q += NT) {
            s.pl[q] = make_ulonglong2(0ull, 0ull);
            s.bits[q] = 0;
        }
        const uint32_t n_ent = column_entries<NT>(B, C, cidx, local, is_obs, gcol, s.ent_m, s.ent_w, s.ent_l,
                                                  s.ent_q, sh.nent, sh.lmax);
        if (n_ent == 0u) { __syncthreads(); continue; }
        const uint32_t lmax = sh.lmax - 1u;
        const uint32_t lmin = s.ent_l[0];
        // a long observable walk is shared by up to three blocks (one work
        // item each): segment k emits the steps emit_hi .. emit_lo and
        // fast-forwards through the steps above emit_hi first (gates undone,
        // nothing emitted or published).  A fast-forward step costs about
        // 0.73 of an emitting one, so segments of equal time emit, from the
        // top: 79 % / 21 % of the walk (two segments), 74.5 % / 20 % / 5.5 %
        // (three).
        const uint32_t n_seg = !is_obs ? 1u
                                       : min(P.obs_segments,
                                             lmax >= 2u * kSplitMinLayers ? 3u : (lmax >= kSplitMinLayers ? 2u : 1u));
        if (seg >= n_seg) { __syncthreads(); continue; }
        int b1 = -1, b2 = -1;                             // segment boundaries
        if (n_seg == 2u) b1 = max(1, (int)(3u * lmax / 14u));
        if (n_seg == 3u) {
            b1 = max(2, (int)(51u * lmax / 200u));
            b2 = min(b1 - 1, max(1, (int)(11u * lmax / 200u)));
        }
        const int emit_hi = seg == 0u ? (int)lmax : (seg == 1u ? b1 - 1 : b2 - 1);
        const int emit_lo = seg + 1u == n_seg ? -1 : (seg == 0u ? b1 : b2);
        const LayerGeo geo = layer_geo(nq);
        const unsigned char *qbase = B.qidx + (size_t)C.qidx_off * 16u;
        const uint2 *lbase = B.lists + 2ull * C.op_base;
        const uint4 *seg_g = B.layer_seg + C.layer_base;
        auto slot_of = [&](int L) -> uint32_t { return (uint32_t)(L + 1) % nring; };

        // ---- walker warps.  Warp 0 walks; a step of more than 64 candidates
        // is split over all walker warps (the helpers wait on a named barrier
        // in between): the activity pass over the candidates, a barrier, the
        // gates undone over the active list, a barrier.  The owner rule
        // leaves every plane a single writer, so the warps need no other
        // synchronisation; list positions come from shared counters.
        auto wsync = [&]() {
            if (WW == 1u) __syncwarp();
            else asm volatile("bar.sync 1, %0;" ::"n"(WW * 32u) : "memory");
        };
        // a position for n entries of this warp's ballot (one shared atomic)
        auto take = [&](uint32_t *ctr, uint32_t n) -> uint32_t {
            uint32_t o = 0;
            if (lane == 0u && n) o = atomicAdd(ctr, n);
            return __shfl_sync(0xFFFFFFFFu, o, 0);
        };
        auto large_activity = [&](uint32_t wid, int Lc, uint32_t np, uint32_t nc, const uint16_t *prv, uint16_t *abl,
                                  ulonglong2 *tbl, uint32_t *tgl, bool snp, uint32_t stamp) {
            for (uint32_t base = 64u * wid; base < nc; base += 64u * WW) {
                const uint32_t i0 = base + lane, i1 = base + lane + 32u;
                uint32_t q0 = 0, q1 = 0;
                if (i0 < nc) q0 = i0 < np ? prv[i0] : s.add[i0 - np];
                if (i1 < nc) q1 = i1 < np ? prv[i1] : s.add[i1 - np];
                const ulonglong2 p0 = s.pl[q0], p1 = s.pl[q1];
                const bool a0 = i0 < nc && (p0.x | p0.y) != 0ull;
                const bool a1 = i1 < nc && (p1.x | p1.y) != 0ull;
                if (i0 < nc) s.bits[q0] = a0 ? kActive : (unsigned char)0;
                if (i1 < nc) s.bits[q1] = a1 ? kActive : (unsigned char)0;
                if (a0 && snp) { tbl[q0] = p0; tgl[q0] = stamp; }
                if (a1 && snp) { tbl[q1] = p1; tgl[q1] = stamp; }
                if (Lc < 0 && ((a0 && p0.y != 0ull) || (a1 && p1.y != 0ull)))
                    report(B.status, GP_ERR_NONDETERMINISTIC, cidx, 0xFFFFFFFFu, gcol);
                const unsigned m0 = __ballot_sync(0xFFFFFFFFu, a0), m1 = __ballot_sync(0xFFFFFFFFu, a1);
                const uint32_t o = take(&sh.wcnt[0], (uint32_t)(__popc(m0) + __popc(m1)));
                if (a0) abl[o + __popc(m0 & lt_mask)] = (uint16_t)q0;
                if (a1) abl[o + __popc(m0) + __popc(m1 & lt_mask)] = (uint16_t)q1;
            }
        };
        auto undo = [&](uint32_t q, ulonglong2 P, uint32_t g, bool act, int Lc) -> uint32_t {
            if (!act) return kNone;
            const uint32_t k = g >> 28, pay = g & 0x0FFFFFFFu;
            if (k >= GV_CX_C) {
                const bool pact = s.bits[pay] == kActive;
                if (pact && (k == GV_CX_T || k == GV_CZ_B)) return kNone;
                const ulonglong2 Q = s.pl[pay];
                const bool cxc = k == GV_CX_C, cxt = k == GV_CX_T, cz = !cxc && !cxt;
                // CX(c,t): x_c ^= x_t, z_t ^= z_c; CZ(a,b): x_a ^= z_b, x_b ^= z_a
                const unsigned long long ox = P.x ^ (cxc ? Q.x : 0ull) ^ (cz ? Q.y : 0ull);
                const unsigned long long oz = P.y ^ (cxt ? Q.y : 0ull);
                const unsigned long long px = Q.x ^ (cxt ? P.x : 0ull) ^ (cz ? P.y : 0ull);
                const unsigned long long pz = Q.y ^ (cxc ? P.y : 0ull);
                s.pl[q] = make_ulonglong2(ox, oz);
                s.pl[pay] = make_ulonglong2(px, pz);
                return pay;
            }
            if (k == K_H) { s.pl[q] = make_ulonglong2(P.y, P.x); return kNone; }
            if (k == K_S) { s.pl[q] = make_ulonglong2(P.x ^ P.y, P.y); return kNone; }
            if (k == GV_NONE) return kNone;
            // measurements and resets
            ulonglong2 t = P;
            if (k <= K_MR) {
                if (t.y != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, cidx, (uint32_t)Lc, gcol);
                if (k != K_M) t = make_ulonglong2(0ull, 0ull);
                if (k != K_R) t.x ^= meas_word_at(s.ent_m, s.ent_w, n_ent, pay);
            } else {
                if (t.x != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, cidx, (uint32_t)Lc, gcol);
                if (k != K_MX) t = make_ulonglong2(0ull, 0ull);
                if (k != K_RX) t.y ^= meas_word_at(s.ent_m, s.ent_w, n_ent, pay);
            }
            s.pl[q] = t;
            return kNone;
        };
        auto large_undo = [&](uint32_t wid, int Lc, uint32_t na, const uint16_t *abl, const Window &vw) {
            for (uint32_t base = 32u * wid; base < na; base += 32u * WW) {
                const uint32_t i = base + lane;
                const uint32_t q = i < na ? abl[i] : 0u;
                const ulonglong2 P = s.pl[q];
                const uint32_t partner = undo(q, P, i < na ? vw.gate[q] : 0u, i < na, Lc);
                const bool add = partner != kNone && s.bits[partner] == 0;
                if (add) s.bits[partner] = kAdded;
                const unsigned m = __ballot_sync(0xFFFFFFFFu, add);
                const uint32_t o = take(&sh.wcnt[1], (uint32_t)__popc(m));
                if (add) s.add[o + __popc(m & lt_mask)] = (uint16_t)partner;
            }
        };
        if (walker && warp != 0u) {
            // ---- helper walker warps: large steps of warp 0's walk
            for (;;) {
                wsync();
                const WalkStep ws = sh.wstep;
                if (ws.cmd == 0u) break;
                const Window vw = sh.desc[ws.slot];
                large_activity(warp, ws.L, ws.n_prev, ws.n_cand, ws.prev, ws.ab, tab_of(s, ws.b), tag_of(s, ws.b),
                               ws.snap != 0u, ws.stamp);
                wsync();
                if (ws.L >= 0) large_undo(warp, ws.L, sh.wcnt[0], ws.ab, vw);
                wsync();
            }
        } else if (walker && warp == 0u) {
            // ---- walker: candidates of a step = the active qubits of the
            // last step, then the qubits the last step added
            uint32_t n_prev = 0, n_add = 0, cur = n_ent;
            int L = (int)lmax;
            bool ok = true;
            uint32_t slot = slot_of(L);
            // fast-forward steps (L > emit_hi) keep their active lists in the
            // two act buffers alternately, arranged so that the last one lands
            // where the first emitting step reads its predecessor's
            uint32_t ff_buf = 0u;
            if (emit_hi < (int)lmax) {
                const uint32_t n_ff = lmax - (uint32_t)emit_hi;
                ff_buf = ((st & 1u) ^ 1u) ^ ((n_ff - 1u) & 1u);
            }
            // the gates of L undone for one candidate (registers from the
            // activity pass): the owner of a two-qubit gate (its active
            // qubit, or its control / first qubit when both are active)
            // updates both planes; returns the partner it touched
            for (;;) {
                const bool ff = L > emit_hi;
                const bool snap = !ff;            // a snapshot is published for the emitters
                const uint32_t b = st & 1u;
                if (!wait_warp(&sh.win_full[slot], (full_par >> slot) & 1u)) { ok = false; break; }
                full_par ^= 1u << slot;
                const Window v = sh.desc[slot];
                if (snap) {
                    if ((tfree_pend >> b) & 1u) {
                        if (!wait_warp(&sh.tab_free[b], (tfree_par >> b) & 1u)) { ok = false; break; }
                        tfree_par ^= 1u << b;
                    }
                    tfree_pend |= 1u << b;
                }
                const uint16_t *prev = ff ? act_of(s, ff_buf ^ 1u) : act_of(s, b ^ 1u);
                ulonglong2 *const tb = tab_of(s, b);
                uint32_t *const tg = tag_of(s, b);
                uint16_t *const ab = ff ? act_of(s, ff_buf) : act_of(s, b);
                const uint32_t n_cand = n_prev + n_add;
                uint32_t n_act = 0, n_new = 0;
                // activity and snapshot of candidates c0, c1 (one lane's pair)
                auto activity = [&](uint32_t i0, uint32_t i1, uint32_t &q0, uint32_t &q1, ulonglong2 &p0, ulonglong2 &p1,
                                    uint32_t &g0, uint32_t &g1, bool &a0, bool &a1) {
                    q0 = q1 = 0;
                    if (i0 < n_cand) q0 = i0 < n_prev ? prev[i0] : s.add[i0 - n_prev];
                    if (i1 < n_cand) q1 = i1 < n_prev ? prev[i1] : s.add[i1 - n_prev];
                    p0 = s.pl[q0];
                    p1 = s.pl[q1];
                    g0 = L >= 0 ? v.gate[q0] : 0u;
                    g1 = L >= 0 ? v.gate[q1] : 0u;
                    a0 = i0 < n_cand && (p0.x | p0.y) != 0ull;
                    a1 = i1 < n_cand && (p1.x | p1.y) != 0ull;
                    if (i0 < n_cand) s.bits[q0] = a0 ? kActive : (unsigned char)0;
                    if (i1 < n_cand) s.bits[q1] = a1 ? kActive : (unsigned char)0;
                    if (a0 && snap) { tb[q0] = p0; tg[q0] = st; }
                    if (a1 && snap) { tb[q1] = p1; tg[q1] = st; }
                    if (L < 0 && ((a0 && p0.y != 0ull) || (a1 && p1.y != 0ull)))
                        report(B.status, GP_ERR_NONDETERMINISTIC, cidx, 0xFFFFFFFFu, gcol);
                    const unsigned m0 = __ballot_sync(0xFFFFFFFFu, a0), m1 = __ballot_sync(0xFFFFFFFFu, a1);
                    if (a0) ab[n_act + __popc(m0 & lt_mask)] = (uint16_t)q0;
                    n_act += __popc(m0);
                    if (a1) ab[n_act + __popc(m1 & lt_mask)] = (uint16_t)q1;
                    n_act += __popc(m1);
                };
                auto append = [&](uint32_t partner) {
                    const bool add = partner != kNone && s.bits[partner] == 0;
                    if (add) s.bits[partner] = kAdded;
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, add);
                    if (add) s.add[n_new + __popc(m & lt_mask)] = (uint16_t)partner;
                    n_new += __popc(m);
                };
                auto publish = [&]() {
                    if (!snap) {
                        __syncwarp();
                        return;
                    }
                    if (lane == 0u) sh.step[b] = StepDesc{L, n_act, slot, 0u};
                    __syncwarp();
                    if (lane == 0u) mbar_arrive(&sh.tab_full[b]);
                };
                if (n_cand <= 32u) {
                    // the step's candidates stay in registers (one per lane)
                    uint32_t q0 = 0;
                    if (lane < n_cand) q0 = lane < n_prev ? prev[lane] : s.add[lane - n_prev];
                    const ulonglong2 p0 = s.pl[q0];
                    const uint32_t g0 = L >= 0 ? v.gate[q0] : 0u;
                    const bool a0 = lane < n_cand && (p0.x | p0.y) != 0ull;
                    if (lane < n_cand) s.bits[q0] = a0 ? kActive : (unsigned char)0;
                    if (a0 && snap) { tb[q0] = p0; tg[q0] = st; }
                    if (L < 0 && a0 && p0.y != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, cidx, 0xFFFFFFFFu, gcol);
                    const unsigned m0 = __ballot_sync(0xFFFFFFFFu, a0);
                    if (a0) ab[__popc(m0 & lt_mask)] = (uint16_t)q0;
                    n_act = __popc(m0);
                    publish();
                    if (L >= 0) append(undo(q0, p0, g0, a0, L));
                } else if (n_cand <= 64u) {
                    // two per lane
                    uint32_t q0, q1, g0, g1;
                    ulonglong2 p0, p1;
                    bool a0, a1;
                    activity(lane, lane + 32u, q0, q1, p0, p1, g0, g1, a0, a1);
                    publish();
                    if (L >= 0) {
                        append(undo(q0, p0, g0, a0, L));
                        append(undo(q1, p1, g1, a1, L));
                    }
                } else {
                    // more than 64 candidates: the helper walker warps join in
                    if (lane == 0u) {
                        sh.wcnt[0] = sh.wcnt[1] = 0u;
                        sh.wstep = WalkStep{L, n_prev, n_cand, slot, ab, prev, b, snap ? 1u : 0u, st, 1u};
                    }
                    wsync();                                // the helpers wake
                    large_activity(0u, L, n_prev, n_cand, prev, ab, tb, tg, snap, st);
                    wsync();                                // every candidate classified
                    n_act = sh.wcnt[0];
                    publish();
                    if (L >= 0) large_undo(0u, L, n_act, ab, v);
                    wsync();                                // the helpers are done
                    n_new = sh.wcnt[1];
                }
                if (L >= 0) {
                // measurements of the column at L on inactive qubits
                    if (cur > 0u && s.ent_l[cur - 1u] == (uint32_t)L) {
                        uint32_t l0 = 0, h0 = cur;
                        while (l0 < h0) {
                            const uint32_t mid = (l0 + h0) >> 1;
                            if (s.ent_l[mid] < (uint32_t)L) l0 = mid + 1; else h0 = mid;
                        }
                        for (uint32_t base = l0; base < cur; base += 32u) {
                            const uint32_t i = base + lane;
                            bool add = false;
                            uint32_t q = 0;
                            if (i < cur) {
                                const unsigned long long w = s.ent_w[i];
                                const uint32_t qv = s.ent_q[i];
                                q = qv & 0x7FFFFFFFu;
                                // an active qubit had the word applied by its gate above
                                if (w != 0ull && s.bits[q] == 0) {
                                    if (qv >> 31) s.pl[q].y ^= w; else s.pl[q].x ^= w;
                                    s.bits[q] = kAdded;
                                    add = true;
                                }
                            }
                            const unsigned m = __ballot_sync(0xFFFFFFFFu, add);
                            if (add) s.add[n_new + __popc(m & lt_mask)] = (uint16_t)q;
                            n_new += __popc(m);
                        }
                        cur = l0;
                    }
                }
                __syncwarp();
                // the emitters see no fast-forward step: the walker releases
                // its window for them too
                if (lane == 0u) {
                    if (ff) mbar_arrive_count(&sh.win_free[slot], NE + 1u);
                    else mbar_arrive(&sh.win_free[slot]);
                }
                if (ff) ff_buf ^= 1u;
                else st++;
                slot = slot == 0u ? nring - 1u : slot - 1u;   // window L - 1
                n_prev = n_act;
                n_add = n_new;
                if (L < 0) break;
                if (emit_lo >= 0 && L == emit_lo) break;        // the segment's last step
                if (L == 0) { L = -1; continue; }
                if (n_prev + n_add == 0u && (uint32_t)(L - 1) < lmin) break;
                L--;
            }
            // the helpers leave
            if (WW > 1u) {
                if (lane == 0u) sh.wstep.cmd = 0u;
                wsync();
            }
            if (ok) {
                // the end-of-column step: the emitters leave on it
                const uint32_t b = st & 1u;
                if ((tfree_pend >> b) & 1u) {
                    if (!wait_warp(&sh.tab_free[b], (tfree_par >> b) & 1u)) ok = false;
                    else tfree_par ^= 1u << b;
                }
                if (ok) {
                    tfree_pend |= 1u << b;
                    if (lane == 0u) {
                        sh.step[b] = StepDesc{0, 0u, 0u, 1u};
                        sh.stop_layer = L;
                    }
                    __syncwarp();
                    if (lane == 0u) mbar_arrive(&sh.tab_full[b]);
                    st++;
                }
            }
            if (lane == 0u) *(volatile uint32_t *)&sh.walk_done = 1u;
        } else if (!producer) {
            // ---- emitters: the noise rows of each published step, one
            // mask word per Pauli component (mechanism) of each row
            for (;;) {
                const uint32_t b = st & 1u;
                if (!wait_warp(&sh.tab_full[b], (tfull_par >> b) & 1u)) break;
                tfull_par ^= 1u << b;
                const StepDesc sd = sh.step[b];
                if (sd.end) {
                    __syncwarp();
                    if (lane == 0u) mbar_arrive(&sh.tab_free[b]);
                    st++;
                    break;
                }
                // the walker waited for the window before it published the
                // step, so the window's contents are visible here through the
                // step's release and acquire
                const uint32_t slot = sd.slot;
                const Window v = sh.desc[slot];
                const ulonglong2 *const tb = tab_of(s, b);
                const uint32_t *const tg = tag_of(s, b);
                const uint16_t *const ab = act_of(s, b);
                const uint32_t n_act = sd.n_act;
                const bool after = sd.layer >= 0;
                const uint32_t stamp = st;
                // planes of qubit x in this step (0 unless x is active)
                auto planes = [&](uint32_t x) -> ulonglong2 {
                    const uint32_t t = tg[x];
                    const ulonglong2 p = tb[x];
                    return t == stamp ? p : make_ulonglong2(0ull, 0ull);
                };
                warp_prefetch();
                // A wide step's work is dealt out twice, so that every lane
                // has work whatever the row kinds: each emitter warp takes a
                // contiguous share of the active qubits, 32 at a time (one
                // per lane); their (qubit, noise row) pairs go one per lane;
                // then the Pauli components of those rows (one mechanism
                // each), again one per lane.  A lane finds its pair or its
                // component by a binary search over the lanes' running
                // counts and fetches what it needs from the lane holding it.
                auto row_word = [&](uint2 r, uint32_t q) -> unsigned long long {
                    const uint32_t kind = row_kind(r);
                    if (kind < K_XERR) return 0ull;
                    const uint32_t ra = row_a(r), rb = row_b(r);
                    const bool two = kind == K_DEP2;
                    const ulonglong2 pa = planes(ra);
                    const ulonglong2 pb = two ? planes(rb) : make_ulonglong2(0ull, 0ull);
                    if (two && q == rb && (pa.x | pa.y) != 0ull) return 0ull;
                    const uint32_t nc = two ? nc_dep2 : (kind == K_DEP1 ? nc_dep1 : 1u);
                    if (l16 >= nc) return 0ull;
                    const unsigned long long codes =
                        two ? 0x0EBF7D639CA25184ull : (kind == K_DEP1 ? 0x321ull : (kind == K_XERR ? 1ull : 2ull));
                    const uint32_t code = (uint32_t)(codes >> (4u * l16)) & 0xFu;
                    return ((code & 1u) ? pa.x : 0ull) ^ ((code & 2u) ? pa.y : 0ull) ^
                           ((code & 4u) ? pb.x : 0ull) ^ ((code & 8u) ? pb.y : 0ull);
                };
                auto scan = [&](uint32_t x) -> uint32_t {     // inclusive, over the lanes
#pragma unroll
                    for (uint32_t o = 1; o < 32u; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                        if (lane >= o) x += y;
                    }
                    return x;
                };
                // the lane whose range of the running count holds j
                auto lane_of = [&](uint32_t incl, uint32_t j) -> uint32_t {
                    uint32_t lo = 0;
#pragma unroll
                    for (uint32_t h = 16; h; h >>= 1) {
                        const uint32_t y = __shfl_sync(0xFFFFFFFFu, incl, lo + h - 1u);
                        if (y <= j) lo += h;
                    }
                    return lo;
                };
                auto emit = [&](uint32_t mech, unsigned long long w) {
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, w != 0ull);
                    if (m == 0u) return;
                    const uint32_t cnt = (uint32_t)__popc(m);
                    if (!warp_room(cnt)) return;
                    if (w != 0ull)
                        B.records[ck_pos + __popc(m & lt_mask)] =
                            make_uint4(mech_base + mech, col_tag, (uint32_t)w, (uint32_t)(w >> 32));
                    ck_pos += cnt;
                };
                if (!WIDE || n_act <= 4u * NE) {
                    // a narrow step (an observable's walk): each half-warp
                    // takes one active qubit and evaluates its rows two at a
                    // time, one Pauli component per lane -- the shortest
                    // chain per step
                    for (uint32_t base = 2u * ew; base < n_act; base += 2u * NE) {
                        const uint32_t c = base + half;
                        const bool valid = c < n_act;
                        const uint32_t q = valid ? ab[c] : 0u;
                        uint32_t a0 = 0, a1 = 0;
                        if (after) { a0 = v.aoff[q]; a1 = v.aoff[q + 1u]; }
                        const uint32_t b0 = v.boff[q], b1 = v.boff[q + 1u];
                        const uint32_t na = valid ? a1 - a0 : 0u;
                        const uint32_t n = valid ? na + (b1 - b0) : 0u;
                        const uint32_t nmax = max(n, __shfl_xor_sync(0xFFFFFFFFu, n, 16));
                        for (uint32_t i = 0; i < nmax; i += 2u) {
                            uint2 r0 = make_uint2(0u, 0u), r1 = make_uint2(0u, 0u);
                            if (i < n) r0 = v.lists[i < na ? a0 + i : v.n_after + b0 + (i - na)];
                            if (i + 1u < n) r1 = v.lists[i + 1u < na ? a0 + i + 1u : v.n_after + b0 + (i + 1u - na)];
                            const unsigned long long w0 = row_word(r0, q), w1 = row_word(r1, q);
                            emit(r0.y + l16, w0);
                            emit(r1.y + l16, w1);
                        }
                    }
                } else {
                    const uint32_t per = (n_act + NE - 1u) / NE;
                    const uint32_t c_lo = min(ew * per, n_act), c_hi = min(c_lo + per, n_act);
                    for (uint32_t c0 = c_lo; c0 < c_hi; c0 += 32u) {
                        const uint32_t c = c0 + lane;
                        const uint32_t q = c < c_hi ? ab[c] : 0u;
                        uint32_t a0 = 0, na = 0, b0 = 0, nb = 0;
                        if (c < c_hi) {
                            if (after) {
                                a0 = v.aoff[q];
                                na = v.aoff[q + 1u] - a0;
                            }
                            b0 = v.boff[q];
                            nb = v.boff[q + 1u] - b0;
                        }
                        const uint32_t rinc = scan(na + nb);
                        const uint32_t n_rows = __shfl_sync(0xFFFFFFFFu, rinc, 31);
                        for (uint32_t j0 = 0; j0 < n_rows; j0 += 32u) {
                            // this lane's (qubit, row) pair
                            const uint32_t j = j0 + lane;
                            const uint32_t o = lane_of(rinc, j);
                            const uint32_t oq = __shfl_sync(0xFFFFFFFFu, q, o);
                            const uint32_t oa0 = __shfl_sync(0xFFFFFFFFu, a0, o);
                            const uint32_t ona = __shfl_sync(0xFFFFFFFFu, na, o);
                            const uint32_t ob0 = __shfl_sync(0xFFFFFFFFu, b0, o);
                            const uint32_t k = j - __shfl_sync(0xFFFFFFFFu, rinc - na - nb, o);
                            uint2 r = make_uint2(0u, 0u);
                            if (j < n_rows) r = v.lists[k < ona ? oa0 + k : v.n_after + ob0 + (k - ona)];
                            // the row's components (a two-qubit row listed
                            // under both qubits is emitted from its first
                            // qubit when that one is active)
                            const uint32_t kind = row_kind(r);
                            uint32_t nc = 0;
                            if (j < n_rows && kind >= K_XERR) {
                                const bool two = kind == K_DEP2;
                                nc = two ? nc_dep2 : (kind == K_DEP1 ? nc_dep1 : 1u);
                                if (two && oq == row_b(r) && tg[row_a(r)] == stamp) nc = 0u;
                            }
                            const uint32_t cinc = scan(nc);
                            const uint32_t n_comp = __shfl_sync(0xFFFFFFFFu, cinc, 31);
                            for (uint32_t i0 = 0; i0 < n_comp; i0 += 32u) {
                                // this lane's component: its row from the lane
                                // holding it, the planes from the snapshot
                                const uint32_t i = i0 + lane;
                                const uint32_t ro = lane_of(cinc, i);
                                const uint32_t comp = i - __shfl_sync(0xFFFFFFFFu, cinc - nc, ro);
                                const uint2 rr = make_uint2(__shfl_sync(0xFFFFFFFFu, r.x, ro), __shfl_sync(0xFFFFFFFFu, r.y, ro));
                                const uint32_t rm = rr.y;
                                unsigned long long w = 0ull;
                                if (i < n_comp) {
                                    const uint32_t rk = row_kind(rr);
                                    const ulonglong2 pa = planes(row_a(rr));
                                    const ulonglong2 pb = rk == K_DEP2 ? planes(row_b(rr)) : make_ulonglong2(0ull, 0ull);
                                    const unsigned long long codes =
                                        rk == K_DEP2 ? 0x0EBF7D639CA25184ull
                                                     : (rk == K_DEP1 ? 0x321ull : (rk == K_XERR ? 1ull : 2ull));
                                    const uint32_t code = (uint32_t)(codes >> (4u * comp)) & 0xFu;
                                    w = ((code & 1u) ? pa.x : 0ull) ^ ((code & 2u) ? pa.y : 0ull) ^
                                        ((code & 4u) ? pb.x : 0ull) ^ ((code & 8u) ? pb.y : 0ull);
                                }
                                emit(rm + comp, w);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0u) {
                    mbar_arrive(&sh.tab_free[b]);
                    mbar_arrive(&sh.win_free[slot]);
                }
                st++;
            }
        } else {
            // ---- producer: windows lmax, lmax - 1, ..., -1 until the walker
            // leaves the column, each into a slot its last window released
            auto post = [&](int L) {
                const uint32_t need = L > 0 ? (uint32_t)L : 0u;
                if (seg_lo == 0xFFFFFFFFu || need < seg_lo || (uint32_t)L + 1u >= seg_lo + (uint32_t)kSegCache) {
                    seg_lo = (uint32_t)L + 2u > (uint32_t)kSegCache ? (uint32_t)L + 2u - (uint32_t)kSegCache : 0u;
                    const uint32_t n = min((uint32_t)kSegCache, C.n_layers + 1u - seg_lo);
                    __syncwarp();
                    for (uint32_t i = lane; i < n; i += 32u) s.segc[i] = seg_g[seg_lo + i];
                    __syncwarp();
                }
                if (lane != 0u) return;
                const uint4 s1 = s.segc[L + 1 - (int)seg_lo];
                const uint32_t n_after = L >= 0 ? s.segc[L - (int)seg_lo].y : 0u;
                const uint32_t list_start = 2u * s1.x - n_after;
                const uint32_t list_n = n_after + s1.z;
                const uint32_t slot = slot_of(L);
                Window &d = sh.desc[slot];
                d.n_after = n_after;
                if (nbuf >= 2u && list_n + 1u <= list_cap) {
                    unsigned char *dst = s.win + (size_t)slot * wbytes;
                    const unsigned char *qsrc = L >= 0 ? qbase + (size_t)L * geo.bytes + 2u * geo.qb : qbase;
                    const uint32_t qbytes = L >= 0 ? 4u * geo.nq4 + 4u * geo.qb : 2u * geo.qb;
                    const uint32_t delta = list_start & 1u;
                    const uint32_t lbytes = list_n ? ((list_n + delta) * 8u + 15u) & ~15u : 0u;
                    d.lists = reinterpret_cast<const uint2 *>(dst + windex) + delta;
                    if (L >= 0) {
                        d.gate = reinterpret_cast<const uint32_t *>(dst);
                        d.aoff = reinterpret_cast<const uint16_t *>(dst + 4u * geo.nq4);
                        d.boff = d.aoff + geo.qb;
                    } else {
                        d.gate = nullptr;
                        d.aoff = nullptr;
                        d.boff = reinterpret_cast<const uint16_t *>(dst);
                    }
                    mbar_expect_tx(&sh.win_full[slot], qbytes + lbytes);
                    bulk_load(dst, qsrc, qbytes, &sh.win_full[slot]);
                    if (lbytes) bulk_load(dst + windex, lbase + list_start - delta, lbytes, &sh.win_full[slot]);
                } else {
                    d.lists = lbase + list_start;
                    if (L >= 0) {
                        const unsigned char *p = qbase + (size_t)L * geo.bytes + 2u * geo.qb;
                        d.gate = reinterpret_cast<const uint32_t *>(p);
                        d.aoff = reinterpret_cast<const uint16_t *>(p + 4u * geo.nq4);
                        d.boff = d.aoff + geo.qb;
                    } else {
                        d.gate = nullptr;
                        d.aoff = nullptr;
                        d.boff = reinterpret_cast<const uint16_t *>(qbase);
                    }
                    mbar_arrive(&sh.win_full[slot]);
                }
            };
            volatile uint32_t *const done_v = &sh.walk_done;
            int Lp = (int)lmax;
            while (Lp >= -1) {
                const uint32_t slot = slot_of(Lp);
                if ((free_pend >> slot) & 1u) {
                    uint32_t got = 0;
                    if (lane == 0u) {
                        uint32_t it = 0;
                        for (; it < wlim; it++) {
                            if (mbar_try_wait(&sh.win_free[slot], (free_par >> slot) & 1u)) { got = 1u; break; }
                            if ((it & 15u) == 15u && (*done_v || *tmo_v)) break;
                        }
                        if (it == wlim) *tmo_v = 1u;
                    }
                    if (!__shfl_sync(0xFFFFFFFFu, got, 0)) break;
                    free_par ^= 1u << slot;
                    free_pend &= ~(1u << slot);
                }
                const uint32_t stop = lane == 0u ? (*done_v | *tmo_v) : 0u;
                if (__shfl_sync(0xFFFFFFFFu, stop, 0)) break;
                if (!stall) {
                    post(Lp);
                    post_par ^= 1u << slot;
                    posted_any |= 1u << slot;
                }
                free_pend |= 1u << slot;
                Lp--;
            }
            if (lane == 0u) sh.posted_lo = Lp + 1;
        }
        __syncthreads();
        if (!sh.tmo) {
            // windows posted below the walk's last layer were never used:
            // their copies land (consumers absorb the phase), and no release
            // comes for them
            const int stop_layer = sh.stop_layer, posted_lo = sh.posted_lo;
            for (int k2 = stop_layer - 1; k2 >= posted_lo; k2--) {
                const uint32_t slot = slot_of(k2);
                if (producer) {
                    free_pend &= ~(1u << slot);
                } else if (warp == 0u) {
                    // the walker warp that tracks the window phases
                    if (!wait_bar(&sh.win_full[slot], (full_par >> slot) & 1u)) break;
                    full_par ^= 1u << slot;
                }
            }
        }
        __syncthreads();
        if (sh.tmo) {
            if (threadIdx.x == 0) report(B.status, GP_ERR_TIMEOUT, 1u, gcol, 0u);
            break;
        }
    }
    flush_chunks();
    // The grouping's first kernel adds into every mechanism's key and stores
    // its words into the mechanism's inline slots: after an L2 flush (or
    // another compile) those lines are in DRAM, and each atomic or partial
    // store waits for its sector.  The first quarter of the blocks that
    // walked, in the order they run out of work, prefetch the two arrays into
    // L2 while the last walks finish; the last blocks, which end the kernel,
    // issue nothing.  Only when the arrays fit well within L2.
    if (threadIdx.x == 0 && sh.worked) {
        const size_t nm = min(B.status->n_mech, P.max_mech);
        const size_t bytes = nm * (sizeof(unsigned long long) +
                                   kInlineWords * (sizeof(uint32_t) + sizeof(unsigned long long)));
        if (nm && bytes <= P.l2_prefetch_max) {
            const uint32_t R = max(1u, min(gridDim.x, P.n_items) / 4u);
            const uint32_t t = atomicAdd(&B.status->pf_ticket, 1u);
            if (t < R) {
                l2_prefetch_share(B.mech_key, (nm * sizeof(unsigned long long)) & ~(size_t)15u, t, R);
                l2_prefetch_share(B.inl_col, nm * kInlineWords * sizeof(uint32_t), t, R);
                l2_prefetch_share(B.inl_word, nm * kInlineWords * sizeof(unsigned long long), t, R);
            }
        }
    }
    // copies still in flight (after a timeout) land before the block exits
    if (producer && lane == 0u) {
        for (uint32_t i = 0; i < nring; i++)
            if ((posted_any >> i) & 1u) mbar_wait_bounded(&sh.win_full[i], ((post_par >> i) & 1u) ^ 1u);
    }
}

}  // namespace

size_t stage1_dynamic_smem_limit(int device) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    cudaFuncAttributes fa{};
    size_t stat = 0;
    for (uint32_t split : {0u, 1u, 2u})
        for (uint32_t t : {128u, 256u, 512u, 1024u}) {
            if (cudaFuncGetAttributes(&fa, stage1_kernel_ptr(t, split)) != cudaSuccess) return 0;
            stat = std::max(stat, fa.sharedSizeBytes);
        }
    return (size_t)optin > stat ? (size_t)optin - stat : 0;
}

Stage1Shape stage1_shape(uint32_t maxq, uint32_t blocks_per_sm, size_t limit) {
    Stage1Shape sh{};
    // k blocks per SM share the SM's shared memory (1 KB of it reserved per block)
    const size_t per_sm = limit + 1024;
    const size_t budget = blocks_per_sm > 1 ? std::min(limit, per_sm / blocks_per_sm - 1024) : limit;
    const uint32_t wi = window_index_bytes(maxq);
    // the role-split walk when its tables and at least two windows fit, else
    // the block-wide walk.  The deepest ring whose windows hold a whole layer
    // (about two list entries per qubit: every noise row after the gates of
    // L and before those of L + 1, two-qubit rows twice) is preferred; a
    // window that does not fit is read from global memory, which costs more
    // than a shallower ring.
    const size_t layer_entries = 2 * (size_t)maxq + 64;
    for (int split = 1; split >= 0; split--) {
        const size_t base = split ? split_base_bytes(maxq) : smem_base_bytes(maxq);
        for (uint32_t pass = 0; pass < 2; pass++)
        for (uint32_t nbuf = split ? 4u : 3u; nbuf >= 2; nbuf--) {
            const size_t want = pass == 0 ? layer_entries : 512;
            if (budget < base + (size_t)nbuf * (wi + want * 8)) continue;
            size_t cap = (budget - base) / nbuf;
            cap = (cap - wi) / 8;
            cap = std::min<size_t>(cap, 4096) & ~(size_t)15;
            sh.nbuf = nbuf;
            sh.list_cap = (uint32_t)cap;
            sh.wbytes = wi + (uint32_t)cap * 8;
            sh.smem = base + (size_t)nbuf * sh.wbytes;
            sh.split = (uint32_t)split;
            return sh;
        }
    }
    // no room for window buffers: every window is read from global memory
    sh.nbuf = 0;
    sh.list_cap = 0;
    sh.wbytes = 0;
    sh.smem = smem_base_bytes(maxq);
    sh.split = 0;
    return sh;
}

const void *stage1_kernel_ptr(uint32_t threads, uint32_t split) {
    if (split == 2u) {
        switch (threads) {
        case 128: return (const void *)stage1_split_kernel<128, true>;
        case 256: return (const void *)stage1_split_kernel<256, true>;
        case 1024: return (const void *)stage1_split_kernel<1024, true>;
        default: return (const void *)stage1_split_kernel<512, true>;
        }
    }
    if (split) {
        switch (threads) {
        case 128: return (const void *)stage1_split_kernel<128, false>;
        case 256: return (const void *)stage1_split_kernel<256, false>;
        case 1024: return (const void *)stage1_split_kernel<1024, false>;
        default: return (const void *)stage1_split_kernel<512, false>;
        }
    }
    switch (threads) {
    case 128: return (const void *)stage1_kernel<128>;
    case 256: return (const void *)stage1_kernel<256>;
    case 1024: return (const void *)stage1_kernel<1024>;
    default: return (const void *)stage1_kernel<512>;
    }
}

void launch_stage1(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t maxq, const Stage1Shape &sh, bool wide,
                   cudaStream_t s, uint32_t *launches) {
    // records per warp chunk: the chunk tails the warps may leave unused fit
    // the pool's slack (kPoolSlack records)
    const uint64_t warps = (uint64_t)grid * (threads / 32u - 1u);
    uint32_t wchunk = (uint32_t)std::min<uint64_t>(256, kPoolSlack / std::max<uint64_t>(warps, 1)) & ~31u;
    if (wchunk < 32u) wchunk = 32u;
    if (sh.split && wide) {
        switch (threads) {
        case 128: stage1_split_kernel<128, true><<<grid, 128, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        case 256: stage1_split_kernel<256, true><<<grid, 256, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        case 1024: stage1_split_kernel<1024, true><<<grid, 1024, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        default: stage1_split_kernel<512, true><<<grid, 512, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        }
    } else if (sh.split) {
        switch (threads) {
        case 128: stage1_split_kernel<128, false><<<grid, 128, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        case 256: stage1_split_kernel<256, false><<<grid, 256, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        case 1024: stage1_split_kernel<1024, false><<<grid, 1024, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        default: stage1_split_kernel<512, false><<<grid, 512, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        }
    } else {
        switch (threads) {
        case 128: stage1_kernel<128><<<grid, 128, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        case 256: stage1_kernel<256><<<grid, 256, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        case 1024: stage1_kernel<1024><<<grid, 1024, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        default: stage1_kernel<512><<<grid, 512, sh.smem, s>>>(b, maxq, sh.nbuf, sh.list_cap, sh.wbytes, wchunk); break;
        }
    }
    *launches += 1;
}

}  // namespace gpdem
