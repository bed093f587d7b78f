// stage2.cu -- probability aggregation (Sec. 3.2) and the adjoint.
//
// Stage 1 leaves mask-word records {mechanism, column, word} in a pool (every
// position of the pool handed out is either a record or marked empty).
// Stage 2:
//   scatter    per record: one 64-bit atomic add into the mechanism's key
//              (word count in the low byte, the sum of its words' hashes
//              above: equal masks give equal keys whatever the order the
//              words arrive in), whose old value says where the word goes:
//              one of the mechanism's kInlineWords slots, or its overflow
//              list
//   group      one thread per mechanism: hash the key, claim or join a slot
//              of an open-addressing table whose claims are verified on the
//              whole mask (word count and every (column, word) pair), so the
//              grouping is exact whatever the hash does; keep the smallest
//              member and add t_i = -log(1 - 2 q_i) to the class sum as an
//              exact 128-bit fixed-point integer: 1 - 2P = prod(1 - 2 q_i) =
//              exp(-sum t_i) (Eq. pmerge), and integer addition makes the sum
//              independent of the order in which the atomics land
//   compact    classes are numbered by their smallest member: a two-pass scan
//              whose input is read straight from the table (1 and the class's
//              detector count for the smallest member of a class, else 0)
//              lists the leaders in edge order with their detector offsets;
//              then one thread per hyperedge writes it: ascending detector
//              ids, observable word, P = -expm1(-T) / 2 and
//              w = log1p(-P) - log(P)
//   finalize   per-mechanism class ids; keys, overflow heads and used table
//              slots are cleared for the next compile
//   backward   dP/dp_i = (1 - 2P) / 2 * dt_i/dp and dw/dP = -1 / (P (1 - P)),
//              summed per noise location in fixed point
// Every grid is fixed by the driver's bounds, so the whole sequence can be
// captured once and replayed.
#include <algorithm>

#include "common.cuh"

namespace gpdem {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;                          // elements per thread
constexpr uint32_t kScanBlock = kScanThreads * kScanPer;

__device__ __forceinline__ uint2 add2(uint2 a, uint2 b) { return make_uint2(a.x + b.x, a.y + b.y); }

// block-wide exclusive scan of two channels
__device__ __forceinline__ uint2 block_scan2(uint2 v, uint32_t *tmp, uint2 &total) {
    uint32_t tx, ty;
    const uint32_t ex = block_exclusive_scan<kScanThreads>(v.x, tmp, tx);
    const uint32_t ey = block_exclusive_scan<kScanThreads>(v.y, tmp, ty);
    total = make_uint2(tx, ty);
    return make_uint2(ex, ey);
}

// ---- hierarchical exclusive scan of uint2 values ---------------------------
// Chunks of kScanBlock values; each block takes chunks blockIdx.x,
// blockIdx.x + gridDim.x, ... (trip counts uniform over the block, so the
// barriers of the block scans are reached by every thread), and the grid is
// capped by the SM count rather than sized by the driver's bounds.
// Pass 1: the sum of every chunk.
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint2 *in, const uint32_t *n_ptr,
                                                                   uint2 *bsum, const Status *st) {
    if (st->code != 0u) return;
    const uint32_t n = *n_ptr;
    const uint32_t nb = (n + kScanBlock - 1) / kScanBlock;
    __shared__ uint32_t tmp[kScanThreads / 32];
    for (uint32_t c = blockIdx.x; c < nb; c += gridDim.x) {
        const uint32_t b0 = c * kScanBlock;
        uint2 acc = make_uint2(0, 0);
        for (int k = 0; k < kScanPer; k++) {
            const uint32_t i = b0 + threadIdx.x * kScanPer + k;
            if (i < n) acc = add2(acc, in[i]);
        }
        uint2 tot;
        block_scan2(acc, tmp, tot);
        if (threadIdx.x == 0) bsum[c] = tot;
    }
}

// Pass 2: exclusive prefix of every value.  Each chunk adds up the sums of
// the chunks before it itself (a few hundred values), so no separate pass
// scans the chunk sums; block 0 also writes out[n] = the total.
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const uint2 *in, const uint32_t *n_ptr,
                                                                 const uint2 *bsum, uint2 *out, const Status *st) {
    if (st->code != 0u) return;
    const uint32_t n = *n_ptr;
    const uint32_t nb = (n + kScanBlock - 1) / kScanBlock;
    __shared__ uint32_t tmp[kScanThreads / 32];
    if (blockIdx.x == 0) {
        uint2 all = make_uint2(0, 0);
        for (uint32_t i = threadIdx.x; i < nb; i += kScanThreads) all = add2(all, bsum[i]);
        uint2 tot;
        block_scan2(all, tmp, tot);
        if (threadIdx.x == 0) out[n] = tot;
    }
    for (uint32_t c = blockIdx.x; c < nb; c += gridDim.x) {
        const uint32_t b0 = c * kScanBlock;
        uint2 before = make_uint2(0, 0);
        for (uint32_t i = threadIdx.x; i < c; i += kScanThreads) before = add2(before, bsum[i]);
        uint2 prefix;
        block_scan2(before, tmp, prefix);
        uint2 v[kScanPer];
        uint2 acc = make_uint2(0, 0);
        for (int k = 0; k < kScanPer; k++) {
            const uint32_t i = b0 + threadIdx.x * kScanPer + k;
            v[k] = i < n ? in[i] : make_uint2(0, 0);
            acc = add2(acc, v[k]);
        }
        uint2 tot;
        uint2 run = add2(block_scan2(acc, tmp, tot), prefix);
        for (int k = 0; k < kScanPer; k++) {
            const uint32_t i = b0 + threadIdx.x * kScanPer + k;
            if (i < n) out[i] = run;
            run = add2(run, v[k]);
        }
    }
}


// ---- per-mechanism words ----------------------------------------------------
// Hash of one (column, word) pair; a mechanism's key adds these up (mod 2^64,
// low byte masked off for the word count).
__device__ __forceinline__ unsigned long long word_hash(uint32_t col, unsigned long long w) {
    return mix64(w ^ (0x9E3779B97F4A7C15ull * (col + 1ull)));
}

// Each thread moves kScatterILP records per round, with every load and atomic
// of the round in flight before the first store (the kernel is bound by their
// latency).
constexpr int kScatterILP = 3;

__global__ void __launch_bounds__(512, 4) scatter_kernel(Buffers B) {
    if (B.status->code != 0u) return;
    const Params &P = *B.params;
    const uint32_t n = min(B.status->rec_count, P.rec_cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kScatterILP * stride) {
        uint4 r[kScatterILP];
#pragma unroll
        for (int u = 0; u < kScatterILP; u++) {
            const uint32_t i = i0 + u * stride;
            r[u] = i < n ? __ldcs(&B.records[i]) : make_uint4(kNone, 0u, 0u, 0u);
        }
        uint32_t k[kScatterILP];
#pragma unroll
        for (int u = 0; u < kScatterILP; u++) {
            if (r[u].x == kNone) continue;
            const unsigned long long w = ((unsigned long long)r[u].w << 32) | r[u].z;
            const unsigned long long add = (word_hash(r[u].y, w) & ~0xFFull) | 1ull;
            k[u] = (uint32_t)(atomicAdd(&B.mech_key[r[u].x], add) & 0xFFull);
        }
#pragma unroll
        for (int u = 0; u < kScatterILP; u++) {
            if (r[u].x == kNone) continue;
            const uint32_t m = r[u].x;
            const unsigned long long w = ((unsigned long long)r[u].w << 32) | r[u].z;
            if (k[u] < (uint32_t)kInlineWords) {
                B.inl_col[(size_t)kInlineWords * m + k[u]] = r[u].y;
                B.inl_word[(size_t)kInlineWords * m + k[u]] = w;
            } else {
                const uint32_t j = atomicAdd(&B.status->ov_count, 1u);
                if (j < P.ov_cap) {
                    const uint32_t next = atomicExch(&B.ov_head[m], j);
                    B.ov_rec[j] = make_uint4(r[u].y, r[u].z, r[u].w, next);
                    B.ov_mech[j] = m;
                } else {
                    report(B.status, GP_ERR_CAPACITY, 11u, j, P.ov_cap);
                }
            }
        }
    }
}

// the (column, word) pairs of mechanism m with `cnt` words: the inline slots,
// then its overflow list
__device__ __forceinline__ void load_words(const Buffers &B, uint32_t m, uint32_t cnt, uint32_t *col,
                                           unsigned long long *w) {
    const uint4 c4 = *reinterpret_cast<const uint4 *>(&B.inl_col[(size_t)kInlineWords * m]);
    const ulonglong2 w01 = *reinterpret_cast<const ulonglong2 *>(&B.inl_word[(size_t)kInlineWords * m]);
    const ulonglong2 w23 = *reinterpret_cast<const ulonglong2 *>(&B.inl_word[(size_t)kInlineWords * m + 2]);
    col[0] = c4.x; col[1] = c4.y; col[2] = c4.z; col[3] = c4.w;
    w[0] = w01.x; w[1] = w01.y; w[2] = w23.x; w[3] = w23.y;
    if (cnt > (uint32_t)kInlineWords) {
        uint32_t j = B.ov_head[m];
        for (uint32_t i = kInlineWords; i < cnt && j != kNone; i++) {
            const uint4 r = B.ov_rec[j];
            col[i] = r.x;
            w[i] = ((unsigned long long)r.z << 32) | r.y;
            j = r.w;
        }
    }
}

// mask of mechanism rep equal to the words col/w of a mechanism with cnt
// words (exact): the counts agree and every word of rep is found at its
// column among them (columns are distinct within a mask)
__device__ __forceinline__ bool same_mask(const Buffers &B, uint32_t rep, uint32_t cnt, const uint32_t *col,
                                          const unsigned long long *w) {
    if ((uint32_t)(B.mech_key[rep] & 0xFFull) != cnt) return false;
    uint32_t rc[kMaxMaskWords];
    unsigned long long rw[kMaxMaskWords];
    load_words(B, rep, cnt, rc, rw);
    for (uint32_t j = 0; j < cnt; j++) {
        uint32_t i = 0;
        while (i < cnt && col[i] != rc[j]) i++;
        if (i == cnt || w[i] != rw[j]) return false;
    }
    return true;
}

// the same for masks of at most kInlineWords words, everything in registers
__device__ __forceinline__ bool same_mask_inline(const Buffers &B, uint32_t rep, uint32_t cnt,
                                                 const uint32_t (&col)[kInlineWords],
                                                 const unsigned long long (&w)[kInlineWords]) {
    if ((uint32_t)(B.mech_key[rep] & 0xFFull) != cnt) return false;
    const uint4 c4 = *reinterpret_cast<const uint4 *>(&B.inl_col[(size_t)kInlineWords * rep]);
    const ulonglong2 w01 = *reinterpret_cast<const ulonglong2 *>(&B.inl_word[(size_t)kInlineWords * rep]);
    const ulonglong2 w23 = *reinterpret_cast<const ulonglong2 *>(&B.inl_word[(size_t)kInlineWords * rep + 2]);
    const uint32_t rc[kInlineWords] = {c4.x, c4.y, c4.z, c4.w};
    const unsigned long long rw[kInlineWords] = {w01.x, w01.y, w23.x, w23.y};
    bool ok = true;
#pragma unroll
    for (int j = 0; j < kInlineWords; j++) {
        if ((uint32_t)j >= cnt) break;
        bool found = false;
#pragma unroll
        for (int i = 0; i < kInlineWords; i++)
            found |= (uint32_t)i < cnt && col[i] == rc[j] && w[i] == rw[j];
        ok &= found;
    }
    return ok;
}

// Claim or join the class of mechanism m (hash h, detector count dets of
// its mask) in the open-addressing table; eq(rep) says whether the claimant
// rep of a slot with the same tag has the same mask.  Returns the slot, or
// kNone when the table is full.
template <class Eq>
__device__ __forceinline__ uint32_t claim_or_join(const Buffers &B, unsigned long long h, uint32_t m,
                                                  uint32_t cap_mask, uint32_t dets, Eq eq) {
    const uint32_t key_hi = (uint32_t)(h >> 32);
    const unsigned long long mine = ((unsigned long long)key_hi << 32) | m;
    uint32_t pos = (uint32_t)h & cap_mask;
    for (uint32_t probe = 0; probe <= cap_mask; probe++) {
        unsigned long long e = __ldcg(&B.table[pos].entry);
        if (e == kEmpty) {
            const unsigned long long old = atomicCAS(&B.table[pos].entry, kEmpty, mine);
            if (old == kEmpty) {
                B.table[pos].cls = dets;      // the claim records the class's detector count
                return pos;
            }
            e = old;
        }
        if ((uint32_t)(e >> 32) == key_hi && eq((uint32_t)e)) return pos;
        pos = (pos + 1u) & cap_mask;
    }
    return kNone;
}

__global__ void __launch_bounds__(512, 4) group_kernel(Buffers B) {
    const Params &P = *B.params;
    if (B.status->code != 0u) return;
    const uint32_t N = B.status->n_mech, S = P.mask_words;
    const uint32_t cap_mask = (1u << P.table_log2) - 1u;
    const float *noise = P.noise;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
        const unsigned long long key = B.mech_key[m];
        const uint32_t cnt = (uint32_t)(key & 0xFFull);
        if (cnt == 0u) { B.slot_of[m] = kNone; continue; }
        if (cnt > S) {
            report(B.status, GP_ERR_CAPACITY, 4u, m, cnt);
            B.slot_of[m] = kNone;
            continue;
        }
        const unsigned long long info = B.mech_info[m];
        const uint32_t loc = (uint32_t)info;
        const uint32_t kind = (uint32_t)(info >> 32) & 0xFFu;
        const float p = noise[loc];
        if (!(p >= 0.0f && p <= channel_pmax(kind))) {
            report(B.status, GP_ERR_INVALID, 5u, loc, __float_as_uint(p));
            B.slot_of[m] = kNone;
            continue;
        }
        if (p == 0.0f) { B.slot_of[m] = kNone; continue; }
        float c, k;
        channel_ck(kind, c, k);
        float t = -log1pf(-c * p) / k;
        if (!(t < 1048576.0f)) t = 1048576.0f;     // q = 1/2 saturates P at 1/2
        // collisions cost probes, never correctness (claims are verified on
        // the whole mask)
        const unsigned long long h = weaken_hash(mix64(key ^ 0x243F6A8885A308D3ull), P.weak_hash);
        uint32_t slot;
        if (cnt <= (uint32_t)kInlineWords) {
            const uint4 c4 = *reinterpret_cast<const uint4 *>(&B.inl_col[(size_t)kInlineWords * m]);
            const ulonglong2 w01 = *reinterpret_cast<const ulonglong2 *>(&B.inl_word[(size_t)kInlineWords * m]);
            const ulonglong2 w23 = *reinterpret_cast<const ulonglong2 *>(&B.inl_word[(size_t)kInlineWords * m + 2]);
            const uint32_t col[kInlineWords] = {c4.x, c4.y, c4.z, c4.w};
            const unsigned long long w[kInlineWords] = {w01.x, w01.y, w23.x, w23.y};
            uint32_t dets = 0;
#pragma unroll
            for (int i = 0; i < kInlineWords; i++)
                if ((uint32_t)i < cnt && !(col[i] & kObsColFlag)) dets += __popcll(w[i]);
            slot = claim_or_join(B, h, m, cap_mask, dets,
                                 [&](uint32_t rep) { return same_mask_inline(B, rep, cnt, col, w); });
        } else {
            uint32_t col[kMaxMaskWords];
            unsigned long long w[kMaxMaskWords];
            load_words(B, m, cnt, col, w);
            uint32_t dets = 0;
            for (uint32_t i = 0; i < cnt; i++)
                if (!(col[i] & kObsColFlag)) dets += __popcll(w[i]);
            slot = claim_or_join(B, h, m, cap_mask, dets,
                                 [&](uint32_t rep) { return same_mask(B, rep, cnt, col, w); });
        }
        if (slot == kNone) {
            report(B.status, GP_ERR_CAPACITY, 6u, m, cap_mask + 1u);
            B.slot_of[m] = kNone;
            continue;
        }
        B.slot_of[m] = slot;
        atomicMin(&B.table[slot].min, m);
        unsigned long long lo, hi;
        to_fixed(t, kProbShift, lo, hi);
        acc128_add(&B.table[slot].acc_lo, lo, hi);
    }
}

// ---- compaction scan: classes numbered by their smallest member ------------
// Input of mechanism i: (1, the detector count its class's claim left in the
// slot) when i is the smallest member of its class, else (0, 0).
__device__ __forceinline__ uint2 leader_in(const Buffers &B, uint32_t i) {
    const uint32_t slot = B.slot_of[i];
    if (slot == kNone) return make_uint2(0u, 0u);
    const uint2 mc = *reinterpret_cast<const uint2 *>(&B.table[slot].min);
    return mc.x == i ? make_uint2(1u, mc.y) : make_uint2(0u, 0u);
}

__global__ void __launch_bounds__(kScanThreads) leader_reduce_kernel(Buffers B) {
    if (B.status->code != 0u) return;
    const uint32_t n = B.status->n_mech;
    const uint32_t nb = (n + kScanBlock - 1) / kScanBlock;
    __shared__ uint32_t tmp[kScanThreads / 32];
    for (uint32_t c = blockIdx.x; c < nb; c += gridDim.x) {
        const uint32_t b0 = c * kScanBlock;
        uint2 v[kScanPer];
#pragma unroll
        for (int k = 0; k < kScanPer; k++) {
            const uint32_t i = b0 + threadIdx.x * kScanPer + k;
            v[k] = i < n ? leader_in(B, i) : make_uint2(0u, 0u);
        }
        uint2 acc = make_uint2(0u, 0u);
#pragma unroll
        for (int k = 0; k < kScanPer; k++) acc = add2(acc, v[k]);
        // the inputs, once, for the second pass (coalesced 8-byte writes)
#pragma unroll
        for (int k = 0; k < kScanPer; k++) {
            const uint32_t i = b0 + threadIdx.x * kScanPer + k;
            if (i < n) B.scan_val[i] = v[k];
        }
        uint2 tot;
        block_scan2(acc, tmp, tot);
        if (threadIdx.x == 0) B.scan_bsum[c] = tot;
    }
}

// Each chunk adds up the sums of the chunks before it itself; every leader
// gets its edge index (its rank) and detector offset: edge_mech[e] = leader,
// det_off[e] = offset.  Block 0 writes the totals (edge count, detector
// entries, det_off[E]) and checks them against the bounds.
__global__ void __launch_bounds__(kScanThreads) leader_down_kernel(Buffers B) {
    if (B.status->code != 0u) return;
    const uint32_t n = B.status->n_mech;
    const uint32_t nb = (n + kScanBlock - 1) / kScanBlock;
    __shared__ uint32_t tmp[kScanThreads / 32];
    if (blockIdx.x == 0) {
        uint2 all = make_uint2(0, 0);
        for (uint32_t i = threadIdx.x; i < nb; i += kScanThreads) all = add2(all, B.scan_bsum[i]);
        uint2 tot;
        block_scan2(all, tmp, tot);
        if (threadIdx.x == 0) {
            if ((unsigned long long)tot.y > B.params->max_det_entries) {
                report(B.status, GP_ERR_CAPACITY, 7u, tot.y,
                       (uint32_t)(B.params->max_det_entries > 0xFFFFFFFFull ? 0xFFFFFFFFull
                                                                            : B.params->max_det_entries));
            } else {
                B.status->n_edges = tot.x;
                B.status->n_det_entries = tot.y;
                B.det_off[tot.x] = tot.y;
            }
        }
    }
    for (uint32_t c = blockIdx.x; c < nb; c += gridDim.x) {
        const uint32_t b0 = c * kScanBlock;
        uint2 before = make_uint2(0, 0);
        for (uint32_t i = threadIdx.x; i < c; i += kScanThreads) before = add2(before, B.scan_bsum[i]);
        uint2 prefix;
        block_scan2(before, tmp, prefix);
        uint2 v[kScanPer];
        uint2 acc = make_uint2(0, 0);
#pragma unroll
        for (int k = 0; k < kScanPer; k++) {
            const uint32_t i = b0 + threadIdx.x * kScanPer + k;
            v[k] = i < n ? B.scan_val[i] : make_uint2(0u, 0u);
            acc = add2(acc, v[k]);
        }
        uint2 tot;
        uint2 run = add2(block_scan2(acc, tmp, tot), prefix);
#pragma unroll
        for (int k = 0; k < kScanPer; k++) {
            if (v[k].x) {
                B.edge_mech[run.x] = b0 + threadIdx.x * kScanPer + k;
                B.det_off[run.x] = run.y;
            }
            run = add2(run, v[k]);
        }
    }
}

__global__ void compact_write_kernel(Buffers B) {
    if (B.status->code != 0u) return;
    const uint32_t E = B.status->n_edges;
    const uint32_t lane = threadIdx.x & 31u;
    // host output (when set): the same arrays, written into host memory too
    const Params &P = *B.params;
    uint32_t *const h_off = reinterpret_cast<uint32_t *>(P.h_det_off);
    uint32_t *const h_idx = reinterpret_cast<uint32_t *>(P.h_det_idx);
    unsigned long long *const h_obs = reinterpret_cast<unsigned long long *>(P.h_obs);
    float *const h_prob = reinterpret_cast<float *>(P.h_prob);
    float *const h_lo = reinterpret_cast<float *>(P.h_logodds);
    const uint64_t h_ecap = P.h_edges_cap, h_dcap = P.h_det_cap;
    if (h_off && E == 0u && blockIdx.x == 0 && threadIdx.x == 0) h_off[0] = 0u;
    for (uint32_t base = blockIdx.x * blockDim.x; base < E; base += gridDim.x * blockDim.x) {
        const uint32_t e = base + threadIdx.x;
        uint32_t b = 0xFFFFFFFFu;
        uint32_t d0 = 0u, d1 = 0u;          // this edge's detector ids [d0, d1)
        if (e < E) {
            const uint32_t m = B.edge_mech[e];
            uint32_t d = B.det_off[e];
            d0 = d;
            const uint32_t slot = B.slot_of[m];
            const unsigned long long info = B.mech_info[m];
            b = (uint32_t)(info >> 48);
            const uint32_t col_base = B.circ[b].col_base;
            const uint32_t cnt = (uint32_t)(B.mech_key[m] & 0xFFull);
            uint32_t col[kMaxMaskWords];
            unsigned long long w[kMaxMaskWords];
            load_words(B, m, cnt, col, w);
            unsigned long long obs = 0ull;
            // words in ascending column order (selection), so the detector
            // ids come out ascending
            uint32_t prev = 0u;
            for (uint32_t k = 0; k < cnt; k++) {
                uint32_t cmin = 0xFFFFFFFFu, jmin = 0u;
                for (uint32_t j = 0; j < cnt; j++) {
                    const uint32_t c = col[j];
                    if ((k == 0u || c > prev) && c < cmin) { cmin = c; jmin = j; }
                }
                prev = cmin;
                unsigned long long x = w[jmin];
                if (cmin & kObsColFlag) { obs ^= x; continue; }
                const uint32_t base_id = (cmin - col_base) * 64u;
                while (x) {
                    const int bit = __ffsll((long long)x) - 1;
                    B.det_idx[d++] = base_id + (uint32_t)bit;
                    x &= x - 1ull;
                }
            }
            d1 = d;
            const TabSlot &ts = B.table[slot];
            const float T = fixed_to_float(ts.acc_lo, ts.acc_hi, kProbShift);
            const float Pc = -0.5f * expm1f(-T);
            const float lo = log1pf(-Pc) - logf(Pc);
            B.obs_mask[e] = obs;
            B.prob[e] = Pc;
            B.logodds[e] = lo;
            B.class_slot[e] = slot;
            B.edge_circ[e] = b;
            B.table[slot].cls = e;
            if (h_off && e < h_ecap) {
                h_off[e] = d0;
                h_obs[e] = obs;
                h_prob[e] = Pc;
                h_lo[e] = lo;
                if (e + 1u == E && E <= h_ecap) h_off[E] = d1;
            }
        }
        if (h_off) {
            // the warp's edges are consecutive, so their detector ids are one
            // range: copied to the host lane by lane (coalesced stores)
            __syncwarp();
            const uint32_t lo_w = __shfl_sync(0xFFFFFFFFu, d0, 0);
            const unsigned has = __ballot_sync(0xFFFFFFFFu, e < E);
            const uint32_t hi_w = has ? __shfl_sync(0xFFFFFFFFu, d1, 31 - __clz(has)) : lo_w;
            for (uint32_t i = lo_w + lane; i < hi_w && i < h_dcap; i += 32u) h_idx[i] = B.det_idx[i];
        }
        // edges per circuit: one atomic per circuit present in the warp
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
        if (e < E && (uint32_t)(__ffs(peers) - 1) == lane) atomicAdd(&B.circ_edges[b], (uint32_t)__popc(peers));
    }
}

// per-mechanism class ids and cleared keys (four consecutive mechanisms per
// thread: one 16-byte load of their slots, one 16-byte store of their ids,
// two of their keys), used table slots cleared (one edge per thread),
// overflow heads reset: disjoint fields, one pass
__global__ void finalize_kernel(Buffers B) {
    if (B.status->code != 0u) return;
    const uint32_t N = B.status->n_mech, E = B.status->n_edges;
    const uint32_t OV = min(B.status->ov_count, B.params->ov_cap);
    const uint32_t N4 = (N + 3u) / 4u;
    const uint32_t M = max(max(N4, E), OV);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        const uint32_t cs = i < E ? B.class_slot[i] : kNone;
        const uint32_t om = i < OV ? B.ov_mech[i] : kNone;
        if (i < N4) {
            const bool full = 4u * i + 3u < N;
            uint32_t sl[4];
            if (full) {
                const uint4 v = *reinterpret_cast<const uint4 *>(&B.slot_of[4u * i]);
                sl[0] = v.x; sl[1] = v.y; sl[2] = v.z; sl[3] = v.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++) sl[u] = 4u * i + u < N ? B.slot_of[4u * i + u] : kNone;
            }
            int32_t cl[4];
#pragma unroll
            for (int u = 0; u < 4; u++) cl[u] = sl[u] == kNone ? -1 : (int32_t)B.table[sl[u]].cls;
            if (full) {
                *reinterpret_cast<int4 *>(&B.mech_class[4u * i]) = make_int4(cl[0], cl[1], cl[2], cl[3]);
                ulonglong2 *k2 = reinterpret_cast<ulonglong2 *>(&B.mech_key[4u * i]);
                k2[0] = make_ulonglong2(0ull, 0ull);
                k2[1] = make_ulonglong2(0ull, 0ull);
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (4u * i + u < N) {
                        B.mech_class[4u * i + u] = cl[u];
                        B.mech_key[4u * i + u] = 0ull;
                    }
            }
        }
        if (om != kNone) B.ov_head[om] = kNone;
        // cls is left alone: other threads may still be reading it (a claim
        // overwrites it in the next compile)
        if (cs != kNone) {
            TabSlot &ts = B.table[cs];
            ts.entry = kEmpty;
            ts.min = kNone;
            *reinterpret_cast<uint4 *>(&ts.acc_lo) = make_uint4(0u, 0u, 0u, 0u);   // acc_lo, acc_hi
        }
    }
}

__global__ void backward_mech_kernel(Buffers B, const float *g_prob, const float *g_logodds, uint32_t N) {
    const float *noise = B.params->noise;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
        const int32_t e = B.mech_class[m];
        if (e < 0) continue;
        const unsigned long long info = B.mech_info[m];
        const uint32_t loc = (uint32_t)info;
        const uint32_t kind = (uint32_t)(info >> 32) & 0xFFu;
        const float p = noise[loc];
        const float Pc = B.prob[e];
        const float one_m_2P = 1.0f - 2.0f * Pc;
        if (one_m_2P <= 0.0f) continue;            // saturated class: P = 1/2
        const float gp = g_prob ? g_prob[e] : 0.0f;
        const float gw = g_logodds ? g_logodds[e] : 0.0f;
        const float gbar = gp - gw / (Pc * (1.0f - Pc));
        float c, k;
        channel_ck(kind, c, k);
        const float dtdp = (c / k) / (1.0f - c * p);
        const float g = gbar * 0.5f * one_m_2P * dtdp;
        acc128_add_signed(&B.gacc[2 * (size_t)loc], g, kGradShift);
    }
}

__global__ void backward_loc_kernel(Buffers B, float *g_noise, uint32_t n_loc) {
    for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n_loc; l += gridDim.x * blockDim.x) {
        const unsigned long long lo = B.gacc[2 * (size_t)l], hi = B.gacc[2 * (size_t)l + 1];
        g_noise[l] = fixed_to_float_signed(lo, hi, kGradShift);
        B.gacc[2 * (size_t)l] = 0ull;
        B.gacc[2 * (size_t)l + 1] = 0ull;
    }
}

__global__ void init_table_kernel(TabSlot *t, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        t[i].entry = kEmpty;
        t[i].min = kNone;
        t[i].cls = 0;
        t[i].acc_lo = 0ull;
        t[i].acc_hi = 0ull;
    }
}

}  // namespace

// exclusive scan of n (read on the device) uint2 values: out[i] = sum of
// in[0..i), out[n] = the total; chunks of 2048 values, two passes (the
// server's selection scans)
static uint32_t scan_grid(uint32_t max_n, uint32_t n_sms) {
    const uint32_t chunks = (max_n + kScanBlock - 1) / kScanBlock;
    return std::max(1u, std::min(chunks, 8u * std::max(n_sms, 1u)));
}

void launch_scan(const Buffers &B, const uint2 *in, const uint32_t *n_ptr, uint2 *out, uint32_t max_n, uint32_t n_sms,
                 cudaStream_t s, uint32_t *launches) {
    const uint32_t grid1 = scan_grid(max_n, n_sms);
    scan_reduce_kernel<<<grid1, kScanThreads, 0, s>>>(in, n_ptr, B.scan_bsum, B.status);
    scan_down_kernel<<<grid1, kScanThreads, 0, s>>>(in, n_ptr, B.scan_bsum, out, B.status);
    *launches += 2;
}

void launch_group(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t max_mech, cudaStream_t s,
                  uint32_t *launches) {
    (void)max_mech;
    scatter_kernel<<<grid, threads, 0, s>>>(b);
    group_kernel<<<grid, threads, 0, s>>>(b);
    *launches += 2;
}

void launch_compact(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t max_mech, uint32_t n_sms,
                    cudaStream_t s, uint32_t *launches) {
    const uint32_t grid1 = scan_grid(max_mech, n_sms);
    leader_reduce_kernel<<<grid1, kScanThreads, 0, s>>>(b);
    leader_down_kernel<<<grid1, kScanThreads, 0, s>>>(b);
    compact_write_kernel<<<grid, threads, 0, s>>>(b);
    finalize_kernel<<<grid, threads, 0, s>>>(b);
    *launches += 4;
}

void launch_backward(const Buffers &b, const float *g_prob, const float *g_logodds, float *g_noise,
                     uint32_t n_mech, uint32_t n_loc, uint32_t grid, uint32_t threads, cudaStream_t s,
                     uint32_t *launches) {
    backward_mech_kernel<<<grid, threads, 0, s>>>(b, g_prob, g_logodds, n_mech);
    backward_loc_kernel<<<grid, threads, 0, s>>>(b, g_noise, n_loc);
    *launches += 2;
}

void launch_init_table(TabSlot *t, size_t n, cudaStream_t s) {
    init_table_kernel<<<1024, 256, 0, s>>>(t, n);
}

}  // namespace gpdem
