// stage2.cu -- probability aggregation (Sec. 3.2) and the adjoint.
//
// scatter    records of stage 1 {mechanism, column, word} are appended to
//            per-mechanism slots (the pool cleans itself as it is read)
// group      one thread per mechanism: sort its mask words by column, hash
//            them, insert into an open-addressing table whose claims are
//            verified word by word (so grouping is exact whatever the hash
//            does), and add t_i = -log(1 - 2 q_i) to the class sum as an
//            exact 128-bit fixed-point integer.  Sums of t give
//            1 - 2P = prod(1 - 2 q_i) = exp(-sum t_i) (Eq. pmerge), and integer
//            addition makes them independent of the order the atomics land.
// compact    classes are numbered by their smallest mechanism id (a scan of
//            "is leader" flags), then each leader writes its hyperedge: the
//            ascending detector list, the observable word, P = -expm1(-T)/2 and
//            w = log1p(-P) - log(P).
// finalize   per-mechanism class ids; the table slots that were used are
//            cleared for the next compile.
// backward   dP/dp_i = (1 - 2P)/2 * dt_i/dp and dw/dP = -1 / (P (1 - P)),
//            summed per noise location in fixed point.
#include "common.cuh"

namespace gpdem {

namespace {

// Load the mask words of mechanism m, sorted by column id (insertion sort;
// masks hold a handful of words).
__device__ __forceinline__ uint32_t load_sorted(const Buffers &B, uint32_t m, uint32_t S, uint32_t cnt,
                                                uint32_t *col, unsigned long long *w) {
    const size_t base = (size_t)m * S;
    for (uint32_t i = 0; i < cnt; i++) {
        uint32_t c = B.slot_col[base + i];
        unsigned long long x = B.slot_word[base + i];
        uint32_t j = i;
        while (j > 0 && col[j - 1] > c) { col[j] = col[j - 1]; w[j] = w[j - 1]; j--; }
        col[j] = c;
        w[j] = x;
    }
    return cnt;
}

__device__ __forceinline__ bool same_mask(const Buffers &B, uint32_t rep, uint32_t S, uint32_t cnt,
                                          const uint32_t *col, const unsigned long long *w) {
    if (__ldcg(&B.mech_cnt[rep]) != cnt) return false;
    uint32_t c2[kMaxMaskWords];
    unsigned long long w2[kMaxMaskWords];
    load_sorted(B, rep, S, cnt, c2, w2);
    for (uint32_t i = 0; i < cnt; i++)
        if (c2[i] != col[i] || w2[i] != w[i]) return false;
    return true;
}

__global__ void scatter_kernel(Buffers B) {
    if (*(volatile uint32_t *)&B.status->code != 0u) return;
    const Params &P = *B.params;
    const uint32_t n = min(B.status->rec_count, P.rec_cap), S = P.mask_words;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 r = B.records[i];
        if (r.x == kNone) continue;
        B.records[i].x = kNone;
        const uint32_t pos = atomicAdd(&B.mech_cnt[r.x], 1u);
        if (pos < S) {
            B.slot_col[(size_t)r.x * S + pos] = r.y;
            B.slot_word[(size_t)r.x * S + pos] = ((unsigned long long)r.w << 32) | r.z;
        } else {
            report(B.status, GP_ERR_CAPACITY, 4u, r.x, pos + 1);
        }
    }
}

__global__ void group_kernel(Buffers B) {
    const Params &P = *B.params;
    if (*(volatile uint32_t *)&B.status->code != 0u) return;
    const uint32_t N = B.status->n_mech, S = P.mask_words;
    const uint32_t cap_mask = (1u << P.table_log2) - 1u;
    const float *noise = P.noise;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
        const uint32_t cnt = B.mech_cnt[m];
        if (cnt == 0u || cnt > S) { B.slot_of[m] = kNone; continue; }
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
        uint32_t col[kMaxMaskWords];
        unsigned long long w[kMaxMaskWords];
        load_sorted(B, m, S, cnt, col, w);
        unsigned long long h = 0x243F6A8885A308D3ull;
        for (uint32_t i = 0; i < cnt; i++) {
            h = mix64(h ^ (0x9E3779B97F4A7C15ull * (col[i] + 1ull)));
            h = mix64(h ^ w[i]);
        }
        const uint32_t key_hi = (uint32_t)(h >> 32);
        const unsigned long long mine = ((unsigned long long)key_hi << 32) | m;
        uint32_t pos = (uint32_t)h & cap_mask, slot = kNone;
        for (uint32_t probe = 0; probe <= cap_mask; probe++) {
            unsigned long long e = __ldcg(&B.table[pos]);
            if (e == kEmpty) {
                const unsigned long long old = atomicCAS(&B.table[pos], kEmpty, mine);
                if (old == kEmpty) { slot = pos; break; }
                e = old;
            }
            if ((uint32_t)(e >> 32) == key_hi && same_mask(B, (uint32_t)e, S, cnt, col, w)) { slot = pos; break; }
            pos = (pos + 1u) & cap_mask;
        }
        if (slot == kNone) {
            report(B.status, GP_ERR_CAPACITY, 6u, m, cap_mask + 1u);
            B.slot_of[m] = kNone;
            continue;
        }
        B.slot_of[m] = slot;
        atomicMin(&B.tab_min[slot], m);
        unsigned long long lo, hi;
        to_fixed(t, kProbShift, lo, hi);
        acc128_add(&B.tab_acc[2 * (size_t)slot], lo, hi);
    }
}

// leader flag and detector count of mechanism m
__device__ __forceinline__ uint2 leader_info(const Buffers &B, uint32_t m, uint32_t S) {
    const uint32_t slot = B.slot_of[m];
    if (slot == kNone || B.tab_min[slot] != m) return make_uint2(0, 0);
    const uint32_t cnt = B.mech_cnt[m];
    uint32_t dets = 0;
    for (uint32_t i = 0; i < cnt; i++) {
        const size_t sidx = (size_t)m * S + i;
        if (!(B.slot_col[sidx] & kObsColFlag)) dets += __popcll(B.slot_word[sidx]);
    }
    return make_uint2(1, dets);
}

constexpr int kScanThreads = 256;
constexpr int kPerThread = kMechPerBlockScan / kScanThreads;

__global__ void __launch_bounds__(kScanThreads) compact_count_kernel(Buffers B) {
    if (*(volatile uint32_t *)&B.status->code != 0u) return;
    const uint32_t N = B.status->n_mech, S = B.params->mask_words;
    const uint32_t m0 = blockIdx.x * kMechPerBlockScan;
    if (m0 >= N) return;
    uint2 acc = make_uint2(0, 0);
    for (int i = 0; i < kPerThread; i++) {
        const uint32_t m = m0 + threadIdx.x * kPerThread + i;
        if (m < N) { const uint2 v = leader_info(B, m, S); acc.x += v.x; acc.y += v.y; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xFFFFFFFFu, acc.x, o);
        acc.y += __shfl_down_sync(0xFFFFFFFFu, acc.y, o);
    }
    __shared__ uint2 red[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint2 s = make_uint2(0, 0);
        for (int w = 0; w < kScanThreads / 32; w++) { s.x += red[w].x; s.y += red[w].y; }
        B.blk_sums[blockIdx.x] = s;
    }
}

// one block: exclusive scan of the per-block (edges, detector ids) counts
__global__ void __launch_bounds__(kScanThreads) compact_scan_kernel(Buffers B) {
    if (*(volatile uint32_t *)&B.status->code != 0u) return;
    const uint32_t N = B.status->n_mech;
    const uint32_t nb = (N + kMechPerBlockScan - 1) / kMechPerBlockScan;
    __shared__ uint32_t warp_tmp[kScanThreads / 32];
    __shared__ uint32_t carry_e, carry_d;
    if (threadIdx.x == 0) { carry_e = 0; carry_d = 0; }
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += kScanThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint2 v = i < nb ? B.blk_sums[i] : make_uint2(0, 0);
        uint32_t te, td;
        const uint32_t oe = block_exclusive_scan<kScanThreads>(v.x, warp_tmp, te);
        const uint32_t od = block_exclusive_scan<kScanThreads>(v.y, warp_tmp, td);
        if (i < nb) B.blk_off[i] = make_uint2(carry_e + oe, carry_d + od);
        __syncthreads();
        if (threadIdx.x == 0) { carry_e += te; carry_d += td; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        B.status->n_edges = carry_e;
        B.status->n_det_entries = carry_d;
        B.status->n_scan_blocks = nb;
        if ((unsigned long long)carry_d > B.params->max_det_entries)
            report(B.status, GP_ERR_CAPACITY, 7u, carry_d, (uint32_t)(B.params->max_det_entries > 0xFFFFFFFFull ? 0xFFFFFFFFull : B.params->max_det_entries));
        else
            B.det_off[carry_e] = carry_d;
    }
}

__global__ void __launch_bounds__(kScanThreads) compact_write_kernel(Buffers B) {
    if (*(volatile uint32_t *)&B.status->code != 0u) return;
    const uint32_t N = B.status->n_mech, S = B.params->mask_words;
    const uint32_t m0 = blockIdx.x * kMechPerBlockScan;
    if (m0 >= N) return;
    uint2 v[kPerThread];
    uint32_t ne = 0, nd = 0;
    for (int i = 0; i < kPerThread; i++) {
        const uint32_t m = m0 + threadIdx.x * kPerThread + i;
        v[i] = (m < N) ? leader_info(B, m, S) : make_uint2(0, 0);
        ne += v[i].x;
        nd += v[i].y;
    }
    __shared__ uint32_t warp_tmp[kScanThreads / 32];
    uint32_t te, td;
    const uint2 boff = B.blk_off[blockIdx.x];
    uint32_t e = block_exclusive_scan<kScanThreads>(ne, warp_tmp, te) + boff.x;
    uint32_t d = block_exclusive_scan<kScanThreads>(nd, warp_tmp, td) + boff.y;
    for (int i = 0; i < kPerThread; i++) {
        if (!v[i].x) continue;
        const uint32_t m = m0 + threadIdx.x * kPerThread + i;
        const uint32_t slot = B.slot_of[m];
        const unsigned long long info = B.mech_info[m];
        const uint32_t b = (uint32_t)(info >> 48);
        const uint32_t col_base = B.circ[b].col_base;
        uint32_t col[kMaxMaskWords];
        unsigned long long w[kMaxMaskWords];
        const uint32_t cnt = load_sorted(B, m, S, B.mech_cnt[m], col, w);
        unsigned long long obs = 0ull;
        uint32_t dd = d;
        for (uint32_t j = 0; j < cnt; j++) {
            if (col[j] & kObsColFlag) { obs ^= w[j]; continue; }
            unsigned long long x = w[j];
            const uint32_t base_id = (col[j] - col_base) * 64u;
            while (x) {
                const int bit = __ffsll((long long)x) - 1;
                B.det_idx[dd++] = base_id + (uint32_t)bit;
                x &= x - 1ull;
            }
        }
        const float T = fixed_to_float(B.tab_acc[2 * (size_t)slot], B.tab_acc[2 * (size_t)slot + 1], kProbShift);
        const float Pc = -0.5f * expm1f(-T);
        B.det_off[e] = d;
        B.obs_mask[e] = obs;
        B.prob[e] = Pc;
        B.logodds[e] = log1pf(-Pc) - logf(Pc);
        B.class_slot[e] = slot;
        B.edge_circ[e] = b;
        B.tab_class[slot] = e;
        d = dd;
        e++;
    }
    // edges per circuit: one atomic per circuit present in the warp
    for (int i = 0; i < kPerThread; i++) {
        const uint32_t m = m0 + threadIdx.x * kPerThread + i;
        const bool lead = v[i].x != 0u;
        const uint32_t b = lead ? (uint32_t)(B.mech_info[m] >> 48) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
        if (lead && (__ffs(peers) - 1) == (int)(threadIdx.x & 31u))
            atomicAdd(&B.circ_edges[b], (uint32_t)__popc(peers));
    }
}

__global__ void finalize_mech_kernel(Buffers B) {
    if (*(volatile uint32_t *)&B.status->code != 0u) return;
    const uint32_t N = B.status->n_mech;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
        const uint32_t slot = B.slot_of[m];
        B.mech_class[m] = (slot == kNone) ? -1 : (int32_t)B.tab_class[slot];
        B.mech_cnt[m] = 0u;
    }
}

__global__ void finalize_table_kernel(Buffers B) {
    if (*(volatile uint32_t *)&B.status->code != 0u) return;
    const uint32_t E = B.status->n_edges;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const uint32_t slot = B.class_slot[e];
        B.table[slot] = kEmpty;
        B.tab_min[slot] = kNone;
        B.tab_acc[2 * (size_t)slot] = 0ull;
        B.tab_acc[2 * (size_t)slot + 1] = 0ull;
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

}  // namespace

void launch_group(const Buffers &b, uint32_t grid, uint32_t threads, cudaStream_t s, uint32_t *launches) {
    scatter_kernel<<<grid, threads, 0, s>>>(b);
    group_kernel<<<grid, threads, 0, s>>>(b);
    *launches += 2;
}

void launch_compact(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t max_scan_blocks,
                    uint32_t max_mech, cudaStream_t s, uint32_t *launches) {
    (void)max_mech;
    compact_count_kernel<<<max_scan_blocks, kScanThreads, 0, s>>>(b);
    compact_scan_kernel<<<1, kScanThreads, 0, s>>>(b);
    compact_write_kernel<<<max_scan_blocks, kScanThreads, 0, s>>>(b);
    finalize_mech_kernel<<<grid, threads, 0, s>>>(b);
    finalize_table_kernel<<<grid, threads, 0, s>>>(b);
    *launches += 5;
}

void launch_backward(const Buffers &b, const float *g_prob, const float *g_logodds, float *g_noise,
                     uint32_t n_mech, uint32_t n_loc, uint32_t grid, uint32_t threads, cudaStream_t s,
                     uint32_t *launches) {
    backward_mech_kernel<<<grid, threads, 0, s>>>(b, g_prob, g_logodds, n_mech);
    backward_loc_kernel<<<grid, threads, 0, s>>>(b, g_noise, n_loc);
    *launches += 2;
}

}  // namespace gpdem
