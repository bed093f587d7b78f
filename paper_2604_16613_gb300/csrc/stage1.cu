// stage1.cu -- error-equivalence-class generation (Sec. 3.1).
//
// The straight-line program of Eq. slp is linear over GF(2), so every 64
// detectors (one "word column") can be propagated on their own.  A thread
// block takes one word column at a time from a work queue and keeps, in
// shared memory, two 64-bit bit-planes per qubit of that column:
//   xs[q] bit j = detector j flips under an X error on q at the current time
//   zs[q] bit j = the same for a Z error.
// It walks the TICK layers backward from the latest measurement of the
// column's detectors (Eq. init-slp seeds the bits there) and stops once every
// plane is zero and no earlier measurement of the column remains, so each
// column only pays for the layers its detecting regions cover.  Per layer:
//   P1  mask words of noise rows that act before the layer's gates of the
//       previous (later-in-time) layer, and the qubit -> gate-row table of
//       this layer (double-buffered by layer parity)
//   P2  mask words of noise rows that act after this layer's gates
//   P3  the gates undone backward (H swaps the planes, S: x ^= z,
//       CX(c,t): x_c ^= x_t and z_t ^= z_c, CZ(a,b): x_a ^= z_b and
//       x_b ^= z_a; measurements XOR in the column's detector bits; resets
//       clear the planes after checking determinism).
// A noise component's mask word is the XOR of the planes named by its Pauli
// (Y = X xor Z; two-qubit terms combine both qubits, Sec. 2.3.4); non-zero
// words are appended to the mechanism's slots with one atomic counter per
// mechanism.
#include "common.cuh"

namespace gpdem {

namespace {

struct Smem {
    unsigned long long *xs, *zs;
    uint32_t *gtab[2];
    uint32_t *ent_m;
    unsigned long long *ent_w;
};

__device__ __forceinline__ Smem carve(unsigned char *base, uint32_t maxq) {
    Smem s;
    s.xs = reinterpret_cast<unsigned long long *>(base);
    s.zs = s.xs + maxq;
    s.ent_w = s.zs + maxq;
    s.gtab[0] = reinterpret_cast<uint32_t *>(s.ent_w + kMaxEntries);
    s.gtab[1] = s.gtab[0] + maxq;
    s.ent_m = s.gtab[1] + maxq;
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

// Emit the mask words of the noise rows of layer [rs, re) that act on the
// requested side of the layer's gates (before == true: before the gates).
template <int NT>
__device__ __forceinline__ void emit_layer(const Buffers &B, const CircuitDev &C, const Smem &s,
                                           uint32_t rs, uint32_t re, const uint32_t *gtab,
                                           bool before, uint32_t gcol_tag, uint32_t b,
                                           uint32_t level, uint32_t S) {
    for (uint32_t r = rs + threadIdx.x; r < re; r += NT) {
        const uint4 op = __ldg(&C.ops[r]);
        const uint32_t k = op.x;
        if (!is_noise(k)) continue;
        const uint32_t a = op.y;
        const uint32_t ga = gtab[a];
        const bool bef_a = (ga >= rs && ga < re && ga > r);
        bool side = bef_a;
        unsigned long long xa = s.xs[a], za = s.zs[a], xb = 0ull, zb = 0ull;
        if (k == K_DEP2) {
            const uint32_t bq = op.z;
            const uint32_t gb = gtab[bq];
            const bool bef_b = (gb >= rs && gb < re && gb > r);
            if (bef_b != bef_a) {
                report(B.status, GP_ERR_INVALID, 3u, b, r);
                continue;
            }
            xb = s.xs[bq];
            zb = s.zs[bq];
        }
        if (side != before) continue;
        if ((xa | za | xb | zb) == 0ull) continue;
        const uint32_t nc = n_comp(k, level);
        const uint32_t mbase = C.mech_base + B.aux[C.op_base + r];
        for (uint32_t c = 0; c < nc; c++) {
            const uint32_t code = comp_planes(k, c);
            unsigned long long w = 0ull;
            if (code & 1u) w ^= xa;
            if (code & 2u) w ^= za;
            if (code & 4u) w ^= xb;
            if (code & 8u) w ^= zb;
            if (w == 0ull) continue;
            const uint32_t mech = mbase + c;
            const uint32_t idx = atomicAdd(&B.mech_cnt[mech], 1u);
            if (idx == 0u) {
                B.mech_info[mech] = (unsigned long long)(C.loc_base + op.w) |
                                    ((unsigned long long)k << 32) |
                                    ((unsigned long long)c << 40) |
                                    ((unsigned long long)b << 48);
            }
            if (idx < S) {
                const size_t slot = (size_t)mech * S + idx;
                B.slot_col[slot] = gcol_tag;
                B.slot_word[slot] = w;
            } else {
                report(B.status, GP_ERR_CAPACITY, 4u, mech, idx + 1);
            }
        }
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) stage1_kernel(Buffers B, uint32_t maxq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem s = carve(smem_raw, maxq);
    const Params &P = *B.params;
    const uint32_t level = P.level, S = P.mask_words;
    __shared__ uint32_t s_item, s_bail, s_nent, s_lmax, s_lmin;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(&B.status->queue_head, 1u);
            s_bail = (*(volatile uint32_t *)&B.status->code) != 0u;
            s_nent = 0;
            s_lmax = 0;
            s_lmin = 0xFFFFFFFFu;
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= P.n_items || s_bail) break;
        const uint32_t gcol = B.items[item];
        const uint32_t b = B.col_circ[gcol];
        const CircuitDev &C = B.circ[b];
        const uint32_t local = gcol - C.col_base;
        const bool is_obs = (C.n_obs > 0u) && (local == C.n_cols - 1u);
        const uint32_t gcol_tag = gcol | (is_obs ? kObsColFlag : 0u);
        const uint32_t nq = C.n_qubits;

        for (uint32_t q = threadIdx.x; q < nq; q += NT) {
            s.xs[q] = 0ull;
            s.zs[q] = 0ull;
            s.gtab[0][q] = kNone;
            s.gtab[1][q] = kNone;
        }
        // (measurement, word) entries of this column (Eq. init-slp)
        if (!is_obs) {
            const uint32_t j0 = local * 64u, j1 = min(j0 + 64u, C.n_det);
            for (uint32_t j = j0 + threadIdx.x; j < j1; j += NT) {
                const uint32_t row = B.det_row[C.det_base + j];
                const uint4 op = C.ops[row];
                const uint32_t mb = B.aux[C.op_base + row];
                for (uint32_t i = 0; i < op.z; i++) {
                    const uint32_t e = atomicAdd(&s_nent, 1u);
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
                    const uint32_t e = atomicAdd(&s_nent, 1u);
                    if (e < (uint32_t)kMaxEntries) {
                        s.ent_m[e] = mb - C.recs[op.y + i];
                        s.ent_w[e] = 1ull << op.w;
                    }
                }
            }
        }
        __syncthreads();
        const uint32_t n_ent_raw = s_nent;
        if (n_ent_raw > (uint32_t)kMaxEntries) {
            if (threadIdx.x == 0) report(B.status, GP_ERR_CAPACITY, 5u, gcol, n_ent_raw);
            __syncthreads();
            continue;
        }
        const uint32_t n_ent = n_ent_raw;
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
            atomicMax(&s_lmax, L);
            atomicMin(&s_lmin, L);
        }
        __syncthreads();
        const uint32_t lmax = s_lmax, lmin = s_lmin;
        const uint32_t m_lo = s.ent_m[0], m_hi = s.ent_m[n_ent - 1];
        const uint32_t *ls = B.layer_start + C.layer_base;

        // backward wave over the layers
        uint32_t L = lmax;
        bool stopped = false;
        for (;;) {
            const uint32_t rs = ls[L], re = ls[L + 1];
            // P1: before-gate noise of layer L+1, and the gate table of layer L
            if (L < lmax) emit_layer<NT>(B, C, s, re, ls[L + 2], s.gtab[(L + 1) & 1u], true, gcol_tag, b, level, S);
            uint32_t *gt = s.gtab[L & 1u];
            for (uint32_t r = rs + threadIdx.x; r < re; r += NT) {
                const uint4 op = __ldg(&C.ops[r]);
                if (!is_gate(op.x)) continue;
                const uint32_t old = atomicExch(&gt[op.y], r);
                bool dup = (old != kNone && old >= rs && old < re);
                if (is_gate2(op.x)) {
                    const uint32_t old2 = atomicExch(&gt[op.z], r);
                    dup |= (old2 != kNone && old2 >= rs && old2 < re);
                }
                if (dup) report(B.status, GP_ERR_INVALID, 4u, b, r);
            }
            __syncthreads();
            // P2: after-gate noise of layer L (planes are still zero at lmax)
            if (L < lmax) emit_layer<NT>(B, C, s, rs, re, gt, false, gcol_tag, b, level, S);
            __syncthreads();
            // P3: undo the gates of layer L
            for (uint32_t r = rs + threadIdx.x; r < re; r += NT) {
                const uint4 op = __ldg(&C.ops[r]);
                const uint32_t k = op.x, a = op.y;
                switch (k) {
                case K_H: { const unsigned long long t = s.xs[a]; s.xs[a] = s.zs[a]; s.zs[a] = t; break; }
                case K_S: s.xs[a] ^= s.zs[a]; break;
                case K_CX: s.xs[a] ^= s.xs[op.z]; s.zs[op.z] ^= s.zs[a]; break;
                case K_CZ: { const unsigned long long za = s.zs[a], zb = s.zs[op.z]; s.xs[a] ^= zb; s.xs[op.z] ^= za; break; }
                case K_R: case K_M: case K_MR: {
                    if (s.zs[a] != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, r, gcol);
                    if (k == K_R || k == K_MR) { s.xs[a] = 0ull; s.zs[a] = 0ull; }
                    if (k != K_R) s.xs[a] ^= meas_word(s, n_ent, B.aux[C.op_base + r], m_lo, m_hi);
                    break;
                }
                case K_RX: case K_MX: case K_MRX: {
                    if (s.xs[a] != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, r, gcol);
                    if (k == K_RX || k == K_MRX) { s.xs[a] = 0ull; s.zs[a] = 0ull; }
                    if (k != K_RX) s.zs[a] ^= meas_word(s, n_ent, B.aux[C.op_base + r], m_lo, m_hi);
                    break;
                }
                default: break;
                }
            }
            int nonzero = 0;
            if (L <= lmin) {
                for (uint32_t q = threadIdx.x; q < nq; q += NT)
                    if ((s.xs[q] | s.zs[q]) != 0ull) { nonzero = 1; break; }
            }
            const int any = __syncthreads_or(nonzero);
            if (L <= lmin && !any) { stopped = true; break; }
            if (L == 0u) break;
            L--;
        }
        if (!stopped) {
            // before-gate noise of layer 0, then the |0> initial state
            emit_layer<NT>(B, C, s, ls[0], ls[1], s.gtab[0], true, gcol_tag, b, level, S);
            for (uint32_t q = threadIdx.x; q < nq; q += NT)
                if (s.zs[q] != 0ull) report(B.status, GP_ERR_NONDETERMINISTIC, b, 0xFFFFFFFFu, gcol);
        }
        __syncthreads();
    }
}

}  // namespace

size_t stage1_smem_bytes(uint32_t maxq) {
    return (size_t)maxq * (8 + 8 + 4 + 4) + (size_t)kMaxEntries * (8 + 4);
}

const void *stage1_kernel_ptr(uint32_t threads) {
    switch (threads) {
    case 128: return (const void *)stage1_kernel<128>;
    case 512: return (const void *)stage1_kernel<512>;
    default: return (const void *)stage1_kernel<256>;
    }
}

void launch_stage1(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t maxq, cudaStream_t s,
                   uint32_t *launches) {
    const size_t smem = stage1_smem_bytes(maxq);
    switch (threads) {
    case 128: stage1_kernel<128><<<grid, 128, smem, s>>>(b, maxq); break;
    case 512: stage1_kernel<512><<<grid, 512, smem, s>>>(b, maxq); break;
    default: stage1_kernel<256><<<grid, 256, smem, s>>>(b, maxq); break;
    }
    *launches += 1;
}

}  // namespace gpdem
