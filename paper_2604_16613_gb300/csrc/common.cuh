// common.cuh -- device-side structures and helpers shared by the kernels of
// the detector-error-model compiler (lowering, stage 1, stage 2, adjoint).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gpdem.h"

namespace gpdem {

// ---------------------------------------------------------------------------
// limits and constants
// ---------------------------------------------------------------------------
constexpr int kRowTile = 512;           // circuit rows per lowering tile
constexpr int kLowerThreads = 256;      // 2 rows per thread
constexpr int kMaxEntries = 1024;       // (measurement, word) pairs per column
constexpr int kMaxMaskWords = 16;       // hard cap of mask words per mechanism
constexpr int kInlineWords = 4;         // mask words kept beside each mechanism;
                                        // the rest go to the overflow list
constexpr int kMechPerBlockScan = 1024; // mechanisms per compaction block
constexpr uint64_t kPoolSlack = 1ull << 22;  // record-pool slack for unused chunk tails
constexpr int kPackThreads = 1024;      // layer index block size
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr unsigned long long kEmpty = 0xFFFFFFFFFFFFFFFFull;
// stage-1 work item: column id | segment << kSegShift (segments of a long
// observable walk that separate blocks share)
constexpr uint32_t kSegShift = 30;
constexpr uint32_t kColMask = (1u << kSegShift) - 1u;
constexpr uint32_t kMaxSegments = 3;
constexpr uint32_t kMaxObsWords = 8;      // observable word columns per circuit
constexpr uint32_t kObsColFlag = 0x80000000u;   // set on the column id of an
                                                // observable word in a mask

// ---------------------------------------------------------------------------
// per-circuit descriptor (one per circuit of a batch)
// ---------------------------------------------------------------------------
struct CircuitDev {
    const uint4 *ops;          // rows {kind, a, b, c}
    const uint32_t *recs;      // record lookbacks
    uint32_t n_ops, n_recs;
    uint32_t n_qubits, n_det, n_obs, n_loc;
    uint32_t col_base, n_cols; // global word columns: detector words, then
                               // n_ocols observable words
    uint32_t n_ocols, obs_per; // observable words; observables per word
                               // (word k holds observables k*obs_per ..)
    uint32_t pad0, pad1;
    uint32_t det_base, loc_base, op_base, tile_first;
    uint32_t n_tiles;
    // filled by the lowering kernels
    uint32_t n_layers, layer_base;
    uint32_t n_meas, meas_base;
    uint32_t n_mech, mech_base;
    uint32_t qidx_off;         // start of the circuit's layer index blocks
                               // (16-byte units)
};
static_assert(sizeof(CircuitDev) % 16 == 0, "CircuitDev alignment");

// compile-wide parameters (uploaded once per compile)
struct Params {
    uint32_t n_circuits;
    uint32_t n_tiles;
    uint32_t n_items;           // stage-1 work items (= total columns)
    uint32_t level;
    uint32_t n_cols_total;
    uint32_t n_loc_total;
    uint32_t table_log2;        // hash table capacity = 1 << table_log2
    uint32_t mask_words;        // S: slots per mechanism
    uint64_t max_det_entries;
    uint32_t max_mech;
    uint32_t max_layer_slots;
    uint32_t max_meas;
    uint32_t max_ops;
    const float *noise;         // concatenated noise vectors
    uint32_t rec_cap;           // capacity of the record pool
    uint32_t max_qubits;
    uint64_t qidx_cap16;        // capacity of the layer index arena (16-byte units)
    // test knobs (gp_debug)
    uint32_t weak_hash;         // 0 full hash, 1 constant tag, 2 constant hash
    uint32_t wait_limit;        // polls of a bounded wait (never 0 on the device)
    uint32_t stall_windows;     // 1: stage 1 stages no window
    uint32_t ov_cap;            // capacity of the overflow word list
    uint32_t obs_segments;      // most work items of one observable walk
    uint64_t l2_prefetch_max;   // bytes of per-mechanism grouping arrays stage 1
                                // prefetches into L2 (0: none; about 3/4 of L2)
    // host output (0: none): the hyperedges also written into host memory
    unsigned long long h_det_off, h_det_idx, h_obs, h_prob, h_logodds;
    uint64_t h_edges_cap, h_det_cap;
};

// device status block (read back by the host after every compile)
struct Status {
    uint32_t code;              // first gp_status error reported
    uint32_t info[3];
    uint32_t n_mech;            // total mechanisms (lowering)
    uint32_t n_edges;           // hyperedges
    uint32_t n_det_entries;
    uint32_t n_scan_blocks;
    uint32_t queue_head;        // stage-1 work queue
    uint32_t rec_count;         // records handed out from the pool
    uint32_t ov_count;          // overflow words taken (mechanisms with more
                                // than kInlineWords words)
    uint32_t pf_ticket;         // stage-1 blocks that ran out of work (L2 prefetch)
    uint32_t pad[4];
};

// one slot of the grouping hash table (one 32-byte sector)
struct TabSlot {
    unsigned long long entry;   // key_hi << 32 | claiming mechanism, or kEmpty
    uint32_t min;               // smallest member mechanism
    uint32_t cls;               // detector count of the mask (set by the claim),
                                // then the hyperedge index once compacted
    unsigned long long acc_lo;  // 128-bit fixed-point sum of t over members
    unsigned long long acc_hi;
};
static_assert(sizeof(TabSlot) == 32, "TabSlot is one sector");

// all device buffers of a driver (pointers into the workspace)
struct Buffers {
    Params *params;
    CircuitDev *circ;
    uint2 *tiles;               // {circuit, first row}
    uint32_t *items;            // stage-1 work order: global column ids
    uint32_t *col_circ;         // circuit of each global column
    uint4 *ops_arena;
    uint32_t *recs_arena;
    float *noise_arena;
    uint32_t *aux;              // per row (indexed by op_base + row)
    uint2 *lists;               // two slots per row: the per-qubit lists of
                                // packed noise rows of each layer (before-gate
                                // lists at the layer's start, after-gate
                                // lists ending at the layer's end)
    unsigned char *qidx;        // per layer: qubit index block (layer_block)
    uint4 *layer_seg;           // per layer slot: {first row, after-gate list
                                // entries, before-gate list entries, 0}
    uint4 *records;             // mask-word records {mech, column, word lo, hi}
    uint4 *tile_sums, *tile_off;
    uint32_t *layer_start;      // per circuit: n_layers + 1 row offsets
    uint2 *meas_lq;             // per measurement: {layer, qubit | x-basis << 31}
    uint32_t *det_row;          // per detector: its row
    uint32_t *obs_rows;         // per circuit (at op_base): OBSERVABLE rows
    uint32_t *obs_count;        // per circuit
    unsigned long long *mech_key;    // per mechanism: word count (low byte) plus
                                // the sum of its words' hashes (grouping key);
                                // zero between compiles
    uint32_t *edge_mech;        // per hyperedge: its class's smallest mechanism
    unsigned long long *mech_info;   // loc | kind << 32 | comp << 40 | circuit << 48
    uint32_t *inl_col;          // per mechanism, kInlineWords slots: column ids
                                // (kObsColFlag on the observable word)
    unsigned long long *inl_word;    // ... and the words
    uint4 *ov_rec;              // overflow words {column, word lo, word hi, next}
    uint32_t *ov_mech;          // mechanism of each overflow word
    uint32_t *ov_head;          // per mechanism: first overflow word or kNone
    uint32_t *slot_of;          // per mechanism: hash-table slot or kNone
    int32_t *mech_class;        // per mechanism: edge or -1
    TabSlot *table;             // grouping hash table
    uint2 *scan_val;            // per mechanism: scan input
    uint2 *comp_off;            // per mechanism: (edge, detector id) offsets, n + 1
    uint2 *scan_bsum;           // scans: per-block sums
    uint32_t *det_off;          // n_edges + 1
    uint32_t *det_idx;
    unsigned long long *obs_mask;
    float *prob, *logodds;
    uint32_t *class_slot, *edge_circ;
    uint32_t *circ_edges;       // per circuit edge counts
    unsigned long long *gacc;   // adjoint accumulators (lo, hi) per location
    Status *status;
};

// ---------------------------------------------------------------------------
// row kinds (flat format)
// ---------------------------------------------------------------------------
enum Kind : uint32_t {
    K_TICK = 0, K_R = 1, K_M = 2, K_MR = 3, K_RX = 4, K_MX = 5, K_MRX = 6, K_NOP = 7,
    K_H = 8, K_S = 9, K_CX = 10, K_CZ = 11, K_DET = 16, K_OBS = 17,
    K_XERR = 32, K_ZERR = 33, K_DEP1 = 34, K_DEP2 = 35
};

__host__ __device__ inline bool is_measure(uint32_t k) {
    return k == K_M || k == K_MR || k == K_MX || k == K_MRX;
}
__host__ __device__ inline bool is_noise(uint32_t k) { return k >= K_XERR && k <= K_DEP2; }
__host__ __device__ inline bool is_gate1(uint32_t k) { return (k >= K_R && k <= K_MRX) || k == K_H || k == K_S; }
__host__ __device__ inline bool is_gate2(uint32_t k) { return k == K_CX || k == K_CZ; }
__host__ __device__ inline bool is_gate(uint32_t k) { return is_gate1(k) || is_gate2(k); }

// number of Pauli components a noise row contributes at a level
__host__ __device__ inline uint32_t n_comp(uint32_t kind, uint32_t level) {
    switch (kind) {
    case K_XERR: case K_ZERR: return 1;
    case K_DEP1: return level == 0 ? 2u : 3u;
    case K_DEP2: return level == 0 ? 6u : (level == 1 ? 10u : 15u);
    default: return 0;
    }
}

// Which plane words make up component c: bit0 = X plane of the first qubit,
// bit1 = Z plane of the first qubit, bit2 / bit3 the same for the second.
// One-qubit depolarising: X, Z, Y.  Two-qubit: the level-0 terms
// IX IZ XI XX ZI ZZ, then the level-1 terms IY XZ YI ZX, then the level-2
// terms XY YX YY YZ ZY (Table tab:correlation-level).
__device__ __forceinline__ uint32_t comp_planes(uint32_t kind, uint32_t c) {
    // packed 4-bit codes, component 0 in the lowest nibble
    const unsigned long long dep2 = 0x0EBF7D639CA25184ull;  // IX..ZY as listed above
    switch (kind) {
    case K_XERR: return 1u;
    case K_ZERR: return 2u;
    case K_DEP1: return (0x321u >> (4 * c)) & 0xFu;
    default: return (uint32_t)((dep2 >> (4 * c)) & 0xFull);
    }
}

// t = -log(1 - 2 q) of one component of a channel with parameter p.  With
// the independent-component decomposition 1 - 2q = (1 - c p)^(1/k):
// X/Z errors c = 2, k = 1; DEPOLARIZE1 c = 4/3, k = 2; DEPOLARIZE2 c = 16/15,
// k = 8.
__device__ __forceinline__ void channel_ck(uint32_t kind, float &c, float &k) {
    switch (kind) {
    case K_DEP1: c = 4.0f / 3.0f; k = 2.0f; break;
    case K_DEP2: c = 16.0f / 15.0f; k = 8.0f; break;
    default: c = 2.0f; k = 1.0f; break;
    }
}
__device__ __forceinline__ float channel_pmax(uint32_t kind) {
    return kind == K_DEP1 ? 0.75f : (kind == K_DEP2 ? 0.9375f : 0.5f);
}

// packed rows: kind (6 bits) | qubit a (13 bits) | qubit b (13 bits), aux
__host__ __device__ inline uint2 pack_row(uint32_t kind, uint32_t a, uint32_t b, uint32_t aux) {
    return make_uint2((kind << 26) | (a << 13) | b, aux);
}
__host__ __device__ inline uint32_t row_kind(uint2 r) { return r.x >> 26; }
__host__ __device__ inline uint32_t row_a(uint2 r) { return (r.x >> 13) & 0x1FFFu; }
__host__ __device__ inline uint32_t row_b(uint2 r) { return r.x & 0x1FFFu; }

// ---------------------------------------------------------------------------
// per-layer qubit index (written by the lowering, read by the stage-1 walk)
// ---------------------------------------------------------------------------
// Block of layer L of a circuit with nq qubits, blocks of one circuit
// consecutive (L = 0 .. n_layers, the last one for the end sentinel):
//   boff[qb]   u16  before-gate list offsets of L: q's rows are entries
//                   [boff[q], boff[q+1]) of the before-gate lists of L
//   gate[nq4]  u32  q's gate in L as seen from q (gate_view), 0 for none
//   aoff[qb]   u16  after-gate list offsets of L
// with nq4 = nq rounded up to 4 and qb = nq + 1 rounded up to 8, so every
// part is 16-byte aligned.  One walk step at L reads gate(L), aoff(L) and
// boff(L + 1): a single contiguous range.
struct LayerGeo {
    uint32_t nq4, qb, bytes;    // bytes of one block (multiple of 16)
};
__host__ __device__ inline LayerGeo layer_geo(uint32_t nq) {
    LayerGeo g;
    g.nq4 = (nq + 3u) & ~3u;
    g.qb = (nq + 1u + 7u) & ~7u;
    g.bytes = 4u * g.nq4 + 4u * g.qb;
    return g;
}
constexpr uint32_t kMaxLayerRows = 32767;   // rows of one TICK layer (u16 list offsets)

// A gate seen from one of its qubits: kind (4 bits) << 28 | payload, payload
// the measurement index for R/M/MR/RX/MX/MRX and the other qubit for the
// two-qubit gates.  One-qubit kinds keep their row kind.
enum GateView : uint32_t {
    GV_NONE = 0, GV_CX_C = 10, GV_CZ_A = 11, GV_CX_T = 12, GV_CZ_B = 13
};
constexpr uint32_t kMaxMeasurements = 1u << 28;

// ---------------------------------------------------------------------------
// shared-memory barriers and 1-D bulk (TMA) copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive on behalf of `count` participants
__device__ __forceinline__ void mbar_arrive_count(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// arrive on the barrier and announce `bytes` of transaction for this phase
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared, completion counted on the barrier
// (addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// bounded wait: false if the phase did not complete within `limit` polls
constexpr uint32_t kWaitPolls = 1u << 22;   // default limit of a bounded wait
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity,
                                                  uint32_t limit = kWaitPolls) {
    for (uint32_t it = 0; it < limit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------------------
// status reporting: the first error wins
// ---------------------------------------------------------------------------
__device__ __forceinline__ void report(Status *st, uint32_t code, uint32_t a, uint32_t b, uint32_t c) {
    if (atomicCAS(&st->code, 0u, code) == 0u) {
        st->info[0] = a;
        st->info[1] = b;
        st->info[2] = c;
    }
}

// block-uniform test of the status code (every thread of the block gets
// thread 0's reading, so an early return never splits a block that later
// meets a barrier); call it where all threads of the block are present
__device__ __forceinline__ bool status_set(Status *st) {
    __shared__ uint32_t code;
    __syncthreads();
    if (threadIdx.x == 0) code = *(volatile uint32_t *)&st->code;
    __syncthreads();
    return code != 0u;
}

// ---------------------------------------------------------------------------
// exact 128-bit fixed-point accumulation (scheduling-independent sums)
// ---------------------------------------------------------------------------
// value v >= 0 as an unsigned integer v * 2^shift, split (lo, hi)
__device__ __forceinline__ void to_fixed(float v, int shift, unsigned long long &lo, unsigned long long &hi) {
    lo = 0; hi = 0;
    if (!(v > 0.0f)) return;
    int e;
    float f = frexpf(v, &e);                        // v = f * 2^e, f in [0.5, 1)
    unsigned long long mant = (unsigned long long)ldexpf(f, 24);  // 24-bit integer
    int s = e - 24 + shift;                         // v * 2^shift = mant * 2^s
    if (s <= -64) return;
    if (s < 0) { lo = mant >> (-s); return; }
    if (s < 64) {
        lo = mant << s;
        hi = (s == 0) ? 0ull : (mant >> (64 - s));
        if (s + 24 <= 64) hi = 0ull;
    } else if (s < 128) {
        hi = mant << (s - 64);
    } else {
        hi = 0x7FFFFFFFFFFFFFFFull;                 // saturate (not reached for clamped inputs)
    }
}

__device__ __forceinline__ void acc128_add(unsigned long long *acc, unsigned long long lo, unsigned long long hi) {
    if (lo) {
        unsigned long long old = atomicAdd(&acc[0], lo);
        if (old + lo < old) hi += 1ull;             // carry out of the low word
    }
    if (hi) atomicAdd(&acc[1], hi);
}

// signed: two's complement modulo 2^128
__device__ __forceinline__ void acc128_add_signed(unsigned long long *acc, float v, int shift) {
    unsigned long long lo, hi;
    to_fixed(fabsf(v), shift, lo, hi);
    if (v < 0.0f) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    acc128_add(acc, lo, hi);
}

__device__ __forceinline__ float fixed_to_float(unsigned long long lo, unsigned long long hi, int shift) {
    return ldexpf((float)hi, 64 - shift) + ldexpf((float)lo, -shift);
}

__device__ __forceinline__ float fixed_to_float_signed(unsigned long long lo, unsigned long long hi, int shift) {
    bool neg = (hi >> 63) != 0ull;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    float v = fixed_to_float(lo, hi, shift);
    return neg ? -v : v;
}

constexpr int kProbShift = 96;   // class sums of t = -log(1-2q): 2^-96 resolution
constexpr int kGradShift = 64;   // adjoint sums: 2^-64 resolution

// ---------------------------------------------------------------------------
// hashing of masks (any well-mixed 64-bit function works: grouping verifies
// whole masks).  Finaliser of splitmix64 (Steele, Lea and Flood 2014).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// the grouping hash under the weak-hash test modes: 1 keeps the table
// position (low half) but gives every mask the same tag (high half), 2 gives
// every mask the same hash
__device__ __forceinline__ unsigned long long weaken_hash(unsigned long long h, uint32_t mode) {
    return mode == 0u ? h : (mode == 1u ? (h & 0xFFFFFFFFull) : 0ull);
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of uint32 (blockDim.x a multiple of 32, <= 1024)
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *smem_warp, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < NT / 32) ? smem_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) smem_warp[lane] = w;
    }
    __syncthreads();
    uint32_t warp_prefix = warp ? smem_warp[warp - 1] : 0u;
    total = smem_warp[NT / 32 - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

}  // namespace gpdem

// kernel entry points (implemented in lower.cu, stage1.cu, stage2.cu)
namespace gpdem {
// one host -> device copy done by the device (all byte counts multiples of 4)
struct CopyJob {
    const void *src;
    void *dst;
    uint64_t bytes;
};
void launch_gather_host(const CopyJob *jobs, uint32_t n_jobs, uint64_t max_bytes, uint32_t n_sms, cudaStream_t s);
void launch_lowering(const Buffers &b, uint32_t n_tiles, uint32_t layer_slots, uint32_t max_qubits, uint32_t n_sms,
                     cudaStream_t s, uint32_t *launches);
cudaError_t lowering_setup(uint32_t max_qubits);
// shared-memory shape of the stage-1 walk: window buffers, list entries a
// buffer holds, bytes of a buffer and of the whole block, and which walk
// (1: role-split, 0: block-wide)
struct Stage1Shape {
    uint32_t nbuf, list_cap, wbytes;
    size_t smem;
    uint32_t split;
};
// limit: dynamic shared memory one block may take (opt-in maximum less the
// kernel's static shared memory)
Stage1Shape stage1_shape(uint32_t max_qubits, uint32_t blocks_per_sm, size_t limit);
size_t stage1_dynamic_smem_limit(int device);
// wide: the role-split walk's emitters deal the rows of wide steps out
// lane by lane (the kernel instance with that path)
void launch_stage1(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t max_qubits, const Stage1Shape &shape,
                   bool wide, cudaStream_t s, uint32_t *launches);
// split: 0 block-wide walk, 1 role-split walk, 2 role-split walk with wide emission
const void *stage1_kernel_ptr(uint32_t threads, uint32_t split);
void launch_group(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t max_mech, cudaStream_t s, uint32_t *launches);
void launch_compact(const Buffers &b, uint32_t grid, uint32_t threads, uint32_t max_mech, uint32_t n_sms, cudaStream_t s,
                    uint32_t *launches);
void launch_init_table(TabSlot *t, size_t n, cudaStream_t s);
// the device buffers of a driver (for the server's selection kernels)
const Buffers &driver_buffers(const gp_driver *d);
uint32_t driver_max_det_entries(const gp_driver *d);
uint32_t driver_sms(const gp_driver *d);      // SMs of the driver's device
void launch_scan(const Buffers &B, const uint2 *in, const uint32_t *n_ptr, uint2 *out, uint32_t max_n, uint32_t n_sms,
                 cudaStream_t s, uint32_t *launches);
void launch_backward(const Buffers &b, const float *g_prob, const float *g_logodds, float *g_noise,
                     uint32_t n_mech, uint32_t n_loc, uint32_t grid, uint32_t threads, cudaStream_t s, uint32_t *launches);
}  // namespace gpdem
