// serve.cu -- cycle-streaming server (include/gpserve.h).
//
// Host side: per-patch state (declared logicals, per-cycle sizes, pending
// requests), pinned staging of submitted cycles, the scheduler step.
// Device side, per step:
//   - the new cycles are copied into their patches' resident rings;
//   - assemble: one launch copies every window's cycles from the rings into
//     the batch arena, shifting record and location indices to the window,
//     emptying the detectors of records-only cycles and appending the rows
//     that close a window with the declared logicals; noise rows are left
//     out (made NOP rows) where no delivered hyperedge can hold their
//     mechanisms: in a window's last H cycles unless the window ends its
//     patch, and in its records-only cycles when only the horizon test
//     would read them and that test is moot (a final window, or a window of
//     registered cycles whose pattern passed it before);
//   - the windows are compiled as one batch (gp_compile_batch);
//   - seal (one captured graph of four kernels): a horizon test per window
//     (no mechanism of a records-only cycle c flips a detector after cycle
//     c + H: those detectors all lie in the window, so a violation shows);
//     the request slot of every hyperedge (the request whose cycle holds its
//     smallest detector; none when that cycle is not sealed yet), counted
//     per chunk of a window's hyperedges; the request starts (slot, then
//     window order); and every delivered hyperedge written, with
//     patch-global detector ids, straight into a pinned host buffer.  Every
//     request's hyperedges thus come out contiguous, and the host hands out
//     slices.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <set>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "gpserve.h"

using namespace gpdem;

namespace gpdem {
void set_last_error(const std::string &msg);
}

namespace {

gp_status sfail(gp_status code, const std::string &msg) {
    set_last_error(msg);
    return code;
}

#define SV_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return sfail(GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// one cycle of one window, or the rows closing a window
struct SegDesc {
    const uint4 *ops;
    const uint32_t *recs;
    const float *noise;
    uint32_t n_ops, n_recs, n_loc;
    uint32_t dst_ops, dst_recs, dst_loc;
    uint32_t rec_shift, loc_shift;
    uint32_t flags;             // kSegRecordsOnly | kSegNoNoise
    uint32_t pad;
};
// kSegNoNoise: the cycle's noise rows become NOP rows (no mechanisms)
constexpr uint32_t kSegRecordsOnly = 1u, kSegNoNoise = 4u;
constexpr size_t kMaxVerified = 1024;   // tested window patterns kept per patch

// what a window seals
struct SealDesc {
    uint32_t det_lo, det_hi;    // window-local detector range of the sealed cycles
    uint32_t take_no_det;       // final window: also hyperedges without detectors
    uint32_t det_base;          // patch-global id of window-local detector 0
    uint32_t n_mech_rec;        // mechanisms of the records-only cycles (0: no check)
    uint32_t n_rec;             // records-only cycles
    uint32_t n_cyc;             // cycles of the window (entries of its cycle table - 1)
    int32_t r_off;              // request slot of cycle j of the window: min(j + r_off, r_max)
    uint32_t r_max;
    uint32_t pad[3];
};
// per records-only cycle j of a window: (end of its mechanisms, first
// window-local detector it may not flip)

constexpr int kSegBlocksY = 8;

__global__ void __launch_bounds__(256) assemble_kernel(const SegDesc *seg, uint32_t n_seg, uint4 *ops,
                                                       uint32_t *recs, float *noise) {
    const uint32_t s = blockIdx.x;
    if (s >= n_seg) return;
    const SegDesc d = seg[s];
    const uint32_t stride = gridDim.y * blockDim.x, t0 = blockIdx.y * blockDim.x + threadIdx.x;
    for (uint32_t i = t0; i < d.n_ops; i += stride) {
        uint4 op = d.ops[i];
        const uint32_t k = op.x;
        if (k == K_DET || k == K_OBS) {
            op.y += d.rec_shift;
            if ((d.flags & kSegRecordsOnly) && k == K_DET) op.z = 0u;
        } else if (is_noise(k)) {
            if (d.flags & kSegNoNoise) op = make_uint4(K_NOP, 0u, 0u, 0u);
            else op.w += d.loc_shift;
        }
        ops[d.dst_ops + i] = op;
    }
    for (uint32_t i = t0; i < d.n_recs; i += stride) recs[d.dst_recs + i] = d.recs[i];
    for (uint32_t i = t0; i < d.n_loc; i += stride)
        noise[d.dst_loc + i] = d.noise[i];
}

// What the select phase of a step needs beyond the compile: the windows,
// the request slots and the pinned step buffer.  The host fills a pinned
// copy before each step; a copy inside the captured select graph brings it
// to the device, so the graph's kernels never change.
struct SealOut {
    uint32_t *doff, *det;
    float *prob, *logodds;
    unsigned long long *obs;
};
struct SelParams {
    uint32_t n_win, n_slots;        // windows; request slots (most requests of a window)
    uint64_t edges_cap, det_cap;    // of the pinned step buffer
    SealOut host;                   // the pinned step buffer
};

// The select phase reads a window's hyperedges in chunks of kSelChunk, one
// per thread of a block; a chunk never spans two windows.
constexpr uint32_t kSelChunk = 1024;
constexpr uint32_t kSelThreads = kSelChunk;
constexpr uint32_t kMaxSlots = 512;     // request slots: max_cycles_per_step at most

// device scratch of the select phase
struct SelScratch {
    uint32_t *win_e0;               // n_win + 1: first hyperedge of each window
    uint32_t *chunk0;               // n_win + 1: first chunk of each window
    uint2 *chunk_tot;               // per chunk and slot: delivered (edges, detector ids), then their output base
    unsigned long long *tot;        // per slot and window: packed totals (edges << 32 | ids), then starts
    uint2 *starts;                  // per slot: n_win + 1 output starts (device copy)
};

// the window holding chunk c: the last w < n_win with chunk0[w] <= c
__device__ __forceinline__ uint32_t chunk_window(const uint32_t *chunk0, uint32_t n_win, uint32_t c) {
    uint32_t lo = 0, hi = n_win;
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (chunk0[mid] <= c) lo = mid; else hi = mid;
    }
    return lo;
}

// first hyperedge and first chunk of every window (from the compile's
// per-circuit counts); clears the horizon flags
__global__ void sel_prep_kernel(Buffers B, const SelParams *sp, SelScratch sc, uint32_t *horizon) {
    const uint32_t n_win = sp->n_win;
    if (threadIdx.x == 0) {
        uint32_t e = 0, c = 0;
        for (uint32_t w = 0; w < n_win; w++) {
            sc.win_e0[w] = e;
            sc.chunk0[w] = c;
            const uint32_t n = B.circ_edges[w];
            e += n;
            c += (n + kSelChunk - 1u) / kSelChunk;
        }
        sc.win_e0[n_win] = e;
        sc.chunk0[n_win] = c;
    }
    for (uint32_t w = threadIdx.x; w < n_win; w += blockDim.x) horizon[w] = 0u;
}

// Per hyperedge: the request slot that delivers it (its smallest detector
// lies in the cycle that request seals), stored with its detector count;
// per chunk: the delivered hyperedges and detector ids of every slot.
// Then the horizon test: a mechanism of records-only cycle c flipping a
// detector after cycle c + H means the window's horizon was too short.
__global__ void __launch_bounds__(kSelThreads, 1) sel_count_kernel(Buffers B, const SealDesc *seal, const uint32_t *cyc_tab,
                                                                uint32_t tab_stride, const uint2 *rec_tab,
                                                                uint32_t max_h, const SelParams *sp, SelScratch sc,
                                                                uint32_t *horizon) {
    extern __shared__ uint2 slot_cnt[];   // n_slots
    const uint32_t n_win = sp->n_win, R = sp->n_slots, n_chunks = sc.chunk0[n_win];
    for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const uint32_t w = chunk_window(sc.chunk0, n_win, c);
        for (uint32_t i = threadIdx.x; i < R; i += blockDim.x) slot_cnt[i] = make_uint2(0u, 0u);
        __syncthreads();
        const uint32_t e = sc.win_e0[w] + (c - sc.chunk0[w]) * kSelChunk + threadIdx.x;
        uint32_t key = 0u, nd = 0u;            // key: slot + 1, or 0 (not delivered this step)
        if (e < sc.win_e0[w + 1]) {
            const SealDesc &sd = seal[w];
            const uint32_t o0 = B.det_off[e], o1 = B.det_off[e + 1];
            nd = o1 - o0;
            if (o1 > o0) {
                const uint32_t d0 = B.det_idx[o0];          // detector lists are ascending
                if (d0 >= sd.det_lo && d0 < sd.det_hi) {
                    // cycle of d0 within the window: last j with tab[j] <= d0
                    const uint32_t *tab = cyc_tab + (size_t)w * tab_stride;
                    uint32_t lo = 0, hi = sd.n_cyc;
                    while (hi - lo > 1u) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (tab[mid] <= d0) lo = mid; else hi = mid;
                    }
                    key = (uint32_t)min((int32_t)lo + sd.r_off, (int32_t)sd.r_max) + 1u;
                }
            } else if (sd.take_no_det) {
                key = sd.r_max + 1u;
            }
            B.scan_val[e] = make_uint2(key, nd);
        }
        // one shared add per slot and warp
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
        const uint32_t sum = __reduce_add_sync(peers, nd);
        if (key != 0u && (threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1)) {
            atomicAdd(&slot_cnt[key - 1u].x, (uint32_t)__popc(peers));
            atomicAdd(&slot_cnt[key - 1u].y, sum);
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < R; i += blockDim.x) sc.chunk_tot[(size_t)c * R + i] = slot_cnt[i];
        __syncthreads();
    }
    for (uint32_t w = blockIdx.x; w < n_win; w += gridDim.x) {
        const uint32_t m0 = B.circ[w].mech_base, n = seal[w].n_mech_rec, nr = seal[w].n_rec;
        const uint2 *tab = rec_tab + (size_t)w * max_h;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const int32_t cls = B.mech_class[m0 + i];
            if (cls < 0) continue;
            const uint32_t o0 = B.det_off[cls], o1 = B.det_off[cls + 1];
            if (o1 == o0) continue;
            uint32_t j = 0;
            while (j + 1u < nr && tab[j].x <= i) j++;
            if (B.det_idx[o1 - 1u] >= tab[j].y) horizon[w] = 1u;
        }
    }
}

// Output order: request slot, then window, then hyperedge.  Totals per
// (slot, window), their exclusive scan (the request starts, also written to
// the host), each chunk's base within its request, and the last detector
// offset of every request (offsets are per request, and request (r, w) is
// the (r n_win + w)-th, so its offsets sit r n_win + w entries after its
// hyperedges).  One block.
__global__ void __launch_bounds__(kSelThreads) sel_starts_kernel(const SelParams *sp, SelScratch sc, uint2 *starts_host) {
    __shared__ unsigned long long warp_tot[kSelThreads / 32];
    const uint32_t n_win = sp->n_win, R = sp->n_slots, P = R * n_win;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t r = i / n_win, w = i % n_win;
        unsigned long long t = 0ull;
        for (uint32_t c = sc.chunk0[w]; c < sc.chunk0[w + 1]; c++) {
            const uint2 v = sc.chunk_tot[(size_t)c * R + r];
            t += ((unsigned long long)v.x << 32) + v.y;
        }
        sc.tot[i] = t;
    }
    __syncthreads();
    unsigned long long run = 0ull;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long v = i < P ? sc.tot[i] : 0ull;
        unsigned long long x = v;
        for (uint32_t o = 1; o < 32u; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31u) warp_tot[warp] = x;
        __syncthreads();
        unsigned long long before = 0ull, all = 0ull;
        for (uint32_t k = 0; k < blockDim.x / 32u; k++) {
            if (k < warp) before += warp_tot[k];
            all += warp_tot[k];
        }
        if (i < P) sc.tot[i] = run + before + x - v;
        run += all;
        __syncthreads();
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < R * (n_win + 1u); i += blockDim.x) {
        const uint32_t r = i / (n_win + 1u), w = i % (n_win + 1u);
        const unsigned long long v = w < n_win ? sc.tot[r * n_win + w] : (r + 1u < R ? sc.tot[(r + 1u) * n_win] : run);
        const uint2 st = make_uint2((uint32_t)(v >> 32), (uint32_t)v);
        sc.starts[i] = st;
        starts_host[i] = st;
    }
    const SealOut out = sp->host;
    const uint64_t edges_cap = sp->edges_cap;
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint32_t r = i / n_win, w = i % n_win;
        const unsigned long long b0 = sc.tot[i];
        unsigned long long b = b0;
        for (uint32_t c = sc.chunk0[w]; c < sc.chunk0[w + 1]; c++) {
            const uint2 v = sc.chunk_tot[(size_t)c * R + r];
            sc.chunk_tot[(size_t)c * R + r] = make_uint2((uint32_t)(b >> 32), (uint32_t)b);
            b += ((unsigned long long)v.x << 32) + v.y;
        }
        const uint64_t at = (b >> 32) + (uint64_t)r * n_win + w;
        if (at < edges_cap) out.doff[at] = (uint32_t)b - (uint32_t)b0;
    }
}

// Every delivered hyperedge written straight into the pinned step buffer at
// its place: the chunk's base in its request, plus those of the same slot
// before it in the chunk (per warp, then across warps).
__global__ void __launch_bounds__(kSelThreads, 1) sel_write_kernel(Buffers B, const SealDesc *seal, const SelParams *sp,
                                                                SelScratch sc) {
    extern __shared__ uint2 warp_cnt[];   // [warp][slot]
    const uint32_t n_win = sp->n_win, R = sp->n_slots, n_chunks = sc.chunk0[n_win];
    const SealOut out = sp->host;
    const uint64_t edges_cap = sp->edges_cap, det_cap = sp->det_cap;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    constexpr uint32_t kWarps = kSelThreads / 32u;
    for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const uint32_t w = chunk_window(sc.chunk0, n_win, c);
        for (uint32_t i = threadIdx.x; i < kWarps * R; i += blockDim.x) warp_cnt[i] = make_uint2(0u, 0u);
        __syncthreads();
        const uint32_t e = sc.win_e0[w] + (c - sc.chunk0[w]) * kSelChunk + threadIdx.x;
        const uint2 kv = e < sc.win_e0[w + 1] ? B.scan_val[e] : make_uint2(0u, 0u);
        const uint32_t key = kv.x, nd = kv.y;
        // rank and detector-id prefix among this warp's hyperedges of the same slot
        uint32_t rank = 0, dpre = 0;
        unsigned todo = __ballot_sync(0xFFFFFFFFu, key != 0u);
        while (todo) {
            const uint32_t k = __shfl_sync(0xFFFFFFFFu, key, __ffs(todo) - 1);
            const bool mine = key == k;
            uint32_t x = mine ? nd : 0u;
            for (uint32_t o = 1; o < 32u; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
            const unsigned m = __ballot_sync(0xFFFFFFFFu, mine);
            if (mine) {
                rank = (uint32_t)__popc(m & lt);
                dpre = x - nd;
            }
            if (lane == 0u) warp_cnt[warp * R + (k - 1u)] = make_uint2((uint32_t)__popc(m), total);
            todo &= ~m;
        }
        __syncthreads();
        for (uint32_t r = threadIdx.x; r < R; r += blockDim.x) {
            uint2 run = make_uint2(0u, 0u);
            for (uint32_t k = 0; k < kWarps; k++) {
                const uint2 t = warp_cnt[k * R + r];
                warp_cnt[k * R + r] = run;
                run.x += t.x;
                run.y += t.y;
            }
        }
        __syncthreads();
        if (key != 0u) {
            const uint32_t r = key - 1u;
            const uint2 base = sc.chunk_tot[(size_t)c * R + r], wb = warp_cnt[warp * R + r];
            const uint64_t pos = (uint64_t)base.x + wb.x + rank, dpos = (uint64_t)base.y + wb.y + dpre;
            if (pos < edges_cap) {
                out.prob[pos] = B.prob[e];
                out.logodds[pos] = B.logodds[e];
                out.obs[pos] = B.obs_mask[e];
            }
            const uint64_t at = pos + (uint64_t)r * n_win + w;
            if (at < edges_cap) out.doff[at] = (uint32_t)(dpos - sc.starts[r * (n_win + 1u) + w].y);
        }
        // the detector ids of each slot's hyperedges in this warp form one
        // contiguous range of the output: the warp writes it lane by lane
        // (consecutive lanes, consecutive words), each lane finding the
        // hyperedge of its word by a binary search over the running counts
        const uint32_t o0 = key != 0u ? B.det_off[e] : 0u;
        const uint32_t db = seal[w].det_base;
        unsigned todo2 = __ballot_sync(0xFFFFFFFFu, key != 0u);
        while (todo2) {
            const uint32_t k = __shfl_sync(0xFFFFFFFFu, key, __ffs(todo2) - 1);
            const bool mine = key == k;
            uint32_t x = mine ? nd : 0u;
            for (uint32_t o = 1; o < 32u; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
            const uint32_t excl = x - (mine ? nd : 0u);
            const uint2 base = sc.chunk_tot[(size_t)c * R + (k - 1u)], wb = warp_cnt[warp * R + (k - 1u)];
            const uint64_t g0 = (uint64_t)base.y + wb.y;
            for (uint32_t t0 = 0; t0 < total; t0 += 32u) {
                const uint32_t t = t0 + lane;
                uint32_t lo = 0;                       // first lane whose running count exceeds t
                for (uint32_t h = 16; h; h >>= 1) {
                    const uint32_t y = __shfl_sync(0xFFFFFFFFu, x, lo + h - 1u);
                    if (y <= t) lo += h;
                }
                const uint32_t so0 = __shfl_sync(0xFFFFFFFFu, o0, lo);
                const uint32_t sex = __shfl_sync(0xFFFFFFFFu, excl, lo);
                if (t < total && g0 + t < det_cap) out.det[g0 + t] = B.det_idx[so0 + (t - sex)] + db;
            }
            todo2 &= ~__ballot_sync(0xFFFFFFFFu, mine);
        }
        __syncthreads();
    }
}

uint32_t n_comp_host(uint32_t kind, uint32_t level) {
    switch (kind) {
    case K_XERR: case K_ZERR: return 1;
    case K_DEP1: return level == 0 ? 2u : 3u;
    case K_DEP2: return level == 0 ? 6u : (level == 1 ? 10u : 15u);
    default: return 0;
    }
}

struct CycleInfo {
    uint32_t n_ops, n_recs, n_loc, n_meas, n_det, n_ticks;
    uint32_t mech[3];           // mechanisms at L0, L1, L2
    uint64_t det_base, meas_base;
    // where the cycle lives on the device once stepped (ring slot or
    // registered copy)
    const uint4 *src_ops;
    const uint32_t *src_recs;
    const float *src_noise;
    int32_t reg = -1;           // the registered cycle it repeats, or -1
};

// what a cycle's rows fix, whatever the patch saw before it: its counts and
// how far its records look back past its own start
struct CycleScan {
    CycleInfo ci;               // counts (bases unset)
    uint64_t reach = 0;         // measurements before the cycle the furthest record reaches
    uint64_t reach_row = 0;     // the row holding that record
    int64_t obs_row = -1;       // first OBSERVABLE_INCLUDE row, if any
};

// a cycle registered once by its patch: its scan and device copies of its
// rows, records and noise (the windows read it from there)
struct Registered {
    uint4 *d_ops = nullptr;
    uint32_t *d_recs = nullptr;
    float *d_noise = nullptr;
    CycleScan scan;             // its rows scanned at registration
};

// pinned host copy of one step's delivered hyperedges, shared by the
// requests it serves until they are released
struct OutBuf {
    uint32_t *doff = nullptr, *det = nullptr;
    float *prob = nullptr, *logodds = nullptr;
    unsigned long long *obs = nullptr;
    uint64_t edges_cap = 0, det_cap = 0;    // doff holds edges_cap + offs_extra entries
    uint32_t refs = 0;
};
const uint32_t kNoOffsets[1] = {0};

struct Request {
    uint64_t id = 0;
    uint32_t patch = 0, cycle = 0;
    bool final = false, done = false;
    uint32_t stage = 0;          // pinned staging slot of the submitted cycle
    int32_t reg = -1;            // or the registered cycle it repeats
    gp_status status = GP_OK;
    uint64_t t_arrival = 0, t_done = 0;
    // delivered hyperedges: a slice of a shared step buffer
    OutBuf *buf = nullptr;
    uint32_t n_edges = 0;
    uint64_t n_det = 0;
    const uint32_t *det_offsets = kNoOffsets, *det_idx = nullptr;
    const unsigned long long *obs = nullptr;
    const float *prob = nullptr, *logodds = nullptr;
};

struct Patch {
    bool open = false;
    uint32_t n_qubits = 0, H = 1, n_obs = 0;
    std::vector<uint32_t> virt_q;        // distinct logical qubits, measured in this order
    std::vector<uint32_t> virt_recs;     // per logical: lookbacks into those measurements
    std::vector<uint32_t> virt_off;      // n_obs + 1
    uint4 *ring_ops = nullptr;
    uint32_t *ring_recs = nullptr;
    float *ring_noise = nullptr;
    std::vector<CycleInfo> cycles;       // every submitted cycle
    std::vector<Registered> registered;
    uint32_t next_step = 0;              // first cycle not yet stepped
    bool final_submitted = false;
    // windows of registered cycles whose horizon test passed, by their
    // cycles' registered ids: the same rows give the same test, so such a
    // window leaves its records-only cycles' noise out and is not tested
    std::set<std::vector<int32_t>> verified;
    std::deque<uint64_t> pending;        // submitted, not yet stepped (cycle order)
};

}  // namespace

struct gp_server {
    gp_server_config cfg{};
    uint32_t W = 0;                      // ring slots per patch: 3 max_horizon + K
    uint32_t n_sms = 1;
    uint32_t extra_ops = 0, extra_recs = 0;
    gp_driver *drv = nullptr;
    // device memory
    unsigned char *dmem = nullptr;
    uint4 *arena_ops = nullptr;
    uint32_t *arena_recs = nullptr;
    float *arena_noise = nullptr;
    // the seal block: per window its SealDesc, record table and cycle table,
    // laid out alike in device memory and at the start of h_desc, so that
    // one copy brings it over (the segment descriptors and closing rows are
    // read by the assembly straight from pinned host memory)
    uint64_t sealblk_bytes = 0;
    SealDesc *d_seal = nullptr;
    uint2 *d_rec_tab = nullptr;
    uint32_t *d_cyc_tab = nullptr;       // per window: detector offset of each cycle
    SelScratch sel{};                    // select-phase scratch
    SelParams *d_sel = nullptr;          // the select phase's per-step parameters
    SelParams *h_sel = nullptr;          // ... their pinned host copy
    cudaStream_t cap_stream = nullptr;   // captures the select graph
    cudaGraphExec_t sel_exec = nullptr;  // the select phase
    float times[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // last step: build, compile, select, hand-out,
                                                 // then the compile's device stages (us)
    uint64_t out_edges_cap = 0, out_det_cap = 0;
    // pinned host memory
    unsigned char *h_desc = nullptr;     // seal block | segs | extra ops | extra recs
    size_t h_desc_bytes = 0;
    uint4 *h_stage_ops = nullptr;
    uint32_t *h_stage_recs = nullptr;
    float *h_stage_noise = nullptr;
    std::vector<uint32_t> free_stage;
    uint32_t *h_horizon = nullptr;       // per window: horizon too short (written by the device)
    uint2 *h_starts = nullptr;           // per request slot and window: output starts (ditto)
    std::vector<OutBuf *> out_pool;
    // state
    std::vector<Patch> patches;
    std::unordered_map<uint64_t, Request> requests;
    std::vector<uint64_t> completed;
    uint64_t next_request = 1;
    uint32_t n_pending = 0;
};

namespace {

template <class T> T *carve_dev(unsigned char *base, uint64_t &off, uint64_t count) {
    off = (off + 255) & ~255ull;
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
}

void free_registered(Patch &p) {
    for (Registered &r : p.registered) {
        if (r.d_ops) cudaFree(r.d_ops);
        if (r.d_recs) cudaFree(r.d_recs);
        if (r.d_noise) cudaFree(r.d_noise);
    }
    p.registered.clear();
}

void free_outbuf(OutBuf *b) {
    if (!b) return;
    void *ptrs[] = {b->doff, b->det, b->prob, b->logodds, b->obs};
    for (void *p : ptrs)
        if (p) cudaFreeHost(p);
    delete b;
}

void free_host(gp_server *s) {
    for (Patch &p : s->patches) free_registered(p);
    void *ptrs[] = {s->h_desc, s->h_stage_ops, s->h_stage_recs, s->h_stage_noise, s->h_horizon, s->h_starts, s->h_sel};
    for (void *p : ptrs)
        if (p) cudaFreeHost(p);
    for (OutBuf *b : s->out_pool) free_outbuf(b);
    s->out_pool.clear();
}

// a free step buffer holding `edges` hyperedges (plus `extra` detector
// offsets) and `dets` detector ids, allocated when none fits.  A new buffer
// has twice the room asked for (within the device outputs' capacity), so a
// load that grows pins host memory a few times, not at every new largest
// step.
OutBuf *take_outbuf(gp_server *s, uint64_t edges, uint64_t extra, uint64_t dets) {
    for (OutBuf *b : s->out_pool)
        if (b->refs == 0 && b->edges_cap >= edges + extra && b->det_cap >= dets) return b;
    OutBuf *b = new (std::nothrow) OutBuf();
    if (!b) return nullptr;
    const uint64_t cap_e = s->out_edges_cap + extra, cap_d = std::max<uint64_t>(s->out_det_cap, 1);
    const uint64_t ne = std::max(edges + extra, std::min(std::max<uint64_t>(2 * (edges + extra), 1u << 16), cap_e));
    const uint64_t nd = std::max(dets, std::min(std::max<uint64_t>(2 * dets, 1u << 18), cap_d));
    if (cudaMallocHost(&b->doff, 4 * ne) != cudaSuccess || cudaMallocHost(&b->det, 4 * nd) != cudaSuccess ||
        cudaMallocHost(&b->prob, 4 * ne) != cudaSuccess || cudaMallocHost(&b->logodds, 4 * ne) != cudaSuccess ||
        cudaMallocHost(&b->obs, 8 * ne) != cudaSuccess) {
        free_outbuf(b);
        return nullptr;
    }
    b->edges_cap = ne;
    b->det_cap = nd;
    s->out_pool.push_back(b);
    return b;
}

void drop_result(Request &r) {
    if (r.buf) r.buf->refs--;
    r.buf = nullptr;
    r.n_edges = 0;
    r.n_det = 0;
    r.det_offsets = kNoOffsets;
    r.det_idx = nullptr;
    r.obs = nullptr;
    r.prob = r.logodds = nullptr;
}

void finish(gp_server *s, Request &r, gp_status st, uint64_t t) {
    r.status = st;
    r.done = true;
    r.t_done = t;
    if (st != GP_OK) drop_result(r);
    s->completed.push_back(r.id);
}

}  // namespace

extern "C" {

gp_status gp_server_create(const gp_server_config *config, gp_server **out) {
    if (!config || !out) return sfail(GP_ERR_INVALID, "null argument");
    *out = nullptr;
    const gp_server_config &c = *config;
    if (!c.max_patches || !c.max_batch || !c.max_cycles_per_step || !c.max_horizon || !c.max_pending ||
        !c.max_qubits || !c.max_cycle_ops || !c.max_cycle_layers)
        return sfail(GP_ERR_INVALID, "server config: every count must be positive (recs, locations, measurements, "
                                     "detectors, mechanisms and logical qubits may be zero)");
    if (c.max_qubits > 8192) return sfail(GP_ERR_INVALID, "server config: max_qubits above 8192");
    if (c.max_batch > c.max_patches) return sfail(GP_ERR_INVALID, "server config: max_batch above max_patches");
    if (c.max_cycles_per_step > kMaxSlots) return sfail(GP_ERR_INVALID, "server config: max_cycles_per_step above 512");
    gp_server *s = new (std::nothrow) gp_server();
    if (!s) return sfail(GP_ERR_CAPACITY, "out of host memory");
    auto cleanup = [&](gp_status st) { gp_server_destroy(s); return st; };
    s->cfg = c;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return cleanup(sfail(GP_ERR_CUDA, "querying the device failed"));
        s->n_sms = (uint32_t)std::max(sms, 1);
    }
    s->W = 3u * c.max_horizon + c.max_cycles_per_step;
    s->extra_ops = 1u + c.max_logical_qubits + 64u;
    s->extra_recs = c.max_logical_qubits;
    const uint64_t W = s->W, Bt = c.max_batch;
    gp_bounds b{};
    b.max_circuits = c.max_batch;
    b.max_qubits = c.max_qubits;
    const uint64_t ops = Bt * (W * c.max_cycle_ops + s->extra_ops);
    const uint64_t recs = Bt * (W * c.max_cycle_recs + s->extra_recs);
    const uint64_t layers = Bt * (W * c.max_cycle_layers + 2);
    const uint64_t meas = Bt * (W * c.max_cycle_measurements + c.max_logical_qubits);
    const uint64_t dets = Bt * W * c.max_cycle_detectors;
    const uint64_t locs = Bt * W * c.max_cycle_locations;
    const uint64_t mech = Bt * W * std::max<uint32_t>(c.max_cycle_mechanisms, 1);
    if (ops > 0xFFFFFFFFull || recs > 0xFFFFFFFFull || layers > 0xFFFFFFFFull || meas > (1ull << 28) ||
        dets > 0xFFFFFFFFull || locs > 0xFFFFFFFFull || mech > 0x7FFFFFFFull)
        return cleanup(sfail(GP_ERR_CAPACITY, "server config: a batch of windows exceeds the compiler's 32-bit sizes"));
    b.max_ops = ops;
    b.max_recs = std::max<uint64_t>(recs, 1);
    b.max_layers = (uint32_t)layers;
    b.max_measurements = (uint32_t)std::max<uint64_t>(meas, 1);
    b.max_detectors = (uint32_t)std::max<uint64_t>(dets, 1);
    b.max_locations = (uint32_t)std::max<uint64_t>(locs, 1);
    b.max_mechanisms = (uint32_t)mech;
    // device memory: driver workspace + rings + arena + descriptors + outputs
    uint64_t ws = 0;
    {
        const gp_status st = gp_workspace_size(&b, &ws);
        if (st != GP_OK) return cleanup(st);
    }
    const uint64_t max_det_entries = 16ull * b.max_mechanisms;
    s->out_edges_cap = b.max_mechanisms;
    s->out_det_cap = std::min<uint64_t>(max_det_entries, 0xFFFFFFFFull);
    const uint64_t nseg = Bt * (W + 1);
    s->sealblk_bytes = Bt * sizeof(SealDesc) + Bt * c.max_horizon * sizeof(uint2) + Bt * (W + 1) * sizeof(uint32_t);
    auto layout = [&](unsigned char *base) {
        uint64_t off = 0;
        for (uint32_t p = 0; p < c.max_patches; p++) {
            uint4 *o = carve_dev<uint4>(base, off, W * c.max_cycle_ops);
            uint32_t *r = carve_dev<uint32_t>(base, off, std::max<uint64_t>(W * c.max_cycle_recs, 1));
            float *n = carve_dev<float>(base, off, std::max<uint64_t>(W * c.max_cycle_locations, 1));
            if (base) {
                s->patches[p].ring_ops = o;
                s->patches[p].ring_recs = r;
                s->patches[p].ring_noise = n;
            }
        }
        s->arena_ops = carve_dev<uint4>(base, off, ops);
        s->arena_recs = carve_dev<uint32_t>(base, off, std::max<uint64_t>(recs, 1));
        s->arena_noise = carve_dev<float>(base, off, std::max<uint64_t>(locs, 1));
        unsigned char *blk = carve_dev<unsigned char>(base, off, s->sealblk_bytes);
        if (base) {
            s->d_seal = reinterpret_cast<SealDesc *>(blk);
            s->d_rec_tab = reinterpret_cast<uint2 *>(blk + Bt * sizeof(SealDesc));
            s->d_cyc_tab = reinterpret_cast<uint32_t *>(blk + Bt * sizeof(SealDesc) + Bt * c.max_horizon * sizeof(uint2));
        }
        const uint64_t K = c.max_cycles_per_step, max_chunks = s->out_edges_cap / kSelChunk + Bt + 1;
        SelScratch sc{};
        sc.win_e0 = carve_dev<uint32_t>(base, off, Bt + 1);
        sc.chunk0 = carve_dev<uint32_t>(base, off, Bt + 1);
        sc.chunk_tot = carve_dev<uint2>(base, off, max_chunks * K);
        sc.tot = carve_dev<unsigned long long>(base, off, K * Bt);
        sc.starts = carve_dev<uint2>(base, off, K * (Bt + 1));
        if (base) s->sel = sc;
        s->d_sel = carve_dev<SelParams>(base, off, 1);
        return off;
    };
    s->patches.resize(c.max_patches);
    const uint64_t own = layout(nullptr);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return cleanup(sfail(GP_ERR_CUDA, "cudaMemGetInfo failed"));
    const uint64_t margin = 256ull << 20;
    if (ws + own + margin > free_b)
        return cleanup(sfail(GP_ERR_CAPACITY, "server needs " + std::to_string((ws + own) >> 20) +
                                                  " MiB of device memory, " + std::to_string(free_b >> 20) + " MiB free"));
    if (cudaMalloc(&s->dmem, own) != cudaSuccess) return cleanup(sfail(GP_ERR_CUDA, "cudaMalloc of the server arena failed"));
    layout(s->dmem);
    {
        const gp_status st = gp_driver_create(&b, nullptr, 0, &s->drv);
        if (st != GP_OK) return cleanup(st);
        gp_enable_timing(s->drv, 1);
        // windows are a few cycles long, so their detector columns, not an
        // observable's long walk, set stage 1: wide emission by default
        gp_tuning t{};
        gp_get_tuning(s->drv, &t);
        t.stage1_wide_emit = 1;
        const gp_status ts = gp_set_tuning(s->drv, &t);
        if (ts != GP_OK) return cleanup(ts);
    }
    // pinned staging
    s->h_desc_bytes = ((s->sealblk_bytes + 15u) & ~(uint64_t)15u) + nseg * sizeof(SegDesc) + Bt * s->extra_ops * sizeof(uint4) +
                      Bt * s->extra_recs * sizeof(uint32_t);
    if (cudaMallocHost(&s->h_desc, s->h_desc_bytes) != cudaSuccess ||
        cudaMallocHost(&s->h_stage_ops, sizeof(uint4) * (uint64_t)c.max_pending * c.max_cycle_ops) != cudaSuccess ||
        cudaMallocHost(&s->h_stage_recs, sizeof(uint32_t) * std::max<uint64_t>((uint64_t)c.max_pending * c.max_cycle_recs, 1)) != cudaSuccess ||
        cudaMallocHost(&s->h_stage_noise, sizeof(float) * std::max<uint64_t>((uint64_t)c.max_pending * c.max_cycle_locations, 1)) != cudaSuccess ||
        cudaMallocHost(&s->h_horizon, sizeof(uint32_t) * Bt) != cudaSuccess ||
        cudaMallocHost(&s->h_starts, sizeof(uint2) * (uint64_t)c.max_cycles_per_step * (Bt + 1)) != cudaSuccess ||
        cudaMallocHost(&s->h_sel, sizeof(SelParams)) != cudaSuccess)
        return cleanup(sfail(GP_ERR_CUDA, "cudaMallocHost of the server staging failed"));
    if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(sfail(GP_ERR_CUDA, "cudaStreamCreate failed"));
    for (uint32_t i = 0; i < c.max_pending; i++) s->free_stage.push_back(c.max_pending - 1 - i);
    *out = s;
    return GP_OK;
}

void gp_server_destroy(gp_server *s) {
    if (!s) return;
    if (s->sel_exec) cudaGraphExecDestroy(s->sel_exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->drv) gp_driver_destroy(s->drv);
    if (s->dmem) cudaFree(s->dmem);
    free_host(s);
    delete s;
}

gp_status gp_server_open_patch(gp_server *s, const gp_patch_spec *spec, uint32_t *patch) {
    if (!s || !spec || !patch) return sfail(GP_ERR_INVALID, "null argument");
    const gp_server_config &c = s->cfg;
    if (spec->n_qubits == 0 || spec->n_qubits > c.max_qubits) return sfail(GP_ERR_INVALID, "patch: n_qubits outside 1..max_qubits");
    if (spec->horizon == 0 || spec->horizon > c.max_horizon) return sfail(GP_ERR_INVALID, "patch: horizon outside 1..max_horizon");
    if (spec->n_observables > 64) return sfail(GP_ERR_INVALID, "patch: at most 64 logicals");
    if (spec->n_observables && (!spec->logical_qubits || !spec->logical_offsets))
        return sfail(GP_ERR_INVALID, "patch: null logical arrays");
    uint32_t slot = kNone;
    for (uint32_t p = 0; p < c.max_patches; p++)
        if (!s->patches[p].open) { slot = p; break; }
    if (slot == kNone) return sfail(GP_ERR_CAPACITY, "all max_patches patches are open");
    Patch np;
    np.ring_ops = s->patches[slot].ring_ops;
    np.ring_recs = s->patches[slot].ring_recs;
    np.ring_noise = s->patches[slot].ring_noise;
    np.open = true;
    np.n_qubits = spec->n_qubits;
    np.H = spec->horizon;
    np.n_obs = spec->n_observables;
    const uint32_t total = spec->n_observables ? spec->logical_offsets[spec->n_observables] : 0u;
    if (total > c.max_logical_qubits) return sfail(GP_ERR_INVALID, "patch: logicals larger than max_logical_qubits");
    std::vector<uint32_t> qs;
    for (uint32_t k = 0; k < spec->n_observables; k++) {
        if (spec->logical_offsets[k] > spec->logical_offsets[k + 1]) return sfail(GP_ERR_INVALID, "patch: logical offsets decrease");
        for (uint32_t i = spec->logical_offsets[k]; i < spec->logical_offsets[k + 1]; i++) {
            if (spec->logical_qubits[i] >= spec->n_qubits) return sfail(GP_ERR_INVALID, "patch: logical qubit out of range");
            qs.push_back(spec->logical_qubits[i]);
        }
    }
    std::sort(qs.begin(), qs.end());
    qs.erase(std::unique(qs.begin(), qs.end()), qs.end());
    np.virt_q = qs;
    np.virt_off.push_back(0);
    for (uint32_t k = 0; k < spec->n_observables; k++) {
        for (uint32_t i = spec->logical_offsets[k]; i < spec->logical_offsets[k + 1]; i++) {
            const uint32_t idx = (uint32_t)(std::lower_bound(qs.begin(), qs.end(), spec->logical_qubits[i]) - qs.begin());
            np.virt_recs.push_back((uint32_t)qs.size() - idx);
        }
        np.virt_off.push_back((uint32_t)np.virt_recs.size());
    }
    s->patches[slot] = std::move(np);
    *patch = slot;
    return GP_OK;
}

gp_status gp_server_close_patch(gp_server *s, uint32_t patch) {
    if (!s || patch >= s->cfg.max_patches || !s->patches[patch].open) return sfail(GP_ERR_INVALID, "no such open patch");
    Patch &p = s->patches[patch];
    if (!p.pending.empty()) return sfail(GP_ERR_INVALID, "patch has pending cycles");
    free_registered(p);
    Patch empty;
    empty.ring_ops = p.ring_ops;
    empty.ring_recs = p.ring_recs;
    empty.ring_noise = p.ring_noise;
    p = std::move(empty);
    return GP_OK;
}

}  // extern "C"

namespace {

// The select phase, captured once as a graph on the server's own stream and
// replayed on the caller's: bring the step's parameters to the device, then
// four kernels (windows' first hyperedges and chunks; per-chunk slot counts
// and the horizon test; request starts; the writes into the pinned step
// buffer).  The starts and horizon flags are written to pinned host memory
// by the kernels themselves.  Every size and pointer that changes from step
// to step is read on the device from the parameter block, so one graph
// serves every step.
gp_status ensure_select_graph(gp_server *s) {
    if (s->sel_exec) return GP_OK;
    const gp_server_config &c = s->cfg;
    const Buffers &B = driver_buffers(s->drv);
    const uint32_t grid = 2u * s->n_sms;
    const size_t smem_count = (size_t)c.max_cycles_per_step * sizeof(uint2);
    const size_t smem_write = (size_t)(kSelThreads / 32u) * c.max_cycles_per_step * sizeof(uint2);
    if (smem_write > 48u * 1024u &&
        cudaFuncSetAttribute(sel_write_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_write) != cudaSuccess)
        return sfail(GP_ERR_CUDA, "select graph: shared memory of the write kernel");
    cudaStream_t cs = s->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return sfail(GP_ERR_CUDA, std::string("select graph capture: ") + cudaGetErrorString(e));
    cudaMemcpyAsync(s->d_sel, s->h_sel, sizeof(SelParams), cudaMemcpyHostToDevice, cs);
    sel_prep_kernel<<<1, 256, 0, cs>>>(B, s->d_sel, s->sel, s->h_horizon);
    sel_count_kernel<<<grid, kSelThreads, smem_count, cs>>>(B, s->d_seal, s->d_cyc_tab, s->W + 1u, s->d_rec_tab,
                                                            c.max_horizon, s->d_sel, s->sel, s->h_horizon);
    sel_starts_kernel<<<1, kSelThreads, 0, cs>>>(s->d_sel, s->sel, s->h_starts);
    sel_write_kernel<<<grid, kSelThreads, smem_write, cs>>>(B, s->d_seal, s->d_sel, s->sel);
    cudaGraph_t g = nullptr;
    const cudaError_t launch_err = cudaGetLastError();
    e = cudaStreamEndCapture(cs, &g);
    if (launch_err != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return sfail(GP_ERR_CUDA, std::string("select graph capture: ") +
                                      cudaGetErrorString(launch_err != cudaSuccess ? launch_err : e));
    }
    e = cudaGraphInstantiate(&s->sel_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->sel_exec = nullptr;
        return sfail(GP_ERR_CUDA, std::string("select graph instantiate: ") + cudaGetErrorString(e));
    }
    return GP_OK;
}

// checks of a cycle about to become patch p's next one; fills its sizes
gp_status scan_cycle(const gp_server *s, const Patch &p, const gp_circuit *cyc, const float *noise, CycleScan &sc) {
    const gp_server_config &c = s->cfg;
    if (cyc->n_ops > c.max_cycle_ops || cyc->n_recs > c.max_cycle_recs || cyc->n_locations > c.max_cycle_locations ||
        cyc->n_detectors > c.max_cycle_detectors)
        return sfail(GP_ERR_CAPACITY, "cycle larger than the server's per-cycle bounds");
    if (cyc->n_qubits > p.n_qubits) return sfail(GP_ERR_INVALID, "cycle uses more qubits than its patch");
    if (cyc->n_observables != p.n_obs) return sfail(GP_ERR_INVALID, "cycle's n_observables differs from its patch's logicals");
    if ((cyc->n_ops && !cyc->ops) || (cyc->n_recs && !cyc->recs) || (cyc->n_locations && !noise))
        return sfail(GP_ERR_INVALID, "null cycle arrays");
    const uint4 *ops = reinterpret_cast<const uint4 *>(cyc->ops);
    sc = CycleScan{};
    CycleInfo &ci = sc.ci;
    ci.n_ops = (uint32_t)cyc->n_ops;
    ci.n_recs = (uint32_t)cyc->n_recs;
    ci.n_loc = cyc->n_locations;
    uint64_t meas = 0;          // measurements of the cycle before the row
    uint32_t n_det = 0;
    for (uint64_t i = 0; i < cyc->n_ops; i++) {
        const uint4 op = ops[i];
        const uint32_t k = op.x;
        if (k == K_TICK) ci.n_ticks++;
        else if (is_measure(k)) meas++;
        else if (is_noise(k)) {
            for (uint32_t l = 0; l < 3; l++) ci.mech[l] += n_comp_host(k, l);
            if (op.w >= cyc->n_locations) return sfail(GP_ERR_INVALID, "cycle row " + std::to_string(i) + ": location out of range");
        } else if (k == K_DET || k == K_OBS) {
            if (k == K_OBS && sc.obs_row < 0) sc.obs_row = (int64_t)i;
            if (k == K_DET) n_det++;
            if ((uint64_t)op.y + op.z > cyc->n_recs) return sfail(GP_ERR_INVALID, "cycle row " + std::to_string(i) + ": records out of range");
            for (uint32_t j = 0; j < op.z; j++) {
                const uint32_t lb = cyc->recs[op.y + j];
                if (lb == 0) return sfail(GP_ERR_INVALID, "cycle row " + std::to_string(i) + ": record lookback refers to no earlier measurement");
                if (lb > meas && lb - meas > sc.reach) {
                    sc.reach = lb - meas;
                    sc.reach_row = i;
                }
            }
        }
    }
    ci.n_meas = (uint32_t)meas;
    ci.n_det = n_det;
    if (n_det != cyc->n_detectors) return sfail(GP_ERR_INVALID, "cycle's n_detectors differs from its DETECTOR rows");
    if (ci.n_meas > c.max_cycle_measurements || ci.n_ticks + 1 > c.max_cycle_layers || ci.mech[2] > c.max_cycle_mechanisms)
        return sfail(GP_ERR_CAPACITY, "cycle larger than the server's per-cycle bounds");
    return GP_OK;
}

// the checks that depend on the patch's history: a scanned cycle placed as the
// patch's next one (its bases set)
gp_status admit_cycle(const Patch &p, const CycleScan &sc, bool final, CycleInfo &ci) {
    if (p.final_submitted) return sfail(GP_ERR_INVALID, "patch already ended with a final cycle");
    if (sc.obs_row >= 0 && !final)
        return sfail(GP_ERR_INVALID, "cycle row " + std::to_string(sc.obs_row) +
                                         ": observables are declared per patch; only a final cycle may define them");
    const uint32_t t = (uint32_t)p.cycles.size();
    ci = sc.ci;
    ci.det_base = t ? p.cycles[t - 1].det_base + p.cycles[t - 1].n_det : 0;
    ci.meas_base = t ? p.cycles[t - 1].meas_base + p.cycles[t - 1].n_meas : 0;
    // a record of row i looks back lb measurements from meas_base + (the
    // cycle's measurements before i); the furthest reaches `reach` before
    // the cycle's start, which must lie within the last H cycles
    const uint64_t horizon_meas = t >= p.H ? p.cycles[t - p.H].meas_base : 0;
    if (sc.reach > ci.meas_base)
        return sfail(GP_ERR_INVALID, "cycle row " + std::to_string(sc.reach_row) + ": record lookback refers to no earlier measurement");
    if (ci.meas_base - sc.reach < horizon_meas)
        return sfail(GP_ERR_HORIZON, "cycle row " + std::to_string(sc.reach_row) + ": record lookback reaches more than H cycles back");
    return GP_OK;
}

uint64_t enqueue(gp_server *s, uint32_t patch, const CycleInfo &ci, bool final, uint32_t stage, int32_t reg,
                 uint64_t t_arrival_ns) {
    Patch &p = s->patches[patch];
    p.cycles.push_back(ci);
    if (final) p.final_submitted = true;
    Request r;
    r.id = s->next_request++;
    r.patch = patch;
    r.cycle = (uint32_t)p.cycles.size() - 1u;
    r.final = final;
    r.stage = stage;
    r.reg = reg;
    r.t_arrival = t_arrival_ns ? t_arrival_ns : now_ns();
    const uint64_t id = r.id;
    p.pending.push_back(id);
    s->requests.emplace(id, std::move(r));
    s->n_pending++;
    return id;
}

}  // namespace

extern "C" {

gp_status gp_server_submit(gp_server *s, uint32_t patch, const gp_circuit *cyc, const float *noise, int final,
                           uint64_t t_arrival_ns, uint64_t *request) {
    if (!s || !cyc || !request) return sfail(GP_ERR_INVALID, "null argument");
    const gp_server_config &c = s->cfg;
    if (patch >= c.max_patches || !s->patches[patch].open) return sfail(GP_ERR_INVALID, "no such open patch");
    CycleInfo ci;
    {
        CycleScan sc;
        gp_status st = scan_cycle(s, s->patches[patch], cyc, noise, sc);
        if (st == GP_OK) st = admit_cycle(s->patches[patch], sc, final != 0, ci);
        if (st != GP_OK) return st;
    }
    if (s->free_stage.empty()) return sfail(GP_ERR_CAPACITY, "max_pending cycles are queued");
    // stage the cycle (pinned) until its step uploads it
    const uint32_t slot = s->free_stage.back();
    s->free_stage.pop_back();
    if (cyc->n_ops) memcpy(s->h_stage_ops + (uint64_t)slot * c.max_cycle_ops, cyc->ops, cyc->n_ops * sizeof(uint4));
    if (cyc->n_recs) memcpy(s->h_stage_recs + (uint64_t)slot * c.max_cycle_recs, cyc->recs, cyc->n_recs * sizeof(uint32_t));
    if (cyc->n_locations) memcpy(s->h_stage_noise + (uint64_t)slot * c.max_cycle_locations, noise, cyc->n_locations * sizeof(float));
    *request = enqueue(s, patch, ci, final != 0, slot, -1, t_arrival_ns);
    return GP_OK;
}

gp_status gp_server_register_cycle(gp_server *s, uint32_t patch, const gp_circuit *cyc, const float *noise,
                                   uint32_t *cycle_id) {
    if (!s || !cyc || !cycle_id) return sfail(GP_ERR_INVALID, "null argument");
    const gp_server_config &c = s->cfg;
    if (patch >= c.max_patches || !s->patches[patch].open) return sfail(GP_ERR_INVALID, "no such open patch");
    Registered r;
    {
        // the rows are scanned once here; a submission only places the scan
        const gp_status st = scan_cycle(s, s->patches[patch], cyc, noise, r.scan);
        if (st != GP_OK) return st;
    }
    if (cudaMalloc(&r.d_ops, sizeof(uint4) * std::max<uint64_t>(cyc->n_ops, 1)) != cudaSuccess ||
        cudaMalloc(&r.d_recs, sizeof(uint32_t) * std::max<uint64_t>(cyc->n_recs, 1)) != cudaSuccess ||
        cudaMalloc(&r.d_noise, sizeof(float) * std::max<uint32_t>(cyc->n_locations, 1)) != cudaSuccess ||
        (cyc->n_ops && cudaMemcpy(r.d_ops, cyc->ops, sizeof(uint4) * cyc->n_ops, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (cyc->n_recs && cudaMemcpy(r.d_recs, cyc->recs, sizeof(uint32_t) * cyc->n_recs, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (cyc->n_locations && cudaMemcpy(r.d_noise, noise, sizeof(float) * cyc->n_locations, cudaMemcpyHostToDevice) != cudaSuccess)) {
        Patch tmp;
        tmp.registered.push_back(r);
        free_registered(tmp);
        return sfail(GP_ERR_CUDA, "device copy of a registered cycle failed");
    }
    Patch &p = s->patches[patch];
    p.registered.push_back(r);
    *cycle_id = (uint32_t)p.registered.size() - 1u;
    return GP_OK;
}

gp_status gp_server_submit_registered(gp_server *s, uint32_t patch, uint32_t cycle_id, int final,
                                      uint64_t t_arrival_ns, uint64_t *request) {
    if (!s || !request) return sfail(GP_ERR_INVALID, "null argument");
    const gp_server_config &c = s->cfg;
    if (patch >= c.max_patches || !s->patches[patch].open) return sfail(GP_ERR_INVALID, "no such open patch");
    Patch &p = s->patches[patch];
    if (cycle_id >= p.registered.size()) return sfail(GP_ERR_INVALID, "no such registered cycle");
    if (s->n_pending >= c.max_pending) return sfail(GP_ERR_CAPACITY, "max_pending cycles are queued");
    const Registered &r = p.registered[cycle_id];
    CycleInfo ci;
    {
        const gp_status st = admit_cycle(p, r.scan, final != 0, ci);
        if (st != GP_OK) return st;
    }
    *request = enqueue(s, patch, ci, final != 0, 0u, (int32_t)cycle_id, t_arrival_ns);
    return GP_OK;
}

gp_status gp_server_step(gp_server *s, gp_level level, void *stream, uint32_t *n_completed) {
    if (!s) return sfail(GP_ERR_INVALID, "null argument");
    if ((int)level < 0 || (int)level > 2) return sfail(GP_ERR_INVALID, "level must be GP_L0, GP_L1 or GP_L2");
    if (n_completed) *n_completed = 0;
    const uint64_t t_start = now_ns();
    const gp_server_config &c = s->cfg;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // patches with pending cycles, oldest request first
    std::vector<std::pair<uint64_t, uint32_t>> order;
    for (uint32_t p = 0; p < c.max_patches; p++) {
        const Patch &P = s->patches[p];
        if (P.open && !P.pending.empty()) order.push_back({s->requests.at(P.pending.front()).t_arrival, p});
    }
    if (order.empty()) return GP_OK;
    std::sort(order.begin(), order.end());
    if (order.size() > c.max_batch) order.resize(c.max_batch);

    struct Win {
        uint32_t patch, t_a, t_b, c0, n_rec;
        bool final;
        std::vector<uint64_t> reqs;
        std::vector<uint64_t> det_off;   // window-local detector offset per cycle c0..t_b+1
        std::vector<int32_t> key;        // registered ids of cycles c0..t_b
        bool keyed = false, known = false;
    };
    std::vector<Win> wins;
    // h_desc: the seal block (as in device memory), then the segment
    // descriptors and closing rows that the assembly reads from here
    SealDesc *hseal = reinterpret_cast<SealDesc *>(s->h_desc);
    uint2 *hrtab = reinterpret_cast<uint2 *>(hseal + c.max_batch);
    uint32_t *hctab = reinterpret_cast<uint32_t *>(hrtab + (uint64_t)c.max_batch * c.max_horizon);
    SegDesc *hseg = reinterpret_cast<SegDesc *>(s->h_desc + ((s->sealblk_bytes + 15u) & ~(uint64_t)15u));
    const uint64_t nseg_cap = (uint64_t)c.max_batch * (s->W + 1);
    uint4 *hxops = reinterpret_cast<uint4 *>(hseg + nseg_cap);
    uint32_t *hxrecs = reinterpret_cast<uint32_t *>(hxops + (uint64_t)c.max_batch * s->extra_ops);
    std::vector<gp_circuit> circ;
    uint32_t nseg = 0;
    uint64_t a_ops = 0, a_recs = 0, a_loc = 0, x_ops = 0, x_recs = 0;
    for (const auto &pr : order) {
        const uint32_t pi = pr.second;
        Patch &P = s->patches[pi];
        Win w;
        w.patch = pi;
        w.t_a = P.next_step;
        w.t_b = w.t_a;
        w.final = false;
        for (uint64_t id : P.pending) {
            const Request &r = s->requests.at(id);
            if (r.cycle != w.t_a + (uint32_t)w.reqs.size() || w.reqs.size() >= c.max_cycles_per_step) break;
            w.reqs.push_back(id);
            w.t_b = r.cycle;
            if (r.final) { w.final = true; break; }
        }
        w.c0 = w.t_a > 3u * P.H ? w.t_a - 3u * P.H : 0u;
        w.n_rec = w.c0 > 0 ? P.H : 0u;
        // upload the new cycles into their ring slots
        for (uint64_t id : w.reqs) {
            const Request &r = s->requests.at(id);
            CycleInfo &ci = P.cycles[r.cycle];
            ci.reg = r.reg;
            if (r.reg >= 0) {
                // a registered cycle is read from its device copy
                const Registered &g = P.registered[r.reg];
                ci.src_ops = g.d_ops;
                ci.src_recs = g.d_recs;
                ci.src_noise = g.d_noise;
                continue;
            }
            const uint32_t slot = r.cycle % s->W;
            ci.src_ops = P.ring_ops + (uint64_t)slot * c.max_cycle_ops;
            ci.src_recs = P.ring_recs + (uint64_t)slot * c.max_cycle_recs;
            ci.src_noise = P.ring_noise + (uint64_t)slot * c.max_cycle_locations;
            if (ci.n_ops)
                SV_CUDA(cudaMemcpyAsync(P.ring_ops + (uint64_t)slot * c.max_cycle_ops, s->h_stage_ops + (uint64_t)r.stage * c.max_cycle_ops,
                                        ci.n_ops * sizeof(uint4), cudaMemcpyHostToDevice, st));
            if (ci.n_recs)
                SV_CUDA(cudaMemcpyAsync(P.ring_recs + (uint64_t)slot * c.max_cycle_recs, s->h_stage_recs + (uint64_t)r.stage * c.max_cycle_recs,
                                        ci.n_recs * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
            if (ci.n_loc)
                SV_CUDA(cudaMemcpyAsync(P.ring_noise + (uint64_t)slot * c.max_cycle_locations,
                                        s->h_stage_noise + (uint64_t)r.stage * c.max_cycle_locations, ci.n_loc * sizeof(float),
                                        cudaMemcpyHostToDevice, st));
        }
        // a window of registered cycles that passed the horizon test before
        // passes it again: its records-only cycles' noise is left out
        w.keyed = !w.final && w.n_rec > 0;
        for (uint32_t k = w.c0; k <= w.t_b; k++) {
            w.key.push_back(P.cycles[k].reg);
            if (P.cycles[k].reg < 0) w.keyed = false;
        }
        w.known = w.keyed && P.verified.count(w.key) != 0;
        // segments of the window
        gp_circuit g{};
        const uint64_t ops0 = a_ops, recs0 = a_recs, loc0 = a_loc;
        uint32_t n_det = 0, mech_rec = 0;
        w.det_off.push_back(0);
        for (uint32_t k = w.c0; k <= w.t_b; k++) {
            const CycleInfo &ci = P.cycles[k];
            SegDesc &d = hseg[nseg++];
            d.ops = ci.src_ops;
            d.recs = ci.src_recs;
            d.noise = ci.src_noise;
            d.n_ops = ci.n_ops;
            d.n_recs = ci.n_recs;
            d.n_loc = ci.n_loc;
            d.dst_ops = (uint32_t)a_ops;
            d.dst_recs = (uint32_t)a_recs;
            d.dst_loc = (uint32_t)a_loc;
            d.rec_shift = (uint32_t)(a_recs - recs0);
            d.loc_shift = (uint32_t)(a_loc - loc0);
            const bool rec_only = k < w.c0 + w.n_rec;
            // a mechanism of the last H cycles of a window that does not end
            // the patch only flips detectors of those cycles or later, after
            // every cycle the window seals: its hyperedge is not delivered,
            // and no delivered hyperedge has its mask, so it is left out
            const bool unsealed = !w.final && k + P.H > w.t_b;
            // a records-only cycle's mechanisms only serve the horizon test
            // (none is in a delivered hyperedge when H holds): a final window
            // and a known window leave them out
            const bool untested = rec_only && (w.final || w.known);
            d.flags = (rec_only ? kSegRecordsOnly : 0u) | (unsealed || untested ? kSegNoNoise : 0u);
            d.pad = 0;
            if (rec_only && !untested) mech_rec += ci.mech[(int)level];
            a_ops += ci.n_ops;
            a_recs += ci.n_recs;
            a_loc += ci.n_loc;
            n_det += ci.n_det;
            w.det_off.push_back(n_det);
        }
        if (!w.final) {
            // the rows closing the window: TICK, Z measurements of the logical
            // qubits, one observable per logical
            const uint64_t xo0 = x_ops, xr0 = x_recs;
            hxops[x_ops++] = make_uint4(K_TICK, 0, 0, 0);
            for (uint32_t q : P.virt_q) hxops[x_ops++] = make_uint4(K_M, q, 0, 0);
            const uint32_t rbase = (uint32_t)(a_recs - recs0);
            for (uint32_t k = 0; k < P.n_obs; k++)
                hxops[x_ops++] = make_uint4(K_OBS, rbase + P.virt_off[k], P.virt_off[k + 1] - P.virt_off[k], k);
            for (uint32_t v : P.virt_recs) hxrecs[x_recs++] = v;
            SegDesc &d = hseg[nseg++];
            d.ops = hxops + xo0;
            d.recs = hxrecs + xr0;
            d.noise = nullptr;
            d.n_ops = (uint32_t)(x_ops - xo0);
            d.n_recs = (uint32_t)(x_recs - xr0);
            d.n_loc = 0;
            d.dst_ops = (uint32_t)a_ops;
            d.dst_recs = (uint32_t)a_recs;
            d.dst_loc = (uint32_t)a_loc;
            d.rec_shift = 0;
            d.loc_shift = 0;
            d.flags = 0;
            d.pad = 0;
            a_ops += d.n_ops;
            a_recs += d.n_recs;
        }
        g.ops = reinterpret_cast<const uint32_t *>(s->arena_ops + ops0);
        g.n_ops = a_ops - ops0;
        g.recs = s->arena_recs + recs0;
        g.n_recs = a_recs - recs0;
        g.n_qubits = P.n_qubits;
        g.n_detectors = n_det;
        g.n_observables = P.n_obs;
        g.n_locations = (uint32_t)(a_loc - loc0);
        circ.push_back(g);
        // sealed cycles [lo, hi)
        SealDesc &sd = hseal[wins.size()];
        const uint32_t lo = w.t_a > P.H ? w.t_a - P.H : 0u;
        const uint32_t hi = w.final ? w.t_b + 1u : (w.t_b + 1u > P.H ? w.t_b + 1u - P.H : 0u);
        if (hi > lo) {
            sd.det_lo = (uint32_t)w.det_off[std::max(lo, w.c0) - w.c0];
            sd.det_hi = (uint32_t)w.det_off[hi - w.c0];
        } else {
            sd.det_lo = sd.det_hi = 0;
        }
        sd.take_no_det = w.final ? 1u : 0u;
        sd.det_base = (uint32_t)P.cycles[w.c0].det_base;
        // a final or known window has no records-only mechanisms to test
        sd.n_mech_rec = mech_rec;
        sd.n_rec = w.n_rec;
        sd.n_cyc = w.t_b - w.c0 + 1u;
        sd.r_off = (int32_t)(w.c0 + P.H) - (int32_t)w.t_a;
        sd.r_max = w.t_b - w.t_a;
        sd.pad[0] = sd.pad[1] = sd.pad[2] = 0;
        for (uint32_t j = 0; j <= sd.n_cyc; j++) hctab[wins.size() * (s->W + 1u) + j] = (uint32_t)w.det_off[j];
        {
            uint32_t mend = 0;
            for (uint32_t j = 0; j < w.n_rec; j++) {
                mend += P.cycles[w.c0 + j].mech[(int)level];
                hrtab[wins.size() * c.max_horizon + j] = make_uint2(mend, (uint32_t)w.det_off[j + P.H + 1]);
            }
        }
        wins.push_back(std::move(w));
    }
    const uint32_t n_win = (uint32_t)wins.size();
    // descriptors and closing rows: one copy each
    // descriptors: one copy of the seal block; the assembly reads the
    // segment descriptors and closing rows from pinned host memory
    SV_CUDA(cudaMemcpyAsync(s->d_seal, s->h_desc, s->sealblk_bytes, cudaMemcpyHostToDevice, st));
    assemble_kernel<<<dim3(nseg, kSegBlocksY), 256, 0, st>>>(hseg, nseg, s->arena_ops, s->arena_recs, s->arena_noise);
    SV_CUDA(cudaGetLastError());
    const uint64_t t_built = now_ns();
    gp_dem_view view{};
    gp_status cst = gp_compile_batch(s->drv, circ.data(), n_win, s->arena_noise, 1, level, stream, &view);
    const uint64_t t_compiled = now_ns();
    std::vector<uint32_t> win_status(n_win, GP_OK);
    uint32_t n_slots = 0;
    for (const Win &w : wins) n_slots = std::max<uint32_t>(n_slots, (uint32_t)w.reqs.size());
    const uint32_t rs = n_win + 1u;             // entries of one slot's row of starts
    OutBuf *ob = nullptr;
    if (cst == GP_OK && view.n_edges) {
        // the step buffer is taken before the select phase, for the batch's
        // whole output (the sealed part is at most that), so the kernels can
        // fill it and one synchronisation ends the step
        if (view.n_det_entries > 0xFFFFFFFFull)
            cst = sfail(GP_ERR_CAPACITY, "a step's detector ids exceed 32 bits");
        if (cst == GP_OK) {
            ob = take_outbuf(s, view.n_edges, (uint64_t)n_slots * n_win, view.n_det_entries);
            if (!ob) cst = sfail(GP_ERR_CUDA, "cudaMallocHost of a result buffer failed");
        }
        if (cst == GP_OK) {
            *s->h_sel = SelParams{n_win, n_slots, ob->edges_cap, ob->det_cap,
                                  SealOut{ob->doff, ob->det, ob->prob, ob->logodds, ob->obs}};
            const gp_status gs = ensure_select_graph(s);
            if (gs != GP_OK) cst = gs;
        }
        if (cst == GP_OK) {
            SV_CUDA(cudaGraphLaunch(s->sel_exec, st));
            SV_CUDA(cudaStreamSynchronize(st));
            const uint2 tot = s->h_starts[(size_t)(n_slots - 1u) * rs + n_win];
            if (tot.x + (uint64_t)n_slots * n_win > ob->edges_cap || tot.y > ob->det_cap)
                cst = sfail(GP_ERR_CAPACITY, "sealed output larger than the step's whole output");
            for (uint32_t w = 0; w < n_win; w++) {
                if (s->h_horizon[w]) win_status[w] = GP_ERR_HORIZON;
                // a tested window's pattern passes from now on
                Patch &P = s->patches[wins[w].patch];
                if (wins[w].keyed && !wins[w].known && win_status[w] == GP_OK && P.verified.size() < kMaxVerified)
                    P.verified.insert(wins[w].key);
            }
        }
    }
    const uint64_t t_selected = now_ns();
    // every request's hyperedges are one slice of the step buffer
    if (cst == GP_OK && ob) {
        for (uint32_t w = 0; w < n_win; w++) {
            if (win_status[w] != GP_OK) continue;
            const Win &W_ = wins[w];
            for (uint32_t r = 0; r < (uint32_t)W_.reqs.size(); r++) {
                const uint2 a = s->h_starts[(size_t)r * rs + w], z = s->h_starts[(size_t)r * rs + w + 1];
                Request &q = s->requests.at(W_.reqs[r]);
                q.buf = ob;
                ob->refs++;
                q.n_edges = z.x - a.x;
                q.n_det = z.y - a.y;
                q.det_offsets = ob->doff + a.x + r * n_win + w;
                q.det_idx = ob->det + a.y;
                q.obs = ob->obs + a.x;
                q.prob = ob->prob + a.x;
                q.logodds = ob->logodds + a.x;
            }
        }
    }
    const uint64_t t_done = now_ns();
    uint32_t done = 0;
    for (uint32_t w = 0; w < n_win; w++) {
        Win &W_ = wins[w];
        Patch &P = s->patches[W_.patch];
        for (uint64_t id : W_.reqs) {
            Request &r = s->requests.at(id);
            finish(s, r, cst != GP_OK ? cst : (gp_status)win_status[w], t_done);
            if (r.reg < 0) s->free_stage.push_back(r.stage);
            P.pending.pop_front();
            s->n_pending--;
            done++;
        }
        P.next_step = W_.t_b + 1;
    }
    if (n_completed) *n_completed = done;
    s->times[0] = (float)(t_built - t_start) * 1e-3f;
    s->times[1] = (float)(t_compiled - t_built) * 1e-3f;
    s->times[2] = (float)(t_selected - t_compiled) * 1e-3f;
    s->times[3] = (float)(t_done - t_selected) * 1e-3f;
    gp_last_timing(s->drv, s->times + 4);
    return cst;
}

gp_status gp_server_set_tuning(gp_server *s, const gp_tuning *t) {
    if (!s || !t) return sfail(GP_ERR_INVALID, "null argument");
    return gp_set_tuning(s->drv, t);
}

gp_status gp_server_last_timing(const gp_server *s, float times_us[8]) {
    if (!s || !times_us) return sfail(GP_ERR_INVALID, "null argument");
    for (int i = 0; i < 8; i++) times_us[i] = s->times[i];
    return GP_OK;
}

gp_status gp_server_submit_registered_many(gp_server *s, uint32_t n, const uint32_t *patches,
                                           const uint32_t *cycle_ids, const uint8_t *finals,
                                           const uint64_t *t_arrival_ns, uint64_t *requests, uint32_t *n_done) {
    if (!s || !n_done || (n && (!patches || !cycle_ids || !requests))) return sfail(GP_ERR_INVALID, "null argument");
    *n_done = 0;
    for (uint32_t i = 0; i < n; i++) {
        const gp_status st = gp_server_submit_registered(s, patches[i], cycle_ids[i], finals ? finals[i] : 0,
                                                         t_arrival_ns ? t_arrival_ns[i] : 0, &requests[i]);
        if (st != GP_OK) return st;
        *n_done = i + 1;
    }
    return GP_OK;
}

gp_status gp_server_drain(gp_server *s, uint32_t cap, uint64_t *ids, uint64_t *t_arrival_ns, uint64_t *t_done_ns,
                          uint32_t *n_edges, int32_t *status, uint32_t *n) {
    if (!s || !n || (cap && (!ids || !t_arrival_ns || !t_done_ns || !n_edges || !status)))
        return sfail(GP_ERR_INVALID, "null argument");
    const uint32_t k = (uint32_t)std::min<size_t>(cap, s->completed.size());
    for (uint32_t i = 0; i < k; i++) {
        auto it = s->requests.find(s->completed[i]);
        ids[i] = s->completed[i];
        if (it == s->requests.end()) {
            t_arrival_ns[i] = t_done_ns[i] = 0;
            n_edges[i] = 0;
            status[i] = GP_ERR_INVALID;
            continue;
        }
        t_arrival_ns[i] = it->second.t_arrival;
        t_done_ns[i] = it->second.t_done;
        n_edges[i] = it->second.n_edges;
        status[i] = (int32_t)it->second.status;
        drop_result(it->second);
        s->requests.erase(it);
    }
    s->completed.erase(s->completed.begin(), s->completed.begin() + k);
    *n = k;
    return GP_OK;
}

gp_status gp_server_completed(gp_server *s, uint64_t *ids, uint32_t cap, uint32_t *n) {
    if (!s || !n || (cap && !ids)) return sfail(GP_ERR_INVALID, "null argument");
    const uint32_t k = (uint32_t)std::min<size_t>(cap, s->completed.size());
    for (uint32_t i = 0; i < k; i++) ids[i] = s->completed[i];
    s->completed.erase(s->completed.begin(), s->completed.begin() + k);
    *n = k;
    return GP_OK;
}

gp_status gp_server_result(const gp_server *s, uint64_t request, gp_sealed_view *out) {
    if (!s || !out) return sfail(GP_ERR_INVALID, "null argument");
    auto it = s->requests.find(request);
    if (it == s->requests.end() || !it->second.done) return sfail(GP_ERR_INVALID, "unknown or pending request");
    const Request &r = it->second;
    out->request = r.id;
    out->patch = r.patch;
    out->cycle = r.cycle;
    out->status = r.status;
    out->n_edges = r.n_edges;
    out->n_det_entries = r.n_det;
    out->det_offsets = r.det_offsets;
    out->det_idx = r.det_idx;
    out->obs_mask = reinterpret_cast<const uint64_t *>(r.obs);
    out->prob = r.prob;
    out->logodds = r.logodds;
    out->t_arrival_ns = r.t_arrival;
    out->t_done_ns = r.t_done;
    return GP_OK;
}

gp_status gp_server_release(gp_server *s, uint64_t request) {
    if (!s) return sfail(GP_ERR_INVALID, "null argument");
    auto it = s->requests.find(request);
    if (it == s->requests.end() || !it->second.done) return sfail(GP_ERR_INVALID, "unknown or pending request");
    drop_result(it->second);
    s->requests.erase(it);
    return GP_OK;
}

}  // extern "C"
