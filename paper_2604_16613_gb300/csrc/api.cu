// api.cu -- host side of the C ABI declared in include/gpdem.h.
//
// A driver owns one device workspace (caller-provided or allocated here) that
// is carved into every buffer the pipeline needs, sized from gp_bounds
// (Sec. 3.4: buffers are built once for a maximal circuit and reused), plus
// pinned host staging for the per-compile parameter block.  A compile fills
// the parameter block on the host, uploads it with one copy, launches the
// kernels on the caller's stream and reads back a small status block.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

using namespace gpdem;

namespace {

thread_local std::string g_last_error;

gp_status fail(gp_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define GP_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

struct Layout {
    // sizes derived from the bounds
    uint32_t max_tiles, max_cols, max_layer_slots, S, table_log2, max_scan_blocks;
    uint64_t max_det_entries;
    uint64_t qidx_cap16;         // layer index arena, 16-byte units
    uint64_t rec_cap;
    uint32_t ov_cap;             // overflow words (beyond kInlineWords per mechanism)
    // byte offsets in the workspace
    uint64_t total = 0;
    uint64_t params_bytes = 0;   // Params + Status + circuits + tiles + items + col_circ
};

struct Carver {
    unsigned char *base;
    uint64_t off = 0;
    template <class T> T *take(uint64_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

bool bounds_ok(const gp_bounds &b, std::string &why) {
    if (b.max_circuits == 0 || b.max_qubits == 0 || b.max_ops == 0 || b.max_mechanisms == 0) {
        why = "bounds: max_circuits, max_qubits, max_ops and max_mechanisms must be positive";
        return false;
    }
    if (b.max_qubits > 8192) { why = "bounds: max_qubits above 8192 does not fit stage-1 shared memory"; return false; }
    if (b.max_mask_words > (uint32_t)kMaxMaskWords) { why = "bounds: max_mask_words above 16"; return false; }
    if (b.max_ops > 0xFFFFFFFFull || b.max_recs > 0xFFFFFFFFull) { why = "bounds: max_ops and max_recs must fit 32 bits"; return false; }
    if (b.max_mechanisms > 0x7FFFFFFFu) { why = "bounds: max_mechanisms too large"; return false; }
    if (b.max_measurements > kMaxMeasurements) { why = "bounds: max_measurements above 2^28"; return false; }
    return true;
}

Layout make_layout(const gp_bounds &b) {
    Layout L;
    L.max_tiles = (uint32_t)((b.max_ops + kRowTile - 1) / kRowTile) + b.max_circuits;
    L.max_cols = b.max_detectors / 64u + (1u + kMaxObsWords) * b.max_circuits + 1u;
    L.max_layer_slots = b.max_layers + 2u * b.max_circuits;
    L.S = b.max_mask_words ? b.max_mask_words : (uint32_t)kMaxMaskWords;
    // classes never outnumber mechanisms: at least 1.5 slots per mechanism
    // keeps the open-addressing load factor below 2/3
    uint32_t lg = 10;
    while ((double)(1ull << lg) < 1.5 * (double)b.max_mechanisms) lg++;
    L.table_log2 = lg;
    L.max_scan_blocks = (b.max_mechanisms + kMechPerBlockScan - 1) / kMechPerBlockScan;
    L.max_det_entries = b.max_det_entries ? b.max_det_entries : 16ull * b.max_mechanisms;
    // mask words over all mechanisms: four per mechanism on average (the
    // workloads here average 2 to 2.5), plus the unused chunk tails that
    // stage-1 warps may leave
    L.rec_cap = std::min<uint64_t>(4ull * b.max_mechanisms + kPoolSlack, 0xFFFFFFF0ull);
    // words beyond the inline slots: the workloads here put 0 to 6 % of their
    // mechanisms above four words; a quarter of the mechanisms plus 2^16 spare
    L.ov_cap = (uint32_t)std::min<uint64_t>((uint64_t)b.max_mechanisms / 4u + 65536u, 0xFFFFFFF0ull);
    // one qubit index block per layer slot at the widest circuit
    L.qidx_cap16 = (uint64_t)L.max_layer_slots * (layer_geo(b.max_qubits).bytes / 16u);
    return L;
}

// carve every buffer; with base == nullptr only the size is computed
Buffers carve_buffers(const gp_bounds &bd, const Layout &L, unsigned char *base, uint64_t *total,
                      uint64_t *params_bytes) {
    Buffers B{};
    Carver c{base};
    // parameter block (one host->device copy per compile)
    B.params = c.take<Params>(1);
    B.status = c.take<Status>(1);
    B.circ = c.take<CircuitDev>(bd.max_circuits);
    B.tiles = c.take<uint2>(L.max_tiles);
    B.items = c.take<uint32_t>(L.max_cols + (kMaxSegments - 1u) * kMaxObsWords * bd.max_circuits);   // + segment items
    B.col_circ = c.take<uint32_t>(L.max_cols);
    if (params_bytes) *params_bytes = align_up(c.off, 256);
    B.ops_arena = c.take<uint4>(bd.max_ops);
    B.recs_arena = c.take<uint32_t>(std::max<uint64_t>(bd.max_recs, 1));
    B.noise_arena = c.take<float>(std::max<uint32_t>(bd.max_locations, 1));
    B.aux = c.take<uint32_t>(bd.max_ops);
    B.lists = c.take<uint2>(2ull * bd.max_ops + 4);
    B.qidx = c.take<unsigned char>(16ull * L.qidx_cap16);
    B.layer_seg = c.take<uint4>(L.max_layer_slots + 1);
    B.records = c.take<uint4>(L.rec_cap);
    B.tile_sums = c.take<uint4>(L.max_tiles);
    B.tile_off = c.take<uint4>(L.max_tiles);
    B.layer_start = c.take<uint32_t>(L.max_layer_slots + 1);
    B.meas_lq = c.take<uint2>(std::max<uint32_t>(bd.max_measurements, 1));
    B.det_row = c.take<uint32_t>(std::max<uint32_t>(bd.max_detectors, 1));
    B.obs_rows = c.take<uint32_t>(bd.max_ops);
    B.obs_count = c.take<uint32_t>(bd.max_circuits);
    B.mech_key = c.take<unsigned long long>(bd.max_mechanisms);
    B.mech_info = c.take<unsigned long long>(bd.max_mechanisms);
    B.inl_col = c.take<uint32_t>((uint64_t)kInlineWords * bd.max_mechanisms);
    B.inl_word = c.take<unsigned long long>((uint64_t)kInlineWords * bd.max_mechanisms);
    B.ov_rec = c.take<uint4>(L.ov_cap);
    B.ov_mech = c.take<uint32_t>(L.ov_cap);
    B.ov_head = c.take<uint32_t>(bd.max_mechanisms);
    B.slot_of = c.take<uint32_t>(bd.max_mechanisms);
    B.mech_class = c.take<int32_t>(bd.max_mechanisms);
    B.table = c.take<TabSlot>(1ull << L.table_log2);
    B.scan_val = c.take<uint2>(bd.max_mechanisms);
    B.comp_off = c.take<uint2>((uint64_t)bd.max_mechanisms + 1);
    {
        const uint64_t nb = ((uint64_t)bd.max_mechanisms + 2047) / 2048;
        B.scan_bsum = c.take<uint2>(nb + 1);
    }
    B.det_off = c.take<uint32_t>((uint64_t)bd.max_mechanisms + 1);
    B.det_idx = c.take<uint32_t>(L.max_det_entries);
    B.obs_mask = c.take<unsigned long long>(bd.max_mechanisms);
    B.prob = c.take<float>(bd.max_mechanisms);
    B.logodds = c.take<float>(bd.max_mechanisms);
    B.class_slot = c.take<uint32_t>(bd.max_mechanisms);
    B.edge_mech = c.take<uint32_t>(bd.max_mechanisms);
    B.edge_circ = c.take<uint32_t>(bd.max_mechanisms);
    B.circ_edges = c.take<uint32_t>(bd.max_circuits);
    B.gacc = c.take<unsigned long long>(2ull * std::max<uint32_t>(bd.max_locations, 1));
    if (total) *total = align_up(c.off, 256);
    return B;
}

}  // namespace

namespace gpdem {
// lets other translation units report through gp_last_error()
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace gpdem

struct gp_driver {
    gp_bounds bounds{};
    Layout L{};
    int device = 0, n_sms = 0;
    uint64_t l2_bytes = 0;          // the device's L2 cache
    size_t smem_limit = 0;          // dynamic shared memory a stage-1 block may take
    unsigned char *ws = nullptr;
    bool own_ws = false;
    uint64_t ws_bytes = 0, params_bytes = 0;
    Buffers B{};
    // pinned host staging
    unsigned char *h_params = nullptr;
    Status *h_status = nullptr;
    uint32_t *h_circ_edges = nullptr;
    uint4 *h_ops = nullptr;
    uint32_t *h_recs = nullptr;
    float *h_noise = nullptr;
    // host inputs: gathered by the device straight from the caller's arrays
    // when it can address pageable host memory coherently, else staged
    bool coherent_host = false;
    CopyJob *h_jobs = nullptr;      // pinned: 3 jobs per circuit (at least 8)
    // last result
    bool have_result = false;
    gp_dem_view view{};
    std::vector<uint32_t> edge_offsets;
    uint32_t n_loc_total = 0;
    // the compile pipeline captured as one CUDA graph (re-captured when the
    // tuning or the timing switch changes)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool exec_timing = false;
    gp_tuning exec_tuning{0, 0, 0, 0, 0, 0, 0};
    uint32_t graph_kernels = 0;
    // tuning / instrumentation / test knobs
    gp_tuning tuning{512, 0, 512, 8, 4, kMaxSegments, 0};
    gp_debug debug{0, 0, 0, 0};
    gp_host_output host_out{};          // edges_cap == 0: none
    bool timing = false;
    cudaEvent_t ev[5] = {};
    float times[4] = {0, 0, 0, 0};
    uint32_t launches = 0;
};

namespace gpdem {
const Buffers &driver_buffers(const gp_driver *d) { return d->B; }
uint32_t driver_sms(const gp_driver *d) { return (uint32_t)d->n_sms; }
uint32_t driver_max_det_entries(const gp_driver *d) {
    return (uint32_t)std::min<uint64_t>(d->L.max_det_entries, 0xFFFFFFFFull);
}
}  // namespace gpdem

namespace {

gp_status full_reset(gp_driver *d, cudaStream_t s) {
    const Layout &L = d->L;
    launch_init_table(d->B.table, (size_t)1 << L.table_log2, s);
    GP_CUDA(cudaGetLastError());
    GP_CUDA(cudaMemsetAsync(d->B.mech_key, 0, sizeof(unsigned long long) * (size_t)d->bounds.max_mechanisms, s));
    GP_CUDA(cudaMemsetAsync(d->B.ov_head, 0xFF, sizeof(uint32_t) * (size_t)d->bounds.max_mechanisms, s));
    GP_CUDA(cudaMemsetAsync(d->B.gacc, 0, 2 * sizeof(unsigned long long) * std::max<uint32_t>(d->bounds.max_locations, 1), s));
    GP_CUDA(cudaMemsetAsync(d->B.records, 0xFF, sizeof(uint4) * L.rec_cap, s));
    GP_CUDA(cudaMemsetAsync(d->B.lists, 0, sizeof(uint2) * (2ull * d->bounds.max_ops + 4), s));
    GP_CUDA(cudaMemsetAsync(d->B.qidx, 0, 16ull * L.qidx_cap16, s));
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
}

const char *stage_name(uint32_t code) {
    switch (code) {
    case GP_ERR_INVALID: return "invalid circuit or noise";
    case GP_ERR_NONDETERMINISTIC: return "a detector or observable is not deterministic";
    case GP_ERR_CAPACITY: return "exceeds the driver's bounds";
    case GP_ERR_TIMEOUT: return "device wait timed out";
    default: return "error";
    }
}

std::string describe(const Status &st) {
    char buf[320];
    const uint32_t a = st.info[0], b = st.info[1], c = st.info[2];
    switch (st.code) {
    case GP_ERR_INVALID:
        if (a == 1) snprintf(buf, sizeof buf, "circuit %u: header says %s but the rows hold %u detectors", b, "n_detectors differs", c);
        else if (a == 2) snprintf(buf, sizeof buf, "circuit %u row %u: malformed row (kind, qubit, location, observable index or record lookback)", b, c);
        else if (a == 3) snprintf(buf, sizeof buf, "circuit %u row %u: two-qubit noise acts before a gate on one qubit and after a gate on the other within one TICK layer", b, c);
        else if (a == 4) snprintf(buf, sizeof buf, "circuit %u row %u: a qubit takes part in two gates within one TICK layer", b, c);
        else if (a == 5) { float p; memcpy(&p, &c, 4); snprintf(buf, sizeof buf, "noise location %u: probability %g is outside the channel's range", b, (double)p); }
        else snprintf(buf, sizeof buf, "invalid input (%u, %u, %u)", a, b, c);
        break;
    case GP_ERR_NONDETERMINISTIC:
        if (b == 0xFFFFFFFFu) snprintf(buf, sizeof buf, "circuit %u: a detector or observable of word column %u anticommutes with the initial |0> state", a, c);
        else snprintf(buf, sizeof buf, "circuit %u layer %u: a detector or observable of word column %u anticommutes with a reset or measurement", a, b, c);
        break;
    case GP_ERR_CAPACITY:
        if (a == 1) snprintf(buf, sizeof buf, "%u layer slots needed, bound allows %u", b, c);
        else if (a == 2) snprintf(buf, sizeof buf, "%u measurements, bound allows %u", b, c);
        else if (a == 3) snprintf(buf, sizeof buf, "%u mechanisms, bound allows %u", b, c);
        else if (a == 4) snprintf(buf, sizeof buf, "mechanism %u has %u non-zero mask words, more than max_mask_words", b, c);
        else if (a == 5) snprintf(buf, sizeof buf, "word column %u references %u (measurement, detector) pairs; at most %d", b, c, kMaxEntries);
        else if (a == 6) snprintf(buf, sizeof buf, "hash table of %u slots is full", c);
        else if (a == 7) snprintf(buf, sizeof buf, "%u detector ids in the hyperedges, bound allows %u", b, c);
        else if (a == 8) snprintf(buf, sizeof buf, "mask-word pool of %u entries is full (it holds 4 words per mechanism of max_mechanisms on average plus 2^22 spare)", c);
        else if (a == 9) snprintf(buf, sizeof buf, "circuit %u: the per-layer qubit index needs %u x 16 bytes, more than max_layers x max_qubits allow", b, c);
        else if (a == 10) snprintf(buf, sizeof buf, "circuit %u layer %u: more than %u rows in one TICK layer", b, c, kMaxLayerRows);
        else if (a == 11) snprintf(buf, sizeof buf, "overflow list of %u mask words is full (mechanisms with more than %d words keep the rest there; it holds a quarter of max_mechanisms plus 65536)", c, kInlineWords);
        else snprintf(buf, sizeof buf, "capacity exceeded (%u, %u, %u)", a, b, c);
        break;
    default:
        snprintf(buf, sizeof buf, "%s (%u, %u, %u)", stage_name(st.code), a, b, c);
    }
    return buf;
}

// Everything a compile runs on the device, with grid sizes fixed by the
// bounds (work beyond the actual sizes exits at once), so the sequence can be
// captured once and replayed: parameter upload, lowering, stage 1 (persistent
// blocks over a work queue), grouping, compaction, status read-back.
gp_status enqueue_pipeline(gp_driver *d, cudaStream_t s, uint32_t *kernels) {
    const gp_bounds &bd = d->bounds;
    const Layout &L = d->L;
    const uint32_t grid2 = (uint32_t)d->n_sms * d->tuning.stage2_blocks_per_sm;
    // stage-1 blocks per SM: 0 = one block with the deepest window ring
    const uint32_t want = d->tuning.stage1_blocks_per_sm ? d->tuning.stage1_blocks_per_sm : 1u;
    const Stage1Shape shape1 = stage1_shape(bd.max_qubits, want, d->smem_limit);
    if (shape1.smem > d->smem_limit) return fail(GP_ERR_CAPACITY, "stage 1 does not fit in shared memory with these bounds");
    int occ = 1;
    const bool wide = shape1.split && d->tuning.stage1_wide_emit;
    GP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stage1_kernel_ptr(d->tuning.stage1_threads, wide ? 2u : shape1.split),
                                                          (int)d->tuning.stage1_threads, shape1.smem));
    if (occ < 1) return fail(GP_ERR_CAPACITY, "stage 1 does not fit on an SM with these bounds");
    const uint32_t bps = std::min<uint32_t>(want, (uint32_t)occ);
    const uint32_t grid1 = std::min<uint32_t>((uint32_t)d->n_sms * bps, std::max<uint32_t>(L.max_cols, 1u));
    GP_CUDA(cudaMemcpyAsync(d->B.params, d->h_params, d->params_bytes, cudaMemcpyHostToDevice, s));
    if (d->timing) GP_CUDA(cudaEventRecordWithFlags(d->ev[0], s, cudaEventRecordExternal));
    launch_lowering(d->B, L.max_tiles, L.max_layer_slots, bd.max_qubits, (uint32_t)d->n_sms, s, kernels);
    if (d->timing) GP_CUDA(cudaEventRecordWithFlags(d->ev[1], s, cudaEventRecordExternal));
    launch_stage1(d->B, grid1, d->tuning.stage1_threads, bd.max_qubits, shape1, wide, s, kernels);
    if (d->timing) GP_CUDA(cudaEventRecordWithFlags(d->ev[2], s, cudaEventRecordExternal));
    launch_group(d->B, grid2, d->tuning.stage2_threads, bd.max_mechanisms, s, kernels);
    if (d->timing) GP_CUDA(cudaEventRecordWithFlags(d->ev[3], s, cudaEventRecordExternal));
    launch_compact(d->B, grid2, d->tuning.stage2_threads, bd.max_mechanisms, (uint32_t)d->n_sms, s, kernels);
    if (d->timing) GP_CUDA(cudaEventRecordWithFlags(d->ev[4], s, cudaEventRecordExternal));
    GP_CUDA(cudaGetLastError());
    GP_CUDA(cudaMemcpyAsync(d->h_status, d->B.status, sizeof(Status), cudaMemcpyDeviceToHost, s));
    GP_CUDA(cudaMemcpyAsync(d->h_circ_edges, d->B.circ_edges, sizeof(uint32_t) * bd.max_circuits,
                            cudaMemcpyDeviceToHost, s));
    return GP_OK;
}

// the launch shapes (the observable split only changes the work order the
// host writes per compile)
bool same_tuning(const gp_tuning &a, const gp_tuning &b) {
    return a.stage1_threads == b.stage1_threads && a.stage1_blocks_per_sm == b.stage1_blocks_per_sm &&
           a.stage2_threads == b.stage2_threads && a.stage2_blocks_per_sm == b.stage2_blocks_per_sm &&
           a.stage1_wide_emit == b.stage1_wide_emit;
}

gp_status ensure_graph(gp_driver *d) {
    if (d->exec && d->exec_timing == d->timing && same_tuning(d->exec_tuning, d->tuning)) return GP_OK;
    if (d->exec) {
        cudaGraphExecDestroy(d->exec);
        d->exec = nullptr;
    }
    uint32_t kernels = 0;
    GP_CUDA(cudaStreamBeginCapture(d->cap_stream, cudaStreamCaptureModeThreadLocal));
    const gp_status st = enqueue_pipeline(d, d->cap_stream, &kernels);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(d->cap_stream, &g);
    if (st != GP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(GP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&d->exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        d->exec = nullptr;
        return fail(GP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
    }
    d->exec_timing = d->timing;
    d->exec_tuning = d->tuning;
    d->graph_kernels = kernels;
    return GP_OK;
}

}  // namespace

extern "C" {

const char *gp_last_error(void) { return g_last_error.c_str(); }

gp_status gp_workspace_size(const gp_bounds *bounds, uint64_t *bytes) {
    if (!bounds || !bytes) return fail(GP_ERR_INVALID, "null argument");
    std::string why;
    if (!bounds_ok(*bounds, why)) return fail(GP_ERR_INVALID, why);
    const Layout L = make_layout(*bounds);
    uint64_t total = 0;
    carve_buffers(*bounds, L, nullptr, &total, nullptr);
    *bytes = total;
    return GP_OK;
}

gp_status gp_driver_create(const gp_bounds *bounds, void *d_workspace, uint64_t workspace_bytes, gp_driver **out) {
    if (!bounds || !out) return fail(GP_ERR_INVALID, "null argument");
    *out = nullptr;
    std::string why;
    if (!bounds_ok(*bounds, why)) return fail(GP_ERR_INVALID, why);
    gp_driver *d = new (std::nothrow) gp_driver();
    if (!d) return fail(GP_ERR_CAPACITY, "out of host memory");
    d->bounds = *bounds;
    d->L = make_layout(*bounds);
    uint64_t total = 0, pbytes = 0;
    carve_buffers(*bounds, d->L, nullptr, &total, &pbytes);
    d->ws_bytes = total;
    d->params_bytes = pbytes;
    auto cleanup = [&](gp_status st) { gp_driver_destroy(d); return st; };
    if (cudaGetDevice(&d->device) != cudaSuccess) return cleanup(fail(GP_ERR_CUDA, "cudaGetDevice failed"));
    if (cudaDeviceGetAttribute(&d->n_sms, cudaDevAttrMultiProcessorCount, d->device) != cudaSuccess)
        return cleanup(fail(GP_ERR_CUDA, "cudaDeviceGetAttribute failed"));
    if (d_workspace) {
        if (workspace_bytes < total) return cleanup(fail(GP_ERR_INVALID, "workspace smaller than gp_workspace_size"));
        if (reinterpret_cast<uintptr_t>(d_workspace) % 256) return cleanup(fail(GP_ERR_INVALID, "workspace must be 256-byte aligned"));
        d->ws = static_cast<unsigned char *>(d_workspace);
    } else {
        cudaError_t e = cudaMalloc(&d->ws, total);
        if (e != cudaSuccess) return cleanup(fail(GP_ERR_CUDA, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e)));
        d->own_ws = true;
    }
    d->B = carve_buffers(*bounds, d->L, d->ws, nullptr, nullptr);
    // pinned staging
    if (cudaMallocHost(&d->h_params, pbytes) != cudaSuccess ||
        cudaMallocHost(&d->h_status, sizeof(Status)) != cudaSuccess ||
        cudaMallocHost(&d->h_circ_edges, sizeof(uint32_t) * bounds->max_circuits) != cudaSuccess ||
        cudaMallocHost(&d->h_ops, sizeof(uint4) * bounds->max_ops) != cudaSuccess ||
        cudaMallocHost(&d->h_recs, sizeof(uint32_t) * std::max<uint64_t>(bounds->max_recs, 1)) != cudaSuccess ||
        cudaMallocHost(&d->h_noise, sizeof(float) * std::max<uint32_t>(bounds->max_locations, 1)) != cudaSuccess ||
        cudaMallocHost(&d->h_jobs, sizeof(CopyJob) * std::max<uint64_t>(3ull * bounds->max_circuits, 8)) != cudaSuccess)
        return cleanup(fail(GP_ERR_CUDA, "cudaMallocHost staging failed"));
    {
        int pageable = 0, host_tables = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, d->device) == cudaSuccess &&
            cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, d->device) ==
                cudaSuccess)
            d->coherent_host = pageable == 1 && host_tables == 1;
        // GPDEM_STAGE_HOST_INPUTS=1 keeps the staged copies (both paths are
        // tested against each other)
        const char *env = getenv("GPDEM_STAGE_HOST_INPUTS");
        if (env && env[0] == '1') d->coherent_host = false;
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, d->device) == cudaSuccess && l2 > 0)
            d->l2_bytes = (uint64_t)l2;
    }
    for (int i = 0; i < 5; i++)
        if (cudaEventCreate(&d->ev[i]) != cudaSuccess) return cleanup(fail(GP_ERR_CUDA, "cudaEventCreate failed"));
    if (cudaStreamCreateWithFlags(&d->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(GP_ERR_CUDA, "cudaStreamCreate failed"));
    // initial state of the self-cleaning structures
    cudaStream_t s = 0;
    gp_status st = full_reset(d, s);
    if (st != GP_OK) return cleanup(st);
    // shared memory above the default 48 KB: the stage-1 walk and the
    // per-layer index kernel
    d->smem_limit = stage1_dynamic_smem_limit(d->device);
    if (d->smem_limit == 0) return cleanup(fail(GP_ERR_CUDA, "querying the shared-memory limit failed"));
    for (uint32_t split : {0u, 1u, 2u})
        for (uint32_t t : {128u, 256u, 512u, 1024u}) {
            if (cudaFuncSetAttribute(stage1_kernel_ptr(t, split), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)d->smem_limit) != cudaSuccess)
                return cleanup(fail(GP_ERR_CUDA, "cudaFuncSetAttribute(stage1 shared memory) failed"));
        }
    if (lowering_setup(bounds->max_qubits) != cudaSuccess)
        return cleanup(fail(GP_ERR_CUDA, "cudaFuncSetAttribute(layer index shared memory) failed"));
    *out = d;
    return GP_OK;
}

void gp_driver_destroy(gp_driver *d) {
    if (!d) return;
    if (d->own_ws && d->ws) cudaFree(d->ws);
    if (d->h_params) cudaFreeHost(d->h_params);
    if (d->h_status) cudaFreeHost(d->h_status);
    if (d->h_circ_edges) cudaFreeHost(d->h_circ_edges);
    if (d->h_ops) cudaFreeHost(d->h_ops);
    if (d->h_recs) cudaFreeHost(d->h_recs);
    if (d->h_noise) cudaFreeHost(d->h_noise);
    if (d->h_jobs) cudaFreeHost(d->h_jobs);
    for (int i = 0; i < 5; i++)
        if (d->ev[i]) cudaEventDestroy(d->ev[i]);
    if (d->exec) cudaGraphExecDestroy(d->exec);
    if (d->cap_stream) cudaStreamDestroy(d->cap_stream);
    delete d;
}

gp_status gp_set_tuning(gp_driver *d, const gp_tuning *t) {
    if (!d || !t) return fail(GP_ERR_INVALID, "null argument");
    auto ok_threads = [](uint32_t x) { return x == 128 || x == 256 || x == 512; };
    if (!(ok_threads(t->stage1_threads) || t->stage1_threads == 1024) || !ok_threads(t->stage2_threads) ||
        t->stage2_blocks_per_sm == 0 ||
        t->stage2_blocks_per_sm > 64 || t->stage1_blocks_per_sm > 64 || t->obs_words == 0 ||
        t->obs_words > kMaxObsWords || t->obs_segments == 0 || t->obs_segments > kMaxSegments ||
        t->stage1_wide_emit > 1)
        return fail(GP_ERR_INVALID, "tuning: stage-1 threads 128..1024, stage-2 threads 128..512 (powers of two); "
                                    "blocks per SM 1..64; observable words 1..8; observable segments 1..3; "
                                    "wide emission 0 or 1");
    d->tuning = *t;
    return GP_OK;
}

gp_status gp_get_tuning(const gp_driver *d, gp_tuning *t) {
    if (!d || !t) return fail(GP_ERR_INVALID, "null argument");
    *t = d->tuning;
    return GP_OK;
}

gp_status gp_set_host_output(gp_driver *d, const gp_host_output *o) {
    if (!d) return fail(GP_ERR_INVALID, "null argument");
    if (!o) {
        d->host_out = gp_host_output{};
        return GP_OK;
    }
    if (!o->det_offsets || !o->det_idx || !o->obs_mask || !o->prob || !o->logodds || o->edges_cap == 0)
        return fail(GP_ERR_INVALID, "host output: every array and a positive edges_cap are needed");
    const void *arrays[5] = {o->det_offsets, o->det_idx, o->obs_mask, o->prob, o->logodds};
    for (int i = 0; i < 5; i++) {
        if (reinterpret_cast<uintptr_t>(arrays[i]) % (i == 2 ? 8u : 4u))
            return fail(GP_ERR_INVALID, "host output: misaligned array");
        if (!d->coherent_host) {
            // without coherent access only page-locked memory is addressable
            cudaPointerAttributes a{};
            if (cudaPointerGetAttributes(&a, arrays[i]) != cudaSuccess || a.type != cudaMemoryTypeHost) {
                cudaGetLastError();
                return fail(GP_ERR_INVALID, "host output: memory the device cannot address (page-lock it)");
            }
        }
    }
    d->host_out = *o;
    return GP_OK;
}

gp_status gp_set_debug(gp_driver *d, const gp_debug *dbg) {
    if (!d || !dbg) return fail(GP_ERR_INVALID, "null argument");
    if (dbg->weak_hash > 2u || dbg->stall_windows > 1u || dbg->reserved != 0u)
        return fail(GP_ERR_INVALID, "debug: weak_hash 0..2, stall_windows 0 or 1, reserved 0");
    d->debug = *dbg;
    return GP_OK;
}

gp_status gp_enable_timing(gp_driver *d, int enable) {
    if (!d) return fail(GP_ERR_INVALID, "null argument");
    d->timing = enable != 0;
    return GP_OK;
}

gp_status gp_last_timing(const gp_driver *d, float times_us[4]) {
    if (!d || !times_us) return fail(GP_ERR_INVALID, "null argument");
    for (int i = 0; i < 4; i++) times_us[i] = d->times[i];
    return GP_OK;
}

uint32_t gp_last_launch_count(const gp_driver *d) { return d ? d->launches : 0u; }

gp_status gp_result_view(const gp_driver *d, gp_dem_view *out) {
    if (!d || !out) return fail(GP_ERR_INVALID, "null argument");
    if (!d->have_result) return fail(GP_ERR_INVALID, "no successful compile on this driver");
    *out = d->view;
    return GP_OK;
}

gp_status gp_result_to_host(gp_driver *d, uint32_t *det_offsets, uint32_t *det_idx, uint64_t *obs_mask, float *prob,
                            float *logodds, void *stream) {
    if (!d) return fail(GP_ERR_INVALID, "null argument");
    if (!d->have_result) return fail(GP_ERR_INVALID, "no successful compile on this driver");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const gp_dem_view &v = d->view;
    struct Part { void *dst; const void *src; uint64_t bytes; };
    const Part parts[5] = {
        {det_offsets, v.det_offsets, 4ull * (v.n_edges + 1ull)},
        {det_idx, v.det_idx, 4ull * v.n_det_entries},
        {obs_mask, v.obs_mask, 8ull * v.n_edges},
        {prob, v.prob, 4ull * v.n_edges},
        {logodds, v.logodds, 4ull * v.n_edges},
    };
    uintptr_t bits = 0;
    for (const Part &p : parts) bits |= reinterpret_cast<uintptr_t>(p.dst);
    if (d->coherent_host && (bits & 3u) == 0u) {
        // one device pass writes every array into host memory
        uint32_t nj = 0;
        uint64_t max_bytes = 0;
        for (const Part &p : parts) {
            if (!p.dst || !p.bytes) continue;
            d->h_jobs[nj++] = CopyJob{p.src, p.dst, p.bytes};
            max_bytes = std::max(max_bytes, p.bytes);
        }
        launch_gather_host(d->h_jobs, nj, max_bytes, (uint32_t)d->n_sms, s);
        GP_CUDA(cudaGetLastError());
    } else {
        for (const Part &p : parts)
            if (p.dst && p.bytes) GP_CUDA(cudaMemcpyAsync(p.dst, p.src, p.bytes, cudaMemcpyDeviceToHost, s));
    }
    GP_CUDA(cudaStreamSynchronize(s));
    return GP_OK;
}

// the device gathers host arrays with 4-byte (or 16-byte) loads, so every
// source must be 4-byte aligned; other callers go through the staged copies
static bool host_words_aligned(const gp_circuit *circuits, uint32_t n, const float *noise) {
    uintptr_t bits = reinterpret_cast<uintptr_t>(noise);
    for (uint32_t b = 0; b < n; b++)
        bits |= reinterpret_cast<uintptr_t>(circuits[b].ops) | reinterpret_cast<uintptr_t>(circuits[b].recs);
    return (bits & 3u) == 0u;
}

gp_status gp_compile_batch(gp_driver *d, const gp_circuit *circuits, uint32_t n_circuits, const float *noise,
                           int inputs_on_device, gp_level level, void *stream, gp_dem_view *out) {
    if (!d || !circuits || n_circuits == 0) return fail(GP_ERR_INVALID, "null argument or empty batch");
    if ((int)level < 0 || (int)level > 2) return fail(GP_ERR_INVALID, "level must be GP_L0, GP_L1 or GP_L2");
    const gp_bounds &bd = d->bounds;
    const Layout &L = d->L;
    if (n_circuits > bd.max_circuits) return fail(GP_ERR_CAPACITY, "more circuits than max_circuits");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    d->have_result = false;
    d->launches = 0;

    // ---- host-side parameter block ----------------------------------------
    Params *P = reinterpret_cast<Params *>(d->h_params);
    const uint64_t off_status = reinterpret_cast<unsigned char *>(d->B.status) - reinterpret_cast<unsigned char *>(d->B.params);
    const uint64_t off_circ = reinterpret_cast<unsigned char *>(d->B.circ) - reinterpret_cast<unsigned char *>(d->B.params);
    const uint64_t off_tiles = reinterpret_cast<unsigned char *>(d->B.tiles) - reinterpret_cast<unsigned char *>(d->B.params);
    const uint64_t off_items = reinterpret_cast<unsigned char *>(d->B.items) - reinterpret_cast<unsigned char *>(d->B.params);
    const uint64_t off_colc = reinterpret_cast<unsigned char *>(d->B.col_circ) - reinterpret_cast<unsigned char *>(d->B.params);
    memset(P, 0, sizeof(Params));
    memset(d->h_params + off_status, 0, sizeof(Status));
    CircuitDev *hc = reinterpret_cast<CircuitDev *>(d->h_params + off_circ);
    uint2 *htiles = reinterpret_cast<uint2 *>(d->h_params + off_tiles);
    uint32_t *hitems = reinterpret_cast<uint32_t *>(d->h_params + off_items);
    uint32_t *hcolc = reinterpret_cast<uint32_t *>(d->h_params + off_colc);

    uint64_t ops_total = 0, recs_total = 0, det_total = 0, loc_total = 0;
    uint32_t cols_total = 0, tiles_total = 0;
    for (uint32_t b = 0; b < n_circuits; b++) {
        const gp_circuit &c = circuits[b];
        if (c.n_ops && !c.ops) return fail(GP_ERR_INVALID, "circuit " + std::to_string(b) + ": null ops");
        if (c.n_recs && !c.recs) return fail(GP_ERR_INVALID, "circuit " + std::to_string(b) + ": null recs");
        if (c.n_qubits > bd.max_qubits) return fail(GP_ERR_CAPACITY, "circuit " + std::to_string(b) + ": more qubits than max_qubits");
        if (c.n_observables > 64) return fail(GP_ERR_INVALID, "circuit " + std::to_string(b) + ": at most 64 observables");
        if (c.n_ops > 0xFFFFFFFFull || c.n_recs > 0xFFFFFFFFull) return fail(GP_ERR_CAPACITY, "circuit too long");
        CircuitDev &C = hc[b];
        memset(&C, 0, sizeof C);
        C.n_ops = (uint32_t)c.n_ops;
        C.n_recs = (uint32_t)c.n_recs;
        C.n_qubits = c.n_qubits;
        C.n_det = c.n_detectors;
        C.n_obs = c.n_observables;
        C.n_loc = c.n_locations;
        C.op_base = (uint32_t)ops_total;
        C.det_base = (uint32_t)det_total;
        C.loc_base = (uint32_t)loc_total;
        C.col_base = cols_total;
        // the observables split evenly over up to obs_words word columns
        C.n_ocols = std::min(c.n_observables, d->tuning.obs_words);
        C.obs_per = C.n_ocols ? (c.n_observables + C.n_ocols - 1u) / C.n_ocols : 0u;
        if (C.n_ocols) C.n_ocols = (c.n_observables + C.obs_per - 1u) / C.obs_per;
        C.n_cols = (c.n_detectors + 63u) / 64u + C.n_ocols;
        C.tile_first = tiles_total;
        C.n_tiles = (uint32_t)((c.n_ops + kRowTile - 1) / kRowTile);
        ops_total += c.n_ops;
        recs_total += c.n_recs;
        det_total += c.n_detectors;
        loc_total += c.n_locations;
        cols_total += C.n_cols;
        tiles_total += C.n_tiles;
        if (ops_total > bd.max_ops) return fail(GP_ERR_CAPACITY, "total rows exceed max_ops");
        if (recs_total > bd.max_recs) return fail(GP_ERR_CAPACITY, "total record lookbacks exceed max_recs");
        if (det_total > bd.max_detectors) return fail(GP_ERR_CAPACITY, "total detectors exceed max_detectors");
        if (loc_total > bd.max_locations) return fail(GP_ERR_CAPACITY, "total noise locations exceed max_locations");
        if (cols_total > L.max_cols || tiles_total > L.max_tiles || cols_total > kColMask)
            return fail(GP_ERR_CAPACITY, "batch too large for the driver");
    }
    // stage-1 work order: observable words first (they span whole circuits;
    // with the role-split walk each is obs_segments items, one per segment,
    // the latest-starting first), then detector words in order
    const uint32_t want1 = d->tuning.stage1_blocks_per_sm ? d->tuning.stage1_blocks_per_sm : 1u;
    const bool split_walk = stage1_shape(bd.max_qubits, want1, d->smem_limit).split != 0u;
    uint32_t ni = 0;
    for (uint32_t b = 0; b < n_circuits; b++) {
        const CircuitDev &C = hc[b];
        for (uint32_t k = 0; k < C.n_cols; k++) hcolc[C.col_base + k] = b;
    }
    const uint32_t n_seg = split_walk ? d->tuning.obs_segments : 1u;
    for (uint32_t k = n_seg; k-- > 0;)
        for (uint32_t b = 0; b < n_circuits; b++) {
            const CircuitDev &C = hc[b];
            for (uint32_t o = C.n_cols - C.n_ocols; o < C.n_cols; o++) hitems[ni++] = (C.col_base + o) | (k << kSegShift);
        }
    for (uint32_t b = 0; b < n_circuits; b++) {
        const CircuitDev &C = hc[b];
        const uint32_t nd = C.n_cols - C.n_ocols;
        for (uint32_t k = 0; k < nd; k++) hitems[ni++] = C.col_base + k;
    }
    for (uint32_t b = 0, t = 0; b < n_circuits; b++)
        for (uint32_t k = 0; k < hc[b].n_tiles; k++) htiles[t++] = make_uint2(b, k * (uint32_t)kRowTile);

    // inputs: device pointers as given, or host arrays staged into the arenas
    if (inputs_on_device) {
        for (uint32_t b = 0; b < n_circuits; b++) {
            hc[b].ops = reinterpret_cast<const uint4 *>(circuits[b].ops);
            hc[b].recs = circuits[b].recs;
            if (reinterpret_cast<uintptr_t>(circuits[b].ops) % 16)
                return fail(GP_ERR_INVALID, "device ops must be 16-byte aligned");
        }
        P->noise = noise;
    } else if (d->coherent_host && host_words_aligned(circuits, n_circuits, noise)) {
        // the device reads the caller's arrays itself (no host copy)
        if (loc_total && !noise) return fail(GP_ERR_INVALID, "null noise");
        uint32_t nj = 0;
        uint64_t max_bytes = 0, r0 = 0;
        auto job = [&](const void *src, void *dst, uint64_t bytes) {
            if (!bytes) return;
            d->h_jobs[nj++] = CopyJob{src, dst, bytes};
            max_bytes = std::max(max_bytes, bytes);
        };
        for (uint32_t b = 0; b < n_circuits; b++) {
            const gp_circuit &c = circuits[b];
            hc[b].ops = d->B.ops_arena + hc[b].op_base;
            hc[b].recs = d->B.recs_arena + r0;
            job(c.ops, d->B.ops_arena + hc[b].op_base, c.n_ops * sizeof(uint4));
            job(c.recs, d->B.recs_arena + r0, c.n_recs * sizeof(uint32_t));
            r0 += c.n_recs;
        }
        job(noise, d->B.noise_arena, loc_total * sizeof(float));
        launch_gather_host(d->h_jobs, nj, max_bytes, (uint32_t)d->n_sms, s);
        GP_CUDA(cudaGetLastError());
        P->noise = d->B.noise_arena;
    } else {
        for (uint32_t b = 0; b < n_circuits; b++) {
            const gp_circuit &c = circuits[b];
            if (c.n_ops) memcpy(d->h_ops + hc[b].op_base, c.ops, c.n_ops * sizeof(uint4));
            hc[b].ops = d->B.ops_arena + hc[b].op_base;
        }
        uint64_t r0 = 0;
        for (uint32_t b = 0; b < n_circuits; b++) {
            const gp_circuit &c = circuits[b];
            if (c.n_recs) memcpy(d->h_recs + r0, c.recs, c.n_recs * sizeof(uint32_t));
            hc[b].recs = d->B.recs_arena + r0;
            r0 += c.n_recs;
        }
        if (loc_total) {
            if (!noise) return fail(GP_ERR_INVALID, "null noise");
            memcpy(d->h_noise, noise, loc_total * sizeof(float));
        }
        if (ops_total) GP_CUDA(cudaMemcpyAsync(d->B.ops_arena, d->h_ops, ops_total * sizeof(uint4), cudaMemcpyHostToDevice, s));
        if (recs_total) GP_CUDA(cudaMemcpyAsync(d->B.recs_arena, d->h_recs, recs_total * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        if (loc_total) GP_CUDA(cudaMemcpyAsync(d->B.noise_arena, d->h_noise, loc_total * sizeof(float), cudaMemcpyHostToDevice, s));
        P->noise = d->B.noise_arena;
    }
    if (loc_total && !P->noise) return fail(GP_ERR_INVALID, "null noise");
    P->n_circuits = n_circuits;
    P->n_tiles = tiles_total;
    P->n_items = ni;
    P->level = (uint32_t)level;
    P->n_cols_total = cols_total;
    P->n_loc_total = (uint32_t)loc_total;
    P->table_log2 = L.table_log2;
    P->mask_words = L.S;
    P->max_det_entries = L.max_det_entries;
    P->max_mech = bd.max_mechanisms;
    P->max_layer_slots = L.max_layer_slots;
    P->max_meas = bd.max_measurements;
    P->max_ops = (uint32_t)bd.max_ops;
    P->rec_cap = (uint32_t)L.rec_cap;
    P->max_qubits = bd.max_qubits;
    P->qidx_cap16 = L.qidx_cap16;
    P->weak_hash = d->debug.weak_hash;
    P->wait_limit = d->debug.wait_limit ? d->debug.wait_limit : kWaitPolls;
    P->stall_windows = d->debug.stall_windows;
    P->ov_cap = L.ov_cap;
    P->obs_segments = n_seg;
    P->l2_prefetch_max = d->l2_bytes / 4u * 3u;
    const gp_host_output &ho = d->host_out;
    P->h_det_off = reinterpret_cast<unsigned long long>(ho.edges_cap ? ho.det_offsets : nullptr);
    P->h_det_idx = reinterpret_cast<unsigned long long>(ho.det_idx);
    P->h_obs = reinterpret_cast<unsigned long long>(ho.obs_mask);
    P->h_prob = reinterpret_cast<unsigned long long>(ho.prob);
    P->h_logodds = reinterpret_cast<unsigned long long>(ho.logodds);
    P->h_edges_cap = ho.edges_cap;
    P->h_det_cap = ho.det_cap;
    // ---- pipeline: one graph launch ----------------------------------------------
    {
        const gp_status gs = ensure_graph(d);
        if (gs != GP_OK) return gs;
    }
    GP_CUDA(cudaGraphLaunch(d->exec, s));
    d->launches = d->graph_kernels;
    GP_CUDA(cudaStreamSynchronize(s));
    if (d->timing) {
        for (int i = 0; i < 4; i++) {
            float ms = 0;
            GP_CUDA(cudaEventElapsedTime(&ms, d->ev[i], d->ev[i + 1]));
            d->times[i] = ms * 1000.0f;
        }
    }
    const Status st = *d->h_status;
    if (st.code != 0) {
        const std::string msg = describe(st);
        full_reset(d, s);
        return fail((gp_status)st.code, msg);
    }
    if (d->host_out.edges_cap &&
        (st.n_edges + 1ull > d->host_out.edges_cap + 1ull || st.n_det_entries > d->host_out.det_cap))
        return fail(GP_ERR_CAPACITY, "host output: the compile's hyperedges exceed its capacities");
    // ---- result view -----------------------------------------------------------
    d->n_loc_total = (uint32_t)loc_total;
    d->edge_offsets.assign(n_circuits + 1, 0);
    for (uint32_t b = 0; b < n_circuits; b++) d->edge_offsets[b + 1] = d->edge_offsets[b] + d->h_circ_edges[b];
    gp_dem_view &v = d->view;
    v.n_circuits = n_circuits;
    v.n_edges = st.n_edges;
    v.n_det_entries = st.n_det_entries;
    v.n_mechanisms = st.n_mech;
    v.det_offsets = d->B.det_off;
    v.det_idx = d->B.det_idx;
    v.obs_mask = reinterpret_cast<const uint64_t *>(d->B.obs_mask);
    v.prob = d->B.prob;
    v.logodds = d->B.logodds;
    v.edge_circuit = d->B.edge_circ;
    v.mech_class = d->B.mech_class;
    v.edge_offsets = d->edge_offsets.data();
    d->have_result = true;
    if (out) *out = v;
    return GP_OK;
}

gp_status gp_compile(gp_driver *d, const gp_circuit *circuit, const float *noise, int inputs_on_device,
                     gp_level level, void *stream, gp_dem_view *out) {
    return gp_compile_batch(d, circuit, 1, noise, inputs_on_device, level, stream, out);
}

gp_status gp_backward(gp_driver *d, const float *g_prob, const float *g_logodds, float *g_noise, void *stream) {
    if (!d || !g_noise) return fail(GP_ERR_INVALID, "null argument");
    if (!d->have_result) return fail(GP_ERR_INVALID, "gp_backward needs a successful compile first");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    d->launches = 0;
    const uint32_t grid2 = (uint32_t)d->n_sms * d->tuning.stage2_blocks_per_sm;
    launch_backward(d->B, g_prob, g_logodds, g_noise, d->view.n_mechanisms, d->n_loc_total, grid2,
                    d->tuning.stage2_threads, s, &d->launches);
    GP_CUDA(cudaGetLastError());
    return GP_OK;
}

}  // extern "C"
