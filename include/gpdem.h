/*
 * gpdem.h -- C ABI of the GB300 detector-error-model compiler.
 *
 * The library turns realised, fully unrolled, noisy Clifford circuits into
 * decoding hypergraphs (detector error models, Sec. 2.1.4 of the GreenPeas
 * paper) entirely on one GPU:
 *
 *   lowering          the flat circuit rows are scanned into TICK layers,
 *                     measurement records and mechanism numbering
 *                     (Sec. 2.3.1, "lowering the realised circuit");
 *   stage 1           detector sensitivities are propagated backward through
 *                     the layers as 64-bit bit-planes, one detector word per
 *                     thread block, and every error mechanism receives the
 *                     words of its flip mask (Sec. 3.1, Eqs. slp/init-slp,
 *                     Sec. 2.3.4 for Y and two-qubit components);
 *   stage 2           mechanisms are grouped by exact mask equality and the
 *                     probabilities of each class are combined as
 *                     P = (1 - prod(1 - 2 q_i)) / 2 (Eq. pmerge, Sec. 3.2),
 *                     and the hyperedges are compacted.
 * An adjoint kernel returns d(loss)/d(noise) for losses linear in the
 * hyperedge probabilities and log-odds weights.
 *
 * Conventions
 *  - Every entry point returns gp_status; GP_OK is 0.  On failure
 *    gp_last_error() returns a message for the calling thread.  No entry
 *    point throws, aborts or traps.
 *  - Pointers marked "host" are read before the call returns and stay owned
 *    by the caller.  Pointers marked "device" are CUDA device addresses on
 *    the driver's device; they must stay valid until the work that reads
 *    them has finished (gp_compile reads them before returning; the noise
 *    vector of a compile is read again by gp_backward).
 *  - Result arrays are device memory owned by the driver and valid until the
 *    next gp_compile / gp_compile_batch on the same driver.
 *  - A driver is not thread-safe; use one driver per host thread.
 *  - All work is issued on the caller's CUDA stream (cudaStream_t passed as
 *    void*, NULL = legacy default stream).
 */
#ifndef GPDEM_H
#define GPDEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GP_OK = 0,
    GP_ERR_INVALID = 1,          /* malformed circuit or argument            */
    GP_ERR_NONDETERMINISTIC = 2, /* a detector/observable is not determined  */
    GP_ERR_CAPACITY = 3,         /* exceeds the driver's bounds              */
    GP_ERR_CUDA = 4,             /* a CUDA runtime call failed               */
    GP_ERR_TIMEOUT = 5,          /* a bounded device wait gave up            */
    GP_ERR_HORIZON = 6           /* serving window exceeded                  */
} gp_status;

/* Correlation level (Table tab:correlation-level, Sec. 3.3).  Two-qubit
 * depolarising channels keep 6 / 10 / 15 Pauli components; one-qubit
 * depolarising channels keep X and Z at L0 and X, Y, Z at L1 and L2. */
typedef enum { GP_L0 = 0, GP_L1 = 1, GP_L2 = 2 } gp_level;

/* Flat circuit row kinds (rows are 4 x uint32 = {kind, a, b, c}).
 *   TICK                      layer boundary
 *   R, M, MR, RX, MX, MRX     a = qubit
 *   H, S                      a = qubit
 *   CX                        a = control, b = target
 *   CZ                        a, b = qubits
 *   DETECTOR                  a = offset into recs, b = number of records
 *   OBSERVABLE_INCLUDE        a = offset, b = number of records, c = index (< 64)
 *   X_ERROR, Z_ERROR,
 *   DEPOLARIZE1               a = qubit, c = noise location
 *   DEPOLARIZE2               a, b = qubits, c = noise location
 *   NOP                       no operation (the row is ignored; the server
 *                             blanks the noise rows it leaves out with it)
 * recs[] holds measurement-record lookbacks k >= 1 (k-th most recent
 * measurement before the annotation).  Between two TICKs a qubit takes part
 * in at most one gate; a noise row on a qubit that still has a gate later in
 * the same layer acts before that gate, otherwise after it (a two-qubit noise
 * row must be on the same side for both qubits).  Violations give
 * GP_ERR_INVALID. */
enum {
    GP_TICK = 0, GP_R = 1, GP_M = 2, GP_MR = 3, GP_RX = 4, GP_MX = 5, GP_MRX = 6, GP_NOP = 7,
    GP_H = 8, GP_S = 9, GP_CX = 10, GP_CZ = 11,
    GP_DETECTOR = 16, GP_OBSERVABLE_INCLUDE = 17,
    GP_X_ERROR = 32, GP_Z_ERROR = 33, GP_DEPOLARIZE1 = 34, GP_DEPOLARIZE2 = 35
};

/* Channel parameter p per noise location: X_ERROR / Z_ERROR flip with
 * probability p (0 <= p <= 1/2); DEPOLARIZE1 applies each non-identity Pauli
 * with p/3 (p <= 3/4); DEPOLARIZE2 each of the fifteen with p/15
 * (p <= 15/16).  Locations with p = 0 contribute no mechanism. */

typedef struct {
    const uint32_t *ops;      /* n_ops x 4 rows (host or device)            */
    uint64_t n_ops;
    const uint32_t *recs;     /* n_recs lookbacks (host or device)          */
    uint64_t n_recs;
    uint32_t n_qubits;        /* qubits are 0 .. n_qubits-1                 */
    uint32_t n_detectors;     /* must equal the number of DETECTOR rows     */
    uint32_t n_observables;   /* 1 + largest observable index, <= 64        */
    uint32_t n_locations;     /* length of this circuit's noise vector      */
} gp_circuit;

/* Capacity of a driver (Sec. 3.4, buffer reuse: a driver built for a maximal
 * circuit serves every circuit within these bounds without allocating).
 * Totals are summed over the circuits of one batch. */
typedef struct {
    uint32_t max_circuits;        /* circuits per batch                       */
    uint32_t max_qubits;          /* qubits of the widest circuit (<= 8192)  */
    uint64_t max_ops;             /* total rows                               */
    uint64_t max_recs;            /* total record lookbacks                   */
    uint32_t max_layers;          /* total TICK layers                        */
    uint32_t max_measurements;    /* total measurements                       */
    uint32_t max_detectors;       /* total detectors                          */
    uint32_t max_locations;       /* total noise locations                    */
    uint32_t max_mechanisms;      /* total error mechanisms                   */
    uint32_t max_mask_words;      /* non-zero 64-bit words in one mechanism's
                                     mask (0 = default 16, at most 16); the
                                     pool for all words holds 4 per mechanism
                                     of max_mechanisms on average            */
    uint64_t max_det_entries;     /* total detector ids over all hyperedges
                                     (0 = 16 x max_mechanisms)                */
} gp_bounds;

/* Device-resident view of the last compile's result (all device pointers,
 * driver-owned, valid until the next compile on the driver). */
typedef struct {
    uint32_t n_circuits;
    uint32_t n_edges;             /* hyperedges over all circuits             */
    uint64_t n_det_entries;
    uint32_t n_mechanisms;        /* mechanisms over all circuits (incl. those
                                     that flip nothing)                      */
    uint32_t pad;
    const uint32_t *det_offsets;  /* n_edges + 1; edge e's detectors are
                                     det_idx[det_offsets[e] .. det_offsets[e+1]) */
    const uint32_t *det_idx;      /* ascending detector indices (per circuit) */
    const uint64_t *obs_mask;     /* bit k = observable k                     */
    const float *prob;            /* P of the class (Eq. pmerge), FP32        */
    const float *logodds;         /* w = log((1 - P) / P), FP32               */
    const uint32_t *edge_circuit; /* circuit of each edge                     */
    const int32_t *mech_class;    /* n_mechanisms: edge of each mechanism or -1.
                                     Mechanisms are numbered circuit by circuit,
                                     noise rows in row order, and within a row
                                     the components in the order of
                                     tab:correlation-level (one-qubit channels
                                     X, Z, Y; two-qubit IX IZ XI XX ZI ZZ, then
                                     IY XZ YI ZX, then XY YX YY YZ ZY), keeping
                                     only those of the compile's level.       */
    const uint32_t *edge_offsets; /* HOST array, n_circuits + 1: circuit b owns
                                     edges [edge_offsets[b], edge_offsets[b+1]) */
} gp_dem_view;

typedef struct gp_driver gp_driver;

/* Device bytes a driver with these bounds needs (the workspace that
 * gp_driver_create carves its buffers from). */
gp_status gp_workspace_size(const gp_bounds *bounds, uint64_t *bytes);

/* Create a driver on the current CUDA device (Sec. 3.4, buffer reuse: the
 * paper builds its driver once from a maximal circuit, then compiles every
 * realised circuit within it into the same buffers; here the maximal circuit
 * is given by its bounds).  d_workspace: device memory of
 * at least gp_workspace_size bytes, 256-byte aligned, owned by the caller and
 * kept alive until gp_driver_destroy; NULL lets the driver allocate (and
 * free) its own.  Pinned host staging buffers are allocated here, never
 * during a compile.  Returns GP_ERR_INVALID for unusable bounds. */
gp_status gp_driver_create(const gp_bounds *bounds, void *d_workspace,
                           uint64_t workspace_bytes, gp_driver **out);
void gp_driver_destroy(gp_driver *drv);

/* Compile a batch of circuits into one set of hyperedges (Secs. 3.1-3.2).
 * circuits: host array of n_circuits descriptors; their ops/recs pointers are
 * device addresses if inputs_on_device, else host addresses.  noise: the
 * concatenation of every circuit's noise vector (sum of n_locations floats),
 * device or host likewise.  Host arrays are read by the device itself when
 * it addresses pageable host memory coherently (a Grace-Blackwell node) and
 * every array is 4-byte aligned; otherwise they are copied through the
 * driver's pinned staging buffers.  On GP_OK *out describes the result.  The
 * call returns after the work has finished on `stream` (it reads back a small
 * status block).  Errors: GP_ERR_INVALID (malformed rows, noise outside a
 * channel's range), GP_ERR_NONDETERMINISTIC, GP_ERR_CAPACITY, GP_ERR_CUDA. */
gp_status gp_compile_batch(gp_driver *drv, const gp_circuit *circuits,
                           uint32_t n_circuits, const float *noise,
                           int inputs_on_device, gp_level level, void *stream,
                           gp_dem_view *out);

/* gp_compile_batch with one circuit: the paper's just-in-time compile of one
 * realised circuit into its decoding hypergraph (Secs. 3.1-3.2; its usage
 * listing, lst:basic-example, builds the driver once and then compiles each
 * realised circuit with its noise vector).  Same arguments, ownership and
 * errors as gp_compile_batch with n_circuits = 1. */
gp_status gp_compile(gp_driver *drv, const gp_circuit *circuit,
                     const float *noise, int inputs_on_device, gp_level level,
                     void *stream, gp_dem_view *out);

/* Vector-Jacobian product of the last compile (not in the paper; used to fit
 * noise parameters): given device arrays g_prob[n_edges] and
 * g_logodds[n_edges] (either may be NULL = zeros), writes
 *   g_noise[l] = sum_e g_prob[e] dP_e/dp_l + g_logodds[e] dw_e/dp_l
 * for every location l of the batch (device array, length = total
 * n_locations).  Uses dP/dq_i = prod_{j != i} (1 - 2 q_j) over the class of
 * mechanism i and dw/dP = -1 / (P (1 - P)).  Accumulation is exact
 * fixed-point, so the result does not depend on scheduling. */
gp_status gp_backward(gp_driver *drv, const float *g_prob,
                      const float *g_logodds, float *g_noise, void *stream);

/* View of the last successful compile: the detector error model of
 * Sec. 2.1.4 (hyperedges as detector lists with observable masks,
 * probabilities and weights), as device arrays owned by the driver and
 * valid until its next compile.  GP_ERR_INVALID when the driver holds no
 * successful compile. */
gp_status gp_result_view(const gp_driver *drv, gp_dem_view *out);

/* Host copy of the last successful compile's hyperedges into caller-owned
 * host arrays (any may be NULL to skip it): det_offsets[n_edges + 1],
 * det_idx[n_det_entries], obs_mask[n_edges], prob[n_edges],
 * logodds[n_edges].  On a device that addresses host memory coherently, and
 * with every array 4-byte aligned, one device pass writes them all; else
 * one asynchronous copy per array.  Returns after the copies have finished
 * on `stream`.  Errors: GP_ERR_INVALID (no result), GP_ERR_CUDA. */
gp_status gp_result_to_host(gp_driver *drv, uint32_t *det_offsets, uint32_t *det_idx,
                            uint64_t *obs_mask, float *prob, float *logodds, void *stream);

/* Host output (not in the paper): caller-owned arrays in host memory that
 * every later compile on the driver also fills, from its compaction kernel,
 * with the hyperedges of gp_result_to_host -- so no separate copy follows
 * the compile.  det_offsets holds edges_cap + 1 entries, obs_mask, prob and
 * logodds edges_cap, det_idx det_cap.  The memory must be addressable by the
 * device: page-locked (cudaHostAlloc / cudaHostRegister), or any host memory
 * on a device that reads pageable memory coherently.  The arrays are 4-byte
 * aligned (obs_mask 8), owned by the caller and must outlive their use; they
 * are complete when the compile returns.  A compile whose hyperedges exceed
 * a capacity fails with GP_ERR_CAPACITY (the arrays then hold what fitted). */
typedef struct {
    uint32_t *det_offsets;
    uint32_t *det_idx;
    uint64_t *obs_mask;
    float *prob;
    float *logodds;
    uint64_t edges_cap;
    uint64_t det_cap;
} gp_host_output;
/* out == NULL turns the host output off.  Errors: GP_ERR_INVALID (a NULL
 * array, misaligned or non-addressable memory, zero edges_cap). */
gp_status gp_set_host_output(gp_driver *drv, const gp_host_output *out);

/* Tunable launch and work-split parameters (picked by the package's
 * autotuner; not in the paper).  None changes a compile's result.
 *   obs_words     the observables of a circuit are split evenly over
 *                 min(n_observables, obs_words) word columns, each walked on
 *                 its own (Sec. 3.1 walks one observable word); a mechanism
 *                 then carries one mask word per column it flips, so
 *                 bounds.max_mask_words counts these words.
 *   obs_segments  the most work items one observable column's walk is split
 *                 over in time (each fast-forwards to its own part).
 *   stage1_wide_emit  1: steps of many active qubits have their noise rows
 *                 and Pauli components dealt out one per lane (faster wide
 *                 detector columns, e.g. non-local codes; a slightly slower
 *                 observable walk); 0: one active qubit per half-warp. */
typedef struct {
    uint32_t stage1_threads;      /* 128, 256, 512 or 1024                    */
    uint32_t stage1_blocks_per_sm;/* resident blocks per SM for stage 1 (0 = max) */
    uint32_t stage2_threads;      /* 128, 256 or 512                          */
    uint32_t stage2_blocks_per_sm;/* grid = SMs x this for grid-stride kernels */
    uint32_t obs_words;           /* 1..8                                     */
    uint32_t obs_segments;        /* 1..3                                     */
    uint32_t stage1_wide_emit;    /* 0 or 1                                   */
} gp_tuning;
gp_status gp_set_tuning(gp_driver *drv, const gp_tuning *t);
gp_status gp_get_tuning(const gp_driver *drv, gp_tuning *t);

/* Per-stage device times of the last compile in microseconds, measured with
 * CUDA events on the compile's stream when timing is enabled (enable != 0).
 * times[0] lowering, [1] stage 1, [2] grouping + reduction, [3] compaction. */
gp_status gp_enable_timing(gp_driver *drv, int enable);
gp_status gp_last_timing(const gp_driver *drv, float times_us[4]);

/* Number of kernel launches issued by the last compile / backward call. */
uint32_t gp_last_launch_count(const gp_driver *drv);

/* Thread-local message describing the last failure on this thread (not in
 * the paper: the error channel of this C interface).  The pointer stays
 * valid until the next failing call on the same thread. */
const char *gp_last_error(void);

/* Test knobs (not in the paper).  They exist so that the test-suite can
 * reach code paths that real inputs almost never take:
 *   weak_hash     0: the grouping hash as designed.  1: every mask gets the
 *                 same 32-bit tag, so every probe that meets another class's
 *                 slot must tell the masks apart by comparing them word by
 *                 word.  2: every mask also gets the same first slot (one
 *                 probe chain for all classes; small circuits only).
 *                 Grouping stays exact in every mode; only speed changes.
 *   wait_limit    polls before a bounded device wait gives up and the
 *                 compile returns GP_ERR_TIMEOUT (0: 2^22, the default).
 *   stall_windows 1: stage 1 stages no layer window, so the first wait of
 *                 every walk can only run out (the timeout path, without a
 *                 hang and without a copy in flight).
 * The knobs apply to the driver's later compiles until changed; a driver
 * starts with all of them 0. */
typedef struct {
    uint32_t weak_hash;
    uint32_t wait_limit;
    uint32_t stall_windows;
    uint32_t reserved;            /* must be 0 */
} gp_debug;
gp_status gp_set_debug(gp_driver *drv, const gp_debug *dbg);

/* Class probabilities for callers that may not allocate device memory.
 *
 * (The paper has no counterpart: this is a service entry point.)  A decoder
 * host in a real-time feedback loop with a fixed memory budget, or a process
 * whose device memory is owned by another framework, may be unable to call
 * cudaMalloc: it cannot take the allocator's device-wide locks or accept the
 * implicit synchronisation an allocation can bring.  This call needs no
 * driver and allocates nothing.  Given, in device memory, the class of each
 * of n_mech mechanisms (mech_class[i] in [0, n_classes), anything else is
 * skipped) and each mechanism's component probability q[i] in [0, 1/2], it
 * writes prob[c] = (1 - prod_{i in c} (1 - 2 q_i)) / 2 and, if logodds is not
 * NULL, logodds[c] = log((1 - prob[c]) / prob[c]) for every class c: the
 * same combination as gp_compile's (Eq. pmerge), equal to it within the
 * library's FP32 tolerance but not bit for bit (gp_compile starts from the
 * channel parameter p, this call from the component probability q).
 * Members with q = 0 contribute nothing, q >= 1/2 saturates the class at
 * prob = 1/2 (logodds 0), and a class with no member of positive q gets
 * prob = 0 and logodds = +infinity.  All pointers are device
 * pointers owned by the caller; work is queued on `stream` and the call
 * returns without waiting for it.
 *
 * Its scratch is a built-in device array of 2^19 classes (8 MiB), which every
 * GPU that loads the library keeps until the process exits.  More than
 * 524,288 classes gives GP_ERR_CAPACITY.  The first call on a device looks up
 * that array's address on the current device and remembers it; make that
 * first call before any stream capture.  A device reset (cudaDeviceReset)
 * after that first call is not supported: the remembered address would be
 * stale.  Each call zeroes the part of the
 * array it uses before using it, but all calls share the one array: calls
 * whose work overlaps on the GPU (different streams or host threads) race and
 * must be serialised by the caller. */
gp_status gp_pmerge_noalloc(const int32_t *mech_class, const float *q, uint32_t n_mech,
                            uint32_t n_classes, float *prob, float *logodds, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GPDEM_H */
