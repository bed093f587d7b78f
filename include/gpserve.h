/*
 * gpserve.h -- C ABI of the cycle-streaming server built on gpdem.h.
 *
 * A patch is a memory experiment that arrives one QEC cycle at a time
 * (continuous serving of per-cycle requests).  The paper compiles whole
 * realised circuits and reports compile time per cycle (Sec. 4); the
 * server turns that into per-cycle answers with a bounded amount of work:
 *
 *   - every patch keeps its last 3H + K cycles resident in device memory
 *     (H: how many cycles back a detector's sensitivity and its records
 *     reach, declared per patch; K: cycles merged into one step);
 *   - a step takes, for each patch with pending cycles t_a..t_b (at most K),
 *     one window circuit of cycles c0..t_b, c0 = max(0, t_a - 3H), assembled
 *     on the device from the resident cycles: the first H cycles of the
 *     window (when c0 > 0) only supply measurement records (their detectors
 *     are emptied), and, unless t_b is the patch's final cycle, the window
 *     is closed by a Z measurement of every qubit of the declared logicals
 *     and one observable per logical, so observable bits are those of the
 *     logical frame at the cycle boundary; the noise of its last H cycles
 *     is then left out (their mechanisms only flip detectors after every
 *     cycle the window seals, so no delivered hyperedge holds one), and so
 *     is the noise of its records-only cycles once a window of the same
 *     registered cycles has passed the horizon test below;
 *   - all windows of a step are compiled in one batched launch
 *     (gp_compile_batch), and a hyperedge is delivered with request t when
 *     its smallest detector lies in cycle t - H (the final request of a
 *     patch also takes every later hyperedge and those without detectors).
 * Over a whole stream the delivered hyperedges are exactly those of the
 * full-circuit compile.  A mechanism of a records-only cycle inside a
 * delivered hyperedge, or a record lookback past H cycles, means H is too
 * small: the affected requests fail with GP_ERR_HORIZON.
 *
 * Conventions are those of gpdem.h.  A server is not thread-safe.  Request
 * results are host memory owned by the server, valid until
 * gp_server_release() or gp_server_destroy().
 */
#ifndef GPSERVE_H
#define GPSERVE_H

#include "gpdem.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Capacity of a server (fixed at creation; device memory for all of it is
 * taken at once, and creation fails with GP_ERR_CAPACITY when the device's
 * free memory cannot hold it). */
typedef struct {
    uint32_t max_patches;            /* patches open at once                        */
    uint32_t max_batch;              /* windows (patches) compiled in one step      */
    uint32_t max_cycles_per_step;    /* K: pending cycles merged into one window    */
    uint32_t max_horizon;            /* largest H a patch may declare (>= 1)        */
    uint32_t max_pending;            /* submitted, not yet stepped cycles (all)     */
    uint32_t max_qubits;             /* per patch, <= 8192                          */
    uint32_t max_cycle_ops;          /* rows of one cycle                           */
    uint32_t max_cycle_recs;         /* record lookbacks of one cycle               */
    uint32_t max_cycle_locations;    /* noise locations of one cycle                */
    uint32_t max_cycle_measurements;
    uint32_t max_cycle_detectors;
    uint32_t max_cycle_mechanisms;   /* Pauli components of one cycle at L2         */
    uint32_t max_cycle_layers;       /* TICK rows of one cycle + 1                  */
    uint32_t max_logical_qubits;     /* per patch: sum over logicals of their sizes */
} gp_server_config;

/* A patch.  Logical k is measured as the parity of Z measurements of its
 * qubits (host arrays, copied). */
typedef struct {
    uint32_t n_qubits;
    uint32_t horizon;                 /* H >= 1                                   */
    uint32_t n_observables;           /* declared logicals, <= 64                 */
    const uint32_t *logical_qubits;   /* host: concatenated supports              */
    const uint32_t *logical_offsets;  /* host: n_observables + 1 offsets          */
} gp_patch_spec;

/* What one request delivered.  det_idx holds patch-global detector ids
 * (declaration order over the whole stream). */
typedef struct {
    uint64_t request;
    uint32_t patch;
    uint32_t cycle;                   /* the cycle this request appended          */
    gp_status status;                 /* GP_OK, or why the request failed         */
    uint32_t n_edges;
    uint64_t n_det_entries;
    const uint32_t *det_offsets;      /* host, n_edges + 1                        */
    const uint32_t *det_idx;          /* host                                     */
    const uint64_t *obs_mask;         /* host                                     */
    const float *prob;                /* host                                     */
    const float *logodds;             /* host                                     */
    uint64_t t_arrival_ns;            /* steady clock (CLOCK_MONOTONIC)           */
    uint64_t t_done_ns;
} gp_sealed_view;

typedef struct gp_server gp_server;

/* Create a server on the current CUDA device.  Errors: GP_ERR_INVALID
 * (zero or out-of-range fields), GP_ERR_CAPACITY (not enough free device
 * memory), GP_ERR_CUDA. */
gp_status gp_server_create(const gp_server_config *config, gp_server **out);
void gp_server_destroy(gp_server *srv);

/* Open a patch; *patch receives its id.  GP_ERR_CAPACITY when max_patches
 * are open, GP_ERR_INVALID for a spec outside the configuration. */
gp_status gp_server_open_patch(gp_server *srv, const gp_patch_spec *spec, uint32_t *patch);
/* Close a patch with no pending cycles (GP_ERR_INVALID otherwise). */
gp_status gp_server_close_patch(gp_server *srv, uint32_t patch);

/* Queue the next cycle of a patch (host arrays, copied before return).
 * The cycle's rows follow gp_circuit: detector and observable rows index
 * the cycle's own record array, noise rows its own locations; record
 * lookbacks are relative and may reach into the patch's earlier cycles, at
 * most H cycles back (else GP_ERR_HORIZON).  noise: host, n_locations.
 * final != 0 ends the patch: its observables must be defined by the cycle's
 * own OBSERVABLE_INCLUDE rows (non-final cycles may not have any).
 * t_arrival_ns: the request's arrival time on the steady clock, 0 = now.
 * *request receives the request id. */
gp_status gp_server_submit(gp_server *srv, uint32_t patch, const gp_circuit *cycle, const float *noise,
                           int final, uint64_t t_arrival_ns, uint64_t *request);

/* Register a cycle a patch repeats (a steady-state syndrome round): it is
 * copied once into device memory and submitted by id.  Its rows are checked
 * here (the errors gp_server_submit reports for a cycle's own rows and
 * sizes); each submission checks only what depends on the patch's history
 * (record lookback and horizon, observables only in a final cycle, no cycle
 * after the final one).  *cycle_id receives its id.  The registered cycles
 * of a patch are freed when it closes. */
gp_status gp_server_register_cycle(gp_server *srv, uint32_t patch, const gp_circuit *cycle, const float *noise,
                                   uint32_t *cycle_id);
gp_status gp_server_submit_registered(gp_server *srv, uint32_t patch, uint32_t cycle_id, int final,
                                      uint64_t t_arrival_ns, uint64_t *request);

/* Submit n registered cycles at once (patches[i], cycle_ids[i], finals[i],
 * t_arrival_ns[i]; host arrays).  Stops at the first failure: *n_done
 * receives how many were queued, requests[0 .. *n_done) their ids, and the
 * failure is returned. */
gp_status gp_server_submit_registered_many(gp_server *srv, uint32_t n, const uint32_t *patches,
                                           const uint32_t *cycle_ids, const uint8_t *finals,
                                           const uint64_t *t_arrival_ns, uint64_t *requests, uint32_t *n_done);

/* One scheduling step: up to max_batch patches with pending cycles (oldest
 * first), up to K cycles each, compiled in one batched launch on the
 * caller's stream; returns when their results are on the host.
 * *n_completed receives the number of requests finished (successfully or
 * not).  A failure confined to some patches (GP_ERR_HORIZON) fails only
 * their requests; a failure of the batch itself fails all of them and is
 * returned. */
gp_status gp_server_step(gp_server *srv, gp_level level, void *stream, uint32_t *n_completed);

/* Microseconds of the last step: host wall clock of building the windows
 * and uploading cycles and descriptors, of the batched compile, of selecting
 * and copying back the sealed hyperedges and of handing them to the
 * requests; then the compile's device stages (lowering, stage 1, grouping,
 * compaction) as gp_last_timing reports them. */
gp_status gp_server_last_timing(const gp_server *srv, float times_us[8]);

/* Launch and work-split parameters of the server's compiles (gp_tuning,
 * gp_set_tuning's checks); none changes a result.  A server starts with the
 * driver's defaults and stage1_wide_emit = 1 (its windows are short, so
 * detector columns set the walk's time).  Not in the paper. */
gp_status gp_server_set_tuning(gp_server *srv, const gp_tuning *t);

/* Ids of requests finished since the last call (at most cap; *n receives
 * the count). */
gp_status gp_server_completed(gp_server *srv, uint64_t *ids, uint32_t cap, uint32_t *n);

/* Finished requests, oldest first, at most cap: id, arrival and completion
 * times, hyperedges delivered and status (host arrays of cap entries); their
 * results are released.  *n receives the count. */
gp_status gp_server_drain(gp_server *srv, uint32_t cap, uint64_t *ids, uint64_t *t_arrival_ns, uint64_t *t_done_ns,
                          uint32_t *n_edges, int32_t *status, uint32_t *n);

/* Result of a finished request (GP_ERR_INVALID for an unknown or pending
 * one). */
gp_status gp_server_result(const gp_server *srv, uint64_t request, gp_sealed_view *out);
/* Forget a finished request's result. */
gp_status gp_server_release(gp_server *srv, uint64_t request);

#ifdef __cplusplus
}
#endif

#endif /* GPSERVE_H */
