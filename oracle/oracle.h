/*
 * oracle.h -- plain, serial FP64 reference for the detector error model.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the GPU library; it is
 * called by the test-suite, by the package smoke check and by the benchmark's
 * CPU-baseline leg, never by the product path.  It shares no code, header or
 * table with the CUDA library.
 *
 * What it computes (Sec. 2.1.4-2.3.4 of the GreenPeas paper):
 *   - every error mechanism E_i (one Pauli component of one noise site with
 *     probability q_i > 0) and the exact set of detectors and observables it
 *     flips, by backtracking detector sensitivities (Sec. 2.1.5, Eqs. slp and
 *     init-slp) with sparse sorted sets;
 *   - the partition of mechanisms by equal flip set (error equivalence
 *     classes, Sec. 2.1.4);
 *   - per class P = q_1 [+] q_2 [+] ... with a [+] b = a(1-b) + b(1-a)
 *     (Eq. pmerge), evaluated as P = -expm1(sum log1p(-2 q_i)) / 2, and the
 *     log-odds weight w = log((1-P)/P);
 *   - the gradient of a linear loss sum_c gP_c P_c + gW_c w_c with respect
 *     to the per-location noise vector.
 *
 * Circuit format: the flat (kind, a, b, c) rows described in
 * paper_2604_16613_gb300/circuits.py, read here with this file's own
 * constants.
 */
#ifndef GREENPEAS_ORACLE_H
#define GREENPEAS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_dem orc_dem;

/* status codes */
#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_NONDETERMINISTIC 2
#define ORC_NOMEM 3

/* Analyse a circuit.  ops: n_ops rows of 4 uint32; recs: lookbacks;
 * noise: n_locations channel parameters; level: 0, 1 or 2 (Table
 * tab:correlation-level).  On success *out owns every array below. */
int orc_analyze(const uint32_t *ops, uint64_t n_ops, const uint32_t *recs,
                uint64_t n_recs, uint32_t n_qubits, const double *noise,
                uint32_t n_locations, int level, orc_dem **out,
                char *err, int err_len);
void orc_free(orc_dem *dem);

uint32_t orc_n_detectors(const orc_dem *d);
uint32_t orc_n_observables(const orc_dem *d);

/* mechanisms (those with q > 0 and a non-empty flip set), in the order the
 * backward walk met them */
uint64_t orc_n_mechanisms(const orc_dem *d);
const uint64_t *orc_mech_op(const orc_dem *d);      /* op row of the noise site */
const uint32_t *orc_mech_comp(const orc_dem *d);    /* component index          */
const uint32_t *orc_mech_loc(const orc_dem *d);     /* noise location           */
const double *orc_mech_q(const orc_dem *d);         /* component probability    */
const uint64_t *orc_mech_mask_off(const orc_dem *d);/* n+1 offsets              */
const uint32_t *orc_mech_mask(const orc_dem *d);    /* sorted ids: detectors
                                                      0..D-1, observables D+k */
const uint64_t *orc_mech_class(const orc_dem *d);   /* class of each mechanism  */

/* classes, sorted by flip set */
uint64_t orc_n_classes(const orc_dem *d);
const uint64_t *orc_class_mask_off(const orc_dem *d);
const uint32_t *orc_class_mask(const orc_dem *d);
const double *orc_class_p(const orc_dem *d);        /* log1p/expm1 form        */
const double *orc_class_p_iter(const orc_dem *d);   /* iterated [+] form       */
const double *orc_class_w(const orc_dem *d);
const uint64_t *orc_class_size(const orc_dem *d);

/* g_noise[loc] = d/dp_loc sum_c (gP[c] P_c + gW[c] w_c); classes indexed as
 * above.  g_noise has n_locations entries and is overwritten. */
void orc_gradient(const orc_dem *d, const double *gP, const double *gW,
                  double *g_noise);

#ifdef __cplusplus
}
#endif
#endif
