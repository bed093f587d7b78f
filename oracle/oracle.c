/*
 * oracle.c -- plain, serial FP64 reference for the detector error model.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Nothing here is tuned: sets are
 * sorted uint32 arrays, the backward walk visits one circuit row at a time,
 * grouping sorts whole flip sets, and every probability is FP64.
 */
#include "oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* circuit row kinds (flat format) */
enum {
    K_TICK = 0, K_R = 1, K_M = 2, K_MR = 3, K_RX = 4, K_MX = 5, K_MRX = 6,
    K_H = 8, K_S = 9, K_CX = 10, K_CZ = 11,
    K_DETECTOR = 16, K_OBS = 17,
    K_XERR = 32, K_ZERR = 33, K_DEP1 = 34, K_DEP2 = 35
};

/* ---- sorted id sets ---------------------------------------------------- */
typedef struct { uint32_t *v; uint32_t n, cap; } idset;

static int set_reserve(idset *s, uint32_t cap) {
    if (cap <= s->cap) return 0;
    uint32_t nc = s->cap ? s->cap : 4;
    while (nc < cap) nc *= 2;
    uint32_t *nv = (uint32_t *)realloc(s->v, (size_t)nc * sizeof(uint32_t));
    if (!nv) return -1;
    s->v = nv;
    s->cap = nc;
    return 0;
}

/* out = a XOR b (symmetric difference); out must differ from a and b */
static int set_xor(idset *out, const idset *a, const idset *b) {
    if (set_reserve(out, a->n + b->n)) return -1;
    uint32_t i = 0, j = 0, k = 0;
    while (i < a->n && j < b->n) {
        if (a->v[i] < b->v[j]) out->v[k++] = a->v[i++];
        else if (a->v[i] > b->v[j]) out->v[k++] = b->v[j++];
        else { i++; j++; }
    }
    while (i < a->n) out->v[k++] = a->v[i++];
    while (j < b->n) out->v[k++] = b->v[j++];
    out->n = k;
    return 0;
}

/* a ^= b using tmp as scratch */
static int set_xor_inplace(idset *a, const idset *b, idset *tmp) {
    if (b->n == 0) return 0;
    if (set_xor(tmp, a, b)) return -1;
    idset t = *a; *a = *tmp; *tmp = t;
    return 0;
}

/* toggle one id (used while building measurement -> id lists) */
static int set_toggle(idset *s, uint32_t id) {
    uint32_t i = 0;
    while (i < s->n && s->v[i] < id) i++;
    if (i < s->n && s->v[i] == id) {
        memmove(s->v + i, s->v + i + 1, (size_t)(s->n - i - 1) * sizeof(uint32_t));
        s->n--;
        return 0;
    }
    if (set_reserve(s, s->n + 1)) return -1;
    memmove(s->v + i + 1, s->v + i, (size_t)(s->n - i) * sizeof(uint32_t));
    s->v[i] = id;
    s->n++;
    return 0;
}

/* ---- result ------------------------------------------------------------ */
struct orc_dem {
    uint32_t n_det, n_obs, n_loc;
    uint64_t n_mech;
    uint64_t *mech_op;
    uint32_t *mech_comp, *mech_loc, *mech_kind;
    double *mech_q;
    uint64_t *mech_mask_off;
    uint32_t *mech_mask;
    uint64_t *mech_class;
    uint64_t n_class;
    uint64_t *class_mask_off;
    uint32_t *class_mask;
    double *class_p, *class_p_iter, *class_w;
    uint64_t *class_size;
    uint64_t *class_members;      /* mechanisms grouped by class */
    uint64_t *class_member_off;
    double *noise;                /* copy of the noise vector (for gradients) */
};

/* ---- Pauli components per channel and level ----------------------------
 * A Pauli on one qubit is (x, z) with X = (1,0), Z = (0,1), Y = (1,1).
 * DEPOLARIZE1 components in order X, Z, Y: level 0 keeps X and Z, levels 1
 * and 2 keep all three.  DEPOLARIZE2 components follow Table
 * tab:correlation-level: the six level-0 terms, then the four level-1
 * terms, then the five level-2 terms; each is (first qubit, second qubit).
 */
/* pauli codes: 0 = I, 1 = X, 2 = Z, 3 = Y */
static const int DEP1_COMP[3] = {1, 2, 3};                /* X Z Y */
static const int DEP2_COMP[15][2] = {
    {0, 1}, {0, 2}, {1, 0}, {1, 1}, {2, 0}, {2, 2},   /* IX IZ XI XX ZI ZZ */
    {0, 3}, {1, 2}, {3, 0}, {2, 1},                   /* IY XZ YI ZX       */
    {1, 3}, {3, 1}, {3, 3}, {3, 2}, {2, 3}            /* XY YX YY YZ ZY    */
};
static int pauli_x(int p) { return p == 1 || p == 3; }
static int pauli_z(int p) { return p == 2 || p == 3; }

static int n_components(uint32_t kind, int level) {
    switch (kind) {
    case K_XERR: case K_ZERR: return 1;
    case K_DEP1: return level == 0 ? 2 : 3;
    case K_DEP2: return level == 0 ? 6 : (level == 1 ? 10 : 15);
    default: return 0;
    }
}

/* Independent-component probability of one Pauli term of a channel with
 * parameter p.  X_ERROR / Z_ERROR: q = p.  DEPOLARIZE1 (each of the three
 * non-identity Paulis with probability p/3) is reproduced exactly by three
 * independent components with q = (1 - sqrt(1 - 4p/3)) / 2; DEPOLARIZE2
 * (each of fifteen with p/15) by fifteen independent components with
 * q = (1 - (1 - 16p/15)^(1/8)) / 2. */
static double component_q(uint32_t kind, double p) {
    switch (kind) {
    case K_XERR: case K_ZERR: return p;
    case K_DEP1: return 0.5 * (1.0 - sqrt(1.0 - 4.0 * p / 3.0));
    case K_DEP2: return 0.5 * (1.0 - pow(1.0 - 16.0 * p / 15.0, 0.125));
    default: return 0.0;
    }
}

static double component_dq_dp(uint32_t kind, double p) {
    switch (kind) {
    case K_XERR: case K_ZERR: return 1.0;
    case K_DEP1: return (1.0 / 3.0) / sqrt(1.0 - 4.0 * p / 3.0);
    case K_DEP2: return (1.0 / 15.0) * pow(1.0 - 16.0 * p / 15.0, -0.875);
    default: return 0.0;
    }
}

static double channel_p_max(uint32_t kind) {
    switch (kind) {
    case K_XERR: case K_ZERR: return 0.5;
    case K_DEP1: return 0.75;
    case K_DEP2: return 15.0 / 16.0;
    default: return 0.0;
    }
}

/* ---- growable arrays --------------------------------------------------- */
#define GROW(ptr, cap, need, type)                                               \
    do {                                                                         \
        if ((need) > (cap)) {                                                    \
            uint64_t nc_ = (cap) ? (cap) : 64;                                   \
            while (nc_ < (need)) nc_ *= 2;                                       \
            type *np_ = (type *)realloc((ptr), nc_ * sizeof(type));              \
            if (!np_) goto nomem;                                                \
            (ptr) = np_;                                                         \
            (cap) = nc_;                                                         \
        }                                                                        \
    } while (0)

static void seterr(char *err, int len, const char *fmt, ...) {
    if (!err || len <= 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, (size_t)len, fmt, ap);
    va_end(ap);
}

/* ---- merge sort of indices with a context comparator ------------------- */
typedef int (*cmp_fn)(uint64_t, uint64_t, const void *);

static int merge_sort(uint64_t *a, uint64_t n, cmp_fn cmp, const void *ctx) {
    uint64_t *b = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!b) return -1;
    for (uint64_t w = 1; w < n; w *= 2) {
        for (uint64_t lo = 0; lo < n; lo += 2 * w) {
            uint64_t mid = lo + w < n ? lo + w : n;
            uint64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            uint64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) b[k++] = cmp(a[j], a[i], ctx) < 0 ? a[j++] : a[i++];
            while (i < mid) b[k++] = a[i++];
            while (j < hi) b[k++] = a[j++];
        }
        memcpy(a, b, n * sizeof(uint64_t));
    }
    free(b);
    return 0;
}

typedef struct { const uint64_t *off; const uint32_t *ids; } mask_ctx;

static int cmp_mask(uint64_t x, uint64_t y, const void *vctx) {
    const mask_ctx *c = (const mask_ctx *)vctx;
    uint64_t xa = c->off[x], xb = c->off[x + 1], ya = c->off[y], yb = c->off[y + 1];
    while (xa < xb && ya < yb) {
        if (c->ids[xa] != c->ids[ya]) return c->ids[xa] < c->ids[ya] ? -1 : 1;
        xa++; ya++;
    }
    if (xa < xb) return 1;
    if (ya < yb) return -1;
    return 0;
}

/* ---- main analysis ----------------------------------------------------- */
int orc_analyze(const uint32_t *ops, uint64_t n_ops, const uint32_t *recs,
                uint64_t n_recs, uint32_t n_qubits, const double *noise,
                uint32_t n_locations, int level, orc_dem **out,
                char *err, int err_len) {
    int status = ORC_OK;
    orc_dem *d = NULL;
    idset *xs = NULL, *zs = NULL, *meas_ids = NULL;
    idset t1 = {0}, t2 = {0}, t3 = {0};
    uint64_t n_meas = 0, n_det = 0;
    uint32_t n_obs = 0;
    uint64_t *meas_before = NULL;   /* per row: measurements strictly before it */
    uint64_t mech_cap = 0, mask_cap = 0;
    uint64_t *order = NULL;

    *out = NULL;
    if (level < 0 || level > 2) { seterr(err, err_len, "level must be 0, 1 or 2"); return ORC_INVALID; }

    /* pass 1: validate rows, count measurements / detectors / observables */
    meas_before = (uint64_t *)malloc((n_ops + 1) * sizeof(uint64_t));
    if (!meas_before) goto nomem;
    for (uint64_t i = 0; i < n_ops; i++) {
        const uint32_t *o = ops + 4 * i;
        uint32_t k = o[0];
        meas_before[i] = n_meas;
        switch (k) {
        case K_TICK: break;
        case K_R: case K_RX: case K_H: case K_S:
        case K_M: case K_MR: case K_MX: case K_MRX:
            if (o[1] >= n_qubits) { seterr(err, err_len, "row %llu: qubit %u out of range", (unsigned long long)i, o[1]); status = ORC_INVALID; goto fail; }
            if (k == K_M || k == K_MR || k == K_MX || k == K_MRX) n_meas++;
            break;
        case K_CX: case K_CZ:
            if (o[1] >= n_qubits || o[2] >= n_qubits || o[1] == o[2]) { seterr(err, err_len, "row %llu: bad two-qubit targets", (unsigned long long)i); status = ORC_INVALID; goto fail; }
            break;
        case K_DETECTOR: case K_OBS:
            if ((uint64_t)o[1] + o[2] > n_recs) { seterr(err, err_len, "row %llu: record list out of range", (unsigned long long)i); status = ORC_INVALID; goto fail; }
            for (uint32_t r = 0; r < o[2]; r++) {
                uint32_t lb = recs[o[1] + r];
                if (lb == 0 || lb > n_meas) { seterr(err, err_len, "row %llu: record lookback %u refers to no earlier measurement", (unsigned long long)i, lb); status = ORC_INVALID; goto fail; }
            }
            if (k == K_DETECTOR) n_det++;
            else if (o[3] + 1 > n_obs) n_obs = o[3] + 1;
            break;
        case K_XERR: case K_ZERR: case K_DEP1: case K_DEP2: {
            if (o[1] >= n_qubits || (k == K_DEP2 && (o[2] >= n_qubits || o[1] == o[2]))) { seterr(err, err_len, "row %llu: bad noise targets", (unsigned long long)i); status = ORC_INVALID; goto fail; }
            if (o[3] >= n_locations) { seterr(err, err_len, "row %llu: location %u out of range", (unsigned long long)i, o[3]); status = ORC_INVALID; goto fail; }
            double p = noise[o[3]];
            if (!(p >= 0.0 && p <= channel_p_max(k))) { seterr(err, err_len, "location %u: probability %g outside the channel's range", o[3], p); status = ORC_INVALID; goto fail; }
            break;
        }
        default:
            seterr(err, err_len, "row %llu: unknown kind %u", (unsigned long long)i, k);
            status = ORC_INVALID;
            goto fail;
        }
    }
    meas_before[n_ops] = n_meas;
    if (n_det + n_obs > 0xFFFFFFFFull || n_obs > 0xFFFFFFu) { seterr(err, err_len, "too many detectors"); status = ORC_INVALID; goto fail; }

    /* pass 2: measurement -> ids it belongs to (Eq. init-slp: each
     * measurement of a detector toggles that detector's bit) */
    meas_ids = (idset *)calloc(n_meas ? n_meas : 1, sizeof(idset));
    if (!meas_ids) goto nomem;
    {
        uint64_t det = 0;
        for (uint64_t i = 0; i < n_ops; i++) {
            const uint32_t *o = ops + 4 * i;
            if (o[0] != K_DETECTOR && o[0] != K_OBS) continue;
            uint32_t id = o[0] == K_DETECTOR ? (uint32_t)det++ : (uint32_t)(n_det + o[3]);
            for (uint32_t r = 0; r < o[2]; r++) {
                uint64_t m = meas_before[i] - recs[o[1] + r];
                if (set_toggle(&meas_ids[m], id)) goto nomem;
            }
        }
    }

    d = (orc_dem *)calloc(1, sizeof(orc_dem));
    if (!d) goto nomem;
    d->n_det = (uint32_t)n_det;
    d->n_obs = n_obs;
    d->n_loc = n_locations;
    d->noise = (double *)malloc((n_locations ? n_locations : 1) * sizeof(double));
    if (!d->noise) goto nomem;
    if (n_locations) memcpy(d->noise, noise, n_locations * sizeof(double));

    xs = (idset *)calloc(n_qubits ? n_qubits : 1, sizeof(idset));
    zs = (idset *)calloc(n_qubits ? n_qubits : 1, sizeof(idset));
    if (!xs || !zs) goto nomem;

    /* pass 3: backward walk (Sec. 2.1.5 backtracking; Eq. slp).
     * xs[q] = ids flipped by an X error on q at the current time point,
     * zs[q] = ids flipped by a Z error. */
    {
        uint64_t n_mask = 0;
        uint64_t m = n_meas;
        for (uint64_t ii = n_ops; ii-- > 0;) {
            const uint32_t *o = ops + 4 * ii;
            uint32_t k = o[0], a = o[1], b = o[2];
            switch (k) {
            case K_TICK: case K_DETECTOR: case K_OBS: break;
            case K_H: { idset t = xs[a]; xs[a] = zs[a]; zs[a] = t; break; }
            case K_S:  /* X before S is Y after */
                if (set_xor_inplace(&xs[a], &zs[a], &t1)) goto nomem;
                break;
            case K_CX: /* X_c -> X_c X_t ; Z_t -> Z_c Z_t */
                if (set_xor_inplace(&xs[a], &xs[b], &t1)) goto nomem;
                if (set_xor_inplace(&zs[b], &zs[a], &t1)) goto nomem;
                break;
            case K_CZ: /* X_a -> X_a Z_b ; X_b -> Z_a X_b */
                if (set_xor_inplace(&xs[a], &zs[b], &t1)) goto nomem;
                if (set_xor_inplace(&xs[b], &zs[a], &t1)) goto nomem;
                break;
            case K_R: case K_MR: case K_RX: case K_MRX: case K_M: case K_MX: {
                int xbasis = (k == K_RX || k == K_MX || k == K_MRX);
                int resets = (k == K_R || k == K_MR || k == K_RX || k == K_MRX);
                int measures = (k == K_M || k == K_MR || k == K_MX || k == K_MRX);
                if (resets) {
                    /* the state right after a reset is an eigenstate of the
                     * basis operator; a detecting region that anticommutes
                     * with it makes the detector random */
                    if ((xbasis ? xs[a].n : zs[a].n) != 0) {
                        seterr(err, err_len, "row %llu: detector/observable %u anticommutes with a reset", (unsigned long long)ii, xbasis ? xs[a].v[0] : zs[a].v[0]);
                        status = ORC_NONDETERMINISTIC;
                        goto fail;
                    }
                    xs[a].n = 0;
                    zs[a].n = 0;
                }
                if (measures) {
                    m--;
                    if ((xbasis ? xs[a].n : zs[a].n) != 0) {
                        seterr(err, err_len, "row %llu: detector/observable %u anticommutes with a measurement", (unsigned long long)ii, xbasis ? xs[a].v[0] : zs[a].v[0]);
                        status = ORC_NONDETERMINISTIC;
                        goto fail;
                    }
                    /* an error that anticommutes with the measured operator
                     * flips the outcome */
                    if (set_xor_inplace(xbasis ? &zs[a] : &xs[a], &meas_ids[m], &t1)) goto nomem;
                }
                break;
            }
            case K_XERR: case K_ZERR: case K_DEP1: case K_DEP2: {
                double p = noise[o[3]];
                int nc = n_components(k, level);
                double q = component_q(k, p);
                if (!(q > 0.0)) break;
                for (int c = 0; c < nc; c++) {
                    int pa, pb = 0;
                    if (k == K_XERR) pa = 1;
                    else if (k == K_ZERR) pa = 2;
                    else if (k == K_DEP1) pa = DEP1_COMP[c];
                    else { pa = DEP2_COMP[c][0]; pb = DEP2_COMP[c][1]; }
                    /* mask = XOR of the sensitivity sets of the component's
                     * X and Z parts (Sec. 2.3.4) */
                    t2.n = 0;
                    if (pauli_x(pa)) { if (set_xor(&t3, &t2, &xs[a])) goto nomem; idset t = t2; t2 = t3; t3 = t; }
                    if (pauli_z(pa)) { if (set_xor(&t3, &t2, &zs[a])) goto nomem; idset t = t2; t2 = t3; t3 = t; }
                    if (pauli_x(pb)) { if (set_xor(&t3, &t2, &xs[b])) goto nomem; idset t = t2; t2 = t3; t3 = t; }
                    if (pauli_z(pb)) { if (set_xor(&t3, &t2, &zs[b])) goto nomem; idset t = t2; t2 = t3; t3 = t; }
                    if (t2.n == 0) continue;   /* flips nothing: not a mechanism */
                    uint64_t i = d->n_mech++;
                    if (d->n_mech > mech_cap) {
                        uint64_t cap2 = mech_cap ? 2 * mech_cap : 1024;
                        uint64_t *a1 = (uint64_t *)realloc(d->mech_op, cap2 * sizeof(uint64_t));
                        if (a1) d->mech_op = a1;
                        uint32_t *a2 = (uint32_t *)realloc(d->mech_comp, cap2 * sizeof(uint32_t));
                        if (a2) d->mech_comp = a2;
                        uint32_t *a3 = (uint32_t *)realloc(d->mech_loc, cap2 * sizeof(uint32_t));
                        if (a3) d->mech_loc = a3;
                        uint32_t *a4 = (uint32_t *)realloc(d->mech_kind, cap2 * sizeof(uint32_t));
                        if (a4) d->mech_kind = a4;
                        double *a5 = (double *)realloc(d->mech_q, cap2 * sizeof(double));
                        if (a5) d->mech_q = a5;
                        uint64_t *a6 = (uint64_t *)realloc(d->mech_mask_off, (cap2 + 1) * sizeof(uint64_t));
                        if (a6) d->mech_mask_off = a6;
                        if (!a1 || !a2 || !a3 || !a4 || !a5 || !a6) goto nomem;
                        mech_cap = cap2;
                    }
                    d->mech_op[i] = ii;
                    d->mech_comp[i] = (uint32_t)c;
                    d->mech_loc[i] = o[3];
                    d->mech_kind[i] = k;
                    d->mech_q[i] = q;
                    d->mech_mask_off[i] = n_mask;
                    GROW(d->mech_mask, mask_cap, n_mask + t2.n, uint32_t);
                    memcpy(d->mech_mask + n_mask, t2.v, t2.n * sizeof(uint32_t));
                    n_mask += t2.n;
                    d->mech_mask_off[i + 1] = n_mask;
                }
                break;
            }
            default: break;
            }
        }
        if (d->n_mech == 0) {
            d->mech_mask_off = (uint64_t *)calloc(1, sizeof(uint64_t));
            if (!d->mech_mask_off) goto nomem;
        }
    }
    /* the circuit starts in |0...0>: every region must commute with Z_q */
    for (uint32_t q = 0; q < n_qubits; q++) {
        if (zs[q].n != 0) {
            seterr(err, err_len, "detector/observable %u anticommutes with the initial |0> state of qubit %u", zs[q].v[0], q);
            status = ORC_NONDETERMINISTIC;
            goto fail;
        }
    }

    /* group mechanisms with equal flip sets (Sec. 2.1.4) */
    {
        uint64_t n = d->n_mech;
        order = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
        d->mech_class = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
        if (!order || !d->mech_class) goto nomem;
        for (uint64_t i = 0; i < n; i++) order[i] = i;
        mask_ctx ctx = {d->mech_mask_off, d->mech_mask};
        if (merge_sort(order, n, cmp_mask, &ctx)) goto nomem;
        uint64_t nc = 0;
        for (uint64_t i = 0; i < n; i++)
            if (i == 0 || cmp_mask(order[i - 1], order[i], &ctx) != 0) nc++;
        d->n_class = nc;
        d->class_mask_off = (uint64_t *)malloc((nc + 1) * sizeof(uint64_t));
        d->class_p = (double *)malloc((nc ? nc : 1) * sizeof(double));
        d->class_p_iter = (double *)malloc((nc ? nc : 1) * sizeof(double));
        d->class_w = (double *)malloc((nc ? nc : 1) * sizeof(double));
        d->class_size = (uint64_t *)calloc(nc ? nc : 1, sizeof(uint64_t));
        d->class_member_off = (uint64_t *)malloc((nc + 1) * sizeof(uint64_t));
        d->class_members = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
        if (!d->class_mask_off || !d->class_p || !d->class_p_iter || !d->class_w ||
            !d->class_size || !d->class_member_off || !d->class_members) goto nomem;
        uint64_t total_ids = 0, c = (uint64_t)-1;
        for (uint64_t i = 0; i < n; i++) {
            uint64_t mi = order[i];
            if (i == 0 || cmp_mask(order[i - 1], mi, &ctx) != 0) {
                c++;
                d->class_member_off[c] = i;
                total_ids += d->mech_mask_off[mi + 1] - d->mech_mask_off[mi];
            }
            d->mech_class[mi] = c;
            d->class_members[i] = mi;
            d->class_size[c]++;
        }
        d->class_member_off[nc] = n;
        d->class_mask = (uint32_t *)malloc((total_ids ? total_ids : 1) * sizeof(uint32_t));
        if (!d->class_mask) goto nomem;
        uint64_t pos = 0;
        for (uint64_t cc = 0; cc < nc; cc++) {
            uint64_t rep = d->class_members[d->class_member_off[cc]];
            uint64_t len = d->mech_mask_off[rep + 1] - d->mech_mask_off[rep];
            d->class_mask_off[cc] = pos;
            memcpy(d->class_mask + pos, d->mech_mask + d->mech_mask_off[rep], len * sizeof(uint32_t));
            pos += len;
            /* Eq. pmerge: P = q_1 [+] q_2 [+] ...; closed form
             * 1 - 2P = prod (1 - 2 q_i), evaluated with log1p / expm1 */
            double s = 0.0, pit = 0.0;
            for (uint64_t j = d->class_member_off[cc]; j < d->class_member_off[cc + 1]; j++) {
                double q = d->mech_q[d->class_members[j]];
                s += log1p(-2.0 * q);
                pit = pit * (1.0 - q) + q * (1.0 - pit);
            }
            double P = -0.5 * expm1(s);
            d->class_p[cc] = P;
            d->class_p_iter[cc] = pit;
            d->class_w[cc] = log1p(-P) - log(P);
        }
        d->class_mask_off[nc] = pos;
    }

    free(order);
    free(meas_before);
    for (uint64_t i = 0; i < n_meas; i++) free(meas_ids[i].v);
    free(meas_ids);
    for (uint32_t q = 0; q < n_qubits; q++) { free(xs[q].v); free(zs[q].v); }
    free(xs); free(zs);
    free(t1.v); free(t2.v); free(t3.v);
    *out = d;
    return ORC_OK;

nomem:
    seterr(err, err_len, "out of memory");
    status = ORC_NOMEM;
fail:
    free(order);
    free(meas_before);
    if (meas_ids) { for (uint64_t i = 0; i < n_meas; i++) free(meas_ids[i].v); free(meas_ids); }
    if (xs) { for (uint32_t q = 0; q < n_qubits; q++) free(xs[q].v); free(xs); }
    if (zs) { for (uint32_t q = 0; q < n_qubits; q++) free(zs[q].v); free(zs); }
    free(t1.v); free(t2.v); free(t3.v);
    orc_free(d);
    return status;
}

void orc_free(orc_dem *d) {
    if (!d) return;
    free(d->mech_op); free(d->mech_comp); free(d->mech_loc); free(d->mech_kind);
    free(d->mech_q); free(d->mech_mask_off); free(d->mech_mask); free(d->mech_class);
    free(d->class_mask_off); free(d->class_mask); free(d->class_p); free(d->class_p_iter);
    free(d->class_w); free(d->class_size); free(d->class_members); free(d->class_member_off);
    free(d->noise);
    free(d);
}

uint32_t orc_n_detectors(const orc_dem *d) { return d->n_det; }
uint32_t orc_n_observables(const orc_dem *d) { return d->n_obs; }
uint64_t orc_n_mechanisms(const orc_dem *d) { return d->n_mech; }
const uint64_t *orc_mech_op(const orc_dem *d) { return d->mech_op; }
const uint32_t *orc_mech_comp(const orc_dem *d) { return d->mech_comp; }
const uint32_t *orc_mech_loc(const orc_dem *d) { return d->mech_loc; }
const double *orc_mech_q(const orc_dem *d) { return d->mech_q; }
const uint64_t *orc_mech_mask_off(const orc_dem *d) { return d->mech_mask_off; }
const uint32_t *orc_mech_mask(const orc_dem *d) { return d->mech_mask; }
const uint64_t *orc_mech_class(const orc_dem *d) { return d->mech_class; }
uint64_t orc_n_classes(const orc_dem *d) { return d->n_class; }
const uint64_t *orc_class_mask_off(const orc_dem *d) { return d->class_mask_off; }
const uint32_t *orc_class_mask(const orc_dem *d) { return d->class_mask; }
const double *orc_class_p(const orc_dem *d) { return d->class_p; }
const double *orc_class_p_iter(const orc_dem *d) { return d->class_p_iter; }
const double *orc_class_w(const orc_dem *d) { return d->class_w; }
const uint64_t *orc_class_size(const orc_dem *d) { return d->class_size; }

/* Gradient of L = sum_c gP_c P_c + gW_c w_c with respect to each location's
 * channel parameter.  For a member i of class c,
 *   dP_c/dq_i = prod_{j != i} (1 - 2 q_j)        (derivative of Eq. pmerge)
 *   dw_c/dP_c = -1 / (P_c (1 - P_c))
 * and dq_i/dp follows the component decomposition of the channel. */
void orc_gradient(const orc_dem *d, const double *gP, const double *gW, double *g_noise) {
    for (uint32_t l = 0; l < d->n_loc; l++) g_noise[l] = 0.0;
    for (uint64_t c = 0; c < d->n_class; c++) {
        double P = d->class_p[c];
        double gbar = gP[c] - gW[c] / (P * (1.0 - P));
        uint64_t lo = d->class_member_off[c], hi = d->class_member_off[c + 1];
        for (uint64_t j = lo; j < hi; j++) {
            uint64_t i = d->class_members[j];
            double prod = 1.0;
            for (uint64_t k = lo; k < hi; k++)
                if (k != j) prod *= 1.0 - 2.0 * d->mech_q[d->class_members[k]];
            uint32_t loc = d->mech_loc[i];
            g_noise[loc] += gbar * prod * component_dq_dp(d->mech_kind[i], d->noise[loc]);
        }
    }
}
