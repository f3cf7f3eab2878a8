/*
 * acref.c -- plain FP64 evaluator of compiled arithmetic circuits (oracle; test
 * infrastructure only, and the timed CPU baseline).  It reads the compiled-AC
 * byte format on its own (no code shared with the GPU library) and evaluates
 * one column at a time, node by node, in the order the nodes are stored
 * (children always precede parents), with C99 double complex arithmetic.
 *
 *  upward pass   Sec. 3.3.1 (Table 5): leaves take their values -- indicators
 *                from the evidence (1 if observed true or unobserved, else 0),
 *                parameters from the gate angles -- and every + / x node
 *                combines its children; the root is the network polynomial.
 *  downward pass Sec. 3.3.2 (Darwiche's differential approach): the adjoint of
 *                the root is 1; a child of a + node receives the parent's
 *                adjoint, a child of a x node receives the parent's adjoint
 *                times the product of its siblings; adjoints add over parents.
 *  gradient      chain rule through the parameter leaves: d f / d angle_k =
 *                sum over leaves of angle k of adjoint * d leaf / d angle_k.
 *  sampling      the chain rule P(x) = prod_j P(x_j | x_<j), each factor from
 *                two upward passes (evidence x_<j, and x_<j with X_j = 0).
 * Parity unpinned: none.  The passes and the gradient are pinned against the
 * density-matrix and brute-force oracles and hand-built ACs
 * (tests/test_oracle_pins.py, tests/test_acref_and_compiler.py); the sampler is
 * pinned index for index against the density-matrix chain rule on noisy
 * circuits of up to 10 qubits (tests/test_oracle_sampler_pins.py).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

typedef struct {
    uint32_t kind, n_qubits, n_angles, n_vars, n_nodes, n_edges, n_levels, n_leaves, root, n_ind;
    const uint32_t *var_card;
    const int32_t *var_tag;
    const uint32_t *level_off;
    const uint8_t *op;
    const uint32_t *child_off;
    const uint32_t *child;
    const int32_t *leaf_a, *leaf_b;
    const double *leaf_coef;
    uint8_t *buf; /* private copy of the bytes */
    cplx *val, *adj;
} oac;

static int take(uint64_t *off, uint64_t len, uint64_t bytes, uint64_t *start) {
    *off = (*off + 7) & ~(uint64_t)7;
    if (*off + bytes > len) return -1;
    *start = *off;
    *off += bytes;
    return 0;
}

int oac_open(const uint8_t *bytes, uint64_t len, oac **out) {
    if (!bytes || len < 64 || !out) return -1;
    uint32_t h[16];
    memcpy(h, bytes, 64);
    if (h[0] != 0x43414B51u || h[1] != 1u) return -2;
    oac *a = (oac *)calloc(1, sizeof(oac));
    if (!a) return -3;
    a->buf = (uint8_t *)malloc(len);
    if (!a->buf) { free(a); return -3; }
    memcpy(a->buf, bytes, len);
    a->kind = h[2]; a->n_qubits = h[3]; a->n_angles = h[4]; a->n_vars = h[5];
    a->n_nodes = h[6]; a->n_edges = h[7]; a->n_levels = h[8]; a->n_leaves = h[9];
    a->root = h[10]; a->n_ind = h[11];
    uint64_t off = 64, s;
    int bad = 0;
    bad |= take(&off, len, 4ull * a->n_vars, &s); a->var_card = (const uint32_t *)(a->buf + s);
    bad |= take(&off, len, 4ull * a->n_vars, &s); a->var_tag = (const int32_t *)(a->buf + s);
    bad |= take(&off, len, 4ull * (a->n_levels + 1), &s); a->level_off = (const uint32_t *)(a->buf + s);
    bad |= take(&off, len, 1ull * a->n_nodes, &s); a->op = a->buf + s;
    bad |= take(&off, len, 4ull * (a->n_nodes + 1), &s); a->child_off = (const uint32_t *)(a->buf + s);
    bad |= take(&off, len, 4ull * a->n_edges, &s); a->child = (const uint32_t *)(a->buf + s);
    bad |= take(&off, len, 4ull * a->n_leaves, &s); a->leaf_a = (const int32_t *)(a->buf + s);
    bad |= take(&off, len, 4ull * a->n_leaves, &s); a->leaf_b = (const int32_t *)(a->buf + s);
    bad |= take(&off, len, 16ull * a->n_leaves, &s); a->leaf_coef = (const double *)(a->buf + s);
    if (bad || a->root >= a->n_nodes) { free(a->buf); free(a); return -2; }
    a->val = (cplx *)malloc(sizeof(cplx) * (a->n_nodes ? a->n_nodes : 1));
    a->adj = (cplx *)malloc(sizeof(cplx) * (a->n_nodes ? a->n_nodes : 1));
    if (!a->val || !a->adj) { free(a->val); free(a->adj); free(a->buf); free(a); return -3; }
    *out = a;
    return 0;
}

void oac_close(oac *a) {
    if (!a) return;
    free(a->val); free(a->adj); free(a->buf); free(a);
}

void oac_info(const oac *a, int64_t *o) {
    o[0] = a->kind; o[1] = a->n_qubits; o[2] = a->n_angles; o[3] = a->n_vars; o[4] = a->n_ind;
    o[5] = a->n_nodes; o[6] = a->n_edges; o[7] = a->n_levels; o[8] = a->n_leaves; o[9] = a->root;
}

/* value of g(t) and of g'(t) for the four leaf functions */
static cplx leaf_fn(int fn, double t) {
    switch (fn) {
        case 0: return cos(0.5 * t);
        case 1: return sin(0.5 * t);
        case 2: return cexp(-0.5 * I * t);
        default: return cexp(0.5 * I * t);
    }
}
static cplx leaf_fn_deriv(int fn, double t) {
    switch (fn) {
        case 0: return -0.5 * sin(0.5 * t);
        case 1: return 0.5 * cos(0.5 * t);
        case 2: return -0.5 * I * cexp(-0.5 * I * t);
        default: return 0.5 * I * cexp(0.5 * I * t);
    }
}

static cplx indicator(int8_t e, int32_t value) {
    if (e == -1) return 1.0;
    if (e == -2) return value == 0 ? 1.0 : -1.0;
    return (e == value) ? 1.0 : 0.0;
}

/* upward pass; fills a->val; returns the root value */
static cplx up(oac *a, const double *angles, const int8_t *ev) {
    for (uint32_t i = 0; i < a->n_nodes; ++i) {
        const uint8_t o = a->op[i];
        cplx v;
        if (o == 0) {
            v = indicator(ev[a->leaf_a[i]], a->leaf_b[i]);
        } else if (o == 1) {
            cplx c = a->leaf_coef[2 * i] + I * a->leaf_coef[2 * i + 1];
            v = c * leaf_fn(a->leaf_b[i], angles[a->leaf_a[i]]);
        } else if (o == 2) {
            v = a->leaf_coef[2 * i] + I * a->leaf_coef[2 * i + 1];
        } else if (o == 3) {
            v = 0.0;
            for (uint32_t e = a->child_off[i]; e < a->child_off[i + 1]; ++e) v += a->val[a->child[e]];
        } else {
            v = 1.0;
            for (uint32_t e = a->child_off[i]; e < a->child_off[i + 1]; ++e) v *= a->val[a->child[e]];
        }
        a->val[i] = v;
    }
    return a->val[a->root];
}

/* downward pass after up(); fills a->adj with d root / d node */
static void down(oac *a) {
    for (uint32_t i = 0; i < a->n_nodes; ++i) a->adj[i] = 0.0;
    a->adj[a->root] = 1.0;
    for (uint32_t i = a->n_nodes; i-- > 0;) {
        const cplx d = a->adj[i];
        if (a->op[i] == 3) {
            for (uint32_t e = a->child_off[i]; e < a->child_off[i + 1]; ++e) a->adj[a->child[e]] += d;
        } else if (a->op[i] == 4) {
            for (uint32_t e = a->child_off[i]; e < a->child_off[i + 1]; ++e) {
                cplx others = 1.0;
                for (uint32_t f = a->child_off[i]; f < a->child_off[i + 1]; ++f)
                    if (f != e) others *= a->val[a->child[f]];
                a->adj[a->child[e]] += d * others;
            }
        }
    }
}

void oac_up(oac *a, const double *angles, const int8_t *ev, double *root) {
    cplx r = up(a, angles, ev);
    root[0] = creal(r);
    root[1] = cimag(r);
}

/* node values of the last upward pass, [n_nodes][2] */
void oac_values(const oac *a, double *out) {
    for (uint32_t i = 0; i < a->n_nodes; ++i) {
        out[2 * i] = creal(a->val[i]);
        out[2 * i + 1] = cimag(a->val[i]);
    }
}

/* root and the adjoint of every indicator leaf, [n_ind][2] */
void oac_marginals(oac *a, const double *angles, const int8_t *ev, double *root, double *ind_adj) {
    cplx r = up(a, angles, ev);
    down(a);
    if (root) { root[0] = creal(r); root[1] = cimag(r); }
    for (uint32_t i = 0; i < a->n_ind; ++i) {
        ind_adj[2 * i] = creal(a->adj[i]);
        ind_adj[2 * i + 1] = cimag(a->adj[i]);
    }
}

/* value += w Re f;  grad[k] += w Re d f / d angle_k */
void oac_gradient(oac *a, const double *angles, const int8_t *ev, double w, double *value, double *grad) {
    cplx r = up(a, angles, ev);
    down(a);
    *value += w * creal(r);
    for (uint32_t i = 0; i < a->n_leaves; ++i) {
        if (a->op[i] != 1) continue;
        cplx c = a->leaf_coef[2 * i] + I * a->leaf_coef[2 * i + 1];
        cplx dl = c * leaf_fn_deriv(a->leaf_b[i], angles[a->leaf_a[i]]);
        grad[a->leaf_a[i]] += w * creal(a->adj[i] * dl);
    }
}

static uint64_t splitmix64_k(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* chain-rule sampler (density AC): bits[s] = outcome index of sample s */
int oac_sample(oac *a, const double *angles, uint64_t seed, int32_t shots, uint64_t *bits) {
    const uint32_t n = a->n_qubits;
    int8_t *ev = (int8_t *)malloc(a->n_vars ? a->n_vars : 1);
    if (!ev) return -3;
    for (int32_t s = 0; s < shots; ++s) {
        for (uint32_t v = 0; v < a->n_vars; ++v) ev[v] = -1;
        uint64_t idx = 0;
        for (uint32_t j = 0; j < n; ++j) {
            const double P = creal(up(a, angles, ev));
            ev[j] = 0;
            const double p0 = creal(up(a, angles, ev));
            const double u = (double)(splitmix64_k(seed, (uint64_t)s * n + j + 1) >> 11) * (1.0 / 9007199254740992.0);
            const int bit = (u * P >= p0) ? 1 : 0;
            ev[j] = (int8_t)bit;
            idx = (idx << 1) | (uint64_t)bit;
        }
        bits[s] = idx;
    }
    free(ev);
    return 0;
}
