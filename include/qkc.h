/*
 * qkc.h -- C-ABI of the GB300 arithmetic-circuit engine for noisy variational
 * quantum circuits (Huang, Holtzen, Millstein, Van den Broeck, Martonosi,
 * "Logical Abstractions for Noisy Variational Quantum Algorithm Simulation",
 * ASPLOS 2021).
 *
 * The engine follows the paper's statement of the problem (Sec. 1, Sec. 3.2,
 * Sec. 3.3): a noisy circuit is compiled once into an arithmetic circuit (AC),
 * and the AC is then queried many times with new gate parameters and new
 * evidence -- amplitudes and probabilities by an upward pass (Sec. 3.3.1,
 * Table 5), every partial derivative by a downward pass (Sec. 3.3.2), and
 * samples of the output distribution.
 *
 * Conventions for every call below.
 *  - Pointers whose name ends in _dev are device memory owned by the caller
 *    (for example PyTorch tensors); the library never frees them.  Pointers
 *    without that suffix are host memory.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *    take a stream are asynchronous on it and write no host memory; the
 *    caller synchronises before reading results.
 *  - Every call returns a qkc_status; on failure a message is kept per host
 *    thread and returned by qkc_last_error().  No call aborts or traps.
 *  - An AC handle is not thread safe: calls on one handle must be issued from
 *    one host thread (or serialised by the caller) and on one stream at a time,
 *    because the handle owns its scratch buffers.
 *  - Outcome bit order: qubit 0 is the most significant bit of an outcome index.
 */
#ifndef QKC_H
#define QKC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QKC_OK = 0,
    QKC_ERR_ARG = 1,         /* a size, pointer or code is out of range               */
    QKC_ERR_FORMAT = 2,      /* a compiled-AC byte buffer is malformed                 */
    QKC_ERR_NOMEM = 3,       /* host or device allocation failed                      */
    QKC_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the name)      */
    QKC_ERR_TIMEOUT = 5,     /* a bounded wait ran out                                */
    QKC_ERR_UNSUPPORTED = 6, /* the query needs another AC kind                        */
    QKC_ERR_TOO_LARGE = 7    /* the AC would exceed the compiler's node budget         */
} qkc_status;

/* ------------------------------------------------------------------ circuits
 * One circuit operation (24 bytes).  `kind` codes:
 *   gates     H=0 X=1 Y=2 Z=3 RX=4 RY=5 RZ=6 CNOT=7 (q0 control, q1 target) CZ=8
 *   channels  DEP1=16 (symmetric depolarising, Kraus sqrt(1-p) I, sqrt(p/3) X, Y, Z)
 *             DEP2=17 (two-qubit depolarising on q0,q1: sqrt(1-p) I(x)I and
 *                      sqrt(p/15) for each of the 15 other Pauli products)
 *             AD=18   (amplitude damping, p = gamma)
 *             PD=19   (phase damping, p = gamma; the paper's Sec. 2.2 Kraus pair,
 *                      with the sign of Table 3b on the damping operator)
 *             PF=20   (phase flip: sqrt(1-p) I, sqrt(p) Z)
 *             BF=21   (bit flip:   sqrt(1-p) I, sqrt(p) X)
 * RX/RY/RZ(theta) = exp(-i theta P/2) with theta = angles[angle].  q1 = -1 for
 * one-qubit operations.  Noise strengths are fixed at compile time.
 */
typedef struct {
    int32_t kind;
    int32_t q0;
    int32_t q1;
    int32_t angle;
    double p;
} qkc_op;

enum { QKC_AC_AMPLITUDE = 0, QKC_AC_DENSITY = 1, QKC_AC_DENSITY_STEPS = 2, QKC_AC_TRAJECTORY = 3 };
enum { QKC_ORDER_AUTO = 0, QKC_ORDER_MINFILL = 1, QKC_ORDER_MINWEIGHT = 2, QKC_ORDER_CREATION = 3 };

/*
 * qkc_compile -- noisy circuit -> Bayesian network -> arithmetic circuit.
 *
 * Sec. 3.1 (conditional amplitude tables, Tables 3a-3c: the table of a gate is
 * the transpose of its unitary; multi-qubit gates must be monomial so only the
 * target gets a new node; a noise channel gets a random-variable node), Sec. 3.2
 * (knowledge compilation, with the simplifications of Table 4: known initial
 * states substituted, 0/1 parameters folded into the structure, every other
 * parameter kept as a leaf, intermediate qubit states summed out).  The
 * compiler used here is symbolic variable elimination with a min-fill order
 * (the paper names variable elimination as its first approach, Sec. 3.2)
 * instead of CNF + c2d.
 *
 * kind QKC_AC_AMPLITUDE: the paper's AC.  Its network polynomial is
 *   f(lambda) = sum_{x,r} prod lambda_{x_j} prod lambda_{r_k} A(x, r)
 * over output qubits x and noise random variables r (Table 5).
 * kind QKC_AC_DENSITY: the AC of the doubled network (ket copy with the tables
 * above, bra copy with their complex conjugates, noise variables and output
 * variables shared by both copies), whose polynomial is
 *   f(lambda) = sum_x prod_j lambda_{x_j} <x| rho |x>,
 * so partial evidence gives marginal probabilities exactly (this construction
 * is this library's reading of Sec. 3.3; the paper itself enumerates r).
 * kind QKC_AC_DENSITY_STEPS: one density AC per sampling step j = 0..n-1,
 * compiled into one node set (equal sub-ACs shared), each from the operations
 * in the backward light cone of qubits 0..j only.  Root j gives the marginal of
 * qubits <= j exactly, so the chain-rule sampler (Sec. 3.3) evaluates at step
 * j only the part of the circuit that can affect it.  The paper has no such
 * construction; it is this library's answer to its sampling cost.  Supported
 * by qkc_evaluate (the last root: the whole circuit) and qkc_sample only.
 *
 * `order` is one of QKC_ORDER_*; `max_nodes` bounds the node store during
 * compilation (0 = 2^31-1; intermediate nodes the final AC drops count too),
 * above it QKC_ERR_TOO_LARGE.  QKC_ORDER_AUTO eliminates each circuit with
 * min-fill and with min-weight on copies of the node store and keeps the order
 * that adds fewer nodes (their table-size estimates ignore sharing and dropped
 * zero entries and can be off severalfold); for DENSITY_STEPS it also compiles
 * the whole AC with min-fill and with min-weight throughout and returns the
 * smaller of those two when it has at least 10% fewer nodes (so it costs up to
 * about five compilations).  On success *out_bytes is a malloc'd buffer in the
 * compiled-AC format below; release it with qkc_free_bytes.
 */
qkc_status qkc_compile(const qkc_op *ops, int32_t n_ops, int32_t n_qubits, int32_t n_angles,
                       int32_t kind, int32_t order, int64_t max_nodes,
                       uint8_t **out_bytes, uint64_t *out_len);
void qkc_free_bytes(uint8_t *bytes);

/*
 * qkc_plan -- an elimination order's estimate, without building nodes (for
 * QKC_ORDER_AUTO: the order with the smaller estimate, which qkc_compile then
 * checks against the other by building both): *table_entries = sum over
 * eliminated variables of the product of the
 * cardinalities of the variable and its neighbours (about the node count), and
 * *max_log2_table = log2 of the largest such table (the order's width in bits).
 * Lets a caller reject a circuit whose AC would not fit before compiling it.
 */
qkc_status qkc_plan(const qkc_op *ops, int32_t n_ops, int32_t n_qubits, int32_t n_angles, int32_t kind,
                    int32_t order, double *table_entries, double *max_log2_table);

/*
 * Compiled-AC byte format (little endian, version 1).  Header of 16 uint32:
 *   [0] magic 0x43414B51 ("QKAC")  [1] version = 1  [2] kind  [3] n_qubits
 *   [4] n_angles  [5] n_vars  [6] n_nodes  [7] n_edges  [8] n_levels
 *   [9] n_leaves  [10] root  [11] n_ind  [12] n_roots (kind
 *   QKC_AC_DENSITY_STEPS: n_qubits, else 0)  [13] branch probabilities
 *   (kind QKC_AC_TRAJECTORY: the noise indicator count, else 0)  [14..15] 0
 * then these arrays, each starting on an 8-byte boundary:
 *   var_card[n_vars] u32      cardinality of each indicator variable
 *   var_tag[n_vars]  i32      qubit index of an output variable, or -1-k for
 *                             the noise variable of the k-th channel
 *   level_off[n_levels+1] u32 nodes of level L are [level_off[L], level_off[L+1])
 *   op[n_nodes] u8            0 IND, 1 PARAM, 2 CONST, 3 ADD, 4 MUL
 *   child_off[n_nodes+1] u32  children of node i are child[child_off[i] ..]
 *   child[n_edges] u32        every child has a lower level than its parent
 *   leaf_a[n_leaves] i32      IND: variable; PARAM: angle slot; CONST: -1
 *   leaf_b[n_leaves] i32      IND: value; PARAM: function (0 cos(t/2),
 *                             1 sin(t/2), 2 exp(-i t/2), 3 exp(+i t/2)); CONST: 0
 *   leaf_coef[n_leaves][2] f64 PARAM: complex coefficient c (leaf = c g(t));
 *                             CONST: the value; IND: (1, 0)
 *   roots[n_roots] u32        (light-cone steps only) root of step j; the
 *                             last is the header's root
 *   prior[header[13]] f64     (TRAJECTORY only) branch probability of every
 *                             noise indicator value, in (variable, value) order
 * Level 0 holds exactly the leaves.  Nodes 0 .. n_ind-1 are the indicator
 * leaves lambda_{v=k} in (variable, value) order, one per value of every
 * variable.  MUL nodes have exactly two children; ADD nodes two or more.
 */

/* ------------------------------------------------------------------ engine */
typedef struct qkc_ctx qkc_ctx; /* opaque: one CUDA device */
typedef struct qkc_ac qkc_ac;   /* opaque: one AC resident on the device + scratch */

typedef struct {
    int32_t kind, n_qubits, n_angles, n_vars, n_ind, precision;
    int64_t n_nodes, n_edges, n_levels, n_leaves, max_level_width;
    int64_t device_bytes;       /* structure bytes resident on the device   */
    int64_t reserved_columns;   /* columns the scratch currently holds      */
} qkc_ac_info;

/* Bind a context to CUDA device `device`. */
qkc_status qkc_ctx_create(int device, qkc_ctx **out);
void qkc_ctx_destroy(qkc_ctx *ctx);

/*
 * qkc_load_ac -- copy a compiled AC (host bytes, caller keeps them) to the
 * device of `ctx` (Sec. 3.2.2: compile once, reuse across simulations).
 * precision 32: node values complex FP32 with a power-of-two scale per
 * (level, column); 64: complex FP64.  Blocks until the copy is done.
 */
qkc_status qkc_load_ac(qkc_ctx *ctx, const uint8_t *bytes, uint64_t len, int32_t precision,
                       qkc_ac **out);
void qkc_free_ac(qkc_ac *ac);
qkc_status qkc_get_info(const qkc_ac *ac, qkc_ac_info *out);

/*
 * qkc_reserve -- size the AC's device scratch for up to `max_vectors` parameter
 * vectors and `max_columns` evaluation columns (grows, never shrinks).  Calls
 * that need more scratch than reserved grow it themselves, which synchronises
 * the device; reserve first to keep them asynchronous.
 */
qkc_status qkc_reserve(qkc_ac *ac, int64_t max_vectors, int64_t max_columns);

/*
 * qkc_set_tile_limit -- cap the column tile of this AC (0 = default: values and
 * adjoints each within 30% of the device memory; otherwise >= 64, rounded down
 * to a multiple of 64).  Calls with more columns than the tile process them in
 * tiles.  Lets many resident ACs share one device (serving).  Takes effect on
 * the next scratch growth; set it before the first query.
 */
qkc_status qkc_set_tile_limit(qkc_ac *ac, int64_t max_tile_columns);

/*
 * qkc_set_params -- bind gate parameters (Sec. 3.2.1, Table 4: parameters are
 * weight variables resolved at simulation time).  angles_dev is [n_vectors]
 * [n_angles] float64, row-major.  Every PARAM leaf gets c g(angle) per vector.
 */
qkc_status qkc_set_params(qkc_ac *ac, const double *angles_dev, int64_t n_vectors, void *stream);

/*
 * Evidence (Sec. 3.3.1: indicators are 1 for the observed value and 0 for the
 * others; unobserved variables have every indicator at 1).  evidence_dev is
 * [n_cols][n_vars] int8: -1 free, k >= 0 observed value k, -2 Pauli-Z sign
 * (binary variables only: lambda_0 = 1, lambda_1 = -1, so the density AC
 * returns <Z...Z> on those qubits).  col_vec_dev [n_cols] int32 names the
 * parameter vector of each column (< n_vectors of the last qkc_set_params).
 *
 * qkc_evaluate -- upward pass (Sec. 3.3.1): out_dev[c] = f(lambda_c) as
 * (re, im) float64, [n_cols][2].
 */
qkc_status qkc_evaluate(qkc_ac *ac, const int32_t *col_vec_dev, const int8_t *evidence_dev,
                        int64_t n_cols, double *out_dev, void *stream);

/*
 * qkc_reevaluate -- incremental upward pass after a parameter update that
 * touched one angle slot (memoisation across queries, Sec. 3.2.2: the AC is
 * compiled once and re-evaluated as parameters change; here only the part that
 * changed is recomputed).  Call it after qkc_set_params has bound new angles
 * that differ from those of the preceding evaluation in slot angle_slot only;
 * it binds that slot's parameter leaves again, recomputes their ancestors (the
 * slot's "dirty cone", found on first use of the slot and kept) for the columns
 * of the preceding qkc_evaluate, and writes out_dev[c] as qkc_evaluate would.
 * Preconditions, checked where the library can: the previous call on this AC
 * that touched its node values was qkc_evaluate or qkc_reevaluate with the same
 * col_vec_dev pointer (same contents) and n_cols, and n_cols fits one tile
 * (qkc_get_info's reserved columns; see qkc_reserve); else QKC_ERR_ARG.  The
 * caller must not have changed any other angle slot.  FP64: the same values
 * as a fresh qkc_evaluate; FP32: each level keeps the scale exponent of the
 * preceding pass, so values agree with a fresh pass up to rounding.
 */
qkc_status qkc_reevaluate(qkc_ac *ac, int32_t angle_slot, const int32_t *col_vec_dev, int64_t n_cols,
                          double *out_dev, void *stream);

/*
 * qkc_marginals -- upward then downward pass (Sec. 3.3.2, the differential
 * approach the paper cites): marg_dev[c][i] = d f / d lambda_i for every
 * indicator leaf i (n_ind of them, (variable, value) order) as (re, im)
 * float64, [n_cols][n_ind][2].  Because f is multilinear in the indicators,
 * for a density AC this is P(e without X_j, X_j = v) for every qubit j and
 * value v.  root_dev (nullable) receives f, [n_cols][2].
 */
qkc_status qkc_marginals(qkc_ac *ac, const int32_t *col_vec_dev, const int8_t *evidence_dev,
                         int64_t n_cols, double *root_dev, double *marg_dev, void *stream);

/*
 * qkc_gradient -- weighted expectation and its gradient in the gate angles.
 * For every vector v:  value_dev[v] = sum_{c: col_vec[c]=v} w_c Re f(lambda_c)
 * and grad_dev[v][k] = d value_dev[v] / d angle_k, with w = weight_dev [n_cols]
 * float64.  With one column per Z-string term and w_c its coefficient this is
 * <H> and its gradient.  The derivative is the downward pass taken to the
 * PARAM leaves, chained with d leaf / d angle (holomorphic chain rule).
 * value_dev [n_vectors], grad_dev [n_vectors][n_angles] float64.
 */
qkc_status qkc_gradient(qkc_ac *ac, const int32_t *col_vec_dev, const int8_t *evidence_dev,
                        const double *weight_dev, int64_t n_cols, int64_t n_vectors,
                        double *value_dev, double *grad_dev, void *stream);

/*
 * qkc_sample -- exact qubit-by-qubit conditional sampling of the output
 * distribution (Sec. 3.3.2 gives the sampling task; the paper's own sampler
 * is Gibbs MCMC, this one is the exact chain rule it compares against,
 * "ideal sampling").  Needs a DENSITY AC, or a DENSITY_STEPS AC, whose step j
 * takes p0 and P from root j (the light cone of qubits <= j) and otherwise runs
 * the same way (same draws, same decisions up to rounding).
 * For vector v, sample s, qubit j: u = (SplitMix64_k(seeds[v]) >> 11) 2^-53
 * with k = s*n_qubits + j + 1 (the k-th output of a SplitMix64 stream);
 * p0 = P(x_<j, X_j = 0), P = P(x_<j); x_j = 1 iff u * P >= p0, in float64.
 * Samples of one vector that share a prefix share one evaluation, and that one
 * upward pass gives both branch probabilities of the step: the indicator of
 * X_j = 1 is set to the imaginary unit, so the density polynomial (real and
 * linear in qubit j's indicators) returns P(x_<j, X_j = 0) + i P(x_<j, X_j = 1)
 * and P = their sum.  No probability is carried from one step to the next as a
 * difference (whose relative error would double with every 1-branch).
 * TRAJECTORY ACs (mixed-unitary channels only): every sample first draws its
 * noise trajectory r -- for noise variable i, u = (SplitMix64_k(~seeds[v]) >> 11)
 * 2^-53 with k = s*n_noise + i + 1, and r_i is the smallest value k with
 * u < p_0 + ... + p_k (the branch probabilities stored in the AC), else the
 * last -- and is then sampled as above with its noise variables observed at r,
 * which draws P(x) = sum_r P(r) P(x | r) exactly.  Samples without any error
 * share the groups of their vector, and so do samples of one vector that drew
 * the same error trajectory (found by hashing, then compared byte for byte).
 * bits_dev [n_vectors][max_shots] uint64: outcome index of each sample
 * (entries s >= shots[v] are left untouched).  shots_dev [n_vectors] int32.
 * total_shots: a host-side upper bound on sum_v min(shots[v], max_shots) used
 * to size the launches (<= 0: n_vectors x max_shots); an understated bound
 * never makes a kernel read or write out of range -- the excess samples are
 * dropped and qkc_check_status reports it.
 */
qkc_status qkc_sample(qkc_ac *ac, const uint64_t *seeds_dev, const int32_t *shots_dev,
                      int64_t n_vectors, int64_t max_shots, int64_t total_shots, uint64_t *bits_dev,
                      void *stream);

/*
 * qkc_sample_probs -- qkc_sample, and also probs_dev [n_vectors][max_shots] float64: for every
 * sample the probability P(x) of its outcome as the sampler computed it: the branch probability
 * P(x_<n-1, X_n-1 = x_n-1) of the last step's pass (for a TRAJECTORY AC, P(r, x) of the sample's
 * trajectory).  Entries s >= shots[v] are left untouched; -1 marks a sample dropped by an
 * understated total_shots.  It lets a caller state each sample's probability (for example to
 * weight or score samples) and check the sampler's arithmetic against an exact P(x).
 */
qkc_status qkc_sample_probs(qkc_ac *ac, const uint64_t *seeds_dev, const int32_t *shots_dev,
                            int64_t n_vectors, int64_t max_shots, int64_t total_shots, uint64_t *bits_dev,
                            double *probs_dev, void *stream);

/*
 * qkc_gibbs -- the paper's Markov-chain sampler (Sec. 3.3.2) on an AMPLITUDE AC:
 * chains over full assignments of the indicator variables (outputs and noise
 * variables) whose stationary distribution is proportional to |A(x, r)|^2, so
 * the output marginal is the noisy outcome distribution.  One update of
 * variable V is an upward and a downward pass at the chain's assignment: the
 * adjoint of lambda_{V=v} is the amplitude of the assignment with V set to v
 * (the polynomial is multilinear), and V is redrawn with probability
 * |A|^2 / sum |A|^2.  Systematic scan over the variables in index order,
 * n_sweeps sweeps per call.  Chain c uses the parameter vector col_vec_dev[c]
 * and, for the update of variable V in sweep t (counting from sweep_offset),
 * the uniform (SplitMix64_k(seeds_dev[c]) >> 11) 2^-53 with
 * k = t * n_vars + V + 1; the new value is the smallest v with
 * u * sum_w |A_w|^2 < sum_{w <= v} |A_w|^2, in FP64.
 * state_dev [n_chains][n_vars] int8: in, an assignment with nonzero amplitude;
 * out, the last one.  samples_dev [n_chains][n_sweeps] uint64 (nullable): the
 * outcome index after every sweep.  Variables may have at most 16 values.
 */
qkc_status qkc_gibbs(qkc_ac *ac, const int32_t *col_vec_dev, const uint64_t *seeds_dev, int64_t n_chains,
                     int8_t *state_dev, int64_t n_sweeps, int64_t sweep_offset, uint64_t *samples_dev,
                     void *stream);

/*
 * qkc_set_sampler -- how qkc_sample evaluates its columns.  mode 1 (default):
 * memoised -- at qubit j a node's value depends only on the vector and on the
 * prefix bits of the qubits < j in the node's indicator support, so nodes with
 * a small such support are evaluated once per (vector, key) instead of once
 * per prefix group (same results), when estimated cheaper than mode 0.
 * mode 2: memoised whenever the slots fit.  mode 0: every node once per group.
 * memo_budget_bytes caps the device memory of the memoised values (0: 40% of
 * the device memory and at most 60% of what is free); the sampler picks the
 * largest key width that fits, and falls back to mode 0 when none does or when
 * the memoised passes are estimated to cost more than the per-group ones.  When
 * the slots of every sampling step fit the budget side by side, they are kept
 * for the whole call and every step's per-slot tier is computed before the
 * first step (in one launch, or one per level index); otherwise each step
 * reuses the same slots.  The memoised values' allocation only grows, up to the
 * budget, and lasts until the AC is freed.
 */
qkc_status qkc_set_sampler(qkc_ac *ac, int32_t mode, int64_t memo_budget_bytes);

/*
 * qkc_check_status -- waits for the device and reports (then clears) the AC's
 * device-side error word: QKC_ERR_ARG if a qkc_sample call was given a
 * total_shots below the sum of its shots (the samples beyond the bound were
 * dropped and their entries are invalid).
 */
qkc_status qkc_check_status(qkc_ac *ac);

/*
 * qkc_evaluate_static -- the upward pass of qkc_evaluate (same arguments, same
 * results), but it allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- a serving loop that
 * must never stall on the implicit device synchronisation cudaMalloc/cudaFree
 * can cause, or a host application whose own memory pool has claimed the
 * device memory and forbids other allocations.  The caller still passes every
 * input and output buffer, and the AC's parameters must already be bound by
 * qkc_set_params (which allocates, once, outside the hot loop).
 *
 * Scratch is one file-scope device array of QKC_STATIC_SCRATCH_BYTES (64 MiB),
 * held by every GPU that loads this library until the process exits.  Columns
 * are processed in tiles of the largest multiple of 64 that fits it: node
 * values (8 bytes per node per column in FP32, 16 in FP64) plus, in FP32, two
 * int32 words per level per column.  An AC that needs more than the array for
 * a 64-column tile is rejected with QKC_ERR_TOO_LARGE (FP32: about 130K nodes).
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  Every call uses the same array and leaves its contents behind;
 * nothing a call reads is left over from an earlier call, but calls whose
 * work overlaps on the GPU (other streams, other host threads, other AC
 * handles) race on the array: serialise them.  A call also rewrites the AC
 * handle's own pass descriptor, so any other call on the same handle
 * (qkc_evaluate, qkc_marginals, qkc_sample, ...) whose work overlaps it on
 * another stream races with it too, as calls on one handle always do.
 */
#define QKC_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
qkc_status qkc_evaluate_static(qkc_ac *ac, const int32_t *col_vec_dev, const int8_t *evidence_dev,
                               int64_t n_cols, double *out_dev, void *stream);

/*
 * Measurement support (no counterpart in the paper).  qkc_stats_enable resets
 * the counters and, when enable != 0, records a pair of CUDA events around
 * every chain of level kernels (upward or downward pass of one column tile)
 * issued by later calls on this AC, with the number of columns that chain
 * processed, up to max_records chains.  qkc_get_stats waits for the recorded
 * events and returns the launch count of this library's kernels and, per pass
 * kind, the summed event time and the algorithmic bytes the level kernels move:
 * upward  (E + N - leaves) x elem per column (child reads, node writes);
 * downward (E + E_mul + N - 1) x elem per column (parent adjoints, siblings of
 * products, node writes); elem = 8 (FP32 complex) or 16 (FP64 complex).
 * A memoised sampling pass moves (children + 1) x elem per tier-A slot and per
 * tier-B node and group column.
 */
typedef struct {
    int64_t launches, records;
    int64_t up_passes, up_columns, up_launches;
    double up_ms, up_bytes;
    int64_t down_passes, down_columns, down_launches;
    double down_ms, down_bytes;
    int64_t memo_passes, memo_columns;  /* memoised sampling passes (qkc_set_sampler mode 1) */
    double memo_ms, memo_bytes;         /* both tiers */
    double memo_a_ms, memo_a_bytes;     /* tier A alone (the per-slot part of memo_ms / memo_bytes) */
    double up_edges, down_edges, memo_edges;  /* child references actually evaluated (one per child of a
                                                 computed node per column or slot; downward: one per
                                                 parent entry visited) */
} qkc_stats;
qkc_status qkc_stats_enable(qkc_ac *ac, int32_t enable, int64_t max_records);
qkc_status qkc_get_stats(qkc_ac *ac, qkc_stats *out);

/* Message of the last failed call on this host thread ("" if none). */
const char *qkc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QKC_H */
