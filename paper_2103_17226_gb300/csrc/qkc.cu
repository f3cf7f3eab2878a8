// qkc.cu -- GB300 (sm_103a) runtime and kernels for batched arithmetic-circuit
// evaluation: parameter binding, upward pass, downward pass, marginals, angle
// gradients and chain-rule sampling (the operations of Sec. 3.3 of Huang et al.,
// ASPLOS 2021, batched over many parameter vectors and evidence columns).
//
// Data layout in HBM (one AC, one column tile of T columns, T a multiple of 64):
//   values  V[node][T]  complex (float2 or double2), the batch dimension contiguous
//   adjoint A[node][T]  same layout (downward pass)
//   scale   S[level][T] int32, FP32 only: node n of level L holds m with
//           value = m * 2^S[L][col]; obs[level][T] = max exponent seen in the level
// Structure: level-sorted CSR (child_off/child), a transposed CSR of (parent,
// sibling) pairs for the pull-based downward pass, and node_level.
//
// Kernel shape: one launch per AC level; a warp owns a block of NB consecutive
// nodes of the level and one chunk of 64 (FP32) or 32 (FP64) columns, so every
// child gather is a coalesced 512-byte row segment (float4 / double2 per lane),
// and the node's structure words are warp-uniform broadcasts.
#include "../../include/qkc.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

extern "C" void qkc_set_error_(const char *msg) { g_last_error = msg ? msg : ""; }
extern "C" const char *qkc_last_error(void) { return g_last_error.c_str(); }

static qkc_status fail(qkc_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static qkc_status fail(qkc_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define QKC_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(QKC_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                                    \
    } while (0)

#define QKC_LAUNCH_CHECK()                                                                      \
    do {                                                                                        \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess)                                                                  \
            return fail(QKC_ERR_CUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                    \
    } while (0)

namespace {

enum : uint8_t { OP_IND = 0, OP_PARAM = 1, OP_CONST = 2, OP_ADD = 3, OP_MUL = 4 };
constexpr int NB = 8;          // nodes per warp item
constexpr int NBB = 32;        // tier-B nodes per warp item (memoised passes)
static_assert(NBB == 32, "memoB_level_f32 splits a node block of 32 by shifts");
constexpr int TPB = 256;       // threads per block
constexpr int OBS_EMPTY = -1000;
constexpr int64_t MEMO_RUN_T = 1024;           // tier-A levels with at most this many threads per vector
                                               // are walked in runs by one launch
constexpr int64_t MEMO_ALL_T = 4096;           // every step's tier A in one launch (a block per step and
                                               // vector) when no tier-A level is wider than this, else
                                               // a launch per level index
constexpr int64_t MEMO_INLINE_SCALE_B = 4096;  // tier-B sets up to this size form level scales inline
constexpr int64_t MEMO_RUN_B = NBB;            // FP32 tier-B levels of one node block (at most 32 nodes) are walked
                                               // in runs by one launch ...
constexpr int MEMO_RUN_LV = 16;                // ... of at most 16 levels and 512 nodes (shared memory)
constexpr int64_t MEMO_RUN_NODES = 512;
constexpr int MEMO_BKEYS = 32;  // per step, the distinct tier-A child supports whose group keys are tabled
constexpr int MEMO_APLANS = 7;  // log2 of the compress plans per step for scattered tier-A key masks
constexpr int MEMO_MARGIN = 2;  // early steps: memoise a node when its key space is >= 4x smaller than V 2^j

// ------------------------------------------------------------------ device helpers
// 2^k as a float: 0 below 2^-126, 2^127 above; no branches (the exponent field clamped to [0, 254])
__device__ __forceinline__ float pow2f(int k) { return __int_as_float(min(max(k + 127, 0), 254) << 23); }
__device__ __forceinline__ int exp_of(float2 v) {
    // exponent field of max(|re|, |im|) minus the bias (-127 for zero / denormals)
    int a = __float_as_int(v.x) & 0x7fffffff, b = __float_as_int(v.y) & 0x7fffffff;
    int m = a > b ? a : b;
    return (m >> 23) - 127;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Programmatic dependent launch: a kernel of the sampling chain is launched with programmatic stream
// serialisation, so it may be scheduled while the kernel before it in the stream finishes; its first
// act is to wait for that kernel's completion (and memory), then to let the next one be scheduled.
// Launched without the attribute, both instructions return at once.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

struct DevAC {
    const uint8_t *op;
    const uint32_t *child_off;
    const uint32_t *child;
    const uint16_t *node_level;
    const uint32_t *par_off;
    const int2 *par;          // (parent, sibling or -1)
    const int32_t *ind_var;   // [n_ind]
    const int32_t *ind_val;
    const int32_t *param_angle;  // [n_param]
    const int32_t *param_fn;
    const double2 *param_coef;
    const double2 *const_val;    // [n_const]
    const uint32_t *cl_off;      // child-level lists per level (FP32 scaling)
    const uint16_t *cl;
    int n_ind, n_param, n_const, n_vars, n_angles, n_qubits;
};

// ------------------------------------------------------------------ parameter binding
// One thread per (param leaf, vector): leaf = coef * g(angle).
template <typename C>
__global__ void bind_params_kernel(DevAC ac, const double *angles, int64_t n_vec, int64_t pv_pitch, C *pv) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)ac.n_param * n_vec;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int p = (int)(t / n_vec);
        int64_t v = t % n_vec;
        double th = angles[v * ac.n_angles + ac.param_angle[p]];
        double s, c;
        sincos(0.5 * th, &s, &c);
        double gr, gi;
        switch (ac.param_fn[p]) {
            case 0: gr = c; gi = 0.0; break;
            case 1: gr = s; gi = 0.0; break;
            case 2: gr = c; gi = -s; break;
            default: gr = c; gi = s; break;
        }
        double2 k = ac.param_coef[p];
        double re = k.x * gr - k.y * gi, im = k.x * gi + k.y * gr;
        C out;
        out.x = re;
        out.y = im;
        pv[(int64_t)p * pv_pitch + v] = out;
    }
}

// ------------------------------------------------------------------ leaf binding (level 0)
// Evidence source: either an explicit [cols][n_vars] int8 array, or a sampling
// prefix (qubits < j fixed to the prefix bits, qubit j fixed to 0, rest free).
struct EvSrc {
    const int8_t *ev;          // explicit evidence (may be null)
    const uint64_t *prefix;    // per column prefix bits (sampling)
    int j;                     // prefix length; the qubit j is fixed to 0 if clamp
    int clamp;
    const int32_t *col_vec;    // column -> parameter vector (null: identity)
    const int32_t *n_active;   // device count of active columns (null: use host count)
    int64_t n_vec;             // bound vectors; out-of-range map entries are clamped
    // sampling a TRAJECTORY AC: the noise variables (indicator variables n_qubits ..) are observed at
    // the trajectory of the sample that owns the column's group (col_traj[col], -1: every branch 0)
    const int8_t *traj;        // [samples][n_noise]
    const int32_t *col_traj;
    int n_noise;
};

// Everything that changes from one pass to the next lives in device memory, so the
// per-level launch sequence of a pass can be captured once as a CUDA graph and replayed.
struct PassDesc {
    EvSrc es;
    const void *pv;       // parameter leaf values [n_param][pv_pitch]
    int64_t pv_pitch;
    int64_t col0, ncols;  // first global column of this tile, columns in the tile (host bound)
};
__global__ void set_desc(PassDesc *dst, PassDesc v) {
    pdl_begin();
    *dst = v;
}
__device__ __forceinline__ int64_t desc_cols(const PassDesc &d) {
    int64_t n = d.ncols;
    if (d.es.n_active) n = min(n, (int64_t)(*d.es.n_active) - d.col0);
    return n;
}

__device__ __forceinline__ int64_t vec_of(const EvSrc &e, int64_t gc) {
    int64_t v = e.col_vec ? (int64_t)e.col_vec[gc] : gc;
    return v < 0 ? 0 : (v >= e.n_vec ? e.n_vec - 1 : v);
}

__device__ __forceinline__ int ev_code(const EvSrc &e, const DevAC &ac, int64_t col, int var) {
    if (e.ev) return e.ev[col * ac.n_vars + var];
    if (var >= ac.n_qubits) {  // a noise variable of a TRAJECTORY AC: the group's branch
        const int32_t t = e.col_traj ? e.col_traj[col] : -1;
        return t < 0 ? 0 : (int)e.traj[(int64_t)t * e.n_noise + (var - ac.n_qubits)];
    }
    int q = var;  // the output variables are the qubits
    if (q < e.j) return (int)((e.prefix[col] >> (e.j - 1 - q)) & 1ull);
    if (q == e.j && e.clamp) return -3;
    return -1;
}
// Indicator value for an evidence code: -1 free (1), -2 Pauli-Z sign (1, -1), k observed (1 at k);
// -3 "split" (1 for value 0, the imaginary unit for value 1).  The density polynomial is real and
// linear in each qubit's pair of indicators, so with qubit j split one upward pass returns
// P(e, X_j = 0) + i P(e, X_j = 1): both branch probabilities of a sampling step, each computed
// afresh (never one as a difference of two others).
__device__ __forceinline__ double2 ind_value(int code, int val) {
    if (code == -1) return make_double2(1.0, 0.0);
    if (code == -2) return make_double2(val == 0 ? 1.0 : -1.0, 0.0);
    if (code == -3) return val == 0 ? make_double2(1.0, 0.0) : make_double2(0.0, 1.0);
    return make_double2(code == val ? 1.0 : 0.0, 0.0);
}

// FP32 leaves; also initialises the level-0 scale (0) and observed exponent.
__global__ void bind_leaves_f32(DevAC ac, const PassDesc *pd, int64_t pitch, float2 *V, int *obs, int n_leaves) {
    const PassDesc d = *pd;
    const EvSrc &es = d.es;
    const int64_t col0 = d.col0, ncols = desc_cols(d), pv_pitch = d.pv_pitch;
    const float2 *pv = static_cast<const float2 *>(d.pv);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_leaves * pitch;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t / pitch);
        int64_t c = t % pitch;
        if (c >= ncols) continue;
        int64_t gc = col0 + c;
        float2 v;
        if (i < ac.n_ind) {
            const double2 lam = ind_value(ev_code(es, ac, gc, ac.ind_var[i]), ac.ind_val[i]);
            v = make_float2((float)lam.x, (float)lam.y);
        } else if (i < ac.n_ind + ac.n_param) {
            v = pv[(int64_t)(i - ac.n_ind) * pv_pitch + vec_of(es, gc)];
        } else {
            double2 k = ac.const_val[i - ac.n_ind - ac.n_param];
            v = make_float2((float)k.x, (float)k.y);
        }
        V[(int64_t)i * pitch + c] = v;
        atomicMax(&obs[c], exp_of(v));
    }
}

__global__ void bind_leaves_f64(DevAC ac, const PassDesc *pd, int64_t pitch, double2 *V, int n_leaves) {
    const PassDesc d = *pd;
    const EvSrc &es = d.es;
    const int64_t col0 = d.col0, ncols = desc_cols(d), pv_pitch = d.pv_pitch;
    const double2 *pv = static_cast<const double2 *>(d.pv);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_leaves * pitch;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t / pitch);
        int64_t c = t % pitch;
        if (c >= ncols) continue;
        int64_t gc = col0 + c;
        double2 v;
        if (i < ac.n_ind) {
            v = ind_value(ev_code(es, ac, gc, ac.ind_var[i]), ac.ind_val[i]);
        } else if (i < ac.n_ind + ac.n_param) {
            v = pv[(int64_t)(i - ac.n_ind) * pv_pitch + vec_of(es, gc)];
        } else {
            v = ac.const_val[i - ac.n_ind - ac.n_param];
        }
        V[(int64_t)i * pitch + c] = v;
    }
}

// ------------------------------------------------------------------ per-level scale (FP32)
// S[L][c] = max over the child levels L' of level L (the lists cl_off/cl: every child level in a
// full pass, those holding tier-B nodes in a memoised one) of S[L'][c] + obs[L'][c]; obs[L][c]
// reset.  Order-independent, so deterministic and per column.
__global__ void level_scale_kernel(const uint32_t *cl_off, const uint16_t *cl, int L, int64_t pitch, int floor_zero,
                                   int *S, int *obs) {
    pdl_begin();
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= pitch) return;
    int s = INT_MIN;
    for (uint32_t k = cl_off[L]; k < cl_off[L + 1]; ++k) {
        int Lp = cl[k];
        int o = obs[(int64_t)Lp * pitch + c];
        if (o == OBS_EMPTY) continue;  // no value of that level in this column (its scale is unused)
        int cand = S[(int64_t)Lp * pitch + c] + o;
        s = max(s, cand);
    }
    if (s == INT_MIN) s = 0;
    if (floor_zero && s < 0) s = 0;  // the level also reads unscaled values (memoised sampling)
    S[(int64_t)L * pitch + c] = s;
    obs[(int64_t)L * pitch + c] = OBS_EMPTY;
}

// The observed exponents of the listed levels back to empty: a memoised pass computes only its
// tier-B levels, and the level scales read the observed exponents of those levels and their child
// levels alone.
__global__ void obs_reset(int *obs, const int32_t *levels, int nlev, int64_t pitch) {
    pdl_begin();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < (int64_t)nlev * pitch) obs[(int64_t)levels[i / pitch] * pitch + i % pitch] = OBS_EMPTY;
}

// ------------------------------------------------------------------ upward pass, one level
struct LevelArgs {
    uint32_t lo, hi;   // node range of the level
    int L;
    int64_t pitch;     // columns per node row in the buffer
};

// FP32: lane holds 2 columns (one float4), warp covers 64 columns.
__global__ void __launch_bounds__(TPB) up_level_f32(DevAC ac, LevelArgs a, const PassDesc *pd,
                                                     float2 *__restrict__ V, const int *__restrict__ S,
                                                     int *__restrict__ obs) {
    const int64_t ncols = desc_cols(*pd);
    if (ncols <= 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (ncols + 63) >> 6;
    const int64_t nblk = (a.hi - a.lo + NB - 1) / NB;
    const int64_t items = nblk * nchunks;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t hp = a.pitch >> 1;  // float4 per row
    float4 *V4 = reinterpret_cast<float4 *>(V);
    for (int64_t it = wid; it < items; it += nw) {
        const int64_t chunk = it % nchunks;
        const int64_t blk = it / nchunks;
        const int64_t col = chunk * 64 + lane * 2;
        if (col >= ncols) continue;
        const int2 sL = *reinterpret_cast<const int2 *>(S + (int64_t)a.L * a.pitch + col);
        int m0 = -127, m1 = -127;
        const uint32_t n0 = a.lo + (uint32_t)blk * NB;
        const uint32_t n1 = min(a.hi, n0 + NB);
        for (uint32_t n = n0; n < n1; ++n) {
            const uint8_t o = ac.op[n];
            const uint32_t e0 = ac.child_off[n], e1 = ac.child_off[n + 1];
            float4 r;
            if (o == OP_MUL) {
                const uint32_t ca = ac.child[e0], cb = ac.child[e0 + 1];
                const int la = ac.node_level[ca], lb = ac.node_level[cb];
                const float4 va = __ldg(V4 + (int64_t)ca * hp + (col >> 1));
                const float4 vb = __ldg(V4 + (int64_t)cb * hp + (col >> 1));
                const int2 sa = __ldg(reinterpret_cast<const int2 *>(S + (int64_t)la * a.pitch + col));
                const int2 sb = __ldg(reinterpret_cast<const int2 *>(S + (int64_t)lb * a.pitch + col));
                float2 p0 = cmul(make_float2(va.x, va.y), make_float2(vb.x, vb.y));
                float2 p1 = cmul(make_float2(va.z, va.w), make_float2(vb.z, vb.w));
                p0 = cscale(p0, pow2f(sa.x + sb.x - sL.x));
                p1 = cscale(p1, pow2f(sa.y + sb.y - sL.y));
                r = make_float4(p0.x, p0.y, p1.x, p1.y);
            } else {
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (uint32_t e = e0; e < e1; ++e) {
                    const uint32_t c = ac.child[e];
                    const int lc = ac.node_level[c];
                    const float4 v = __ldg(V4 + (int64_t)c * hp + (col >> 1));
                    const int2 sc = __ldg(reinterpret_cast<const int2 *>(S + (int64_t)lc * a.pitch + col));
                    const float f0 = pow2f(sc.x - sL.x), f1 = pow2f(sc.y - sL.y);
                    acc.x += v.x * f0; acc.y += v.y * f0;
                    acc.z += v.z * f1; acc.w += v.w * f1;
                }
                r = acc;
            }
            V4[(int64_t)n * hp + (col >> 1)] = r;
            m0 = max(m0, exp_of(make_float2(r.x, r.y)));
            m1 = max(m1, exp_of(make_float2(r.z, r.w)));
        }
        atomicMax(obs + (int64_t)a.L * a.pitch + col, m0);
        if (col + 1 < ncols) atomicMax(obs + (int64_t)a.L * a.pitch + col + 1, m1);
    }
}

// FP64: lane holds 1 column (one double2), warp covers 32 columns.  No scaling.
__global__ void __launch_bounds__(TPB) up_level_f64(DevAC ac, LevelArgs a, const PassDesc *pd,
                                                     double2 *__restrict__ V) {
    const int64_t ncols = desc_cols(*pd);
    if (ncols <= 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (ncols + 31) >> 5;
    const int64_t nblk = (a.hi - a.lo + NB - 1) / NB;
    const int64_t items = nblk * nchunks;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = wid; it < items; it += nw) {
        const int64_t chunk = it % nchunks;
        const int64_t blk = it / nchunks;
        const int64_t col = chunk * 32 + lane;
        if (col >= ncols) continue;
        const uint32_t n0 = a.lo + (uint32_t)blk * NB;
        const uint32_t n1 = min(a.hi, n0 + NB);
        for (uint32_t n = n0; n < n1; ++n) {
            const uint8_t o = ac.op[n];
            const uint32_t e0 = ac.child_off[n], e1 = ac.child_off[n + 1];
            double2 r;
            if (o == OP_MUL) {
                const double2 va = __ldg(V + (int64_t)ac.child[e0] * a.pitch + col);
                const double2 vb = __ldg(V + (int64_t)ac.child[e0 + 1] * a.pitch + col);
                r = cmul(va, vb);
            } else {
                r = make_double2(0.0, 0.0);
                for (uint32_t e = e0; e < e1; ++e) {
                    const double2 v = __ldg(V + (int64_t)ac.child[e] * a.pitch + col);
                    r.x += v.x; r.y += v.y;
                }
            }
            V[(int64_t)n * a.pitch + col] = r;
        }
    }
}

// ------------------------------------------------------------------ incremental upward pass
// After qkc_set_params changed one angle slot: the slot's parameter leaves are bound again and
// only their ancestors (the slot's dirty cone, by level) are recomputed over the tile of the
// preceding evaluation, with the arithmetic of up_level_*; every other node keeps its value
// and every level keeps its FP32 scale.
template <typename C>
__global__ void rebind_param_leaves(const uint32_t *leaves, int nleaves, const PassDesc *pd, int64_t pitch, C *V,
                                    int n_ind) {
    const PassDesc d = *pd;
    const int64_t ncols = desc_cols(d);
    const C *pv = static_cast<const C *>(d.pv);
    const int64_t total = (int64_t)nleaves * ncols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / ncols, c = t - i * ncols;
        const uint32_t leaf = leaves[i];
        V[(int64_t)leaf * pitch + c] = pv[(int64_t)(leaf - n_ind) * d.pv_pitch + vec_of(d.es, d.col0 + c)];
    }
}

__global__ void __launch_bounds__(TPB) up_list_f32(DevAC ac, LevelArgs a, const uint32_t *nodes, int64_t count,
                                                    const PassDesc *pd, float2 *__restrict__ V,
                                                    const int *__restrict__ S) {
    const int64_t ncols = desc_cols(*pd);
    if (ncols <= 0 || count <= 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (ncols + 63) >> 6;
    const int64_t items = ((count + NB - 1) / NB) * nchunks;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t hp = a.pitch >> 1;
    float4 *V4 = reinterpret_cast<float4 *>(V);
    for (int64_t it = wid; it < items; it += nw) {
        const int64_t chunk = it % nchunks;
        const int64_t blk = it / nchunks;
        const int64_t col = chunk * 64 + lane * 2;
        if (col >= ncols) continue;
        const int2 sL = *reinterpret_cast<const int2 *>(S + (int64_t)a.L * a.pitch + col);
        const int64_t k1 = min(count, (blk + 1) * NB);
        for (int64_t kk = blk * NB; kk < k1; ++kk) {
            const uint32_t n = nodes[kk];
            const uint8_t o = ac.op[n];
            const uint32_t e0 = ac.child_off[n], e1 = ac.child_off[n + 1];
            float4 r;
            if (o == OP_MUL) {
                const uint32_t ca = ac.child[e0], cb = ac.child[e0 + 1];
                const int la = ac.node_level[ca], lb = ac.node_level[cb];
                const float4 va = __ldg(V4 + (int64_t)ca * hp + (col >> 1));
                const float4 vb = __ldg(V4 + (int64_t)cb * hp + (col >> 1));
                const int2 sa = __ldg(reinterpret_cast<const int2 *>(S + (int64_t)la * a.pitch + col));
                const int2 sb = __ldg(reinterpret_cast<const int2 *>(S + (int64_t)lb * a.pitch + col));
                float2 p0 = cmul(make_float2(va.x, va.y), make_float2(vb.x, vb.y));
                float2 p1 = cmul(make_float2(va.z, va.w), make_float2(vb.z, vb.w));
                p0 = cscale(p0, pow2f(sa.x + sb.x - sL.x));
                p1 = cscale(p1, pow2f(sa.y + sb.y - sL.y));
                r = make_float4(p0.x, p0.y, p1.x, p1.y);
            } else {
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (uint32_t e = e0; e < e1; ++e) {
                    const uint32_t c = ac.child[e];
                    const int lc = ac.node_level[c];
                    const float4 v = __ldg(V4 + (int64_t)c * hp + (col >> 1));
                    const int2 sc = __ldg(reinterpret_cast<const int2 *>(S + (int64_t)lc * a.pitch + col));
                    const float f0 = pow2f(sc.x - sL.x), f1 = pow2f(sc.y - sL.y);
                    acc.x += v.x * f0; acc.y += v.y * f0;
                    acc.z += v.z * f1; acc.w += v.w * f1;
                }
                r = acc;
            }
            V4[(int64_t)n * hp + (col >> 1)] = r;
        }
    }
}

__global__ void __launch_bounds__(TPB) up_list_f64(DevAC ac, LevelArgs a, const uint32_t *nodes, int64_t count,
                                                    const PassDesc *pd, double2 *__restrict__ V) {
    const int64_t ncols = desc_cols(*pd);
    if (ncols <= 0 || count <= 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (ncols + 31) >> 5;
    const int64_t items = ((count + NB - 1) / NB) * nchunks;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = wid; it < items; it += nw) {
        const int64_t chunk = it % nchunks;
        const int64_t blk = it / nchunks;
        const int64_t col = chunk * 32 + lane;
        if (col >= ncols) continue;
        const int64_t k1 = min(count, (blk + 1) * NB);
        for (int64_t kk = blk * NB; kk < k1; ++kk) {
            const uint32_t n = nodes[kk];
            const uint8_t o = ac.op[n];
            const uint32_t e0 = ac.child_off[n], e1 = ac.child_off[n + 1];
            double2 r;
            if (o == OP_MUL) {
                const double2 va = __ldg(V + (int64_t)ac.child[e0] * a.pitch + col);
                const double2 vb = __ldg(V + (int64_t)ac.child[e0 + 1] * a.pitch + col);
                r = cmul(va, vb);
            } else {
                r = make_double2(0.0, 0.0);
                for (uint32_t e = e0; e < e1; ++e) {
                    const double2 v = __ldg(V + (int64_t)ac.child[e] * a.pitch + col);
                    r.x += v.x; r.y += v.y;
                }
            }
            V[(int64_t)n * a.pitch + col] = r;
        }
    }
}

// ------------------------------------------------------------------ downward pass, split by fan-out
// Per level, nodes whose parent lists hold at most HEAVY entries are "light": a warp owns NB
// of them x one column chunk and walks each parent list four entries at a time (independent
// loads in flight).  "Heavy" nodes get a whole block per column chunk: its 8 warps take the
// parents round-robin and the partial sums are added in warp order (deterministic).  CONST
// leaves are never visited: their adjoints are not used.
constexpr int HEAVY = 64;

__device__ __forceinline__ float4 down_term_f32(const int2 ps, const float4 *A4, const float4 *V4, const int *S,
                                                const uint16_t *node_level, int64_t hp, int64_t pitch, int64_t col) {
    const float4 dp = A4[(int64_t)ps.x * hp + (col >> 1)];
    if (ps.y < 0) return dp;
    const int ls = node_level[ps.y];
    const float4 vs = __ldg(V4 + (int64_t)ps.y * hp + (col >> 1));
    const int2 ss = __ldg(reinterpret_cast<const int2 *>(S + (int64_t)ls * pitch + col));
    const float2 s0 = cscale(make_float2(vs.x, vs.y), pow2f(ss.x));
    const float2 s1 = cscale(make_float2(vs.z, vs.w), pow2f(ss.y));
    const float2 t0 = cmul(make_float2(dp.x, dp.y), s0);
    const float2 t1 = cmul(make_float2(dp.z, dp.w), s1);
    return make_float4(t0.x, t0.y, t1.x, t1.y);
}
__device__ __forceinline__ void acc4(float4 &a, const float4 b) { a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w; }

struct DownArgs {
    const uint32_t *nodes;  // node ids of this level's light (or heavy) list
    int64_t count;
    int64_t pitch;
};

__global__ void __launch_bounds__(TPB) down_light_f32(DevAC ac, DownArgs a, const PassDesc *pd, const float2 *__restrict__ V,
                                                       const int *__restrict__ S, float2 *A) {
    const int64_t ncols = pd->ncols;
    if (ncols <= 0 || a.count <= 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (ncols + 63) >> 6;
    const int64_t nblk = (a.count + NB - 1) / NB;
    const int64_t items = nblk * nchunks;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t hp = a.pitch >> 1;
    const float4 *V4 = reinterpret_cast<const float4 *>(V);
    float4 *A4 = reinterpret_cast<float4 *>(A);
    for (int64_t it = wid; it < items; it += nw) {
        const int64_t chunk = it % nchunks;
        const int64_t blk = it / nchunks;
        const int64_t col = chunk * 64 + lane * 2;
        if (col >= ncols) continue;
        const int64_t k1 = min(a.count, (blk + 1) * NB);
        for (int64_t k = blk * NB; k < k1; ++k) {
            const uint32_t n = a.nodes[k];
            const uint32_t e1 = ac.par_off[n + 1];
            uint32_t e = ac.par_off[n];
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (; e + 4 <= e1; e += 4) {
                const int2 p0 = ac.par[e], p1 = ac.par[e + 1], p2 = ac.par[e + 2], p3 = ac.par[e + 3];
                const float4 t0 = down_term_f32(p0, A4, V4, S, ac.node_level, hp, a.pitch, col);
                const float4 t1 = down_term_f32(p1, A4, V4, S, ac.node_level, hp, a.pitch, col);
                const float4 t2 = down_term_f32(p2, A4, V4, S, ac.node_level, hp, a.pitch, col);
                const float4 t3 = down_term_f32(p3, A4, V4, S, ac.node_level, hp, a.pitch, col);
                acc4(acc, t0); acc4(acc, t1); acc4(acc, t2); acc4(acc, t3);
            }
            for (; e < e1; ++e) acc4(acc, down_term_f32(ac.par[e], A4, V4, S, ac.node_level, hp, a.pitch, col));
            A4[(int64_t)n * hp + (col >> 1)] = acc;
        }
    }
}

__global__ void __launch_bounds__(TPB) down_heavy_f32(DevAC ac, DownArgs a, const PassDesc *pd, const float2 *__restrict__ V,
                                                       const int *__restrict__ S, float2 *A) {
    __shared__ float4 part[TPB / 32][32];
    const int64_t ncols = pd->ncols;
    const int64_t nchunks = (ncols + 63) >> 6;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t hp = a.pitch >> 1;
    const float4 *V4 = reinterpret_cast<const float4 *>(V);
    float4 *A4 = reinterpret_cast<float4 *>(A);
    for (int64_t it = blockIdx.x; it < a.count * nchunks; it += gridDim.x) {
        const int64_t chunk = it % nchunks;
        const uint32_t n = a.nodes[it / nchunks];
        const int64_t col = chunk * 64 + lane * 2;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (col < ncols)
            for (uint32_t e = ac.par_off[n] + w; e < ac.par_off[n + 1]; e += TPB / 32)
                acc4(acc, down_term_f32(ac.par[e], A4, V4, S, ac.node_level, hp, a.pitch, col));
        part[w][lane] = acc;
        __syncthreads();
        if (w == 0 && col < ncols) {
            float4 t = part[0][lane];
            for (int k = 1; k < TPB / 32; ++k) acc4(t, part[k][lane]);
            A4[(int64_t)n * hp + (col >> 1)] = t;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double2 down_term_f64(const int2 ps, const double2 *A, const double2 *V, int64_t pitch,
                                                 int64_t col) {
    const double2 dp = A[(int64_t)ps.x * pitch + col];
    if (ps.y < 0) return dp;
    return cmul(dp, __ldg(V + (int64_t)ps.y * pitch + col));
}

__global__ void __launch_bounds__(TPB) down_light_f64(DevAC ac, DownArgs a, const PassDesc *pd, const double2 *__restrict__ V,
                                                       double2 *A) {
    const int64_t ncols = pd->ncols;
    if (ncols <= 0 || a.count <= 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (ncols + 31) >> 5;
    const int64_t nblk = (a.count + NB - 1) / NB;
    const int64_t items = nblk * nchunks;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = wid; it < items; it += nw) {
        const int64_t chunk = it % nchunks;
        const int64_t blk = it / nchunks;
        const int64_t col = chunk * 32 + lane;
        if (col >= ncols) continue;
        const int64_t k1 = min(a.count, (blk + 1) * NB);
        for (int64_t k = blk * NB; k < k1; ++k) {
            const uint32_t n = a.nodes[k];
            const uint32_t e1 = ac.par_off[n + 1];
            uint32_t e = ac.par_off[n];
            double2 acc = make_double2(0.0, 0.0);
            for (; e + 4 <= e1; e += 4) {
                const int2 p0 = ac.par[e], p1 = ac.par[e + 1], p2 = ac.par[e + 2], p3 = ac.par[e + 3];
                const double2 t0 = down_term_f64(p0, A, V, a.pitch, col), t1 = down_term_f64(p1, A, V, a.pitch, col);
                const double2 t2 = down_term_f64(p2, A, V, a.pitch, col), t3 = down_term_f64(p3, A, V, a.pitch, col);
                acc.x += t0.x; acc.y += t0.y; acc.x += t1.x; acc.y += t1.y;
                acc.x += t2.x; acc.y += t2.y; acc.x += t3.x; acc.y += t3.y;
            }
            for (; e < e1; ++e) {
                const double2 t = down_term_f64(ac.par[e], A, V, a.pitch, col);
                acc.x += t.x; acc.y += t.y;
            }
            A[(int64_t)n * a.pitch + col] = acc;
        }
    }
}

__global__ void __launch_bounds__(TPB) down_heavy_f64(DevAC ac, DownArgs a, const PassDesc *pd, const double2 *__restrict__ V,
                                                       double2 *A) {
    __shared__ double2 part[TPB / 32][32];
    const int64_t ncols = pd->ncols;
    const int64_t nchunks = (ncols + 31) >> 5;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t it = blockIdx.x; it < a.count * nchunks; it += gridDim.x) {
        const int64_t chunk = it % nchunks;
        const uint32_t n = a.nodes[it / nchunks];
        const int64_t col = chunk * 32 + lane;
        double2 acc = make_double2(0.0, 0.0);
        if (col < ncols)
            for (uint32_t e = ac.par_off[n] + w; e < ac.par_off[n + 1]; e += TPB / 32) {
                const double2 t = down_term_f64(ac.par[e], A, V, a.pitch, col);
                acc.x += t.x; acc.y += t.y;
            }
        part[w][lane] = acc;
        __syncthreads();
        if (w == 0 && col < ncols) {
            double2 t = part[0][lane];
            for (int k = 1; k < TPB / 32; ++k) { t.x += part[k][lane].x; t.y += part[k][lane].y; }
            A[(int64_t)n * a.pitch + col] = t;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ memoised sampling
// How a tier-B node finds a tier-A child's slot from a group's prefix (bit q = x_q): the
// child's key is the prefix bits at the child's support m, packed into the low bits, computed
// by the mask-compress of Warren (Hacker's Delight, 2nd ed., Sec. 7-4) with its six
// shift masks mv[i] (bits moving right by 2^i in round i) precomputed on the host.
struct KeyPlan {
    int64_t off;     // the child's tier-A block (units)
    uint64_t m;      // the child's support among the qubits < j
    uint64_t mv[6];  // compress masks of m
    uint32_t k;      // |m|
    int32_t mid;     // row of the step's group-key table holding this support's keys, -1 if none
};

// At sampling step j a group's evidence fixes qubits < j to its prefix and qubit j to 0, so a
// node's value depends only on the vector and on the prefix bits of the qubits < j in the
// node's indicator support sigma(n).  With k = |sigma(n) & jmask| such bits, a node needs at
// most V * 2^k distinct values.  Nodes with k <= t_j ("tier A") are computed once per
// (vector, key) on a dense slot space -- slot = vector * 2^k + key, key bit i = prefix bit of
// the i-th smallest qubit of sigma(n) & jmask -- instead of once per group; tier A is closed
// under children (sigma(child) is a subset of sigma(parent)).  The other nodes ("tier B") are
// computed per group as before and read tier-A children through their key.  Tier-A values are
// unscaled; a tier-B level that reads one keeps its scale exponent at least 0.
struct MemoDesc {
    int64_t V;            // vectors
    int32_t j, clamp;
    uint64_t jmask;       // qubits < j
    const void *pv;       // parameter leaf values
    int64_t pv_pitch;
    void *VA;             // tier-A values
    const int64_t *offu;  // per node: start of its tier-A block in units (x V slots), -1 for tier B
    const uint64_t *sigma;
    const uint32_t *emask;  // per child edge of a tier-A node: the child's key bits in the parent's key,
                            // or (bit 31 set) the index of a key plan in aplan for a scattered mask
    const uint4 *brec;      // per child edge of a tier-B node, in node order (layout: BChild below)
    const KeyPlan *kplan;  // per tier-A child of a tier-B node (this step)
    const KeyPlan *aplan;  // per distinct scattered child-key mask of tier-A parents (this step)
    const KeyPlan *bplan;  // the step's tabled supports (nbm of them) ...
    int32_t nbm;
    uint32_t *keys;        // ... and their keys per group column of the tile: keys[row * kpitch + column]
    int64_t kpitch;
    const uint32_t *bcl_off;  // per level: its child levels that hold tier-B nodes in this step,
    const uint16_t *bcl;      // bcl[bcl_off[L] .. bcl_off[L + 1]) (the level scales read those alone)
};

__device__ __forceinline__ uint32_t plan_key(const KeyPlan *kp, uint64_t x, bool narrow) {
    if (narrow) {  // every qubit < j < 32: 32-bit words, five rounds
        uint32_t y = (uint32_t)x & (uint32_t)__ldg(&kp->m);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const uint32_t t = y & (uint32_t)__ldg(&kp->mv[i]);
            y = (y ^ t) | (t >> (1 << i));
        }
        return y;
    }
    uint64_t y = x & __ldg(&kp->m);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint64_t t = y & __ldg(&kp->mv[i]);
        y = (y ^ t) | (t >> (1 << i));
    }
    return (uint32_t)y;
}
__global__ void set_memo_desc(MemoDesc *dst, MemoDesc v) {
    pdl_begin();
    *dst = v;
}

// bits of x selected by mask m, packed into the low bits in order (contiguous runs take a shift)
__device__ __forceinline__ uint32_t extract_bits(uint64_t x, uint64_t m) {
    if (m == 0) return 0u;
    const int z = __ffsll((long long)m) - 1;
    const uint64_t r = m >> z;
    if ((r & (r + 1)) == 0) return (uint32_t)((x >> z) & r);
    uint32_t out = 0;
    for (int i = 0; m; ++i) {
        const uint64_t b = m & (~m + 1);
        if (x & b) out |= 1u << i;
        m ^= b;
    }
    return out;
}

template <typename C>
__device__ __forceinline__ C memo_leaf(const DevAC &ac, const MemoDesc &md, uint32_t n, int64_t vec, uint32_t key) {
    C r;
    const uint8_t o = ac.op[n];
    if (o == OP_IND) {
        const int q = ac.ind_var[n], val = ac.ind_val[n];
        double lam = 1.0, lim = 0.0;
        if (q < md.j) lam = ((int)(key & 1u) == val) ? 1.0 : 0.0;
        else if (q == md.j && md.clamp) {  // split: 1 for X_j = 0, the imaginary unit for X_j = 1
            lam = (val == 0) ? 1.0 : 0.0;
            lim = (val == 0) ? 0.0 : 1.0;
        }
        r.x = lam;
        r.y = lim;
    } else if (o == OP_PARAM) {
        r = static_cast<const C *>(md.pv)[(int64_t)(n - ac.n_ind) * md.pv_pitch + vec];
    } else {
        const double2 k = ac.const_val[n - ac.n_ind - ac.n_param];
        r.x = k.x;
        r.y = k.y;
    }
    return r;
}

// Tier-A nodes of one level, grouped by key width: the group's nodes are nodes[nb ..] and
// their unit blocks (2^k units each, one unit = one key of one vector) start t0 units into the
// level, in the same order, so a unit index gives its node and key by a shift.
struct MemoAGroup {
    uint32_t t0, nb, k, u0;  // first thread, first node, key width, first unit (within the level)
};

// Key widths from which a thread evaluates four slots of one node (keys key0 + 32 r, r < 4, with
// bits 5-6 of key0 clear): the node and its children are looked up once, and since the packing
// of bits is OR-linear, a child key is ck(key0) | ck(32 r), two per-child constants.
constexpr int MEMO_QUAD_K = 7;

// One thread's tier-A work at level-local thread index t for vector vec: one slot, or four slots of
// one node (keys key0 + 32 r) from key width MEMO_QUAD_K.
template <typename C>
__device__ __forceinline__ void memoA_slot(const DevAC &ac, const MemoDesc &md, C *VA, const uint32_t *nodes,
                                           const MemoAGroup *grp, int ng, int64_t u0, int64_t vec, uint32_t t) {
    int gi = 0;
    while (gi + 1 < ng && __ldg(&grp[gi + 1].t0) <= t) ++gi;
    const uint32_t t0 = __ldg(&grp[gi].t0), nb = __ldg(&grp[gi].nb), ug = __ldg(&grp[gi].u0);
    const int k = (int)__ldg(&grp[gi].k);
    const uint32_t q = t - t0;
    const bool quad = k >= MEMO_QUAD_K;
    const uint32_t rel = quad ? (((q >> 5) << 7) | (q & 31u)) : q;  // first unit within the group
    const uint32_t nl = rel >> k;
    const uint32_t key0 = rel & ((1u << k) - 1u);
    const uint32_t n = nodes[nb + nl];
    C r[4];
    const uint8_t o = ac.op[n];
    if (o <= OP_CONST) {  // leaves have at most one key bit: one slot
        r[0] = memo_leaf<C>(ac, md, n, vec, key0);
    } else {
        const uint32_t e0 = ac.child_off[n], e1 = ac.child_off[n + 1];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            r[i].x = (o == OP_MUL) ? 1 : 0;
            r[i].y = 0;
        }
        const uint32_t full = (1u << k) - 1u;
        for (uint32_t e = e0; e < e1; ++e) {
            const uint32_t c = ac.child[e];
            const uint32_t me = md.emask[e];  // the child's key bits inside this node's key
            int kc;
            uint32_t ck0, m;
            if (me == full) {  // same key space: same key
                kc = k;
                ck0 = key0;
                m = full;
            } else if (me & 0x80000000u) {
                const KeyPlan *kp = md.aplan + (me & 0x7fffffffu);
                kc = (int)__ldg(&kp->k);
                m = (uint32_t)__ldg(&kp->m);
                ck0 = plan_key(kp, key0, true);
            } else {
                kc = __popc(me);
                m = me;
                ck0 = extract_bits(key0, me);
            }
            const uint32_t d1 = ((m >> 5) & 1u) ? 1u << __popc(m & 31u) : 0u;  // ck(32)
            const uint32_t d2 = ((m >> 6) & 1u) ? 1u << __popc(m & 63u) : 0u;  // ck(64)
            const C *src = VA + md.V * md.offu[c] + (vec << kc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i > 0 && !quad) break;
                const C v = src[ck0 | ((i & 1) ? d1 : 0u) | ((i & 2) ? d2 : 0u)];
                if (o == OP_MUL) {
                    C mm;
                    mm.x = r[i].x * v.x - r[i].y * v.y;
                    mm.y = r[i].x * v.y + r[i].y * v.x;
                    r[i] = mm;
                } else {
                    r[i].x += v.x;
                    r[i].y += v.y;
                }
            }
        }
    }
    C *dst = VA + md.V * (u0 + ug + ((int64_t)nl << k)) + (vec << k) + key0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i > 0 && !quad) break;
        dst[32 * i] = r[i];
    }
}

// One level of tier A: a thread per slot, or per four slots of one node, of the level's tier-A
// blocks (vector, node, key).
template <typename C>
__global__ void __launch_bounds__(TPB, sizeof(C) == 8 ? 8 : 1) memoA_level(DevAC ac, const MemoDesc *mdp,
                                                                          const uint32_t *nodes,
                                                    const MemoAGroup *grp, int ng, int64_t u0, uint32_t T) {
    pdl_begin();
    if (T == 0 || ng <= 0) return;
    const MemoDesc md = *mdp;
    C *VA = static_cast<C *>(md.VA);
    const uint32_t nblk = (T + TPB - 1) / TPB;
    const int64_t items = md.V * (int64_t)nblk;
    // block item b covers vector b / nblk and threads (b % nblk) * TPB + thread; quotient and
    // remainder are stepped along the grid-stride loop rather than divided every time
    int64_t vec = blockIdx.x / nblk;
    uint32_t rb = blockIdx.x % nblk;
    const uint32_t dq = gridDim.x / nblk, dr = gridDim.x % nblk;
    for (int64_t b = blockIdx.x; b < items; b += gridDim.x) {
        const uint32_t t = rb * TPB + threadIdx.x;
        if (t < T) memoA_slot<C>(ac, md, VA, nodes, grp, ng, u0, vec, t);
        rb += dr;
        vec += dq;
        if (rb >= nblk) {
            rb -= nblk;
            ++vec;
        }
    }
}

// A run of consecutive small tier-A levels in one launch: a block per vector walks the levels in
// order, its threads covering each level's slots, with a block barrier between levels (a slot reads
// only slots of its own vector on lower levels).
struct MemoARunLevel {
    uint32_t i0, g0, ng, T;  // first node and first group (within the step), groups, threads per vector
    int64_t u0;              // first unit of the level
};
template <typename C>
__global__ void __launch_bounds__(TPB) memoA_run(DevAC ac, const MemoDesc *mdp, const uint32_t *nodes,
                                                  const MemoAGroup *grp, const MemoARunLevel *lv, int nlv) {
    pdl_begin();
    const MemoDesc md = *mdp;
    C *VA = static_cast<C *>(md.VA);
    for (int64_t vec = blockIdx.x; vec < md.V; vec += gridDim.x) {
        for (int l = 0; l < nlv; ++l) {
            const MemoARunLevel L = lv[l];
            for (uint32_t t = threadIdx.x; t < L.T; t += blockDim.x)
                memoA_slot<C>(ac, md, VA, nodes + L.i0, grp + L.g0, (int)L.ng, L.u0, vec, t);
            __syncthreads();
        }
    }
}

// Every step's tier A in one launch, when every step's slots are resident side by side: a block per
// (step, vector) walks all of the step's tier-A levels (each level's slots by the block's threads,
// then a barrier).  Tier A depends on the parameters alone, not on the sampled prefixes, and each
// step's levels form a chain of small dependent levels; so the steps run concurrently instead of one
// chain per step.  Pairs are taken in `order` (the steps with the most tier-A work first).
struct MemoAStep {
    int64_t node_base, grp_base;  // the step's first tier-A node and group
    uint32_t lv0, lv1;            // its tier-A levels in the level list
};
template <typename C>
__global__ void __launch_bounds__(TPB) memoA_all(DevAC ac, const MemoDesc *mdesc, const uint32_t *nodes,
                                                  const MemoAGroup *grp, const MemoARunLevel *lv,
                                                  const MemoAStep *steps, const int32_t *order, int nq, int64_t V) {
    pdl_begin();
    for (int64_t p = blockIdx.x; p < (int64_t)nq * V; p += gridDim.x) {
        const int j = order[p / V];
        const int64_t vec = p % V;
        const MemoDesc md = mdesc[j];
        C *VA = static_cast<C *>(md.VA);
        const MemoAStep st = steps[j];
        for (uint32_t l = st.lv0; l < st.lv1; ++l) {
            const MemoARunLevel L = lv[l];
            for (uint32_t t = threadIdx.x; t < L.T; t += blockDim.x)
                memoA_slot<C>(ac, md, VA, nodes + st.node_base + L.i0, grp + st.grp_base + L.g0, (int)L.ng, L.u0,
                              vec, t);
            __syncthreads();
        }
    }
}

// Every step's tier A at once when some tier-A level is too wide for memoA_all: a launch per level
// index covers that level in every step that has tier-A nodes there (levels in increasing order, so a
// slot's children are done), grid-striding over (step, vector, thread block) items like memoA_level.
// The steps' memo descriptors are staged in shared memory.  A step's levels then no longer wait on one
// another's launches step by step: D launches replace a launch per (step, tier-A item).
struct MemoALvlStep {
    int64_t node_off, grp_off, u0;  // the step's first tier-A node and group of the level, first unit
    uint32_t T, ng;                 // threads per vector, groups
    int32_t j, pad;                 // the step
};
constexpr int MEMO_LVL_STEPS = 64;  // steps per level (a memoised AC has at most 63 qubits)
template <typename C>
__global__ void __launch_bounds__(TPB, sizeof(C) == 8 ? 8 : 1) memoA_lvl_all(DevAC ac, const MemoDesc *mdesc,
                                                                            const uint32_t *nodes,
                                                                            const MemoAGroup *grp,
                                                                            const MemoALvlStep *ls, int nls) {
    pdl_begin();
    __shared__ MemoDesc smd[MEMO_LVL_STEPS];
    __shared__ int64_t pre[MEMO_LVL_STEPS + 1];  // block items before each step's
    for (int i = threadIdx.x; i < nls; i += blockDim.x) smd[i] = mdesc[ls[i].j];
    __syncthreads();
    const int64_t V = smd[0].V;
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (int i = 0; i < nls; ++i) pre[i + 1] = pre[i] + V * (int64_t)((ls[i].T + TPB - 1) / TPB);
    }
    __syncthreads();
    const int64_t items = pre[nls];
    int s = 0;
    for (int64_t b = blockIdx.x; b < items; b += gridDim.x) {
        while (pre[s + 1] <= b) ++s;  // items only grow along the loop
        const MemoALvlStep L = ls[s];
        const uint32_t nblk = (L.T + TPB - 1) / TPB;
        const int64_t r = b - pre[s];
        const int64_t vec = r / nblk;
        const uint32_t t = (uint32_t)(r - vec * nblk) * TPB + threadIdx.x;
        if (t < L.T)
            memoA_slot<C>(ac, smd[s], static_cast<C *>(smd[s].VA), nodes + L.node_off, grp + L.grp_off, (int)L.ng,
                          L.u0, vec, t);
    }
}

// The group-key table of one tile: for every group column and tabled support, the column's
// prefix bits on that support, packed (read by tier-B nodes for their tier-A children).  Only
// columns below the tile's group count are written.
__global__ void memo_keys(const PassDesc *pd, const MemoDesc *mdp) {
    pdl_begin();
    const int64_t ncols = desc_cols(*pd);
    const int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const MemoDesc md = *mdp;
    const int64_t g = pd->col0 + col;
    const uint64_t pre = md.j ? __brevll(pd->es.prefix[g] << (64 - md.j)) : 0ull;  // qubit order
    const bool narrow = md.j <= 32;
    for (int r = 0; r < md.nbm; ++r) md.keys[(int64_t)r * md.kpitch + col] = plan_key(md.bplan + r, pre, narrow);
}

// One level of tier B (FP32): as up_level_f32 over a node list, tier-A children read by key.
// The level's scale exponent in one column, from its child levels' scales and observed exponents
// (the rule of level_scale_kernel: child levels with no value in the column are skipped).  A memoised
// pass lists, per level, only the child levels that hold tier-B nodes in its step: the others are not
// computed there, so they have no value in any column.
__device__ __forceinline__ int level_scale_col(const uint32_t *cl_off, const uint16_t *cl, int L, int64_t pitch,
                                               int floor_zero, const int *S, const int *obs, int64_t c) {
    int s = INT_MIN;
    for (uint32_t k = __ldg(cl_off + L), k1 = __ldg(cl_off + L + 1); k < k1; ++k) {
        const int Lp = __ldg(cl + k);
        const int o = obs[(int64_t)Lp * pitch + c];
        if (o == OBS_EMPTY) continue;
        s = max(s, S[(int64_t)Lp * pitch + c] + o);
    }
    if (s == INT_MIN) s = 0;
    if (floor_zero && s < 0) s = 0;
    return s;
}

// What a tier-B kernel needs of the memo and pass descriptors, read once into registers (a reference
// into global memory would be re-read after every store, which the compiler cannot prove disjoint).
struct BView {
    const float4 *V4c;     // the lane's first column in row 0 of the value tile
    const int *Sc;         // ... in level 0 of the scale words
    const uint32_t *Kc;    // ... in row 0 of the group-key table
    const float2 *VA;      // tier-A slots
    const KeyPlan *kplan;  // key plans (untabled supports)
    const uint64_t *prefix;
    int64_t hp, pitch, kpitch, Vn, g0;
    uint32_t vec[4];       // the lane's four columns' vectors
    int j, nv;             // nv: the lane's columns inside the tile (1..4)
    bool narrow;
};

// One child of a tier-B node for a lane's four columns: values and scale exponents (for a tabled
// tier-A child, first its four keys).  Its edge record (uint4) says where the values live:
//   x bit 31 set: a tier-B child, x & 0x7fffffff = its row of the value tile, y = its level;
//   else a tier-A child: x = 1 + its key plan, y = key width | (1 + group-key table row, 0 if
//   the support is not tabled) << 8, (z, w) = its tier-A block offset in units (64 bits).
// A tier-A slot holds an unscaled value: exponent 0.
struct BChild {
    float4 a, b;  // columns 0-1 and 2-3: (re, im, re, im)
    int4 s;
};

// Issue the loads of one child's four column values (tier B) or keys (tier-A, tabled); an
// untabled tier-A child's keys are formed here from the group prefixes.  NC: tier-B rows and scale
// words through the read-only path (they were written by earlier launches); else plain loads (a run
// reads rows it wrote itself).
template <bool NC = true>
__device__ __forceinline__ void bchild_issue(const uint4 r, BChild &c, const BView &w) {
    if (r.x & 0x80000000u) {
        const float4 *row = w.V4c + (int64_t)(r.x & 0x7fffffffu) * w.hp;
        const int4 *sc = reinterpret_cast<const int4 *>(w.Sc + (int64_t)r.y * w.pitch);
        if (NC) {
            c.a = __ldg(row);
            c.b = __ldg(row + 1);
            c.s = __ldg(sc);
        } else {
            c.a = row[0];
            c.b = row[1];
            c.s = *sc;
        }
    } else {
        const int mid = (int)(r.y >> 8) - 1;
        if (mid >= 0) {  // tabled: the four columns' keys (col is a multiple of 4, so is the pitch)
            const uint4 kk = *reinterpret_cast<const uint4 *>(w.Kc + (int64_t)mid * w.kpitch);
            // no key is stored past the tile's last column: those columns reuse the first one's
            c.s = make_int4((int)kk.x, (int)(w.nv > 1 ? kk.y : kk.x), (int)(w.nv > 2 ? kk.z : kk.x),
                            (int)(w.nv > 3 ? kk.w : kk.x));
        } else {  // the group prefixes in qubit order (bit q = x_q), compressed to the child's support
            const KeyPlan *kp = w.kplan + (r.x - 1u);
            int k[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t g = w.g0 + (i < w.nv ? i : 0);
                const uint64_t pre = w.j ? __brevll(w.prefix[g] << (64 - w.j)) : 0ull;
                k[i] = (int)plan_key(kp, pre, w.narrow);
            }
            c.s = make_int4(k[0], k[1], k[2], k[3]);
        }
    }
}
// Second stage for a tier-A child: its four slots, read by key.
__device__ __forceinline__ void bchild_slots(const uint4 r, BChild &c, const BView &w) {
    if (r.x & 0x80000000u) return;
    const int kc = (int)(r.y & 0xffu);
    const float2 *blk = w.VA + w.Vn * (int64_t)(((uint64_t)r.w << 32) | r.z);
    const float2 v0 = blk[((uint64_t)w.vec[0] << kc) | (uint32_t)c.s.x];
    const float2 v1 = blk[((uint64_t)w.vec[1] << kc) | (uint32_t)c.s.y];
    const float2 v2 = blk[((uint64_t)w.vec[2] << kc) | (uint32_t)c.s.z];
    const float2 v3 = blk[((uint64_t)w.vec[3] << kc) | (uint32_t)c.s.w];
    c.a = make_float4(v0.x, v0.y, v1.x, v1.y);
    c.b = make_float4(v2.x, v2.y, v3.x, v3.y);
    c.s = make_int4(0, 0, 0, 0);
}

__device__ __forceinline__ float2 mul_scaled(float ax, float ay, float bx, float by, int e) {
    return cscale(cmul(make_float2(ax, ay), make_float2(bx, by)), pow2f(e));
}

// The per-launch part of a tier-B kernel's view of its descriptors.
__device__ __forceinline__ void bview_init(BView &w, const PassDesc *pd, const MemoDesc *mdp, int64_t pitch) {
    w.VA = static_cast<const float2 *>(mdp->VA);
    w.kplan = mdp->kplan;
    w.prefix = pd->es.prefix;
    w.hp = pitch >> 1;
    w.pitch = pitch;
    w.kpitch = mdp->kpitch;
    w.Vn = mdp->V;
    w.j = mdp->j;
    w.narrow = w.j <= 32;
}
// The per-column part: the lane's four columns starting at tile column col (col < ncols).
__device__ __forceinline__ void bview_cols(BView &w, int64_t col, int64_t ncols, int64_t col0, const int32_t *col_vec,
                                           int64_t n_vec, const float4 *V4, const int *S, const uint32_t *keys) {
    w.nv = (int)min((int64_t)4, ncols - col);
    w.g0 = col0 + col;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t g = w.g0 + (i < w.nv ? i : 0);
        int64_t v = col_vec ? (int64_t)col_vec[g] : g;
        v = v < 0 ? 0 : (v >= n_vec ? n_vec - 1 : v);
        w.vec[i] = (uint32_t)v;
    }
    w.V4c = V4 + (col >> 1);
    w.Sc = S + col;
    w.Kc = keys + col;
}
// Stage a node block's descriptors (first edge record, degree | op << 24) and first two edge records
// in the warp's shared arrays (lane i: node i).
__device__ __forceinline__ void bstage(uint2 *sd, uint4 (*sr)[2], const uint2 *bdesc, const uint4 *brec, int nn,
                                       int lane) {
    __syncwarp();
    if (lane < nn) {
        const uint2 d = __ldg(bdesc + lane);
        const uint32_t deg = d.y & 0xffffffu;
        sd[lane] = d;
        const uint4 r0 = __ldg(brec + d.x);
        sr[lane][0] = r0;
        sr[lane][1] = deg >= 2u ? __ldg(brec + d.x + 1) : r0;  // a node's own records only
    }
    __syncwarp();
}
// The staged nodes 0 .. nn-1 for the lane's four columns: per node, both children's loads are issued
// (tile rows and scale words, or group keys), then the tier-A slots by key, and only then is the node
// combined and stored at dst[i * hp]; mx tracks each column's largest stored magnitude.
template <bool NC = true>
__device__ __forceinline__ void bnodes(const uint2 *sd, const uint4 (*sr)[2], int nn, const int sl[4], float4 *dst,
                                       const BView &w, const uint4 *brec, float mx[4]) {
    for (int i = 0; i < nn; ++i) {
        const uint2 dsc = sd[i];
        const uint32_t deg = dsc.y & 0xffffffu, o = dsc.y >> 24;
        const uint4 r0 = sr[i][0], r1 = sr[i][1];
        BChild x, y;
        bchild_issue<NC>(r0, x, w);
        if (deg >= 2u) bchild_issue<NC>(r1, y, w);
        bchild_slots(r0, x, w);
        if (deg >= 2u) bchild_slots(r1, y, w);
        float2 q[4];
        if (o == OP_MUL) {
            q[0] = mul_scaled(x.a.x, x.a.y, y.a.x, y.a.y, x.s.x + y.s.x - sl[0]);
            q[1] = mul_scaled(x.a.z, x.a.w, y.a.z, y.a.w, x.s.y + y.s.y - sl[1]);
            q[2] = mul_scaled(x.b.x, x.b.y, y.b.x, y.b.y, x.s.z + y.s.z - sl[2]);
            q[3] = mul_scaled(x.b.z, x.b.w, y.b.z, y.b.w, x.s.w + y.s.w - sl[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = make_float2(0.f, 0.f);
            auto add = [&](const BChild &c) {
                const float f0 = pow2f(c.s.x - sl[0]), f1 = pow2f(c.s.y - sl[1]);
                const float f2 = pow2f(c.s.z - sl[2]), f3 = pow2f(c.s.w - sl[3]);
                q[0].x += c.a.x * f0; q[0].y += c.a.y * f0;
                q[1].x += c.a.z * f1; q[1].y += c.a.w * f1;
                q[2].x += c.b.x * f2; q[2].y += c.b.y * f2;
                q[3].x += c.b.z * f3; q[3].y += c.b.w * f3;
            };
            add(x);
            if (deg >= 2u) add(y);
            for (uint32_t e = 2; e < deg; ++e) {  // children beyond the second: one at a time
                const uint4 r = __ldg(brec + dsc.x + e);
                BChild z;
                bchild_issue<NC>(r, z, w);
                bchild_slots(r, z, w);
                add(z);
            }
        }
        float4 *d = dst + (int64_t)i * w.hp;
        d[0] = make_float4(q[0].x, q[0].y, q[1].x, q[1].y);
        d[1] = make_float4(q[2].x, q[2].y, q[3].x, q[3].y);
#pragma unroll
        for (int k = 0; k < 4; ++k) mx[k] = fmaxf(mx[k], fmaxf(fabsf(q[k].x), fabsf(q[k].y)));
    }
}
// The level's scale exponent for the lane's columns: formed from its child levels (floor: the level
// reads unscaled tier-A values) or read from S.
__device__ __forceinline__ void blevel_scale(const MemoDesc *mdp, int L, int64_t pitch, bool inline_scale, int floor_zero,
                                             const int *S, const int *obs, int64_t col, int nv, int sl[4]) {
    if (inline_scale) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            sl[i] = i < nv ? level_scale_col(mdp->bcl_off, mdp->bcl, L, pitch, floor_zero, S, obs, col + i) : 0;
    } else {
        const int4 t4 = *reinterpret_cast<const int4 *>(S + (int64_t)L * pitch + col);
        sl[0] = t4.x; sl[1] = t4.y; sl[2] = t4.z; sl[3] = t4.w;
    }
}
__device__ __forceinline__ void bstore_scale(int *S, int L, int64_t pitch, int64_t col, int nv, const int sl[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (i < nv) S[(int64_t)L * pitch + col + i] = sl[i];
}
__device__ __forceinline__ void bobserve(int *obs, int L, int64_t pitch, int64_t col, int nv, const float mx[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < nv) atomicMax(obs + (int64_t)L * pitch + col + k, (__float_as_int(mx[k]) >> 23) - 127);
}

// One level of tier B (FP32): as up_level_f32 over a node list, tier-A children read by key.
// A warp item is 32 tier-B nodes x 128 columns, four consecutive columns per lane (two float4
// per child row: a 1 KB segment per warp).  The item's node descriptors and first two edge
// records are staged in shared memory by one coalesced load; then, per node, the loads of both
// children are issued (tile rows and scale words, or group keys), then the tier-A slots by key,
// and only then is the node combined and stored.  Four columns per lane spread the per-node work
// (records, decoding, addresses) over twice the bytes of a two-column lane.  The arithmetic (and
// its order) is that of up_level_f32, so values equal the per-group sampler's bit for bit.  The
// level's largest exponent per column is tracked as the largest magnitude (the exponent is
// monotonic in it) and taken once per item.
// a.hi bit 0: the level reads unscaled tier-A values (its scale is at least 0); bit 1: this kernel
// forms the level's scale itself (the items of the level's first node block write it).
__global__ void __launch_bounds__(TPB, 3) memoB_level_f32(DevAC ac, LevelArgs a, const uint2 *bdesc, int64_t count,
                                                        const PassDesc *pd,
                                                        const MemoDesc *mdp, float2 *__restrict__ V,
                                                        int *__restrict__ S, int *__restrict__ obs) {
    pdl_begin();
    __shared__ uint2 sdesc[TPB / 32][NBB];
    __shared__ uint4 srec[TPB / 32][NBB][2];
    const int64_t ncols = desc_cols(*pd);
    if (ncols <= 0 || count <= 0) return;
    const uint4 *brec = mdp->brec;
    const int64_t col0 = pd->col0;
    const int32_t *col_vec = pd->es.col_vec;
    const int64_t n_vec = pd->es.n_vec;
    const uint32_t *keys = mdp->keys;
    BView w;
    bview_init(w, pd, mdp, a.pitch);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    // Work items (node block of 32, 128-column chunk), node-block major, dealt round-robin over the
    // warps: at any time the warps share a node block, so its tier-A children stay in L2.  Whole
    // rounds take whole items; the items left (fewer than a round) are cut into 2^sub_log2 parts of
    // 32 >> sub_log2 nodes, so that the last round is not a few warps doing whole items.
    const uint32_t nchunks = (uint32_t)((ncols + 127) >> 7);
    const uint32_t cnt = (uint32_t)count;
    const uint32_t nblk = (cnt + NBB - 1) / NBB;
    const uint32_t items = nblk * nchunks;  // < 2^32 (the level's rows of the tile would exceed 4 TB)
    const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t full = items / nw * nw, rem = items - full;
    float4 *V4 = reinterpret_cast<float4 *>(V);
    // one item: nodes n0 .. n0 + nn - 1 of the level in chunk `chunk`
    auto item = [&](uint32_t n0, int nn, uint32_t chunk) {
        const int64_t col = (int64_t)chunk * 128 + lane * 4;
        bstage(sdesc[wp], srec[wp], bdesc + n0, brec, nn, lane);
        if (col >= ncols) return;
        bview_cols(w, col, ncols, col0, col_vec, n_vec, V4, S, keys);
        int sl[4];
        blevel_scale(mdp, a.L, a.pitch, (a.hi & 2u) != 0, (int)(a.hi & 1u), S, obs, col, w.nv, sl);
        if ((a.hi & 2u) && n0 == 0) bstore_scale(S, a.L, a.pitch, col, w.nv, sl);
        float mx[4] = {0.f, 0.f, 0.f, 0.f};
        bnodes(sdesc[wp], srec[wp], nn, sl, V4 + (int64_t)(a.lo + n0) * w.hp + (col >> 1), w, brec, mx);
        bobserve(obs, a.L, a.pitch, col, w.nv, mx);
    };
    {  // whole rounds: item = node block * nchunks + chunk, stepped by the warp count without division
        uint32_t blk = wid / nchunks, chunk = wid % nchunks;
        const uint32_t dq = nw / nchunks, dr = nw % nchunks;
        for (uint32_t it = wid; it < full; it += nw) {
            const uint32_t b = blk, c = chunk;
            chunk += dr;
            blk += dq;
            if (chunk >= nchunks) {
                chunk -= nchunks;
                ++blk;
            }
            item(b * NBB, (int)min((uint32_t)NBB, cnt - b * NBB), c);
        }
    }
    if (rem == 0) return;
    // the last, partial round in parts: the part size that needs the fewest node-times, at about
    // three per item of overhead
    uint32_t sub_log2 = 0, best = 0xffffffffu;
    for (uint32_t sl = 0; sl <= 3; ++sl) {
        const uint32_t cost = (((rem << sl) + nw - 1) / nw) * ((uint32_t)(NBB >> sl) + 3u);
        if (cost < best) best = cost, sub_log2 = sl;
    }
    const uint32_t nsub = rem << sub_log2;
    for (uint32_t t = wid; t < nsub; t += nw) {
        const uint32_t it = full + (t >> sub_log2);
        const uint32_t blk = it / nchunks, chunk = it - blk * nchunks;
        const uint32_t n0 = blk * NBB + ((t & ((1u << sub_log2) - 1u)) << (5 - sub_log2));
        if (n0 >= cnt) continue;  // an empty part of the level's last node block (warp-uniform)
        item(n0, (int)min((uint32_t)NBB >> sub_log2, cnt - n0), chunk);
    }
}

// A run of consecutive small tier-B levels in one launch: a warp per 64-column chunk (two columns per
// lane) walks the levels in order, every node of each level for its own columns.  A level reads only
// lower levels of the same columns, and each lane reads back only what it wrote itself (tile rows,
// scale words, observed exponents of its columns), so no barrier is needed -- and a step whose tier B
// is a chain of small levels costs one launch instead of one per level (and no scale launches).  The
// nodes of a level are taken two at a time: the loads of both nodes' children are issued before
// either is combined, so a lane has four child rows in flight.  The arithmetic (and its order) is
// that of up_level_f32.  Each lane owns its columns, so the levels' observed exponents are stored,
// not reduced.
struct MemoBRunLevel {
    uint32_t b0, count;  // first tier-B row of the level within the step, its tier-B nodes
    int32_t L, floor0;   // level, whether it reads unscaled tier-A values
};
// A run lane's view: its two columns.
struct RView {
    float4 *V4c;           // the lane's columns in row 0 of the value tile
    const int *Sc;         // ... in level 0 of the scale words
    const uint32_t *Kc;    // ... in row 0 of the group-key table
    const float2 *VA;      // tier-A slots
    const KeyPlan *kplan;  // key plans (untabled supports)
    const uint64_t *pre;   // the group prefixes, at the lane's first column
    uint32_t hp, pitch, kpitch, Vn;
    uint32_t vec0, vec1;   // the columns' vectors
    int j;
    bool narrow, two;      // two: the second column is inside the tile
};
// One child of a run-level node for the lane's two columns (the edge record as for BChild).
struct RChild {
    float4 v;  // (re, im) of column 0, then of column 1
    int2 s;    // scale exponents; for a tier-A child, first its keys
};
// An untabled tier-A child's keys in the lane's two columns: the group prefixes in qubit order
// (bit q = x_q), compressed to the child's support (rare: out of line).
__device__ __noinline__ int2 rkeys_untabled(const KeyPlan *kp, const uint64_t *pre, int j, bool two, bool narrow) {
    const uint64_t p0 = j ? __brevll(pre[0] << (64 - j)) : 0ull;
    const uint64_t p1 = j ? __brevll(pre[two ? 1 : 0] << (64 - j)) : 0ull;
    return make_int2((int)plan_key(kp, p0, narrow), (int)plan_key(kp, p1, narrow));
}
__device__ __forceinline__ void rchild_issue(const uint4 r, RChild &c, const RView &w) {
    if (r.x & 0x80000000u) {  // rows written by this launch or earlier ones: plain loads
        c.v = w.V4c[(int64_t)(r.x & 0x7fffffffu) * w.hp];
        c.s = *reinterpret_cast<const int2 *>(w.Sc + (int64_t)r.y * w.pitch);
    } else {
        const int mid = (int)(r.y >> 8) - 1;
        if (mid >= 0) {  // no key is stored past the tile's last column: that column reuses the first one's
            const uint2 kk = *reinterpret_cast<const uint2 *>(w.Kc + (int64_t)mid * w.kpitch);
            c.s = make_int2((int)kk.x, (int)(w.two ? kk.y : kk.x));
        } else {
            c.s = rkeys_untabled(w.kplan + (r.x - 1u), w.pre, w.j, w.two, w.narrow);
        }
    }
}
__device__ __forceinline__ void rchild_slots(const uint4 r, RChild &c, const RView &w) {
    if (r.x & 0x80000000u) return;
    const int kc = (int)(r.y & 0xffu);
    const float2 *blk = w.VA + w.Vn * (int64_t)(((uint64_t)r.w << 32) | r.z);
    const float2 v0 = blk[((uint64_t)w.vec0 << kc) | (uint32_t)c.s.x];
    const float2 v1 = blk[((uint64_t)w.vec1 << kc) | (uint32_t)c.s.y];
    c.v = make_float4(v0.x, v0.y, v1.x, v1.y);
    c.s = make_int2(0, 0);
}
// A node's value in the lane's two columns from its loaded children x (and y: degree >= 2); children
// beyond the second are loaded here, one at a time (X: the node may have more than two).
template <bool X>
__device__ __forceinline__ float4 rcombine(uint2 dsc, const RChild &x, const RChild &y, int sl0, int sl1,
                                           const uint4 *brec, const RView &w) {
    const uint32_t deg = dsc.y & 0xffffffu, o = dsc.y >> 24;
    float2 q0, q1;
    if (o == OP_MUL) {
        q0 = mul_scaled(x.v.x, x.v.y, y.v.x, y.v.y, x.s.x + y.s.x - sl0);
        q1 = mul_scaled(x.v.z, x.v.w, y.v.z, y.v.w, x.s.y + y.s.y - sl1);
    } else {
        float f0 = pow2f(x.s.x - sl0), f1 = pow2f(x.s.y - sl1);
        q0 = make_float2(x.v.x * f0, x.v.y * f0);
        q1 = make_float2(x.v.z * f1, x.v.w * f1);
        if (deg >= 2u) {
            f0 = pow2f(y.s.x - sl0);
            f1 = pow2f(y.s.y - sl1);
            q0.x += y.v.x * f0; q0.y += y.v.y * f0;
            q1.x += y.v.z * f1; q1.y += y.v.w * f1;
        }
        for (uint32_t e = 2; X && e < deg; ++e) {  // children beyond the second
            const uint4 r = __ldg(brec + dsc.x + e);
            RChild z;
            rchild_issue(r, z, w);
            rchild_slots(r, z, w);
            f0 = pow2f(z.s.x - sl0);
            f1 = pow2f(z.s.y - sl1);
            q0.x += z.v.x * f0; q0.y += z.v.y * f0;
            q1.x += z.v.z * f1; q1.y += z.v.w * f1;
        }
    }
    return make_float4(q0.x, q0.y, q1.x, q1.y);
}
// fuse bit 0: the run is the step's first tier-B launch and forms the tile's group keys itself (what
// memo_keys does, for the lane's columns); bit 1: the run holds the step's root (tier-B row rrow on
// level Lroot) and writes each column's root value (what memo_root does).
// The block stages the whole run's node descriptors and first two edge records in shared memory once
// (dynamic shared memory: 40 bytes per node), and each warp keeps, per run level and column, the level's
// scale plus observed exponent there, so a level's scale reads global memory only for child levels
// outside the run: a level then costs its nodes' child loads alone.
__global__ void __launch_bounds__(TPB, 4) memoB_run_f32(const MemoBRunLevel *lv, int nlv, const uint2 *bdesc,
                                                      const PassDesc *pd, const MemoDesc *mdp, int64_t pitch,
                                                      float2 *__restrict__ V, int *__restrict__ S,
                                                      int *__restrict__ obs, int fuse, int64_t rrow, int Lroot,
                                                      double2 *__restrict__ out) {
    pdl_begin();
    extern __shared__ uint4 run_smem[];
    __shared__ MemoBRunLevel slv[MEMO_RUN_LV];
    const int64_t ncols = desc_cols(*pd);
    if (ncols <= 0 || ((ncols + 63) >> 6) <= (int64_t)gridDim.x) return;  // few chunks: memoB_runc_f32
    const uint4 *brec = mdp->brec;
    // the run's rows are consecutive: [base, base + ntot)
    const uint32_t base = lv[0].b0, ntot = lv[nlv - 1].b0 + lv[nlv - 1].count - base;
    uint4 *srec = run_smem;                                              // [ntot][2]
    uint2 *sdesc = reinterpret_cast<uint2 *>(srec + 2 * (size_t)ntot);  // [ntot]
    int *se = reinterpret_cast<int *>(sdesc + ntot);                     // [nlv][warps][64]
    for (uint32_t i = threadIdx.x; i < ntot; i += blockDim.x) {
        const uint2 d = __ldg(bdesc + base + i);
        const uint4 r0 = __ldg(brec + d.x);
        sdesc[i] = d;
        srec[2 * i] = r0;
        srec[2 * i + 1] = (d.y & 0xffffffu) >= 2u ? __ldg(brec + d.x + 1) : r0;
    }
    if (threadIdx.x < nlv) slv[threadIdx.x] = lv[threadIdx.x];
    __syncthreads();
    const int64_t col0 = pd->col0;
    const int32_t *col_vec = pd->es.col_vec;
    const int64_t n_vec = pd->es.n_vec;
    const uint64_t *prefix = pd->es.prefix;
    const uint32_t *cl_off = mdp->bcl_off;
    const uint16_t *cl = mdp->bcl;
    const int j = mdp->j;
    RView w;
    w.VA = static_cast<const float2 *>(mdp->VA);
    w.kplan = mdp->kplan;
    w.hp = (uint32_t)(pitch >> 1);
    w.pitch = (uint32_t)pitch;
    w.kpitch = (uint32_t)mdp->kpitch;
    w.Vn = (uint32_t)mdp->V;
    w.j = j;
    w.narrow = j <= 32;
    uint32_t *keys = mdp->keys;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t nchunks = (ncols + 63) >> 6;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float4 *V4 = reinterpret_cast<float4 *>(V);
    int2 *se_w = reinterpret_cast<int2 *>(se) + (size_t)wp * 32 + lane;  // level l at se_w[l * warps * 32]
    const int se_step = (TPB / 32) * 32;
    if (fuse & 1) {  // the group keys of the lane's columns (the same chunks as below), per tabled support
        const KeyPlan *bplan = mdp->bplan;
        const int nbm = mdp->nbm;
        const bool narrow = j <= 32;
        for (int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; chunk < nchunks; chunk += nw) {
            const int64_t col = chunk * 64 + lane * 2;
            if (col >= ncols) continue;
            const bool two = col + 1 < ncols;
            const uint64_t p0 = j ? __brevll(prefix[col0 + col] << (64 - j)) : 0ull;
            const uint64_t p1 = two && j ? __brevll(prefix[col0 + col + 1] << (64 - j)) : 0ull;
            for (int r = 0; r < nbm; ++r) {
                uint32_t *kr = keys + (int64_t)r * mdp->kpitch + col;
                kr[0] = plan_key(bplan + r, p0, narrow);
                if (two) kr[1] = plan_key(bplan + r, p1, narrow);
            }
        }
    }
    for (int64_t chunk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; chunk < nchunks; chunk += nw) {
        const int64_t col = chunk * 64 + lane * 2;  // even, and the pitch is a multiple of 64
        if (col >= ncols) continue;  // the lane has no column (no barrier follows)
        w.two = col + 1 < ncols;
        const int64_t g0 = col0 + col, g1 = w.two ? g0 + 1 : g0;
        int64_t v0 = col_vec ? (int64_t)col_vec[g0] : g0, v1 = col_vec ? (int64_t)col_vec[g1] : g1;
        v0 = v0 < 0 ? 0 : (v0 >= n_vec ? n_vec - 1 : v0);
        v1 = v1 < 0 ? 0 : (v1 >= n_vec ? n_vec - 1 : v1);
        w.vec0 = (uint32_t)v0;
        w.vec1 = (uint32_t)v1;
        w.pre = prefix + g0;
        w.V4c = V4 + (col >> 1);
        w.Sc = S + col;
        w.Kc = keys + col;
        for (int l = 0; l < nlv; ++l) {
            const MemoBRunLevel L = slv[l];
            // the level's scale (the rule of level_scale_col): child levels of this run from shared
            // memory, the others from their scale and observed-exponent words
            int s0 = INT_MIN, s1 = INT_MIN;
            for (uint32_t k = __ldg(cl_off + L.L), k1 = __ldg(cl_off + L.L + 1); k < k1; ++k) {
                const int Lp = __ldg(cl + k);
                int r = l - 1;
                while (r >= 0 && slv[r].L != Lp) --r;
                if (r >= 0) {
                    const int2 e = se_w[r * se_step];
                    s0 = max(s0, e.x);
                    s1 = max(s1, e.y);
                } else {
                    const int2 o = *reinterpret_cast<const int2 *>(obs + (int64_t)Lp * pitch + col);
                    const int2 sc = *reinterpret_cast<const int2 *>(S + (int64_t)Lp * pitch + col);
                    if (o.x != OBS_EMPTY) s0 = max(s0, sc.x + o.x);
                    if (o.y != OBS_EMPTY) s1 = max(s1, sc.y + o.y);
                }
            }
            if (s0 == INT_MIN) s0 = 0;
            if (s1 == INT_MIN) s1 = 0;
            if (L.floor0) {
                s0 = max(s0, 0);
                s1 = max(s1, 0);
            }
            if (!w.two) s1 = 0;
            const int sl0 = s0, sl1 = s1;
            float mx0 = 0.f, mx1 = 0.f;
            const uint32_t r0 = L.b0 - base;
            float4 *dst = w.V4c + (int64_t)L.b0 * w.hp;
            const int nn = (int)L.count;
            for (int i = 0; i < nn;) {  // two nodes at a time where both have at most two children
                const uint2 d0 = sdesc[r0 + i];
                const uint2 d1 = sdesc[r0 + (i + 1 < nn ? i + 1 : i)];
                const uint32_t deg0 = d0.y & 0xffffffu, deg1 = d1.y & 0xffffffu;
                const uint4 *q0r = srec + 2 * (size_t)(r0 + i);
                RChild x0, y0;
                y0.v = make_float4(0.f, 0.f, 0.f, 0.f);
                y0.s = make_int2(0, 0);
                if (i + 1 < nn && deg0 <= 2u && deg1 <= 2u) {
                    const uint4 *q1r = q0r + 2;
                    RChild x1, y1;
                    y1.v = make_float4(0.f, 0.f, 0.f, 0.f);
                    y1.s = make_int2(0, 0);
                    rchild_issue(q0r[0], x0, w);
                    if (deg0 == 2u) rchild_issue(q0r[1], y0, w);
                    rchild_issue(q1r[0], x1, w);
                    if (deg1 == 2u) rchild_issue(q1r[1], y1, w);
                    rchild_slots(q0r[0], x0, w);
                    if (deg0 == 2u) rchild_slots(q0r[1], y0, w);
                    rchild_slots(q1r[0], x1, w);
                    if (deg1 == 2u) rchild_slots(q1r[1], y1, w);
                    const float4 q = rcombine<false>(d0, x0, y0, sl0, sl1, brec, w);
                    const float4 p = rcombine<false>(d1, x1, y1, sl0, sl1, brec, w);
                    dst[(int64_t)i * w.hp] = q;
                    dst[(int64_t)(i + 1) * w.hp] = p;
                    mx0 = fmaxf(mx0, fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fmaxf(fabsf(p.x), fabsf(p.y))));
                    mx1 = fmaxf(mx1, fmaxf(fmaxf(fabsf(q.z), fabsf(q.w)), fmaxf(fabsf(p.z), fabsf(p.w))));
                    i += 2;
                } else {
                    rchild_issue(q0r[0], x0, w);
                    if (deg0 >= 2u) rchild_issue(q0r[1], y0, w);
                    rchild_slots(q0r[0], x0, w);
                    if (deg0 >= 2u) rchild_slots(q0r[1], y0, w);
                    const float4 q = rcombine<true>(d0, x0, y0, sl0, sl1, brec, w);
                    dst[(int64_t)i * w.hp] = q;
                    mx0 = fmaxf(mx0, fmaxf(fabsf(q.x), fabsf(q.y)));
                    mx1 = fmaxf(mx1, fmaxf(fabsf(q.z), fabsf(q.w)));
                    i += 1;
                }
            }
            int *sw = S + (int64_t)L.L * pitch + col, *ow = obs + (int64_t)L.L * pitch + col;
            const int e0 = (__float_as_int(mx0) >> 23) - 127, e1 = (__float_as_int(mx1) >> 23) - 127;
            se_w[l * se_step] = make_int2(sl0 + e0, sl1 + e1);
            if (w.two) {
                *reinterpret_cast<int2 *>(sw) = make_int2(sl0, sl1);
                *reinterpret_cast<int2 *>(ow) = make_int2(e0, e1);
            } else {
                sw[0] = sl0;
                ow[0] = e0;
            }
        }
        if (fuse & 2) {  // the root's value in the lane's columns, unscaled to FP64
            const float4 q = w.V4c[rrow * (int64_t)w.hp];
            const int *sr = S + (int64_t)Lroot * pitch + col;
            const int64_t gc = col0 + col;
            out[gc] = make_double2(ldexp((double)q.x, sr[0]), ldexp((double)q.y, sr[0]));
            if (w.two) out[gc + 1] = make_double2(ldexp((double)q.z, sr[1]), ldexp((double)q.w, sr[1]));
        }
    }
}
// The same run when the tile has no more 64-column chunks than the launch has blocks (the early sampling
// steps, a few groups per vector): a block per chunk, its 8 warps sharing the chunk's columns (two per
// lane, as above) and splitting each level's nodes (warp w: nodes w, w + 8, ...), with a block barrier
// between levels; a level's observed exponent is the largest over the warps, reduced in shared memory.
// The chain of levels then costs a level's nodes divided by 8 instead of by 1, with the same arithmetic
// (every warp forms the same scales), so values equal memoB_run_f32's bit for bit.  Launched beside
// memoB_run_f32 with the same grid; exactly one of the two has work.
__global__ void __launch_bounds__(TPB, 4) memoB_runc_f32(const MemoBRunLevel *lv, int nlv, const uint2 *bdesc,
                                                       const PassDesc *pd, const MemoDesc *mdp, int64_t pitch,
                                                       float2 *__restrict__ V, int *__restrict__ S,
                                                       int *__restrict__ obs, int fuse, int64_t rrow, int Lroot,
                                                       double2 *__restrict__ out) {
    pdl_begin();
    extern __shared__ uint4 run_smem[];
    __shared__ MemoBRunLevel slv[MEMO_RUN_LV];
    __shared__ float2 smx[2][TPB / 32][32];  // per level parity, warp and lane: the warp's largest magnitudes
    const int64_t ncols = desc_cols(*pd);
    const int64_t nchunks = (ncols + 63) >> 6;
    if (ncols <= 0 || nchunks > (int64_t)gridDim.x) return;  // many chunks: memoB_run_f32
    const uint4 *brec = mdp->brec;
    const uint32_t base = lv[0].b0, ntot = lv[nlv - 1].b0 + lv[nlv - 1].count - base;
    uint4 *srec = run_smem;
    uint2 *sdesc = reinterpret_cast<uint2 *>(srec + 2 * (size_t)ntot);
    int *se = reinterpret_cast<int *>(sdesc + ntot);
    for (uint32_t i = threadIdx.x; i < ntot; i += blockDim.x) {
        const uint2 d = __ldg(bdesc + base + i);
        const uint4 r0 = __ldg(brec + d.x);
        sdesc[i] = d;
        srec[2 * i] = r0;
        srec[2 * i + 1] = (d.y & 0xffffffu) >= 2u ? __ldg(brec + d.x + 1) : r0;
    }
    if (threadIdx.x < nlv) slv[threadIdx.x] = lv[threadIdx.x];
    __syncthreads();
    const int64_t col0 = pd->col0;
    const int32_t *col_vec = pd->es.col_vec;
    const int64_t n_vec = pd->es.n_vec;
    const uint64_t *prefix = pd->es.prefix;
    const uint32_t *cl_off = mdp->bcl_off;
    const uint16_t *cl = mdp->bcl;
    const int j = mdp->j;
    RView w;
    w.VA = static_cast<const float2 *>(mdp->VA);
    w.kplan = mdp->kplan;
    w.hp = (uint32_t)(pitch >> 1);
    w.pitch = (uint32_t)pitch;
    w.kpitch = (uint32_t)mdp->kpitch;
    w.Vn = (uint32_t)mdp->V;
    w.j = j;
    w.narrow = j <= 32;
    uint32_t *keys = mdp->keys;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nwarp = TPB / 32;
    float4 *V4 = reinterpret_cast<float4 *>(V);
    int2 *se_w = reinterpret_cast<int2 *>(se) + (size_t)wp * 32 + lane;
    const int se_step = nwarp * 32;
    for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {  // one chunk a block
        const int64_t col = chunk * 64 + lane * 2;
        const bool active = col < ncols;
        w.two = col + 1 < ncols;
        const int64_t g0 = col0 + (active ? col : 0), g1 = w.two ? g0 + 1 : g0;
        if (fuse & 1) {  // the chunk's group keys: the warps split the tabled supports
            const KeyPlan *bplan = mdp->bplan;
            const uint64_t p0 = j ? __brevll(prefix[g0] << (64 - j)) : 0ull;
            const uint64_t p1 = j ? __brevll(prefix[g1] << (64 - j)) : 0ull;
            for (int r = wp, nbm = mdp->nbm; r < nbm && active; r += nwarp) {
                uint32_t *kr = keys + (int64_t)r * mdp->kpitch + col;
                kr[0] = plan_key(bplan + r, p0, w.narrow);
                if (w.two) kr[1] = plan_key(bplan + r, p1, w.narrow);
            }
            __syncthreads();
        }
        int64_t v0 = col_vec ? (int64_t)col_vec[g0] : g0, v1 = col_vec ? (int64_t)col_vec[g1] : g1;
        v0 = v0 < 0 ? 0 : (v0 >= n_vec ? n_vec - 1 : v0);
        v1 = v1 < 0 ? 0 : (v1 >= n_vec ? n_vec - 1 : v1);
        w.vec0 = (uint32_t)v0;
        w.vec1 = (uint32_t)v1;
        w.pre = prefix + g0;
        w.V4c = V4 + ((active ? col : 0) >> 1);
        w.Sc = S + (active ? col : 0);
        w.Kc = keys + (active ? col : 0);
        for (int l = 0; l < nlv; ++l) {
            const MemoBRunLevel L = slv[l];
            int s0 = INT_MIN, s1 = INT_MIN;
            if (active) {
                for (uint32_t k = __ldg(cl_off + L.L), k1 = __ldg(cl_off + L.L + 1); k < k1; ++k) {
                    const int Lp = __ldg(cl + k);
                    int r = l - 1;
                    while (r >= 0 && slv[r].L != Lp) --r;
                    if (r >= 0) {
                        const int2 e = se_w[r * se_step];
                        s0 = max(s0, e.x);
                        s1 = max(s1, e.y);
                    } else {
                        const int2 o = *reinterpret_cast<const int2 *>(obs + (int64_t)Lp * pitch + col);
                        const int2 sc = *reinterpret_cast<const int2 *>(S + (int64_t)Lp * pitch + col);
                        if (o.x != OBS_EMPTY) s0 = max(s0, sc.x + o.x);
                        if (o.y != OBS_EMPTY) s1 = max(s1, sc.y + o.y);
                    }
                }
            }
            if (s0 == INT_MIN) s0 = 0;
            if (s1 == INT_MIN) s1 = 0;
            if (L.floor0) {
                s0 = max(s0, 0);
                s1 = max(s1, 0);
            }
            if (!w.two) s1 = 0;
            const int sl0 = s0, sl1 = s1;
            int *sw = S + (int64_t)L.L * pitch + (active ? col : 0), *ow = obs + (int64_t)L.L * pitch + (active ? col : 0);
            if (wp == 0 && active) {  // the level's scale, read by the next levels' warps after the barrier
                if (w.two) *reinterpret_cast<int2 *>(sw) = make_int2(sl0, sl1);
                else sw[0] = sl0;
            }
            float mx0 = 0.f, mx1 = 0.f;
            const uint32_t r0 = L.b0 - base;
            float4 *dst = w.V4c + (int64_t)L.b0 * w.hp;
            const int nn = (int)L.count;
            for (int i = wp; i < nn && active;) {  // this warp's nodes: i, i + 8, ...; two at a time
                const int i1 = i + nwarp;
                const uint2 d0 = sdesc[r0 + i];
                const uint2 d1 = sdesc[r0 + (i1 < nn ? i1 : i)];
                const uint32_t deg0 = d0.y & 0xffffffu, deg1 = d1.y & 0xffffffu;
                const uint4 *q0r = srec + 2 * (size_t)(r0 + i);
                RChild x0, y0;
                y0.v = make_float4(0.f, 0.f, 0.f, 0.f);
                y0.s = make_int2(0, 0);
                if (i1 < nn && deg0 <= 2u && deg1 <= 2u) {
                    const uint4 *q1r = srec + 2 * (size_t)(r0 + i1);
                    RChild x1, y1;
                    y1.v = make_float4(0.f, 0.f, 0.f, 0.f);
                    y1.s = make_int2(0, 0);
                    rchild_issue(q0r[0], x0, w);
                    if (deg0 == 2u) rchild_issue(q0r[1], y0, w);
                    rchild_issue(q1r[0], x1, w);
                    if (deg1 == 2u) rchild_issue(q1r[1], y1, w);
                    rchild_slots(q0r[0], x0, w);
                    if (deg0 == 2u) rchild_slots(q0r[1], y0, w);
                    rchild_slots(q1r[0], x1, w);
                    if (deg1 == 2u) rchild_slots(q1r[1], y1, w);
                    const float4 q = rcombine<false>(d0, x0, y0, sl0, sl1, brec, w);
                    const float4 p = rcombine<false>(d1, x1, y1, sl0, sl1, brec, w);
                    dst[(int64_t)i * w.hp] = q;
                    dst[(int64_t)i1 * w.hp] = p;
                    mx0 = fmaxf(mx0, fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fmaxf(fabsf(p.x), fabsf(p.y))));
                    mx1 = fmaxf(mx1, fmaxf(fmaxf(fabsf(q.z), fabsf(q.w)), fmaxf(fabsf(p.z), fabsf(p.w))));
                    i += 2 * nwarp;
                } else {
                    rchild_issue(q0r[0], x0, w);
                    if (deg0 >= 2u) rchild_issue(q0r[1], y0, w);
                    rchild_slots(q0r[0], x0, w);
                    if (deg0 >= 2u) rchild_slots(q0r[1], y0, w);
                    const float4 q = rcombine<true>(d0, x0, y0, sl0, sl1, brec, w);
                    dst[(int64_t)i * w.hp] = q;
                    mx0 = fmaxf(mx0, fmaxf(fabsf(q.x), fabsf(q.y)));
                    mx1 = fmaxf(mx1, fmaxf(fabsf(q.z), fabsf(q.w)));
                    i += nwarp;
                }
            }
            smx[l & 1][wp][lane] = make_float2(mx0, mx1);
            __syncthreads();  // the level's rows (global) and every warp's magnitudes are visible
            for (int u = 0; u < nwarp; ++u) {
                const float2 m = smx[l & 1][u][lane];
                mx0 = fmaxf(mx0, m.x);
                mx1 = fmaxf(mx1, m.y);
            }
            const int e0 = (__float_as_int(mx0) >> 23) - 127, e1 = (__float_as_int(mx1) >> 23) - 127;
            se_w[l * se_step] = make_int2(sl0 + e0, sl1 + e1);
            if (wp == 0 && active) {  // the observed exponents: read only by later launches
                if (w.two) *reinterpret_cast<int2 *>(ow) = make_int2(e0, e1);
                else ow[0] = e0;
            }
        }
        if ((fuse & 2) && wp == 0 && active) {  // the root's value in the lane's columns, unscaled to FP64
            const float4 q = w.V4c[rrow * (int64_t)w.hp];
            const int *sr = S + (int64_t)Lroot * pitch + col;
            const int64_t gc = col0 + col;
            out[gc] = make_double2(ldexp((double)q.x, sr[0]), ldexp((double)q.y, sr[0]));
            if (w.two) out[gc + 1] = make_double2(ldexp((double)q.z, sr[1]), ldexp((double)q.w, sr[1]));
        }
        __syncthreads();  // before the next chunk reuses the shared magnitudes
    }
}
// Dynamic shared memory of a run of nlv levels and ntot nodes.
static size_t run_smem_bytes(int nlv, int64_t ntot) {
    return (size_t)ntot * (2 * sizeof(uint4) + sizeof(uint2)) + (size_t)nlv * (TPB / 32) * 32 * sizeof(int2);
}

// One level of tier B (FP64, unscaled).
__global__ void __launch_bounds__(TPB) memoB_level_f64(LevelArgs a, const uint2 *bdesc, int64_t count,
                                                        const PassDesc *pd, const MemoDesc *mdp,
                                                        double2 *__restrict__ V) {
    pdl_begin();
    const int64_t ncols = desc_cols(*pd);
    if (ncols <= 0 || count <= 0) return;
    const MemoDesc md = *mdp;
    const double2 *VA = static_cast<const double2 *>(md.VA);
    const bool narrow = md.j <= 32;
    const EvSrc es = pd->es;
    const int64_t col0 = pd->col0;
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (ncols + 31) >> 5;
    const int64_t items = ((count + NBB - 1) / NBB) * nchunks;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t blk = wid / nchunks, chunk = wid % nchunks;
    const int64_t dq = nw / nchunks, dr = nw % nchunks;
    for (int64_t it = wid; it < items; it += nw) {
        const int64_t col = chunk * 32 + lane;
        const int64_t blk_i = blk;
        chunk += dr;
        blk += dq;
        if (chunk >= nchunks) {
            chunk -= nchunks;
            ++blk;
        }
        if (col >= ncols) continue;
        const int64_t g = col0 + col;
        const int64_t vec = vec_of(es, g);
        const uint64_t pre = md.j ? __brevll(es.prefix[g] << (64 - md.j)) : 0ull;  // qubit order
        const int64_t k1 = min(count, (blk_i + 1) * NBB);
        for (int64_t kk = blk_i * NBB; kk < k1; ++kk) {
            const uint2 dsc = __ldg(bdesc + kk);
            const uint32_t r0 = dsc.x, deg = dsc.y & 0xffffffu, o = dsc.y >> 24;
            double2 r = make_double2(o == OP_MUL ? 1.0 : 0.0, 0.0);
            for (uint32_t e = 0; e < deg; ++e) {
                const uint32_t eo = __ldg(md.brec + r0 + e).x;
                double2 v;
                if (eo & 0x80000000u) {  // tier B: the child's row of the tile
                    v = __ldg(V + (int64_t)(eo & 0x7fffffffu) * a.pitch + col);
                } else {
                    const KeyPlan *kp = md.kplan + (eo - 1u);
                    const int mid = __ldg(&kp->mid);
                    const uint32_t key = mid >= 0 ? md.keys[(int64_t)mid * md.kpitch + col] : plan_key(kp, pre, narrow);
                    v = VA[md.V * __ldg(&kp->off) + ((vec << (int)__ldg(&kp->k)) | (int64_t)key)];
                }
                if (o == OP_MUL) r = cmul(r, v);
                else { r.x += v.x; r.y += v.y; }
            }
            V[(int64_t)(a.lo + kk) * a.pitch + col] = r;
        }
    }
}

// Root value of every active group column: from the tier-A slots or the tier-B tile.
__global__ void memo_root(const MemoDesc *mdp, const PassDesc *pd, uint32_t root, int Lroot, int64_t rrow,
                          const void *Vb, const int *S, int64_t pitch, int prec32, double2 *out) {
    pdl_begin();
    const int64_t ncols = desc_cols(*pd);
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const MemoDesc md = *mdp;
    const int64_t g = pd->col0 + c;
    const int64_t off = md.offu[root];
    double2 r;
    if (off >= 0) {
        const uint64_t rc = md.sigma[root] & md.jmask;
        const uint64_t pre = md.j ? __brevll(pd->es.prefix[g] << (64 - md.j)) : 0ull;
        const int64_t sl = md.V * off + ((vec_of(pd->es, g) << __popcll(rc)) | (int64_t)extract_bits(pre, rc));
        if (prec32) {
            const float2 v = static_cast<const float2 *>(md.VA)[sl];
            r = make_double2(v.x, v.y);
        } else {
            r = static_cast<const double2 *>(md.VA)[sl];
        }
    } else if (prec32) {  // tier B: the root's row of the tile
        const float2 m = static_cast<const float2 *>(Vb)[rrow * pitch + c];
        const int sc = S[(int64_t)Lroot * pitch + c];
        r = make_double2(ldexp((double)m.x, sc), ldexp((double)m.y, sc));
    } else {
        r = static_cast<const double2 *>(Vb)[rrow * pitch + c];
    }
    out[g] = r;
}

// ------------------------------------------------------------------ Gibbs sampling (amplitude AC)
// Redraw variable `var` of every chain from |A(state with var = v)|^2, where the amplitudes are
// the adjoints of the indicator leaves of `var` after an upward and a downward pass at the
// chain's full assignment.  Decision in FP64: the smallest v with u * W < W_0 + ... + W_v.
template <typename C>
__global__ void gibbs_choose(const C *A, int64_t pitch, int64_t col0, int64_t ncols, int var, int card,
                             int ind0, int n_vars, const uint64_t *seeds, uint64_t k, int8_t *state) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int64_t g = col0 + c;
    double w[16];
    double tot = 0.0;
    for (int v = 0; v < card; ++v) {
        const C a = A[(int64_t)(ind0 + v) * pitch + c];
        w[v] = (double)a.x * (double)a.x + (double)a.y * (double)a.y;
        tot += w[v];
    }
    if (!(tot > 0.0)) return;  // keep the current value (no neighbour has weight)
    uint64_t z = seeds[g] + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    const double target = u * tot;
    double acc = 0.0;
    int pick = card - 1;
    for (int v = 0; v < card; ++v) {
        acc += w[v];
        if (target < acc) { pick = v; break; }
    }
    state[g * n_vars + var] = (int8_t)pick;
}

// outcome index of every chain (output variables are the qubits 0 .. n_qubits-1)
__global__ void gibbs_record(const int8_t *state, int64_t n_chains, int n_vars, int n_qubits, int64_t n_sweeps,
                             int64_t sweep, uint64_t *samples) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    uint64_t x = 0;
    for (int q = 0; q < n_qubits; ++q) x = (x << 1) | (uint64_t)(state[c * n_vars + q] & 1);
    samples[c * n_sweeps + sweep] = x;
}

// ------------------------------------------------------------------ small kernels
// root value of every active column, in FP64 (FP32 mantissa times 2^S)
__global__ void root_f32(const float2 *V, const int *S, int64_t pitch, uint32_t root, int Lroot, int64_t ncols,
                         const int32_t *n_active, int64_t col0, double2 *out) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n_active) ncols = min(ncols, (int64_t)(*n_active) - col0);
    if (c >= ncols) return;
    float2 m = V[(int64_t)root * pitch + c];
    int s = S[(int64_t)Lroot * pitch + c];
    out[col0 + c] = make_double2(ldexp((double)m.x, s), ldexp((double)m.y, s));
}
__global__ void root_f64(const double2 *V, int64_t pitch, uint32_t root, int64_t ncols, const int32_t *n_active,
                         int64_t col0, double2 *out) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n_active) ncols = min(ncols, (int64_t)(*n_active) - col0);
    if (c >= ncols) return;
    out[col0 + c] = V[(int64_t)root * pitch + c];
}

template <typename C>
__global__ void seed_root(C *A, int64_t pitch, uint32_t root, const PassDesc *pd) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= pd->ncols) return;
    C one;
    one.x = 1;
    one.y = 0;
    A[(int64_t)root * pitch + c] = one;
}

template <typename C>
__global__ void gather_marginals(const C *A, int64_t pitch, int n_ind, int64_t ncols, int64_t col0, double2 *out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)n_ind * ncols;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = t / n_ind;
        int i = (int)(t % n_ind);
        C a = A[(int64_t)i * pitch + c];
        out[(col0 + c) * n_ind + i] = make_double2((double)a.x, (double)a.y);
    }
}

// value[v] += w Re f ; grad[v][k] += w Re(adjoint * d leaf / d angle_k)
template <typename C>
__global__ void gradient_accumulate(DevAC ac, const C *A, int64_t pitch, int64_t ncols, int64_t col0,
                                    const int32_t *col_vec, int64_t n_vectors, const double *angles,
                                    const double *weight, const double2 *rootv, double *value, double *grad) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)(ac.n_param + 1) * ncols;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int p = (int)(t / ncols);
        int64_t c = t % ncols;
        int64_t gc = col0 + c;
        int64_t v = col_vec[gc];
        v = v < 0 ? 0 : (v >= n_vectors ? n_vectors - 1 : v);  // out-of-range entries are clamped
        double w = weight[gc];
        if (p == ac.n_param) {
            atomicAdd(value + v, w * rootv[gc].x);
            continue;
        }
        int k = ac.param_angle[p];
        double th = angles[v * ac.n_angles + k];
        double s, co;
        sincos(0.5 * th, &s, &co);
        double gr, gi;
        switch (ac.param_fn[p]) {
            case 0: gr = -0.5 * s; gi = 0.0; break;
            case 1: gr = 0.5 * co; gi = 0.0; break;
            case 2: gr = -0.5 * s; gi = -0.5 * co; break;   // (-i/2) e^{-it/2}
            default: gr = -0.5 * s; gi = 0.5 * co; break;   // (+i/2) e^{+it/2}
        }
        double2 kc = ac.param_coef[p];
        double dr = kc.x * gr - kc.y * gi, di = kc.x * gi + kc.y * gr;
        C a = A[(int64_t)(ac.n_ind + p) * pitch + c];
        double contrib = (double)a.x * dr - (double)a.y * di;
        atomicAdd(grad + v * ac.n_angles + k, w * contrib);
    }
}

// ------------------------------------------------------------------ sampling kernels
__device__ __forceinline__ uint64_t splitmix64_k(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void sample_init(int64_t n_vec, int64_t max_shots, const int32_t *shots, int32_t *s_group,
                            uint64_t *s_bits, int32_t *g_vec, uint64_t *g_prefix, int32_t *g_count) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n_vec) {
        g_vec[t] = (int32_t)t;
        g_prefix[t] = 0;
    }
    if (t == 0) *g_count = (int32_t)n_vec;
    if (t < n_vec * max_shots) {
        s_group[t] = (int32_t)(t / max_shots);
        s_bits[t] = 0;
    }
    (void)shots;
}

// TRAJECTORY ACs (mixed-unitary channels, E_k = sqrt(p_k) U_k): the noise branches of every sample
// are drawn from their state-independent probabilities, so P(x) = sum_r P(r) P(x | r) is sampled
// exactly by drawing r first.  Uniform of sample s, noise variable i: (SplitMix64_k(~seed) >> 11)
// 2^-53, k = s * n_noise + i + 1 (a second stream per vector); the branch is the smallest k with
// u < cdf_k (the cumulative branch probabilities in value order), else the last.  err[t] marks a
// sample with some branch other than 0.
__global__ void traj_draw(int64_t n_vec, int64_t max_shots, const int32_t *shots, const uint64_t *seeds,
                          int n_noise, const int32_t *noise_off, const double *cdf, int8_t *traj, int32_t *err) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    const int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v]) {
        err[t] = 0;
        return;
    }
    const uint64_t sd = ~seeds[v];
    int any = 0;
    for (int i = 0; i < n_noise; ++i) {
        uint64_t z = sd + ((uint64_t)s * (uint64_t)n_noise + (uint64_t)i + 1ull) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        const int o = noise_off[i], card = noise_off[i + 1] - o;
        int r = card - 1;
        for (int k = 0; k < card - 1; ++k)
            if (u < cdf[o + k]) { r = k; break; }
        traj[t * n_noise + i] = (int8_t)r;
        any |= r != 0;
    }
    err[t] = any;
}

// Samples of one vector that drew the same error trajectory share one group: every sample with an
// error inserts (vector, trajectory) into an open-addressing table (one 64-bit word per slot: high
// half of the key's hash, 1 + the first sample that claimed it); a sample whose trajectory equals a
// claimed slot's byte for byte joins that sample.  rep[t] = the representative sample of t (t itself
// when it claimed a slot, or when no slot was found within the probe limit: then it keeps its own
// group, which is still exact).  Which equal sample represents a group may vary from run to run;
// a group's values depend only on its vector, trajectory and prefix, so the samples do not.
__global__ void traj_dedup(int64_t n_vec, int64_t max_shots, const int32_t *err, const int8_t *traj, int n_noise,
                           unsigned long long *table, uint64_t tmask, int32_t *rep) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    rep[t] = (int32_t)t;
    if (!err[t]) return;
    const int64_t v = t / max_shots;
    const int8_t *r = traj + t * n_noise;
    uint64_t h = 0x9E3779B97F4A7C15ull * (uint64_t)(v + 1);
    for (int i = 0; i < n_noise; ++i) {
        h ^= (uint64_t)(uint8_t)r[i] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 0xBF58476D1CE4E5B9ull;
    }
    h ^= h >> 31;
    const unsigned long long mine = ((unsigned long long)(h >> 32) << 32) | (unsigned long long)(t + 1);
    uint64_t slot = h & tmask;
    for (int probe = 0; probe < 4096; ++probe, slot = (slot + 1) & tmask) {
        const unsigned long long cur = atomicCAS(table + slot, 0ull, mine);
        if (cur == 0ull) return;  // claimed: t represents its (vector, trajectory)
        if ((cur >> 32) != (h >> 32)) continue;
        const int64_t o = (int64_t)(cur & 0xffffffffull) - 1;
        if (o / max_shots != v) continue;
        const int8_t *ro = traj + o * n_noise;
        bool same = true;
        for (int i = 0; i < n_noise && same; ++i) same = ro[i] == r[i];
        if (same) {
            rep[t] = (int32_t)o;
            return;
        }
    }
}
__global__ void traj_rep_flags(int64_t n, const int32_t *err, const int32_t *rep, int32_t *flag) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) flag[t] = (err[t] && rep[t] == (int32_t)t) ? 1 : 0;
}

// The first groups of a trajectory sampling call: group v holds vector v's samples whose trajectory
// has no error (all share the branches 0); the samples with one error trajectory (equal samples of a
// vector) share a group, n_vec + the rank of their representative, carrying that trajectory.
__global__ void traj_groups(int64_t n_vec, int64_t max_shots, const int32_t *shots, const int32_t *err,
                            const int32_t *rep, const int32_t *flag, const int32_t *pos, const int32_t *bsum,
                            int32_t *s_group, uint64_t *s_bits, int32_t *g_vec, uint64_t *g_prefix, int32_t *g_traj,
                            int32_t *g_count) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = n_vec * max_shots;
    if (t < n_vec) {
        g_vec[t] = (int32_t)t;
        g_prefix[t] = 0;
        g_traj[t] = -1;
    }
    if (t == n - 1) *g_count = (int32_t)n_vec + pos[t] + bsum[t >> 10] + flag[t];
    if (t >= n) return;
    const int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v]) return;
    s_bits[t] = 0;
    if (!err[t]) {
        s_group[t] = (int32_t)v;
        return;
    }
    const int32_t o = rep[t];
    const int32_t g = (int32_t)n_vec + pos[o] + bsum[o >> 10];
    s_group[t] = g;
    if (o == (int32_t)t) {
        g_vec[g] = (int32_t)v;
        g_prefix[g] = 0;
        g_traj[g] = (int32_t)t;
    }
}
__global__ void set_count(int32_t *dst, int32_t v) { *dst = v; }

// Decide bit j of every live sample; mark the child group (2g + bit).  pv[g] = (P(x_<j, X_j = 0),
// P(x_<j, X_j = 1)) of the sample's group from this step's pass; P(x_<j) is their sum.
__global__ void sample_decide(int64_t n_vec, int64_t max_shots, const int32_t *shots, const uint64_t *seeds, int j,
                              int n_qubits, const double2 *pv, int32_t *s_group,
                              uint64_t *s_bits, int32_t *flag, const int32_t *g_count, int32_t *status) {
    pdl_begin();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v]) return;
    int g = s_group[t];
    if (g < 0 || g >= *g_count) {  // a sample dropped by an understated shot total
        atomicExch(status, 1);
        return;
    }
    const double p0 = pv[g].x, P = pv[g].x + pv[g].y;
    uint64_t k = (uint64_t)s * (uint64_t)n_qubits + (uint64_t)j + 1ull;
    double u = (double)(splitmix64_k(seeds[v], k) >> 11) * (1.0 / 9007199254740992.0);
    int bit = (u * P >= p0) ? 1 : 0;
    s_bits[t] = (s_bits[t] << 1) | (uint64_t)bit;
    flag[2 * g + bit] = 1;
}

// exclusive scan of flag[0..n) into pos (block-local pass), block sums in bsum
__global__ void scan_block(const int32_t *flag, const int32_t *n_dev, int mult, int32_t *pos, int32_t *bsum) {
    pdl_begin();
    __shared__ int32_t sh[1024];
    const int64_t n = (int64_t)(*n_dev) * mult;
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    int32_t x = (i < n) ? flag[i] : 0;
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int32_t y = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += y;
        __syncthreads();
    }
    if (i < n) pos[i] = sh[threadIdx.x] - x;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = sh[1023];
}
__global__ void scan_sums(int32_t *bsum, int64_t nb) {
    pdl_begin();
    // single block: exclusive scan of nb block sums
    __shared__ int32_t carry;
    __shared__ int32_t sh[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        int32_t x = (i < nb) ? bsum[i] : 0;
        sh[threadIdx.x] = x;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int32_t y = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < nb) bsum[i] = carry + sh[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sh[1023];
        __syncthreads();
    }
}

// Build the next groups from the marked children and remap every sample.
__global__ void sample_regroup(const int32_t *g_count_old, const int32_t *flag, const int32_t *pos,
                               const int32_t *bsum, const int32_t *g_vec, const uint64_t *g_prefix,
                               const double2 *pv, int32_t *g_vec_n, uint64_t *g_prefix_n,
                               double *g_P_n, int32_t *g_count_new, int64_t nflag, const int32_t *g_traj,
                               int32_t *g_traj_n) {
    pdl_begin();
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t n = min((int64_t)(2LL * (*g_count_old)), nflag);  // only the scanned child slots
    if (k >= n) return;
    int32_t id = pos[k] + bsum[k >> 10];
    if (k == n - 1) *g_count_new = id + flag[k];
    if (!flag[k]) return;
    int64_t g = k >> 1;
    int bit = (int)(k & 1);
    g_vec_n[id] = g_vec[g];
    g_prefix_n[id] = (g_prefix[g] << 1) | (uint64_t)bit;
    if (g_traj) g_traj_n[id] = g_traj[g];
    g_P_n[id] = bit ? pv[g].y : pv[g].x;  // the child's probability P(x_<j+1), from this step's pass
}
__global__ void sample_remap(int64_t n_vec, int64_t max_shots, const int32_t *shots, const int32_t *pos,
                             const int32_t *bsum, int32_t *s_group, const uint64_t *s_bits, int64_t nflag,
                             int32_t *status) {
    pdl_begin();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v] || s_group[t] < 0) return;
    int64_t k = 2LL * s_group[t] + (int64_t)(s_bits[t] & 1ull);
    if (k >= nflag) {  // beyond the host bound (understated shot total): drop the sample
        s_group[t] = -1;
        atomicExch(status, 1);
        return;
    }
    s_group[t] = pos[k] + bsum[k >> 10];
}
// Outcome index of every sample and, when asked (probs non-null), the probability P(x) its group
// carried through the chain rule (the product of the conditionals the decisions compared against).
__global__ void sample_write(int64_t n_vec, int64_t max_shots, const int32_t *shots, const uint64_t *s_bits,
                             uint64_t *bits, const int32_t *s_group, const double *g_P, const int32_t *g_count,
                             double *probs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v]) return;
    bits[t] = s_bits[t];
    if (probs) {
        const int g = s_group[t];
        probs[t] = (g >= 0 && g < *g_count) ? g_P[g] : -1.0;  // -1: a sample dropped by an understated total
    }
}

// active column count of one timed pass, for the live roofline (stats mode)
__global__ void stat_record(const int32_t *n_active, int64_t col0, int64_t ncols, int64_t *dst) {
    int64_t c = ncols;
    if (n_active) c = min(ncols, (int64_t)(*n_active) - col0);
    *dst = c > 0 ? c : 0;
}

inline unsigned grid_for(int64_t work, int64_t per_block = TPB, int64_t cap = 152LL * 64) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace

// ------------------------------------------------------------------ handles
struct qkc_ctx {
    int device;
    int sm_count;
    size_t total_mem;
    int memoB_blocks_per_sm = 0;  // resident blocks of memoB_level_f32 (occupancy), 0 until queried
};

template <typename T>
static cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

struct qkc_ac {
    qkc_ctx *ctx = nullptr;
    int prec = 32;
    uint32_t kind, n_qubits, n_angles, n_vars, N, E, D, n_leaves, root, n_ind, n_param, n_const;
    std::vector<uint32_t> level_off;
    int64_t max_width = 0;
    int64_t n_mul_edges = 0;  // parent entries that carry a sibling (children of products)
    // downward-pass work lists: per level, light and heavy nodes (CONST leaves left out)
    std::vector<int64_t> light_off, heavy_off;
    uint32_t *d_light = nullptr, *d_heavy = nullptr;
    int64_t down_edges = 0;   // parent entries visited by the downward pass
    int64_t down_sib = 0;     // ... of which carry a sibling (product parents)
    int64_t struct_bytes = 0;
    // device structure
    uint8_t *d_op = nullptr;
    uint32_t *d_child_off = nullptr, *d_child = nullptr, *d_par_off = nullptr, *d_cl_off = nullptr;
    int2 *d_par = nullptr;
    uint16_t *d_node_level = nullptr, *d_cl = nullptr;
    int32_t *d_ind_var = nullptr, *d_ind_val = nullptr, *d_param_angle = nullptr, *d_param_fn = nullptr;
    double2 *d_param_coef = nullptr, *d_const_val = nullptr;
    // scratch
    int64_t vec_cap = 0;      // parameter vectors the param table holds
    int64_t n_vec = 0;        // vectors bound by the last set_params
    void *d_pv = nullptr;     // [n_param][vec_cap]
    const double *last_angles = nullptr;  // not owned; for gradient chaining
    int64_t tile = 0;         // columns per tile (multiple of 64)
    int64_t tile_limit = 0;   // caller's cap on the tile (0: 35% of device memory)
    void *d_V = nullptr;      // [N][tile]
    void *d_A = nullptr;      // [N][tile], allocated by the first downward pass
    bool adj_ok = false;
    int *d_S = nullptr, *d_obs = nullptr;  // [D][tile]
    uint32_t vrows = 0;                    // node rows of the value buffer d_V (N, or fewer for step ACs)
    std::vector<uint32_t> roots;           // per sampling step: its root (all the root but for step ACs)
    std::vector<int> root_lev;             // per step: the root's level
    int root_L = 0;                        // level of the root
    uint32_t *d_keys = nullptr;            // [MEMO_BKEYS][tile]: the memoised sampler's group-key table
    // TRAJECTORY ACs: noise variables, their cumulative branch probabilities, and the sampler's
    // per-sample trajectories and per-group trajectory owners
    int n_noise = 0;
    double *d_cdf = nullptr;        // per noise value, cumulative within its variable
    int32_t *d_noise_off = nullptr; // [n_noise + 1] first value of each noise variable in d_cdf
    int8_t *d_traj = nullptr;       // [samples][n_noise] branch of every noise variable
    int32_t *d_err = nullptr;       // [samples] the sample's trajectory has a branch other than 0
    int32_t *d_rep = nullptr;       // [samples] the sample representing its (vector, trajectory)
    unsigned long long *d_table = nullptr;  // [table_size] dedup table of error trajectories
    uint64_t table_size = 0;
    int32_t *d_g_traj[2] = {nullptr, nullptr};       // per group: sample whose trajectory it carries, -1: none
    int64_t traj_cap = 0;
    double2 *d_root = nullptr;  // [root_cap]
    int64_t root_cap = 0;
    // sampling scratch
    int64_t samp_cap = 0, grp_cap = 0;
    int32_t *d_s_group = nullptr, *d_flag = nullptr, *d_pos = nullptr, *d_bsum = nullptr, *d_gcount = nullptr;
    uint64_t *d_s_bits = nullptr;
    int32_t *d_g_vec[2] = {nullptr, nullptr};
    uint64_t *d_g_prefix[2] = {nullptr, nullptr};
    double *d_g_P[2] = {nullptr, nullptr};

    PassDesc *d_desc = nullptr;  // the pass descriptor the level kernels read
    // memoised sampling: indicator support of every node, per-cap step metadata, tier-A slots
    std::vector<uint64_t> sigma;
    std::vector<uint32_t> var_card;               // cardinality of every indicator variable
    std::vector<uint32_t> h_child_off, h_child;  // host copy of the structure (density ACs)
    std::vector<uint32_t> h_cl_off;              // child-level lists per level (host copy)
    std::vector<uint16_t> h_cl;
    std::vector<uint8_t> h_op;  // node ops (host copy, memoised-pass metadata)
    std::vector<int32_t> h_param_angle;  // angle slot of every parameter leaf
    // incremental re-evaluation: the dirty cone of every angle slot (built on first use), and
    // whether the tile still holds the last qkc_evaluate's values (one tile, its columns)
    struct DirtyCone {
        uint32_t *d_nodes = nullptr, *d_leaves = nullptr;
        std::vector<int64_t> lvl;  // [D + 1] offsets of each level's nodes in d_nodes
        int nleaves = 0;
    };
    std::vector<DirtyCone *> cones;
    bool eval_ok = false;
    int64_t eval_cols = 0;
    const int32_t *eval_colvec = nullptr;
    uint64_t *d_sigma = nullptr;
    MemoDesc *d_mdesc = nullptr;  // one memo descriptor per step
    // a captured launch sequence and the buffers it was captured with: the scratch generation changes
    // with every reallocation of a buffer a sequence names (values, scales, adjoints, roots), so a
    // graph is captured again whenever any of them moved, not only the value tile
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const void *V = nullptr, *A = nullptr;
        int64_t pitch = 0;
        uint64_t gen = 0;
    };
    uint64_t scratch_gen = 1;
    struct MemoMeta {
        int cap = 0;
        int64_t max_units = 0;
        std::vector<int64_t> unit_base{0};  // per step: its first unit when every step's slots are resident
        MemoARunLevel *d_alllv = nullptr;   // every step's tier-A levels (memoA_all)
        MemoALvlStep *d_lvs = nullptr;      // per level, the steps with tier-A nodes there (memoA_lvl_all)
        std::vector<int64_t> lvs_off;       // [D + 1] offsets into d_lvs
        MemoAStep *d_asteps = nullptr;      // per step: its bases and levels in d_alllv
        int32_t *d_aorder = nullptr;        // the steps by tier-A work, largest first
        int64_t all_T = 0;                  // the largest threads per vector of any tier-A level
        std::vector<std::vector<int64_t>> a_lvl, u_lvl, b_lvl, g_lvl;  // per step, [D + 1]
        std::vector<std::vector<int64_t>> t_lvl;                        // per step and level: tier-A threads
        struct AItem { int L; int64_t off; int cnt; int64_t nodes = 0; };  // one launch: level L, or a run of
                                                                         // cnt levels (tier B: of `nodes` nodes)
        std::vector<std::vector<AItem>> a_items;        // per step, in level order
        MemoARunLevel *d_runlv = nullptr;               // the runs' levels, all steps
        std::vector<std::vector<AItem>> b_items;        // per step: tier-B launches (a level, or a run of cnt levels)
        std::vector<int64_t> rst_base, rst_cnt;         // per step: levels whose observed exponents are reset
        int32_t *d_rst = nullptr;
        uint32_t *d_bclo = nullptr;                     // per step, per level (D + 1 entries a step): where
        uint16_t *d_bcl = nullptr;                      // its child levels holding tier-B nodes start in d_bcl
        MemoBRunLevel *d_brunlv = nullptr;              // the tier-B runs' levels, all steps
        std::vector<std::vector<uint8_t>> floor0;               // per step, [D]
        std::vector<int64_t> a_base, b_base, offu_base, g_base;  // per step
        std::vector<double> a_bytes_slot, b_bytes_col;           // per step: algorithmic bytes per slot unit / column
        std::vector<double> a_edges_slot, b_edges_col;           // per step: child references per vector / column
        uint32_t *d_a_nodes = nullptr;
        MemoAGroup *d_a_grp = nullptr;  // tier-A key-width groups, per step and level
        int64_t *d_offu = nullptr;
        uint32_t *d_emask = nullptr;    // [step][edge]: a child's key bits inside its tier-A parent's key
        uint2 *d_bdesc = nullptr;       // per step, per tier-B node (tier-B order): (first edge record,
                                        // degree | op << 24)
        uint4 *d_brec = nullptr;        // per step, per edge of a tier-B node: where its child's values live
                                        // (a tier-B child's tile row and level, or a tier-A child's key plan,
                                        // key width, group-key table row and block offset; see BChild)
        std::vector<int64_t> br_base;   // per step: first edge record
        std::vector<int64_t> root_row;  // per step: the root's tier-B row, -1 when the root is tier A
        std::vector<int> fuse;          // per step: its first tier-B run forms the group keys (bit 0), its
                                        // last run writes the root values (bit 1)
        int64_t max_rows = 0;           // tier-B nodes of the largest step (rows of the value tile)
        KeyPlan *d_kplan = nullptr;     // key plans of the tier-A children of tier-B nodes, per step
        KeyPlan *d_aplan = nullptr;     // key plans of scattered child-key masks of tier-A nodes, per step
        std::vector<int64_t> kp_base, ap_base;  // per step: first key plan of each kind
        KeyPlan *d_bplan = nullptr;     // per step: the tabled supports (group-key table rows)
        std::vector<int64_t> bp_base, bp_cnt;
        std::vector<GraphSlot> gA, gB;  // captured launch sequences per step
    };
    std::vector<MemoMeta *> memo;  // indexed by cap
    void *d_VA = nullptr;
    int64_t va_bytes = 0;
    int sampler = 1;  // 1: memoised when estimated cheaper, 2: memoised whenever it fits, 0: per group
    int64_t memo_budget = 0;  // bytes for memoised slots (0: automatic)
    int32_t *d_status = nullptr; // device-side error word (sampling input checks)
    GraphSlot g_up, g_down;
    // stats: launches of this library's kernels, and (when enabled) CUDA events around
    // every chain of level kernels with the number of columns it processed
    int64_t launches = 0;
    bool timing = false;
    struct Rec {  // kind 0 up, 1 down, 2/3 memo tier B/A
        cudaEvent_t e0, e1;
        int kind;
        double fixed_bytes, col_bytes, fixed_edges, col_edges;
    };
    std::vector<Rec> recs;
    int64_t *d_statcols = nullptr;
    int64_t statcap = 0;

    DevAC dev() const {
        DevAC d;
        d.op = d_op; d.child_off = d_child_off; d.child = d_child; d.node_level = d_node_level;
        d.par_off = d_par_off; d.par = d_par; d.ind_var = d_ind_var; d.ind_val = d_ind_val;
        d.param_angle = d_param_angle; d.param_fn = d_param_fn; d.param_coef = d_param_coef;
        d.const_val = d_const_val; d.cl_off = d_cl_off; d.cl = d_cl;
        d.n_ind = (int)n_ind; d.n_param = (int)n_param; d.n_const = (int)n_const; d.n_vars = (int)n_vars;
        d.n_angles = (int)n_angles; d.n_qubits = (int)n_qubits;
        return d;
    }
    size_t elem() const { return prec == 32 ? sizeof(float2) : sizeof(double2); }
};

extern "C" qkc_status qkc_ctx_create(int device, qkc_ctx **out) {
    if (!out) return fail(QKC_ERR_ARG, "qkc_ctx_create: out is null");
    int n = 0;
    QKC_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(QKC_ERR_ARG, "qkc_ctx_create: device %d of %d", device, n);
    QKC_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    QKC_CUDA(cudaGetDeviceProperties(&prop, device));
    qkc_ctx *c = new (std::nothrow) qkc_ctx;
    if (!c) return fail(QKC_ERR_NOMEM, "qkc_ctx_create: out of host memory");
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->total_mem = prop.totalGlobalMem;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->memoB_blocks_per_sm, memoB_level_f32, TPB, 0) != cudaSuccess ||
        c->memoB_blocks_per_sm < 1) {
        cudaGetLastError();
        c->memoB_blocks_per_sm = 4;
    }
    // tier-B runs stage up to MEMO_RUN_NODES nodes and MEMO_RUN_LV levels in dynamic shared memory
    if (cudaFuncSetAttribute(memoB_run_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)run_smem_bytes(MEMO_RUN_LV, MEMO_RUN_NODES)) != cudaSuccess ||
        cudaFuncSetAttribute(memoB_runc_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)run_smem_bytes(MEMO_RUN_LV, MEMO_RUN_NODES)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(QKC_ERR_CUDA, "qkc_ctx_create: cannot size the shared memory of the tier-B run kernel");
    }
    *out = c;
    return QKC_OK;
}

extern "C" void qkc_ctx_destroy(qkc_ctx *ctx) { delete ctx; }

static void free_scratch(qkc_ac *a) {
    ++a->scratch_gen;
    cudaFree(a->d_pv); a->d_pv = nullptr;
    cudaFree(a->d_V); a->d_V = nullptr;
    cudaFree(a->d_A); a->d_A = nullptr; a->adj_ok = false;
    cudaFree(a->d_S); a->d_S = nullptr;
    cudaFree(a->d_obs); a->d_obs = nullptr;
    cudaFree(a->d_keys); a->d_keys = nullptr;
    cudaFree(a->d_root); a->d_root = nullptr;
    cudaFree(a->d_s_group); cudaFree(a->d_flag); cudaFree(a->d_pos); cudaFree(a->d_bsum);
    cudaFree(a->d_gcount); cudaFree(a->d_s_bits);
    a->d_s_group = a->d_flag = a->d_pos = a->d_bsum = a->d_gcount = nullptr;
    a->d_s_bits = nullptr;
    for (int i = 0; i < 2; ++i) {
        cudaFree(a->d_g_vec[i]); cudaFree(a->d_g_prefix[i]); cudaFree(a->d_g_P[i]); cudaFree(a->d_g_traj[i]);
        a->d_g_vec[i] = nullptr; a->d_g_prefix[i] = nullptr; a->d_g_P[i] = nullptr; a->d_g_traj[i] = nullptr;
    }
    cudaFree(a->d_traj); cudaFree(a->d_err); cudaFree(a->d_rep); cudaFree(a->d_table);
    a->d_traj = nullptr; a->d_err = a->d_rep = nullptr; a->d_table = nullptr; a->table_size = 0;
    a->vec_cap = a->tile = a->root_cap = a->samp_cap = a->grp_cap = a->traj_cap = 0;
}

static void drop_records(qkc_ac *a) {
    for (auto &r : a->recs) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    a->recs.clear();
}

extern "C" void qkc_free_ac(qkc_ac *a) {
    if (!a) return;
    cudaSetDevice(a->ctx->device);
    cudaDeviceSynchronize();
    drop_records(a);
    cudaFree(a->d_statcols);
    if (a->g_up.exec) cudaGraphExecDestroy(a->g_up.exec);
    if (a->g_down.exec) cudaGraphExecDestroy(a->g_down.exec);
    cudaFree(a->d_desc);
    cudaFree(a->d_status);
    cudaFree(a->d_sigma);
    cudaFree(a->d_cdf); cudaFree(a->d_noise_off);
    for (auto *c : a->cones)
        if (c) { cudaFree(c->d_nodes); cudaFree(c->d_leaves); delete c; }
    cudaFree(a->d_mdesc);
    cudaFree(a->d_VA);
    for (auto *m : a->memo) {
        if (!m) continue;
        cudaFree(m->d_a_nodes); cudaFree(m->d_a_grp); cudaFree(m->d_offu);
        cudaFree(m->d_emask); cudaFree(m->d_runlv); cudaFree(m->d_brunlv); cudaFree(m->d_rst); cudaFree(m->d_alllv); cudaFree(m->d_lvs); cudaFree(m->d_asteps); cudaFree(m->d_aorder); cudaFree(m->d_bclo); cudaFree(m->d_bcl); cudaFree(m->d_bdesc); cudaFree(m->d_brec); cudaFree(m->d_kplan); cudaFree(m->d_aplan); cudaFree(m->d_bplan);
        for (auto &g : m->gA) if (g.exec) cudaGraphExecDestroy(g.exec);
        for (auto &g : m->gB) if (g.exec) cudaGraphExecDestroy(g.exec);
        delete m;
    }
    free_scratch(a);
    cudaFree(a->d_op); cudaFree(a->d_child_off); cudaFree(a->d_child); cudaFree(a->d_par_off);
    cudaFree(a->d_par); cudaFree(a->d_node_level); cudaFree(a->d_cl_off); cudaFree(a->d_cl);
    cudaFree(a->d_ind_var); cudaFree(a->d_ind_val); cudaFree(a->d_param_angle); cudaFree(a->d_param_fn);
    cudaFree(a->d_param_coef); cudaFree(a->d_const_val);
    cudaFree(a->d_light); cudaFree(a->d_heavy);
    delete a;
}

// ---- parse + validate + upload
static bool take(uint64_t &off, uint64_t len, uint64_t bytes, uint64_t &start) {
    off = (off + 7) & ~(uint64_t)7;
    if (off + bytes > len || off + bytes < off) return false;
    start = off;
    off += bytes;
    return true;
}

template <typename T>
static qkc_status upload(T **dst, const T *src, size_t count, int64_t &bytes) {
    QKC_CUDA(dalloc(dst, count));
    if (count) QKC_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    bytes += (int64_t)(count * sizeof(T));
    return QKC_OK;
}

extern "C" qkc_status qkc_load_ac(qkc_ctx *ctx, const uint8_t *bytes, uint64_t len, int32_t precision,
                                  qkc_ac **out) {
    if (!ctx || !bytes || !out) return fail(QKC_ERR_ARG, "qkc_load_ac: null argument");
    if (precision != 32 && precision != 64) return fail(QKC_ERR_ARG, "qkc_load_ac: precision must be 32 or 64");
    if (len < 64) return fail(QKC_ERR_FORMAT, "qkc_load_ac: buffer shorter than the header");
    uint32_t h[16];
    std::memcpy(h, bytes, 64);
    if (h[0] != 0x43414B51u || h[1] != 1u) return fail(QKC_ERR_FORMAT, "qkc_load_ac: bad magic or version");
    const uint32_t kind = h[2], nq = h[3], na = h[4], nv = h[5], N = h[6], E = h[7], D = h[8], nl = h[9],
                   root = h[10], nind = h[11];
    if (kind > 3 || nq == 0 || nq > 64 || N == 0 || D == 0 || D > 65535 || nl > N || root >= N || nind > nl ||
        h[12] != (kind == QKC_AC_DENSITY_STEPS ? nq : 0u) || (kind != QKC_AC_TRAJECTORY && h[13] != 0u) ||
        (kind == QKC_AC_TRAJECTORY && nv < nq))
        return fail(QKC_ERR_FORMAT, "qkc_load_ac: inconsistent header");
    uint64_t off = 64, s_card, s_tag, s_lo, s_op, s_coff, s_child, s_la, s_lb, s_lc;
    bool ok = take(off, len, 4ull * nv, s_card) && take(off, len, 4ull * nv, s_tag) &&
              take(off, len, 4ull * (D + 1), s_lo) && take(off, len, 1ull * N, s_op) &&
              take(off, len, 4ull * (N + 1), s_coff) && take(off, len, 4ull * E, s_child) &&
              take(off, len, 4ull * nl, s_la) && take(off, len, 4ull * nl, s_lb) && take(off, len, 16ull * nl, s_lc);
    uint64_t s_roots = 0;
    if (ok && kind == QKC_AC_DENSITY_STEPS) ok = take(off, len, 4ull * nq, s_roots);
    uint64_t s_prior = 0;
    if (ok && kind == QKC_AC_TRAJECTORY) ok = take(off, len, 8ull * h[13], s_prior);
    if (!ok) return fail(QKC_ERR_FORMAT, "qkc_load_ac: buffer too short for its arrays");
    auto rd = [&](uint64_t s, size_t i, size_t w) {
        uint64_t v = 0;
        std::memcpy(&v, bytes + s + i * w, w);
        return v;
    };
    std::vector<uint32_t> card(nv), lo(D + 1), coff(N + 1), child(E);
    std::vector<int32_t> la(nl), lb(nl);
    std::vector<uint8_t> op(N);
    std::vector<double> lc(2ull * nl);
    for (uint32_t i = 0; i < nv; ++i) card[i] = (uint32_t)rd(s_card, i, 4);
    for (uint32_t i = 0; i <= D; ++i) lo[i] = (uint32_t)rd(s_lo, i, 4);
    std::memcpy(op.data(), bytes + s_op, N);
    std::memcpy(coff.data(), bytes + s_coff, 4ull * (N + 1));
    if (E) std::memcpy(child.data(), bytes + s_child, 4ull * E);
    if (nl) {
        std::memcpy(la.data(), bytes + s_la, 4ull * nl);
        std::memcpy(lb.data(), bytes + s_lb, 4ull * nl);
        std::memcpy(lc.data(), bytes + s_lc, 16ull * nl);
    }
    // validation: levels, ops, children, leaf payloads
    if (lo[0] != 0 || lo[D] != N || lo[1] != nl) return fail(QKC_ERR_FORMAT, "qkc_load_ac: bad level offsets");
    for (uint32_t l = 0; l < D; ++l)
        if (lo[l + 1] < lo[l]) return fail(QKC_ERR_FORMAT, "qkc_load_ac: level offsets not sorted");
    if (coff[0] != 0 || coff[N] != E) return fail(QKC_ERR_FORMAT, "qkc_load_ac: bad child offsets");
    std::vector<uint16_t> lev(N);
    for (uint32_t l = 0; l < D; ++l)
        for (uint32_t i = lo[l]; i < lo[l + 1]; ++i) lev[i] = (uint16_t)l;
    uint32_t n_ind = 0, n_param = 0;
    std::vector<uint32_t> ind_off(nv + 1, 0);
    for (uint32_t i = 0; i < nv; ++i) ind_off[i + 1] = ind_off[i] + card[i];
    if (ind_off[nv] != nind) return fail(QKC_ERR_FORMAT, "qkc_load_ac: indicator count mismatch");
    for (uint32_t i = 0; i < N; ++i) {
        if (coff[i + 1] < coff[i]) return fail(QKC_ERR_FORMAT, "qkc_load_ac: child offsets not sorted");
        const uint32_t deg = coff[i + 1] - coff[i];
        if (i < nl) {
            if (op[i] > OP_CONST || deg) return fail(QKC_ERR_FORMAT, "qkc_load_ac: node %u: bad leaf", i);
            if (op[i] == OP_IND) {
                if (i != n_ind) return fail(QKC_ERR_FORMAT, "qkc_load_ac: indicator leaves not first");
                ++n_ind;
                if (la[i] < 0 || (uint32_t)la[i] >= nv || lb[i] < 0 || (uint32_t)lb[i] >= card[la[i]] ||
                    ind_off[la[i]] + (uint32_t)lb[i] != i)
                    return fail(QKC_ERR_FORMAT, "qkc_load_ac: node %u: bad indicator", i);
            } else if (op[i] == OP_PARAM) {
                if (i != n_ind + n_param) return fail(QKC_ERR_FORMAT, "qkc_load_ac: PARAM leaves out of order");
                ++n_param;
                if (la[i] < 0 || (uint32_t)la[i] >= na || lb[i] < 0 || lb[i] > 3)
                    return fail(QKC_ERR_FORMAT, "qkc_load_ac: node %u: bad parameter leaf", i);
            }
        } else {
            if (op[i] == OP_MUL && deg != 2) return fail(QKC_ERR_FORMAT, "qkc_load_ac: node %u: MUL arity", i);
            if (op[i] == OP_ADD && deg < 1) return fail(QKC_ERR_FORMAT, "qkc_load_ac: node %u: empty ADD", i);
            if (op[i] != OP_ADD && op[i] != OP_MUL) return fail(QKC_ERR_FORMAT, "qkc_load_ac: node %u: op", i);
            for (uint32_t e = coff[i]; e < coff[i + 1]; ++e)
                if (child[e] >= N || lev[child[e]] >= lev[i])
                    return fail(QKC_ERR_FORMAT, "qkc_load_ac: node %u: child not on a lower level", i);
        }
    }
    if (n_ind != nind) return fail(QKC_ERR_FORMAT, "qkc_load_ac: indicator leaves missing");
    // TRAJECTORY: the branch probabilities of every noise variable (variables nq .. nv-1), checked
    // to form a distribution, kept as cumulative sums for drawing trajectories
    std::vector<double> cdf;
    std::vector<int32_t> noise_off;
    if (kind == QKC_AC_TRAJECTORY) {
        for (uint32_t v = 0; v < nq; ++v)
            if (card[v] != 2) return fail(QKC_ERR_FORMAT, "qkc_load_ac: output variable %u is not binary", v);
        uint64_t want = 0;
        for (uint32_t v = nq; v < nv; ++v) want += card[v];
        if (want != h[13]) return fail(QKC_ERR_FORMAT, "qkc_load_ac: %u branch probabilities for %llu noise values",
                                       h[13], (unsigned long long)want);
        std::vector<double> pr(h[13]);
        if (h[13]) std::memcpy(pr.data(), bytes + s_prior, 8ull * h[13]);
        uint32_t k = 0;
        for (uint32_t v = nq; v < nv; ++v) {
            noise_off.push_back((int32_t)k);
            double acc = 0.0;
            for (uint32_t x = 0; x < card[v]; ++x, ++k) {
                if (!(pr[k] >= 0.0 && pr[k] <= 1.0)) return fail(QKC_ERR_FORMAT, "qkc_load_ac: bad branch probability");
                acc += pr[k];
                cdf.push_back(acc);
            }
            if (std::fabs(acc - 1.0) > 1e-9)
                return fail(QKC_ERR_FORMAT, "qkc_load_ac: branch probabilities of noise variable %u sum to %.17g", v, acc);
        }
        noise_off.push_back((int32_t)k);
    }
    std::vector<uint32_t> roots(nq, root);  // the root of every sampling step
    if (kind == QKC_AC_DENSITY_STEPS) {
        std::memcpy(roots.data(), bytes + s_roots, 4ull * nq);
        for (uint32_t j = 0; j < nq; ++j)
            if (roots[j] >= N) return fail(QKC_ERR_FORMAT, "qkc_load_ac: step root %u out of range", j);
        if (roots[nq - 1] != root) return fail(QKC_ERR_FORMAT, "qkc_load_ac: the last step root is not the root");
    } else if (lev[root] != D - 1 || lo[D - 1] + 1 != lo[D]) {
        return fail(QKC_ERR_FORMAT, "qkc_load_ac: root is not alone on the top level");
    }
    // transposed CSR of (parent, sibling)
    std::vector<uint32_t> poff(N + 1, 0);
    for (uint32_t e = 0; e < E; ++e) poff[child[e] + 1]++;
    for (uint32_t i = 0; i < N; ++i) poff[i + 1] += poff[i];
    std::vector<int2> par(E);
    std::vector<uint32_t> fillp(poff.begin(), poff.end() - 1);
    for (uint32_t p = nl; p < N; ++p) {
        for (uint32_t e = coff[p]; e < coff[p + 1]; ++e) {
            int sib = -1;
            if (op[p] == OP_MUL) sib = (int)child[coff[p] + (e == coff[p] ? 1 : 0)];
            par[fillp[child[e]]++] = make_int2((int)p, sib);
        }
    }
    // downward-pass work lists (level order; CONST leaves never need an adjoint)
    std::vector<uint32_t> light, heavy;
    std::vector<int64_t> light_off(D + 1, 0), heavy_off(D + 1, 0);
    int64_t down_edges = 0, down_sib = 0;
    for (uint32_t l = 0; l < D; ++l) {
        for (uint32_t i = lo[l]; i < lo[l + 1]; ++i) {
            if (op[i] == OP_CONST) continue;
            const uint32_t fo = poff[i + 1] - poff[i];
            down_edges += fo;
            for (uint32_t e = poff[i]; e < poff[i + 1]; ++e) down_sib += par[e].y >= 0;
            (fo > (uint32_t)HEAVY ? heavy : light).push_back(i);
        }
        light_off[l + 1] = (int64_t)light.size();
        heavy_off[l + 1] = (int64_t)heavy.size();
    }
    // child-level lists per level
    std::vector<uint32_t> cloff(D + 1, 0);
    std::vector<uint16_t> cl;
    {
        std::vector<int> seen(D, -1);
        for (uint32_t l = 0; l < D; ++l) {
            for (uint32_t i = lo[l]; i < lo[l + 1]; ++i)
                for (uint32_t e = coff[i]; e < coff[i + 1]; ++e) {
                    uint16_t cl_ = lev[child[e]];
                    if (seen[cl_] != (int)l) { seen[cl_] = (int)l; cl.push_back(cl_); }
                }
            cloff[l + 1] = (uint32_t)cl.size();
        }
    }
    std::vector<int32_t> ind_var(nind), ind_val(nind), p_angle(n_param), p_fn(n_param);
    std::vector<double2> p_coef(n_param), c_val(nl - nind - n_param);
    for (uint32_t i = 0; i < nind; ++i) { ind_var[i] = la[i]; ind_val[i] = lb[i]; }
    for (uint32_t i = 0; i < n_param; ++i) {
        p_angle[i] = la[nind + i]; p_fn[i] = lb[nind + i];
        p_coef[i] = make_double2(lc[2 * (nind + i)], lc[2 * (nind + i) + 1]);
    }
    for (uint32_t i = nind + n_param; i < nl; ++i) {
        if (op[i] != OP_CONST) return fail(QKC_ERR_FORMAT, "qkc_load_ac: leaf order");
        c_val[i - nind - n_param] = make_double2(lc[2 * i], lc[2 * i + 1]);
    }
    QKC_CUDA(cudaSetDevice(ctx->device));
    qkc_ac *a = new (std::nothrow) qkc_ac;
    if (!a) return fail(QKC_ERR_NOMEM, "qkc_load_ac: out of host memory");
    a->ctx = ctx; a->prec = precision; a->kind = kind; a->n_qubits = nq; a->n_angles = na; a->n_vars = nv;
    a->N = N; a->E = E; a->D = D; a->n_leaves = nl; a->root = root; a->n_ind = nind; a->n_param = n_param;
    a->roots = roots;
    a->n_noise = kind == QKC_AC_TRAJECTORY ? (int)(nv - nq) : 0;
    a->root_L = (int)lev[root];
    for (uint32_t j = 0; j < nq; ++j) a->root_lev.push_back((int)lev[roots[j]]);
    a->n_const = nl - nind - n_param; a->level_off = lo;
    a->var_card = card;
    for (uint32_t i = nl; i < N; ++i)
        if (op[i] == OP_MUL) a->n_mul_edges += coff[i + 1] - coff[i];
    a->light_off = light_off;
    a->heavy_off = heavy_off;
    a->down_edges = down_edges;
    a->down_sib = down_sib;
    for (uint32_t l = 0; l < D; ++l) a->max_width = std::max<int64_t>(a->max_width, lo[l + 1] - lo[l]);
    qkc_status st = QKC_OK;
    int64_t &b = a->struct_bytes;
    if ((st = upload(&a->d_op, op.data(), N, b)) || (st = upload(&a->d_child_off, coff.data(), N + 1, b)) ||
        (st = upload(&a->d_child, child.data(), E, b)) || (st = upload(&a->d_par_off, poff.data(), N + 1, b)) ||
        (st = upload(&a->d_par, par.data(), E, b)) || (st = upload(&a->d_node_level, lev.data(), N, b)) ||
        (st = upload(&a->d_cl_off, cloff.data(), D + 1, b)) || (st = upload(&a->d_cl, cl.data(), cl.size(), b)) ||
        (st = upload(&a->d_ind_var, ind_var.data(), nind, b)) || (st = upload(&a->d_ind_val, ind_val.data(), nind, b)) ||
        (st = upload(&a->d_param_angle, p_angle.data(), n_param, b)) ||
        (st = upload(&a->d_param_fn, p_fn.data(), n_param, b)) ||
        (st = upload(&a->d_param_coef, p_coef.data(), n_param, b)) ||
        (st = upload(&a->d_const_val, c_val.data(), c_val.size(), b)) ||
        (st = upload(&a->d_light, light.data(), light.size(), b)) ||
        (st = upload(&a->d_heavy, heavy.data(), heavy.size(), b))) {
        qkc_free_ac(a);
        return st;
    }
    a->h_cl_off = cloff;    // child-level lists per level (the memoised passes' resets)
    a->h_cl = cl;
    a->h_child_off = coff;  // host copy of the structure (memoised passes, dirty cones)
    a->h_child = child;
    a->h_op = op;
    a->h_param_angle = p_angle;
    if (kind == QKC_AC_DENSITY || kind == QKC_AC_DENSITY_STEPS) {  // indicator supports (memoised sampling)
        a->sigma.assign(N, 0ull);
        for (uint32_t i = 0; i < nind; ++i) a->sigma[i] = 1ull << (uint32_t)ind_var[i];
        for (uint32_t i = nl; i < N; ++i)
            for (uint32_t e = coff[i]; e < coff[i + 1]; ++e) a->sigma[i] |= a->sigma[child[e]];
        if ((st = upload(&a->d_sigma, a->sigma.data(), N, b))) {
            qkc_free_ac(a);
            return st;
        }
    }
    if (kind == QKC_AC_TRAJECTORY &&
        ((st = upload(&a->d_cdf, cdf.data(), cdf.size(), b)) ||
         (st = upload(&a->d_noise_off, noise_off.data(), noise_off.size(), b)))) {
        qkc_free_ac(a);
        return st;
    }
    if (cudaMalloc((void **)&a->d_mdesc, sizeof(MemoDesc) * std::max<size_t>(1, a->n_qubits)) != cudaSuccess ||
        cudaMalloc((void **)&a->d_desc, sizeof(PassDesc)) != cudaSuccess ||
        cudaMalloc((void **)&a->d_status, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(a->d_status, 0, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        qkc_free_ac(a);
        return fail(QKC_ERR_NOMEM, "qkc_load_ac: cannot allocate the pass descriptor");
    }
    *out = a;
    return QKC_OK;
}

extern "C" qkc_status qkc_get_info(const qkc_ac *a, qkc_ac_info *o) {
    if (!a || !o) return fail(QKC_ERR_ARG, "qkc_get_info: null argument");
    o->kind = (int32_t)a->kind; o->n_qubits = (int32_t)a->n_qubits; o->n_angles = (int32_t)a->n_angles;
    o->n_vars = (int32_t)a->n_vars; o->n_ind = (int32_t)a->n_ind; o->precision = a->prec;
    o->n_nodes = a->N; o->n_edges = a->E; o->n_levels = a->D; o->n_leaves = a->n_leaves;
    o->max_level_width = a->max_width; o->device_bytes = a->struct_bytes; o->reserved_columns = a->tile;
    return QKC_OK;
}

// ---- scratch management
static qkc_status ensure_vectors(qkc_ac *a, int64_t nvec) {
    if (nvec <= a->vec_cap) return QKC_OK;
    QKC_CUDA(cudaDeviceSynchronize());
    cudaFree(a->d_pv);
    a->d_pv = nullptr;
    a->vec_cap = 0;
    QKC_CUDA(cudaMalloc(&a->d_pv, std::max<size_t>(1, (size_t)a->n_param * nvec * a->elem())));
    a->vec_cap = nvec;
    return QKC_OK;
}

// Column tile: values for `cols` columns, rounded up to 64, capped so that the
// value buffer (and, when a downward pass needs it, the adjoint buffer of the
// same shape) each stay within 25% of the device memory.
// The value tile: `rows` node rows (0: every node; the memoised passes of a step AC need only
// the largest step's tier-B rows) x a multiple of 64 columns, at least `cols` when it fits.
static qkc_status ensure_tile(qkc_ac *a, int64_t cols, uint32_t rows = 0) {
    if (rows == 0) rows = a->N;
    int64_t want = (cols + 63) / 64 * 64;
    if (want < 64) want = 64;
    const int64_t per_col = (int64_t)rows * (int64_t)a->elem() + 8LL * a->D + 4LL * MEMO_BKEYS;
    int64_t cap = (int64_t)((double)a->ctx->total_mem * 0.30) / std::max<int64_t>(1, per_col);
    if (const char *env = std::getenv("QKC_MAX_TILE_COLUMNS")) {  // smaller tiles (tests of the tiled path)
        const long long lim = std::atoll(env);
        if (lim > 0) cap = std::min<int64_t>(cap, lim);
    }
    if (a->tile_limit > 0) cap = std::min<int64_t>(cap, a->tile_limit);
    cap = cap / 64 * 64;
    if (cap < 64) return fail(QKC_ERR_NOMEM, "qkc: AC too large for one 64-column tile");
    want = std::min(want, cap);
    if (want <= a->tile && rows <= a->vrows) return QKC_OK;
    QKC_CUDA(cudaDeviceSynchronize());
    a->eval_ok = false;
    ++a->scratch_gen;
    cudaFree(a->d_V); cudaFree(a->d_A); cudaFree(a->d_S); cudaFree(a->d_obs); cudaFree(a->d_keys);
    a->d_V = a->d_A = nullptr; a->d_S = a->d_obs = nullptr; a->d_keys = nullptr; a->tile = 0; a->adj_ok = false;
    cudaError_t e1 = cudaMalloc(&a->d_V, (size_t)rows * want * a->elem());
    cudaError_t e3 = cudaMalloc((void **)&a->d_S, sizeof(int) * (size_t)a->D * want);
    cudaError_t e4 = cudaMalloc((void **)&a->d_obs, sizeof(int) * (size_t)a->D * want);
    cudaError_t e5 = cudaMalloc((void **)&a->d_keys, sizeof(uint32_t) * (size_t)MEMO_BKEYS * want);
    if (e1 || e3 || e4 || e5) {
        cudaFree(a->d_V); cudaFree(a->d_S); cudaFree(a->d_obs); cudaFree(a->d_keys);
        a->d_V = nullptr; a->d_S = a->d_obs = nullptr; a->d_keys = nullptr;
        cudaGetLastError();
        return fail(QKC_ERR_NOMEM, "qkc: cannot allocate a %lld-column tile", (long long)want);
    }
    a->tile = want;
    a->vrows = rows;
    return QKC_OK;
}

static qkc_status ensure_adj(qkc_ac *a) {
    if (a->adj_ok) return QKC_OK;
    QKC_CUDA(cudaDeviceSynchronize());
    ++a->scratch_gen;
    cudaFree(a->d_A);
    a->d_A = nullptr;
    cudaError_t e = cudaMalloc(&a->d_A, (size_t)a->N * a->tile * a->elem());
    if (e) {
        cudaGetLastError();
        return fail(QKC_ERR_NOMEM, "qkc: cannot allocate the adjoint buffer (%lld columns)", (long long)a->tile);
    }
    a->adj_ok = true;
    return QKC_OK;
}

static qkc_status ensure_roots(qkc_ac *a, int64_t n) {
    if (n <= a->root_cap) return QKC_OK;
    QKC_CUDA(cudaDeviceSynchronize());
    ++a->scratch_gen;
    cudaFree(a->d_root);
    a->d_root = nullptr;
    a->root_cap = 0;
    QKC_CUDA(cudaMalloc((void **)&a->d_root, sizeof(double2) * (size_t)std::max<int64_t>(1, n)));
    a->root_cap = n;
    return QKC_OK;
}

extern "C" qkc_status qkc_reserve(qkc_ac *a, int64_t max_vectors, int64_t max_columns) {
    if (!a || max_vectors < 0 || max_columns < 0) return fail(QKC_ERR_ARG, "qkc_reserve: bad argument");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    qkc_status st;
    if ((st = ensure_vectors(a, max_vectors))) return st;
    if (max_columns > 0) {
        if ((st = ensure_tile(a, max_columns))) return st;
        if ((st = ensure_roots(a, max_columns))) return st;
    }
    return QKC_OK;
}

extern "C" qkc_status qkc_set_tile_limit(qkc_ac *a, int64_t max_tile_columns) {
    if (!a || max_tile_columns < 0) return fail(QKC_ERR_ARG, "qkc_set_tile_limit: bad argument");
    if (max_tile_columns > 0 && max_tile_columns < 64)
        return fail(QKC_ERR_ARG, "qkc_set_tile_limit: the tile holds at least 64 columns");
    a->tile_limit = max_tile_columns;
    return QKC_OK;
}

extern "C" qkc_status qkc_set_params(qkc_ac *a, const double *angles, int64_t n_vec, void *stream) {
    if (!a || n_vec <= 0 || (!angles && a->n_angles > 0)) return fail(QKC_ERR_ARG, "qkc_set_params: bad argument");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    qkc_status st = ensure_vectors(a, n_vec);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (a->n_param > 0) {
        const int64_t work = (int64_t)a->n_param * n_vec;
        if (a->prec == 32)
            bind_params_kernel<float2><<<grid_for(work), TPB, 0, s>>>(a->dev(), angles, n_vec, a->vec_cap,
                                                                      (float2 *)a->d_pv);
        else
            bind_params_kernel<double2><<<grid_for(work), TPB, 0, s>>>(a->dev(), angles, n_vec, a->vec_cap,
                                                                       (double2 *)a->d_pv);
        ++a->launches;
        QKC_LAUNCH_CHECK();
    }
    a->n_vec = n_vec;
    a->last_angles = angles;
    return QKC_OK;
}

// ---- one upward pass over a column tile [col0, col0 + ncols)
// Opens a timed record (stats mode): event before the level-kernel chain; the
// active column count is written by a tiny kernel so device-side counts work.
static qkc_status rec_begin(qkc_ac *a, int kind, const int32_t *n_active, int64_t col0, int64_t ncols,
                            cudaStream_t s) {
    if (!a->timing) return QKC_OK;
    if ((int64_t)a->recs.size() >= a->statcap) return QKC_OK;  // record buffer full: stop recording
    qkc_ac::Rec r;
    r.kind = kind;
    r.fixed_bytes = 0.0;
    r.col_bytes = 0.0;
    r.fixed_edges = 0.0;
    r.col_edges = 0.0;
    QKC_CUDA(cudaEventCreate(&r.e0));
    QKC_CUDA(cudaEventCreate(&r.e1));
    stat_record<<<1, 1, 0, s>>>(n_active, col0, ncols, a->d_statcols + a->recs.size());
    ++a->launches;
    QKC_CUDA(cudaEventRecord(r.e0, s));
    a->recs.push_back(r);
    return QKC_OK;
}
static qkc_status rec_end(qkc_ac *a, size_t idx, cudaStream_t s) {
    if (!a->timing || idx >= a->recs.size()) return QKC_OK;
    QKC_CUDA(cudaEventRecord(a->recs[idx].e1, s));
    return QKC_OK;
}

// The launches of one upward pass over a tile of `pitch` columns (levels 0 .. D-1). Every
// kernel reads the pass descriptor a->d_desc, and grids are sized for a full tile, so the
// same sequence serves any column count: it is captured once as a CUDA graph and replayed.
static void launch_up_sequence(qkc_ac *a, cudaStream_t s, void *V, int *S, int *obs, int64_t pitch) {
    const DevAC d = a->dev();
    const int sms = a->ctx->sm_count;
    const PassDesc *pd = a->d_desc;
    const unsigned gs = (unsigned)((pitch + TPB - 1) / TPB);
    if (a->prec == 32) {
        // level 0: leaves (S[0] = 0 and obs[0] reset by the scale kernel, then observed)
        level_scale_kernel<<<gs, TPB, 0, s>>>(d.cl_off, d.cl, 0, pitch, 0, S, obs);
        bind_leaves_f32<<<grid_for((int64_t)a->n_leaves * pitch), TPB, 0, s>>>(d, pd, pitch, (float2 *)V, obs,
                                                                              (int)a->n_leaves);
        for (uint32_t L = 1; L < a->D; ++L) {
            level_scale_kernel<<<gs, TPB, 0, s>>>(d.cl_off, d.cl, (int)L, pitch, 0, S, obs);
            LevelArgs la{a->level_off[L], a->level_off[L + 1], (int)L, pitch};
            const int64_t items = ((int64_t)(la.hi - la.lo + NB - 1) / NB) * ((pitch + 63) / 64);
            up_level_f32<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(d, la, pd, (float2 *)V, S, obs);
        }
    } else {
        bind_leaves_f64<<<grid_for((int64_t)a->n_leaves * pitch), TPB, 0, s>>>(d, pd, pitch, (double2 *)V,
                                                                              (int)a->n_leaves);
        for (uint32_t L = 1; L < a->D; ++L) {
            LevelArgs la{a->level_off[L], a->level_off[L + 1], (int)L, pitch};
            const int64_t items = ((int64_t)(la.hi - la.lo + NB - 1) / NB) * ((pitch + 31) / 32);
            up_level_f64<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(d, la, pd, (double2 *)V);
        }
    }
}
static int64_t up_sequence_launches(const qkc_ac *a) {
    return a->prec == 32 ? 2 + 2 * (int64_t)(a->D - 1) : 1 + (int64_t)(a->D - 1);
}

// The launches of one downward pass over the current tile (levels D-1 .. 0).
static void launch_down_sequence(qkc_ac *a, cudaStream_t s) {
    const int64_t pitch = a->tile;
    const DevAC d = a->dev();
    const int sms = a->ctx->sm_count;
    const PassDesc *pd = a->d_desc;
    const unsigned g = (unsigned)((pitch + TPB - 1) / TPB);
    const int64_t cw = a->prec == 32 ? 64 : 32;  // columns per warp chunk
    if (a->prec == 32) seed_root<float2><<<g, TPB, 0, s>>>((float2 *)a->d_A, pitch, a->root, pd);
    else seed_root<double2><<<g, TPB, 0, s>>>((double2 *)a->d_A, pitch, a->root, pd);
    for (int L = (int)a->D - 2; L >= 0; --L) {
        const int64_t nl = a->light_off[L + 1] - a->light_off[L], nh = a->heavy_off[L + 1] - a->heavy_off[L];
        if (nl) {
            DownArgs da{a->d_light + a->light_off[L], nl, pitch};
            const int64_t items = ((nl + NB - 1) / NB) * ((pitch + cw - 1) / cw);
            const unsigned gl = grid_for(items * 32, TPB, (int64_t)sms * 8);
            if (a->prec == 32)
                down_light_f32<<<gl, TPB, 0, s>>>(d, da, pd, (const float2 *)a->d_V, a->d_S, (float2 *)a->d_A);
            else
                down_light_f64<<<gl, TPB, 0, s>>>(d, da, pd, (const double2 *)a->d_V, (double2 *)a->d_A);
        }
        if (nh) {
            DownArgs da{a->d_heavy + a->heavy_off[L], nh, pitch};
            const unsigned gh = (unsigned)std::min<int64_t>(nh * ((pitch + cw - 1) / cw), (int64_t)sms * 8);
            if (a->prec == 32)
                down_heavy_f32<<<gh, TPB, 0, s>>>(d, da, pd, (const float2 *)a->d_V, a->d_S, (float2 *)a->d_A);
            else
                down_heavy_f64<<<gh, TPB, 0, s>>>(d, da, pd, (const double2 *)a->d_V, (double2 *)a->d_A);
        }
    }
}
static int64_t down_sequence_launches(const qkc_ac *a) {
    int64_t n = 1;
    for (int L = (int)a->D - 2; L >= 0; --L)
        n += (a->light_off[L + 1] > a->light_off[L]) + (a->heavy_off[L + 1] > a->heavy_off[L]);
    return n;
}

// Capture (or reuse) the graph of one pass kind; rebuilt when the tile buffers move.
static qkc_status pass_graph(qkc_ac *a, bool down, cudaGraphExec_t *out) {
    qkc_ac::GraphSlot &g = down ? a->g_down : a->g_up;
    if (g.exec && g.V == a->d_V && g.A == a->d_A && g.pitch == a->tile && g.gen == a->scratch_gen) {
        *out = g.exec;
        return QKC_OK;
    }
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    cudaStream_t cs;
    QKC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (down) launch_down_sequence(a, cs);
        else launch_up_sequence(a, cs, a->d_V, a->d_S, a->d_obs, a->tile);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
        }
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return fail(QKC_ERR_CUDA, "qkc: capturing the %s-pass graph failed: %s", down ? "downward" : "upward",
                    cudaGetErrorString(e));
    }
    g.V = a->d_V;
    g.A = a->d_A;
    g.pitch = a->tile;
    g.gen = a->scratch_gen;
    *out = g.exec;
    return QKC_OK;
}

static qkc_status run_up(qkc_ac *a, const EvSrc &es, int64_t col0, int64_t ncols, cudaStream_t s) {
    qkc_status st;
    cudaGraphExec_t exec;
    if ((st = pass_graph(a, false, &exec))) return st;
    PassDesc desc{es, a->d_pv, a->vec_cap, col0, ncols};
    set_desc<<<1, 1, 0, s>>>(a->d_desc, desc);
    ++a->launches;
    QKC_LAUNCH_CHECK();
    const size_t ri = a->recs.size();
    if ((st = rec_begin(a, 0, es.n_active, col0, ncols, s))) return st;
    QKC_CUDA(cudaGraphLaunch(exec, s));
    a->launches += up_sequence_launches(a);
    if ((st = rec_end(a, ri, s))) return st;
    return QKC_OK;
}

// Root values of a tile's columns: the AC's root, or (step >= 0) the root of that sampling step.
static qkc_status run_roots(qkc_ac *a, int64_t col0, int64_t ncols, const int32_t *n_active, cudaStream_t s,
                            int step = -1) {
    const unsigned g = (unsigned)((ncols + TPB - 1) / TPB);
    const uint32_t r = step < 0 ? a->root : a->roots[step];
    const int Lr = step < 0 ? a->root_L : a->root_lev[step];
    if (a->prec == 32)
        root_f32<<<g, TPB, 0, s>>>((const float2 *)a->d_V, a->d_S, a->tile, r, Lr, ncols, n_active, col0, a->d_root);
    else
        root_f64<<<g, TPB, 0, s>>>((const double2 *)a->d_V, a->tile, r, ncols, n_active, col0, a->d_root);
    ++a->launches;
    QKC_LAUNCH_CHECK();
    return QKC_OK;
}

static qkc_status run_down(qkc_ac *a, int64_t ncols, cudaStream_t s) {
    qkc_status st;
    cudaGraphExec_t exec;
    if ((st = pass_graph(a, true, &exec))) return st;
    PassDesc desc{EvSrc{nullptr, nullptr, 0, 0, nullptr, nullptr, 1}, a->d_pv, a->vec_cap, 0, ncols};
    set_desc<<<1, 1, 0, s>>>(a->d_desc, desc);
    ++a->launches;
    QKC_LAUNCH_CHECK();
    const size_t ri = a->recs.size();
    if ((st = rec_begin(a, 1, nullptr, 0, ncols, s))) return st;
    QKC_CUDA(cudaGraphLaunch(exec, s));
    a->launches += down_sequence_launches(a);
    if ((st = rec_end(a, ri, s))) return st;
    return QKC_OK;
}

static qkc_status check_query(qkc_ac *a, const int32_t *col_vec, const int8_t *ev, int64_t n_cols, const char *who) {
    if (!a) return fail(QKC_ERR_ARG, "%s: null AC", who);
    if (n_cols < 0 || (n_cols > 0 && !ev)) return fail(QKC_ERR_ARG, "%s: bad evidence or column count", who);
    if (a->n_vec <= 0 && a->n_param > 0) return fail(QKC_ERR_ARG, "%s: qkc_set_params has not been called", who);
    if (!col_vec && n_cols > a->n_vec && a->n_param > 0)
        return fail(QKC_ERR_ARG, "%s: %lld columns but %lld parameter vectors and no column map", who,
                    (long long)n_cols, (long long)a->n_vec);
    (void)col_vec;
    return QKC_OK;
}

extern "C" qkc_status qkc_evaluate(qkc_ac *a, const int32_t *col_vec, const int8_t *ev, int64_t n_cols,
                                   double *out, void *stream) {
    qkc_status st = check_query(a, col_vec, ev, n_cols, "qkc_evaluate");
    if (st) return st;
    a->eval_ok = false;
    if (n_cols == 0) return QKC_OK;
    if (!out) return fail(QKC_ERR_ARG, "qkc_evaluate: out is null");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    if ((st = ensure_tile(a, n_cols)) || (st = ensure_roots(a, n_cols))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < n_cols; c0 += a->tile) {
        const int64_t nc = std::min<int64_t>(a->tile, n_cols - c0);
        EvSrc es{ev, nullptr, 0, 0, col_vec, nullptr, std::max<int64_t>(1, a->n_vec)};
        if ((st = run_up(a, es, c0, nc, s))) return st;
        if ((st = run_roots(a, c0, nc, nullptr, s))) return st;
    }
    QKC_CUDA(cudaMemcpyAsync(out, a->d_root, sizeof(double2) * n_cols, cudaMemcpyDeviceToDevice, s));
    a->eval_ok = n_cols <= a->tile;  // one tile: its node values stay for qkc_reevaluate
    a->eval_cols = n_cols;
    a->eval_colvec = col_vec;
    return QKC_OK;
}

// The dirty cone of angle slot k: its parameter leaves and every node above one of them, by level.
static qkc_status dirty_cone(qkc_ac *a, int k, qkc_ac::DirtyCone **out) {
    if (a->cones.empty()) a->cones.assign(a->n_angles, nullptr);
    if (a->cones[k]) {
        *out = a->cones[k];
        return QKC_OK;
    }
    const uint32_t N = a->N, D = a->D;
    std::vector<char> dirty(N, 0);
    std::vector<uint32_t> leaves, nodes;
    for (uint32_t i = 0; i < a->n_param; ++i)
        if (a->h_param_angle[i] == k) {
            dirty[a->n_ind + i] = 1;
            leaves.push_back(a->n_ind + i);
        }
    auto *c = new qkc_ac::DirtyCone;
    c->lvl.assign(D + 1, 0);
    for (uint32_t L = 1; L < D; ++L) {  // children sit on lower levels, so one sweep by level suffices
        for (uint32_t n = a->level_off[L]; n < a->level_off[L + 1]; ++n) {
            for (uint32_t e = a->h_child_off[n]; e < a->h_child_off[n + 1] && !dirty[n]; ++e)
                if (dirty[a->h_child[e]]) dirty[n] = 1;
            if (dirty[n]) nodes.push_back(n);
        }
        c->lvl[L + 1] = (int64_t)nodes.size();
    }
    c->nleaves = (int)leaves.size();
    int64_t b = 0;
    qkc_status st;
    if ((st = upload(&c->d_nodes, nodes.data(), nodes.size(), b)) ||
        (st = upload(&c->d_leaves, leaves.data(), leaves.size(), b))) {
        cudaFree(c->d_nodes);
        cudaFree(c->d_leaves);
        delete c;
        return st;
    }
    a->cones[k] = c;
    *out = c;
    return QKC_OK;
}

extern "C" qkc_status qkc_reevaluate(qkc_ac *a, int32_t angle_slot, const int32_t *col_vec, int64_t n_cols,
                                     double *out, void *stream) {
    if (!a || n_cols < 0 || (n_cols > 0 && !out) || angle_slot < 0 || angle_slot >= (int32_t)a->n_angles)
        return fail(QKC_ERR_ARG, "qkc_reevaluate: bad argument");
    if (n_cols == 0) return QKC_OK;
    if (!a->eval_ok || a->eval_cols != n_cols || a->eval_colvec != col_vec)
        return fail(QKC_ERR_ARG, "qkc_reevaluate: must follow qkc_evaluate (or qkc_reevaluate) on this AC with the "
                                 "same col_vec and n_cols, within one tile, and no other pass in between");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    qkc_ac::DirtyCone *cone = nullptr;
    qkc_status st = dirty_cone(a, angle_slot, &cone);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    EvSrc es{nullptr, nullptr, 0, 0, col_vec, nullptr, std::max<int64_t>(1, a->n_vec)};
    set_desc<<<1, 1, 0, s>>>(a->d_desc, PassDesc{es, a->d_pv, a->vec_cap, 0, n_cols});
    ++a->launches;
    const DevAC d = a->dev();
    const int64_t pitch = a->tile;
    if (cone->nleaves > 0) {
        const unsigned g = grid_for((int64_t)cone->nleaves * n_cols);
        if (a->prec == 32)
            rebind_param_leaves<float2><<<g, TPB, 0, s>>>(cone->d_leaves, cone->nleaves, a->d_desc, pitch,
                                                          (float2 *)a->d_V, (int)a->n_ind);
        else
            rebind_param_leaves<double2><<<g, TPB, 0, s>>>(cone->d_leaves, cone->nleaves, a->d_desc, pitch,
                                                           (double2 *)a->d_V, (int)a->n_ind);
        ++a->launches;
    }
    const int sms = a->ctx->sm_count;
    for (uint32_t L = 1; L < a->D; ++L) {
        const int64_t i0 = cone->lvl[L], i1 = cone->lvl[L + 1];
        if (i1 == i0) continue;
        const int64_t cw = a->prec == 32 ? 64 : 32;
        const int64_t items = ((i1 - i0 + NB - 1) / NB) * ((n_cols + cw - 1) / cw);
        const unsigned g = grid_for(items * 32, TPB, (int64_t)sms * 8);
        LevelArgs la{0, 0, (int)L, pitch};
        if (a->prec == 32)
            up_list_f32<<<g, TPB, 0, s>>>(d, la, cone->d_nodes + i0, i1 - i0, a->d_desc, (float2 *)a->d_V, a->d_S);
        else
            up_list_f64<<<g, TPB, 0, s>>>(d, la, cone->d_nodes + i0, i1 - i0, a->d_desc, (double2 *)a->d_V);
        ++a->launches;
    }
    QKC_LAUNCH_CHECK();
    if ((st = run_roots(a, 0, n_cols, nullptr, s))) return st;
    QKC_CUDA(cudaMemcpyAsync(out, a->d_root, sizeof(double2) * n_cols, cudaMemcpyDeviceToDevice, s));
    return QKC_OK;
}

extern "C" qkc_status qkc_marginals(qkc_ac *a, const int32_t *col_vec, const int8_t *ev, int64_t n_cols,
                                    double *root_out, double *marg_out, void *stream) {
    qkc_status st = check_query(a, col_vec, ev, n_cols, "qkc_marginals");
    if (st) return st;
    a->eval_ok = false;
    if (a->kind == QKC_AC_DENSITY_STEPS)  // the downward pass needs the root alone on the top level
        return fail(QKC_ERR_UNSUPPORTED, "qkc_marginals: not on a DENSITY_STEPS AC (use its DENSITY AC)");
    if (n_cols == 0) return QKC_OK;
    if (!marg_out) return fail(QKC_ERR_ARG, "qkc_marginals: marg_out is null");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    if ((st = ensure_tile(a, n_cols)) || (st = ensure_roots(a, n_cols)) || (st = ensure_adj(a))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < n_cols; c0 += a->tile) {
        const int64_t nc = std::min<int64_t>(a->tile, n_cols - c0);
        EvSrc es{ev, nullptr, 0, 0, col_vec, nullptr, std::max<int64_t>(1, a->n_vec)};
        if ((st = run_up(a, es, c0, nc, s))) return st;
        if ((st = run_roots(a, c0, nc, nullptr, s))) return st;
        if ((st = run_down(a, nc, s))) return st;
        const int64_t work = (int64_t)a->n_ind * nc;
        if (a->prec == 32)
            gather_marginals<float2><<<grid_for(work), TPB, 0, s>>>((const float2 *)a->d_A, a->tile, (int)a->n_ind, nc,
                                                                   c0, (double2 *)marg_out);
        else
            gather_marginals<double2><<<grid_for(work), TPB, 0, s>>>((const double2 *)a->d_A, a->tile, (int)a->n_ind,
                                                                    nc, c0, (double2 *)marg_out);
        ++a->launches;
        QKC_LAUNCH_CHECK();
    }
    if (root_out)
        QKC_CUDA(cudaMemcpyAsync(root_out, a->d_root, sizeof(double2) * n_cols, cudaMemcpyDeviceToDevice, s));
    return QKC_OK;
}

extern "C" qkc_status qkc_gradient(qkc_ac *a, const int32_t *col_vec, const int8_t *ev, const double *weight,
                                   int64_t n_cols, int64_t n_vectors, double *value, double *grad, void *stream) {
    qkc_status st = check_query(a, col_vec, ev, n_cols, "qkc_gradient");
    if (st) return st;
    a->eval_ok = false;
    if (a->kind == QKC_AC_DENSITY_STEPS)
        return fail(QKC_ERR_UNSUPPORTED, "qkc_gradient: not on a DENSITY_STEPS AC (use its DENSITY AC)");
    if (!col_vec || !weight || !value || !grad || n_vectors <= 0 || n_vectors > a->n_vec)
        return fail(QKC_ERR_ARG, "qkc_gradient: needs col_vec, weight, value, grad and 0 < n_vectors <= bound vectors");
    if (!a->last_angles) return fail(QKC_ERR_ARG, "qkc_gradient: qkc_set_params has not been called");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    QKC_CUDA(cudaMemsetAsync(value, 0, sizeof(double) * n_vectors, s));
    QKC_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * n_vectors * std::max<uint32_t>(1, a->n_angles), s));
    if (n_cols == 0) return QKC_OK;
    if ((st = ensure_tile(a, n_cols)) || (st = ensure_roots(a, n_cols)) || (st = ensure_adj(a))) return st;
    for (int64_t c0 = 0; c0 < n_cols; c0 += a->tile) {
        const int64_t nc = std::min<int64_t>(a->tile, n_cols - c0);
        EvSrc es{ev, nullptr, 0, 0, col_vec, nullptr, std::max<int64_t>(1, a->n_vec)};
        if ((st = run_up(a, es, c0, nc, s))) return st;
        if ((st = run_roots(a, c0, nc, nullptr, s))) return st;
        if ((st = run_down(a, nc, s))) return st;
        const int64_t work = (int64_t)(a->n_param + 1) * nc;
        if (a->prec == 32)
            gradient_accumulate<float2><<<grid_for(work), TPB, 0, s>>>(a->dev(), (const float2 *)a->d_A, a->tile, nc, c0,
                                                                      col_vec, n_vectors, a->last_angles, weight,
                                                                      a->d_root, value, grad);
        else
            gradient_accumulate<double2><<<grid_for(work), TPB, 0, s>>>(a->dev(), (const double2 *)a->d_A, a->tile, nc,
                                                                       c0, col_vec, n_vectors, a->last_angles, weight,
                                                                       a->d_root, value, grad);
        ++a->launches;
        QKC_LAUNCH_CHECK();
    }
    return QKC_OK;
}

// ---- sampling
static qkc_status ensure_sampling(qkc_ac *a, int64_t n_samples, int64_t n_groups) {
    if (n_samples <= a->samp_cap && n_groups <= a->grp_cap) return QKC_OK;
    QKC_CUDA(cudaDeviceSynchronize());
    const int64_t ns = std::max(n_samples, a->samp_cap), ng = std::max(n_groups, a->grp_cap);
    cudaFree(a->d_s_group); cudaFree(a->d_s_bits); cudaFree(a->d_flag); cudaFree(a->d_pos); cudaFree(a->d_bsum);
    cudaFree(a->d_gcount);
    for (int i = 0; i < 2; ++i) { cudaFree(a->d_g_vec[i]); cudaFree(a->d_g_prefix[i]); cudaFree(a->d_g_P[i]); }
    a->samp_cap = a->grp_cap = 0;
    const int64_t nflag = 2 * ng;
    const int64_t nblk = (nflag + 1023) / 1024 + 1;
    QKC_CUDA(dalloc(&a->d_s_group, ns));
    QKC_CUDA(dalloc(&a->d_s_bits, ns));
    QKC_CUDA(dalloc(&a->d_flag, nflag));
    QKC_CUDA(dalloc(&a->d_pos, nflag));
    QKC_CUDA(dalloc(&a->d_bsum, nblk));
    QKC_CUDA(dalloc(&a->d_gcount, 2));
    for (int i = 0; i < 2; ++i) {
        QKC_CUDA(dalloc(&a->d_g_vec[i], ng));
        QKC_CUDA(dalloc(&a->d_g_prefix[i], ng));
        QKC_CUDA(dalloc(&a->d_g_P[i], ng));
    }
    if (a->kind == QKC_AC_TRAJECTORY) {
        for (int i = 0; i < 2; ++i) {
            cudaFree(a->d_g_traj[i]);
            a->d_g_traj[i] = nullptr;
            QKC_CUDA(dalloc(&a->d_g_traj[i], ng));
        }
        cudaFree(a->d_traj);
        cudaFree(a->d_err);
        cudaFree(a->d_rep);
        cudaFree(a->d_table);
        a->d_traj = nullptr;
        a->d_err = a->d_rep = nullptr;
        a->d_table = nullptr;
        a->table_size = 1;
        while (a->table_size < 2 * (uint64_t)ns) a->table_size <<= 1;
        QKC_CUDA(dalloc(&a->d_traj, (size_t)ns * (size_t)std::max(1, a->n_noise)));
        QKC_CUDA(dalloc(&a->d_err, ns));
        QKC_CUDA(dalloc(&a->d_rep, ns));
        QKC_CUDA(dalloc(&a->d_table, a->table_size));
    }
    a->samp_cap = ns;
    a->grp_cap = ng;
    return QKC_OK;
}


// ---- memoised sampling (host side)
// The six shift masks of Warren's mask-compress (Hacker's Delight, 2nd ed., Sec. 7-4): round i
// moves the bits of mv[i] right by 2^i; the count of mask zeros to the right of each bit is
// formed by a parallel prefix XOR.
static void compress_masks(uint64_t m, uint64_t mv[6]) {
    uint64_t mk = ~m << 1;
    for (int i = 0; i < 6; ++i) {
        uint64_t mp = mk ^ (mk << 1);
        mp ^= mp << 2;
        mp ^= mp << 4;
        mp ^= mp << 8;
        mp ^= mp << 16;
        mp ^= mp << 32;
        const uint64_t v = mp & m;
        mv[i] = v;
        m = (m ^ v) | (v >> (1 << i));
        mk &= ~mp;
    }
}

static qkc_ac::MemoMeta *memo_meta(qkc_ac *a, int cap, qkc_status *st) {
    *st = QKC_OK;
    if ((int)a->memo.size() <= cap) a->memo.resize(cap + 1, nullptr);
    if (a->memo[cap]) return a->memo[cap];
    auto *m = new qkc_ac::MemoMeta;
    m->cap = cap;
    const int nq = (int)a->n_qubits;
    const uint32_t N = a->N, D = a->D;
    std::vector<uint32_t> an, bn, emask;
    std::vector<uint2> bdesc;
    std::vector<uint4> brec;  // edge records of tier-B nodes (layout: BChild)
    std::vector<uint16_t> lev(N);
    for (uint32_t L = 0; L < D; ++L)
        for (uint32_t n = a->level_off[L]; n < a->level_off[L + 1]; ++n) lev[n] = (uint16_t)L;
    std::vector<int64_t> offu;
    std::vector<MemoAGroup> grp;
    std::vector<KeyPlan> kplan, aplan, bplan;
    std::vector<MemoARunLevel> runlv;
    m->a_items.assign(nq, {});
    m->b_items.assign(nq, {});
    std::vector<MemoBRunLevel> brunlv;
    std::vector<MemoARunLevel> alllv;
    std::vector<MemoAStep> asteps;
    std::vector<int32_t> rst;
    std::vector<uint16_t> bcl;
    std::vector<uint32_t> bclo;
    std::vector<int32_t> plan_of;  // per node: its key plan in this step, -1 if none yet
    std::vector<int64_t> row_of;   // per node: its tier-B row in this step
    std::vector<char> reach;       // per node: reachable from this step's root
    std::vector<uint32_t> dfs;
    emask.assign((size_t)nq * a->E, 0u);
    const std::vector<uint32_t> &child_off = a->h_child_off, &child = a->h_child;
    m->a_lvl.assign(nq, std::vector<int64_t>(D + 1, 0));
    m->u_lvl = m->a_lvl;
    m->b_lvl = m->a_lvl;
    m->g_lvl = m->a_lvl;
    m->t_lvl = m->a_lvl;
    m->floor0.assign(nq, std::vector<uint8_t>(D, 0));
    std::vector<std::pair<int, uint32_t>> al;  // (key width, node) of one level's tier A
    for (int j = 0; j < nq; ++j) {
        const uint64_t jmask = j == 0 ? 0ull : (j >= 64 ? ~0ull : ((1ull << j) - 1ull));
        // a node is memoised when its key has at most t bits: early steps have at most V 2^j
        // groups, so t = j - MEMO_MARGIN keeps the key space 2^MEMO_MARGIN times smaller; later
        // steps stop at the cap, about half the shots per vector
        const int t = std::min(cap, std::max(0, j - MEMO_MARGIN));
        m->a_base.push_back((int64_t)an.size());
        m->b_base.push_back((int64_t)bn.size());
        m->g_base.push_back((int64_t)grp.size());
        m->kp_base.push_back((int64_t)kplan.size());
        m->ap_base.push_back((int64_t)aplan.size());
        m->bp_base.push_back((int64_t)bplan.size());
        m->br_base.push_back((int64_t)brec.size());
        plan_of.assign(N, -1);
        row_of.assign(N, -1);
        // the step's nodes: those its root reaches (all of a single-root AC's computed nodes)
        reach.assign(N, 0);
        dfs.assign(1, a->roots[j]);
        reach[a->roots[j]] = 1;
        while (!dfs.empty()) {
            const uint32_t v = dfs.back();
            dfs.pop_back();
            for (uint32_t e = child_off[v]; e < child_off[v + 1]; ++e)
                if (!reach[child[e]]) {
                    reach[child[e]] = 1;
                    dfs.push_back(child[e]);
                }
        }
        m->offu_base.push_back((int64_t)offu.size());
        const size_t ob = offu.size();
        offu.resize(ob + N, -1);
        int64_t units = 0;
        double abytes = 0.0, bbytes = 0.0, aedges = 0.0, bedges = 0.0;
        for (uint32_t L = 0; L < D; ++L) {
            // leaves are always memoised (at most one key bit, V * 2 slots): the memoised pass
            // binds no leaf per group, so every leaf a per-group node reads must be here
            al.clear();
            for (uint32_t n = a->level_off[L]; n < a->level_off[L + 1]; ++n) {
                if (!reach[n]) continue;
                const int k = __builtin_popcountll(a->sigma[n] & jmask);
                if (k <= t || n < a->n_leaves) al.push_back({k, n});
            }
            // widest keys first; within a width, node order
            std::stable_sort(al.begin(), al.end(), [](const std::pair<int, uint32_t> &x,
                                                      const std::pair<int, uint32_t> &y) { return x.first > y.first; });
            const int64_t u0 = units, i0 = (int64_t)an.size();
            int64_t th = 0;  // threads of the level (one per slot, or per four slots from MEMO_QUAD_K)
            for (size_t i = 0; i < al.size(); ++i) {
                const int k = al[i].first;
                const uint32_t n = al[i].second;
                if (i == 0 || k != al[i - 1].first)
                    grp.push_back(MemoAGroup{(uint32_t)th, (uint32_t)((int64_t)an.size() - i0), (uint32_t)k,
                                             (uint32_t)(units - u0)});
                th += k >= MEMO_QUAD_K ? (1ll << k) / 4 : (1ll << k);
                offu[ob + n] = units;
                an.push_back(n);
                units += 1ll << k;
                const double deg = (double)(child_off[n + 1] - child_off[n]);
                abytes += (double)(1ll << k) * (deg + 1.0);
                aedges += (double)(1ll << k) * deg;
                const uint64_t rn = a->sigma[n] & jmask;
                for (uint32_t e = child_off[n]; e < child_off[n + 1]; ++e) {
                    const uint64_t rc = a->sigma[child[e]] & jmask;
                    uint32_t me = 0;  // positions of rc's qubits among rn's, in qubit order
                    int pos = 0;
                    for (uint64_t r = rn; r; r &= r - 1, ++pos)
                        if (rc & (r & (~r + 1))) me |= 1u << pos;
                    const uint32_t run = me ? me >> __builtin_ctz(me) : 0u;
                    if (run & (run + 1u)) {  // scattered: a compress plan (at most 2^MEMO_APLANS per step)
                        int64_t idx = -1;
                        for (int64_t i = m->ap_base[j]; i < (int64_t)aplan.size() && idx < 0; ++i)
                            if (aplan[i].m == me) idx = i - m->ap_base[j];
                        if (idx < 0 && (int64_t)aplan.size() - m->ap_base[j] < (1 << MEMO_APLANS)) {
                            KeyPlan kp{};
                            kp.m = me;
                            compress_masks(me, kp.mv);
                            kp.k = (uint32_t)__builtin_popcount(me);
                            idx = (int64_t)aplan.size() - m->ap_base[j];
                            aplan.push_back(kp);
                        }
                        if (idx >= 0) me = 0x80000000u | (uint32_t)idx;
                    }
                    emask[(size_t)j * a->E + e] = me;
                }
            }
            for (uint32_t n = a->level_off[L]; n < a->level_off[L + 1]; ++n) {
                if (!reach[n] || offu[ob + n] >= 0) continue;
                row_of[n] = (int64_t)bn.size() - m->b_base[j];  // tier-B values are stored by row
                bn.push_back(n);
                const uint32_t deg = child_off[n + 1] - child_off[n];
                if (deg > 0xffffffu) {  // a descriptor holds a 24-bit degree: no memoised passes
                    delete m;
                    return nullptr;
                }
                bdesc.push_back(make_uint2((uint32_t)((int64_t)brec.size() - m->br_base[j]),
                                           deg | ((uint32_t)a->h_op[n] << 24)));
                bbytes += (double)(child_off[n + 1] - child_off[n]) + 1.0;
                bedges += (double)(child_off[n + 1] - child_off[n]);
                for (uint32_t e = child_off[n]; e < child_off[n + 1]; ++e) {
                    const uint32_t c = child[e];
                    const int64_t oc = offu[ob + c];
                    if (oc < 0) {  // a tier-B child: its row
                        brec.push_back(make_uint4(0x80000000u | (uint32_t)row_of[c], lev[c], 0u, 0u));
                    } else {
                        m->floor0[j][L] = 1;
                        if (plan_of[c] < 0) {
                            KeyPlan kp{};
                            kp.off = oc;
                            kp.m = a->sigma[c] & jmask;
                            compress_masks(kp.m, kp.mv);
                            kp.k = (uint32_t)__builtin_popcountll(kp.m);
                            kp.mid = -1;  // a row of the group-key table for this support, when there is room
                            for (int64_t i = m->bp_base[j]; i < (int64_t)bplan.size() && kp.mid < 0; ++i)
                                if (bplan[i].m == kp.m) kp.mid = (int32_t)(i - m->bp_base[j]);
                            if (kp.mid < 0 && (int64_t)bplan.size() - m->bp_base[j] < MEMO_BKEYS) {
                                kp.mid = (int32_t)((int64_t)bplan.size() - m->bp_base[j]);
                                bplan.push_back(kp);
                            }
                            plan_of[c] = (int32_t)((int64_t)kplan.size() - m->kp_base[j]);
                            kplan.push_back(kp);
                        }
                        const KeyPlan &kp = kplan[m->kp_base[j] + plan_of[c]];
                        brec.push_back(make_uint4((uint32_t)plan_of[c] + 1u, kp.k | ((uint32_t)(kp.mid + 1) << 8),
                                                  (uint32_t)((uint64_t)kp.off & 0xffffffffu),
                                                  (uint32_t)((uint64_t)kp.off >> 32)));
                    }
                }
            }
            m->a_lvl[j][L + 1] = (int64_t)an.size() - m->a_base[j];
            m->u_lvl[j][L + 1] = units;
            m->b_lvl[j][L + 1] = (int64_t)bn.size() - m->b_base[j];
            m->g_lvl[j][L + 1] = (int64_t)grp.size() - m->g_base[j];
            m->t_lvl[j][L] = th;
        }
        m->bp_cnt.push_back((int64_t)bplan.size() - m->bp_base[j]);
        {  // tier-B launches: consecutive small levels form one run (FP32: a warp per 64-column chunk walks
           // them), of at most MEMO_RUN_LV levels and MEMO_RUN_NODES nodes
            std::vector<uint32_t> pend;
            int64_t pend_nodes = 0;
            auto flush = [&]() {
                if (pend.size() >= 2) {
                    m->b_items[j].push_back({-1, (int64_t)brunlv.size(), (int)pend.size(), pend_nodes});
                    for (uint32_t L : pend)
                        brunlv.push_back(MemoBRunLevel{(uint32_t)m->b_lvl[j][L],
                                                       (uint32_t)(m->b_lvl[j][L + 1] - m->b_lvl[j][L]), (int32_t)L,
                                                       (int32_t)m->floor0[j][L]});
                } else if (pend.size() == 1) {
                    m->b_items[j].push_back({(int)pend[0], 0, 0});
                }
                pend.clear();
                pend_nodes = 0;
            };
            for (uint32_t L = 1; L < D; ++L) {
                const int64_t cnt = m->b_lvl[j][L + 1] - m->b_lvl[j][L];
                if (cnt == 0) continue;
                if (a->prec == 32 && cnt <= MEMO_RUN_B) {
                    if ((int)pend.size() == MEMO_RUN_LV || pend_nodes + cnt > MEMO_RUN_NODES) flush();
                    pend.push_back(L);
                    pend_nodes += cnt;
                } else {
                    flush();
                    m->b_items[j].push_back({(int)L, 0, 0});
                }
            }
            flush();
            int fz = 0;
            const auto &bi = m->b_items[j];
            if (!bi.empty() && bi.front().cnt > 0 && m->bp_cnt[j] > 0) fz |= 1;
            if (!bi.empty() && bi.back().cnt > 0 && row_of[a->roots[j]] >= 0 &&
                brunlv.back().L == (int32_t)a->root_lev[j])
                fz |= 2;
            m->fuse.push_back(fz);
        }
        {  // every tier-A level of the step, in order (memoA_all)
            MemoAStep st{m->a_base[j], m->g_base[j], (uint32_t)alllv.size(), 0u};
            for (uint32_t L = 0; L < D; ++L) {
                if (m->a_lvl[j][L + 1] == m->a_lvl[j][L]) continue;
                alllv.push_back(MemoARunLevel{(uint32_t)m->a_lvl[j][L], (uint32_t)m->g_lvl[j][L],
                                              (uint32_t)(m->g_lvl[j][L + 1] - m->g_lvl[j][L]),
                                              (uint32_t)m->t_lvl[j][L], m->u_lvl[j][L]});
                m->all_T = std::max<int64_t>(m->all_T, m->t_lvl[j][L]);
            }
            st.lv1 = (uint32_t)alllv.size();
            asteps.push_back(st);
        }
        {  // tier-A launches: consecutive small levels form one run (a block per vector walks them)
            std::vector<uint32_t> pend;
            auto flush = [&]() {
                if (pend.size() >= 2) {
                    m->a_items[j].push_back({-1, (int64_t)runlv.size(), (int)pend.size()});
                    for (uint32_t L : pend)
                        runlv.push_back(MemoARunLevel{(uint32_t)m->a_lvl[j][L], (uint32_t)m->g_lvl[j][L],
                                                      (uint32_t)(m->g_lvl[j][L + 1] - m->g_lvl[j][L]),
                                                      (uint32_t)m->t_lvl[j][L], m->u_lvl[j][L]});
                } else if (pend.size() == 1) {
                    m->a_items[j].push_back({(int)pend[0], 0, 0});
                }
                pend.clear();
            };
            for (uint32_t L = 0; L < D; ++L) {
                if (m->a_lvl[j][L + 1] == m->a_lvl[j][L]) continue;
                if (m->t_lvl[j][L] <= MEMO_RUN_T) {
                    pend.push_back(L);
                } else {
                    flush();
                    m->a_items[j].push_back({(int)L, 0, 0});
                }
            }
            flush();
        }
        {  // level scales: per level with tier-B nodes, its child levels that hold tier-B nodes in this
           // step (no other level is computed here); observed exponents reset: the levels of per-level
           // launches that form their scales inline (they take a maximum over node blocks; a run stores
           // its levels' exponents, and the scale kernel resets its own level)
            auto has_b = [&](uint32_t L) { return m->b_lvl[j][L + 1] > m->b_lvl[j][L]; };
            for (uint32_t L = 0; L < D; ++L) {
                bclo.push_back((uint32_t)bcl.size());
                if (L == 0 || !has_b(L)) continue;
                for (uint32_t k = a->h_cl_off[L]; k < a->h_cl_off[L + 1]; ++k)
                    if (has_b((uint32_t)a->h_cl[k])) bcl.push_back(a->h_cl[k]);
            }
            bclo.push_back((uint32_t)bcl.size());
            m->rst_base.push_back((int64_t)rst.size());
            if (a->prec == 32 && m->b_lvl[j][D] <= MEMO_INLINE_SCALE_B)
                for (const auto &it : m->b_items[j])
                    if (it.cnt == 0) rst.push_back((int32_t)it.L);
            m->rst_cnt.push_back((int64_t)rst.size() - m->rst_base[j]);
        }
        m->root_row.push_back(row_of[a->roots[j]]);
        m->max_rows = std::max<int64_t>(m->max_rows, (int64_t)bn.size() - m->b_base[j]);
        m->a_bytes_slot.push_back(abytes * (double)a->elem());
        m->b_bytes_col.push_back(bbytes * (double)a->elem());
        m->a_edges_slot.push_back(aedges);
        m->b_edges_col.push_back(bedges);
        m->max_units = std::max(m->max_units, units);
        m->unit_base.push_back(m->unit_base.back() + units);
    }
    if (m->max_units >= 0xffffffffll) {  // block offsets are stored in 32 bits per edge
        delete m;
        *st = QKC_OK;
        return nullptr;
    }
    std::vector<MemoALvlStep> lvs;  // per level, the steps with tier-A nodes there (memoA_lvl_all)
    m->lvs_off.assign(1, 0);
    for (uint32_t L = 0; L < D; ++L) {
        for (int j = 0; j < nq; ++j) {
            if (m->a_lvl[j][L + 1] == m->a_lvl[j][L]) continue;
            lvs.push_back(MemoALvlStep{m->a_base[j] + m->a_lvl[j][L], m->g_base[j] + m->g_lvl[j][L], m->u_lvl[j][L],
                                       (uint32_t)m->t_lvl[j][L],
                                       (uint32_t)(m->g_lvl[j][L + 1] - m->g_lvl[j][L]), (int32_t)j, 0});
        }
        m->lvs_off.push_back((int64_t)lvs.size());
    }
    std::vector<int32_t> aorder(nq);  // steps by tier-A work, largest first (memoA_all)
    for (int j = 0; j < nq; ++j) aorder[j] = j;
    std::stable_sort(aorder.begin(), aorder.end(),
                     [&](int x, int y) { return m->a_bytes_slot[x] > m->a_bytes_slot[y]; });
    int64_t dummy = 0;
    if ((*st = upload(&m->d_a_nodes, an.data(), an.size(), dummy)) ||
        (*st = upload(&m->d_a_grp, grp.data(), grp.size(), dummy)) ||
        (*st = upload(&m->d_offu, offu.data(), offu.size(), dummy)) ||
        (*st = upload(&m->d_emask, emask.data(), emask.size(), dummy)) ||
        (*st = upload(&m->d_runlv, runlv.data(), runlv.size(), dummy)) ||
        (*st = upload(&m->d_brunlv, brunlv.data(), brunlv.size(), dummy)) ||
        (*st = upload(&m->d_rst, rst.data(), rst.size(), dummy)) ||
        (*st = upload(&m->d_bclo, bclo.data(), bclo.size(), dummy)) ||
        (*st = upload(&m->d_alllv, alllv.data(), alllv.size(), dummy)) ||
        (*st = upload(&m->d_lvs, lvs.data(), lvs.size(), dummy)) ||
        (*st = upload(&m->d_asteps, asteps.data(), asteps.size(), dummy)) ||
        (*st = upload(&m->d_aorder, aorder.data(), aorder.size(), dummy)) ||
        (*st = upload(&m->d_bcl, bcl.data(), bcl.size(), dummy)) ||
        (*st = upload(&m->d_bdesc, bdesc.data(), bdesc.size(), dummy)) ||
        (*st = upload(&m->d_brec, brec.data(), brec.size(), dummy)) ||
        (*st = upload(&m->d_kplan, kplan.data(), kplan.size(), dummy)) ||
        (*st = upload(&m->d_aplan, aplan.data(), aplan.size(), dummy)) ||
        (*st = upload(&m->d_bplan, bplan.data(), bplan.size(), dummy))) {
        cudaFree(m->d_a_nodes); cudaFree(m->d_a_grp); cudaFree(m->d_offu);
        cudaFree(m->d_emask); cudaFree(m->d_runlv); cudaFree(m->d_brunlv); cudaFree(m->d_rst); cudaFree(m->d_alllv); cudaFree(m->d_lvs); cudaFree(m->d_asteps); cudaFree(m->d_aorder); cudaFree(m->d_bclo); cudaFree(m->d_bcl); cudaFree(m->d_bdesc); cudaFree(m->d_brec); cudaFree(m->d_kplan); cudaFree(m->d_aplan); cudaFree(m->d_bplan);
        delete m;
        return nullptr;
    }
    a->memo[cap] = m;
    return m;
}

// Launch a kernel of the sampling chain with programmatic stream serialisation (the kernel begins with
// pdl_begin, so it touches memory only once the kernel before it has completed).
template <typename... P, typename... A>
static void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);  // a failure is left for the caller's launch check
}

// Launch sequences of a memoised pass, captured once per (cap, step) as CUDA graphs.  They
// read the memo descriptor (vectors, step, slots) and the pass descriptor (tile columns), and
// their grids do not depend on the number of vectors or columns.
static void launch_memoA_sequence(qkc_ac *a, const qkc_ac::MemoMeta *m, int j, cudaStream_t s) {
    const DevAC d = a->dev();
    const MemoDesc *md_j = a->d_mdesc + j;
    const unsigned g = (unsigned)(a->ctx->sm_count * 16);
    const unsigned gr = (unsigned)(a->ctx->sm_count * 4);  // run kernels: a block per vector, grid-stride
    const uint32_t *nodes_j = m->d_a_nodes + m->a_base[j];
    const MemoAGroup *grp_j = m->d_a_grp + m->g_base[j];
    for (const auto &it : m->a_items[j]) {
        if (it.cnt > 0) {
            if (a->prec == 32)
                launch_pdl(memoA_run<float2>, gr, TPB, 0, s, d, md_j, nodes_j, grp_j, m->d_runlv + it.off, it.cnt);
            else
                launch_pdl(memoA_run<double2>, gr, TPB, 0, s, d, md_j, nodes_j, grp_j, m->d_runlv + it.off, it.cnt);
            continue;
        }
        const uint32_t L = (uint32_t)it.L;
        const int64_t i0 = m->a_lvl[j][L];
        const int64_t u0 = m->u_lvl[j][L];
        const uint32_t T = (uint32_t)m->t_lvl[j][L];
        const uint32_t *nodes = nodes_j + i0;
        const MemoAGroup *gp = grp_j + m->g_lvl[j][L];
        const int ng = (int)(m->g_lvl[j][L + 1] - m->g_lvl[j][L]);
        if (a->prec == 32) launch_pdl(memoA_level<float2>, g, TPB, 0, s, d, md_j, nodes, gp, ng, u0, T);
        else launch_pdl(memoA_level<double2>, g, TPB, 0, s, d, md_j, nodes, gp, ng, u0, T);
    }
}
static int64_t memoA_launches(const qkc_ac *a, const qkc_ac::MemoMeta *m, int j) {
    (void)a;
    return (int64_t)m->a_items[j].size();
}
static void launch_memoB_sequence(qkc_ac *a, const qkc_ac::MemoMeta *m, int j, cudaStream_t s) {
    const DevAC d = a->dev();
    const MemoDesc *md_j = a->d_mdesc + j;
    const int sms = a->ctx->sm_count;
    const uint32_t D = a->D;
    const int64_t pitch = a->tile;
    if (m->b_lvl[j][D] > 0) {
        const unsigned gs = (unsigned)((pitch + TPB - 1) / TPB);
        if (m->bp_cnt[j] > 0 && !(m->fuse[j] & 1)) launch_pdl(memo_keys, gs, TPB, 0, s, a->d_desc, md_j);
        // FP32 scales: only levels with tier-B nodes are computed, so every level's observed
        // exponent starts empty and the scale kernel runs for those levels alone
        if (a->prec == 32 && m->rst_cnt[j] > 0)
            launch_pdl(obs_reset, (unsigned)((m->rst_cnt[j] * pitch + TPB - 1) / TPB), TPB, 0, s,
                a->d_obs, m->d_rst + m->rst_base[j], (int)m->rst_cnt[j], pitch);
        const bool inline_scale = m->b_lvl[j][D] <= MEMO_INLINE_SCALE_B;
        const uint2 *bd_j = m->d_bdesc + m->b_base[j];
        const uint32_t *cl_off_j = m->d_bclo + (size_t)j * (D + 1);
        const size_t nit = m->b_items[j].size();
        for (size_t ii = 0; ii < nit; ++ii) {
            const auto &it = m->b_items[j][ii];
            if (it.cnt > 0) {  // a run of small levels (FP32): a warp per 64-column chunk walks them
                const int64_t chunks = (pitch + 63) / 64;
                const unsigned g = (unsigned)std::min<int64_t>((chunks + TPB / 32 - 1) / (TPB / 32), (int64_t)sms * 8);
                const int fz = (ii == 0 ? (m->fuse[j] & 1) : 0) | (ii + 1 == nit ? (m->fuse[j] & 2) : 0);
                launch_pdl(memoB_run_f32, g, TPB, run_smem_bytes(it.cnt, it.nodes), s, m->d_brunlv + it.off, it.cnt, bd_j,
                                                                                a->d_desc, md_j, pitch,
                                                 (float2 *)a->d_V, a->d_S, a->d_obs, fz, m->root_row[j],
                                                 a->root_lev[j], a->d_root);
                launch_pdl(memoB_runc_f32, g, TPB, run_smem_bytes(it.cnt, it.nodes), s, m->d_brunlv + it.off, it.cnt, bd_j,
                                                                                a->d_desc, md_j, pitch,
                                                 (float2 *)a->d_V, a->d_S, a->d_obs, fz, m->root_row[j],
                                                 a->root_lev[j], a->d_root);
                continue;
            }
            const uint32_t L = (uint32_t)it.L;
            const int64_t b0 = m->b_lvl[j][L], b1 = m->b_lvl[j][L + 1];
            if (a->prec == 32 && !inline_scale)
                launch_pdl(level_scale_kernel, gs, TPB, 0, s, cl_off_j, m->d_bcl, (int)L, pitch, m->floor0[j][L], a->d_S,
                                                      a->d_obs);
            // lo: the level's first tier-B row; hi: bit 0 reads tier-A values, bit 1 scale formed inline
            LevelArgs la{(uint32_t)b0, (uint32_t)m->floor0[j][L] | (inline_scale ? 2u : 0u), (int)L, pitch};
            if (a->prec == 32) {  // at most one wave of resident blocks (the kernel splits the last round)
                const int64_t items = ((b1 - b0 + NBB - 1) / NBB) * ((pitch + 127) / 128);
                const unsigned g = grid_for(items * 8 * 32, TPB, (int64_t)sms * a->ctx->memoB_blocks_per_sm);
                launch_pdl(memoB_level_f32, g, TPB, 0, s, d, la, bd_j + b0, b1 - b0, a->d_desc, md_j, (float2 *)a->d_V,
                                                   a->d_S, a->d_obs);
            } else {  // a warp per 32 nodes x 32 columns, grid-striding
                const int64_t items = ((b1 - b0 + NBB - 1) / NBB) * ((pitch + 31) / 32);
                const unsigned g = grid_for(items * 32, TPB, (int64_t)sms * 8);
                launch_pdl(memoB_level_f64, g, TPB, 0, s, la, bd_j + b0, b1 - b0, a->d_desc, md_j, (double2 *)a->d_V);
            }
        }
    }
    if (!(m->fuse[j] & 2))
        launch_pdl(memo_root, (unsigned)((pitch + TPB - 1) / TPB), TPB, 0, s, md_j, a->d_desc, a->roots[j], a->root_lev[j],
                                                                      m->root_row[j], a->d_V, a->d_S, pitch,
                                                                      a->prec == 32, a->d_root);
}
static int64_t memoB_launches(const qkc_ac *a, const qkc_ac::MemoMeta *m, int j) {
    int64_t n = (m->fuse[j] & 2) ? 0 : 1;
    if (m->b_lvl[j][a->D] > 0) {
        n += (a->prec == 32 && m->rst_cnt[j] > 0) ? 1 : 0;
        n += m->bp_cnt[j] > 0 && !(m->fuse[j] & 1);
        const int per = (a->prec == 32 && m->b_lvl[j][a->D] > MEMO_INLINE_SCALE_B) ? 2 : 1;
        for (const auto &it : m->b_items[j]) n += it.cnt > 0 ? 2 : per;  // a run: both run kernels
    }
    return n;
}

static qkc_status memo_graph(qkc_ac *a, qkc_ac::MemoMeta *m, int j, bool partB, cudaGraphExec_t *out) {
    auto &slot = partB ? m->gB : m->gA;
    if ((int)slot.size() <= j) slot.resize(a->n_qubits);
    auto &g = slot[j];
    if (g.exec && (!partB || (g.V == a->d_V && g.A == (const void *)a->d_root && g.pitch == a->tile &&
                              g.gen == a->scratch_gen))) {
        *out = g.exec;
        return QKC_OK;
    }
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    cudaStream_t cs;
    QKC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (partB) launch_memoB_sequence(a, m, j, cs);
        else launch_memoA_sequence(a, m, j, cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
        }
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return fail(QKC_ERR_CUDA, "qkc: capturing a memoised-pass graph failed: %s", cudaGetErrorString(e));
    }
    g.V = a->d_V;
    g.A = a->d_root;
    g.pitch = a->tile;
    g.gen = a->scratch_gen;
    *out = g.exec;
    return QKC_OK;
}

// Step j's memo descriptor (into a->d_mdesc + j).  resident: every step's tier-A slots are held at
// once, step j's from unit unit_base[j]; else every step's start at unit 0.
static void set_memo_step(qkc_ac *a, const qkc_ac::MemoMeta *m, int j, int clamp, int64_t n_vec, bool resident,
                          cudaStream_t s) {
    const uint64_t jmask = j == 0 ? 0ull : (j >= 64 ? ~0ull : ((1ull << j) - 1ull));
    char *VA = static_cast<char *>(a->d_VA) + (resident ? n_vec * m->unit_base[j] * (int64_t)a->elem() : 0);
    MemoDesc md{n_vec,    j,         clamp, jmask, a->d_pv, a->vec_cap, VA, m->d_offu + m->offu_base[j],
                a->d_sigma, m->d_emask + (size_t)j * a->E, m->d_brec + m->br_base[j],
                m->d_kplan + m->kp_base[j], m->d_aplan + m->ap_base[j], m->d_bplan + m->bp_base[j],
                (int32_t)m->bp_cnt[j], a->d_keys, a->tile, m->d_bclo + (size_t)j * (a->D + 1), m->d_bcl};
    launch_pdl(set_memo_desc, 1, 1, 0, s, a->d_mdesc + j, md);
    ++a->launches;
}

// The tier-A passes of every step at once (their slots resident side by side), after every step's
// memo descriptor is set: memoA_all (a block per step and vector) when no tier-A level is wider than
// MEMO_ALL_T threads per vector, else memoA_lvl_all per level index.
static qkc_status memo_tierA_all(qkc_ac *a, qkc_ac::MemoMeta *m, int clamp, int64_t n_vec, cudaStream_t s) {
    const int nq = (int)a->n_qubits;
    qkc_status st;
    for (int j = 0; j < nq; ++j) set_memo_step(a, m, j, clamp, n_vec, true, s);
    const size_t ra = a->recs.size();
    if ((st = rec_begin(a, 3, nullptr, 0, 0, s))) return st;
    if (ra < a->recs.size()) {
        for (int j = 0; j < nq; ++j) {
            a->recs[ra].fixed_bytes += (double)n_vec * m->a_bytes_slot[j];
            a->recs[ra].fixed_edges += (double)n_vec * m->a_edges_slot[j];
        }
    }
    const DevAC d = a->dev();
    if (m->all_T <= MEMO_ALL_T) {
        const unsigned g = (unsigned)std::min<int64_t>((int64_t)nq * n_vec, (int64_t)a->ctx->sm_count * 8);
        if (a->prec == 32)
            launch_pdl(memoA_all<float2>, g, TPB, 0, s, d, a->d_mdesc, m->d_a_nodes, m->d_a_grp, m->d_alllv, m->d_asteps,
                                                m->d_aorder, nq, n_vec);
        else
            launch_pdl(memoA_all<double2>, g, TPB, 0, s, d, a->d_mdesc, m->d_a_nodes, m->d_a_grp, m->d_alllv, m->d_asteps,
                                                 m->d_aorder, nq, n_vec);
        ++a->launches;
    } else {
        const unsigned g = (unsigned)(a->ctx->sm_count * 16);
        for (uint32_t L = 0; L < a->D; ++L) {
            const int64_t o0 = m->lvs_off[L], cnt = m->lvs_off[L + 1] - o0;
            if (cnt == 0) continue;
            if (a->prec == 32)
                launch_pdl(memoA_lvl_all<float2>, g, TPB, 0, s, d, a->d_mdesc, m->d_a_nodes, m->d_a_grp, m->d_lvs + o0,
                                                        (int)cnt);
            else
                launch_pdl(memoA_lvl_all<double2>, g, TPB, 0, s, d, a->d_mdesc, m->d_a_nodes, m->d_a_grp, m->d_lvs + o0,
                                                         (int)cnt);
            ++a->launches;
        }
    }
    if ((st = rec_end(a, ra, s))) return st;
    QKC_LAUNCH_CHECK();
    return QKC_OK;
}

// One memoised upward pass of step j over `bound` group columns (device count n_active); with
// resident slots, its tier A was computed beforehand (memo_tierA_all).
static qkc_status memo_pass(qkc_ac *a, qkc_ac::MemoMeta *m, int j, int clamp, int64_t n_vec,
                            const int32_t *n_active, int64_t bound, int cur, bool resident, cudaStream_t s) {
    qkc_status st;
    cudaGraphExec_t gA = nullptr, gB;
    if ((!resident && (st = memo_graph(a, m, j, false, &gA))) || (st = memo_graph(a, m, j, true, &gB))) return st;
    set_memo_step(a, m, j, clamp, n_vec, resident, s);
    if (!resident) {
        const size_t ra = a->recs.size();
        if ((st = rec_begin(a, 3, nullptr, 0, 0, s))) return st;
        if (ra < a->recs.size()) {
            a->recs[ra].fixed_bytes = (double)n_vec * m->a_bytes_slot[j];
            a->recs[ra].fixed_edges = (double)n_vec * m->a_edges_slot[j];
        }
        QKC_CUDA(cudaGraphLaunch(gA, s));  // tier A: once per step
        a->launches += memoA_launches(a, m, j);
        if ((st = rec_end(a, ra, s))) return st;
    }
    const size_t ri = a->recs.size();
    if ((st = rec_begin(a, 2, n_active, 0, bound, s))) return st;
    if (ri < a->recs.size()) {
        a->recs[ri].col_bytes = m->b_bytes_col[j];
        a->recs[ri].col_edges = m->b_edges_col[j];
    }
    const int64_t pitch = a->tile;
    for (int64_t c0 = 0; c0 < bound; c0 += pitch) {  // tier B and the roots, per tile of groups
        const int64_t nc = std::min<int64_t>(pitch, bound - c0);
        EvSrc es{nullptr, a->d_g_prefix[cur], j, clamp, a->d_g_vec[cur], n_active, std::max<int64_t>(1, n_vec)};
        PassDesc desc{es, a->d_pv, a->vec_cap, c0, nc};
        launch_pdl(set_desc, 1, 1, 0, s, a->d_desc, desc);
        ++a->launches;
        QKC_CUDA(cudaGraphLaunch(gB, s));
        a->launches += memoB_launches(a, m, j);
    }
    if ((st = rec_end(a, ri, s))) return st;
    QKC_LAUNCH_CHECK();
    return QKC_OK;
}

extern "C" qkc_status qkc_set_sampler(qkc_ac *a, int32_t mode, int64_t memo_budget_bytes) {
    if (!a || mode < 0 || mode > 2 || memo_budget_bytes < 0)
        return fail(QKC_ERR_ARG, "qkc_set_sampler: mode must be 0, 1 or 2 and the budget >= 0");
    a->sampler = mode;
    a->memo_budget = memo_budget_bytes;
    return QKC_OK;
}

static qkc_status sample_impl(qkc_ac *a, const uint64_t *seeds, const int32_t *shots, int64_t n_vec,
                              int64_t max_shots, int64_t total_shots, uint64_t *bits, double *probs, void *stream) {
    if (!a || !seeds || !shots || !bits || n_vec <= 0 || max_shots < 0)
        return fail(QKC_ERR_ARG, "qkc_sample: bad argument");
    if (a->kind != QKC_AC_DENSITY && a->kind != QKC_AC_DENSITY_STEPS && a->kind != QKC_AC_TRAJECTORY)
        return fail(QKC_ERR_UNSUPPORTED, "qkc_sample: needs a DENSITY, DENSITY_STEPS or TRAJECTORY AC");
    if (n_vec > a->n_vec && a->n_param > 0) return fail(QKC_ERR_ARG, "qkc_sample: more vectors than bound");
    a->eval_ok = false;
    if (max_shots == 0) return QKC_OK;
    if (n_vec * max_shots > (int64_t)INT32_MAX / 2) return fail(QKC_ERR_ARG, "qkc_sample: too many samples");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_samp = n_vec * max_shots;
    // host bound on the live samples, hence on the groups of every step
    const int64_t live = (total_shots > 0 && total_shots < n_samp) ? total_shots : n_samp;
    const int nq = (int)a->n_qubits;
    // TRAJECTORY AC: a group per vector for the samples without error, one per sample with an error
    const bool traj = a->kind == QKC_AC_TRAJECTORY;
    const int64_t max_groups = std::max(n_samp, n_vec) + (traj ? n_vec : 0);
    qkc_status st;
    if ((st = ensure_sampling(a, n_samp, max_groups))) return st;
    // tile sized for the largest step (bounded by the sample count), roots for every group; a step
    // AC sizes its tile once the memoised passes (whose rows it holds) are chosen
    const bool steps = a->kind == QKC_AC_DENSITY_STEPS;
    if ((!steps && (st = ensure_tile(a, max_groups))) || (st = ensure_roots(a, max_groups))) return st;
    // memoised passes: the largest cap (bits per node key) whose tier-A slots fit the budget
    // (the caller's, else 40% of the device memory and 60% of what is free); if the slots
    // cannot be allocated, smaller caps, then the per-group sampler
    qkc_ac::MemoMeta *meta = nullptr;
    // (memoised passes key a node's value by vector and prefix bits alone: not for trajectories)
    const bool memo_ok = a->sampler >= 1 && nq <= 63 && !traj;
    if (memo_ok) {
        // an already built key width whose slots fit the current allocation (no new metadata)
        for (int cap = (int)a->memo.size() - 1; cap >= 1 && !meta; --cap)
            if (a->memo[cap] && n_vec * a->memo[cap]->max_units * (int64_t)a->elem() <= a->va_bytes) meta = a->memo[cap];
    }
    auto memo_budget = [&]() {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
        return a->memo_budget > 0 ? (double)a->memo_budget
                                  : std::min(0.40 * (double)a->ctx->total_mem, 0.6 * (double)(fr + (size_t)a->va_bytes));
    };
    if (memo_ok && !meta) {
        int ks = 0;
        while (ks < 24 && (2ll << ks) <= max_shots) ++ks;  // floor(log2(max_shots))
        const double budget = memo_budget();
        for (int cap = ks - 1; cap >= 1 && !meta; --cap) {
            qkc_ac::MemoMeta *m = memo_meta(a, cap, &st);
            if (st) return st;
            if (!m) continue;
            const int64_t need = n_vec * m->max_units * (int64_t)a->elem();
            if ((double)need > budget) continue;
            if (need > a->va_bytes) {
                QKC_CUDA(cudaDeviceSynchronize());
                cudaFree(a->d_VA);
                a->d_VA = nullptr;
                a->va_bytes = 0;
                if (cudaMalloc(&a->d_VA, (size_t)std::max<int64_t>(need, 256)) != cudaSuccess) {
                    cudaGetLastError();
                    continue;  // try a smaller cap
                }
                a->va_bytes = need;
            }
            meta = m;
        }
    }
    if (meta && a->sampler == 1) {
        // keep the memoised passes only when they are estimated cheaper than evaluating every
        // node per group: bytes weighted by the measured cost per byte of each kernel kind
        // (per-slot tier-A evaluation ~3x, per-group tier-B ~2x the plain upward pass)
        double plain = 0.0, memo = 0.0, groups = (double)n_vec;
        const double per_col = (double)a->elem() * ((double)a->E + (double)(a->N - a->n_leaves));
        for (int j = 0; j < nq; ++j) {
            plain += groups * per_col;
            memo += 3.0 * (double)n_vec * meta->a_bytes_slot[j] + 2.0 * groups * meta->b_bytes_col[j];
            groups = std::min(2.0 * groups, (double)live);
        }
        if (memo >= plain) meta = nullptr;
    }
    // every step's tier-A slots at once, when they fit the budget: the steps' tier-A passes then run
    // concurrently before the first step (one launch, or one per level index when a level is wide)
    bool resident = false;
    if (meta && nq > 1) {
        const int64_t need = n_vec * meta->unit_base[nq] * (int64_t)a->elem();
        if (need <= a->va_bytes) {
            resident = true;
        } else if ((double)need <= memo_budget()) {
            void *p = nullptr;
            if (cudaMalloc(&p, (size_t)need) == cudaSuccess) {
                QKC_CUDA(cudaDeviceSynchronize());
                cudaFree(a->d_VA);
                a->d_VA = p;
                a->va_bytes = need;
                resident = true;
            } else {
                cudaGetLastError();
            }
        }
    }
    if (steps && (st = ensure_tile(a, std::max(n_samp, n_vec),
                                   meta ? (uint32_t)std::max<int64_t>(1, meta->max_rows) : 0u)))
        return st;
    const unsigned gs = (unsigned)((n_samp + TPB - 1) / TPB);
    if (traj) {
        // draw every sample's trajectory, then one group per vector for the error-free samples and
        // one per sample with an error (rank by an exclusive scan of the error flags)
        traj_draw<<<gs, TPB, 0, s>>>(n_vec, max_shots, shots, seeds, a->n_noise, a->d_noise_off, a->d_cdf,
                                     a->d_traj, a->d_err);
        QKC_CUDA(cudaMemsetAsync(a->d_table, 0, sizeof(unsigned long long) * a->table_size, s));
        traj_dedup<<<gs, TPB, 0, s>>>(n_vec, max_shots, a->d_err, a->d_traj, a->n_noise, a->d_table,
                                      a->table_size - 1, a->d_rep);
        traj_rep_flags<<<gs, TPB, 0, s>>>(n_samp, a->d_err, a->d_rep, a->d_flag);
        set_count<<<1, 1, 0, s>>>(a->d_gcount + 1, (int32_t)n_samp);
        const int64_t nb = (n_samp + 1023) / 1024;
        scan_block<<<(unsigned)nb, 1024, 0, s>>>(a->d_flag, a->d_gcount + 1, 1, a->d_pos, a->d_bsum);
        scan_sums<<<1, 1024, 0, s>>>(a->d_bsum, nb);
        traj_groups<<<std::max(gs, (unsigned)((n_vec + TPB - 1) / TPB)), TPB, 0, s>>>(
            n_vec, max_shots, shots, a->d_err, a->d_rep, a->d_flag, a->d_pos, a->d_bsum, a->d_s_group, a->d_s_bits,
            a->d_g_vec[0], a->d_g_prefix[0], a->d_g_traj[0], a->d_gcount);
        a->launches += 7;
    } else {
        sample_init<<<std::max(gs, (unsigned)((n_vec + TPB - 1) / TPB)), TPB, 0, s>>>(
            n_vec, max_shots, shots, a->d_s_group, a->d_s_bits, a->d_g_vec[0], a->d_g_prefix[0], a->d_gcount);
    }
    QKC_LAUNCH_CHECK();
    int cur = 0;
    // evidence of the group columns at step j (prefix bits, trajectory)
    auto group_ev = [&](int j, int clamp, const int32_t *n_active) {
        EvSrc es{nullptr, a->d_g_prefix[cur], j, clamp, a->d_g_vec[cur], n_active, std::max<int64_t>(1, a->n_vec)};
        if (traj) {
            es.traj = a->d_traj;
            es.col_traj = a->d_g_traj[cur];
            es.n_noise = a->n_noise;
        }
        return es;
    };
    if (resident && (st = memo_tierA_all(a, meta, 1, n_vec, s))) return st;
    // groups before the first step (host bound); every step's pass gives both branch probabilities of
    // each group, so no pass for P(empty prefix) is needed
    const int64_t bound0 = traj ? n_vec + live : n_vec;
    int64_t bound = bound0;  // host upper bound of the group count
    for (int j = 0; j < nq; ++j) {
        // (P(prefix, X_j = 0), P(prefix, X_j = 1)) for every group (count on the device, bound on the host)
        int32_t *gcount = a->d_gcount + cur;
        if (meta) {
            if ((st = memo_pass(a, meta, j, 1, n_vec, gcount, bound, cur, resident, s))) return st;
        } else {
            for (int64_t c0 = 0; c0 < bound; c0 += a->tile) {
                const int64_t nc = std::min<int64_t>(a->tile, bound - c0);
                if ((st = run_up(a, group_ev(j, 1, gcount), c0, nc, s))) return st;
                if ((st = run_roots(a, c0, nc, gcount, s, j))) return st;
            }
        }
        const int64_t nflag = 2 * bound;
        QKC_CUDA(cudaMemsetAsync(a->d_flag, 0, sizeof(int32_t) * nflag, s));
        launch_pdl(sample_decide, gs, TPB, 0, s, n_vec, max_shots, shots, seeds, j, nq, a->d_root, a->d_s_group,
                                         a->d_s_bits, a->d_flag, gcount, a->d_status);
        const int64_t nb = (nflag + 1023) / 1024;
        launch_pdl(scan_block, (unsigned)nb, 1024, 0, s, a->d_flag, gcount, 2, a->d_pos, a->d_bsum);
        launch_pdl(scan_sums, 1, 1024, 0, s, a->d_bsum, nb);
        const int nxt = cur ^ 1;
        launch_pdl(sample_regroup, (unsigned)((nflag + TPB - 1) / TPB), TPB, 0, s,
            gcount, a->d_flag, a->d_pos, a->d_bsum, a->d_g_vec[cur], a->d_g_prefix[cur], a->d_root,
            a->d_g_vec[nxt], a->d_g_prefix[nxt], a->d_g_P[nxt], a->d_gcount + nxt, nflag,
            traj ? a->d_g_traj[cur] : nullptr, traj ? a->d_g_traj[nxt] : nullptr);
        launch_pdl(sample_remap, gs, TPB, 0, s, n_vec, max_shots, shots, a->d_pos, a->d_bsum, a->d_s_group, a->d_s_bits,
                                        nflag, a->d_status);
        a->launches += 5;
        QKC_LAUNCH_CHECK();
        cur = nxt;
        bound = std::min<int64_t>(2 * bound, live + (traj ? n_vec : 0));
    }
    sample_write<<<gs, TPB, 0, s>>>(n_vec, max_shots, shots, a->d_s_bits, bits, a->d_s_group, a->d_g_P[cur],
                                    a->d_gcount + cur, probs);
    ++a->launches;
    QKC_LAUNCH_CHECK();
    return QKC_OK;
}

extern "C" qkc_status qkc_sample(qkc_ac *a, const uint64_t *seeds, const int32_t *shots, int64_t n_vec,
                                 int64_t max_shots, int64_t total_shots, uint64_t *bits, void *stream) {
    return sample_impl(a, seeds, shots, n_vec, max_shots, total_shots, bits, nullptr, stream);
}

extern "C" qkc_status qkc_sample_probs(qkc_ac *a, const uint64_t *seeds, const int32_t *shots, int64_t n_vec,
                                       int64_t max_shots, int64_t total_shots, uint64_t *bits, double *probs,
                                       void *stream) {
    if (!probs) return fail(QKC_ERR_ARG, "qkc_sample_probs: probs is null");
    return sample_impl(a, seeds, shots, n_vec, max_shots, total_shots, bits, probs, stream);
}


extern "C" qkc_status qkc_gibbs(qkc_ac *a, const int32_t *col_vec, const uint64_t *seeds, int64_t n_chains,
                                int8_t *state, int64_t n_sweeps, int64_t sweep_offset, uint64_t *samples,
                                void *stream) {
    qkc_status st = check_query(a, col_vec, state, n_chains, "qkc_gibbs");
    if (st) return st;
    a->eval_ok = false;
    if (a->kind != QKC_AC_AMPLITUDE) return fail(QKC_ERR_UNSUPPORTED, "qkc_gibbs: needs an AMPLITUDE AC");
    if (!seeds || n_sweeps < 0 || sweep_offset < 0) return fail(QKC_ERR_ARG, "qkc_gibbs: bad argument");
    if (n_chains == 0 || n_sweeps == 0) return QKC_OK;
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    if ((st = ensure_tile(a, n_chains)) || (st = ensure_roots(a, n_chains)) || (st = ensure_adj(a))) return st;
    std::vector<int> ind0(a->n_vars + 1, 0), card(a->n_vars, 0);
    for (uint32_t v = 0; v < a->n_vars; ++v) {
        card[v] = (int)a->var_card[v];
        ind0[v + 1] = ind0[v] + card[v];
        if (card[v] > 16) return fail(QKC_ERR_UNSUPPORTED, "qkc_gibbs: variable with more than 16 values");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nv = (int)a->n_vars;
    for (int64_t sw = 0; sw < n_sweeps; ++sw) {
        for (int v = 0; v < nv; ++v) {
            const uint64_t k = (uint64_t)(sweep_offset + sw) * (uint64_t)nv + (uint64_t)v + 1ull;
            for (int64_t c0 = 0; c0 < n_chains; c0 += a->tile) {
                const int64_t nc = std::min<int64_t>(a->tile, n_chains - c0);
                EvSrc es{state, nullptr, 0, 0, col_vec, nullptr, std::max<int64_t>(1, a->n_vec)};
                if ((st = run_up(a, es, c0, nc, s))) return st;
                if ((st = run_down(a, nc, s))) return st;
                const unsigned g = (unsigned)((nc + TPB - 1) / TPB);
                if (a->prec == 32)
                    gibbs_choose<float2><<<g, TPB, 0, s>>>((const float2 *)a->d_A, a->tile, c0, nc, v, card[v], ind0[v],
                                                          nv, seeds, k, state);
                else
                    gibbs_choose<double2><<<g, TPB, 0, s>>>((const double2 *)a->d_A, a->tile, c0, nc, v, card[v],
                                                           ind0[v], nv, seeds, k, state);
                ++a->launches;
                QKC_LAUNCH_CHECK();
            }
        }
        if (samples) {
            gibbs_record<<<(unsigned)((n_chains + TPB - 1) / TPB), TPB, 0, s>>>(state, n_chains, nv, (int)a->n_qubits,
                                                                               n_sweeps, sw, samples);
            ++a->launches;
            QKC_LAUNCH_CHECK();
        }
    }
    return QKC_OK;
}

extern "C" qkc_status qkc_check_status(qkc_ac *a) {
    if (!a) return fail(QKC_ERR_ARG, "qkc_check_status: null AC");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    int32_t v = 0;
    QKC_CUDA(cudaMemcpy(&v, a->d_status, sizeof v, cudaMemcpyDeviceToHost));
    if (v) {
        QKC_CUDA(cudaMemset(a->d_status, 0, sizeof(int32_t)));
        return fail(QKC_ERR_ARG, "qkc_check_status: a qkc_sample call was given total_shots below the sum of its "
                                 "shots; samples beyond it were dropped");
    }
    return QKC_OK;
}

extern "C" qkc_status qkc_stats_enable(qkc_ac *a, int32_t enable, int64_t max_records) {
    if (!a || max_records < 0) return fail(QKC_ERR_ARG, "qkc_stats_enable: bad argument");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    QKC_CUDA(cudaDeviceSynchronize());
    drop_records(a);
    if (enable && max_records > a->statcap) {
        cudaFree(a->d_statcols);
        a->d_statcols = nullptr;
        a->statcap = 0;
        QKC_CUDA(cudaMalloc((void **)&a->d_statcols, sizeof(int64_t) * (size_t)max_records));
        a->statcap = max_records;
    }
    a->timing = enable != 0;
    a->launches = 0;
    return QKC_OK;
}

extern "C" qkc_status qkc_get_stats(qkc_ac *a, qkc_stats *o) {
    if (!a || !o) return fail(QKC_ERR_ARG, "qkc_get_stats: bad argument");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    std::memset(o, 0, sizeof(*o));
    o->launches = a->launches;
    if (!a->recs.empty()) {
        std::vector<int64_t> cols(a->recs.size());
        QKC_CUDA(cudaMemcpy(cols.data(), a->d_statcols, sizeof(int64_t) * cols.size(), cudaMemcpyDeviceToHost));
        const double elem = (double)a->elem();
        for (size_t i = 0; i < a->recs.size(); ++i) {
            float ms = 0.f;
            QKC_CUDA(cudaEventSynchronize(a->recs[i].e1));
            QKC_CUDA(cudaEventElapsedTime(&ms, a->recs[i].e0, a->recs[i].e1));
            if (a->recs[i].kind == 2) {  // memoised sampling pass, tier B: per group column
                o->memo_passes += 1;
                o->memo_columns += cols[i];
                o->memo_ms += ms;
                o->memo_bytes += a->recs[i].col_bytes * (double)cols[i];
                o->memo_edges += a->recs[i].col_edges * (double)cols[i];
            } else if (a->recs[i].kind == 3) {  // memoised sampling pass, tier A: per slot
                o->memo_ms += ms;
                o->memo_bytes += a->recs[i].fixed_bytes;
                o->memo_edges += a->recs[i].fixed_edges;
                o->memo_a_ms += ms;
                o->memo_a_bytes += a->recs[i].fixed_bytes;
            } else if (a->recs[i].kind == 0) {
                o->up_passes += 1;
                o->up_columns += cols[i];
                o->up_ms += ms;
                o->up_launches += (int64_t)(a->D - 1);
                // child reads + node writes of the internal nodes (the algorithmic bytes of the level kernels)
                o->up_bytes += elem * ((double)a->E + (double)(a->N - a->n_leaves)) * (double)cols[i];
                o->up_edges += (double)a->E * (double)cols[i];
            } else {
                o->down_passes += 1;
                o->down_columns += cols[i];
                o->down_ms += ms;
                o->down_launches += (int64_t)(a->D - 1);
                // per parent entry: the parent's adjoint (+ the sibling value for a product), one write per node
                // parent adjoint per visited parent entry, sibling value per product parent,
                // one write per visited node (CONST leaves are not visited)
                const double reads = (double)a->down_edges + (double)a->down_sib;
                const double writes = (double)(a->light_off[a->D] + a->heavy_off[a->D]);
                o->down_bytes += elem * (reads + writes) * (double)cols[i];
                o->down_edges += (double)a->down_edges * (double)cols[i];
            }
        }
    }
    o->records = (int64_t)a->recs.size();
    return QKC_OK;
}

// ------------------------------------------------------------------ upward pass without allocation
// Scratch for qkc_evaluate_static: node values and the FP32 per-(level, column)
// scale words of one column tile.  A file-scope device array, so every GPU that
// loads this library holds QKC_STATIC_SCRATCH_BYTES until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[QKC_STATIC_SCRATCH_BYTES];

namespace {
// Device address of g_static_scratch per device, looked up once per device with
// that device current.  In host code the array's name is only a host-side
// stand-in, so kernels must be given this address, never the name.
std::mutex g_static_mu;
void *g_static_ptr[128] = {nullptr};
}  // namespace

static qkc_status static_scratch(int device, void **out) {
    if (device < 0 || device >= 128) return fail(QKC_ERR_ARG, "qkc_evaluate_static: device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(QKC_ERR_CUDA, "qkc_evaluate_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_static_ptr[device] = p;
    }
    *out = g_static_ptr[device];
    return QKC_OK;
}

extern "C" qkc_status qkc_evaluate_static(qkc_ac *a, const int32_t *col_vec, const int8_t *ev, int64_t n_cols,
                                          double *out, void *stream) {
    qkc_status st = check_query(a, col_vec, ev, n_cols, "qkc_evaluate_static");
    if (st) return st;
    if (n_cols == 0) return QKC_OK;
    if (!out) return fail(QKC_ERR_ARG, "qkc_evaluate_static: out is null");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    void *base = nullptr;
    if ((st = static_scratch(a->ctx->device, &base))) return st;
    // tile: the largest multiple of 64 columns whose values (+ FP32 scale words) fit the array
    const int64_t scale_words = a->prec == 32 ? 2LL * a->D * (int64_t)sizeof(int) : 0;
    const int64_t per_col = (int64_t)a->N * (int64_t)a->elem() + scale_words;
    int64_t tile = (int64_t)QKC_STATIC_SCRATCH_BYTES / per_col;
    tile = std::min<int64_t>(tile / 64 * 64, (n_cols + 63) / 64 * 64);
    if (tile < 64)
        return fail(QKC_ERR_TOO_LARGE,
                    "qkc_evaluate_static: this AC needs %lld bytes of scratch for a 64-column tile; the static "
                    "scratch holds %lld bytes",
                    (long long)(per_col * 64), (long long)QKC_STATIC_SCRATCH_BYTES);
    // layout inside the array: values [N][tile], then S [D][tile], then obs [D][tile]
    char *p = static_cast<char *>(base);
    void *V = p;
    int *S = reinterpret_cast<int *>(p + (size_t)a->N * tile * a->elem());
    int *obs = S + (size_t)a->D * tile;
    cudaStream_t s = (cudaStream_t)stream;
    double2 *o = reinterpret_cast<double2 *>(out);
    // Every scratch word a tile reads is written earlier in the same tile (leaves, then each
    // level's scale words, then its values), so nothing left from a previous call is used.
    for (int64_t c0 = 0; c0 < n_cols; c0 += tile) {
        const int64_t nc = std::min<int64_t>(tile, n_cols - c0);
        EvSrc es{ev, nullptr, 0, 0, col_vec, nullptr, std::max<int64_t>(1, a->n_vec)};
        PassDesc desc{es, a->d_pv, a->vec_cap, c0, nc};
        set_desc<<<1, 1, 0, s>>>(a->d_desc, desc);
        launch_up_sequence(a, s, V, S, obs, tile);
        const unsigned gr = (unsigned)((nc + TPB - 1) / TPB);
        if (a->prec == 32)
            root_f32<<<gr, TPB, 0, s>>>((const float2 *)V, S, tile, a->root, a->root_L, nc, nullptr, c0, o);
        else
            root_f64<<<gr, TPB, 0, s>>>((const double2 *)V, tile, a->root, nc, nullptr, c0, o);
        a->launches += 2 + up_sequence_launches(a);
        QKC_LAUNCH_CHECK();
    }
    return QKC_OK;
}
