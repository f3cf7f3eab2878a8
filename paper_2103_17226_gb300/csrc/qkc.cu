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
constexpr int TPB = 256;       // threads per block
constexpr int OBS_EMPTY = -1000;

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float pow2f(int k) {
    if (k < -126) return 0.0f;
    if (k > 127) k = 127;
    return __int_as_float((k + 127) << 23);
}
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
};

__device__ __forceinline__ int64_t vec_of(const EvSrc &e, int64_t gc) {
    int64_t v = e.col_vec ? (int64_t)e.col_vec[gc] : gc;
    return v < 0 ? 0 : (v >= e.n_vec ? e.n_vec - 1 : v);
}

__device__ __forceinline__ int ev_code(const EvSrc &e, const DevAC &ac, int64_t col, int var) {
    if (e.ev) return e.ev[col * ac.n_vars + var];
    int q = var;  // density AC: indicator variables are the qubits
    if (q < e.j) return (int)((e.prefix[col] >> (e.j - 1 - q)) & 1ull);
    if (q == e.j && e.clamp) return 0;
    return -1;
}
__device__ __forceinline__ double ind_value(int code, int val) {
    if (code == -1) return 1.0;
    if (code == -2) return val == 0 ? 1.0 : -1.0;
    return code == val ? 1.0 : 0.0;
}

// FP32 leaves; also initialises the level-0 scale (0) and observed exponent.
__global__ void bind_leaves_f32(DevAC ac, EvSrc es, int64_t col0, int64_t ncols_host, int64_t pitch,
                                const float2 *pv, int64_t pv_pitch, float2 *V, int *obs, int n_leaves) {
    int64_t ncols = ncols_host;
    if (es.n_active) ncols = min(ncols_host, (int64_t)(*es.n_active) - col0);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_leaves * pitch;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t / pitch);
        int64_t c = t % pitch;
        if (c >= ncols) continue;
        int64_t gc = col0 + c;
        float2 v;
        if (i < ac.n_ind) {
            v = make_float2((float)ind_value(ev_code(es, ac, gc, ac.ind_var[i]), ac.ind_val[i]), 0.0f);
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

__global__ void bind_leaves_f64(DevAC ac, EvSrc es, int64_t col0, int64_t ncols_host, int64_t pitch,
                                const double2 *pv, int64_t pv_pitch, double2 *V, int n_leaves) {
    int64_t ncols = ncols_host;
    if (es.n_active) ncols = min(ncols_host, (int64_t)(*es.n_active) - col0);
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_leaves * pitch;
    for (; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t / pitch);
        int64_t c = t % pitch;
        if (c >= ncols) continue;
        int64_t gc = col0 + c;
        double2 v;
        if (i < ac.n_ind) {
            v = make_double2(ind_value(ev_code(es, ac, gc, ac.ind_var[i]), ac.ind_val[i]), 0.0);
        } else if (i < ac.n_ind + ac.n_param) {
            v = pv[(int64_t)(i - ac.n_ind) * pv_pitch + vec_of(es, gc)];
        } else {
            v = ac.const_val[i - ac.n_ind - ac.n_param];
        }
        V[(int64_t)i * pitch + c] = v;
    }
}

// ------------------------------------------------------------------ per-level scale (FP32)
// S[L][c] = max over the child levels L' of level L of S[L'][c] + obs[L'][c];
// obs[L][c] reset.  Order-independent, so deterministic and per column.
__global__ void level_scale_kernel(DevAC ac, int L, int64_t pitch, int64_t ncols, int *S, int *obs) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= pitch) return;
    int s = INT_MIN;
    for (uint32_t k = ac.cl_off[L]; k < ac.cl_off[L + 1]; ++k) {
        int Lp = ac.cl[k];
        int o = obs[(int64_t)Lp * pitch + c];
        if (o == OBS_EMPTY) o = -127;
        int cand = S[(int64_t)Lp * pitch + c] + o;
        s = max(s, cand);
    }
    if (s == INT_MIN) s = 0;
    S[(int64_t)L * pitch + c] = s;
    obs[(int64_t)L * pitch + c] = OBS_EMPTY;
    (void)ncols;
}

// ------------------------------------------------------------------ upward pass, one level
struct LevelArgs {
    uint32_t lo, hi;   // node range of the level
    int L;
    int64_t pitch;     // columns per node row in the buffer
    int64_t ncols;     // active columns of this tile (host bound)
    const int32_t *n_active;  // device-side active count (sampling) or null
    int64_t col0;
};

// FP32: lane holds 2 columns (one float4), warp covers 64 columns.
__global__ void __launch_bounds__(TPB) up_level_f32(DevAC ac, LevelArgs a, float2 *__restrict__ V,
                                                     const int *__restrict__ S, int *__restrict__ obs) {
    int64_t ncols = a.ncols;
    if (a.n_active) ncols = min(a.ncols, (int64_t)(*a.n_active) - a.col0);
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
__global__ void __launch_bounds__(TPB) up_level_f64(DevAC ac, LevelArgs a, double2 *__restrict__ V) {
    int64_t ncols = a.ncols;
    if (a.n_active) ncols = min(a.ncols, (int64_t)(*a.n_active) - a.col0);
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
    int64_t pitch, ncols;
};

__global__ void __launch_bounds__(TPB) down_light_f32(DevAC ac, DownArgs a, const float2 *__restrict__ V,
                                                       const int *__restrict__ S, float2 *A) {
    const int64_t ncols = a.ncols;
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

__global__ void __launch_bounds__(TPB) down_heavy_f32(DevAC ac, DownArgs a, const float2 *__restrict__ V,
                                                       const int *__restrict__ S, float2 *A) {
    __shared__ float4 part[TPB / 32][32];
    const int64_t ncols = a.ncols;
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

__global__ void __launch_bounds__(TPB) down_light_f64(DevAC ac, DownArgs a, const double2 *__restrict__ V,
                                                       double2 *A) {
    const int64_t ncols = a.ncols;
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

__global__ void __launch_bounds__(TPB) down_heavy_f64(DevAC ac, DownArgs a, const double2 *__restrict__ V,
                                                       double2 *A) {
    __shared__ double2 part[TPB / 32][32];
    const int64_t ncols = a.ncols;
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
__global__ void seed_root(C *A, int64_t pitch, uint32_t root, int64_t ncols) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncols) return;
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

__global__ void sample_set_total(const double2 *root, int64_t n_vec, double *g_P) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n_vec) g_P[t] = root[t].x;
}

// Decide bit j of every live sample; mark the child group (2g + bit).
__global__ void sample_decide(int64_t n_vec, int64_t max_shots, const int32_t *shots, const uint64_t *seeds, int j,
                              int n_qubits, const double2 *p0v, const double *g_P, int32_t *s_group,
                              uint64_t *s_bits, int32_t *flag) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v]) return;
    int g = s_group[t];
    double p0 = p0v[g].x, P = g_P[g];
    uint64_t k = (uint64_t)s * (uint64_t)n_qubits + (uint64_t)j + 1ull;
    double u = (double)(splitmix64_k(seeds[v], k) >> 11) * (1.0 / 9007199254740992.0);
    int bit = (u * P >= p0) ? 1 : 0;
    s_bits[t] = (s_bits[t] << 1) | (uint64_t)bit;
    flag[2 * g + bit] = 1;
}

// exclusive scan of flag[0..n) into pos (block-local pass), block sums in bsum
__global__ void scan_block(const int32_t *flag, const int32_t *n_dev, int mult, int32_t *pos, int32_t *bsum) {
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
                               const double *g_P, const double2 *p0v, int32_t *g_vec_n, uint64_t *g_prefix_n,
                               double *g_P_n, int32_t *g_count_new) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t n = 2LL * (*g_count_old);
    if (k >= n) return;
    int32_t id = pos[k] + bsum[k >> 10];
    if (k == n - 1) *g_count_new = id + flag[k];
    if (!flag[k]) return;
    int64_t g = k >> 1;
    int bit = (int)(k & 1);
    g_vec_n[id] = g_vec[g];
    g_prefix_n[id] = (g_prefix[g] << 1) | (uint64_t)bit;
    double p0 = p0v[g].x, P = g_P[g];
    g_P_n[id] = bit ? fmax(P - p0, 0.0) : p0;
}
__global__ void sample_remap(int64_t n_vec, int64_t max_shots, const int32_t *shots, const int32_t *pos,
                             const int32_t *bsum, int32_t *s_group, const uint64_t *s_bits) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v]) return;
    int64_t k = 2LL * s_group[t] + (int64_t)(s_bits[t] & 1ull);
    s_group[t] = pos[k] + bsum[k >> 10];
}
__global__ void sample_write(int64_t n_vec, int64_t max_shots, const int32_t *shots, const uint64_t *s_bits,
                             uint64_t *bits) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_vec * max_shots) return;
    int64_t v = t / max_shots, s = t % max_shots;
    if (s >= shots[v]) return;
    bits[t] = s_bits[t];
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
    double2 *d_root = nullptr;  // [root_cap]
    int64_t root_cap = 0;
    // sampling scratch
    int64_t samp_cap = 0, grp_cap = 0;
    int32_t *d_s_group = nullptr, *d_flag = nullptr, *d_pos = nullptr, *d_bsum = nullptr, *d_gcount = nullptr;
    uint64_t *d_s_bits = nullptr;
    int32_t *d_g_vec[2] = {nullptr, nullptr};
    uint64_t *d_g_prefix[2] = {nullptr, nullptr};
    double *d_g_P[2] = {nullptr, nullptr};

    // stats: launches of this library's kernels, and (when enabled) CUDA events around
    // every chain of level kernels with the number of columns it processed
    int64_t launches = 0;
    bool timing = false;
    struct Rec { cudaEvent_t e0, e1; int kind; };  // kind 0 upward, 1 downward
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
    *out = c;
    return QKC_OK;
}

extern "C" void qkc_ctx_destroy(qkc_ctx *ctx) { delete ctx; }

static void free_scratch(qkc_ac *a) {
    cudaFree(a->d_pv); a->d_pv = nullptr;
    cudaFree(a->d_V); a->d_V = nullptr;
    cudaFree(a->d_A); a->d_A = nullptr; a->adj_ok = false;
    cudaFree(a->d_S); a->d_S = nullptr;
    cudaFree(a->d_obs); a->d_obs = nullptr;
    cudaFree(a->d_root); a->d_root = nullptr;
    cudaFree(a->d_s_group); cudaFree(a->d_flag); cudaFree(a->d_pos); cudaFree(a->d_bsum);
    cudaFree(a->d_gcount); cudaFree(a->d_s_bits);
    a->d_s_group = a->d_flag = a->d_pos = a->d_bsum = a->d_gcount = nullptr;
    a->d_s_bits = nullptr;
    for (int i = 0; i < 2; ++i) {
        cudaFree(a->d_g_vec[i]); cudaFree(a->d_g_prefix[i]); cudaFree(a->d_g_P[i]);
        a->d_g_vec[i] = nullptr; a->d_g_prefix[i] = nullptr; a->d_g_P[i] = nullptr;
    }
    a->vec_cap = a->tile = a->root_cap = a->samp_cap = a->grp_cap = 0;
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
    if (kind > 1 || nq == 0 || nq > 64 || N == 0 || D == 0 || D > 65535 || nl > N || root >= N || nind > nl)
        return fail(QKC_ERR_FORMAT, "qkc_load_ac: inconsistent header");
    uint64_t off = 64, s_card, s_tag, s_lo, s_op, s_coff, s_child, s_la, s_lb, s_lc;
    bool ok = take(off, len, 4ull * nv, s_card) && take(off, len, 4ull * nv, s_tag) &&
              take(off, len, 4ull * (D + 1), s_lo) && take(off, len, 1ull * N, s_op) &&
              take(off, len, 4ull * (N + 1), s_coff) && take(off, len, 4ull * E, s_child) &&
              take(off, len, 4ull * nl, s_la) && take(off, len, 4ull * nl, s_lb) && take(off, len, 16ull * nl, s_lc);
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
    if (lev[root] != D - 1 || lo[D - 1] + 1 != lo[D]) return fail(QKC_ERR_FORMAT, "qkc_load_ac: root is not alone on the top level");
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
            (fo > 64 ? heavy : light).push_back(i);
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
    a->n_const = nl - nind - n_param; a->level_off = lo;
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
// same shape) each stay within 35% of the device memory.
static qkc_status ensure_tile(qkc_ac *a, int64_t cols) {
    int64_t want = (cols + 63) / 64 * 64;
    if (want < 64) want = 64;
    const int64_t per_col = (int64_t)a->N * (int64_t)a->elem() + 8LL * a->D;
    int64_t cap = (int64_t)((double)a->ctx->total_mem * 0.35) / std::max<int64_t>(1, per_col);
    if (const char *env = std::getenv("QKC_MAX_TILE_COLUMNS")) {  // smaller tiles (tests of the tiled path)
        const long long lim = std::atoll(env);
        if (lim > 0) cap = std::min<int64_t>(cap, lim);
    }
    if (a->tile_limit > 0) cap = std::min<int64_t>(cap, a->tile_limit);
    cap = cap / 64 * 64;
    if (cap < 64) return fail(QKC_ERR_NOMEM, "qkc: AC too large for one 64-column tile");
    want = std::min(want, cap);
    if (want <= a->tile) return QKC_OK;
    QKC_CUDA(cudaDeviceSynchronize());
    cudaFree(a->d_V); cudaFree(a->d_A); cudaFree(a->d_S); cudaFree(a->d_obs);
    a->d_V = a->d_A = nullptr; a->d_S = a->d_obs = nullptr; a->tile = 0; a->adj_ok = false;
    cudaError_t e1 = cudaMalloc(&a->d_V, (size_t)a->N * want * a->elem());
    cudaError_t e3 = cudaMalloc((void **)&a->d_S, sizeof(int) * (size_t)a->D * want);
    cudaError_t e4 = cudaMalloc((void **)&a->d_obs, sizeof(int) * (size_t)a->D * want);
    if (e1 || e3 || e4) {
        cudaFree(a->d_V); cudaFree(a->d_S); cudaFree(a->d_obs);
        a->d_V = nullptr; a->d_S = a->d_obs = nullptr;
        cudaGetLastError();
        return fail(QKC_ERR_NOMEM, "qkc: cannot allocate a %lld-column tile", (long long)want);
    }
    a->tile = want;
    return QKC_OK;
}

static qkc_status ensure_adj(qkc_ac *a) {
    if (a->adj_ok) return QKC_OK;
    QKC_CUDA(cudaDeviceSynchronize());
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

static qkc_status run_up(qkc_ac *a, const EvSrc &es, int64_t col0, int64_t ncols, cudaStream_t s) {
    const int64_t pitch = a->tile;
    const DevAC d = a->dev();
    const int sms = a->ctx->sm_count;
    qkc_status st;
    if (a->prec == 32) {
        // level 0: leaves (S[0] = 0 and obs[0] reset by the scale kernel, then observed)
        level_scale_kernel<<<(unsigned)((pitch + TPB - 1) / TPB), TPB, 0, s>>>(d, 0, pitch, ncols, a->d_S, a->d_obs);
        bind_leaves_f32<<<grid_for((int64_t)a->n_leaves * pitch), TPB, 0, s>>>(
            d, es, col0, ncols, pitch, (const float2 *)a->d_pv, a->vec_cap, (float2 *)a->d_V, a->d_obs,
            (int)a->n_leaves);
        QKC_LAUNCH_CHECK();
        a->launches += 2;
        const size_t ri = a->recs.size();
        if ((st = rec_begin(a, 0, es.n_active, col0, ncols, s))) return st;
        for (uint32_t L = 1; L < a->D; ++L) {
            level_scale_kernel<<<(unsigned)((pitch + TPB - 1) / TPB), TPB, 0, s>>>(d, (int)L, pitch, ncols, a->d_S,
                                                                                   a->d_obs);
            LevelArgs la{a->level_off[L], a->level_off[L + 1], (int)L, pitch, ncols, es.n_active, col0};
            const int64_t items = ((int64_t)(la.hi - la.lo + NB - 1) / NB) * ((ncols + 63) / 64);
            up_level_f32<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(d, la, (float2 *)a->d_V, a->d_S,
                                                                                    a->d_obs);
        }
        a->launches += 2 * (int64_t)(a->D - 1);
        if ((st = rec_end(a, ri, s))) return st;
        QKC_LAUNCH_CHECK();
    } else {
        bind_leaves_f64<<<grid_for((int64_t)a->n_leaves * pitch), TPB, 0, s>>>(
            d, es, col0, ncols, pitch, (const double2 *)a->d_pv, a->vec_cap, (double2 *)a->d_V, (int)a->n_leaves);
        QKC_LAUNCH_CHECK();
        a->launches += 1;
        const size_t ri = a->recs.size();
        if ((st = rec_begin(a, 0, es.n_active, col0, ncols, s))) return st;
        for (uint32_t L = 1; L < a->D; ++L) {
            LevelArgs la{a->level_off[L], a->level_off[L + 1], (int)L, pitch, ncols, es.n_active, col0};
            const int64_t items = ((int64_t)(la.hi - la.lo + NB - 1) / NB) * ((ncols + 31) / 32);
            up_level_f64<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(d, la, (double2 *)a->d_V);
        }
        a->launches += (int64_t)(a->D - 1);
        if ((st = rec_end(a, ri, s))) return st;
        QKC_LAUNCH_CHECK();
    }
    return QKC_OK;
}

static qkc_status run_roots(qkc_ac *a, int64_t col0, int64_t ncols, const int32_t *n_active, cudaStream_t s) {
    const unsigned g = (unsigned)((ncols + TPB - 1) / TPB);
    if (a->prec == 32)
        root_f32<<<g, TPB, 0, s>>>((const float2 *)a->d_V, a->d_S, a->tile, a->root, (int)a->D - 1, ncols, n_active,
                                   col0, a->d_root);
    else
        root_f64<<<g, TPB, 0, s>>>((const double2 *)a->d_V, a->tile, a->root, ncols, n_active, col0, a->d_root);
    ++a->launches;
    QKC_LAUNCH_CHECK();
    return QKC_OK;
}

static qkc_status run_down(qkc_ac *a, int64_t ncols, cudaStream_t s) {
    const int64_t pitch = a->tile;
    const DevAC d = a->dev();
    const int sms = a->ctx->sm_count;
    const unsigned g = (unsigned)((ncols + TPB - 1) / TPB);
    qkc_status st;
    const size_t ri = a->recs.size();
    if ((st = rec_begin(a, 1, nullptr, 0, ncols, s))) return st;
    a->launches += (int64_t)a->D;
    if (a->prec == 32) {
        seed_root<float2><<<g, TPB, 0, s>>>((float2 *)a->d_A, pitch, a->root, ncols);
        for (int L = (int)a->D - 2; L >= 0; --L) {
            const int64_t nl = a->light_off[L + 1] - a->light_off[L], nh = a->heavy_off[L + 1] - a->heavy_off[L];
            if (nl) {
                DownArgs da{a->d_light + a->light_off[L], nl, pitch, ncols};
                const int64_t items = ((nl + NB - 1) / NB) * ((ncols + 63) / 64);
                down_light_f32<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(
                    d, da, (const float2 *)a->d_V, a->d_S, (float2 *)a->d_A);
            }
            if (nh) {
                DownArgs da{a->d_heavy + a->heavy_off[L], nh, pitch, ncols};
                const int64_t items = nh * ((ncols + 63) / 64);
                down_heavy_f32<<<(unsigned)std::min<int64_t>(items, (int64_t)sms * 8), TPB, 0, s>>>(
                    d, da, (const float2 *)a->d_V, a->d_S, (float2 *)a->d_A);
                ++a->launches;
            }
        }
    } else {
        seed_root<double2><<<g, TPB, 0, s>>>((double2 *)a->d_A, pitch, a->root, ncols);
        for (int L = (int)a->D - 2; L >= 0; --L) {
            const int64_t nl = a->light_off[L + 1] - a->light_off[L], nh = a->heavy_off[L + 1] - a->heavy_off[L];
            if (nl) {
                DownArgs da{a->d_light + a->light_off[L], nl, pitch, ncols};
                const int64_t items = ((nl + NB - 1) / NB) * ((ncols + 31) / 32);
                down_light_f64<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(
                    d, da, (const double2 *)a->d_V, (double2 *)a->d_A);
            }
            if (nh) {
                DownArgs da{a->d_heavy + a->heavy_off[L], nh, pitch, ncols};
                const int64_t items = nh * ((ncols + 31) / 32);
                down_heavy_f64<<<(unsigned)std::min<int64_t>(items, (int64_t)sms * 8), TPB, 0, s>>>(
                    d, da, (const double2 *)a->d_V, (double2 *)a->d_A);
                ++a->launches;
            }
        }
    }
    if ((st = rec_end(a, ri, s))) return st;
    QKC_LAUNCH_CHECK();
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
    return QKC_OK;
}

extern "C" qkc_status qkc_marginals(qkc_ac *a, const int32_t *col_vec, const int8_t *ev, int64_t n_cols,
                                    double *root_out, double *marg_out, void *stream) {
    qkc_status st = check_query(a, col_vec, ev, n_cols, "qkc_marginals");
    if (st) return st;
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
    a->samp_cap = ns;
    a->grp_cap = ng;
    return QKC_OK;
}

extern "C" qkc_status qkc_sample(qkc_ac *a, const uint64_t *seeds, const int32_t *shots, int64_t n_vec,
                                 int64_t max_shots, uint64_t *bits, void *stream) {
    if (!a || !seeds || !shots || !bits || n_vec <= 0 || max_shots < 0)
        return fail(QKC_ERR_ARG, "qkc_sample: bad argument");
    if (a->kind != QKC_AC_DENSITY) return fail(QKC_ERR_UNSUPPORTED, "qkc_sample: needs a DENSITY AC");
    if (n_vec > a->n_vec && a->n_param > 0) return fail(QKC_ERR_ARG, "qkc_sample: more vectors than bound");
    if (max_shots == 0) return QKC_OK;
    if (n_vec * max_shots > (int64_t)INT32_MAX / 2) return fail(QKC_ERR_ARG, "qkc_sample: too many samples");
    QKC_CUDA(cudaSetDevice(a->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_samp = n_vec * max_shots;
    const int nq = (int)a->n_qubits;
    qkc_status st;
    if ((st = ensure_sampling(a, n_samp, std::max(n_samp, n_vec)))) return st;
    // tile sized for the largest step (bounded by the sample count), roots for every group
    if ((st = ensure_tile(a, std::max(n_samp, n_vec))) || (st = ensure_roots(a, std::max(n_samp, n_vec)))) return st;
    const unsigned gs = (unsigned)((n_samp + TPB - 1) / TPB);
    sample_init<<<std::max(gs, (unsigned)((n_vec + TPB - 1) / TPB)), TPB, 0, s>>>(
        n_vec, max_shots, shots, a->d_s_group, a->d_s_bits, a->d_g_vec[0], a->d_g_prefix[0], a->d_gcount);
    QKC_LAUNCH_CHECK();
    int cur = 0;
    // P(empty prefix) for every vector: all indicators free
    {
        for (int64_t c0 = 0; c0 < n_vec; c0 += a->tile) {
            const int64_t nc = std::min<int64_t>(a->tile, n_vec - c0);
            EvSrc es{nullptr, a->d_g_prefix[cur], 0, 0, a->d_g_vec[cur], nullptr, std::max<int64_t>(1, a->n_vec)};
            if ((st = run_up(a, es, c0, nc, s))) return st;
            if ((st = run_roots(a, c0, nc, nullptr, s))) return st;
        }
        sample_set_total<<<(unsigned)((n_vec + TPB - 1) / TPB), TPB, 0, s>>>(a->d_root, n_vec, a->d_g_P[cur]);
        a->launches += 2;  // init + totals
        QKC_LAUNCH_CHECK();
    }
    int64_t bound = n_vec;  // host upper bound of the group count
    for (int j = 0; j < nq; ++j) {
        // p0 = P(prefix, X_j = 0) for every group (count on the device, bound on the host)
        int32_t *gcount = a->d_gcount + cur;
        for (int64_t c0 = 0; c0 < bound; c0 += a->tile) {
            const int64_t nc = std::min<int64_t>(a->tile, bound - c0);
            EvSrc es{nullptr, a->d_g_prefix[cur], j, 1, a->d_g_vec[cur], gcount, std::max<int64_t>(1, a->n_vec)};
            if ((st = run_up(a, es, c0, nc, s))) return st;
            if ((st = run_roots(a, c0, nc, gcount, s))) return st;
        }
        const int64_t nflag = 2 * bound;
        QKC_CUDA(cudaMemsetAsync(a->d_flag, 0, sizeof(int32_t) * nflag, s));
        sample_decide<<<gs, TPB, 0, s>>>(n_vec, max_shots, shots, seeds, j, nq, a->d_root, a->d_g_P[cur],
                                         a->d_s_group, a->d_s_bits, a->d_flag);
        const int64_t nb = (nflag + 1023) / 1024;
        scan_block<<<(unsigned)nb, 1024, 0, s>>>(a->d_flag, gcount, 2, a->d_pos, a->d_bsum);
        scan_sums<<<1, 1024, 0, s>>>(a->d_bsum, nb);
        const int nxt = cur ^ 1;
        sample_regroup<<<(unsigned)((nflag + TPB - 1) / TPB), TPB, 0, s>>>(
            gcount, a->d_flag, a->d_pos, a->d_bsum, a->d_g_vec[cur], a->d_g_prefix[cur], a->d_g_P[cur], a->d_root,
            a->d_g_vec[nxt], a->d_g_prefix[nxt], a->d_g_P[nxt], a->d_gcount + nxt);
        sample_remap<<<gs, TPB, 0, s>>>(n_vec, max_shots, shots, a->d_pos, a->d_bsum, a->d_s_group, a->d_s_bits);
        a->launches += 5;
        QKC_LAUNCH_CHECK();
        cur = nxt;
        bound = std::min<int64_t>(2 * bound, n_samp);
    }
    sample_write<<<gs, TPB, 0, s>>>(n_vec, max_shots, shots, a->d_s_bits, bits);
    ++a->launches;
    QKC_LAUNCH_CHECK();
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
            if (a->recs[i].kind == 0) {
                o->up_passes += 1;
                o->up_columns += cols[i];
                o->up_ms += ms;
                o->up_launches += (int64_t)(a->D - 1);
                // child reads + node writes of the internal nodes (the algorithmic bytes of the level kernels)
                o->up_bytes += elem * ((double)a->E + (double)(a->N - a->n_leaves)) * (double)cols[i];
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
    const DevAC d = a->dev();
    const int sms = a->ctx->sm_count;
    double2 *o = reinterpret_cast<double2 *>(out);
    // Every scratch word a tile reads is written earlier in the same tile (leaves, then each
    // level's scale words, then its values), so nothing left from a previous call is used.
    for (int64_t c0 = 0; c0 < n_cols; c0 += tile) {
        const int64_t nc = std::min<int64_t>(tile, n_cols - c0);
        EvSrc es{ev, nullptr, 0, 0, col_vec, nullptr, std::max<int64_t>(1, a->n_vec)};
        const unsigned gr = (unsigned)((nc + TPB - 1) / TPB);
        if (a->prec == 32) {
            level_scale_kernel<<<(unsigned)((tile + TPB - 1) / TPB), TPB, 0, s>>>(d, 0, tile, nc, S, obs);
            bind_leaves_f32<<<grid_for((int64_t)a->n_leaves * tile), TPB, 0, s>>>(
                d, es, c0, nc, tile, (const float2 *)a->d_pv, a->vec_cap, (float2 *)V, obs, (int)a->n_leaves);
            for (uint32_t L = 1; L < a->D; ++L) {
                level_scale_kernel<<<(unsigned)((tile + TPB - 1) / TPB), TPB, 0, s>>>(d, (int)L, tile, nc, S, obs);
                LevelArgs la{a->level_off[L], a->level_off[L + 1], (int)L, tile, nc, nullptr, c0};
                const int64_t items = ((int64_t)(la.hi - la.lo + NB - 1) / NB) * ((nc + 63) / 64);
                up_level_f32<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(d, la, (float2 *)V, S, obs);
            }
            root_f32<<<gr, TPB, 0, s>>>((const float2 *)V, S, tile, a->root, (int)a->D - 1, nc, nullptr, c0, o);
            a->launches += 3 + 2 * (int64_t)(a->D - 1);
        } else {
            bind_leaves_f64<<<grid_for((int64_t)a->n_leaves * tile), TPB, 0, s>>>(
                d, es, c0, nc, tile, (const double2 *)a->d_pv, a->vec_cap, (double2 *)V, (int)a->n_leaves);
            for (uint32_t L = 1; L < a->D; ++L) {
                LevelArgs la{a->level_off[L], a->level_off[L + 1], (int)L, tile, nc, nullptr, c0};
                const int64_t items = ((int64_t)(la.hi - la.lo + NB - 1) / NB) * ((nc + 31) / 32);
                up_level_f64<<<grid_for(items * 32, TPB, (int64_t)sms * 8), TPB, 0, s>>>(d, la, (double2 *)V);
            }
            root_f64<<<gr, TPB, 0, s>>>((const double2 *)V, tile, a->root, nc, nullptr, c0, o);
            a->launches += 2 + (int64_t)(a->D - 1);
        }
        QKC_LAUNCH_CHECK();
    }
    return QKC_OK;
}
