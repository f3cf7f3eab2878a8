// qkc_compile.cpp -- noisy circuit -> Bayesian network -> arithmetic circuit (host).
//
// Sec. 3.1: every gate becomes a conditional amplitude table (CAT) whose entry
// A(out = j | in = i) is U[j][i] (Table 3a, "the transpose of the unitary");
// monomial multi-qubit gates give a new node only to the qubit whose basis state
// changes (Table 3c); a noise channel gets a random-variable (rv) node whose CAT
// holds its Kraus operators (Table 3b).  Gates that are diagonal in the
// computational basis (RZ, Z, CZ, phase flip, phase damping) change no basis
// state, so they add a factor over existing nodes and no new node.
//
// Sec. 3.2 / Table 4: known initial states are substituted (initial nodes have a
// single value), entries equal to 0 or 1 are folded into the structure, every
// other number is a leaf (angle-dependent entries are PARAM leaves bound later),
// and intermediate qubit states are summed out so the AC mentions only output
// and noise variables.  Instead of CNF + c2d, the AC is built by symbolic
// variable elimination (the approach the paper starts from, Sec. 3.2) under a
// min-fill order (the elimination-order remark of Sec. 3.2.2), with
// hash-consing so equal sub-expressions are one node.
//
// DENSITY kind: the network is doubled -- a ket copy with the CATs above, a bra
// copy with their complex conjugates, each noise rv shared by both copies and
// each output variable shared by both copies -- so the polynomial is
// sum_x prod lambda_x <x|rho|x>.
// TRAJECTORY kind: the same doubling, but every noise rv has one variable per
// copy and both are tied to the same indicator leaves, so with the noise
// variables observed at a trajectory r the polynomial is
// sum_x prod lambda_x |A(x, r)|^2 (the paper's Table 5 amplitudes, squared).
#include "../../include/qkc.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <unordered_map>
#include <vector>

extern "C" void qkc_set_error_(const char *msg);  // defined with the runtime (qkc.cu)

namespace {

using cplx = std::complex<double>;

enum NodeOp : uint8_t { OP_IND = 0, OP_PARAM = 1, OP_CONST = 2, OP_ADD = 3, OP_MUL = 4 };
enum ParamFn : int32_t { FN_COS = 0, FN_SIN = 1, FN_EXPNEG = 2, FN_EXPPOS = 3 };

constexpr int32_t REF_ZERO = -1;
constexpr int32_t REF_ONE = -2;

struct TooLarge {};

// A symbolic table entry before it becomes a node: 0, 1, a constant, or c*g(angle).
struct Sym {
    enum Kind { ZERO, ONE, CONST, PARAM } kind = ZERO;
    cplx coef = 0.0;
    int32_t angle = -1;
    int32_t fn = 0;

    static Sym zero() { return Sym(); }
    static Sym one() { Sym s; s.kind = ONE; s.coef = 1.0; return s; }
    static Sym cst(cplx v) {
        Sym s;
        if (v == cplx(0.0, 0.0)) return s;
        if (v == cplx(1.0, 0.0)) return one();
        s.kind = CONST; s.coef = v; return s;
    }
    static Sym par(int32_t angle, int32_t fn, cplx c) {
        Sym s; s.kind = PARAM; s.angle = angle; s.fn = fn; s.coef = c; return s;
    }
    Sym conj() const {
        Sym s = *this;
        s.coef = std::conj(coef);
        if (kind == PARAM) {
            if (fn == FN_EXPNEG) s.fn = FN_EXPPOS;
            else if (fn == FN_EXPPOS) s.fn = FN_EXPNEG;
        }
        return s;
    }
};

// ---------------------------------------------------------------- node store
struct NodeStore {
    std::vector<uint8_t> op;
    std::vector<uint32_t> coff;   // child offsets (size = nodes + 1)
    std::vector<int32_t> kids;
    std::vector<int32_t> la, lb;  // leaf payload (for leaves)
    std::vector<cplx> lc;
    // open-addressing hash of node ids
    std::vector<int32_t> slots;
    size_t mask = 0;
    size_t used = 0;
    int64_t max_nodes;

    explicit NodeStore(int64_t maxn) : max_nodes(maxn) {
        coff.push_back(0);
        slots.assign(1 << 16, -1);
        mask = slots.size() - 1;
    }
    int32_t size() const { return (int32_t)op.size(); }

    static uint64_t mix(uint64_t h) {
        h ^= h >> 33; h *= 0xff51afd7ed558ccdULL; h ^= h >> 33; h *= 0xc4ceb9fe1a85ec53ULL;
        h ^= h >> 33; return h;
    }
    static uint64_t dbits(double d) { uint64_t u; std::memcpy(&u, &d, 8); return u; }

    uint64_t hash_node(uint8_t o, const int32_t *k, int nk, int32_t a, int32_t b, cplx c) const {
        uint64_t h = mix(0x1234567ULL + o);
        if (o >= OP_ADD) {
            for (int i = 0; i < nk; ++i) h = mix(h ^ (uint64_t)(uint32_t)k[i] ^ ((uint64_t)i << 40));
        } else {
            h = mix(h ^ (uint64_t)(uint32_t)a);
            h = mix(h ^ ((uint64_t)(uint32_t)b << 7));
            h = mix(h ^ dbits(c.real()));
            h = mix(h ^ dbits(c.imag()) ^ 0x9e37ULL);
        }
        return h;
    }
    uint64_t hash_of(int32_t id) const {
        uint8_t o = op[id];
        if (o >= OP_ADD) return hash_node(o, &kids[coff[id]], coff[id + 1] - coff[id], 0, 0, 0.0);
        return hash_node(o, nullptr, 0, la[id], lb[id], lc[id]);
    }
    bool equal(int32_t id, uint8_t o, const int32_t *k, int nk, int32_t a, int32_t b, cplx c) const {
        if (op[id] != o) return false;
        if (o >= OP_ADD) {
            if ((int)(coff[id + 1] - coff[id]) != nk) return false;
            return std::memcmp(&kids[coff[id]], k, sizeof(int32_t) * nk) == 0;
        }
        return la[id] == a && lb[id] == b && dbits(lc[id].real()) == dbits(c.real()) &&
               dbits(lc[id].imag()) == dbits(c.imag());
    }
    void grow() {
        std::vector<int32_t> old;
        old.swap(slots);
        slots.assign(old.size() * 2, -1);
        mask = slots.size() - 1;
        for (int32_t id : old) {
            if (id < 0) continue;
            size_t s = hash_of(id) & mask;
            while (slots[s] >= 0) s = (s + 1) & mask;
            slots[s] = id;
        }
    }
    int32_t intern(uint8_t o, const int32_t *k, int nk, int32_t a, int32_t b, cplx c) {
        uint64_t h = hash_node(o, k, nk, a, b, c);
        size_t s = h & mask;
        while (slots[s] >= 0) {
            if (equal(slots[s], o, k, nk, a, b, c)) return slots[s];
            s = (s + 1) & mask;
        }
        if ((int64_t)op.size() >= max_nodes) throw TooLarge();
        int32_t id = (int32_t)op.size();
        op.push_back(o);
        for (int i = 0; i < nk; ++i) kids.push_back(k[i]);
        coff.push_back((uint32_t)kids.size());
        la.push_back(a); lb.push_back(b); lc.push_back(c);
        slots[s] = id;
        if (++used * 2 > slots.size()) grow();
        return id;
    }

    int32_t ind(int32_t var, int32_t val) { return intern(OP_IND, nullptr, 0, var, val, cplx(1.0, 0.0)); }
    int32_t cst(cplx v) {
        if (v == cplx(0.0, 0.0)) return REF_ZERO;
        if (v == cplx(1.0, 0.0)) return REF_ONE;
        return intern(OP_CONST, nullptr, 0, -1, 0, v);
    }
    int32_t sym(const Sym &s) {
        switch (s.kind) {
            case Sym::ZERO: return REF_ZERO;
            case Sym::ONE: return REF_ONE;
            case Sym::CONST: return cst(s.coef);
            default: return intern(OP_PARAM, nullptr, 0, s.angle, s.fn, s.coef);
        }
    }
    bool is_const(int32_t r) const { return r >= 0 && op[r] == OP_CONST; }

    int32_t mul(int32_t a, int32_t b) {
        if (a == REF_ZERO || b == REF_ZERO) return REF_ZERO;
        if (a == REF_ONE) return b;
        if (b == REF_ONE) return a;
        if (is_const(a) && is_const(b)) return cst(lc[a] * lc[b]);
        int32_t k[2] = {std::min(a, b), std::max(a, b)};
        return intern(OP_MUL, k, 2, 0, 0, 0.0);
    }
    // Sum of terms (each a ref); ZEROs dropped, constants merged into one constant.
    int32_t add(std::vector<int32_t> &t) {
        cplx csum = 0.0;
        bool have_c = false;
        size_t w = 0;
        for (size_t i = 0; i < t.size(); ++i) {
            int32_t r = t[i];
            if (r == REF_ZERO) continue;
            if (r == REF_ONE) { csum += 1.0; have_c = true; continue; }
            if (is_const(r)) { csum += lc[r]; have_c = true; continue; }
            t[w++] = r;
        }
        t.resize(w);
        if (have_c) {
            int32_t c = cst(csum);
            if (c != REF_ZERO) {
                if (t.empty()) return c;
                if (c == REF_ONE) c = cst_one_leaf();
                t.push_back(c);
            }
        }
        if (t.empty()) return REF_ZERO;
        if (t.size() == 1) return t[0];
        std::sort(t.begin(), t.end());
        return intern(OP_ADD, t.data(), (int)t.size(), 0, 0, 0.0);
    }
    // A CONST leaf holding exactly 1 (only needed as an ADD child or as a lone root).
    int32_t cst_one_leaf() { return intern(OP_CONST, nullptr, 0, -1, 0, cplx(1.0, 0.0)); }
    int32_t cst_zero_leaf() { return intern(OP_CONST, nullptr, 0, -1, 0, cplx(0.0, 0.0)); }
};

// ---------------------------------------------------------------- factors
struct Var {
    int32_t card;
};

struct Factor {
    std::vector<int32_t> vars;   // variables with card > 1, table index: first var most significant
    std::vector<int32_t> tab;    // node refs
    bool alive = true;
};

struct Network {
    std::vector<Var> vars;
    std::vector<Factor> factors;
    NodeStore &ns;
    explicit Network(NodeStore &n) : ns(n) {}

    int32_t new_var(int32_t card) {
        vars.push_back({card});
        return (int32_t)vars.size() - 1;
    }
    // Factor over `scope` (may include card-1 variables, fixed at value 0), entry from fn(assignment).
    void add_factor(const std::vector<int32_t> &scope, const std::function<Sym(const std::vector<int> &)> &fn) {
        Factor f;
        std::vector<int32_t> big;
        for (int32_t v : scope)
            if (vars[v].card > 1) big.push_back(v);
        f.vars = big;
        size_t total = 1;
        for (int32_t v : big) total *= (size_t)vars[v].card;
        f.tab.assign(total, REF_ZERO);
        std::vector<int> asg(scope.size(), 0);
        std::vector<int> digit(big.size(), 0);
        for (size_t idx = 0; idx < total; ++idx) {
            // decode idx into big-var digits (first most significant)
            size_t r = idx;
            for (int i = (int)big.size() - 1; i >= 0; --i) {
                int c = vars[big[i]].card;
                digit[i] = (int)(r % c);
                r /= c;
            }
            for (size_t s = 0, b = 0; s < scope.size(); ++s) {
                if (vars[scope[s]].card > 1) asg[s] = digit[b++];
                else asg[s] = 0;
            }
            f.tab[idx] = ns.sym(fn(asg));
        }
        factors.push_back(std::move(f));
    }
};

// ---------------------------------------------------------------- gate algebra
using Mat2 = std::array<std::array<Sym, 2>, 2>;

Mat2 gate_matrix(int kind, int angle) {
    const double s2 = 1.0 / std::sqrt(2.0);
    Mat2 m;
    const cplx I(0.0, 1.0);
    switch (kind) {
        case 0:  // H
            m[0][0] = Sym::cst(s2); m[0][1] = Sym::cst(s2);
            m[1][0] = Sym::cst(s2); m[1][1] = Sym::cst(-s2);
            break;
        case 1:  // X
            m[0][1] = Sym::one(); m[1][0] = Sym::one();
            break;
        case 2:  // Y = [[0, -i], [i, 0]]
            m[0][1] = Sym::cst(-I); m[1][0] = Sym::cst(I);
            break;
        case 3:  // Z
            m[0][0] = Sym::one(); m[1][1] = Sym::cst(-1.0);
            break;
        case 4:  // RX = [[c, -i s], [-i s, c]]
            m[0][0] = Sym::par(angle, FN_COS, 1.0); m[1][1] = Sym::par(angle, FN_COS, 1.0);
            m[0][1] = Sym::par(angle, FN_SIN, -I); m[1][0] = Sym::par(angle, FN_SIN, -I);
            break;
        case 5:  // RY = [[c, -s], [s, c]]
            m[0][0] = Sym::par(angle, FN_COS, 1.0); m[1][1] = Sym::par(angle, FN_COS, 1.0);
            m[0][1] = Sym::par(angle, FN_SIN, -1.0); m[1][0] = Sym::par(angle, FN_SIN, 1.0);
            break;
        case 6:  // RZ = diag(e^{-i t/2}, e^{+i t/2})
            m[0][0] = Sym::par(angle, FN_EXPNEG, 1.0); m[1][1] = Sym::par(angle, FN_EXPPOS, 1.0);
            break;
        default:
            break;
    }
    return m;
}

bool diagonal(const Mat2 &m) { return m[0][1].kind == Sym::ZERO && m[1][0].kind == Sym::ZERO; }

using KMat = std::array<std::array<cplx, 2>, 2>;

// Kraus operators of the one-qubit channels.
std::vector<KMat> kraus1(int kind, double p) {
    std::vector<KMat> k;
    auto Im = KMat{{{1, 0}, {0, 1}}};
    auto Xm = KMat{{{0, 1}, {1, 0}}};
    auto Ym = KMat{{{0, cplx(0, -1)}, {cplx(0, 1), 0}}};
    auto Zm = KMat{{{1, 0}, {0, -1}}};
    auto scale = [](KMat m, double s) { for (auto &r : m) for (auto &e : r) e *= s; return m; };
    switch (kind) {
        case 16:  // DEP1
            k.push_back(scale(Im, std::sqrt(1.0 - p)));
            k.push_back(scale(Xm, std::sqrt(p / 3.0)));
            k.push_back(scale(Ym, std::sqrt(p / 3.0)));
            k.push_back(scale(Zm, std::sqrt(p / 3.0)));
            break;
        case 18:  // AD
            k.push_back(KMat{{{1, 0}, {0, std::sqrt(1.0 - p)}}});
            k.push_back(KMat{{{0, std::sqrt(p)}, {0, 0}}});
            break;
        case 19:  // PD (sign of the damping operator as in the paper's Table 3b)
            k.push_back(KMat{{{1, 0}, {0, std::sqrt(1.0 - p)}}});
            k.push_back(KMat{{{0, 0}, {0, -std::sqrt(p)}}});
            break;
        case 20:  // PF
            k.push_back(scale(Im, std::sqrt(1.0 - p)));
            k.push_back(scale(Zm, std::sqrt(p)));
            break;
        case 21:  // BF
            k.push_back(scale(Im, std::sqrt(1.0 - p)));
            k.push_back(scale(Xm, std::sqrt(p)));
            break;
        default:
            break;
    }
    return k;
}

KMat pauli(int a) {
    switch (a) {
        case 0: return KMat{{{1, 0}, {0, 1}}};
        case 1: return KMat{{{0, 1}, {1, 0}}};
        case 2: return KMat{{{0, cplx(0, -1)}, {cplx(0, 1), 0}}};
        default: return KMat{{{1, 0}, {0, -1}}};
    }
}

struct Builder {
    NodeStore &ns;
    Network net;
    int n_qubits;
    int kind;
    std::vector<int32_t> ket, bra;   // current variable per qubit
    std::vector<int32_t> ind_vars;   // indicator variables, in indicator order
    std::vector<int32_t> ind_tag;    // qubit index or -1-k for the k-th channel
    int n_channels = 0;

    Builder(NodeStore &n, int nq, int k) : ns(n), net(n), n_qubits(nq), kind(k) {
        for (int q = 0; q < nq; ++q) {
            ket.push_back(net.new_var(1));
            bra.push_back(kind == QKC_AC_DENSITY || kind == QKC_AC_TRAJECTORY ? net.new_var(1) : -1);
        }
    }
    bool dbl() const { return kind == QKC_AC_DENSITY || kind == QKC_AC_TRAJECTORY; }
    // TRAJECTORY kind: every noise variable has a ket-copy and a bra-copy variable, both tied to
    // the same indicator leaves, so observing a trajectory fixes both copies to the same branch
    bool per_copy_noise() const { return kind == QKC_AC_TRAJECTORY; }

    // One-qubit matrix m on copy `cur` (conjugated for the bra copy).
    void apply1(std::vector<int32_t> &cur, int q, const Mat2 &m, bool conj) {
        auto ent = [&](int j, int i) { return conj ? m[j][i].conj() : m[j][i]; };
        int32_t u = cur[q];
        if (diagonal(m)) {
            net.add_factor({u}, [&](const std::vector<int> &a) { return ent(a[0], a[0]); });
        } else {
            int32_t w = net.new_var(2);
            net.add_factor({u, w}, [&](const std::vector<int> &a) { return ent(a[1], a[0]); });
            cur[q] = w;
        }
    }
    void cnot(std::vector<int32_t> &cur, int c, int t) {
        int32_t w = net.new_var(2);
        net.add_factor({cur[c], cur[t], w}, [&](const std::vector<int> &a) {
            return (a[2] == (a[0] ^ a[1])) ? Sym::one() : Sym::zero();
        });
        cur[t] = w;
    }
    void cz(std::vector<int32_t> &cur, int a, int b) {
        net.add_factor({cur[a], cur[b]}, [&](const std::vector<int> &x) {
            return (x[0] & x[1]) ? Sym::cst(-1.0) : Sym::one();
        });
    }
    // Channel with Kraus list on copy `cur`, rv variable r.
    void channel1(std::vector<int32_t> &cur, int q, const std::vector<KMat> &ks, int32_t r, bool conj) {
        bool diag = true;
        for (auto &k : ks) diag = diag && k[0][1] == cplx(0, 0) && k[1][0] == cplx(0, 0);
        auto ent = [&](int kk, int j, int i) {
            cplx v = ks[kk][j][i];
            return Sym::cst(conj ? std::conj(v) : v);
        };
        int32_t u = cur[q];
        if (diag) {
            net.add_factor({u, r}, [&](const std::vector<int> &a) { return ent(a[1], a[0], a[0]); });
        } else {
            int32_t w = net.new_var(2);
            net.add_factor({u, r, w}, [&](const std::vector<int> &a) { return ent(a[1], a[2], a[0]); });
            cur[q] = w;
        }
    }
    void channel2_dep(std::vector<int32_t> &cur, int qa, int qb, double p, int32_t r, bool conj) {
        int32_t wa = net.new_var(2), wb = net.new_var(2);
        const double w0 = std::sqrt(1.0 - p), w1 = std::sqrt(p / 15.0);
        net.add_factor({cur[qa], cur[qb], r, wa, wb}, [&](const std::vector<int> &a) {
            int K = a[2], ka = K >> 2, kb = K & 3;
            cplx v = (K == 0 ? w0 : w1) * pauli(ka)[a[3]][a[0]] * pauli(kb)[a[4]][a[1]];
            return Sym::cst(conj ? std::conj(v) : v);
        });
        cur[qa] = wa;
        cur[qb] = wb;
    }

    void op(const qkc_op &o) {
        const int k = o.kind;
        if (k <= 6) {
            Mat2 m = gate_matrix(k, o.angle);
            apply1(ket, o.q0, m, false);
            if (dbl()) apply1(bra, o.q0, m, true);
        } else if (k == 7) {
            cnot(ket, o.q0, o.q1);
            if (dbl()) cnot(bra, o.q0, o.q1);
        } else if (k == 8) {
            cz(ket, o.q0, o.q1);
            if (dbl()) cz(bra, o.q0, o.q1);
        } else if (k == 17) {
            int32_t r = net.new_var(16);
            const int32_t rb = per_copy_noise() ? net.new_var(16) : r;
            channel2_dep(ket, o.q0, o.q1, o.p, r, false);
            if (dbl()) channel2_dep(bra, o.q0, o.q1, o.p, rb, true);
            const double w1 = o.p / 15.0;
            std::vector<double> pr(16, w1);
            pr[0] = 1.0 - o.p;
            note_rv(r, rb, pr);
        } else {
            auto ks = kraus1(k, o.p);
            int32_t r = net.new_var((int32_t)ks.size());
            const int32_t rb = per_copy_noise() ? net.new_var((int32_t)ks.size()) : r;
            channel1(ket, o.q0, ks, r, false);
            if (dbl()) channel1(bra, o.q0, ks, rb, true);
            // branch probabilities of the mixed-unitary channels (E_k = sqrt(p_k) U_k)
            std::vector<double> pr;
            if (k == 16) pr = {1.0 - o.p, o.p / 3.0, o.p / 3.0, o.p / 3.0};
            else if (k == 20 || k == 21) pr = {1.0 - o.p, o.p};
            note_rv(r, rb, pr);
        }
    }
    void note_rv(int32_t r, int32_t rb, const std::vector<double> &pr) {
        if (!dbl() || per_copy_noise()) {  // noise variables carry indicators (Table 5)
            rv_vars.push_back(r);
            rv_bra.push_back(rb);
            for (double x : pr) prior.push_back(x);
        }
        ++n_channels;
    }
    std::vector<int32_t> rv_vars, rv_bra;
    std::vector<double> prior;  // TRAJECTORY: branch probability of every noise indicator value

    // Close the network: unify bra outputs with ket outputs, add indicator factors.
    void finish() {
        if (dbl()) {
            std::vector<int32_t> ren(net.vars.size());
            for (size_t v = 0; v < ren.size(); ++v) ren[v] = (int32_t)v;
            for (int q = 0; q < n_qubits; ++q) ren[bra[q]] = ket[q];
            for (auto &f : net.factors)
                for (auto &v : f.vars) v = ren[v];
        }
        // indicator variables: outputs first (qubit order), then noise rvs (amplitude kind)
        for (int q = 0; q < n_qubits; ++q) {
            ind_vars.push_back(ket[q]);
            ind_tag.push_back(q);
        }
        for (size_t i = 0; i < rv_vars.size(); ++i) {
            ind_vars.push_back(rv_vars[i]);
            ind_tag.push_back(-1 - (int32_t)i);
        }
        // Every indicator leaf exists, in (variable, value) order, so node ids 0..n_ind-1 are them.
        ind_card.clear();
        for (size_t i = 0; i < ind_vars.size(); ++i) {
            int32_t c = (int32_t)std::max<int32_t>(2, net.vars[ind_vars[i]].card);
            if (ind_tag[i] < 0) c = net.vars[ind_vars[i]].card;
            ind_card.push_back(c);
            for (int32_t v = 0; v < c; ++v) ns.ind((int32_t)i, v);
        }
        for (size_t i = 0; i < ind_vars.size(); ++i) {
            const int32_t var = ind_vars[i];
            Factor f;
            if (net.vars[var].card > 1) {
                f.vars.push_back(var);
                for (int32_t v = 0; v < net.vars[var].card; ++v) f.tab.push_back(ns.ind((int32_t)i, v));
            } else {
                f.tab.push_back(ns.ind((int32_t)i, 0));
            }
            net.factors.push_back(std::move(f));
            if (per_copy_noise() && ind_tag[i] < 0) {  // the bra copy's variable: the same leaves
                const int32_t vb = rv_bra[(size_t)(-1 - ind_tag[i])];
                Factor fb;
                fb.vars.push_back(vb);
                for (int32_t v = 0; v < net.vars[vb].card; ++v) fb.tab.push_back(ns.ind((int32_t)i, v));
                net.factors.push_back(std::move(fb));
            }
        }
    }
    std::vector<int32_t> ind_card;
};

// ---------------------------------------------------------------- elimination order
struct Graph {
    std::vector<std::vector<int32_t>> adj;  // sorted neighbour lists
    std::vector<double> lw;                 // log2 card
};

std::vector<int32_t> elimination_order(const Network &net, int mode, double *cost_out, double *width_out = nullptr) {
    const int nv = (int)net.vars.size();
    std::vector<std::vector<int32_t>> adj(nv);
    std::vector<char> active(nv, 0);
    for (const auto &f : net.factors) {
        for (int32_t a : f.vars) {
            active[a] = 1;
            for (int32_t b : f.vars)
                if (a != b) adj[a].push_back(b);
        }
    }
    for (auto &l : adj) {
        std::sort(l.begin(), l.end());
        l.erase(std::unique(l.begin(), l.end()), l.end());
    }
    std::vector<double> lw(nv);
    for (int v = 0; v < nv; ++v) lw[v] = std::log2((double)std::max(1, net.vars[v].card));
    auto connected = [&](int32_t a, int32_t b) {
        return std::binary_search(adj[a].begin(), adj[a].end(), b);
    };
    auto score = [&](int32_t v) -> std::pair<double, double> {
        double w = lw[v];
        for (int32_t u : adj[v]) w += lw[u];
        if (mode == QKC_ORDER_MINWEIGHT) return {w, (double)adj[v].size()};
        long fill = 0;
        const auto &nb = adj[v];
        for (size_t i = 0; i < nb.size(); ++i)
            for (size_t j = i + 1; j < nb.size(); ++j)
                if (!connected(nb[i], nb[j])) ++fill;
        return {(double)fill, w};
    };
    std::vector<int32_t> order;
    std::vector<std::pair<double, double>> sc(nv);
    std::vector<char> dirty(nv, 1);
    double cost = 0.0, maxw = 0.0;
    int total = 0;
    for (int v = 0; v < nv; ++v) total += active[v];
    if (mode == QKC_ORDER_CREATION) {
        for (int v = 0; v < nv; ++v)
            if (active[v]) order.push_back(v);
    }
    while (mode != QKC_ORDER_CREATION && (int)order.size() < total) {
        int32_t best = -1;
        for (int v = 0; v < nv; ++v) {
            if (!active[v]) continue;
            if (dirty[v]) { sc[v] = score(v); dirty[v] = 0; }
            if (best < 0 || sc[v] < sc[best]) best = v;
        }
        // eliminate best: connect its neighbours, remove it
        const std::vector<int32_t> nb = adj[best];
        double w = lw[best];
        for (int32_t u : nb) w += lw[u];
        cost += std::exp2(w);
        maxw = std::max(maxw, w);
        for (int32_t a : nb) {
            auto &la = adj[a];
            la.erase(std::lower_bound(la.begin(), la.end(), best));
            for (int32_t b : nb) {
                if (a == b) continue;
                auto it = std::lower_bound(la.begin(), la.end(), b);
                if (it == la.end() || *it != b) la.insert(it, b);
            }
        }
        // scores change for the neighbours and their neighbours
        for (int32_t a : nb) {
            dirty[a] = 1;
            for (int32_t b : adj[a]) dirty[b] = 1;
        }
        adj[best].clear();
        active[best] = 0;
        order.push_back(best);
    }
    if (mode == QKC_ORDER_CREATION) {
        // cost estimate for the creation order
        std::vector<std::vector<int32_t>> a2(nv);
        for (const auto &f : net.factors)
            for (int32_t a : f.vars)
                for (int32_t b : f.vars)
                    if (a != b) a2[a].push_back(b);
        for (auto &l : a2) { std::sort(l.begin(), l.end()); l.erase(std::unique(l.begin(), l.end()), l.end()); }
        for (int32_t v : order) {
            double w = lw[v];
            for (int32_t u : a2[v]) w += lw[u];
            cost += std::exp2(w);
            maxw = std::max(maxw, w);
            for (int32_t x : a2[v]) {
                auto &lx = a2[x];
                lx.erase(std::lower_bound(lx.begin(), lx.end(), v));
                for (int32_t y : a2[v]) {
                    if (x == y) continue;
                    auto it = std::lower_bound(lx.begin(), lx.end(), y);
                    if (it == lx.end() || *it != y) lx.insert(it, y);
                }
            }
            a2[v].clear();
        }
    }
    if (cost_out) *cost_out = cost;
    if (width_out) *width_out = maxw;
    return order;
}

// ---------------------------------------------------------------- elimination
void eliminate(Network &net, int32_t x, std::vector<std::vector<int32_t>> &var_factors) {
    NodeStore &ns = net.ns;
    std::vector<int32_t> fs;
    for (int32_t fi : var_factors[x])
        if (net.factors[fi].alive) fs.push_back(fi);
    std::sort(fs.begin(), fs.end());
    fs.erase(std::unique(fs.begin(), fs.end()), fs.end());
    // smaller tables first: their partial products are shared across more entries
    std::stable_sort(fs.begin(), fs.end(), [&](int32_t a, int32_t b) {
        return net.factors[a].tab.size() < net.factors[b].tab.size();
    });
    std::vector<int32_t> U;
    for (int32_t fi : fs)
        for (int32_t v : net.factors[fi].vars) U.push_back(v);
    std::sort(U.begin(), U.end());
    U.erase(std::unique(U.begin(), U.end()), U.end());
    std::vector<int32_t> R;
    for (int32_t v : U)
        if (v != x) R.push_back(v);
    // strides of each factor for every variable of U
    const size_t nf = fs.size();
    std::vector<std::vector<size_t>> stride(nf, std::vector<size_t>(U.size(), 0));
    size_t xpos = 0;
    for (size_t u = 0; u < U.size(); ++u)
        if (U[u] == x) xpos = u;
    for (size_t f = 0; f < nf; ++f) {
        const Factor &F = net.factors[fs[f]];
        size_t s = 1;
        for (int i = (int)F.vars.size() - 1; i >= 0; --i) {
            size_t u = std::lower_bound(U.begin(), U.end(), F.vars[i]) - U.begin();
            stride[f][u] = s;
            s *= (size_t)net.vars[F.vars[i]].card;
        }
    }
    Factor g;
    g.vars = R;
    size_t total = 1;
    for (int32_t v : R) total *= (size_t)net.vars[v].card;
    g.tab.assign(total, REF_ZERO);
    const int cx = net.vars[x].card;
    std::vector<int> digit(U.size(), 0);
    std::vector<size_t> base(nf, 0);
    std::vector<int32_t> terms;
    terms.reserve(cx);
    for (size_t idx = 0; idx < total; ++idx) {
        // decode idx over R (first most significant) into U digits
        size_t r = idx;
        for (int i = (int)R.size() - 1; i >= 0; --i) {
            int c = net.vars[R[i]].card;
            size_t u = std::lower_bound(U.begin(), U.end(), R[i]) - U.begin();
            digit[u] = (int)(r % c);
            r /= c;
        }
        for (size_t f = 0; f < nf; ++f) {
            size_t b = 0;
            for (size_t u = 0; u < U.size(); ++u)
                if (u != xpos) b += stride[f][u] * (size_t)digit[u];
            base[f] = b;
        }
        terms.clear();
        for (int xv = 0; xv < cx; ++xv) {
            int32_t p = REF_ONE;
            for (size_t f = 0; f < nf && p != REF_ZERO; ++f) {
                const Factor &F = net.factors[fs[f]];
                p = ns.mul(p, F.tab[base[f] + stride[f][xpos] * (size_t)xv]);
            }
            if (p != REF_ZERO) terms.push_back(p);
        }
        g.tab[idx] = ns.add(terms);
    }
    for (int32_t fi : fs) {
        net.factors[fi].alive = false;
        std::vector<int32_t>().swap(net.factors[fi].tab);
    }
    int32_t gi = (int32_t)net.factors.size();
    net.factors.push_back(std::move(g));
    for (int32_t v : net.factors[gi].vars) var_factors[v].push_back(gi);
}

// ---------------------------------------------------------------- output
void put_u32(std::vector<uint8_t> &b, uint32_t v) {
    uint8_t t[4];
    std::memcpy(t, &v, 4);
    b.insert(b.end(), t, t + 4);
}
void pad8(std::vector<uint8_t> &b) {
    while (b.size() % 8) b.push_back(0);
}
template <class T>
void put_arr(std::vector<uint8_t> &b, const std::vector<T> &a) {
    pad8(b);
    const uint8_t *p = reinterpret_cast<const uint8_t *>(a.data());
    b.insert(b.end(), p, p + a.size() * sizeof(T));
}

}  // namespace

// The nodes that compiling `circ` with elimination order `mode` adds to the store `ns` (on a copy of
// it: `ns` is unchanged), or -1 when that would exceed `limit` new nodes.  The automatic order takes,
// per circuit, whichever of min-fill and min-weight adds fewer nodes: their table-size estimates
// ignore the sharing of equal sub-ACs and the zero entries the elimination drops, and can pick an
// order that gives several times the nodes.
static int64_t trial_nodes(const NodeStore &ns, const std::vector<qkc_op> &circ, int32_t n_qubits, int32_t bkind,
                           int mode, int64_t limit) {
    NodeStore t = ns;
    t.max_nodes = std::min<int64_t>(ns.max_nodes, (int64_t)ns.size() + std::max<int64_t>(limit, 0));
    try {
        Builder bld(t, n_qubits, bkind);
        for (const qkc_op &o : circ) bld.op(o);
        bld.finish();
        Network &net = bld.net;
        const auto ord = elimination_order(net, mode, nullptr);
        std::vector<std::vector<int32_t>> var_factors(net.vars.size());
        for (size_t fi = 0; fi < net.factors.size(); ++fi)
            for (int32_t v : net.factors[fi].vars) var_factors[v].push_back((int32_t)fi);
        for (int32_t x : ord) eliminate(net, x, var_factors);
        return (int64_t)t.size() - (int64_t)ns.size();
    } catch (const TooLarge &) {
        return -1;
    }
}

static qkc_status compile_one(const qkc_op *ops, int32_t n_ops, int32_t n_qubits, int32_t n_angles,
                              int32_t kind, int32_t order, int64_t max_nodes, uint8_t **out_bytes,
                              uint64_t *out_len) {
    if (!out_bytes || !out_len || n_qubits <= 0 || n_qubits > 64 || n_ops < 0 || (n_ops > 0 && !ops) ||
        n_angles < 0 || kind < QKC_AC_AMPLITUDE || kind > QKC_AC_TRAJECTORY || order < 0 || order > 3) {
        qkc_set_error_("qkc_compile: invalid argument");
        return QKC_ERR_ARG;
    }
    for (int32_t i = 0; i < n_ops; ++i) {
        const qkc_op &o = ops[i];
        const bool two = (o.kind == 7 || o.kind == 8 || o.kind == 17);
        const bool known = (o.kind >= 0 && o.kind <= 8) || (o.kind >= 16 && o.kind <= 21);
        const bool par = (o.kind >= 4 && o.kind <= 6);
        if (!known || o.q0 < 0 || o.q0 >= n_qubits || (two && (o.q1 < 0 || o.q1 >= n_qubits || o.q1 == o.q0)) ||
            (par && (o.angle < 0 || o.angle >= n_angles)) ||
            (o.kind >= 16 && !(o.p >= 0.0 && o.p <= 1.0))) {
            char msg[160];
            std::snprintf(msg, sizeof msg, "qkc_compile: operation %d is invalid (kind %d, qubits %d,%d, angle %d)",
                          i, o.kind, o.q0, o.q1, o.angle);
            qkc_set_error_(msg);
            return QKC_ERR_ARG;
        }
        if (kind == QKC_AC_TRAJECTORY && (o.kind == 18 || o.kind == 19)) {
            char msg[200];
            std::snprintf(msg, sizeof msg, "qkc_compile: operation %d: a TRAJECTORY AC needs mixed-unitary channels "
                                           "(DEP1, DEP2, PF, BF), not amplitude or phase damping", i);
            qkc_set_error_(msg);
            return QKC_ERR_ARG;
        }
    }
    if (max_nodes <= 0 || max_nodes > 0x7fffffffLL) max_nodes = 0x7fffffffLL;
    try {
        NodeStore ns(max_nodes);
        // The circuits to compile: the whole circuit, or (light-cone steps) for every j the
        // operations in the backward light cone of qubits 0..j -- walking the circuit from its
        // end, an operation is kept when it touches a qubit of the growing set, which it then
        // joins.  A dropped operation acts only on qubits traced out at the end and never
        // coupled to qubits <= j afterwards, and is trace preserving, so the marginal of qubits
        // <= j is unchanged.  All circuits share the node store (equal sub-ACs are shared).
        std::vector<std::vector<qkc_op>> circuits;
        if (kind == QKC_AC_DENSITY_STEPS) {
            for (int32_t j = 0; j < n_qubits; ++j) {
                std::vector<char> act(n_qubits, 0);
                for (int32_t q = 0; q <= j; ++q) act[q] = 1;
                std::vector<qkc_op> kept;
                for (int32_t i = n_ops - 1; i >= 0; --i) {
                    const qkc_op &o = ops[i];
                    const bool two = (o.kind == 7 || o.kind == 8 || o.kind == 17);
                    if (act[o.q0] || (two && act[o.q1])) {
                        kept.push_back(o);
                        act[o.q0] = 1;
                        if (two) act[o.q1] = 1;
                    }
                }
                std::reverse(kept.begin(), kept.end());
                circuits.push_back(std::move(kept));
            }
        } else {
            circuits.emplace_back(ops, ops + n_ops);
        }
        const int32_t bkind = kind == QKC_AC_DENSITY_STEPS ? QKC_AC_DENSITY : kind;
        std::vector<int32_t> roots;
        std::vector<int32_t> ind_vars_tag;
        std::vector<uint32_t> ind_card_out;
        std::vector<double> prior;  // TRAJECTORY: branch probabilities of the noise indicator values
        for (const auto &circ : circuits) {
            Builder bld(ns, n_qubits, bkind);
            for (const qkc_op &o : circ) bld.op(o);
            bld.finish();
            Network &net = bld.net;

            // elimination order
            std::vector<int32_t> ord;
            if (order == QKC_ORDER_AUTO) {
                // both orders tried on copies of the store (the one with the smaller estimate first,
                // the other bounded by its count); the one that adds fewer nodes is used
                double c1 = 0, c2 = 0;
                elimination_order(net, QKC_ORDER_MINFILL, &c1);
                elimination_order(net, QKC_ORDER_MINWEIGHT, &c2);
                const int first = c2 < c1 ? QKC_ORDER_MINWEIGHT : QKC_ORDER_MINFILL;
                const int second = first == QKC_ORDER_MINFILL ? QKC_ORDER_MINWEIGHT : QKC_ORDER_MINFILL;
                const int64_t room = ns.max_nodes - (int64_t)ns.size();
                const int64_t n1 = trial_nodes(ns, circ, n_qubits, bkind, first, room);
                const int64_t n2 = trial_nodes(ns, circ, n_qubits, bkind, second, n1 >= 0 ? n1 - 1 : room);
                ord = elimination_order(net, (n2 >= 0 && (n1 < 0 || n2 < n1)) ? second : first, nullptr);
            } else {
                ord = elimination_order(net, order, nullptr);
            }
            std::vector<std::vector<int32_t>> var_factors(net.vars.size());
            for (size_t fi = 0; fi < net.factors.size(); ++fi)
                for (int32_t v : net.factors[fi].vars) var_factors[v].push_back((int32_t)fi);
            for (int32_t x : ord) eliminate(net, x, var_factors);

            // root = product of the remaining scalar factors
            int32_t root = REF_ONE;
            for (auto &f : net.factors)
                if (f.alive) root = ns.mul(root, f.tab.empty() ? REF_ZERO : f.tab[0]);
            if (root == REF_ONE) root = ns.cst_one_leaf();
            if (root == REF_ZERO) root = ns.cst_zero_leaf();
            roots.push_back(root);
            // indicator variables (the same for every circuit: outputs in qubit order, then the
            // noise variables of the amplitude kind)
            ind_vars_tag = bld.ind_tag;
            ind_card_out.assign(bld.ind_card.begin(), bld.ind_card.end());
            prior = bld.prior;
        }
        const int32_t root = roots.back();

        // reachable nodes + the full indicator set
        const int32_t nall = ns.size();
        std::vector<char> keep(nall, 0);
        std::vector<int32_t> stack;
        for (int32_t r : roots)
            if (!keep[r]) { keep[r] = 1; stack.push_back(r); }
        while (!stack.empty()) {
            int32_t v = stack.back();
            stack.pop_back();
            for (uint32_t e = ns.coff[v]; e < ns.coff[v + 1]; ++e) {
                int32_t c = ns.kids[e];
                if (!keep[c]) { keep[c] = 1; stack.push_back(c); }
            }
        }
        for (int32_t v = 0; v < nall; ++v)
            if (ns.op[v] == OP_IND) keep[v] = 1;
        // levels (children always have smaller ids than parents: ids are creation order)
        std::vector<int32_t> level(nall, 0);
        int32_t maxlev = 0;
        for (int32_t v = 0; v < nall; ++v) {
            if (!keep[v] || ns.op[v] < OP_ADD) continue;
            int32_t l = 0;
            for (uint32_t e = ns.coff[v]; e < ns.coff[v + 1]; ++e) l = std::max(l, level[ns.kids[e]]);
            level[v] = l + 1;
            maxlev = std::max(maxlev, l + 1);
        }
        // new numbering: leaves (IND in (var,value) order, PARAM, CONST), then by level, op, id
        std::vector<int32_t> ids;
        for (int32_t v = 0; v < nall; ++v)
            if (keep[v]) ids.push_back(v);
        auto leaf_rank = [&](int32_t v) {
            return ns.op[v] == OP_IND ? 0 : ns.op[v] == OP_PARAM ? 1 : ns.op[v] == OP_CONST ? 2 : 3;
        };
        std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t b) {
            if (level[a] != level[b]) return level[a] < level[b];
            if (level[a] == 0) {
                int ra = leaf_rank(a), rb = leaf_rank(b);
                if (ra != rb) return ra < rb;
                if (ra == 0) {
                    if (ns.la[a] != ns.la[b]) return ns.la[a] < ns.la[b];
                    return ns.lb[a] < ns.lb[b];
                }
                if (ra == 1) {
                    if (ns.la[a] != ns.la[b]) return ns.la[a] < ns.la[b];
                    if (ns.lb[a] != ns.lb[b]) return ns.lb[a] < ns.lb[b];
                }
                return a < b;
            }
            if (ns.op[a] != ns.op[b]) return ns.op[a] > ns.op[b];  // MUL before ADD
            return a < b;
        });
        std::vector<int32_t> newid(nall, -1);
        for (size_t i = 0; i < ids.size(); ++i) newid[ids[i]] = (int32_t)i;
        const uint32_t N = (uint32_t)ids.size();
        const uint32_t D = (uint32_t)maxlev + 1;
        std::vector<uint32_t> level_off(D + 1, 0);
        for (int32_t v : ids) level_off[level[v] + 1]++;
        for (uint32_t l = 0; l < D; ++l) level_off[l + 1] += level_off[l];
        const uint32_t n_leaves = level_off[1];
        std::vector<uint8_t> opv(N);
        std::vector<uint32_t> coff(N + 1, 0);
        std::vector<uint32_t> kids;
        std::vector<int32_t> la(n_leaves), lb(n_leaves);
        std::vector<double> lc(2 * (size_t)n_leaves);
        uint32_t n_ind = 0;
        for (uint32_t i = 0; i < N; ++i) {
            int32_t v = ids[i];
            opv[i] = ns.op[v];
            if (ns.op[v] == OP_IND) ++n_ind;
            if (i < n_leaves) {
                la[i] = ns.la[v];
                lb[i] = ns.lb[v];
                lc[2 * i] = ns.lc[v].real();
                lc[2 * i + 1] = ns.lc[v].imag();
            }
            std::vector<uint32_t> ch;
            for (uint32_t e = ns.coff[v]; e < ns.coff[v + 1]; ++e) ch.push_back((uint32_t)newid[ns.kids[e]]);
            std::sort(ch.begin(), ch.end());
            kids.insert(kids.end(), ch.begin(), ch.end());
            coff[i + 1] = (uint32_t)kids.size();
        }
        std::vector<uint32_t> var_card(ind_card_out);
        std::vector<int32_t> var_tag(ind_vars_tag);
        const uint32_t n_roots = kind == QKC_AC_DENSITY_STEPS ? (uint32_t)roots.size() : 0u;
        const uint32_t n_prior = kind == QKC_AC_TRAJECTORY ? (uint32_t)prior.size() : 0u;
        std::vector<uint8_t> out;
        const uint32_t hdr[16] = {0x43414B51u, 1u, (uint32_t)kind, (uint32_t)n_qubits, (uint32_t)n_angles,
                                  (uint32_t)var_card.size(), N, (uint32_t)kids.size(), D, n_leaves,
                                  (uint32_t)newid[root], n_ind, n_roots, n_prior, 0, 0};
        for (uint32_t h : hdr) put_u32(out, h);
        put_arr(out, var_card);
        put_arr(out, var_tag);
        put_arr(out, level_off);
        put_arr(out, opv);
        put_arr(out, coff);
        put_arr(out, kids);
        put_arr(out, la);
        put_arr(out, lb);
        put_arr(out, lc);
        if (n_roots) {
            std::vector<uint32_t> rr;
            for (int32_t r : roots) rr.push_back((uint32_t)newid[r]);
            put_arr(out, rr);
        }
        if (n_prior) put_arr(out, prior);
        pad8(out);
        uint8_t *buf = (uint8_t *)std::malloc(out.size());
        if (!buf) {
            qkc_set_error_("qkc_compile: out of host memory");
            return QKC_ERR_NOMEM;
        }
        std::memcpy(buf, out.data(), out.size());
        *out_bytes = buf;
        *out_len = out.size();
        return QKC_OK;
    } catch (const TooLarge &) {
        qkc_set_error_("qkc_compile: the AC exceeds max_nodes");
        return QKC_ERR_TOO_LARGE;
    } catch (const std::bad_alloc &) {
        qkc_set_error_("qkc_compile: out of host memory");
        return QKC_ERR_NOMEM;
    }
}

// A step AC under the automatic order: the per-step choice (each step's circuit takes whichever order
// adds fewer nodes to the shared store) is greedy, and one order for every step can share more; so
// min-fill and min-weight throughout are compiled too, and one of them replaces the per-step choice
// when it has at least 10% fewer nodes (a smaller AC is not always a faster one to sample: the split
// of its nodes between the memoised tiers matters too, so small gains are not taken).
extern "C" qkc_status qkc_compile(const qkc_op *ops, int32_t n_ops, int32_t n_qubits, int32_t n_angles,
                                  int32_t kind, int32_t order, int64_t max_nodes, uint8_t **out_bytes,
                                  uint64_t *out_len) {
    qkc_status st = compile_one(ops, n_ops, n_qubits, n_angles, kind, order, max_nodes, out_bytes, out_len);
    if (st != QKC_OK || order != QKC_ORDER_AUTO || kind != QKC_AC_DENSITY_STEPS) return st;
    auto nodes_of = [](const uint8_t *b) {
        uint32_t n;
        std::memcpy(&n, b + 6 * sizeof(uint32_t), sizeof n);  // header word 6: nodes
        return (int64_t)n;
    };
    for (int32_t alt : {QKC_ORDER_MINFILL, QKC_ORDER_MINWEIGHT}) {
        const int64_t best = nodes_of(*out_bytes);
        uint8_t *b = nullptr;
        uint64_t n = 0;
        // (the bound is on the node store, which also holds intermediate nodes the final AC drops)
        const int64_t bound = max_nodes > 0 ? std::min<int64_t>(max_nodes, 16 * best) : 16 * best;
        if (compile_one(ops, n_ops, n_qubits, n_angles, kind, alt, bound, &b, &n) == QKC_OK &&
            (double)nodes_of(b) < 0.9 * (double)best) {
            std::free(*out_bytes);
            *out_bytes = b;
            *out_len = n;
        } else {
            std::free(b);
        }
    }
    qkc_set_error_("");
    return QKC_OK;
}

extern "C" void qkc_free_bytes(uint8_t *bytes) { std::free(bytes); }

extern "C" qkc_status qkc_plan(const qkc_op *ops, int32_t n_ops, int32_t n_qubits, int32_t n_angles,
                               int32_t kind, int32_t order, double *table_entries, double *max_log2_table) {
    if (!table_entries || !max_log2_table || n_qubits <= 0 || n_qubits > 64 || n_ops < 0 ||
        (n_ops > 0 && !ops) || kind < QKC_AC_AMPLITUDE || kind > QKC_AC_TRAJECTORY || order < 0 || order > 3) {
        qkc_set_error_("qkc_plan: invalid argument");
        return QKC_ERR_ARG;
    }
    for (int32_t i = 0; i < n_ops; ++i) {
        const qkc_op &o = ops[i];
        const bool two = (o.kind == 7 || o.kind == 8 || o.kind == 17);
        const bool known = (o.kind >= 0 && o.kind <= 8) || (o.kind >= 16 && o.kind <= 21);
        if (!known || o.q0 < 0 || o.q0 >= n_qubits || (two && (o.q1 < 0 || o.q1 >= n_qubits || o.q1 == o.q0)) ||
            (o.kind >= 4 && o.kind <= 6 && (o.angle < 0 || o.angle >= n_angles))) {
            qkc_set_error_("qkc_plan: invalid operation");
            return QKC_ERR_ARG;
        }
    }
    try {
        NodeStore ns(0x7fffffffLL);
        // light-cone steps: the last step is the whole circuit, the largest of them
        Builder bld(ns, n_qubits, kind == QKC_AC_DENSITY_STEPS ? QKC_AC_DENSITY : kind);
        for (int32_t i = 0; i < n_ops; ++i) bld.op(ops[i]);
        bld.finish();
        double c1 = 0, w1 = 0, c2 = 0, w2 = 0;
        if (order == QKC_ORDER_AUTO) {
            elimination_order(bld.net, QKC_ORDER_MINFILL, &c1, &w1);
            elimination_order(bld.net, QKC_ORDER_MINWEIGHT, &c2, &w2);
            if (c2 < c1) { c1 = c2; w1 = w2; }
        } else {
            elimination_order(bld.net, order, &c1, &w1);
        }
        *table_entries = c1;
        *max_log2_table = w1;
        return QKC_OK;
    } catch (const std::bad_alloc &) {
        qkc_set_error_("qkc_plan: out of host memory");
        return QKC_ERR_NOMEM;
    }
}
