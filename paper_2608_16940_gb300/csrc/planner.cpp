// Fusion planning (§IV-C) and circuit execution.
//
//   - per-gate:   one block per input op (the plain comparator path);
//   - greedy:     extend the current block in circuit order while the union of
//                 targets stays within kmax (the plain width-limit heuristic);
//   - DP:         Eq. dp-recurrence over windows of W ops,
//                 D_i = min_{j in J_i} D_j + Gamma(B(j,i)),
//                 Gamma = 4^k (dense) / 1 (diagonal), ties to the smallest j,
//                 then a greedy cross-window merge (merge neighbours when the
//                 union fits the cap and Gamma(merged) <= Gamma(a) + Gamma(b)),
//                 the whole pipeline repeated on the blocks at most `rounds`
//                 times while the block count falls;
//   - DP-MLP:     the same DP with Gamma(B) = the cost model's predicted
//                 seconds for the block's width and physical target mask; a
//                 diagonal block is one streaming pass, scored as a one-qubit
//                 pass at its lowest physical target.
// Block matrices are formed in FP64 in circuit order, later ops multiplied on
// the left (§IV-C); a block of diagonal ops keeps only its diagonal (Alg. 2,
// diagonal branch) and runs on the streaming kernel, up to QSA_MAX_DIAG wide.
// With opts.layer, a pre-pass first groups the circuit into layer units
// (diagonal gates on at most two qubits, then one-qubit ops whose qubits fit
// one tile), moving an op ahead only of ops it commutes with (the
// semantics-preserving reorder of §IV-C: disjoint targets, or both diagonal);
// the planners then run on the reordered stream, a layer unit counting as one
// pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "qsa.h"
#include "qsa_internal.h"
#include "qsa_runtime.h"
#include "qsa_costmodel.h"

namespace qsa {

namespace {

struct Unit {
    uint64_t mask;       // logical target qubits
    bool diag;
    size_t s, e;         // range of ops (execution order)
    bool prod = false;   // product unit (one-qubit ops on >= 2 qubits), while a block of its own
    bool layer = false;  // layer unit, while a block of its own
    int nd = 0;          // layer unit: its first nd ops are the diagonal part
    bool init = false;   // zero-state prefix (opts.zero_init)
};

using Scorer = double (*)(void* ctx, int width, bool diag, bool prod, uint64_t mask);

// A diagonal or a product block is one streaming pass.
double gamma_score(void*, int width, bool diag, bool prod, uint64_t) {
    return (diag || prod) ? 1.0 : std::ldexp(1.0, 2 * width);
}

struct MlpCtx {
    int n;
    const int32_t* L;
    const CostParams* P;
    std::unordered_map<uint64_t, double> cache;
};

double mlp_score(void* ctx, int width, bool diag, bool prod, uint64_t mask) {
    auto* c = static_cast<MlpCtx*>(ctx);
    diag = diag || prod;   // both run as one streaming pass
    const uint64_t key = mask | (diag ? (1ull << 63) : 0ull);
    auto it = c->cache.find(key);
    if (it != c->cache.end()) return it->second;
    uint64_t pm = 0;
    for (int q = 0; q < c->n; ++q)
        if ((mask >> q) & 1) pm |= 1ull << c->L[q];
    const double v = diag ? costmodel_eval(*c->P, 1, pm & (~pm + 1), c->n, 1)
                          : costmodel_eval(*c->P, width, pm, c->n, 1);
    c->cache[key] = v;
    return v;
}

int popc(uint64_t v) { return __builtin_popcountll(v); }

std::vector<Unit> dp_window(const std::vector<Unit>& u, size_t b, size_t e, int kmax, int kmax_diag, Scorer sc,
                            void* ctx) {
    const size_t h = e - b;
    std::vector<double> D(h + 1, 0.0);
    std::vector<size_t> arg(h + 1, 0);
    for (size_t i = 1; i <= h; ++i) {
        double best = INFINITY;
        size_t bj = i - 1;
        uint64_t mask = 0;
        bool diag = true;
        // walk j downward so the union grows incrementally; keep the
        // smallest j on ties by accepting equal scores as j decreases
        std::vector<std::pair<size_t, double>> cand;
        for (size_t jj = i; jj-- > 0;) {
            mask |= u[b + jj].mask;
            diag = diag && u[b + jj].diag;
            const int w = popc(mask);
            const int cap = diag ? kmax_diag : kmax;
            if (w > cap && jj != i - 1) {
                // widths only grow as j decreases, but a diagonal run can turn
                // dense; the cap of a dense block is >= the diagonal cap, so
                // once the dense cap is exceeded no smaller j is feasible
                if (w > std::max(kmax, kmax_diag)) break;
                continue;
            }
            const double val = D[jj] + sc(ctx, w, diag, jj == i - 1 && (u[b + jj].prod || u[b + jj].layer), mask);
            if (val <= best) {
                best = val;
                bj = jj;
            }
        }
        D[i] = best;
        arg[i] = bj;
    }
    std::vector<Unit> out;
    size_t i = h;
    while (i > 0) {
        size_t j = arg[i];
        Unit m{0, true, u[b + j].s, u[b + i - 1].e};
        for (size_t t = j; t < i; ++t) {
            m.mask |= u[b + t].mask;
            m.diag = m.diag && u[b + t].diag;
        }
        m.prod = i - j == 1 && u[b + j].prod;
        m.layer = i - j == 1 && u[b + j].layer;
        m.nd = m.layer ? u[b + j].nd : 0;
        out.push_back(m);
        i = j;
    }
    std::reverse(out.begin(), out.end());
    return out;
}

std::vector<Unit> merge_pass(const std::vector<Unit>& blocks, int kmax, int kmax_diag, Scorer sc, void* ctx) {
    std::vector<Unit> out;
    if (blocks.empty()) return out;
    Unit cur = blocks[0];
    for (size_t i = 1; i < blocks.size(); ++i) {
        const Unit& nx = blocks[i];
        const uint64_t m = cur.mask | nx.mask;
        const bool dg = cur.diag && nx.diag;
        const int w = popc(m);
        const int cap = dg ? kmax_diag : kmax;
        if (w <= cap && sc(ctx, w, dg, false, m) <=
                            sc(ctx, popc(cur.mask), cur.diag, cur.prod || cur.layer, cur.mask) +
                                sc(ctx, popc(nx.mask), nx.diag, nx.prod || nx.layer, nx.mask)) {
            cur = Unit{m, dg, cur.s, nx.e};
        } else {
            out.push_back(cur);
            cur = nx;
        }
    }
    out.push_back(cur);
    return out;
}

std::vector<Unit> dp_pipeline(const std::vector<Unit>& gates, const qsa_plan_opts& o, Scorer sc, void* ctx) {
    std::vector<Unit> units = gates;
    for (int round = 0; round < o.rounds; ++round) {
        std::vector<Unit> blocks;
        for (size_t b = 0; b < units.size(); b += static_cast<size_t>(o.window)) {
            size_t e = std::min(units.size(), b + static_cast<size_t>(o.window));
            auto w = dp_window(units, b, e, o.kmax, o.kmax_diag, sc, ctx);
            blocks.insert(blocks.end(), w.begin(), w.end());
        }
        blocks = merge_pass(blocks, o.kmax, o.kmax_diag, sc, ctx);
        if (round > 0 && blocks.size() >= units.size()) break;
        units.swap(blocks);
    }
    return units;
}

std::vector<Unit> greedy(const std::vector<Unit>& gates, int kmax) {
    std::vector<Unit> out;
    if (gates.empty()) return out;
    Unit cur = gates[0];
    for (size_t i = 1; i < gates.size(); ++i) {
        uint64_t m = cur.mask | gates[i].mask;
        if (popc(m) > kmax) {
            out.push_back(cur);
            cur = gates[i];
        } else {
            cur = Unit{m, cur.diag && gates[i].diag, cur.s, gates[i].e};
        }
    }
    out.push_back(cur);
    return out;
}

qsa_status validate_ops(const qsa_op* ops, size_t n_ops, int n_qubits) {
    if (n_ops > 0 && !ops) return fail(QSA_E_ARG, "ops is NULL");
    for (size_t i = 0; i < n_ops; ++i) {
        qsa_status st = validate_targets(n_qubits, ops[i].targets, ops[i].k);
        if (st != QSA_OK) return st;
        if (!ops[i].matrix) return fail(QSA_E_ARG, "op matrix is NULL");
        if (ops[i].flags & QSA_OP_DIAG) {
            const size_t d = size_t(1) << ops[i].k;
            for (size_t r = 0; r < d; ++r)
                for (size_t c = 0; c < d; ++c)
                    if (r != c && (ops[i].matrix[2 * (r * d + c)] != 0.0 || ops[i].matrix[2 * (r * d + c) + 1] != 0.0))
                        return fail(QSA_E_ARG, "op flagged QSA_OP_DIAG has a nonzero off-diagonal entry");
        }
    }
    return QSA_OK;
}

qsa_status normalise_opts(const qsa_plan_opts* in, qsa_plan_opts* o) {
    if (in) *o = *in; else qsa_plan_opts_default(o);
    if (o->planner < 0 || o->planner > 3) return fail(QSA_E_ARG, "unknown planner");
    if (o->kmax < 1 || o->kmax > QSA_MAX_K) return fail(QSA_E_ARG, "kmax must be in 1..6");
    if (o->kmax_diag < 1 || o->kmax_diag > QSA_MAX_DIAG) return fail(QSA_E_ARG, "kmax_diag must be in 1..12");
    if (o->window < 1) return fail(QSA_E_ARG, "window must be >= 1");
    if (o->rounds < 1 || o->rounds > 4) return fail(QSA_E_ARG, "rounds must be in 1..4");
    if (o->precision < 0 || o->precision > 1) return fail(QSA_E_ARG, "unknown precision");
    if (o->lowering < 0 || o->lowering > 2) return fail(QSA_E_ARG, "unknown lowering");
    if (o->victim < 0 || o->victim > 1) return fail(QSA_E_ARG, "unknown victim rule");
    if (o->kmax_prod < 0 || o->kmax_prod > QSA_MAX_PROD) return fail(QSA_E_ARG, "kmax_prod must be in 0..11");
    if (o->layer < 0 || o->layer > 1) return fail(QSA_E_ARG, "layer must be 0 or 1");
    if (o->zero_init < 0 || o->zero_init > 1) return fail(QSA_E_ARG, "zero_init must be 0 or 1");
    return QSA_OK;
}

// next_use[i * n + q]: index of the first dense block after block i that
// targets logical qubit q (INT32_MAX for none).
void build_next_use(qsa_plan_s* p) {
    const size_t B = p->blocks.size();
    const int n = p->n;
    p->next_use.assign(B * n, INT32_MAX);
    std::vector<int32_t> cur(n, INT32_MAX);
    for (size_t i = B; i-- > 0;) {
        std::copy(cur.begin(), cur.end(), p->next_use.begin() + i * n);
        const PlanBlock& b = p->blocks[i];
        if (!b.diag && !b.prod && b.layer < 0)
            for (int j = 0; j < b.k; ++j) cur[b.t[j]] = static_cast<int32_t>(i);
    }
}

uint64_t op_mask(const qsa_op& op) {
    uint64_t m = 0;
    for (int j = 0; j < op.k; ++j) m |= 1ull << op.targets[j];
    return m;
}

// Layer pre-pass.  From the front of the pending stream: an op that is neither
// one-qubit nor a diagonal gate on <= 2 qubits is a plain unit; otherwise a
// layer unit is grown over the pending ops in circuit order -- a diagonal
// gate on <= 2 qubits joins the diagonal part if no factor of the unit and no
// skipped non-diagonal op touches its qubits; a one-qubit op joins its
// qubit's factor if no skipped op touches the qubit and the factor qubits'
// positions (layout L) still fit a tile; anything else is skipped and blocks
// its qubits (all ops if it is non-diagonal, non-diagonal ops if diagonal).
// The scan ends after more than 256 skips.  The unit executes its diagonal
// part, then its factor ops (each in circuit order); skipped ops stay pending.
void layer_prepass(const qsa_op* ops, size_t n_ops, int n, const int32_t* L, std::vector<size_t>* order,
                   std::vector<Unit>* units) {
    constexpr int kLookahead = 256;
    std::vector<size_t> pending(n_ops);
    std::iota(pending.begin(), pending.end(), size_t(0));
    std::vector<char> taken(n_ops, 0);
    while (!pending.empty()) {
        const qsa_op& first = ops[pending[0]];
        const bool first_diag = (first.flags & QSA_OP_DIAG) != 0;
        if (!(first.k == 1 || (first_diag && first.k <= 2))) {
            units->push_back(Unit{op_mask(first), first_diag, order->size(), order->size() + 1});
            order->push_back(pending[0]);
            pending.erase(pending.begin());
            continue;
        }
        std::vector<size_t> dpart, fpart;
        uint64_t fq = 0, blocked_nondiag = 0, blocked_all = 0, all = 0;
        std::vector<int> fpos;
        int skips = 0;
        for (size_t idx : pending) {
            const qsa_op& op = ops[idx];
            const uint64_t Q = op_mask(op);
            const bool dg = (op.flags & QSA_OP_DIAG) != 0;
            if (dg && op.k <= 2 && !(Q & fq) && !(Q & blocked_nondiag)) {
                dpart.push_back(idx);
                all |= Q;
                continue;
            }
            if (op.k == 1 && !(Q & blocked_all)) {
                bool fits = (Q & fq) != 0;
                if (!fits) {
                    fpos.push_back(L[op.targets[0]]);
                    fits = layer_fits(n, fpos.data(), static_cast<int>(fpos.size()));
                    fpos.pop_back();
                }
                if (fits) {
                    if (!(Q & fq)) fpos.push_back(L[op.targets[0]]);
                    fpart.push_back(idx);
                    fq |= Q;
                    all |= Q;
                    continue;
                }
            }
            blocked_all |= Q;
            if (!dg) blocked_nondiag |= Q;
            if (++skips > kLookahead) break;
        }
        Unit u{all, false, order->size(), order->size() + dpart.size() + fpart.size()};
        u.layer = true;
        u.nd = static_cast<int>(dpart.size());
        units->push_back(u);
        for (size_t x : dpart) {
            order->push_back(x);
            taken[x] = 1;
        }
        for (size_t x : fpart) {
            order->push_back(x);
            taken[x] = 1;
        }
        std::vector<size_t> rest;
        rest.reserve(pending.size());
        for (size_t x : pending)
            if (!taken[x]) rest.push_back(x);
        pending.swap(rest);
    }
}

// Zero-state prefix: ops are taken in circuit order while each is a one-qubit
// op on a qubit no taken diagonal gate touches, or a diagonal gate on at most
// two qubits.
size_t zero_init_prefix(const qsa_op* ops, size_t n_ops) {
    uint64_t diag_touched = 0;
    for (size_t i = 0; i < n_ops; ++i) {
        const uint64_t Q = op_mask(ops[i]);
        if (ops[i].k == 1 && !(Q & diag_touched)) continue;
        if ((ops[i].flags & QSA_OP_DIAG) && ops[i].k <= 2) {
            diag_touched |= Q;
            continue;
        }
        return i;
    }
    return n_ops;
}

// Units over the execution order *order (the identity unless the layer
// pre-pass moved ops), then the planner; with opts.zero_init the zero-state
// prefix is one unit ahead of the rest.
std::vector<Unit> plan(const qsa_op* ops, size_t n_ops, int n_qubits, const qsa_plan_opts& o, const int32_t* L,
                       std::vector<size_t>* order, const CostModel& model) {
    const size_t P = o.zero_init ? zero_init_prefix(ops, n_ops) : 0;
    if (P > 0) {
        qsa_plan_opts rest_opts = o;
        rest_opts.zero_init = 0;
        std::vector<size_t> rest_order;
        std::vector<Unit> rest = plan(ops + P, n_ops - P, n_qubits, rest_opts, L, &rest_order, model);
        order->clear();
        for (size_t i = 0; i < P; ++i) order->push_back(i);
        for (size_t x : rest_order) order->push_back(x + P);
        std::vector<Unit> units;
        Unit u{0, false, 0, P};
        u.init = true;
        units.push_back(u);
        for (Unit r : rest) {
            r.s += P;
            r.e += P;
            units.push_back(r);
        }
        return units;
    }
    int32_t ident[QSA_MAX_QUBITS];
    for (int q = 0; q < n_qubits; ++q) ident[q] = q;
    order->clear();
    std::vector<Unit> gates;
    if (o.layer && o.planner != QSA_PLAN_PER_GATE) {
        layer_prepass(ops, n_ops, n_qubits, L ? L : ident, order, &gates);
    } else {
        order->resize(n_ops);
        std::iota(order->begin(), order->end(), size_t(0));
    }
    gates.reserve(n_ops);
    for (size_t i = 0; i < n_ops && !(o.layer && o.planner != QSA_PLAN_PER_GATE);) {
        auto one_qubit = [&](size_t x) { return ops[x].k == 1 && !(ops[x].flags & QSA_OP_DIAG); };
        if (o.kmax_prod >= 2 && o.planner != QSA_PLAN_PER_GATE && one_qubit(i)) {
            // product unit: a maximal run of non-diagonal one-qubit ops on at most kmax_prod qubits
            uint64_t m = 1ull << ops[i].targets[0];
            size_t j = i + 1;
            while (j < n_ops && one_qubit(j)) {
                const uint64_t nm = m | (1ull << ops[j].targets[0]);
                if (nm != m && popc(m) == o.kmax_prod) break;
                m = nm;
                ++j;
            }
            Unit u{m, false, i, j};
            u.prod = popc(m) >= 2;
            gates.push_back(u);
            i = j;
            continue;
        }
        uint64_t m = 0;
        for (int j = 0; j < ops[i].k; ++j) m |= 1ull << ops[i].targets[j];
        gates.push_back(Unit{m, (ops[i].flags & QSA_OP_DIAG) != 0, i, i + 1});
        ++i;
    }
    if (o.planner == QSA_PLAN_PER_GATE) return gates;
    if (o.planner == QSA_PLAN_GREEDY) return greedy(gates, o.kmax);
    if (o.planner == QSA_PLAN_DP_MLP) {
        if (!model) return greedy(gates, o.kmax);   // no network: the width-limit heuristic
        if (!L) L = ident;
        MlpCtx ctx{n_qubits, L, model.get(), {}};
        return dp_pipeline(gates, o, mlp_score, &ctx);
    }
    return dp_pipeline(gates, o, gamma_score, nullptr);
}

// M <- E(op) M for the D x D block matrix M (row-major), op on block positions pos[].
void left_multiply(std::vector<std::complex<double>>& M, int u, const int* pos, int k, const double* g) {
    const size_t D = size_t(1) << u, d = size_t(1) << k;
    size_t opmask = 0;
    for (int j = 0; j < k; ++j) opmask |= size_t(1) << pos[j];
    std::vector<size_t> off(d);
    for (size_t c = 0; c < d; ++c) {
        size_t o = 0;
        for (int j = 0; j < k; ++j)
            if ((c >> j) & 1) o |= size_t(1) << pos[j];
        off[c] = o;
    }
    // whole rows at a time (contiguous, real arithmetic): rows x | off[r] of
    // the product are sum_c g[r][c] * rows x | off[c], summed in c order
    double* m = reinterpret_cast<double*>(M.data());
    std::vector<double> in(2 * d * D);
    for (size_t x = 0; x < D; ++x) {
        if (x & opmask) continue;
        for (size_t c = 0; c < d; ++c)
            std::copy(m + 2 * (x | off[c]) * D, m + 2 * ((x | off[c]) * D + D), in.data() + 2 * c * D);
        for (size_t r = 0; r < d; ++r) {
            double* out = m + 2 * (x | off[r]) * D;
            std::fill(out, out + 2 * D, 0.0);
            for (size_t c = 0; c < d; ++c) {
                const double gr = g[2 * (r * d + c)], gi = g[2 * (r * d + c) + 1];
                const double* v = in.data() + 2 * c * D;
                for (size_t col = 0; col < D; ++col) {
                    const double vr = v[2 * col], vi = v[2 * col + 1];
                    out[2 * col] += gr * vr - gi * vi;
                    out[2 * col + 1] += gr * vi + gi * vr;
                }
            }
        }
    }
}

// Fused matrix of ops[s..e) on the ascending union of their targets.
qsa_status fuse_range(const qsa_op* ops, size_t s, size_t e, int32_t* tgt, int* width, std::vector<double>* out) {
    uint64_t m = 0;
    for (size_t i = s; i < e; ++i)
        for (int j = 0; j < ops[i].k; ++j) m |= 1ull << ops[i].targets[j];
    const int u = popc(m);
    if (u > QSA_MAX_K) return fail(QSA_E_ARG, "fused block wider than 6 qubits");
    int t = 0;
    for (int q = 0; q < 64; ++q)
        if ((m >> q) & 1) tgt[t++] = q;
    *width = u;
    const size_t D = size_t(1) << u;
    std::vector<std::complex<double>> M(D * D, 0.0);
    for (size_t i = 0; i < D; ++i) M[i * D + i] = 1.0;
    for (size_t i = s; i < e; ++i) {
        int pos[QSA_MAX_K];
        for (int j = 0; j < ops[i].k; ++j) pos[j] = static_cast<int>(std::find(tgt, tgt + u, ops[i].targets[j]) - tgt);
        left_multiply(M, u, pos, ops[i].k, ops[i].matrix);
    }
    out->resize(2 * D * D);
    for (size_t i = 0; i < D * D; ++i) {
        (*out)[2 * i] = M[i].real();
        (*out)[2 * i + 1] = M[i].imag();
    }
    return QSA_OK;
}

// Diagonal of the fused block of diagonal ops ops[s..e) on the ascending union
// of their targets: entry c is the product, in circuit order, of each op's
// diagonal entry at the bits of c that are its targets.
qsa_status fuse_diag_range(const qsa_op* ops, size_t s, size_t e, int32_t* tgt, int* width, std::vector<double>* out) {
    uint64_t m = 0;
    for (size_t i = s; i < e; ++i)
        for (int j = 0; j < ops[i].k; ++j) m |= 1ull << ops[i].targets[j];
    const int u = popc(m);
    if (u > QSA_MAX_DIAG) return fail(QSA_E_ARG, "diagonal block wider than 12 qubits");
    int t = 0;
    for (int q = 0; q < 64; ++q)
        if ((m >> q) & 1) tgt[t++] = q;
    *width = u;
    const size_t D = size_t(1) << u;
    std::vector<std::complex<double>> d(D, 1.0);
    for (size_t i = s; i < e; ++i) {
        const qsa_op& op = ops[i];
        int pos[QSA_MAX_K];
        for (int j = 0; j < op.k; ++j) pos[j] = static_cast<int>(std::find(tgt, tgt + u, op.targets[j]) - tgt);
        const size_t dk = size_t(1) << op.k;
        for (size_t c = 0; c < D; ++c) {
            size_t gi = 0;
            for (int j = 0; j < op.k; ++j) gi |= ((c >> pos[j]) & 1) << j;
            d[c] = std::complex<double>(op.matrix[2 * (gi * dk + gi)], op.matrix[2 * (gi * dk + gi) + 1]) * d[c];
        }
    }
    out->resize(2 * D);
    for (size_t c = 0; c < D; ++c) {
        (*out)[2 * c] = d[c].real();
        (*out)[2 * c + 1] = d[c].imag();
    }
    return QSA_OK;
}

}  // namespace

}  // namespace qsa

using namespace qsa;

extern "C" {

void qsa_plan_opts_default(qsa_plan_opts* o) {
    if (!o) return;
    o->planner = QSA_PLAN_DP;
    o->kmax = 4;
    o->kmax_diag = 4;
    o->window = 64;
    o->rounds = 4;
    o->precision = QSA_PREC_FP32;
    o->lowering = QSA_LOWER_AUTO;
    o->timing = 0;
    o->victim = QSA_VICTIM_FIRST_FREE;
    o->kmax_prod = 0;
    o->layer = 0;
    o->zero_init = 0;
}

qsa_status qsa_plan_circuit(const qsa_op* ops, size_t n_ops, int n_qubits, const qsa_plan_opts* opts,
                            size_t* block_start, size_t* n_blocks) {
    if (n_qubits < 1 || n_qubits > QSA_MAX_QUBITS) return fail(QSA_E_ARG, "n_qubits must be in 1..34");
    if (!n_blocks || (n_ops > 0 && !block_start)) return fail(QSA_E_ARG, "NULL output");
    qsa_plan_opts o;
    qsa_status st = normalise_opts(opts, &o);
    if (st != QSA_OK) return st;
    st = validate_ops(ops, n_ops, n_qubits);
    if (st != QSA_OK) return st;
    std::vector<size_t> order;
    auto blocks = plan(ops, n_ops, n_qubits, o, nullptr, &order, costmodel_global());
    for (size_t i = 0; i < blocks.size(); ++i) block_start[i] = blocks[i].s;
    *n_blocks = blocks.size();
    return QSA_OK;
}

qsa_status qsa_fuse_ops(const qsa_op* ops, size_t n_ops, int32_t* block_targets_out, int* width_out,
                        double* matrix_out) {
    if (!ops || n_ops == 0 || !block_targets_out || !width_out || !matrix_out) return fail(QSA_E_ARG, "NULL argument");
    for (size_t i = 0; i < n_ops; ++i) {
        qsa_status st = validate_targets(QSA_MAX_QUBITS, ops[i].targets, ops[i].k);
        if (st != QSA_OK) return st;
        if (!ops[i].matrix) return fail(QSA_E_ARG, "op matrix is NULL");
    }
    std::vector<double> M;
    qsa_status st = fuse_range(ops, 0, n_ops, block_targets_out, width_out, &M);
    if (st != QSA_OK) return st;
    std::memcpy(matrix_out, M.data(), sizeof(double) * M.size());
    return QSA_OK;
}

qsa_status qsa_plan_create(const qsa_op* ops, size_t n_ops, int n_qubits, const qsa_plan_opts* opts,
                           const int32_t* layout, qsa_plan* out) {
    return plan_create(ops, n_ops, n_qubits, opts, layout, costmodel_global(), out);
}

}  // extern "C"

namespace qsa {

qsa_status plan_create(const qsa_op* ops, size_t n_ops, int n_qubits, const qsa_plan_opts* opts,
                       const int32_t* layout, const CostModel& model, qsa_plan* out) {
    if (!out) return fail(QSA_E_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > QSA_MAX_QUBITS) return fail(QSA_E_ARG, "n_qubits must be in 1..34");
    qsa_plan_opts o;
    qsa_status st = normalise_opts(opts, &o);
    if (st != QSA_OK) return st;
    st = validate_ops(ops, n_ops, n_qubits);
    if (st != QSA_OK) return st;
    if (layout) {
        uint64_t seen = 0;
        for (int q = 0; q < n_qubits; ++q) {
            if (layout[q] < 0 || layout[q] >= n_qubits || ((seen >> layout[q]) & 1))
                return fail(QSA_E_ARG, "layout is not a bijection");
            seen |= 1ull << layout[q];
        }
    }
    auto* p = new qsa_plan_s();
    p->n = n_qubits;
    p->opts = o;
    p->n_ops = n_ops;
    p->L0.resize(n_qubits);
    for (int q = 0; q < n_qubits; ++q) p->L0[q] = layout ? layout[q] : q;
    auto blocks = plan(ops, n_ops, n_qubits, o, layout, &p->order, model);
    // the ops in execution order
    std::vector<qsa_op> perm(n_ops);
    for (size_t i = 0; i < n_ops; ++i) perm[i] = ops[p->order[i]];
    ops = perm.data();
    p->blocks.resize(blocks.size());
    std::vector<double> M;
    ModulusCarry carry;   // modulus errors of the plan's FP32 constants (error feedback)
    for (size_t i = 0; i < blocks.size(); ++i) {
        const Unit& u = blocks[i];
        PlanBlock& b = p->blocks[i];
        b.off = p->host_mat.size();
        b.first_op = u.s;
        if (u.init) {
            // zero-state preparation: each qubit's one-qubit ops applied to |0>
            // as a one-qubit diagonal on an all-ones input, then the diagonal gates
            PlanLayer pl;
            pl.spec.generate = true;
            std::vector<std::array<std::complex<double>, 2>> a(n_qubits, {1.0, 0.0});
            std::vector<LayerDiagOp> gates;
            uint64_t diag_touched = 0;
            for (size_t x = u.s; x < u.e; ++x) {
                const uint64_t Q = op_mask(ops[x]);
                if (ops[x].k == 1 && !(Q & diag_touched)) {
                    const int q = ops[x].targets[0];
                    const double* g = ops[x].matrix;
                    const std::complex<double> h00(g[0], g[1]), h01(g[2], g[3]), h10(g[4], g[5]), h11(g[6], g[7]);
                    a[q] = {h00 * a[q][0] + h01 * a[q][1], h10 * a[q][0] + h11 * a[q][1]};
                } else {
                    LayerDiagOp d;
                    st = layer_diag_from_op(ops[x], &d);
                    if (st != QSA_OK) {
                        delete p;
                        return st;
                    }
                    gates.push_back(d);
                    diag_touched |= Q;
                }
            }
            for (int q = 0; q < n_qubits; ++q) {
                LayerDiagOp d;
                d.k = 1;
                d.q[0] = q;
                d.d[0] = a[q][0];
                d.d[1] = a[q][1];
                pl.spec.diag.push_back(d);
            }
            pl.spec.diag.insert(pl.spec.diag.end(), gates.begin(), gates.end());
            b.init = true;
            b.layer = static_cast<int>(p->layers.size());
            b.k = 0;
            p->layers.push_back(std::move(pl));
            continue;
        }
        if (u.layer) {
            // diagonal part, then per-qubit factor products (qubits ascending,
            // later ops on the left)
            PlanLayer pl;
            for (size_t x = u.s; x < u.s + static_cast<size_t>(u.nd); ++x) {
                LayerDiagOp d;
                st = layer_diag_from_op(ops[x], &d);
                if (st != QSA_OK) {
                    delete p;
                    return st;
                }
                pl.spec.diag.push_back(d);
            }
            std::map<int, std::array<std::complex<double>, 4>> fac;
            for (size_t x = u.s + static_cast<size_t>(u.nd); x < u.e; ++x) {
                const int q = ops[x].targets[0];
                auto it = fac.find(q);
                std::array<std::complex<double>, 4> f =
                    it == fac.end() ? std::array<std::complex<double>, 4>{1.0, 0.0, 0.0, 1.0} : it->second;
                const double* g = ops[x].matrix;
                std::complex<double> h[4];
                for (int c = 0; c < 4; ++c) h[c] = std::complex<double>(g[2 * c], g[2 * c + 1]);
                fac[q] = {h[0] * f[0] + h[1] * f[2], h[0] * f[1] + h[1] * f[3], h[2] * f[0] + h[3] * f[2],
                          h[2] * f[1] + h[3] * f[3]};
            }
            for (const auto& kv : fac) {
                pl.spec.t.push_back(kv.first);
                pl.spec.f.push_back(kv.second);
            }
            b.layer = static_cast<int>(p->layers.size());
            b.n_diag = u.nd;
            b.k = static_cast<int>(pl.spec.t.size());
            for (int j = 0; j < b.k; ++j) b.t[j] = pl.spec.t[j];
            p->layers.push_back(std::move(pl));
            continue;
        }
        if (u.prod) {
            // per-qubit factors (ascending qubits), each the product of its ops in
            // circuit order, later ops on the left
            b.prod = true;
            int t = 0;
            for (int q = 0; q < 64; ++q)
                if ((u.mask >> q) & 1) b.t[t++] = q;
            b.k = t;
            std::vector<std::complex<double>> F(4 * t);
            for (int j = 0; j < t; ++j) {
                F[4 * j] = 1.0;
                F[4 * j + 3] = 1.0;
            }
            for (size_t x = u.s; x < u.e; ++x) {
                const int j = static_cast<int>(std::find(b.t, b.t + t, ops[x].targets[0]) - b.t);
                const double* g = ops[x].matrix;
                std::complex<double> f[4], h[4];
                for (int c = 0; c < 4; ++c) {
                    f[c] = F[4 * j + c];
                    h[c] = std::complex<double>(g[2 * c], g[2 * c + 1]);
                }
                F[4 * j] = h[0] * f[0] + h[1] * f[2];
                F[4 * j + 1] = h[0] * f[1] + h[1] * f[3];
                F[4 * j + 2] = h[2] * f[0] + h[3] * f[2];
                F[4 * j + 3] = h[2] * f[1] + h[3] * f[3];
            }
            p->host_mat.resize(b.off + 8 * t);
            for (int c = 0; c < 4 * t; ++c) {
                p->host_mat[b.off + 2 * c] = static_cast<float>(F[c].real());
                p->host_mat[b.off + 2 * c + 1] = static_cast<float>(F[c].imag());
            }
        } else if (u.diag) {
            b.diag = true;
            st = fuse_diag_range(ops, u.s, u.e, b.t, &b.k, &M);
            if (st != QSA_OK) {
                delete p;
                return st;
            }
            p->host_mat.resize(b.off + M.size());
            to_float_moduli(M.data(), M.size() / 2, p->host_mat.data() + b.off, 1.0 / static_cast<double>(M.size() / 2),
                            &carry);
        } else if (u.e - u.s == 1) {
            const qsa_op& op = ops[u.s];
            b.k = op.k;
            for (int j = 0; j < op.k; ++j) b.t[j] = op.targets[j];
            const size_t cnt = 2ull << (2 * op.k);
            p->host_mat.resize(b.off + cnt);
            to_float_matrix(op.matrix, op.k, p->host_mat.data() + b.off);
        } else {
            st = fuse_range(ops, u.s, u.e, b.t, &b.k, &M);
            if (st != QSA_OK) {
                delete p;
                return st;
            }
            p->host_mat.resize(b.off + M.size());
            for (size_t j = 0; j < M.size(); ++j) p->host_mat[b.off + j] = static_cast<float>(M[j]);
        }
        p->max_width = std::max(p->max_width, b.k);
        while (p->host_mat.size() % 4) p->host_mat.push_back(0.f);  // 16-byte aligned matrices
    }
    // the zero-state block takes over the layer block after it: the generated
    // product state passes through that block's diagonal part and factors in
    // the same write-only pass (its record is left empty and never referenced)
    if (p->blocks.size() >= 2 && p->blocks[0].init && p->blocks[1].layer >= 0 && !p->blocks[1].init) {
        LayerSpec& a = p->layers[p->blocks[0].layer].spec;
        LayerSpec& b = p->layers[p->blocks[1].layer].spec;
        a.diag.insert(a.diag.end(), b.diag.begin(), b.diag.end());
        a.t = b.t;
        a.f = b.f;
        b = LayerSpec{};
        PlanBlock& b0 = p->blocks[0];
        b0.k = p->blocks[1].k;
        for (int j = 0; j < b0.k; ++j) b0.t[j] = p->blocks[1].t[j];
        b0.n_diag = static_cast<int>(a.diag.size());
        p->blocks.erase(p->blocks.begin() + 1);
    }
    // consecutive layer blocks: the exit phases of each block's factors move
    // to the next block's diagonal part; then every layer block's passes for
    // the plan's layout
    for (size_t i = 0; i + 1 < p->blocks.size(); ++i)
        if (p->blocks[i].layer >= 0 && p->blocks[i + 1].layer >= 0)
            layer_move_exit_phases(&p->layers[p->blocks[i].layer].spec, &p->layers[p->blocks[i + 1].layer].spec);
    for (PlanLayer& pl : p->layers)
        pl.launches = prepare_layer(n_qubits, p->L0.data(), pl.spec, &p->host_layer, &carry);
    build_next_use(p);
    *out = p;
    return QSA_OK;
}

}  // namespace qsa

extern "C" {

qsa_status qsa_plan_promotions(qsa_plan p, const int32_t* layout_in, int victim, uint64_t* promotions,
                               uint64_t* passes, int32_t* layout_out) {
    if (!p) return fail(QSA_E_ARG, "plan is NULL");
    if (victim < 0 || victim > 1) return fail(QSA_E_ARG, "unknown victim rule");
    const int n = p->n;
    int32_t L[QSA_MAX_QUBITS];
    uint64_t seen = 0;
    for (int q = 0; q < n; ++q) {
        L[q] = layout_in ? layout_in[q] : q;
        if (L[q] < 0 || L[q] >= n || ((seen >> L[q]) & 1)) return fail(QSA_E_ARG, "layout is not a bijection");
        seen |= 1ull << L[q];
    }
    const int frames = std::min(kInBlockBits, n);
    uint64_t pr = 0, ps = 0;
    for (size_t i = 0; i < p->blocks.size(); ++i) {
        const PlanBlock& b = p->blocks[i];
        if (b.diag || b.prod || b.layer >= 0) continue;
        int phys[QSA_MAX_K], pa[QSA_MAX_K], pb[QSA_MAX_K];
        for (int j = 0; j < b.k; ++j) phys[j] = L[b.t[j]];
        const int np = choose_promotions(L, n, phys, b.k, frames, victim, p->next_use.data() + i * n, pa, pb);
        if (np < 0) return fail(QSA_E_ARG, "block wider than the in-block frames");
        // swap the logical qubits at each position pair, in order
        for (int m = 0; m < np; ++m) {
            int qa = -1, qb = -1;
            for (int q = 0; q < n; ++q) {
                if (L[q] == pa[m]) qa = q;
                if (L[q] == pb[m]) qb = q;
            }
            L[qa] = pb[m];
            L[qb] = pa[m];
        }
        pr += static_cast<uint64_t>(np);
        ps += np > 0 ? 1 : 0;
    }
    if (promotions) *promotions = pr;
    if (passes) *passes = ps;
    if (layout_out) std::memcpy(layout_out, L, sizeof(int32_t) * n);
    return QSA_OK;
}

qsa_status qsa_plan_exchanges(qsa_plan p, int rank_bits, const int32_t* layout_in, int victim, qsa_exchange* out,
                              size_t capacity, size_t* n_out, int32_t* layout_out) {
    if (!p || !n_out) return fail(QSA_E_ARG, "NULL argument");
    if (victim < 0 || victim > 1) return fail(QSA_E_ARG, "unknown victim rule");
    const int n = p->n;
    if (rank_bits < 1 || rank_bits >= n) return fail(QSA_E_ARG, "rank_bits must be in 1..N-1");
    const int local = n - rank_bits;
    int32_t L[QSA_MAX_QUBITS];
    uint64_t seen = 0;
    for (int q = 0; q < n; ++q) {
        L[q] = layout_in ? layout_in[q] : q;
        if (L[q] < 0 || L[q] >= n || ((seen >> L[q]) & 1)) return fail(QSA_E_ARG, "layout is not a bijection");
        seen |= 1ull << L[q];
    }
    // next use of each logical qubit by a block that needs its qubits local
    // (every block but the diagonal ones: a rank fixes its own rank bits)
    const size_t B = p->blocks.size();
    std::vector<int32_t> next(B * static_cast<size_t>(n), INT32_MAX), cur(n, INT32_MAX);
    for (size_t i = B; i-- > 0;) {
        std::copy(cur.begin(), cur.end(), next.begin() + i * n);
        const PlanBlock& b = p->blocks[i];
        if (!b.diag)
            for (int j = 0; j < b.k; ++j) cur[b.t[j]] = static_cast<int32_t>(i);
    }
    size_t cnt = 0;
    for (size_t i = 0; i < B; ++i) {
        const PlanBlock& b = p->blocks[i];
        if (b.diag) continue;
        if (b.k > local) return fail(QSA_E_ARG, "a block is wider than the local positions of a rank");
        int phys[QSA_MAX_DIAG], pa[QSA_MAX_DIAG], pb[QSA_MAX_DIAG];
        for (int j = 0; j < b.k; ++j) phys[j] = L[b.t[j]];
        const int np = choose_promotions(L, n, phys, b.k, local, victim, next.data() + i * n, pa, pb);
        if (np < 0) return fail(QSA_E_ARG, "not enough free local positions");
        for (int m = 0; m < np; ++m) {
            if (out && cnt < capacity) out[cnt] = qsa_exchange{static_cast<uint64_t>(i), pa[m], pb[m]};
            ++cnt;
            int qa = -1, qb = -1;
            for (int q = 0; q < n; ++q) {
                if (L[q] == pa[m]) qa = q;
                if (L[q] == pb[m]) qb = q;
            }
            L[qa] = pb[m];
            L[qb] = pa[m];
        }
    }
    *n_out = cnt;
    if (layout_out) std::memcpy(layout_out, L, sizeof(int32_t) * n);
    if (cnt > capacity) return fail(QSA_E_RANGE, "capacity smaller than the number of exchanges");
    return QSA_OK;
}

qsa_status qsa_plan_info(qsa_plan p, size_t* n_blocks, size_t* n_ops, int* max_width, size_t* matrix_bytes) {
    if (!p) return fail(QSA_E_ARG, "plan is NULL");
    if (n_blocks) *n_blocks = p->blocks.size();
    if (n_ops) *n_ops = p->n_ops;
    if (max_width) *max_width = p->max_width;
    if (matrix_bytes) *matrix_bytes = p->host_mat.size() * sizeof(float);
    return QSA_OK;
}

qsa_status qsa_plan_blocks(qsa_plan p, size_t* first_op, int32_t* widths, size_t capacity) {
    if (!p) return fail(QSA_E_ARG, "plan is NULL");
    if (capacity < p->blocks.size()) return fail(QSA_E_RANGE, "capacity smaller than the number of blocks");
    for (size_t i = 0; i < p->blocks.size(); ++i) {
        if (first_op) first_op[i] = p->blocks[i].first_op;
        if (widths) widths[i] = p->blocks[i].k;
    }
    return QSA_OK;
}

qsa_status qsa_plan_order(qsa_plan p, size_t* order, size_t capacity) {
    if (!p || !order) return fail(QSA_E_ARG, "NULL argument");
    if (capacity < p->n_ops) return fail(QSA_E_RANGE, "capacity smaller than the number of ops");
    for (size_t i = 0; i < p->n_ops; ++i) order[i] = i < p->order.size() ? p->order[i] : i;
    return QSA_OK;
}

qsa_status qsa_plan_block_kinds(qsa_plan p, int32_t* kinds, int32_t* n_diag, size_t capacity) {
    if (!p) return fail(QSA_E_ARG, "plan is NULL");
    if (capacity < p->blocks.size()) return fail(QSA_E_RANGE, "capacity smaller than the number of blocks");
    for (size_t i = 0; i < p->blocks.size(); ++i) {
        const PlanBlock& b = p->blocks[i];
        if (kinds) kinds[i] = b.init ? 4 : b.layer >= 0 ? 3 : b.prod ? 2 : b.diag ? 1 : 0;
        if (n_diag) n_diag[i] = b.layer >= 0 ? b.n_diag : 0;
    }
    return QSA_OK;
}

qsa_status qsa_plan_destroy(qsa_plan p) {
    if (!p) return fail(QSA_E_ARG, "plan is NULL");
    if (p->d_mat || p->d_layer) cudaDeviceSynchronize();
    if (p->d_mat) dev_free(p->d_mat);
    if (p->d_layer) dev_free(p->d_layer);
    delete p;
    return QSA_OK;
}

qsa_status qsa_plan_execute(qsa_state s, qsa_plan p, qsa_run_stats* stats) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (!p) return fail(QSA_E_ARG, "plan is NULL");
    if (p->n != s->n) return fail(QSA_E_ARG, "plan and state have different qubit counts");
    qsa_run_stats local{};
    qsa_run_stats* rs = stats ? stats : &local;
    *rs = qsa_run_stats{};
    if (p->blocks.empty()) return QSA_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (p->dev != dev) {
        // first execution on this device: upload the fused matrices and the
        // layer payloads once
        if (p->d_mat || p->d_layer) cudaStreamSynchronize(s->stream);
        if (p->d_mat) dev_free(p->d_mat);
        if (p->d_layer) dev_free(p->d_layer);
        p->d_mat = nullptr;
        p->d_layer = nullptr;
        const size_t bytes = p->host_mat.size() * sizeof(float);
        const size_t lbytes = p->host_layer.size();
        cudaError_t e = bytes ? dev_malloc(&p->d_mat, bytes) : cudaSuccess;
        if (e == cudaSuccess && lbytes) e = dev_malloc(&p->d_layer, lbytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (p->d_mat) dev_free(p->d_mat);
            p->d_mat = nullptr;
            p->d_layer = nullptr;
            return fail(QSA_E_NOMEM, "cudaMalloc of plan matrices failed");
        }
        if (bytes) {
            e = cudaMemcpyAsync(p->d_mat, p->host_mat.data(), bytes, cudaMemcpyHostToDevice, s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "plan matrix upload");
        }
        if (lbytes) {
            e = cudaMemcpyAsync(p->d_layer, p->host_layer.data(), lbytes, cudaMemcpyHostToDevice, s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "plan layer upload");
        }
        p->dev = dev;
        rs->h2d_bytes = static_cast<double>(bytes + lbytes);
    }
    const uint64_t l0 = s->launches;
    s->timing = p->opts.timing != 0;
    for (size_t i = 0; i < p->blocks.size(); ++i) {
        const PlanBlock& b = p->blocks[i];
        if (b.init && !s->known_zero) {
            st = fail(QSA_E_STATE, "a zero_init plan needs the state |0..0>");
        } else if (b.layer >= 0) {
            const PlanLayer& pl = p->layers[b.layer];
            if (s->n >= QSA_LAYER_TILE_BITS && std::equal(p->L0.begin(), p->L0.end(), s->L))
                st = run_layer_launches(s, pl.launches, p->d_layer, rs);
            else
                st = apply_layer_logical(s, pl.spec, rs);   // another layout: prepare again
        } else if (b.prod) {
            st = apply_prod_logical(s, b.t, b.k, p->d_mat + b.off, rs);
        } else if (b.diag) {
            st = apply_diag_logical(s, b.t, b.k, p->d_mat + b.off, rs);
        } else if (p->opts.lowering == QSA_LOWER_PERMUTE) {
            // promote the targets into the in-block frames, victims per the plan's rule
            int phys[QSA_MAX_K], pa[QSA_MAX_K], pb[QSA_MAX_K];
            for (int j = 0; j < b.k; ++j) phys[j] = s->L[b.t[j]];
            const int np = choose_promotions(s->L, s->n, phys, b.k, std::min(kInBlockBits, s->n), p->opts.victim,
                                             p->next_use.data() + i * s->n, pa, pb);
            st = np < 0 ? fail(QSA_E_ARG, "block wider than the in-block frames")
                        : permute_positions(s, pa, pb, np, rs);
            if (st == QSA_OK) st = apply_physical(s, phys, b.k, p->d_mat + b.off, p->opts.precision, rs);
        } else {
            st = apply_logical(s, b.t, b.k, p->d_mat + b.off, p->opts.lowering, p->opts.precision, rs);
        }
        if (st != QSA_OK) {
            s->timing = false;
            return st;
        }
    }
    s->timing = false;
    rs->launches = s->launches - l0;
    if (p->opts.timing) {
        collect_timers(s, &rs->seconds);
        return sync_and_check(s, "plan execution");
    }
    return QSA_OK;
}

qsa_status qsa_plan_execute_from_zero(qsa_state s, qsa_plan p, qsa_run_stats* stats) {
    if (!s) return fail(QSA_E_ARG, "state is NULL");
    if (!p) return fail(QSA_E_ARG, "plan is NULL");
    if (p->n != s->n) return fail(QSA_E_ARG, "plan and state have different qubit counts");
    if (!p->blocks.empty() && p->blocks[0].init && s->n >= QSA_LAYER_TILE_BITS && !s->failed) {
        // the preparation pass writes every amplitude: |0..0> in the plan's
        // layout needs no clearing first
        for (int q = 0; q < s->n; ++q) s->L[q] = p->L0[q];
        s->known_zero = true;
    } else {
        qsa_status st = qsa_state_reset(s);
        if (st != QSA_OK) return st;
        for (int q = 0; q < s->n; ++q) s->L[q] = p->L0[q];   // relabelling |0..0> is free
    }
    return qsa_plan_execute(s, p, stats);
}

qsa_status qsa_apply_circuit(qsa_state s, const qsa_op* ops, size_t n_ops, const qsa_plan_opts* opts,
                             qsa_run_stats* stats) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    qsa_plan p = nullptr;
    st = plan_create(ops, n_ops, s->n, opts, s->L, s->cm ? s->cm : costmodel_global(), &p);
    if (st != QSA_OK) return st;
    st = qsa_plan_execute(s, p, stats);
    if (p->d_mat || p->d_layer) {
        // free after the stream has consumed the matrices
        cudaStreamSynchronize(s->stream);
        if (p->d_mat) dev_free(p->d_mat);
        if (p->d_layer) dev_free(p->d_layer);
        p->d_mat = nullptr;
        p->d_layer = nullptr;
    }
    delete p;
    return st;
}

qsa_status qsa_state_counters(qsa_state s, uint64_t* launches) {
    if (!s || !launches) return fail(QSA_E_ARG, "NULL argument");
    *launches = s->launches;
    return QSA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched trajectories
// ---------------------------------------------------------------------------
struct qsa_batch_s {
    int n = 0, n_traj = 0;
    size_t total_ops = 0;
    std::vector<qsa::BatchBlock> blocks;
    std::vector<uint32_t> bstart;
    std::vector<int32_t> order;
    std::vector<float> mats;
    qsa::BatchBlock* d_blocks = nullptr;
    uint32_t* d_bstart = nullptr;
    int32_t* d_order = nullptr;
    float* d_mats = nullptr;
    unsigned* d_queue = nullptr;   // [0] work counter, [1] error word
    uint32_t* d_out = nullptr;     // keys, counts (n_traj * shots each), n_distinct (n_traj)
    size_t out_cap = 0;
    uint64_t shots = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    void* g_states = nullptr;
    uint64_t g_shots = 0, g_seed = 0, g_budget = 0;
    uint64_t launches = 0;
};

namespace {

void batch_free_device(qsa_batch b) {
    for (void* p : {static_cast<void*>(b->d_blocks), static_cast<void*>(b->d_bstart), static_cast<void*>(b->d_order),
                    static_cast<void*>(b->d_mats), static_cast<void*>(b->d_queue), static_cast<void*>(b->d_out)})
        if (p) dev_free(p);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
}

cudaError_t batch_enqueue(qsa_batch b, float2* states, uint64_t shots, uint64_t seed, uint64_t budget, cudaStream_t st) {
    uint32_t* keys = b->d_out;
    uint32_t* cnts = keys + static_cast<size_t>(b->n_traj) * shots;
    uint32_t* nd = cnts + static_cast<size_t>(b->n_traj) * shots;
    cudaError_t e = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    qsa::BatchArgs a{};
    a.states = states;
    a.n = b->n;
    a.n_traj = b->n_traj;
    a.blocks = b->d_blocks;
    a.bstart = b->d_bstart;
    a.order = b->d_order;
    a.mats = b->d_mats;
    a.queue = b->d_queue;
    a.err = reinterpret_cast<int*>(b->d_queue + 1);
    a.budget = budget;
    e = qsa::launch_batch_evolve(a, st, &b->launches);
    if (e != cudaSuccess) return e;
    return qsa::launch_batch_sample(states, b->n, b->n_traj, static_cast<uint32_t>(shots), seed, keys, cnts, nd, st,
                                    &b->launches);
}

}  // namespace

extern "C" {

qsa_status qsa_batch_create(int n_qubits, int n_traj, const qsa_op* ops, const size_t* op_offsets,
                            const qsa_plan_opts* opts, qsa_batch* out) {
    if (!out) return fail(QSA_E_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 22) return fail(QSA_E_ARG, "batched states need 1 <= N <= 22");
    if (n_traj < 1 || !op_offsets) return fail(QSA_E_ARG, "bad trajectory list");
    qsa_plan_opts o;
    qsa_status st = normalise_opts(opts, &o);
    if (st != QSA_OK) return st;
    if (o.kmax > 4) return fail(QSA_E_ARG, "batched trajectories fuse blocks of at most 4 qubits (kmax <= 4)");
    if (o.kmax_diag > o.kmax) return fail(QSA_E_ARG, "batched trajectories need kmax_diag <= kmax");
    if (o.layer) return fail(QSA_E_ARG, "batched trajectories take no layer units");
    if (o.zero_init) return fail(QSA_E_ARG, "batched trajectories take no zero_init prefix");
    if (o.kmax_prod >= 2) return fail(QSA_E_ARG, "batched trajectories do not use product blocks (kmax_prod <= 1)");
    if (op_offsets[0] != 0) return fail(QSA_E_ARG, "op_offsets[0] must be 0");
    for (int t = 0; t < n_traj; ++t)
        if (op_offsets[t + 1] < op_offsets[t]) return fail(QSA_E_ARG, "op_offsets must be non-decreasing");
    st = validate_ops(ops, op_offsets[n_traj], n_qubits);
    if (st != QSA_OK) return st;
    auto* b = new qsa_batch_s();
    b->n = n_qubits;
    b->n_traj = n_traj;
    b->total_ops = op_offsets[n_traj];
    b->bstart.push_back(0);
    std::vector<double> M;
    for (int t = 0; t < n_traj; ++t) {
        const qsa_op* tops = ops + op_offsets[t];
        const size_t cnt = op_offsets[t + 1] - op_offsets[t];
        std::vector<size_t> order;   // the identity: batches take no layer units
        auto units = plan(tops, cnt, n_qubits, o, nullptr, &order, costmodel_global());
        for (const Unit& u : units) {
            int32_t tg[QSA_MAX_K];
            int k = 0;
            const uint32_t off = static_cast<uint32_t>(b->mats.size());
            if (u.e - u.s == 1) {
                k = tops[u.s].k;
                for (int j = 0; j < k; ++j) tg[j] = tops[u.s].targets[j];
                b->mats.resize(off + (2u << (2 * k)));
                to_float_matrix(tops[u.s].matrix, k, b->mats.data() + off);
            } else {
                st = fuse_range(tops, u.s, u.e, tg, &k, &M);
                if (st != QSA_OK) {
                    delete b;
                    return st;
                }
                b->mats.resize(off + M.size());
                for (size_t j = 0; j < M.size(); ++j) b->mats[off + j] = static_cast<float>(M[j]);
            }
            while (b->mats.size() % 4) b->mats.push_back(0.f);
            qsa::BatchBlock bb;
            int phys[QSA_MAX_K];
            for (int j = 0; j < k; ++j) phys[j] = tg[j];
            if (!qsa::make_batch_block(n_qubits, phys, k, off, &bb)) {
                delete b;
                return fail(QSA_E_ARG, "could not tile a fused block");
            }
            b->blocks.push_back(bb);
        }
        b->bstart.push_back(static_cast<uint32_t>(b->blocks.size()));
    }
    // longest trajectories first, so the tail of the queue holds short work
    b->order.resize(n_traj);
    for (int t = 0; t < n_traj; ++t) b->order[t] = t;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return b->bstart[x + 1] - b->bstart[x] > b->bstart[y + 1] - b->bstart[y];
    });
    cudaError_t e = cudaSuccess;
    auto up = [&](void** dst, const void* src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = dev_malloc(dst, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(reinterpret_cast<void**>(&b->d_blocks), b->blocks.data(), b->blocks.size() * sizeof(qsa::BatchBlock));
    up(reinterpret_cast<void**>(&b->d_bstart), b->bstart.data(), b->bstart.size() * sizeof(uint32_t));
    up(reinterpret_cast<void**>(&b->d_order), b->order.data(), b->order.size() * sizeof(int32_t));
    up(reinterpret_cast<void**>(&b->d_mats), b->mats.data(), b->mats.size() * sizeof(float));
    if (e == cudaSuccess) e = dev_malloc(&b->d_queue, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free_device(b);
        delete b;
        return fail(QSA_E_NOMEM, std::string("batch setup: ") + cudaGetErrorString(e));
    }
    *out = b;
    return QSA_OK;
}

qsa_status qsa_batch_info(qsa_batch b, size_t* total_blocks, size_t* total_ops, uint64_t* launches) {
    if (!b) return fail(QSA_E_ARG, "batch is NULL");
    if (total_blocks) *total_blocks = b->blocks.size();
    if (total_ops) *total_ops = b->total_ops;
    if (launches) *launches = b->launches;
    return QSA_OK;
}

qsa_status qsa_batch_run(qsa_batch b, void* dev_states, size_t bytes, uint64_t shots, uint64_t seed,
                         uint64_t budget_cycles, int use_graph, void* cuda_stream, qsa_run_stats* stats) {
    if (!b || !dev_states) return fail(QSA_E_ARG, "NULL argument");
    if (bytes < (static_cast<size_t>(b->n_traj) * sizeof(float2) << b->n))
        return fail(QSA_E_ARG, "state buffer smaller than n_traj * 8 * 2^N bytes");
    if (reinterpret_cast<uintptr_t>(dev_states) % 16) return fail(QSA_E_ARG, "states must be 16-byte aligned");
    if (shots < 1 || shots > 16384) return fail(QSA_E_ARG, "batched sampling takes 1..16384 shots per trajectory");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t need = sizeof(uint32_t) * (2 * static_cast<size_t>(b->n_traj) * shots + b->n_traj);
    if (need > b->out_cap) {
        if (b->d_out) {
            cudaDeviceSynchronize();
            dev_free(b->d_out);
        }
        b->d_out = nullptr;
        b->out_cap = 0;
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            cudaGraphDestroy(b->graph);
            b->gexec = nullptr;
            b->graph = nullptr;
        }
        cudaError_t e = dev_malloc(&b->d_out, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(QSA_E_NOMEM, "cudaMalloc of batch outputs failed");
        }
        b->out_cap = need;
    }
    b->shots = shots;
    float2* states = static_cast<float2*>(dev_states);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaSuccess;
    if (use_graph) {
        const bool fresh = !b->gexec || b->g_states != dev_states || b->g_shots != shots || b->g_seed != seed ||
                           b->g_budget != budget_cycles;
        if (fresh) {
            if (b->gexec) {
                cudaGraphExecDestroy(b->gexec);
                cudaGraphDestroy(b->graph);
                b->gexec = nullptr;
                b->graph = nullptr;
            }
            // one direct run first: it sets the kernels' attributes outside the capture
            e = batch_enqueue(b, states, shots, seed, budget_cycles, b->cap_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap_stream);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t ee = batch_enqueue(b, states, shots, seed, budget_cycles, b->cap_stream);
                e = cudaStreamEndCapture(b->cap_stream, &b->graph);
                if (ee != cudaSuccess) e = ee;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return fail(QSA_E_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
            }
            b->g_states = dev_states;
            b->g_shots = shots;
            b->g_seed = seed;
            b->g_budget = budget_cycles;
        }
        cudaEventRecord(e0, st);
        e = cudaGraphLaunch(b->gexec, st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) b->launches += 2;
    } else {
        cudaEventRecord(e0, st);
        e = batch_enqueue(b, states, shots, seed, budget_cycles, st);
        cudaEventRecord(e1, st);
    }
    unsigned err_word = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err_word, b->d_queue + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
    if (stats) {
        *stats = qsa_run_stats{};
        stats->seconds = ms * 1e-3;
        stats->apply_seconds = ms * 1e-3;
        stats->blocks = b->blocks.size();
        stats->passes = b->blocks.size();
        stats->hbm_bytes = 16.0 * static_cast<double>(1ull << b->n) * static_cast<double>(b->blocks.size());
        stats->launches = use_graph ? 2 : 2;
    }
    if (err_word != 0)
        return fail(QSA_E_TIMEOUT, "batched trajectories: the cycle budget ran out (error word " +
                                       std::to_string(err_word) + "); the states and counts are incomplete");
    return QSA_OK;
}

qsa_status qsa_batch_counts(qsa_batch b, uint32_t* outcomes, uint32_t* counts, uint32_t* n_distinct) {
    if (!b || !b->d_out || !outcomes || !counts || !n_distinct) return fail(QSA_E_ARG, "NULL argument or no run yet");
    const size_t m = static_cast<size_t>(b->n_traj) * b->shots;
    cudaError_t e = cudaMemcpy(outcomes, b->d_out, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(counts, b->d_out + m, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(n_distinct, b->d_out + 2 * m, sizeof(uint32_t) * b->n_traj, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("batch counts: ") + cudaGetErrorString(e));
    return QSA_OK;
}

qsa_status qsa_batch_destroy(qsa_batch b) {
    if (!b) return fail(QSA_E_ARG, "batch is NULL");
    cudaDeviceSynchronize();
    batch_free_device(b);
    delete b;
    return QSA_OK;
}

}  // extern "C"
