// Host side of layer blocks (§IV-D structured fused blocks): tile geometry
// for a set of factor positions, classification of the diagonal ops relative
// to the tile (all-in / cross / out), the 2^12-entry table of the all-in ops
// (formed in FP64), the device payload of each pass, and qsa_apply_layer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "qsa.h"
#include "qsa_internal.h"
#include "qsa_runtime.h"

namespace qsa {

namespace {

constexpr int kTile = QSA_LAYER_TILE_BITS;
constexpr int kLow = QSA_LAYER_LOW_BITS;

// Largest m in [kLow, kTile] with m + #{pos >= m} <= kTile; the tile's extra
// bits are those positions.  For N >= 12 the chosen m gives exactly kTile
// tile bits.
bool layer_geom(const std::vector<int>& pos, LayerGeom* g) {
    for (int m = kTile; m >= kLow; --m) {
        std::vector<int> hi;
        for (int p : pos)
            if (p >= m) hi.push_back(p);
        if (m + static_cast<int>(hi.size()) <= kTile) {
            std::sort(hi.begin(), hi.end());
            g->m = m;
            g->nx = static_cast<int>(hi.size());
            for (int e = 0; e < kTile; ++e) g->xpos[e] = e < g->nx ? hi[e] : 0;
            return g->m + g->nx == kTile;
        }
    }
    return false;
}

int tile_bit(const LayerGeom& g, int p) {
    if (p < g.m) return p;
    for (int e = 0; e < g.nx; ++e)
        if (g.xpos[e] == p) return g.m + e;
    return -1;
}

void align16(std::vector<unsigned char>* b) {
    while (b->size() % 16) b->push_back(0);
}

template <typename T>
size_t append(std::vector<unsigned char>* b, const T* data, size_t count) {
    align16(b);
    const size_t off = b->size();
    b->resize(off + sizeof(T) * count);
    if (count) std::memcpy(b->data() + off, data, sizeof(T) * count);
    return off;
}

float2 f2(std::complex<double> z) { return make_float2(static_cast<float>(z.real()), static_cast<float>(z.imag())); }

float2 f2m(std::complex<double> z, double weight, ModulusCarry* carry) {
    return f2_modulus(z, std::norm(z), weight, carry);
}

// F = diag(p) [[c, -s], [s, c]] diag(q) with q[0] = 1, c = |F00|, s = |F01|;
// false unless the product reproduces F to 1e-10 (a unitary F does).
bool split_rotation(const std::array<std::complex<double>, 4>& F, double* c, double* s, std::complex<double>* p,
                    std::complex<double>* q) {
    const std::complex<double> a = F[0], b = F[1], cc = F[2], d = F[3];
    const double ca = std::abs(a), sb = std::abs(b);
    if (ca == 0.0 && sb == 0.0) return false;
    *c = ca;
    *s = sb;
    q[0] = 1.0;
    if (ca > 0.0 && sb > 0.0) {
        p[0] = a / ca;
        q[1] = -b / (p[0] * sb);
        p[1] = cc / sb;
    } else if (sb == 0.0) {
        p[0] = a / ca;
        q[1] = 1.0;
        p[1] = d / ca;
    } else {
        q[1] = 1.0;
        p[0] = -b / sb;
        p[1] = cc / sb;
    }
    const std::complex<double> rec[4] = {p[0] * ca * q[0], -p[0] * sb * q[1], p[1] * sb * q[0], p[1] * ca * q[1]};
    for (int i = 0; i < 4; ++i)
        if (std::abs(rec[i] - F[i]) > 1e-10) return false;
    return true;
}

// The rotation [[c, -s], [s, c]] runs in the cotangent form when s > c.
bool rotation_cotangent(double c, double s) { return s > c; }

// One pass: factors fsel (indices into spec.f), the diagonal ops if with_diag.
// Returns false when there is nothing to apply.
bool prepare_pass(int n, const int32_t* L, const LayerSpec& spec, const std::vector<int>& fsel, bool with_diag,
                  std::vector<unsigned char>* bytes, LayerLaunch* out, ModulusCarry* carry) {
    std::vector<int> pos;
    for (int j : fsel) pos.push_back(L[spec.t[j]]);
    LayerGeom g;
    if (!layer_geom(pos, &g)) return false;
    (void)n;
    LayerPayload p;
    std::vector<std::array<std::complex<double>, 4>> fac(kTile, {1.0, 0.0, 0.0, 1.0});
    for (size_t i = 0; i < fsel.size(); ++i) {
        const int b = tile_bit(g, pos[i]);
        fac[b] = spec.f[fsel[i]];
        p.active |= 1u << b;
    }
    // rotation mode when every factor splits as diag(p) R diag(q)
    std::vector<double> rc(kTile, 1.0), rs(kTile, 0.0);
    std::vector<std::array<std::complex<double>, 2>> rp(kTile, {1.0, 1.0}), rq(kTile, {1.0, 1.0});
    p.rotation = true;
    for (int b = 0; b < kTile && p.rotation; ++b)
        if ((p.active >> b) & 1u) p.rotation = split_rotation(fac[b], &rc[b], &rs[b], rp[b].data(), rq[b].data());
    // R = kappa M: tangent form (c >= s) M = [[1, -t], [t, 1]], kappa = c;
    // cotangent form M = [[u, -1], [1, u]], kappa = s, computed as (-row 0, row 1)
    // with the sign moved into p0; kappa joins the entry phases q.  The kernel
    // runs the cotangent form as the tangent form with t = -u, whose outputs
    // are row 1 and -row 0 in exchanged places: it leaves them there and the
    // pass reads its later tables and store offsets at the exchanged index
    // (rswap), so the rounds need no per-factor branches.
    std::vector<double> rcoef(kTile, 0.0);
    p.rswap = 0;
    if (p.rotation)
        for (int b = 0; b < kTile; ++b) {
            if (!((p.active >> b) & 1u)) continue;
            double kappa;
            if (rotation_cotangent(rc[b], rs[b])) {
                rcoef[b] = rc[b] / rs[b];
                kappa = rs[b];
                rp[b][0] = -rp[b][0];
                rcoef[b] = -rcoef[b];
                p.rswap |= 1u << b;
            } else {
                rcoef[b] = rs[b] / rc[b];
                kappa = rc[b];
            }
            rq[b][0] *= kappa;
            rq[b][1] *= kappa;
        }
    std::vector<LayerGate> cross, outg;
    uint32_t cross_bits = 0;
    std::vector<std::complex<double>> din;
    if (with_diag) {
        for (const LayerDiagOp& op : spec.diag) {
            const int p0 = L[op.q[0]], b0 = tile_bit(g, p0);
            const int p1 = op.k == 2 ? L[op.q[1]] : -1, b1 = op.k == 2 ? tile_bit(g, p1) : -1;
            if (b0 >= 0 && (op.k == 1 || b1 >= 0)) {
                if (din.empty()) din.assign(1u << kTile, 1.0);
                for (uint32_t j = 0; j < (1u << kTile); ++j) {
                    int c = static_cast<int>((j >> b0) & 1u);
                    if (op.k == 2) c |= static_cast<int>((j >> b1) & 1u) << 1;
                    din[j] *= op.d[c];
                }
            } else if (op.k == 2 && (b0 >= 0) != (b1 >= 0)) {
                // one qubit in the tile (v), one outside (o): d[2 o + v]
                LayerGate G{};
                const bool first_in = b0 >= 0;
                G.a = first_in ? b0 : b1;
                G.b = first_in ? p1 : p0;
                for (int o = 0; o < 2; ++o)
                    for (int v = 0; v < 2; ++v)
                        G.d[2 * o + v] = f2m(op.d[first_in ? (v | (o << 1)) : (o | (v << 1))], 0.25, carry);
                cross.push_back(G);
                cross_bits |= 1u << G.a;
            } else {
                LayerGate G{};
                G.a = p0;
                G.b = p1;
                for (int c = 0; c < (1 << op.k); ++c) G.d[c] = f2m(op.d[c], 1.0 / (1 << op.k), carry);
                outg.push_back(G);
            }
        }
    }
    p.pmask = p.rotation ? (cross_bits | p.active) : (cross_bits & ~p.active);
    if (p.active == 0 && p.pmask == 0 && outg.empty() && din.empty()) return false;
    // rotation mode: each bit's q phases; per round, the product of its bits' p phases
    std::vector<float2> qph(2 * kTile, make_float2(1.f, 0.f)), rpt(48, make_float2(1.f, 0.f));
    // with no per-tile phases the pass multiplies by per-round products of the q phases,
    // the same for every tile: formed here in FP64 and rounded as the pass's constants
    const bool static_tables = p.rotation && cross.empty() && outg.empty();
    std::vector<float2> sph(48, make_float2(1.f, 0.f));
    p.rpmask = 0;
    if (p.rotation) {
        for (int b = 0; b < kTile; ++b)
            if ((p.active >> b) & 1u) {
                // the pass scales by |q|^2 (1 + t^2) with t as rounded: aim q's
                // modulus at the exact rotation's |q|^2 (1 + t^2) over (1 + t_f^2)
                const double tf = static_cast<float>(rcoef[b]);
                const double scale = (1.0 + rcoef[b] * rcoef[b]) / (1.0 + tf * tf);
                qph[2 * b] = f2_modulus(rq[b][0], std::norm(rq[b][0]) * scale, 0.5, static_tables ? nullptr : carry);
                qph[2 * b + 1] =
                    f2_modulus(rq[b][1], std::norm(rq[b][1]) * scale, 0.5, static_tables ? nullptr : carry);
            }
        for (int r = 0; r < 3; ++r)
            for (int i = 0; i < 16; ++i) {
                // the amplitude in place i of the round has the local index i ^ (exchanged bits)
                const int li = i ^ static_cast<int>((p.rswap >> (4 * r)) & 15u);
                std::complex<double> z = 1.0;
                for (int lb = 0; lb < 4; ++lb)
                    if ((p.active >> (4 * r + lb)) & 1u) z *= rp[4 * r + lb][(li >> lb) & 1];
                rpt[16 * r + i] = f2m(z, 1.0 / 16, carry);
                if (std::abs(z - 1.0) > 1e-15) p.rpmask |= 1u << r;
            }
        if (static_tables)
            for (int r = 0; r < 3; ++r)
                for (int i = 0; i < 16; ++i) {
                    std::complex<double> z = 1.0;
                    double m2 = 1.0;
                    for (int lb = 0; lb < 4; ++lb) {
                        const int b = 4 * r + lb, v = (i >> lb) & 1;
                        if (!((p.pmask >> b) & 1u)) continue;
                        const double tf = static_cast<float>(rcoef[b]);
                        z *= rq[b][v];
                        m2 *= std::norm(rq[b][v]) * (1.0 + rcoef[b] * rcoef[b]) / (1.0 + tf * tf);
                    }
                    sph[16 * r + i] = f2_modulus(z, m2, 1.0 / 16, carry);
                }
    }
    std::stable_sort(cross.begin(), cross.end(), [](const LayerGate& x, const LayerGate& y) { return x.a < y.a; });
    p.ncross = static_cast<int>(cross.size());
    p.nout = static_cast<int>(outg.size());
    for (int b = 0, c = 0; b <= kTile; ++b) {
        while (c < p.ncross && cross[c].a < b) ++c;
        p.cstart[b] = c;
    }
    align16(bytes);
    const size_t base = bytes->size();
    std::vector<float2> facf(4 * kTile);
    for (int b = 0; b < kTile; ++b) {
        if (p.rotation)
            facf[b] = make_float2(static_cast<float>(rcoef[b]), 0.f);
        else
            for (int c = 0; c < 4; ++c) facf[4 * b + c] = f2(fac[b][c]);
    }
    if (p.rotation) {
        for (int b = 0; b < kTile; ++b) p.rot[b] = facf[b].x;
        for (int i = 0; i < 48; ++i) {
            p.rp[2 * i] = rpt[i].x;
            p.rp[2 * i + 1] = rpt[i].y;
        }
    }
    p.off_fac = append(bytes, facf.data(), facf.size()) - base;
    p.off_qph = append(bytes, qph.data(), qph.size()) - base;
    p.off_rp = append(bytes, rpt.data(), rpt.size()) - base;
    p.off_sph = append(bytes, sph.data(), sph.size()) - base;
    p.off_cross = append(bytes, cross.data(), cross.size()) - base;
    p.off_out = append(bytes, outg.data(), outg.size()) - base;
    if (!din.empty()) {
        std::vector<float2> df(din.size());
        for (size_t j = 0; j < din.size(); ++j) df[j] = f2m(din[j], 1.0 / (1u << kTile), carry);
        p.off_din = append(bytes, df.data(), df.size()) - base;
        p.has_din = true;
    }
    align16(bytes);
    p.bytes = bytes->size() - base;
    out->g = g;
    out->p = p;
    out->dev_off = base;
    return true;
}

}  // namespace

// Modulus-faithful rounding of the FP32 constants of a plan.  A constant (a
// gate phase, a phase-table entry, an entry phase) multiplies a large share
// of the state, so the modulus error of its rounding changes the norm
// systematically, and circuits that repeat an angle (a QAOA round applies the
// same ZZ phase to every edge) add those errors coherently.  The candidates
// are the nine FP32 numbers one ulp or less from the rounded real and
// imaginary parts (the direction moves by at most about an ulp: a phase
// error, second order in the fidelity).  With a carry the choice is error
// feedback: the candidate whose weighted modulus error brings the carry
// nearest zero, so repeated constants alternate between values just above
// and just below the exact modulus and their errors cancel instead of adding
// up (weight = the share of the state's indices the constant multiplies).
// Without a carry: the smallest modulus error.  Ties go to the smaller error,
// then to the candidate nearer z.
namespace {
// The FP32 neighbour of a finite float toward -inf (up = false) or +inf: the
// same value as std::nextafter, by stepping the bit pattern.
inline float step_float(float x, bool up) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7fffffffu) == 0)
        u = up ? 0x00000001u : 0x80000001u;
    else if ((u >> 31) == (up ? 1u : 0u))
        --u;
    else
        ++u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}
}  // namespace

float2 f2_modulus(std::complex<double> z, double m2, double weight, ModulusCarry* carry) {
    const float r0 = static_cast<float>(z.real()), i0 = static_cast<float>(z.imag());
    const float rs[3] = {step_float(r0, false), r0, step_float(r0, true)};
    const float is[3] = {step_float(i0, false), i0, step_float(i0, true)};
    const double acc = carry ? carry->acc : 0.0;
    const double zr = z.real(), zi = z.imag();
    double rr[3], ii[3];
    for (int a = 0; a < 3; ++a) {
        rr[a] = static_cast<double>(rs[a]) * rs[a];
        ii[a] = static_cast<double>(is[a]) * is[a];
    }
    auto dist = [&](int a, int b) {
        return (rs[a] - zr) * (rs[a] - zr) + (is[b] - zi) * (is[b] - zi);
    };
    int br = 0, bi = 0;
    double bk = 0.0, be = 0.0;
    bool first = true;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double e = rr[a] + ii[b] - m2;
            const double key = std::fabs(acc + weight * e);
            bool take = first || key < bk;
            if (!take && key == bk) {
                const double ae = std::fabs(e), abe = std::fabs(be);
                take = ae < abe || (ae == abe && dist(a, b) < dist(br, bi));
            }
            if (take) {
                first = false;
                bk = key;
                be = e;
                br = a;
                bi = b;
            }
        }
    if (carry) carry->acc += weight * be;
    return make_float2(rs[br], is[bi]);
}

void to_float_moduli(const double* z, size_t count, float* out, double weight, ModulusCarry* carry) {
    for (size_t i = 0; i < count; ++i) {
        const std::complex<double> v(z[2 * i], z[2 * i + 1]);
        const float2 f = f2_modulus(v, std::norm(v), weight, carry);
        out[2 * i] = f.x;
        out[2 * i + 1] = f.y;
    }
}

void layer_move_exit_phases(LayerSpec* from, LayerSpec* to) {
    std::vector<LayerDiagOp> moved;
    for (size_t j = 0; j < from->f.size(); ++j) {
        double c, s;
        std::complex<double> p[2], q[2];
        if (!split_rotation(from->f[j], &c, &s, p, q)) continue;
        // the cotangent form's pass negates p0: hand over -p0 so that it meets 1 there
        if (rotation_cotangent(c, s)) p[0] = -p[0];
        if (std::abs(std::abs(p[0]) - 1.0) > 1e-12 || std::abs(std::abs(p[1]) - 1.0) > 1e-12) continue;
        if (std::abs(p[0] - 1.0) < 1e-15 && std::abs(p[1] - 1.0) < 1e-15) continue;
        auto& F = from->f[j];
        F = {std::conj(p[0]) * F[0], std::conj(p[0]) * F[1], std::conj(p[1]) * F[2], std::conj(p[1]) * F[3]};
        LayerDiagOp d;
        d.k = 1;
        d.q[0] = from->t[j];
        d.d[0] = p[0];
        d.d[1] = p[1];
        moved.push_back(d);
    }
    to->diag.insert(to->diag.begin(), moved.begin(), moved.end());
}

bool layer_fits(int n, const int* pos, int k) {
    const int T = std::min(kTile, n);
    const int low = std::min(kLow, T);
    int hi = 0;
    for (int j = 0; j < k; ++j) hi += pos[j] >= low ? 1 : 0;
    return hi <= T - low;
}

std::vector<LayerLaunch> prepare_layer(int n, const int32_t* L, const LayerSpec& spec,
                                       std::vector<unsigned char>* bytes, ModulusCarry* carry) {
    std::vector<LayerLaunch> out;
    if (n < kTile) return out;
    // factor groups that fit a tile, in target order
    std::vector<std::vector<int>> groups(1);
    int hi = 0;
    for (size_t j = 0; j < spec.t.size(); ++j) {
        const bool high = L[spec.t[j]] >= kLow;
        if (high && hi == kTile - kLow) {
            groups.emplace_back();
            hi = 0;
        }
        groups.back().push_back(static_cast<int>(j));
        hi += high ? 1 : 0;
    }
    for (size_t i = 0; i < groups.size(); ++i) {
        LayerLaunch ll;
        if (prepare_pass(n, L, spec, groups[i], i == 0, bytes, &ll, carry)) {
            // only the first pass generates; later ones read what it wrote
            ll.p.generate = spec.generate && out.empty();
            out.push_back(ll);
        }
    }
    return out;
}

qsa_status run_layer_launches(qsa_state s, const std::vector<LayerLaunch>& ls, const unsigned char* d_base,
                              qsa_run_stats* rs) {
    for (const LayerLaunch& ll : ls) {
        if (ll.p.rotation && (ll.p.ncross > 0 || ll.p.nout > 0)) {
            qsa_status st = ensure_dev(s, &s->d_lrec, &s->lrec_cap, layer_record_bytes(s->n));
            if (st != QSA_OK) return st;
        }
        // the per-tile records first (outside the layer kernel's timer)
        cudaError_t e = launch_layer_records(s->psi, s->n, ll.g, d_base + ll.dev_off, ll.p, s->d_lrec, s->stream,
                                             &s->launches);
        if (e != cudaSuccess) return cuda_fail(s, e, "layer records kernel");
        {
            Timer tm(s, rs ? &rs->layer_seconds : nullptr);
            e = launch_apply_layer(s->psi, s->n, ll.g, d_base + ll.dev_off, ll.p, s->d_lrec, s->stream,
                                   &s->launches);
            tm.stop();
        }
        if (e != cudaSuccess) return cuda_fail(s, e, "layer kernel");
        s->known_zero = false;
        if (rs) {
            rs->passes += 1;
            rs->hbm_bytes += (ll.p.generate ? 8.0 : 16.0) * static_cast<double>(1ull << s->n);
        }
    }
    if (rs) {
        rs->blocks += 1;
        rs->layer_blocks += 1;
    }
    return QSA_OK;
}

qsa_status apply_layer_logical(qsa_state s, const LayerSpec& spec, qsa_run_stats* rs) {
    if (s->n >= kTile) {
        std::vector<unsigned char> bytes;
        const auto ls = prepare_layer(s->n, s->L, spec, &bytes);
        if (ls.empty()) return QSA_OK;
        qsa_status st = ensure_dev(s, reinterpret_cast<void**>(&s->d_mat), &s->mat_cap, bytes.size());
        if (st != QSA_OK) return st;
        // pageable source: the copy is staged before the call returns
        cudaError_t e = cudaMemcpyAsync(s->d_mat, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "layer payload upload");
        return run_layer_launches(s, ls, reinterpret_cast<const unsigned char*>(s->d_mat), rs);
    }
    // small states: the ops one by one on the diagonal and product kernels
    std::vector<float> tab;
    std::vector<size_t> off;
    for (const LayerDiagOp& op : spec.diag) {
        off.push_back(tab.size());
        for (int c = 0; c < (1 << op.k); ++c) {
            tab.push_back(static_cast<float>(op.d[c].real()));
            tab.push_back(static_cast<float>(op.d[c].imag()));
        }
        while (tab.size() % 4) tab.push_back(0.f);
    }
    const size_t foff = tab.size();
    for (const auto& f : spec.f)
        for (int c = 0; c < 4; ++c) {
            tab.push_back(static_cast<float>(f[c].real()));
            tab.push_back(static_cast<float>(f[c].imag()));
        }
    if (spec.generate) {
        cudaError_t e = launch_fill_one(s->psi, s->n, s->stream, &s->launches);
        if (e != cudaSuccess) return cuda_fail(s, e, "fill kernel");
        s->known_zero = false;
    }
    if (tab.empty()) return QSA_OK;
    qsa_status st = ensure_dev(s, reinterpret_cast<void**>(&s->d_mat), &s->mat_cap, tab.size() * sizeof(float));
    if (st != QSA_OK) return st;
    cudaError_t e = cudaMemcpyAsync(s->d_mat, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice,
                                    s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "layer table upload");
    for (size_t i = 0; i < spec.diag.size(); ++i) {
        st = apply_diag_logical(s, spec.diag[i].q, spec.diag[i].k, s->d_mat + off[i], rs);
        if (st != QSA_OK) return st;
    }
    if (!spec.t.empty()) return apply_prod_logical(s, spec.t.data(), static_cast<int>(spec.t.size()), s->d_mat + foff, rs);
    return QSA_OK;
}

qsa_status layer_diag_from_op(const qsa_op& op, LayerDiagOp* out) {
    if (op.k < 1 || op.k > 2) return fail(QSA_E_ARG, "layer diagonal ops act on 1 or 2 qubits");
    if (!op.matrix) return fail(QSA_E_ARG, "op matrix is NULL");
    const int D = 1 << op.k;
    out->k = op.k;
    for (int j = 0; j < op.k; ++j) out->q[j] = op.targets[j];
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            const double re = op.matrix[2 * (r * D + c)], im = op.matrix[2 * (r * D + c) + 1];
            if (r == c)
                out->d[r] = std::complex<double>(re, im);
            else if (re != 0.0 || im != 0.0)
                return fail(QSA_E_ARG, "layer diagonal op has a nonzero off-diagonal entry");
        }
    return QSA_OK;
}

}  // namespace qsa

using namespace qsa;

extern "C" {

qsa_status qsa_apply_layer(qsa_state s, const qsa_op* diag_ops, size_t n_diag, const int32_t* targets, int k,
                           const double* factors) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (k < 0 || k > QSA_MAX_LAYER) return fail(QSA_E_ARG, "k must be in 0..12");
    if (k > 0) {
        st = validate_targets(s->n, targets, k, QSA_MAX_LAYER);
        if (st != QSA_OK) return st;
        if (!factors) return fail(QSA_E_ARG, "factors is NULL");
    }
    if (n_diag > 0 && !diag_ops) return fail(QSA_E_ARG, "diag_ops is NULL");
    LayerSpec spec;
    for (size_t i = 0; i < n_diag; ++i) {
        st = validate_targets(s->n, diag_ops[i].targets, diag_ops[i].k, 2);
        if (st != QSA_OK) return st;
        LayerDiagOp d;
        st = layer_diag_from_op(diag_ops[i], &d);
        if (st != QSA_OK) return st;
        spec.diag.push_back(d);
    }
    for (int j = 0; j < k; ++j) {
        spec.t.push_back(targets[j]);
        std::array<std::complex<double>, 4> f;
        for (int c = 0; c < 4; ++c) f[c] = std::complex<double>(factors[8 * j + 2 * c], factors[8 * j + 2 * c + 1]);
        spec.f.push_back(f);
    }
    return apply_layer_logical(s, spec, nullptr);
}

}  // extern "C"
