// planner.cpp -- host planning for the slab-blocked simulator.
//
// 1. canonicalize(): API gates -> canonical gates with FP64 matrices (host libm only; the
//    device never evaluates transcendental functions).
// 2. Fusion (arXiv 2406.14084, Alg. 2 level 3 and the diagonal fusion of the artifact
//    appendix): a greedy scan merges later gates into the current one when they commute with
//    every gate skipped over and the merged gate stays within a width limit.  Diagonal gates
//    merge into diagonal tables (D<k> gates); dense merges form k-qubit unitaries whose FP64
//    product is U = G_m ... G_1, accepted when the analytic cost model says the merged op is
//    cheaper than the parts.
// 3. Gate-block finding (Eq. 5-7, Alg. 1 findGBs): repeatedly build one slab pass.  Starting
//    from the always-resident low segment bits, scan the remaining ops in order and take every
//    op whose predecessors are done and whose non-diagonal qubits fit the slab (adding their
//    physical positions while there is room); ops that do not fit block their qubits for the
//    rest of the scan.  Diagonal roles (controls, diagonal gates) never need slab residence:
//    outside the slab their bits are constant per CTA.  Uncontrolled SWAP gates only relabel
//    qubits (Sec. II-B) and cost nothing.  In the paper's low-block mode the slab is fixed to
//    the b lowest physical bits and remap passes (Alg. 4) bring needed qubits into it.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>

namespace qs {

namespace {

const double kPi = 3.14159265358979323846;

int popcount(uint64_t x) { return __builtin_popcountll(x); }

// ------------------------------------------------------------------ gate matrices

bool named_matrix(const qs_gate &g, std::vector<cd> &m, bool &diag)
{
    const double th = g.p[0], ph = g.p[1], la = g.p[2];
    const double c = std::cos(th / 2), s = std::sin(th / 2);
    const cd I(0, 1);
    diag = false;
    switch (g.kind) {
    case QS_H: {
        const double r = 1.0 / std::sqrt(2.0);
        m = {r, r, r, -r};
        return true;
    }
    case QS_Y: m = {0.0, -I, I, 0.0}; return true;
    case QS_RX: m = {c, -I * s, -I * s, c}; return true;
    case QS_RY: m = {c, -s, s, c}; return true;
    case QS_U3:
        m = {c, -std::exp(I * la) * s, std::exp(I * ph) * s, std::exp(I * (ph + la)) * c};
        return true;
    case QS_Z: diag = true; m = {1.0, -1.0}; return true;
    case QS_S: diag = true; m = {1.0, I}; return true;
    case QS_SDG: diag = true; m = {1.0, -I}; return true;
    case QS_T: diag = true; m = {1.0, std::exp(I * (kPi / 4))}; return true;
    case QS_TDG: diag = true; m = {1.0, std::exp(-I * (kPi / 4))}; return true;
    case QS_RZ: diag = true; m = {std::exp(-I * (th / 2)), std::exp(I * (th / 2))}; return true;
    case QS_P: diag = true; m = {1.0, std::exp(I * th)}; return true;
    case QS_CZ: diag = true; m = {1.0, 1.0, 1.0, -1.0}; return true;
    case QS_CP: diag = true; m = {1.0, 1.0, 1.0, std::exp(I * th)}; return true;
    case QS_RZZ: {
        diag = true;
        const cd e0 = std::exp(-I * (th / 2)), e1 = std::exp(I * (th / 2));
        m = {e0, e1, e1, e0};
        return true;
    }
    default: return false;
    }
}

int expected_nt(int kind)
{
    switch (kind) {
    case QS_CZ: case QS_CP: case QS_SWAP: case QS_RZZ: return 2;
    case QS_UNITARY: case QS_DIAG: return -1;
    default: return 1;
    }
}

char role_of(const CGate &g, int q)
{
    // 'N' = non-diagonal action on q; 'D' = diagonal action (controls, diagonal gates)
    if (g.cls == C_DIAG) return 'D';
    for (int t : g.tq)
        if (t == q) return 'N';
    return 'D';
}

std::vector<int> all_qubits(const CGate &g)
{
    std::vector<int> v = g.tq;
    v.insert(v.end(), g.cq.begin(), g.cq.end());
    return v;
}

// Dense matrix of g on the ordered qubit list Q (local bit j <-> Q[j]); Q must cover g.
std::vector<cd> embed(const CGate &g, const std::vector<int> &Q)
{
    const int kq = (int)Q.size();
    const size_t D = size_t(1) << kq;
    std::vector<cd> M(D * D, 0.0);
    auto pos = [&](int q) {
        for (int j = 0; j < kq; ++j)
            if (Q[j] == q) return j;
        return -1;
    };
    uint64_t cmask = 0;
    for (int c : g.cq) cmask |= 1ull << pos(c);
    std::vector<int> tp;
    for (int t : g.tq) tp.push_back(pos(t));
    const int kt = (int)tp.size();
    for (size_t col = 0; col < D; ++col) {
        if ((col & cmask) != cmask) {
            M[col * D + col] = 1.0;
            continue;
        }
        uint64_t l = 0;
        for (int j = 0; j < kt; ++j) l |= ((col >> tp[j]) & 1ull) << j;
        uint64_t clear = col;
        for (int j = 0; j < kt; ++j) clear &= ~(1ull << tp[j]);
        switch (g.cls) {
        case C_DENSE: {
            const size_t Dt = size_t(1) << kt;
            for (size_t r = 0; r < Dt; ++r) {
                uint64_t row = clear;
                for (int j = 0; j < kt; ++j) row |= ((r >> j) & 1ull) << tp[j];
                M[row * D + col] = g.m[r * Dt + l];
            }
            break;
        }
        case C_DIAG: M[col * D + col] = g.m[l]; break;
        case C_PERMX: M[(col ^ (1ull << tp[0])) * D + col] = 1.0; break;
        case C_SWAP: {
            const uint64_t b0 = (col >> tp[0]) & 1, b1 = (col >> tp[1]) & 1;
            const uint64_t row = (clear) | (b1 << tp[0]) | (b0 << tp[1]);
            M[row * D + col] = 1.0;
            break;
        }
        }
    }
    return M;
}

// Diagonal entries of a diagonal gate (controls folded in) on the ordered list Q.
std::vector<cd> embed_diag(const CGate &g, const std::vector<int> &Q)
{
    const int kq = (int)Q.size();
    const size_t D = size_t(1) << kq;
    std::vector<cd> d(D, 1.0);
    auto pos = [&](int q) {
        for (int j = 0; j < kq; ++j)
            if (Q[j] == q) return j;
        return -1;
    };
    uint64_t cmask = 0;
    for (int c : g.cq) cmask |= 1ull << pos(c);
    std::vector<int> tp;
    for (int t : g.tq) tp.push_back(pos(t));
    for (size_t x = 0; x < D; ++x) {
        if ((x & cmask) != cmask) continue;
        uint64_t l = 0;
        for (size_t j = 0; j < tp.size(); ++j) l |= ((x >> tp[j]) & 1ull) << j;
        d[x] = g.m[l];
    }
    return d;
}

std::vector<cd> matmul(const std::vector<cd> &A, const std::vector<cd> &B, size_t D)
{
    std::vector<cd> C(D * D, 0.0);
    for (size_t i = 0; i < D; ++i)
        for (size_t k = 0; k < D; ++k) {
            const cd a = A[i * D + k];
            if (a == cd(0.0)) continue;
            for (size_t j = 0; j < D; ++j) C[i * D + j] += a * B[k * D + j];
        }
    return C;
}

std::vector<int> union_qubits(const CGate &a, const CGate &b)
{
    std::vector<int> u = all_qubits(a);
    for (int q : all_qubits(b))
        if (std::find(u.begin(), u.end(), q) == u.end()) u.push_back(q);
    return u;
}

}  // namespace

// ------------------------------------------------------------------ canonicalisation

int canonicalize(const qs_gate *g, size_t ng, int n, std::vector<CGate> &out, std::string &err)
{
    out.clear();
    out.reserve(ng);
    for (size_t i = 0; i < ng; ++i) {
        const qs_gate &x = g[i];
        char buf[160];
        if (x.kind < 0 || x.kind >= QS_NUM_KINDS) {
            snprintf(buf, sizeof buf, "gate %zu: unknown kind %d", i, x.kind);
            err = buf;
            return QS_EINVAL;
        }
        if (x.nt < 1 || x.nt > QS_MAX_TARGETS || x.nc < 0 || x.nc > QS_MAX_CONTROLS) {
            snprintf(buf, sizeof buf, "gate %zu: bad target/control count", i);
            err = buf;
            return QS_EINVAL;
        }
        const int ent = expected_nt(x.kind);
        if (ent > 0 && x.nt != ent) {
            snprintf(buf, sizeof buf, "gate %zu: kind %d needs %d targets", i, x.kind, ent);
            err = buf;
            return QS_EINVAL;
        }
        if (x.kind == QS_CX && x.nc < 1) {
            snprintf(buf, sizeof buf, "gate %zu: CX needs a control", i);
            err = buf;
            return QS_EINVAL;
        }
        uint64_t seen = 0;
        bool bad = false;
        for (int j = 0; j < x.nt + x.nc; ++j) {
            const int q = j < x.nt ? x.t[j] : x.c[j - x.nt];
            if (q < 0 || q >= n || (seen >> q & 1)) bad = true;
            else seen |= 1ull << q;
        }
        if (bad) {
            snprintf(buf, sizeof buf, "gate %zu: qubit out of range or repeated", i);
            err = buf;
            return QS_EINVAL;
        }
        CGate c;
        c.tq.assign(x.t, x.t + x.nt);
        c.cq.assign(x.c, x.c + x.nc);
        const size_t D = size_t(1) << x.nt;
        bool diag = false;
        if (x.kind == QS_X || x.kind == QS_CX) {
            c.cls = C_PERMX;
        } else if (x.kind == QS_SWAP) {
            c.cls = C_SWAP;
        } else if (x.kind == QS_UNITARY || x.kind == QS_DIAG) {
            if (!x.m) {
                snprintf(buf, sizeof buf, "gate %zu: matrix pointer is NULL", i);
                err = buf;
                return QS_EINVAL;
            }
            if (x.kind == QS_DIAG) {
                c.cls = C_DIAG;
                c.m.resize(D);
                for (size_t e = 0; e < D; ++e) c.m[e] = cd(x.m[2 * e], x.m[2 * e + 1]);
            } else {
                std::vector<cd> m(D * D);
                for (size_t e = 0; e < D * D; ++e) m[e] = cd(x.m[2 * e], x.m[2 * e + 1]);
                bool isdiag = true;
                for (size_t r = 0; r < D && isdiag; ++r)
                    for (size_t col = 0; col < D; ++col)
                        if (r != col && m[r * D + col] != cd(0.0)) { isdiag = false; break; }
                if (isdiag) {
                    c.cls = C_DIAG;
                    c.m.resize(D);
                    for (size_t e = 0; e < D; ++e) c.m[e] = m[e * D + e];
                } else {
                    c.cls = C_DENSE;
                    c.m = std::move(m);
                }
            }
        } else {
            if (!named_matrix(x, c.m, diag)) {
                err = "internal: no matrix for gate kind";
                return QS_EINVAL;
            }
            c.cls = diag ? C_DIAG : C_DENSE;
        }
        for (const cd &v : c.m)
            if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) {
                snprintf(buf, sizeof buf, "gate %zu: non-finite matrix entry", i);
                err = buf;
                return QS_EINVAL;
            }
        out.push_back(std::move(c));
    }
    return QS_OK;
}

// ------------------------------------------------------------------ cost model

double op_cost(const CGate &g, qs_dtype dt)
{
    // Units: FP32 FMA issue slots per amplitude of the slab kernel.  FP64 arithmetic is
    // weighted by the measured FP32/FP64 FMA rate ratio of GB300 (~62).  Ops that run inside a
    // register stage cost their arithmetic plus a small per-op overhead; ops that must run on the
    // shared-memory slab (dense on 3+ qubits, diagonal tables wider than 7 qubits) also pay a
    // shared-memory round trip of the whole slab (16 slots for complex64, 32 for complex128).
    const double w = dt == QS_C64 ? 1.0 : 62.0;
    const double smem = dt == QS_C64 ? 16.0 : 32.0;
    const int k = (int)g.tq.size();
    const int nc = (int)g.cq.size();
    const double frac = std::ldexp(1.0, -nc);
    switch (g.cls) {
    case C_DENSE: {
        if (k == 1) {
            // a real 2x2 matrix acts on real and imaginary parts separately: half the FMAs
            bool real = true;
            for (const cd &x : g.m) real = real && x.imag() == 0.0;
            return frac * w * (real ? 4.0 : 8.0) + 1.0;
        }
        if (k <= 2) return frac * w * 4.0 * std::ldexp(1.0, k) + 1.0;
        return frac * w * 4.0 * std::ldexp(1.0, k) + smem + 2.0;
    }
    case C_DIAG: {
        bool cphase = true;
        for (size_t i = 0; i + 1 < g.m.size(); ++i)
            if (g.m[i] != cd(1.0)) cphase = false;
        const int m = k + nc;
        if (cphase) {
            const cd p = g.m.back();
            const double flops = (p == cd(-1.0)) ? 0.5 : w * 4.0;  // sign flip vs complex multiply
            return std::ldexp(1.0, -m) * flops + 1.0;
        }
        // A table over several qubits costs one multiply per amplitude.  Merging phases of
        // distinct qubits into one table is left to the register stages, which combine every
        // register-bit diagonal of a stage into one table at no cost in passes; the extra unit
        // here keeps the fusion pass from building such tables early.
        if (m <= 7) return w * 4.0 + 3.0;
        return w * 4.0 + 3.0 * m + smem + 2.0;
    }
    case C_PERMX: return frac * 1.0 + 1.0;
    case C_SWAP: return frac * 1.0 + 1.0;
    }
    return 0.0;
}

int default_slab_bits(qs_dtype dt) { return dt == QS_C64 ? 13 : 12; }
int default_seg_bits(qs_dtype dt) { return dt == QS_C64 ? 4 : 3; }

// ------------------------------------------------------------------ fusion

namespace {

bool hoistable(const CGate &g, const std::map<int, char> &skipped)
{
    for (int q : all_qubits(g)) {
        auto it = skipped.find(q);
        if (it == skipped.end()) continue;
        if (it->second == 'N' || role_of(g, q) == 'N') return false;
    }
    return true;
}

void note_skipped(const CGate &g, std::map<int, char> &skipped)
{
    for (int q : all_qubits(g)) {
        const char r = role_of(g, q);
        auto it = skipped.find(q);
        if (it == skipped.end()) skipped[q] = r;
        else if (r == 'N') it->second = 'N';
    }
}

// Merge g (applied after cur) into cur if allowed.  Returns true on success.
bool try_merge(CGate &cur, const CGate &g, int kdiag, int kdense, bool force_dense, qs_dtype dt)
{
    std::vector<int> U = union_qubits(cur, g);
    if (cur.cls == C_DIAG && g.cls == C_DIAG) {
        if ((int)U.size() > kdiag) return false;
        std::vector<cd> a = embed_diag(cur, U), b = embed_diag(g, U);
        for (size_t i = 0; i < a.size(); ++i) a[i] *= b[i];
        CGate m;
        m.cls = C_DIAG;
        m.tq = U;
        m.m = std::move(a);
        m.nsrc = cur.nsrc + g.nsrc;
        if (!force_dense && op_cost(m, dt) > op_cost(cur, dt) + op_cost(g, dt) + 1e-9) return false;
        cur = std::move(m);
        return true;
    }
    if (kdense < 1 || (int)U.size() > kdense) return false;
    // dense merge: matrix over U (controls become qubits of the fused gate)
    CGate m;
    m.cls = C_DENSE;
    m.tq = U;
    const size_t D = size_t(1) << U.size();
    m.m = matmul(embed(g, U), embed(cur, U), D);
    m.nsrc = cur.nsrc + g.nsrc;
    if (!force_dense) {
        // keep controls as controls where possible: a merged op is only worth it if cheaper
        if (op_cost(m, dt) > op_cost(cur, dt) + op_cost(g, dt) + 1e-9) return false;
    }
    cur = std::move(m);
    return true;
}

std::vector<CGate> fuse_pass(const std::vector<CGate> &in, int kdiag, int kdense, bool force_dense,
                             bool diag_only, qs_dtype dt)
{
    const int window = 256;
    std::vector<CGate> out;
    std::vector<char> used(in.size(), 0);
    for (size_t i = 0; i < in.size(); ++i) {
        if (used[i]) continue;
        used[i] = 1;
        CGate cur = in[i];
        if (diag_only && cur.cls != C_DIAG) {
            out.push_back(std::move(cur));
            continue;
        }
        std::map<int, char> skipped;
        for (size_t j = i + 1; j < in.size() && j < i + window; ++j) {
            if (used[j]) continue;
            const CGate &g = in[j];
            bool merged = false;
            if (hoistable(g, skipped) && !(diag_only && g.cls != C_DIAG))
                merged = try_merge(cur, g, kdiag, diag_only ? 0 : kdense, force_dense, dt);
            if (merged) {
                used[j] = 1;
                continue;
            }
            note_skipped(g, skipped);
            // stop once every qubit of cur is blocked by a non-diagonal skipped gate
            bool all_blocked = true;
            for (int q : all_qubits(cur)) {
                auto it = skipped.find(q);
                if (it == skipped.end() || it->second != 'N') { all_blocked = false; break; }
            }
            if (all_blocked) break;
        }
        // a fused product that came out as the identity (H then H, RZ then RZ^-1, ...) does
        // nothing: drop it (a uniform phase is kept, it is not the identity)
        bool identity = cur.cls == C_DENSE || cur.cls == C_DIAG;
        if (identity) {
            const size_t D = size_t(1) << cur.tq.size();
            for (size_t r = 0; identity && r < D; ++r)
                for (size_t c = 0; identity && c < (cur.cls == C_DENSE ? D : 1); ++c) {
                    const cd want = (cur.cls == C_DIAG || r == c) ? cd(1.0) : cd(0.0);
                    const cd got = cur.cls == C_DIAG ? cur.m[r] : cur.m[r * D + c];
                    identity = std::abs(got - want) <= 1e-14;
                }
        }
        if (!identity) out.push_back(std::move(cur));
    }
    return out;
}

// ------------------------------------------------------------------ device-op construction

struct Coefs {
    std::vector<cd> &pool;
    uint32_t push(const std::vector<cd> &v)
    {
        const uint32_t off = (uint32_t)pool.size();
        pool.insert(pool.end(), v.begin(), v.end());
        return off;
    }
};

// local_of[p] = slab-local bit of physical position p, or -1 if p is outside the slab.
// phys[] = physical position of each logical qubit at the op's turn.
DevOp make_op(const CGate &g, const std::vector<int> &phys, const int *local_of, Coefs &cf)
{
    DevOp op;
    std::memset(&op, 0, sizeof op);
    std::vector<int> ins;
    uint64_t cmask = 0, ocmask = 0;
    for (int c : g.cq) {
        const int p = phys[c];
        const int l = local_of[p];
        if (l >= 0) {
            cmask |= 1ull << l;
            ins.push_back(l);
        } else {
            ocmask |= 1ull << p;
        }
    }
    switch (g.cls) {
    case C_DENSE:
    case C_PERMX:
    case C_SWAP: {
        op.type = g.cls == C_DENSE ? OP_DENSE : g.cls == C_PERMX ? OP_PERMX : OP_SWAP;
        op.k = (uint8_t)g.tq.size();
        for (size_t j = 0; j < g.tq.size(); ++j) {
            const int l = local_of[phys[g.tq[j]]];
            op.t[j] = (uint8_t)l;
            ins.push_back(l);
        }
        if (g.cls == C_DENSE) op.mat = cf.push(g.m);
        break;
    }
    case C_DIAG: {
        op.type = OP_DIAG;
        // table bits: local qubits first (in tq order), then outer ones
        std::vector<int> locq, outq;
        for (size_t j = 0; j < g.tq.size(); ++j) {
            if (local_of[phys[g.tq[j]]] >= 0) locq.push_back((int)j);
            else outq.push_back((int)j);
        }
        op.k = (uint8_t)locq.size();
        op.nout = (uint8_t)outq.size();
        for (size_t j = 0; j < locq.size(); ++j) op.t[j] = (uint8_t)local_of[phys[g.tq[locq[j]]]];
        for (size_t j = 0; j < outq.size(); ++j) op.outpos[j] = (uint8_t)phys[g.tq[outq[j]]];
        const size_t D = g.m.size();
        std::vector<cd> tab(D);
        for (size_t o = 0; o < D; ++o) {
            size_t idx = 0;
            for (size_t j = 0; j < locq.size(); ++j) idx |= ((o >> locq[j]) & 1) << j;
            for (size_t j = 0; j < outq.size(); ++j) idx |= ((o >> outq[j]) & 1) << (locq.size() + j);
            tab[idx] = g.m[o];
        }
        op.mat = cf.push(tab);
        break;
    }
    }
    std::sort(ins.begin(), ins.end());
    op.nins = (uint8_t)ins.size();
    for (size_t j = 0; j < ins.size(); ++j) op.ins[j] = (uint8_t)ins[j];
    op.cmask = cmask;
    op.ocmask = ocmask;
    return op;
}

struct Sched {
    int gate;
    std::vector<int> phys;  // logical -> physical snapshot
};

// The kernel's XOR swizzle of slab-local indices in shared memory (same map as the device's
// swz<>: complex64 XORs bits 1-3 with bits 5-7 and 9-11, complex128 bits 0-2 with 3-5, 6-8, 9-11).
uint32_t smem_swizzle(uint32_t i, qs_dtype dt)
{
    if (dt == QS_C64) return i ^ (((i >> 4) ^ (i >> 8)) & 0xEu);
    return i ^ (((i >> 3) ^ (i >> 6) ^ (i >> 9)) & 7u);
}

// Split every uncontrolled, complex, non-diagonal 1-qubit gate into Z-Y-Z Euler form,
//   U = g P(beta) R P(delta),   P(phi) = diag(1, e^{i phi}),   R = [[c, -s], [s, c]] (real),
// with c = |U00|, s = |U10|, g = U00 / c, e^{i beta} = U10 / (g s), e^{i delta} = -U01 / (g s)
// (all FP64), and write every uncontrolled 1-qubit diagonal diag(d0, d1) as d0 P(arg d1/d0).
// The real rotation costs half the FMAs of a complex 2x2, and the phases of all qubits between
// two layers of rotations commute, so the register stages merge them into one table.  The
// scalar factors g and d0 are collected into one diagonal placed first (a global phase).
std::vector<CGate> split_one_qubit(const std::vector<CGate> &in)
{
    std::vector<CGate> out;
    out.reserve(in.size() * 2);
    cd G = 1.0;
    for (const CGate &g : in) {
        if (g.cq.empty() && g.tq.size() == 1 && g.cls == C_DIAG) {
            const cd d0 = g.m[0], d1 = g.m[1];
            if (d0 != cd(1.0) && std::abs(d0) > 0.5) {
                G *= d0;
                CGate p = g;
                p.m = {cd(1.0), d1 / d0};
                out.push_back(std::move(p));
                continue;
            }
        } else if (g.cq.empty() && g.tq.size() == 1 && g.cls == C_DENSE) {
            bool real = true;
            for (const cd &x : g.m) real = real && x.imag() == 0.0;
            const cd u00 = g.m[0], u01 = g.m[1], u10 = g.m[2], u11 = g.m[3];
            const double c = std::abs(u00), s = std::abs(u10);
            if (!real && c > 1e-6 && s > 1e-6) {
                const cd gph = u00 / c;
                const cd eb = u10 / (gph * s), ed = -u01 / (gph * s);
                if (std::abs(u11 - gph * eb * ed * c) <= 1e-12) {
                    G *= gph;
                    CGate pd, r, pb;
                    pd.cls = pb.cls = C_DIAG;
                    pd.tq = pb.tq = r.tq = g.tq;
                    pd.m = {cd(1.0), ed};
                    pb.m = {cd(1.0), eb};
                    pd.nsrc = pb.nsrc = 0;
                    r.cls = C_DENSE;
                    r.m = {cd(c), cd(-s), cd(s), cd(c)};
                    r.nsrc = g.nsrc;
                    out.push_back(std::move(pd));
                    out.push_back(std::move(r));
                    out.push_back(std::move(pb));
                    continue;
                }
            }
        }
        out.push_back(g);
    }
    if (G != cd(1.0)) {
        CGate gp;
        gp.cls = C_DIAG;
        gp.tq = {0};
        gp.m = {G, G};
        gp.nsrc = 0;
        out.insert(out.begin(), std::move(gp));
    }
    return out;
}

// A diagonal gate whose entries are all 1 except the last one (all qubits 1): Z, S, T, P, CZ,
// CP and their controlled forms.
bool controlled_phase(const CGate &g, cd &phase)
{
    if (g.cls != C_DIAG || g.m.empty()) return false;
    for (size_t i = 0; i + 1 < g.m.size(); ++i)
        if (g.m[i] != cd(1.0)) return false;
    phase = g.m.back();
    return true;
}

// Merge the register-bit diagonals of one stage (subs [s0, end)) into as few tables as
// possible.  A diagonal on register bits commutes with every other diagonal and with every
// non-diagonal sub whose target bits it does not read, so it may sit anywhere in the interval
// of positions between the nearest conflicting non-diagonal subs before and after it.  The
// fewest positions meeting every interval are found by the greedy interval-stabbing rule
// (sort by right end, place a point at the first uncovered right end).  Each group of two or
// more diagonals whose element-wise product is cheaper as one table (one complex multiply per
// amplitude) than as separate subs becomes one SB_DIAG.  A controlled phase whose condition
// includes slab bits outside the registers or physical bits outside the slab joins too: those
// bits are constant for a thread's group, so they index the table (up to kMergeCondBits of them
// per table).  Diagonal tables that already read such bits stay where they are.
// Condition bits of one merged table when qs_options.merge_bits is 0: 10 for complex128 stages
// in FP64, whose time is FP64 multiplies (QFT-32: 2.23 s with 6 bits, 1.98 s with 10; layered
// circuits within 0.3 %), else 6 (complex64 and double-float stages are slightly slower with
// the larger tables).
int default_merge_bits(const Plan &plan) { return plan.dt == QS_C128 && plan.opt.arith == QS_ARITH_FP64 ? 10 : 6; }

void merge_stage_diagonals(Plan &plan, int s0, int RB, Coefs &cf)
{
    const int kMergeCondBits = plan.opt.merge_bits > 0 ? std::min(plan.opt.merge_bits, 10) : default_merge_bits(plan);
    const int E = 1 << RB;
    std::vector<DevSub> in(plan.subs.begin() + s0, plan.subs.end());
    const int ns = (int)in.size();
    auto target_bits = [](const DevSub &s) -> uint32_t {
        switch (s.type) {
        case SB_G1: case SB_G1R: case SB_G1N: case SB_G1A: case SB_G1NM: case SB_G1AM: case SB_X:
            return 1u << s.j0;
        case SB_G2: case SB_SWAP: return (1u << s.j0) | (1u << s.j1);
        default: return 0;
        }
    };
    auto is_diag = [](const DevSub &s) { return s.type == SB_PHASE || s.type == SB_DIAG; };
    auto eligible = [kMergeCondBits](const DevSub &s) {
        return (s.type == SB_PHASE && __builtin_popcount(s.lcm) + __builtin_popcountll(s.ocm) <= kMergeCondBits) ||
               (s.type == SB_DIAG && s.ndl == 0);
    };
    std::vector<std::vector<cd>> tab(ns);
    std::vector<std::vector<uint8_t>> cond(ns);  // bits (DevSub::dl codes) that must all be 1
    std::vector<uint32_t> reads(ns, 0);
    std::vector<double> cost(ns, 0.0);
    std::vector<int> slot(ns, 0), nd_index;  // nd_index: positions of non-diagonal subs
    for (int i = 0; i < ns; ++i) {
        slot[i] = (int)nd_index.size();
        if (!is_diag(in[i])) {
            nd_index.push_back(i);
            continue;
        }
        if (!eligible(in[i])) continue;
        std::vector<cd> t(E, cd(1.0));
        if (in[i].type == SB_PHASE) {
            const cd p = plan.coef[in[i].mat];
            for (int e = 0; e < E; ++e)
                if ((uint32_t(e) & in[i].scm) == in[i].scm) t[e] = p;
            for (int l = 0; l < 32; ++l)
                if (in[i].lcm >> l & 1) cond[i].push_back((uint8_t)l);
            for (int q = 0; q < 64; ++q)
                if (in[i].ocm >> q & 1) cond[i].push_back((uint8_t)(0x80 | q));
            const double frac = std::ldexp(1.0, -__builtin_popcount(in[i].scm) - (int)cond[i].size());
            cost[i] = E * frac * (p == cd(-1.0) ? 0.25 : 1.0);
        } else {
            for (int e = 0; e < E; ++e) t[e] = plan.coef[in[i].mat + e];
            cost[i] = E;
        }
        for (int j = 0; j < RB; ++j)
            for (int e = 0; e < E; ++e)
                if (t[e] != t[e ^ (1 << j)]) {
                    reads[i] |= 1u << j;
                    break;
                }
        tab[i] = std::move(t);
    }
    const int m = (int)nd_index.size();
    // feasible slot interval [lo, hi] of each eligible diagonal
    std::vector<int> lo(ns, 0), hi(ns, m), cand;
    for (int i = 0; i < ns; ++i) {
        if (tab[i].empty()) continue;
        for (int k = 0; k < slot[i]; ++k)
            if (target_bits(in[nd_index[k]]) & reads[i]) lo[i] = k + 1;
        for (int k = slot[i]; k < m; ++k)
            if (target_bits(in[nd_index[k]]) & reads[i]) {
                hi[i] = k;
                break;
            }
        cand.push_back(i);
    }
    std::sort(cand.begin(), cand.end(), [&](int a, int b) { return hi[a] < hi[b] || (hi[a] == hi[b] && a < b); });
    std::vector<int> point(ns, -1);
    std::vector<std::vector<int>> groups;
    std::vector<std::vector<uint8_t>> gcond;  // union of the members' condition bits
    std::vector<int> gpoint;
    for (int i : cand) {
        if (point[i] >= 0) continue;
        const int p = hi[i];
        std::vector<int> gr;
        std::vector<uint8_t> un;
        for (int j : cand) {
            if (point[j] >= 0 || lo[j] > p || p > hi[j]) continue;
            std::vector<uint8_t> u2 = un;
            for (uint8_t c : cond[j])
                if (std::find(u2.begin(), u2.end(), c) == u2.end()) u2.push_back(c);
            if ((int)u2.size() > kMergeCondBits) continue;  // left for another table
            un = std::move(u2);
            point[j] = p;
            gr.push_back(j);
        }
        groups.push_back(gr);
        gcond.push_back(un);
        gpoint.push_back(p);
    }
    std::vector<char> merged(ns, 0);
    std::vector<std::vector<DevSub>> at(m + 1);
    bool changed = false;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const std::vector<int> &gr = groups[gi];
        double c = 0;
        for (int i : gr) c += cost[i];
        if (gr.size() < 2 || c <= 1.25 * E) continue;
        // table over (condition bits hi, register index e): a member contributes where all of its
        // condition bits are set in hi
        const std::vector<uint8_t> &un = gcond[gi];
        const int ndl = (int)un.size();
        std::vector<cd> t(size_t(E) << ndl, cd(1.0));
        for (int i : gr) {
            uint32_t need = 0;
            for (uint8_t cbit : cond[i]) need |= 1u << (std::find(un.begin(), un.end(), cbit) - un.begin());
            for (uint32_t h = 0; h < (1u << ndl); ++h)
                if ((h & need) == need)
                    for (int e = 0; e < E; ++e) t[(size_t(h) << RB) | e] *= tab[i][e];
            merged[i] = 1;
        }
        DevSub s;
        std::memset(&s, 0, sizeof s);
        s.type = SB_DIAG;
        s.ndl = (uint8_t)ndl;
        for (int j = 0; j < ndl; ++j) s.dl[j] = un[j];
        s.mat = cf.push(t);
        at[gpoint[gi]].push_back(s);
        changed = true;
    }
    if (!changed) return;
    std::vector<DevSub> out;
    int k = 0;
    for (int i = 0; i < ns; ++i) {
        if (!is_diag(in[i])) {
            for (const DevSub &s : at[k]) out.push_back(s);
            ++k;
            out.push_back(in[i]);
            continue;
        }
        if (!merged[i]) out.push_back(in[i]);
    }
    for (const DevSub &s : at[m]) out.push_back(s);
    plan.subs.resize(s0);
    plan.subs.insert(plan.subs.end(), out.begin(), out.end());
}

// Write each uncontrolled real 2x2 sub M of a stage (rotations, reflections such as H) as a real
// scalar times a matrix N with two entries of magnitude 1, so that N costs one FMA per real
// output instead of two.  For an orthogonal M (|m00| = |m11|, |m01| = |m10|):
//   |m00| >= |m01|:  M = m00 [[1, m01/m00], [m10/m00, m11/m00]],  m11/m00 = +1 or -1  (N, NM)
//   otherwise:       M = m01 [[m00/m01, 1], [m10/m01, m11/m01]],  m10/m01 = +1 or -1  (A, AM)
// so every ratio is at most 1 in magnitude.  The scalars of all factored subs are collected into
// one scalar sub of the stage (a diagonal that reads no bit), which the diagonal merge that
// follows folds into a table where one exists.  The matrices are FP64 ratios of the gate's own
// entries (Eq. 2-3 reassociated), so results change only by rounding.
void factor_stage_rotations(Plan &plan, int s0, Coefs &cf)
{
    if (plan.opt.factor == 1) return;
    std::vector<DevSub> in(plan.subs.begin() + s0, plan.subs.end());
    int cand = 0;
    bool has_diag = false;
    for (const DevSub &sb : in) {
        if (sb.type == SB_G1R && !(sb.scm | sb.lcm | sb.ocm)) ++cand;
        if (sb.type == SB_PHASE || sb.type == SB_DIAG) has_diag = true;
    }
    // the stage scalar costs one multiply per amplitude unless a table absorbs it, the same as
    // the FMA one factored sub saves
    if (cand == 0 || (cand < 2 && !has_diag)) return;
    double sigma = 1.0;
    std::vector<DevSub> out;
    out.reserve(in.size() + cand + 1);
    for (const DevSub &sb : in) {
        if (sb.type != SB_G1R || (sb.scm | sb.lcm | sb.ocm)) {
            out.push_back(sb);
            continue;
        }
        const double m00 = plan.coef[sb.mat].real(), m01 = plan.coef[sb.mat + 1].real();
        const double m10 = plan.coef[sb.mat + 2].real(), m11 = plan.coef[sb.mat + 3].real();
        DevSub f = sb;
        double x, y, d;
        bool unit;  // the entry that must be +-1 is, to rounding
        if (std::abs(m00) >= std::abs(m01)) {
            d = m00;
            const double r = d != 0.0 ? m11 / d : 0.0;
            unit = std::abs(std::abs(r) - 1.0) <= 1e-13;
            f.type = r > 0 ? SB_G1N : SB_G1NM;
            x = d != 0.0 ? m01 / d : 0.0;
            y = d != 0.0 ? m10 / d : 0.0;
        } else {
            d = m01;
            const double r = m10 / d;
            unit = std::abs(std::abs(r) - 1.0) <= 1e-13;
            f.type = r > 0 ? SB_G1A : SB_G1AM;
            x = m00 / d;
            y = m11 / d;
        }
        if (d == 0.0 || !unit) {
            out.push_back(sb);  // not orthogonal: keep the full matrix
            continue;
        }
        f.mat = cf.push(std::vector<cd>{cd(x), cd(y)});
        out.push_back(f);
        sigma *= d;
    }
    DevSub sc;
    std::memset(&sc, 0, sizeof sc);
    sc.type = SB_PHASE;
    sc.mat = cf.push(std::vector<cd>{cd(sigma)});
    out.push_back(sc);
    plan.subs.resize(s0);
    plan.subs.insert(plan.subs.end(), out.begin(), out.end());
}

// Split a pass's scheduled ops into register stages (Alg. 2's innermost fusion level applied
// to the register file) and shared-memory ops.  A stage collects ops whose non-diagonal local
// bits fit `RB` register bits; ops are taken in order and may move ahead of skipped ops only if
// they commute with them (same role test as the block finder).
void build_stages(Plan &plan, const std::vector<CGate> &gates, const std::vector<Sched> &sched,
                  const int *local_of, int b, qs_dtype dt, Coefs &cf)
{
    (void)dt;
    const int RB = plan.stage_bits;
    const size_t ns = sched.size();
    std::vector<uint64_t> nb(ns, 0), db(ns, 0);
    std::vector<char> regable(ns, 0), done(ns, 0);
    for (size_t i = 0; i < ns; ++i) {
        const CGate &g = gates[sched[i].gate];
        const std::vector<int> &ph = sched[i].phys;
        for (int t : g.tq) {
            const int l = local_of[ph[t]];
            if (g.cls == C_DIAG) {
                if (l >= 0) db[i] |= 1ull << l;
            } else {
                nb[i] |= 1ull << l;
            }
        }
        for (int c : g.cq) {
            const int l = local_of[ph[c]];
            if (l >= 0) db[i] |= 1ull << l;
        }
        cd ph0;
        bool r = b >= RB && b - RB <= 16;
        if (r) {
            switch (g.cls) {
            case C_DENSE: r = g.tq.size() <= 2; break;
            case C_PERMX: case C_SWAP: r = true; break;
            case C_DIAG: r = controlled_phase(g, ph0) || (g.tq.size() + g.cq.size() <= 7); break;
            }
        }
        regable[i] = r;
    }
    size_t first = 0;
    while (true) {
        while (first < ns && done[first]) ++first;
        if (first >= ns) break;
        if (!regable[first]) {
            plan.ops.push_back(make_op(gates[sched[first].gate], sched[first].phys, local_of, cf));
            done[first] = 1;
            continue;
        }
        uint64_t S = 0, skipN = 0, skipD = 0;
        std::vector<size_t> sub;
        for (size_t j = first; j < ns; ++j) {
            if (done[j]) continue;
            const bool hoist = (nb[j] & (skipN | skipD)) == 0 && (db[j] & skipN) == 0;
            if (!hoist || !regable[j]) {
                skipN |= nb[j];
                skipD |= db[j];
                continue;
            }
            const uint64_t need = nb[j] & ~S;
            if (popcount(S | need) <= RB) {
                S |= need;
                sub.push_back(j);
                done[j] = 1;
            } else {
                skipN |= nb[j];
                skipD |= db[j];
            }
        }
        // fill the register set: bits the stage's diagonal ops read first, then high bits
        uint64_t want = 0;
        for (size_t j : sub) want |= db[j];
        for (int l = b - 1; l >= 0 && popcount(S) < RB; --l)
            if ((want >> l & 1) && !(S >> l & 1)) S |= 1ull << l;
        for (int l = b - 1; l >= 0 && popcount(S) < RB; --l)
            if (!(S >> l & 1)) S |= 1ull << l;
        DevStage st;
        std::memset(&st, 0, sizeof st);
        st.r = (uint8_t)RB;
        int regidx[64];
        for (int l = 0; l < 64; ++l) regidx[l] = -1;
        int nr = 0, nrest = 0;
        for (int l = 0; l < b; ++l) {
            if (S >> l & 1) {
                st.sbits[nr] = (uint8_t)l;
                regidx[l] = nr++;
            } else {
                st.rest[nrest++] = (uint8_t)l;
            }
        }
        st.nrest = (uint8_t)nrest;
        for (int e = 0; e < (1 << RB); ++e) {
            uint32_t o = 0;
            for (int j = 0; j < RB; ++j)
                if (e >> j & 1) o |= 1u << st.sbits[j];
            st.off[e] = (uint16_t)smem_swizzle(o, plan.dt);
        }
        st.sub_begin = (int)plan.subs.size();
        for (size_t j : sub) {
            const CGate &g = gates[sched[j].gate];
            const std::vector<int> &ph = sched[j].phys;
            DevSub s;
            std::memset(&s, 0, sizeof s);
            auto classify = [&](int q) {
                const int l = local_of[ph[q]];
                if (l < 0) s.ocm |= 1ull << ph[q];
                else if (regidx[l] >= 0) s.scm |= 1u << regidx[l];
                else s.lcm |= 1u << l;
            };
            cd phase;
            if (g.cls != C_DIAG)
                for (int c : g.cq) classify(c);
            switch (g.cls) {
            case C_DENSE:
                if (g.tq.size() == 1) {
                    bool real = true;
                    for (const cd &x : g.m) real = real && x.imag() == 0.0;
                    s.type = real ? SB_G1R : SB_G1;
                    s.j0 = (uint8_t)regidx[local_of[ph[g.tq[0]]]];
                    s.mat = cf.push(g.m);
                } else {
                    int j0 = regidx[local_of[ph[g.tq[0]]]], j1 = regidx[local_of[ph[g.tq[1]]]];
                    std::vector<cd> m = g.m;
                    if (j0 > j1) {
                        // exchange the two index bits of rows and columns
                        auto sw = [](int x) { return ((x & 1) << 1) | ((x >> 1) & 1); };
                        for (int r = 0; r < 4; ++r)
                            for (int c = 0; c < 4; ++c) m[sw(r) * 4 + sw(c)] = g.m[r * 4 + c];
                        std::swap(j0, j1);
                    }
                    s.type = SB_G2;
                    s.j0 = (uint8_t)j0;
                    s.j1 = (uint8_t)j1;
                    s.mat = cf.push(m);
                }
                break;
            case C_PERMX:
                s.type = SB_X;
                s.j0 = (uint8_t)regidx[local_of[ph[g.tq[0]]]];
                break;
            case C_SWAP: {
                int j0 = regidx[local_of[ph[g.tq[0]]]], j1 = regidx[local_of[ph[g.tq[1]]]];
                if (j0 > j1) std::swap(j0, j1);
                s.type = SB_SWAP;
                s.j0 = (uint8_t)j0;
                s.j1 = (uint8_t)j1;
                break;
            }
            case C_DIAG:
                if (controlled_phase(g, phase)) {
                    s.type = SB_PHASE;
                    for (int q : g.tq) classify(q);
                    for (int c : g.cq) classify(c);
                    s.mat = cf.push(std::vector<cd>{phase});
                } else {
                    s.type = SB_DIAG;
                    std::vector<int> Q = g.tq;
                    Q.insert(Q.end(), g.cq.begin(), g.cq.end());
                    const int ntq = (int)g.tq.size();
                    std::vector<int> qreg(Q.size(), -1), qhi(Q.size(), -1);
                    int ndl = 0;
                    for (size_t k = 0; k < Q.size(); ++k) {
                        const int l = local_of[ph[Q[k]]];
                        if (l >= 0 && regidx[l] >= 0) {
                            qreg[k] = regidx[l];
                        } else {
                            qhi[k] = ndl;
                            s.dl[ndl++] = l >= 0 ? (uint8_t)l : (uint8_t)(0x80 | ph[Q[k]]);
                        }
                    }
                    s.ndl = (uint8_t)ndl;
                    std::vector<cd> tab(size_t(1) << (RB + ndl));
                    for (size_t hi = 0; hi < (size_t(1) << ndl); ++hi)
                        for (int e = 0; e < (1 << RB); ++e) {
                            bool ctl_ok = true;
                            size_t idx = 0;
                            for (size_t k = 0; k < Q.size(); ++k) {
                                const size_t bit = qreg[k] >= 0 ? ((e >> qreg[k]) & 1) : ((hi >> qhi[k]) & 1);
                                if ((int)k < ntq) idx |= bit << k;
                                else if (!bit) ctl_ok = false;
                            }
                            tab[(hi << RB) | e] = ctl_ok ? g.m[idx] : cd(1.0);
                        }
                    s.mat = cf.push(tab);
                }
                break;
            }
            plan.subs.push_back(s);
        }
        factor_stage_rotations(plan, st.sub_begin, cf);
        merge_stage_diagonals(plan, st.sub_begin, RB, cf);
        st.sub_end = (int)plan.subs.size();
        DevOp op;
        std::memset(&op, 0, sizeof op);
        op.type = OP_STAGE;
        op.mat = (uint32_t)plan.stages.size();
        plan.stages.push_back(st);
        plan.ops.push_back(op);
    }
}

void emit_pass(Plan &plan, const std::vector<CGate> &gates, std::vector<int> S, int lo, int b, int n,
               const std::vector<Sched> &sched, StepKind kind, qs_dtype dt)
{
    // pad the slab up to b bits with the lowest unused positions
    std::set<int> inS(S.begin(), S.end());
    for (int p = 0; (int)inS.size() < b && p < n; ++p) inS.insert(p);
    DevPass P;
    std::memset(&P, 0, sizeof P);
    std::vector<int> hi;
    for (int p : inS)
        if (p >= lo) hi.push_back(p);
    P.b = (int)inS.size();
    P.lo = lo;
    P.nhi = (int)hi.size();
    for (size_t j = 0; j < hi.size(); ++j) P.hipos[j] = (uint8_t)hi[j];
    for (int j = 0; j < 32; ++j) P.perm[j] = (uint8_t)j;
    int local_of[64];
    for (int p = 0; p < 64; ++p) local_of[p] = -1;
    for (int p = 0; p < lo; ++p) local_of[p] = p;
    for (size_t j = 0; j < hi.size(); ++j) local_of[hi[j]] = lo + (int)j;
    Coefs cf{plan.coef};
    P.op_begin = (int)plan.ops.size();
    build_stages(plan, gates, sched, local_of, P.b, dt, cf);
    P.op_end = (int)plan.ops.size();
    P.has_perm = 0;
    plan.steps.push_back({kind, (int)plan.passes.size()});
    plan.passes.push_back(P);
}

// ------------------------------------------------------------------ tensor-core steps

uint16_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
}

float bf16_value(uint16_t h)
{
    const uint32_t u = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Operand images of a 6-qubit gate U for the tensor-core kernel: the real embedding
// E (128 x 128, rows = output index n, columns = input index k, interleaved re/im) split as
// E = E_hi + E_lo in BF16 (from FP64), each stored in the 128-byte-swizzled K-major layout
// (K split into 128-byte atoms of 64 elements stored one after the other for all 128 rows;
// 16-byte chunk c of row r placed at chunk c ^ (r & 7)).
// TF32 value nearest to f (round to nearest even on the 10 stored mantissa bits), as FP32 bits.
uint32_t tf32_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0xFFFu + ((u >> 13) & 1u);
    return u & ~0x1FFFu;
}

float tf32_value(uint32_t u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Image layout of one E matrix: per 128-byte K atom (128 rows x 128 bytes = 16 KiB per part),
// the hi part then the lo part, so that the kernel fetches one atom of both parts with one
// 32 KiB bulk copy.  `hi` and `lo` hold the parts atom after atom.
void append_atoms(std::vector<unsigned char> &out, const unsigned char *hi, const unsigned char *lo, size_t part_bytes)
{
    const size_t atom = size_t(kTcRows) * 128;
    const size_t base = out.size();
    out.resize(base + 2 * part_bytes);
    for (size_t a = 0; a * atom < part_bytes; ++a) {
        std::memcpy(out.data() + base + 2 * a * atom, hi + a * atom, atom);
        std::memcpy(out.data() + base + (2 * a + 1) * atom, lo + a * atom, atom);
    }
}

// TF32 x 3 images: E = E_hi + E_lo in TF32 (from FP64), 4-byte elements in the same swizzled
// K-major layout with 128-byte atoms of 32 elements (four K atoms).
void tc_images_tf32(const std::vector<cd> &U, std::vector<unsigned char> &out)
{
    const int K = kTcK, R = kTcK;
    std::vector<uint32_t> hi(size_t(R) * K), lo(size_t(R) * K);
    for (int j = 0; j < K / 2; ++j)
        for (int l = 0; l < K / 2; ++l) {
            const cd u = U[size_t(j) * (K / 2) + l];
            const double e[2][2] = {{u.real(), -u.imag()}, {u.imag(), u.real()}};
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) {
                    const int n = 2 * j + a, k = 2 * l + c;
                    const double x = e[a][c];
                    const uint32_t h = tf32_rne((float)x);
                    const uint32_t w = tf32_rne((float)(x - (double)tf32_value(h)));
                    const size_t kb = size_t(k) >> 5, kin = size_t(k) & 31;
                    const size_t chunk = kin >> 2, within = kin & 3;
                    const size_t idx = kb * (size_t(R) * 32) + size_t(n) * 32 + ((chunk ^ (n & 7)) << 2) + within;
                    hi[idx] = h;
                    lo[idx] = w;
                }
        }
    append_atoms(out, reinterpret_cast<const unsigned char *>(hi.data()), reinterpret_cast<const unsigned char *>(lo.data()),
                 hi.size() * 4);
}

void tc_images(const std::vector<cd> &U, std::vector<unsigned char> &out)
{
    const int K = kTcK, R = kTcK;
    std::vector<uint16_t> hi(size_t(R) * K), lo(size_t(R) * K);
    for (int j = 0; j < K / 2; ++j)
        for (int l = 0; l < K / 2; ++l) {
            const cd u = U[size_t(j) * (K / 2) + l];
            const double e[2][2] = {{u.real(), -u.imag()}, {u.imag(), u.real()}};
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) {
                    const int n = 2 * j + a, k = 2 * l + c;
                    const double x = e[a][c];
                    const uint16_t h = bf16_rne((float)x);
                    const uint16_t w = bf16_rne((float)(x - (double)bf16_value(h)));
                    const size_t kb = size_t(k) >> 6, kin = size_t(k) & 63;
                    const size_t chunk = kin >> 3, within = kin & 7;
                    const size_t idx = kb * (size_t(R) * 64) + size_t(n) * 64 + ((chunk ^ (n & 7)) << 3) + within;
                    hi[idx] = h;
                    lo[idx] = w;
                }
        }
    append_atoms(out, reinterpret_cast<const unsigned char *>(hi.data()), reinterpret_cast<const unsigned char *>(lo.data()),
                 hi.size() * 2);
}

// The 64x64 block U[t' 64 + j'][t 64 + j] of a 7-qubit matrix (t', t = bit 6 of row, column).
std::vector<cd> tc_block(const std::vector<cd> &U, int tr, int tc)
{
    std::vector<cd> B(size_t(64) * 64);
    for (size_t j = 0; j < 64; ++j)
        for (size_t l = 0; l < 64; ++l) B[j * 64 + l] = U[(size_t(tr) * 64 + j) * 128 + size_t(tc) * 64 + l];
    return B;
}

// A tensor-core step for dense gate g (6 or 7 targets) at the current layout.  A 7th target
// becomes row bit 6 of the slab's 128 x 64 matrix view.
void emit_tc(Plan &plan, const CGate &g, const std::vector<int> &phys, int lo, int n, int mode)
{
    std::set<int> S;
    for (int p = 0; p < lo; ++p) S.insert(p);
    for (int t : g.tq) S.insert(phys[t]);
    for (int p = 0; (int)S.size() < kTcSlabBits && p < n; ++p) S.insert(p);
    DevTc T;
    std::memset(&T, 0, sizeof T);
    std::vector<int> hi;
    for (int p : S)
        if (p >= lo) hi.push_back(p);
    T.slab.b = (int)S.size();
    T.slab.lo = lo;
    T.slab.nhi = (int)hi.size();
    for (size_t j = 0; j < hi.size(); ++j) T.slab.hipos[j] = (uint8_t)hi[j];
    for (int j = 0; j < 32; ++j) T.slab.perm[j] = (uint8_t)j;
    int local_of[64];
    for (int p = 0; p < 64; ++p) local_of[p] = -1;
    for (int p = 0; p < lo; ++p) local_of[p] = p;
    for (size_t j = 0; j < hi.size(); ++j) local_of[hi[j]] = lo + (int)j;
    const int width = (int)g.tq.size();
    uint32_t tmask = 0;
    std::vector<int> tphys;
    for (int j = 0; j < width; ++j) {
        const uint8_t l = (uint8_t)local_of[phys[g.tq[j]]];
        if (j < kTcTargets) T.tpos[j] = l;
        tmask |= 1u << l;
        tphys.push_back(phys[g.tq[j]]);
    }
    int m = 0;
    for (int l = 0; l < kTcSlabBits; ++l)
        if (!(tmask >> l & 1)) T.mpos[m++] = (uint8_t)l;
    if (width == 7) T.mpos[m++] = (uint8_t)local_of[phys[g.tq[6]]];
    T.img = (uint32_t)plan.tc_images.size();
    T.mode = mode;
    T.width = width;
    auto images = [&](const std::vector<cd> &U) {
        if (mode == QS_TC_TF32X3) tc_images_tf32(U, plan.tc_images);
        else tc_images(U, plan.tc_images);
    };
    if (width == 7)
        for (int b = 0; b < 4; ++b) images(tc_block(g.m, b >> 1, b & 1));
    else
        images(g.m);
    plan.tc_coef.push_back((uint32_t)plan.coef.size());
    plan.coef.insert(plan.coef.end(), g.m.begin(), g.m.end());
    plan.tc_phys.push_back(tphys);
    plan.steps.push_back({S_TC, (int)plan.tcs.size()});
    plan.tcs.push_back(T);
}

// Widen a dense gate to 6 targets: identity on added qubits (added as the high index bits).
CGate pad_to_tc(const CGate &g, int n, const std::vector<int> &phys)
{
    CGate r;
    r.cls = C_DENSE;
    r.tq = g.tq;
    r.nsrc = g.nsrc;
    // prefer qubits that already sit in the lowest physical positions
    std::vector<int> byphys(n);
    for (int q = 0; q < n; ++q) byphys[phys[q]] = q;
    for (int p = 0; p < n && (int)r.tq.size() < kTcTargets; ++p) {
        const int q = byphys[p];
        if (std::find(r.tq.begin(), r.tq.end(), q) == r.tq.end()) r.tq.push_back(q);
    }
    const int k = (int)g.tq.size();
    const size_t D = size_t(1) << kTcTargets, d = size_t(1) << k;
    r.m.assign(D * D, 0.0);
    for (size_t row = 0; row < D; ++row)
        for (size_t col = 0; col < D; ++col)
            if ((row >> k) == (col >> k)) r.m[row * D + col] = g.m[(row & (d - 1)) * d + (col & (d - 1))];
    return r;
}

void emit_remap(Plan &plan, int n, int lo, const std::vector<int> &A, const std::vector<int> &B)
{
    std::set<int> inS;
    for (int p = 0; p < lo; ++p) inS.insert(p);
    for (int p : A) inS.insert(p);
    for (int p : B) inS.insert(p);
    (void)n;
    DevPass P;
    std::memset(&P, 0, sizeof P);
    std::vector<int> hi;
    for (int p : inS)
        if (p >= lo) hi.push_back(p);
    P.b = (int)inS.size();
    P.lo = lo;
    P.nhi = (int)hi.size();
    for (size_t j = 0; j < hi.size(); ++j) P.hipos[j] = (uint8_t)hi[j];
    int local_of[64];
    for (int p = 0; p < 64; ++p) local_of[p] = -1;
    for (int p = 0; p < lo; ++p) local_of[p] = p;
    for (size_t j = 0; j < hi.size(); ++j) local_of[hi[j]] = lo + (int)j;
    for (int j = 0; j < 32; ++j) P.perm[j] = (uint8_t)j;
    for (size_t j = 0; j < A.size(); ++j) {
        const int la = local_of[A[j]], lb = local_of[B[j]];
        P.perm[la] = (uint8_t)lb;
        P.perm[lb] = (uint8_t)la;
    }
    P.op_begin = P.op_end = (int)plan.ops.size();
    P.has_perm = 1;
    plan.steps.push_back({S_REMAP, (int)plan.passes.size()});
    plan.passes.push_back(P);
}

int max_remap_pairs(int bmax, int lo) { return std::max(1, (bmax - lo) / 2); }

}  // namespace

// ------------------------------------------------------------------ remap plans

int plan_remap(int n, qs_dtype dt, const std::vector<int> &A, const std::vector<int> &B, Plan &plan,
               std::string &err)
{
    const int lo = std::min(default_seg_bits(dt), n);
    const int bmax = std::min(max_slab_bits(dt), n);
    if (A.size() != B.size()) {
        err = "remap: A and B differ in length";
        return QS_EINVAL;
    }
    uint64_t used = 0;
    for (size_t j = 0; j < A.size(); ++j) {
        for (int p : {A[j], B[j]}) {
            if (p < 0 || p >= n || (used >> p & 1)) {
                err = "remap: positions must be distinct and in range";
                return QS_EINVAL;
            }
            used |= 1ull << p;
        }
    }
    // split into passes whose slab (low segment + pair positions) fits on chip
    std::vector<int> a, b;
    int extra = 0;
    for (size_t j = 0; j < A.size(); ++j) {
        const int add = (A[j] >= lo) + (B[j] >= lo);
        if (extra + add > bmax - lo && !a.empty()) {
            emit_remap(plan, n, lo, a, b);
            a.clear();
            b.clear();
            extra = 0;
        }
        a.push_back(A[j]);
        b.push_back(B[j]);
        extra += add;
    }
    if (!a.empty()) emit_remap(plan, n, lo, a, b);
    return QS_OK;
}

void plan_canonicalize(int n, qs_dtype dt, const std::vector<int> &phys_of, Plan &plan)
{
    const int lo = std::min(default_seg_bits(dt), n);
    const int bmax = std::min(max_slab_bits(dt), n);
    std::vector<int> log_of(n);
    for (int q = 0; q < n; ++q) log_of[phys_of[q]] = q;
    for (int guard = 0; guard < 4 * n + 8; ++guard) {
        bool done = true;
        for (int p = 0; p < n; ++p)
            if (log_of[p] != p) done = false;
        if (done) break;
        std::vector<int> A, B;
        uint64_t used = 0;
        int extra = 0;
        for (int p = 0; p < n; ++p) {
            if (log_of[p] == p) continue;
            const int t = log_of[p];  // position p holds logical t, whose home is position t
            if ((used >> p & 1) || (used >> t & 1)) continue;
            const int add = (p >= lo) + (t >= lo);
            if (extra + add > bmax - lo) continue;
            used |= (1ull << p) | (1ull << t);
            extra += add;
            A.push_back(p);
            B.push_back(t);
        }
        emit_remap(plan, n, lo, A, B);
        for (size_t j = 0; j < A.size(); ++j) std::swap(log_of[A[j]], log_of[B[j]]);
    }
}

// ------------------------------------------------------------------ full plan

int build_plan(const std::vector<CGate> &gates_in, int n, qs_dtype dt, const qs_options &opt,
               Plan &plan, std::string &err)
{
    plan.n = n;
    plan.dt = dt;
    plan.opt = opt;
    {
        const int def = dt == QS_C64 ? kStageBitsC64 : kStageBitsC128;
        int rb = opt.stage_bits > 0 ? opt.stage_bits : def;
        if (rb > def) rb = def;
        if (rb < def - 1) rb = def - 1;
        plan.stage_bits = rb;
    }
    plan.input_gates = (int)gates_in.size();
    const bool lowblock = opt.slab_mode == QS_SLAB_REMAP;

    // ---- slab geometry
    const int lo = opt.seg_bits > 0 ? std::min(opt.seg_bits, n) : std::min(default_seg_bits(dt), n);
    int b = opt.slab_bits > 0 ? opt.slab_bits : default_slab_bits(dt);
    b = std::min(b, std::min(max_slab_bits(dt), n));
    if (b < lo) b = lo;
    if (b - lo > 12) b = lo + 12;
    plan.slab_bits = b;
    plan.seg_bits = lo;
    const int bmax = std::min(max_slab_bits(dt), n);

    // ---- uncontrolled SWAP gates only relabel qubits (Sec. II-B): drop them and rename the
    // qubits of later gates.  True qubit q lives on working qubit sigma[q] afterwards.
    std::vector<int> sigma(n);
    for (int q = 0; q < n; ++q) sigma[q] = q;
    std::vector<CGate> gates;
    gates.reserve(gates_in.size());
    for (const CGate &g0 : gates_in) {
        if (g0.cls == C_SWAP && g0.cq.empty()) {
            std::swap(sigma[g0.tq[0]], sigma[g0.tq[1]]);
            continue;
        }
        CGate g = g0;
        for (int &q : g.tq) q = sigma[q];
        for (int &q : g.cq) q = sigma[q];
        gates.push_back(std::move(g));
    }
    auto finish_layout = [&](const std::vector<int> &phys_w) {
        plan.final_phys_of.assign(n, 0);
        for (int q = 0; q < n; ++q) plan.final_phys_of[q] = phys_w[sigma[q]];
    };

    // ---- fusion (a fused dense gate must still fit one slab pass)
    const bool tc = opt.tc != QS_TC_OFF;
    if (tc) {
        if (dt != QS_C64) {
            err = "the tensor-core path is built for complex64 states";
            return QS_EUNSUPPORTED;
        }
        if (opt.tc != QS_TC_BF16X3 && opt.tc != QS_TC_TF32X3) {
            err = "unknown tensor-core mode";
            return QS_EINVAL;
        }
        if (n < kTcSlabBits || !opt.blocking) {
            err = "the tensor-core path needs blocking and at least 13 qubits";
            return QS_EUNSUPPORTED;
        }
        if (opt.tc_width != 0 && opt.tc_width != 6 && opt.tc_width != 7) {
            err = "tensor-core blocks are 6 or 7 qubits wide";
            return QS_EUNSUPPORTED;
        }
    }
    const int tcw = opt.tc_width == 7 ? 7 : kTcTargets;
    std::vector<char> is_tc;
    if (tc) {
        // Alg. 2 level 3 with F = 6 or 7: merge greedily into dense blocks of at most F qubits;
        // the products are FP64 on the host.  Blocks of 4+ qubits run on the tensor cores (7-qubit
        // blocks as such, narrower ones widened to 6).  Diagonal runs are merged no wider than the
        // blocks by default: wider tables could not join a block and would each cost a pass.
        const int kdiag = opt.diag_bits > 0 ? std::min(opt.diag_bits, kMaxDiagBits) : tcw;
        gates = fuse_pass(gates, kdiag, 0, false, true, dt);
        gates = fuse_pass(gates, kdiag, tcw, true, false, dt);
        for (const CGate &g : gates) is_tc.push_back(g.cls == C_DENSE && g.tq.size() >= 4);
    } else if (opt.fuse_width > 0) {
        const bool euler = opt.euler != 1;
        if (opt.blocking && euler) gates = split_one_qubit(gates);
        const int kdiag = opt.diag_bits > 0 ? std::min(opt.diag_bits, kMaxDiagBits) : 10;
        int kdense = std::min(opt.fuse_width, kMaxDense);
        if (opt.blocking) kdense = std::min(kdense, lowblock ? b : std::max(1, b - lo));
        gates = fuse_pass(gates, kdiag, 0, false, true, dt);
        gates = fuse_pass(gates, kdiag, kdense, opt.fuse_force != 0, false, dt);
    }
    if (is_tc.empty()) is_tc.assign(gates.size(), 0);
    for (size_t gi = 0; gi < gates.size(); ++gi) {
        const CGate &g = gates[gi];
        if (is_tc[gi]) continue;
        if (g.cls == C_DENSE && (int)g.tq.size() > kMaxDense) {
            err = "dense gates wider than 5 qubits need the tensor-core path";
            return QS_EUNSUPPORTED;
        }
        if (g.cls == C_DIAG && (int)g.tq.size() > kMaxDiagBits) {
            err = "diagonal gate wider than 12 qubits";
            return QS_EUNSUPPORTED;
        }
    }
    plan.fused_ops = (int)gates.size();
    double fl = 0;
    for (const CGate &g : gates) {
        const int k = (int)g.tq.size();
        if (g.cls == C_DENSE) fl += 8.0 * std::ldexp(1.0, k) * std::ldexp(1.0, -(int)g.cq.size());
        else if (g.cls == C_DIAG) fl += 6.0;
    }
    plan.flops_per_amp = fl;

    std::vector<int> phys(n), logi(n);
    for (int q = 0; q < n; ++q) phys[q] = logi[q] = q;
    auto is_relabel = [](const CGate &g) { return g.cls == C_SWAP && g.cq.empty(); };
    int ident_local[64];
    for (int p = 0; p < 64; ++p) ident_local[p] = p < n ? p : -1;
    auto emit_unblocked = [&](const CGate &g) {
        Coefs cf{plan.coef};
        DevOp op = make_op(g, phys, ident_local, cf);
        plan.steps.push_back({S_UNBLOCKED, (int)plan.ops.size()});
        plan.ops.push_back(op);
    };

    if (!opt.blocking) {
        // gate-by-gate: one full-state pass per op
        for (const CGate &g : gates) {
            if (is_relabel(g)) {
                std::swap(phys[g.tq[0]], phys[g.tq[1]]);
                continue;
            }
            emit_unblocked(g);
        }
        finish_layout(phys);
        return QS_OK;
    }

    std::vector<char> done(gates.size(), 0);
    size_t first = 0;
    int stalls = 0;
    while (true) {
        while (first < gates.size() && done[first]) ++first;
        if (first >= gates.size()) break;
        if (is_tc[first]) {
            const CGate &g = gates[first];
            emit_tc(plan, g.tq.size() == 7 ? g : pad_to_tc(g, n, phys), phys, lo, n, opt.tc);
            done[first] = 1;
            stalls = 0;
            continue;
        }
        std::set<int> S;
        for (int p = 0; p < (lowblock ? b : lo); ++p) S.insert(p);
        std::map<int, char> skipped;
        std::vector<Sched> sched;
        std::vector<int> wanted;  // low-block mode: logical qubits needed but not resident
        for (size_t i = first; i < gates.size(); ++i) {
            if (done[i]) continue;
            const CGate &g = gates[i];
            if (!hoistable(g, skipped) || is_tc[i]) {
                note_skipped(g, skipped);
                continue;
            }
            if (is_relabel(g)) {
                const int a = g.tq[0], c = g.tq[1];
                std::swap(phys[a], phys[c]);
                logi[phys[a]] = a;
                logi[phys[c]] = c;
                done[i] = 1;
                continue;
            }
            std::vector<int> need;
            if (g.cls != C_DIAG)
                for (int t : g.tq)
                    if (!S.count(phys[t])) need.push_back(phys[t]);
            const bool fits = lowblock ? need.empty() : (int)(S.size() + need.size()) <= b;
            if (fits) {
                for (int p : need) S.insert(p);
                sched.push_back({(int)i, phys});
                done[i] = 1;
            } else {
                if (lowblock)
                    for (int p : need)
                        if (std::find(wanted.begin(), wanted.end(), logi[p]) == wanted.end())
                            wanted.push_back(logi[p]);
                note_skipped(g, skipped);
            }
        }
        if (!sched.empty()) {
            emit_pass(plan, gates, std::vector<int>(S.begin(), S.end()), lo, b, n, sched, S_PASS, dt);
            stalls = 0;
        }
        while (first < gates.size() && done[first]) ++first;
        if (first >= gates.size()) break;
        const int mmax = std::min(max_remap_pairs(bmax, lo), b);
        const CGate &head = gates[first];
        const bool head_fits_alone =
            head.cls == C_DIAG || (lowblock ? (int)head.tq.size() <= mmax : (int)head.tq.size() <= b - lo);
        if (sched.empty() && (!head_fits_alone || stalls > 2)) {
            // the first remaining op cannot be brought into any slab: apply it unblocked
            emit_unblocked(head);
            done[first] = 1;
            stalls = 0;
            continue;
        }
        if (lowblock && !wanted.empty()) {
            // Alg. 4: swap wanted qubits into the low block, evicting block qubits (any position
            // below b) whose next non-diagonal use is farthest away.
            std::vector<int> nextuse(n, 1 << 30);
            int pos = 0;
            for (size_t i = first; i < gates.size(); ++i, ++pos) {
                if (done[i] || gates[i].cls == C_DIAG) continue;
                for (int t : gates[i].tq) nextuse[t] = std::min(nextuse[t], pos);
            }
            // keep the head op's own qubits first in the wanted list
            std::vector<int> want;
            if (head.cls != C_DIAG)
                for (int t : head.tq)
                    if (phys[t] >= b) want.push_back(t);
            for (int q : wanted)
                if (std::find(want.begin(), want.end(), q) == want.end()) want.push_back(q);
            std::vector<int> cand;
            for (int p = 0; p < b; ++p) {
                const int q = logi[p];
                bool head_q = false;
                if (head.cls != C_DIAG)
                    for (int t : head.tq) head_q |= (t == q);
                if (!head_q && std::find(want.begin(), want.end(), q) == want.end()) cand.push_back(p);
            }
            std::stable_sort(cand.begin(), cand.end(),
                             [&](int x, int y) { return nextuse[logi[x]] > nextuse[logi[y]]; });
            std::vector<int> A, B;
            for (size_t j = 0; j < want.size() && (int)A.size() < mmax && j < cand.size(); ++j) {
                A.push_back(cand[j]);
                B.push_back(phys[want[j]]);
            }
            if (!A.empty()) {
                emit_remap(plan, n, lo, A, B);
                for (size_t j = 0; j < A.size(); ++j) {
                    const int qa = logi[A[j]], qb = logi[B[j]];
                    std::swap(phys[qa], phys[qb]);
                    logi[phys[qa]] = qa;
                    logi[phys[qb]] = qb;
                }
            }
        }
        if (sched.empty()) ++stalls;
    }
    finish_layout(phys);
    return QS_OK;
}

}  // namespace qs
