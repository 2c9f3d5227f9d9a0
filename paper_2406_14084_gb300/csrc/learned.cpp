// learned.cpp -- the learned planner: per-step plan features, and the choice among candidate
// plans by the cost-model network.
//
// The greedy planner (Alg. 1-2 with the analytic op cost) fixes the fusion width, the slab
// size and the register-stage width from the caller's options.  The learned planner builds a
// grid of alternatives -- Z-Y-Z split of 1-qubit gates on or off, fusion width 1..5 (widths
// above 2 forced past the analytic check), three slab sizes, two stage widths -- scores every
// step of every distinct candidate with one batched forward launch, and returns the candidate
// whose summed prediction is lowest.  The greedy plan is kept unless a candidate is predicted
// at least 5% faster (a margin over the model's error, about 6% RMS in time).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "learned.h"
#include "model.h"

namespace qs {

namespace {

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

struct StepTally {
    float f[QS_PLAN_FEATURES] = {};
};

void tally_op(const DevOp &op, float *f)
{
    const double act = std::ldexp(1.0, -(popc(op.cmask) + popc(op.ocmask)));
    switch (op.type) {
    case OP_DENSE:
        f[22] += 1;
        f[23] += float(1u << op.k);
        f[26] += float(4.0 * double(1u << op.k) * act);
        f[27] = std::max(f[27], float(op.k));
        if (op.cmask | op.ocmask) f[25] += 1;
        break;
    case OP_DIAG:
        f[24] += 1;
        f[26] += 4.f;
        break;
    case OP_PHASE:
        f[24] += 1;
        f[26] += float(4.0 * act);
        break;
    default:  // PERMX / SWAP
        f[24] += 1;
        if (op.cmask | op.ocmask) f[25] += 1;
        break;
    }
}

void tally_sub(const DevSub &sb, float *f)
{
    const double act = std::ldexp(1.0, -(popc(sb.scm) + popc(sb.lcm) + popc(sb.ocm)));
    const bool ctl = (sb.scm | sb.lcm | sb.ocm) != 0;
    f[15] += 1;
    switch (sb.type) {
    case SB_G1:
        f[16] += 1;
        f[26] += float(8.0 * act);
        f[27] = std::max(f[27], 1.f);
        if (ctl) f[25] += 1;
        break;
    case SB_G1R:
        f[17] += 1;
        f[26] += float(4.0 * act);
        f[27] = std::max(f[27], 1.f);
        if (ctl) f[25] += 1;
        break;
    case SB_G1N:
    case SB_G1A:
    case SB_G1NM:
    case SB_G1AM:
        f[17] += 1;
        f[26] += float(2.0 * act);
        f[27] = std::max(f[27], 1.f);
        break;
    case SB_G2:
        f[18] += 1;
        f[26] += float(16.0 * act);
        f[27] = std::max(f[27], 2.f);
        if (ctl) f[25] += 1;
        break;
    case SB_PHASE:
        f[19] += 1;
        f[26] += float(4.0 * act);
        break;
    case SB_DIAG:
        f[20] += 1;
        f[26] += float(4.0 * act);
        break;
    default:  // SB_X, SB_SWAP
        f[21] += 1;
        if (ctl) f[25] += 1;
        break;
    }
}

}  // namespace

void plan_features(const Plan &p, std::vector<float> &rows)
{
    const int rb = p.stage_bits > 0 ? p.stage_bits : (p.dt == QS_C64 ? kStageBitsC64 : kStageBitsC128);
    for (const Step &s : p.steps) {
        StepTally t;
        float *f = t.f;
        f[0] = float(p.n);
        f[1] = p.dt == QS_C128 ? 1.f : 0.f;
        f[12] = float(rb);
        switch (s.kind) {
        case S_PASS:
        case S_REMAP: {
            const DevPass &P = p.passes[s.index];
            f[s.kind == S_PASS ? 2 : 3] = 1;
            f[6] = float(P.b);
            f[7] = float(P.lo);
            f[8] = float(P.nhi);
            f[9] = P.has_perm ? 1.f : 0.f;
            if (P.nhi > 0) {
                f[10] = float(P.hipos[0]);
                f[11] = float(P.hipos[P.nhi - 1]);
            }
            for (int o = P.op_begin; o < P.op_end; ++o) {
                const DevOp &op = p.ops[o];
                f[13] += 1;
                if (op.type == OP_STAGE) {
                    const DevStage &st = p.stages[op.mat];
                    f[14] += 1;
                    for (int j = st.sub_begin; j < st.sub_end; ++j) tally_sub(p.subs[j], f);
                } else {
                    tally_op(op, f);
                }
            }
            break;
        }
        case S_UNBLOCKED: {
            const DevOp &op = p.ops[s.index];
            f[4] = 1;
            f[6] = float(op.k);
            f[13] = 1;
            tally_op(op, f);
            break;
        }
        case S_TC:
            f[5] = 1;
            f[6] = float(kTcSlabBits);
            f[27] = float(p.tcs[s.index].width);
            break;
        }
        rows.insert(rows.end(), f, f + QS_PLAN_FEATURES);
    }
}

int learned_choose(const std::vector<CGate> &gates, int n, qs_dtype dt, const qs_options &opt, qs_model *model,
                   Plan &greedy, Plan &best, LearnedMeta &meta, std::string &err)
{
    meta = LearnedMeta{};
    int rc = build_plan(gates, n, dt, opt, greedy, err);
    if (rc) return rc;
    meta.chosen = -1;
    if (!model || opt.tc != QS_TC_OFF || !opt.blocking || model_nfeat(model) != QS_PLAN_FEATURES) return QS_OK;

    // candidate grid
    const int bmax = std::min(max_slab_bits(dt), n);
    const int rbmax = dt == QS_C64 ? kStageBitsC64 : kStageBitsC128;
    struct Fuse {
        int width, force;
    };
    const Fuse fuses[] = {{1, 0}, {2, 0}, {3, 1}, {4, 1}, {5, 1}};
    std::vector<qs_options> cand;
    const int merges[] = {6, 8, 10};  // stage-table condition bits
    for (int eu = 1; eu <= 2; ++eu)
        for (const Fuse &fz : fuses)
            for (int sb = std::max(bmax - 2, 6); sb <= bmax; ++sb)
                for (int rb = rbmax - 1; rb <= rbmax; ++rb)
                    for (int mb : merges) {
                        qs_options o = opt;
                        o.planner = QS_PLANNER_GREEDY;
                        o.fuse_width = fz.width;
                        o.fuse_force = fz.force;
                        o.slab_bits = sb;
                        o.stage_bits = rb;
                        o.slab_mode = QS_SLAB_GATHER;
                        o.euler = eu;
                        o.merge_bits = mb;
                        cand.push_back(o);
                    }
    const size_t nc = cand.size();
    std::vector<Plan> plans(nc);
    std::vector<int> ok(nc, 0);
    {
        const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (unsigned w = 0; w < hw; ++w)
            pool.emplace_back([&, w]() {
                for (size_t c = w; c < nc; c += hw) {
                    std::string e;
                    try {
                        ok[c] = build_plan(gates, n, dt, cand[c], plans[c], e) == QS_OK;
                    } catch (...) {
                        ok[c] = 0;
                    }
                }
            });
        for (auto &t : pool) t.join();
    }
    // features; candidates whose step features equal an earlier one's are the same plan
    std::vector<float> rows;
    std::vector<size_t> first_row, nsteps;
    std::vector<int> cidx;  // -1 = greedy
    std::vector<std::vector<float>> seen;
    auto add = [&](const Plan &p, int c) {
        std::vector<float> r;
        plan_features(p, r);
        for (const auto &s : seen)
            if (s == r) return;
        seen.push_back(r);
        first_row.push_back(rows.size() / QS_PLAN_FEATURES);
        nsteps.push_back(r.size() / QS_PLAN_FEATURES);
        cidx.push_back(c);
        rows.insert(rows.end(), r.begin(), r.end());
    };
    add(greedy, -1);
    for (size_t c = 0; c < nc; ++c)
        if (ok[c]) add(plans[c], (int)c);
    meta.candidates = (int)cidx.size();
    const size_t nrows = rows.size() / QS_PLAN_FEATURES;
    std::vector<float> y(nrows);
    rc = model_predict(model, rows.data(), nrows, y.data(), err);
    if (rc) return rc;
    const double scale = std::ldexp(1.0, n - 20);
    std::vector<double> total(cidx.size(), 0.0);
    for (size_t k = 0; k < cidx.size(); ++k)
        for (size_t s = 0; s < nsteps[k]; ++s) total[k] += std::exp(double(y[first_row[k] + s])) * scale;
    meta.greedy_ms = total[0];
    size_t arg = 0;
    for (size_t k = 1; k < total.size(); ++k)
        if (total[k] < total[arg]) arg = k;
    meta.predicted_ms = total[0];
    // the judge (two timed applies) protects against a wrong pick, so a 2 % predicted margin
    // suffices
    if (arg != 0 && total[arg] < 0.98 * total[0]) {
        meta.chosen = cidx[arg];
        meta.predicted_ms = total[arg];
        best = std::move(plans[cidx[arg]]);
    }
    return QS_OK;
}

}  // namespace qs
