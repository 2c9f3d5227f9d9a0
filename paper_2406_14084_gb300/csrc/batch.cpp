// batch.cpp -- host side of the batched persistent launch (qs_batch_* in include/qs.h).
//
// Every circuit is planned with the regular planner (gather slabs, register stages); the
// plans are concatenated into one device buffer with their indices rebased, and the work items
// are listed round by round (all circuits' pass 0, then pass 1, ...), the order the persistent
// kernel's queue hands them out.  A run zeroes the done counters, the queue head and the
// results, launches the kernel once, and reads the per-circuit results back; with
// options.graph the three memsets and the launch are captured once into a CUDA graph and
// replayed.  The autotuner rebuilds the plans for each (slab bits, stage width) candidate,
// times the runs with CUDA events and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "planner.h"
#include "qs_internal.h"

using namespace qs;

namespace qs {
qs_status set_error(qs_status st, const std::string &msg);  // api.cpp
}

struct qs_batch {
    int ncirc = 0;
    qs_dtype dt = QS_C64;
    qs_options opt{};
    std::vector<int> n;
    std::vector<std::vector<CGate>> gates;
    // current build
    int slab_bits = 0, stage_bits = 0, b_max = 0, rounds = 0;
    std::vector<Plan> plans;
    std::vector<BatchCirc> circs;
    std::vector<BatchItem> items;
    unsigned ndone = 0;
    // device memory
    void *states = nullptr;
    size_t state_bytes = 0;
    size_t plan_bytes = 0;
    void *buf = nullptr;  // plan arrays, circuits, items
    BatchArgs args{};
    void *terms_buf = nullptr;
    size_t terms_cap = 0;
    std::vector<BatchTerm> terms_host;
    std::vector<uint64_t> term_key;
    void *ctl = nullptr;  // done counters, head, results
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = 0.0;

    void free_build()
    {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        if (buf) cudaFree(buf);
        buf = nullptr;
        if (ctl) cudaFree(ctl);
        ctl = nullptr;
    }
    ~qs_batch()
    {
        if (stream) cudaStreamSynchronize(stream);
        free_build();
        if (terms_buf) cudaFree(terms_buf);
        if (states) cudaFree(states);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

qs_status cuda_err(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return QS_OK;
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

size_t amp_size(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

template <typename T>
size_t put(std::vector<unsigned char> &h, const std::vector<T> &v)
{
    const size_t off = (h.size() + 255) & ~size_t(255);
    h.resize(off + std::max<size_t>(16, v.size() * sizeof(T)), 0);
    if (!v.empty()) std::memcpy(h.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

// Plan every circuit for the given slab / stage widths and upload the concatenated arrays.
qs_status build(qs_batch *B, int slab_bits, int stage_bits)
{
    B->free_build();
    B->plans.clear();
    B->plans.resize(B->ncirc);
    qs_options o = B->opt;
    o.dtype = B->dt;
    o.slab_bits = slab_bits;
    o.stage_bits = stage_bits;
    o.blocking = 1;
    o.slab_mode = QS_SLAB_GATHER;
    o.tc = QS_TC_OFF;
    std::vector<DevPass> passes;
    std::vector<DevOp> ops;
    std::vector<DevStage> stages;
    std::vector<DevSub> subs;
    std::vector<cd> coef;
    B->circs.assign(B->ncirc, BatchCirc{});
    B->items.clear();
    uint64_t amp_off = 0;
    unsigned done0 = 0;
    int bmax = 0, rounds = 0;
    for (int c = 0; c < B->ncirc; ++c) {
        Plan &p = B->plans[c];
        std::string err;
        int rc = build_plan(B->gates[c], B->n[c], B->dt, o, p, err);
        if (rc) return set_error((qs_status)rc, "circuit " + std::to_string(c) + ": " + err);
        for (const Step &s : p.steps)
            if (s.kind != S_PASS)
                return set_error(QS_EUNSUPPORTED, "circuit " + std::to_string(c) +
                                                      ": batched circuits need slab passes only");
        if (p.steps.empty()) {
            // a circuit without gates still needs one pass to prepare |0..0> and read out
            DevPass P;
            std::memset(&P, 0, sizeof P);
            P.b = std::min(B->n[c], slab_bits);
            P.lo = std::min(default_seg_bits(B->dt), P.b);
            P.nhi = P.b - P.lo;
            for (int j = 0; j < P.nhi; ++j) P.hipos[j] = (uint8_t)(P.lo + j);
            p.passes.push_back(P);
            p.steps.push_back({S_PASS, 0});
            p.final_phys_of.resize(B->n[c]);
            for (int q = 0; q < B->n[c]; ++q) p.final_phys_of[q] = q;
        }
        BatchCirc &C = B->circs[c];
        C.amp_off = amp_off;
        C.n = B->n[c];
        C.npass = (int)p.steps.size();
        C.pass0 = (int)passes.size();
        C.done0 = (int)done0;
        const int b = p.passes[p.steps[0].index].b;
        C.nslab_log = B->n[c] - b;
        bmax = std::max(bmax, b);
        rounds = std::max(rounds, C.npass);
        const int op_base = (int)ops.size(), st_base = (int)stages.size(), sb_base = (int)subs.size();
        const uint32_t cf_base = (uint32_t)coef.size();
        for (const Step &s : p.steps) {
            DevPass P = p.passes[s.index];
            P.op_begin += op_base;
            P.op_end += op_base;
            passes.push_back(P);
        }
        for (DevOp op : p.ops) {
            if (op.type == OP_STAGE) op.mat += (uint32_t)st_base;
            else op.mat += cf_base;
            ops.push_back(op);
        }
        for (DevStage st : p.stages) {
            st.sub_begin += sb_base;
            st.sub_end += sb_base;
            stages.push_back(st);
        }
        for (DevSub sb : p.subs) {
            sb.mat += cf_base;
            subs.push_back(sb);
        }
        coef.insert(coef.end(), p.coef.begin(), p.coef.end());
        amp_off += uint64_t(1) << B->n[c];
        done0 += (unsigned)C.npass;
    }
    // Work items: runs of consecutive slabs of one pass of one circuit, listed round by round.
    // A CTA walks the slabs of a run with its own double buffering, so the queue is read once per
    // run; runs of up to 8 slabs keep at least 256 items per pass of the largest circuits.
    for (int r = 0; r < rounds; ++r)
        for (int c = 0; c < B->ncirc; ++c)
            if (B->circs[c].npass > r) {
                const uint32_t ns = 1u << B->circs[c].nslab_log;
                const uint32_t run = std::max(1u, std::min(8u, ns / 256u));
                for (uint32_t sl = 0; sl < ns; sl += run)
                    B->items.push_back(BatchItem{c, r, sl, (int32_t)std::min(run, ns - sl)});
            }
    B->slab_bits = slab_bits;
    B->stage_bits = B->plans.empty() ? stage_bits : B->plans[0].stage_bits;
    B->b_max = bmax;
    B->rounds = rounds;
    B->ndone = done0;
    // coefficients in the state precision
    std::vector<unsigned char> h;
    const size_t o_pass = put(h, passes), o_ops = put(h, ops), o_st = put(h, stages), o_sb = put(h, subs);
    const size_t o_circ = put(h, B->circs), o_item = put(h, B->items);
    const size_t o_coef = (h.size() + 255) & ~size_t(255);
    // two spare entries: the register stages read a sub-op's first two coefficients ahead
    h.resize(o_coef + (coef.size() + 2) * amp_size(B->dt), 0);
    for (size_t i = 0; i < coef.size(); ++i) {
        if (B->dt == QS_C64) {
            float *f = reinterpret_cast<float *>(h.data() + o_coef) + 2 * i;
            f[0] = (float)coef[i].real();
            f[1] = (float)coef[i].imag();
        } else {
            double *f = reinterpret_cast<double *>(h.data() + o_coef) + 2 * i;
            f[0] = coef[i].real();
            f[1] = coef[i].imag();
        }
    }
    qs_status st = cuda_err(cudaMalloc(&B->buf, h.size()), "batch plan allocation");
    if (st) return st;
    st = cuda_err(cudaMemcpy(B->buf, h.data(), h.size(), cudaMemcpyHostToDevice), "batch plan upload");
    if (st) return st;
    B->plan_bytes = h.size();
    const size_t ctl_bytes = ((size_t(B->ndone) + 1) * sizeof(unsigned) + 255) / 256 * 256 + B->ncirc * sizeof(double);
    st = cuda_err(cudaMalloc(&B->ctl, ctl_bytes), "batch control allocation");
    if (st) return st;
    char *base = static_cast<char *>(B->buf);
    BatchArgs &a = B->args;
    a.circs = reinterpret_cast<const BatchCirc *>(base + o_circ);
    a.items = reinterpret_cast<const BatchItem *>(base + o_item);
    a.nitems = (unsigned)B->items.size();
    a.passes = reinterpret_cast<const DevPass *>(base + o_pass);
    a.ops = reinterpret_cast<const DevOp *>(base + o_ops);
    a.stages = reinterpret_cast<const DevStage *>(base + o_st);
    a.subs = reinterpret_cast<const DevSub *>(base + o_sb);
    a.coef = base + o_coef;
    a.done = static_cast<unsigned *>(B->ctl);
    a.head = a.done + B->ndone;
    a.results = reinterpret_cast<double *>(static_cast<char *>(B->ctl) +
                                           ((size_t(B->ndone) + 1) * sizeof(unsigned) + 255) / 256 * 256);
    a.status = device_status_ptr();
    a.terms = nullptr;
    B->term_key.clear();  // terms must be re-mapped through the new layouts
    return QS_OK;
}

// Map the Z terms of each circuit to physical masks (through its plan's final layout).
qs_status set_terms(qs_batch *B, const qs_pauli_term *terms, size_t nterms)
{
    std::vector<uint64_t> key;
    for (size_t t = 0; t < nterms; ++t) {
        if (terms[t].xmask != 0) return set_error(QS_EUNSUPPORTED, "batched expectations take Z strings only");
        if (!std::isfinite(terms[t].coeff)) return set_error(QS_EINVAL, "non-finite coefficient");
        uint64_t cbits;
        std::memcpy(&cbits, &terms[t].coeff, 8);
        key.push_back(terms[t].zmask);
        key.push_back(cbits);
    }
    if (key == B->term_key && B->args.terms) return QS_OK;
    B->terms_host.clear();
    for (int c = 0; c < B->ncirc; ++c) {
        BatchCirc &C = B->circs[c];
        C.term0 = (int)B->terms_host.size();
        const std::vector<int> &ph = B->plans[c].final_phys_of;
        for (size_t t = 0; t < nterms; ++t) {
            if (B->n[c] < 64 && (terms[t].zmask >> B->n[c])) continue;
            uint64_t m = 0;
            for (int q = 0; q < B->n[c]; ++q)
                if (terms[t].zmask >> q & 1) m |= 1ull << ph[q];
            B->terms_host.push_back(BatchTerm{m, terms[t].coeff});
        }
        C.nterm = (int)B->terms_host.size() - C.term0;
    }
    const size_t bytes = std::max<size_t>(16, B->terms_host.size() * sizeof(BatchTerm));
    if (bytes > B->terms_cap) {
        if (B->terms_buf) cudaFree(B->terms_buf);
        B->terms_buf = nullptr;
        qs_status st = cuda_err(cudaMalloc(&B->terms_buf, bytes), "batch term allocation");
        if (st) return st;
        B->terms_cap = bytes;
    }
    qs_status st = cuda_err(cudaMemcpy(B->terms_buf, B->terms_host.data(), B->terms_host.size() * sizeof(BatchTerm),
                                       cudaMemcpyHostToDevice),
                            "batch term upload");
    if (st) return st;
    // circuit table carries the term ranges
    st = cuda_err(cudaMemcpy(const_cast<BatchCirc *>(B->args.circs), B->circs.data(),
                             B->circs.size() * sizeof(BatchCirc), cudaMemcpyHostToDevice),
                  "batch circuit upload");
    if (st) return st;
    B->args.terms = static_cast<const BatchTerm *>(B->terms_buf);
    B->term_key = key;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return QS_OK;
}

qs_status enqueue(qs_batch *B)
{
    char err[256] = {0};
    const size_t cnt_bytes = (size_t(B->ndone) + 1) * sizeof(unsigned);
    qs_status st = cuda_err(cudaMemsetAsync(B->args.done, 0, cnt_bytes, B->stream), "batch counter reset");
    if (st) return st;
    st = cuda_err(cudaMemsetAsync(B->args.results, 0, B->ncirc * sizeof(double), B->stream), "batch result reset");
    if (st) return st;
    const int rc = launch_batch(B->dt, B->stage_bits, B->states, B->args, B->b_max, B->stream, err, sizeof err);
    return rc ? set_error((qs_status)rc, err) : QS_OK;
}

qs_status run(qs_batch *B, double *host_out)
{
    cudaEventRecord(B->ev0, B->stream);
    if (B->opt.graph) {
        if (!B->graph) {
            cudaGraph_t g = nullptr;
            qs_status st = cuda_err(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal),
                                    "graph capture begin");
            if (st) return st;
            st = enqueue(B);
            cudaError_t e = cudaStreamEndCapture(B->stream, &g);
            if (st) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            st = cuda_err(e, "graph capture end");
            if (st) return st;
            st = cuda_err(cudaGraphInstantiate(&B->graph, g, 0), "graph instantiate");
            cudaGraphDestroy(g);
            if (st) return st;
        }
        qs_status st = cuda_err(cudaGraphLaunch(B->graph, B->stream), "graph launch");
        if (st) return st;
    } else {
        qs_status st = enqueue(B);
        if (st) return st;
    }
    cudaEventRecord(B->ev1, B->stream);
    qs_status st = cuda_err(cudaStreamSynchronize(B->stream), "batch run");
    if (st) return st;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, B->ev0, B->ev1);
    B->last_ms = ms;
    int status = 0;
    if (read_device_status((void *)B->stream, &status) != QS_OK) return set_error(QS_ECUDA, "status read failed");
    if (status == QS_ETIMEOUT) return set_error(QS_ETIMEOUT, "a batched dependency wait ran out; results are invalid");
    if (host_out)
        return cuda_err(cudaMemcpy(host_out, B->args.results, B->ncirc * sizeof(double), cudaMemcpyDeviceToHost),
                        "batch result readback");
    return QS_OK;
}

}  // namespace

#define QS_GUARD_BEGIN try {
#define QS_GUARD_END                                                                             \
    }                                                                                            \
    catch (const std::bad_alloc &) { return set_error(QS_ENOMEM, "host allocation failed"); }    \
    catch (const std::exception &e) { return set_error(QS_EINVAL, e.what()); }                   \
    catch (...) { return set_error(QS_EINVAL, "unknown error"); }

extern "C" {

qs_status qs_batch_create(int ncirc, const int *n, const qs_gate *const *gates, const size_t *ngates,
                          const qs_options *o, qs_batch **out)
{
    QS_GUARD_BEGIN
    if (!out || !n || (ncirc > 0 && (!gates || !ngates)) || ncirc < 1) return set_error(QS_EINVAL, "bad argument");
    qs_options opt;
    if (o) opt = *o;
    else qs_options_default(&opt);
    if (opt.dtype != QS_C64 && opt.dtype != QS_C128) return set_error(QS_EINVAL, "bad dtype");
    if (opt.tc != QS_TC_OFF) return set_error(QS_EUNSUPPORTED, "batched circuits run without the tensor-core path");
    std::unique_ptr<qs_batch> B(new qs_batch());
    B->ncirc = ncirc;
    B->dt = (qs_dtype)opt.dtype;
    B->opt = opt;
    B->n.assign(n, n + ncirc);
    B->gates.resize(ncirc);
    size_t total = 0;
    for (int c = 0; c < ncirc; ++c) {
        if (n[c] < 1 || n[c] > 30) return set_error(QS_EINVAL, "batched circuits take 1..30 qubits");
        std::string err;
        int rc = canonicalize(gates[c], ngates[c], n[c], B->gates[c], err);
        if (rc) return set_error((qs_status)rc, "circuit " + std::to_string(c) + ": " + err);
        total += (size_t(1) << n[c]) * amp_size(B->dt);
    }
    qs_status st = cuda_err(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking), "stream create");
    if (st) return st;
    cudaEventCreate(&B->ev0);
    cudaEventCreate(&B->ev1);
    st = cuda_err(cudaMalloc(&B->states, total), "batch state allocation");
    if (st) return st;
    B->state_bytes = total;
    const int smax = max_slab_bits(B->dt);
    const int sb = opt.slab_bits > 0 ? std::min(opt.slab_bits, smax) : smax;
    st = build(B.get(), sb, opt.stage_bits);
    if (st) return st;
    *out = B.release();
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_apply_batch(qs_batch *b, const qs_pauli_term *terms, size_t nterms, double *host_out)
{
    QS_GUARD_BEGIN
    if (!b || !host_out || (nterms && !terms)) return set_error(QS_EINVAL, "NULL argument");
    qs_status st = set_terms(b, terms, nterms);
    if (st) return st;
    return run(b, host_out);
    QS_GUARD_END
}

qs_status qs_batch_tune(qs_batch *b, const qs_pauli_term *terms, size_t nterms, int *chosen_slab_bits)
{
    QS_GUARD_BEGIN
    if (!b || (nterms && !terms)) return set_error(QS_EINVAL, "NULL argument");
    const int smax = max_slab_bits(b->dt);
    const int def_rb = b->dt == QS_C64 ? kStageBitsC64 : kStageBitsC128;
    double best = 1e300;
    int best_sb = smax, best_rb = def_rb;
    for (int sb = smax - 2; sb <= smax; ++sb)
        for (int rb = def_rb - 1; rb <= def_rb; ++rb) {
            if (sb < rb) continue;
            qs_status st = build(b, sb, rb);
            if (st) return st;
            st = set_terms(b, terms, nterms);
            if (st) return st;
            double t = 1e300;
            for (int rep = 0; rep < 3; ++rep) {
                st = run(b, nullptr);
                if (st) return st;
                if (rep > 0) t = std::min(t, b->last_ms);  // first run warms up
            }
            if (t < best) {
                best = t;
                best_sb = sb;
                best_rb = rb;
            }
        }
    qs_status st = build(b, best_sb, best_rb);
    if (st) return st;
    b->opt.slab_bits = best_sb;
    b->opt.stage_bits = best_rb;
    if (chosen_slab_bits) *chosen_slab_bits = best_sb;
    return set_terms(b, terms, nterms);
    QS_GUARD_END
}

qs_status qs_batch_info_get(const qs_batch *b, qs_batch_info *out)
{
    if (!b || !out) return set_error(QS_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->circuits = b->ncirc;
    out->items = (int32_t)b->items.size();
    out->rounds = b->rounds;
    out->slab_bits = b->slab_bits;
    out->stage_bits = b->stage_bits;
    out->graph = b->opt.graph ? 1 : 0;
    out->state_bytes = (int64_t)b->state_bytes;
    out->last_run_ms = b->last_ms;
    out->plan_bytes = (int64_t)b->plan_bytes;
    return QS_OK;
}

qs_status qs_batch_destroy(qs_batch *b)
{
    QS_GUARD_BEGIN
    delete b;
    return QS_OK;
    QS_GUARD_END
}

}  // extern "C"
