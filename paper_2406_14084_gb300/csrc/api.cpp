// api.cpp -- the extern "C" boundary of libqs.so (declared in include/qs.h).
//
// Every entry point validates its arguments, catches every C++ exception and converts it to
// a qs_status with a thread-local message.  Host-side fault injection for tests: the
// environment variable QS_FAULT=alloc|plan|launch makes the matching step fail with its
// error status before any device work is issued (no GPU fault is ever provoked).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "learned.h"
#include "model.h"
#include "planner.h"
#include "qs_internal.h"

using namespace qs;

namespace {

thread_local std::string g_err;

qs_status fail(qs_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

bool fault(const char *what)
{
    const char *f = std::getenv("QS_FAULT");
    return f && std::strcmp(f, what) == 0;
}

qs_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return QS_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(QS_ENOMEM, std::string(what) + ": out of device memory");
    return fail(QS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t amp_bytes(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

}  // namespace

namespace qs {
// Record an error for qs_last_error (used by the other host translation units).
qs_status set_error(qs_status st, const std::string &msg) { return fail(st, msg); }
}  // namespace qs

namespace {

struct DevPlanBuf {
    void *base = nullptr;
    DevPass *passes = nullptr;
    DevOp *ops = nullptr;
    DevStage *stages = nullptr;
    DevSub *subs = nullptr;
    DevTc *tcs = nullptr;
    unsigned char *images = nullptr;
    void *coef = nullptr;
    void *coef_df = nullptr;  // complex128 plans in double-float form: (h, l) of re, then of im
    int device = -1;
};

}  // namespace

struct qs_state {
    int n = 0;
    qs_dtype dt = QS_C64;
    void *amp = nullptr;
    bool owned = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<int> phys_of;  // logical -> physical
    double *scratch = nullptr;
    size_t scratch_bytes = 0;
    qs_stats_t stats{};
    // profiling: event pairs recorded around launches, folded into stats on qs_stats()
    bool profiling = false;
    struct Timed {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t take_event()
    {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void fold_timings()
    {
        if (pending.empty()) return;
        cudaStreamSynchronize(stream);
        for (const Timed &t : pending) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t.a, t.b);
            switch (t.kind) {
            case 0: stats.pass_ms += ms; break;
            case 1: stats.remap_ms += ms; break;
            case 2: stats.unblocked_ms += ms; break;
            default: stats.tc_ms += ms; break;
            }
            stats.timed_launches++;
            event_pool.push_back(t.a);
            event_pool.push_back(t.b);
        }
        pending.clear();
    }
    ~qs_state()
    {
        for (const Timed &t : pending) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
    }
};

struct qs_plan {
    Plan p;
    DevPlanBuf dev[2];  // per dtype
    // learned planner: the greedy twin (judge), predictions, and the judge's measurements
    std::unique_ptr<qs_plan> alt;
    bool learned = false;
    int candidates = 0, chosen = -1;
    double pred_ms = 0, greedy_pred_ms = 0;
    int judge_state = 2;       // 0: next apply times this plan, 1: times alt, 2: settled
    double judge_ms[2] = {0, 0};
    bool use_alt = false;
    ~qs_plan()
    {
        for (auto &d : dev)
            if (d.base) cudaFree(d.base);
    }
};

namespace {

bool identity_layout(const qs_state *s)
{
    for (int q = 0; q < s->n; ++q)
        if (s->phys_of[q] != q) return false;
    return true;
}

qs_status ensure_scratch(qs_state *s, size_t bytes)
{
    if (s->scratch_bytes >= bytes) return QS_OK;
    if (fault("alloc")) return fail(QS_ENOMEM, "injected allocation failure");
    if (s->scratch) {
        cudaStreamSynchronize(s->stream);
        cudaFree(s->scratch);
        s->scratch = nullptr;
        s->scratch_bytes = 0;
    }
    void *p = nullptr;
    qs_status st = cuda_status(cudaMalloc(&p, bytes), "scratch allocation");
    if (st) return st;
    s->scratch = (double *)p;
    s->scratch_bytes = bytes;
    return QS_OK;
}

qs_status upload(qs_plan *pl, qs_dtype dt)
{
    DevPlanBuf &d = pl->dev[dt];
    int dev = 0;
    cudaGetDevice(&dev);
    if (d.base && d.device == dev) return QS_OK;
    if (d.base) {
        cudaFree(d.base);
        d.base = nullptr;
    }
    const Plan &p = pl->p;
    const size_t np = std::max<size_t>(1, p.passes.size()), no = std::max<size_t>(1, p.ops.size());
    const size_t nc = std::max<size_t>(1, p.coef.size());
    const size_t nst = std::max<size_t>(1, p.stages.size()), nsb = std::max<size_t>(1, p.subs.size());
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_pass = 0, o_ops = al(np * sizeof(DevPass));
    const size_t o_st = o_ops + al(no * sizeof(DevOp)), o_sb = o_st + al(nst * sizeof(DevStage));
    const size_t ntc = std::max<size_t>(1, p.tcs.size()), nim = std::max<size_t>(16, p.tc_images.size());
    const size_t o_tc = o_sb + al(nsb * sizeof(DevSub)), o_im = o_tc + al(ntc * sizeof(DevTc));
    const size_t o_coef = o_im + al(nim);
    // two spare entries: the register stages read a sub-op's first two coefficients ahead
    const bool want_df = dt == QS_C128 && p.opt.arith == QS_ARITH_DF;
    const size_t o_cdf = o_coef + al((nc + 2) * amp_bytes(dt));
    const size_t total = o_cdf + (want_df ? al((nc + 2) * 16) : 0);
    std::vector<unsigned char> h(total, 0);
    if (!p.passes.empty()) std::memcpy(h.data() + o_pass, p.passes.data(), p.passes.size() * sizeof(DevPass));
    if (!p.ops.empty()) std::memcpy(h.data() + o_ops, p.ops.data(), p.ops.size() * sizeof(DevOp));
    if (!p.stages.empty()) std::memcpy(h.data() + o_st, p.stages.data(), p.stages.size() * sizeof(DevStage));
    if (!p.subs.empty()) std::memcpy(h.data() + o_sb, p.subs.data(), p.subs.size() * sizeof(DevSub));
    if (!p.tcs.empty()) std::memcpy(h.data() + o_tc, p.tcs.data(), p.tcs.size() * sizeof(DevTc));
    if (!p.tc_images.empty()) std::memcpy(h.data() + o_im, p.tc_images.data(), p.tc_images.size());
    if (dt == QS_C64) {
        float *f = reinterpret_cast<float *>(h.data() + o_coef);
        for (size_t i = 0; i < p.coef.size(); ++i) {
            f[2 * i] = (float)p.coef[i].real();
            f[2 * i + 1] = (float)p.coef[i].imag();
        }
    } else {
        double *f = reinterpret_cast<double *>(h.data() + o_coef);
        for (size_t i = 0; i < p.coef.size(); ++i) {
            f[2 * i] = p.coef[i].real();
            f[2 * i + 1] = p.coef[i].imag();
        }
    }
    if (want_df) {
        // each FP64 part x as h = fl32(x), l = fl32(x - h): h + l carries about 48 bits of x
        float *f = reinterpret_cast<float *>(h.data() + o_cdf);
        for (size_t i = 0; i < p.coef.size(); ++i) {
            const double parts[2] = {p.coef[i].real(), p.coef[i].imag()};
            for (int r = 0; r < 2; ++r) {
                const float hi = (float)parts[r];
                f[4 * i + 2 * r] = hi;
                f[4 * i + 2 * r + 1] = (float)(parts[r] - (double)hi);
            }
        }
    }
    if (fault("alloc")) return fail(QS_ENOMEM, "injected allocation failure");
    void *base = nullptr;
    qs_status st = cuda_status(cudaMalloc(&base, total), "plan upload allocation");
    if (st) return st;
    st = cuda_status(cudaMemcpy(base, h.data(), total, cudaMemcpyHostToDevice), "plan upload");
    if (st) {
        cudaFree(base);
        return st;
    }
    d.base = base;
    d.device = dev;
    d.passes = reinterpret_cast<DevPass *>((char *)base + o_pass);
    d.ops = reinterpret_cast<DevOp *>((char *)base + o_ops);
    d.stages = reinterpret_cast<DevStage *>((char *)base + o_st);
    d.subs = reinterpret_cast<DevSub *>((char *)base + o_sb);
    d.tcs = reinterpret_cast<DevTc *>((char *)base + o_tc);
    d.images = reinterpret_cast<unsigned char *>((char *)base + o_im);
    d.coef = (char *)base + o_coef;
    d.coef_df = want_df ? (char *)base + o_cdf : nullptr;
    return QS_OK;
}

// Synchronise the state's stream and report a bounded device-side wait that ran out.
qs_status check_device(qs_state *s)
{
    int status = 0;
    if (read_device_status((void *)s->stream, &status) != QS_OK)
        return fail(QS_ECUDA, "reading the device status word failed");
    if (status == QS_ETIMEOUT)
        return fail(QS_ETIMEOUT, "a device-side wait ran out of its iteration budget; results are not valid");
    return QS_OK;
}

// Per-launch event pairs for qs_plan_profile and the learned planner's judge.
struct StepTimer {
    std::vector<cudaEvent_t> ev;  // ev[i] recorded before step i; ev.back() after the last
    ~StepTimer()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    void mark(cudaStream_t s)
    {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev.push_back(e);
    }
    float between(size_t i, size_t j) const
    {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[i], ev[j]);
        return ms;
    }
};

qs_status run_plan(qs_state *s, qs_plan *pl, StepTimer *timer = nullptr)
{
    if (fault("launch")) return fail(QS_ECUDA, "injected launch failure");
    qs_status st = upload(pl, s->dt);
    if (st) return st;
    const DevPlanBuf &d = pl->dev[s->dt];
    const Plan &p = pl->p;
    LaunchCtx c{s->amp, s->n, s->dt, (void *)s->stream};
    char err[256] = {0};
    const int64_t pass_bytes = int64_t(2) * (int64_t(1) << s->n) * (int64_t)amp_bytes(s->dt);
    if (timer) timer->mark(s->stream);
    for (const Step &stp : p.steps) {
        int rc = QS_OK;
        cudaEvent_t ev0 = nullptr;
        if (s->profiling) {
            ev0 = s->take_event();
            cudaEventRecord(ev0, s->stream);
        }
        switch (stp.kind) {
        case S_PASS:
        case S_REMAP: {
            const DevPass &hp = p.passes[stp.index];
            const int rb = p.stage_bits > 0 ? p.stage_bits : (s->dt == QS_C64 ? kStageBitsC64 : kStageBitsC128);
            // double-float form: complex128, requested, and a pass of register stages only
            bool df = d.coef_df != nullptr && stp.kind == S_PASS && !hp.has_perm;
            for (int o = hp.op_begin; df && o < hp.op_end; ++o) df = p.ops[o].type == OP_STAGE;
            const PassArgs pa{d.passes + stp.index, d.ops, d.stages, d.subs, d.coef, rb, d.coef_df, df};
            rc = launch_pass(c, pa, hp, err, sizeof err);
            if (stp.kind == S_PASS) s->stats.passes++;
            else s->stats.remaps++;
            s->stats.bytes_moved += pass_bytes;
            break;
        }
        case S_UNBLOCKED:
            rc = launch_unblocked(c, d.ops + stp.index, p.ops[stp.index], d.coef, err, sizeof err);
            s->stats.unblocked++;
            s->stats.bytes_moved += pass_bytes;
            break;
        case S_TC:
            rc = launch_tc(c, d.tcs + stp.index, p.tcs[stp.index], d.images, err, sizeof err);
            s->stats.tc_gates++;
            s->stats.bytes_moved += pass_bytes;
            break;
        }
        if (s->profiling) {
            cudaEvent_t ev1 = s->take_event();
            cudaEventRecord(ev1, s->stream);
            const int kind = stp.kind == S_PASS ? 0 : stp.kind == S_REMAP ? 1 : stp.kind == S_UNBLOCKED ? 2 : 3;
            s->pending.push_back({ev0, ev1, kind});
            if (s->pending.size() > 4096) s->fold_timings();
        }
        if (rc) return fail((qs_status)rc, err);
        if (timer) timer->mark(s->stream);
    }
    s->stats.plans_applied++;
    return QS_OK;
}

qs_status canonicalize_state(qs_state *s)
{
    if (identity_layout(s)) return QS_OK;
    std::unique_ptr<qs_plan> pl(new qs_plan());
    pl->p.n = s->n;
    pl->p.dt = s->dt;
    plan_canonicalize(s->n, s->dt, s->phys_of, pl->p);
    qs_status st = run_plan(s, pl.get());
    if (st) return st;
    // plan buffers are freed by the destructor; wait so the free cannot race the kernels
    cudaStreamSynchronize(s->stream);
    for (int q = 0; q < s->n; ++q) s->phys_of[q] = q;
    return QS_OK;
}

// Learned planner: greedy plan plus, when the model predicts a faster candidate, that
// candidate with the greedy plan attached as its judge.
qs_status fuse_learned(const std::vector<CGate> &cg, int n, const qs_options &opt, qs_model *model, qs_plan **out)
{
    std::unique_ptr<qs_plan> greedy(new qs_plan()), best(new qs_plan());
    LearnedMeta meta;
    std::string err;
    qs_options gopt = opt;
    gopt.planner = QS_PLANNER_GREEDY;
    int rc = learned_choose(cg, n, (qs_dtype)opt.dtype, gopt, model, greedy->p, best->p, meta, err);
    if (rc) return fail((qs_status)rc, err);
    qs_plan *res;
    if (meta.chosen >= 0) {
        best->alt = std::move(greedy);
        best->judge_state = 0;
        res = best.release();
    } else {
        res = greedy.release();
    }
    res->learned = model != nullptr;
    res->candidates = meta.candidates;
    res->chosen = meta.chosen;
    res->pred_ms = meta.predicted_ms;
    res->greedy_pred_ms = meta.greedy_ms;
    *out = res;
    return QS_OK;
}

#define QS_GUARD_BEGIN try {
#define QS_GUARD_END                                                              \
    }                                                                             \
    catch (const std::bad_alloc &) { return fail(QS_ENOMEM, "host allocation failed"); } \
    catch (const std::exception &e) { return fail(QS_EINVAL, e.what()); }         \
    catch (...) { return fail(QS_EINVAL, "unknown error"); }

}  // namespace

extern "C" {

const char *qs_last_error(void) { return g_err.c_str(); }

const char *qs_version(void) { return "qs-gb300 0.1 (sm_103a)"; }

void qs_options_default(qs_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->fuse_width = 2;
    o->blocking = 1;
    o->slab_bits = 0;
    o->seg_bits = 0;
    o->slab_mode = QS_SLAB_GATHER;
    o->planner = QS_PLANNER_GREEDY;
    o->tc = QS_TC_OFF;
    o->tc_width = 6;
    o->graph = 0;
    o->diag_bits = 0;
    o->dtype = QS_C64;
}

qs_status qs_create_from_buffer(int n, qs_dtype dt, void *dev, void *stream, qs_state **out)
{
    QS_GUARD_BEGIN
    g_err.clear();
    if (!out) return fail(QS_EINVAL, "out is NULL");
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "n must be in [1, 36]");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    if (!dev || (reinterpret_cast<uintptr_t>(dev) & 255)) return fail(QS_EINVAL, "buffer must be non-NULL and 256-byte aligned");
    std::unique_ptr<qs_state> s(new qs_state());
    s->n = n;
    s->dt = dt;
    s->amp = dev;
    s->owned = false;
    s->stream = (cudaStream_t)stream;
    cudaGetDevice(&s->device);
    s->phys_of.resize(n);
    for (int q = 0; q < n; ++q) s->phys_of[q] = q;
    *out = s.release();
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_create(int n, qs_dtype dt, qs_state **out)
{
    QS_GUARD_BEGIN
    g_err.clear();
    if (!out) return fail(QS_EINVAL, "out is NULL");
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "n must be in [1, 36]");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    if (fault("alloc")) return fail(QS_ENOMEM, "injected allocation failure");
    const size_t bytes = (size_t(1) << n) * amp_bytes(dt);
    void *p = nullptr;
    qs_status st = cuda_status(cudaMalloc(&p, bytes), "state allocation");
    if (st) return st;
    std::unique_ptr<qs_state> s(new qs_state());
    s->n = n;
    s->dt = dt;
    s->amp = p;
    s->owned = true;
    s->stream = nullptr;
    cudaGetDevice(&s->device);
    s->phys_of.resize(n);
    for (int q = 0; q < n; ++q) s->phys_of[q] = q;
    LaunchCtx c{s->amp, n, dt, nullptr};
    char err[256] = {0};
    int rc = launch_set_basis(c, 0, err, sizeof err);
    if (rc) {
        cudaFree(p);
        return fail((qs_status)rc, err);
    }
    *out = s.release();
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_destroy(qs_state *s)
{
    QS_GUARD_BEGIN
    if (!s) return QS_OK;
    cudaStreamSynchronize(s->stream);
    if (s->owned && s->amp) cudaFree(s->amp);
    if (s->scratch) cudaFree(s->scratch);
    delete s;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_set_stream(qs_state *s, void *stream)
{
    if (!s) return fail(QS_EINVAL, "state is NULL");
    s->stream = (cudaStream_t)stream;
    return QS_OK;
}

qs_status qs_sync(qs_state *s)
{
    if (!s) return fail(QS_EINVAL, "state is NULL");
    qs_status st = cuda_status(cudaStreamSynchronize(s->stream), "synchronize");
    return st ? st : check_device(s);
}

qs_status qs_set_basis(qs_state *s, uint64_t x)
{
    QS_GUARD_BEGIN
    if (!s) return fail(QS_EINVAL, "state is NULL");
    if (s->n < 64 && (x >> s->n)) return fail(QS_EINVAL, "basis index out of range");
    LaunchCtx c{s->amp, s->n, s->dt, (void *)s->stream};
    char err[256] = {0};
    int rc = launch_set_basis(c, x, err, sizeof err);
    if (rc) return fail((qs_status)rc, err);
    for (int q = 0; q < s->n; ++q) s->phys_of[q] = q;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_get_buffer(qs_state *s, void **dev, int *phys_of)
{
    if (!s) return fail(QS_EINVAL, "state is NULL");
    if (dev) *dev = s->amp;
    if (phys_of)
        for (int q = 0; q < s->n; ++q) phys_of[q] = s->phys_of[q];
    return QS_OK;
}

qs_status qs_canonicalize(qs_state *s)
{
    QS_GUARD_BEGIN
    if (!s) return fail(QS_EINVAL, "state is NULL");
    return canonicalize_state(s);
    QS_GUARD_END
}

qs_status qs_copy_to_host(qs_state *s, uint64_t first, uint64_t count, void *host)
{
    QS_GUARD_BEGIN
    if (!s || (!host && count)) return fail(QS_EINVAL, "NULL argument");
    const uint64_t N = 1ull << s->n;
    if (first > N || count > N - first) return fail(QS_EINVAL, "range outside the state");
    qs_status st = canonicalize_state(s);
    if (st) return st;
    const size_t ab = amp_bytes(s->dt);
    st = cuda_status(cudaMemcpyAsync(host, (char *)s->amp + first * ab, count * ab,
                                     cudaMemcpyDeviceToHost, s->stream),
                     "copy to host");
    if (st) return st;
    st = cuda_status(cudaStreamSynchronize(s->stream), "copy to host");
    return st ? st : check_device(s);
    QS_GUARD_END
}

qs_status qs_copy_from_host(qs_state *s, uint64_t first, uint64_t count, const void *host)
{
    QS_GUARD_BEGIN
    if (!s || (!host && count)) return fail(QS_EINVAL, "NULL argument");
    const uint64_t N = 1ull << s->n;
    if (first > N || count > N - first) return fail(QS_EINVAL, "range outside the state");
    qs_status st = canonicalize_state(s);
    if (st) return st;
    const size_t ab = amp_bytes(s->dt);
    st = cuda_status(cudaMemcpyAsync((char *)s->amp + first * ab, host, count * ab,
                                     cudaMemcpyHostToDevice, s->stream),
                     "copy from host");
    if (st) return st;
    return cuda_status(cudaStreamSynchronize(s->stream), "copy from host");
    QS_GUARD_END
}

qs_status qs_fuse(const qs_gate *g, size_t ng, int n, const qs_options *o, qs_plan **out)
{
    QS_GUARD_BEGIN
    g_err.clear();
    if (!out) return fail(QS_EINVAL, "out is NULL");
    if (!g && ng) return fail(QS_EINVAL, "gates is NULL");
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "n must be in [1, 36]");
    if (fault("plan")) return fail(QS_EINVAL, "injected planning failure");
    qs_options opt;
    if (o) opt = *o;
    else qs_options_default(&opt);
    if (opt.fuse_width < 0 || opt.fuse_width > 7 || opt.slab_bits < 0 || opt.slab_bits > kMaxSlabBits ||
        opt.seg_bits < 0 || opt.seg_bits > 8 || opt.merge_bits < 0 || opt.merge_bits > 10 ||
        (opt.arith != QS_ARITH_FP64 && opt.arith != QS_ARITH_DF) ||
        (opt.slab_mode != QS_SLAB_GATHER && opt.slab_mode != QS_SLAB_REMAP) ||
        (opt.tc != QS_TC_OFF && opt.tc != QS_TC_TF32X3 && opt.tc != QS_TC_BF16X3))
        return fail(QS_EINVAL, "option out of range");
    std::vector<CGate> cg;
    std::string err;
    int rc = canonicalize(g, ng, n, cg, err);
    if (rc) return fail((qs_status)rc, err);
    if (opt.dtype != QS_C64 && opt.dtype != QS_C128) return fail(QS_EINVAL, "bad options dtype");
    if (opt.planner == QS_PLANNER_LEARNED) return fuse_learned(cg, n, opt, default_cost_model(), out);
    std::unique_ptr<qs_plan> pl(new qs_plan());
    // A plan can be applied to either precision; opt.dtype selects the cost model it is
    // optimised for (and the slab size, which must fit shared memory at apply time).
    rc = build_plan(cg, n, (qs_dtype)opt.dtype, opt, pl->p, err);
    if (rc) return fail((qs_status)rc, err);
    *out = pl.release();
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_fuse_learned(const qs_gate *g, size_t ng, int n, const qs_options *o, qs_model *model, qs_plan **out)
{
    QS_GUARD_BEGIN
    g_err.clear();
    if (!out) return fail(QS_EINVAL, "out is NULL");
    if (!g && ng) return fail(QS_EINVAL, "gates is NULL");
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "n must be in [1, 36]");
    qs_options opt;
    if (o) opt = *o;
    else qs_options_default(&opt);
    if (opt.fuse_width < 0 || opt.fuse_width > 7 || opt.slab_bits < 0 || opt.slab_bits > kMaxSlabBits ||
        opt.seg_bits < 0 || opt.seg_bits > 8 || opt.merge_bits < 0 || opt.merge_bits > 10 ||
        (opt.arith != QS_ARITH_FP64 && opt.arith != QS_ARITH_DF) ||
        (opt.slab_mode != QS_SLAB_GATHER && opt.slab_mode != QS_SLAB_REMAP) ||
        (opt.tc != QS_TC_OFF && opt.tc != QS_TC_TF32X3 && opt.tc != QS_TC_BF16X3) ||
        (opt.dtype != QS_C64 && opt.dtype != QS_C128))
        return fail(QS_EINVAL, "option out of range");
    std::vector<CGate> cg;
    std::string err;
    int rc = canonicalize(g, ng, n, cg, err);
    if (rc) return fail((qs_status)rc, err);
    return fuse_learned(cg, n, opt, model, out);
    QS_GUARD_END
}

qs_status qs_plan_destroy(qs_plan *p)
{
    QS_GUARD_BEGIN
    if (p) {
        cudaDeviceSynchronize();
        delete p;
    }
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_plan_info_get(const qs_plan *p, qs_plan_info *out)
{
    if (!p || !out) return fail(QS_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->n = p->p.n;
    for (const Step &s : p->p.steps) {
        if (s.kind == S_PASS) out->passes++;
        else if (s.kind == S_REMAP) out->remaps++;
        else if (s.kind == S_UNBLOCKED) out->unblocked++;
        else if (s.kind == S_TC) out->tc_gates++;
    }
    out->ops = p->p.fused_ops;
    out->input_gates = p->p.input_gates;
    out->slab_bits = p->p.slab_bits;
    out->seg_bits = p->p.seg_bits;
    out->flops_per_amp = p->p.flops_per_amp;
    out->device_bytes = (int64_t)(p->p.passes.size() * sizeof(DevPass) + p->p.ops.size() * sizeof(DevOp) +
                                  p->p.stages.size() * sizeof(DevStage) + p->p.subs.size() * sizeof(DevSub) +
                                  p->p.tcs.size() * sizeof(DevTc) + p->p.tc_images.size() +
                                  p->p.coef.size() * 16);
    out->stages = (int32_t)p->p.stages.size();
    out->stage_ops = (int32_t)p->p.subs.size();
    for (const Step &s : p->p.steps)
        if (s.kind == S_PASS) {
            const DevPass &P = p->p.passes[s.index];
            for (int o = P.op_begin; o < P.op_end; ++o)
                if (p->p.ops[o].type != OP_STAGE) out->smem_ops++;
        }
    out->stage_bits = p->p.stage_bits;
    out->learned = p->learned ? 1 : 0;
    out->candidates = p->candidates;
    out->chosen = p->chosen;
    out->judge_state = p->judge_state;
    out->predicted_ms = p->pred_ms;
    out->greedy_predicted_ms = p->greedy_pred_ms;
    out->judge_ms_learned = p->judge_ms[0];
    out->judge_ms_greedy = p->judge_ms[1];
    out->using_greedy = (p->alt && p->use_alt) ? 1 : 0;
    return QS_OK;
}

qs_status qs_plan_dump(const qs_plan *pl, char *buf, size_t cap, size_t *needed)
{
    QS_GUARD_BEGIN
    if (!pl) return fail(QS_EINVAL, "plan is NULL");
    const Plan &p = pl->p;
    std::string out;
    char tmp[64];
    auto num = [&](long long v) {
        snprintf(tmp, sizeof tmp, " %lld", v);
        out += tmp;
    };
    auto cnum = [&](const cd &v) {
        snprintf(tmp, sizeof tmp, " %.17g %.17g", v.real(), v.imag());
        out += tmp;
    };
    out += "N";
    num(p.n);
    out += "\n";
    auto dump_op = [&](const DevOp &op, const int *phys_of_local, bool unblocked) {
        auto P = [&](int l) { return unblocked ? l : phys_of_local[l]; };
        static const char *names[] = {"DENSE", "DIAG", "PERMX", "SWAP", "PHASE"};
        out += "OP ";
        out += names[op.type];
        const int kt = op.type == OP_DIAG ? op.k + op.nout : op.type == OP_PERMX ? 1 : op.type == OP_SWAP ? 2 : op.k;
        num(kt);
        out += " t";
        if (op.type == OP_DIAG) {
            for (int j = 0; j < op.k; ++j) num(P(op.t[j]));
            for (int j = 0; j < op.nout; ++j) num(op.outpos[j]);
        } else {
            for (int j = 0; j < kt; ++j) num(P(op.t[j]));
        }
        out += " c";
        for (int l = 0; l < 64; ++l)
            if (op.cmask >> l & 1) num(P(l));
        for (int l = 0; l < 64; ++l)
            if (op.ocmask >> l & 1) num(l);
        if (op.type == OP_DENSE || op.type == OP_DIAG) {
            out += " m";
            const size_t cnt = op.type == OP_DENSE ? (size_t(1) << (2 * kt)) : (size_t(1) << kt);
            for (size_t e = 0; e < cnt; ++e) cnum(p.coef[op.mat + e]);
        }
        out += "\n";
    };
    for (const Step &s : p.steps) {
        if (s.kind == S_TC) {
            const DevTc &T = p.tcs[s.index];
            out += "PASS";
            num(T.slab.b);
            num(T.slab.lo);
            for (int j = 0; j < T.slab.nhi; ++j) num(T.slab.hipos[j]);
            out += "\nOP DENSE";
            num(T.width);
            out += " t";
            for (int q : p.tc_phys[s.index]) num(q);
            out += " c m";
            for (size_t e = 0; e < (size_t(1) << (2 * T.width)); ++e) cnum(p.coef[p.tc_coef[s.index] + e]);
            out += "\n";
        } else if (s.kind == S_UNBLOCKED) {
            out += "UNBLOCKED\n";
            dump_op(p.ops[s.index], nullptr, true);
        } else if (s.kind == S_PASS || s.kind == S_REMAP) {
            const DevPass &P = p.passes[s.index];
            int phys_of_local[32];
            for (int l = 0; l < P.lo; ++l) phys_of_local[l] = l;
            for (int j = 0; j < P.nhi; ++j) phys_of_local[P.lo + j] = P.hipos[j];
            if (s.kind == S_REMAP) {
                std::vector<int> A, B;
                for (int l = 0; l < P.b; ++l)
                    if (P.perm[l] > l) {
                        A.push_back(phys_of_local[l]);
                        B.push_back(phys_of_local[P.perm[l]]);
                    }
                out += "REMAP";
                num((long long)A.size());
                for (int a : A) num(a);
                for (int b : B) num(b);
                out += "\n";
                continue;
            }
            out += "PASS";
            num(P.b);
            num(P.lo);
            for (int j = 0; j < P.nhi; ++j) num(P.hipos[j]);
            out += "\n";
            for (int o = P.op_begin; o < P.op_end; ++o) {
                if (p.ops[o].type != OP_STAGE) {
                    dump_op(p.ops[o], phys_of_local, false);
                    continue;
                }
                // a register stage: list its sub-ops as ops in physical positions
                const DevStage &st = p.stages[p.ops[o].mat];
                auto reg_phys = [&](int j) { return phys_of_local[st.sbits[j]]; };
                for (int si = st.sub_begin; si < st.sub_end; ++si) {
                    const DevSub &sb = p.subs[si];
                    std::vector<int> ctl;
                    for (int j = 0; j < st.r; ++j)
                        if (sb.scm >> j & 1) ctl.push_back(reg_phys(j));
                    for (int l = 0; l < 32; ++l)
                        if (sb.lcm >> l & 1) ctl.push_back(phys_of_local[l]);
                    for (int q = 0; q < 64; ++q)
                        if (sb.ocm >> q & 1) ctl.push_back(q);
                    auto head = [&](const char *kind, const std::vector<int> &t, const std::vector<int> &c) {
                        out += "OP ";
                        out += kind;
                        num((long long)t.size());
                        out += " t";
                        for (int q : t) num(q);
                        out += " c";
                        for (int q : c) num(q);
                    };
                    switch (sb.type) {
                    case SB_G1:
                    case SB_G1R:
                    case SB_G2: {
                        std::vector<int> t{reg_phys(sb.j0)};
                        if (sb.type == SB_G2) t.push_back(reg_phys(sb.j1));
                        head("DENSE", t, ctl);
                        out += " m";
                        for (size_t e = 0; e < (sb.type == SB_G2 ? 16u : 4u); ++e) cnum(p.coef[sb.mat + e]);
                        break;
                    }
                    case SB_G1N:
                    case SB_G1NM:
                    case SB_G1A:
                    case SB_G1AM: {
                        head("DENSE", {reg_phys(sb.j0)}, ctl);
                        out += " m";
                        const cd x = p.coef[sb.mat], y = p.coef[sb.mat + 1], one(1.0);
                        if (sb.type == SB_G1N || sb.type == SB_G1NM) {
                            cnum(one); cnum(x); cnum(y); cnum(sb.type == SB_G1N ? one : -one);
                        } else {
                            cnum(x); cnum(one); cnum(sb.type == SB_G1A ? one : -one); cnum(y);
                        }
                        break;
                    }
                    case SB_X: head("PERMX", {reg_phys(sb.j0)}, ctl); break;
                    case SB_SWAP: head("SWAP", {reg_phys(sb.j0), reg_phys(sb.j1)}, ctl); break;
                    case SB_PHASE: {
                        if (ctl.empty()) {
                            // a scalar on every element: a diagonal of equal entries on one qubit
                            head("DIAG", {reg_phys(0)}, {});
                            out += " m";
                            cnum(p.coef[sb.mat]);
                            cnum(p.coef[sb.mat]);
                            break;
                        }
                        // controlled phase: diagonal over every masked qubit, 1 except all-ones
                        head("DIAG", ctl, {});
                        out += " m";
                        const size_t D = size_t(1) << ctl.size();
                        for (size_t e = 0; e + 1 < D; ++e) cnum(cd(1.0));
                        cnum(p.coef[sb.mat]);
                        break;
                    }
                    case SB_DIAG: {
                        std::vector<int> t;
                        for (int j = 0; j < st.r; ++j) t.push_back(reg_phys(j));
                        for (int j = 0; j < sb.ndl; ++j)
                            t.push_back(sb.dl[j] & 0x80 ? (sb.dl[j] & 0x7f) : phys_of_local[sb.dl[j]]);
                        head("DIAG", t, {});
                        out += " m";
                        for (size_t e = 0; e < (size_t(1) << t.size()); ++e) cnum(p.coef[sb.mat + e]);
                        break;
                    }
                    }
                    out += "\n";
                }
            }
        }
    }
    out += "LAYOUT";
    for (int q = 0; q < p.n; ++q) num(p.final_phys_of.empty() ? q : p.final_phys_of[q]);
    out += "\n";
    if (needed) *needed = out.size() + 1;
    if (buf && cap) {
        const size_t m = std::min(cap - 1, out.size());
        std::memcpy(buf, out.data(), m);
        buf[m] = 0;
    }
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_apply_plan(qs_state *s, const qs_plan *p)
{
    QS_GUARD_BEGIN
    if (!s || !p) return fail(QS_EINVAL, "NULL argument");
    if (p->p.n != s->n) return fail(QS_EINVAL, "plan and state have different qubit counts");
    if (p->p.dt != s->dt) return fail(QS_EINVAL, "plan was built for the other precision (options.dtype)");
    const int bmax = max_slab_bits(s->dt);
    for (const DevPass &ps : p->p.passes)
        if (ps.b > bmax) return fail(QS_EINVAL, "plan slab too large for this dtype");
    qs_status st = canonicalize_state(s);
    if (st) return st;
    qs_plan *pl = const_cast<qs_plan *>(p);
    if (pl->alt && pl->judge_state < 2) {
        // the judge: time this plan on its first apply and the greedy twin on the second
        qs_plan *run = pl->judge_state == 0 ? pl : pl->alt.get();
        StepTimer timer;
        st = run_plan(s, run, &timer);
        if (st) return st;
        st = cuda_status(cudaEventSynchronize(timer.ev.back()), "judge timing");
        if (st) return st;
        pl->judge_ms[pl->judge_state] = timer.between(0, timer.ev.size() - 1);
        if (++pl->judge_state == 2) pl->use_alt = pl->judge_ms[1] < pl->judge_ms[0];
        s->phys_of = run->p.final_phys_of;
        return QS_OK;
    }
    qs_plan *run = (pl->alt && pl->use_alt) ? pl->alt.get() : pl;
    st = run_plan(s, run);
    if (st) return st;
    s->phys_of = run->p.final_phys_of;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_plan_profile(qs_state *s, const qs_plan *p, float *step_ms, size_t cap)
{
    QS_GUARD_BEGIN
    if (!s || !p || (!step_ms && cap)) return fail(QS_EINVAL, "NULL argument");
    if (p->p.n != s->n) return fail(QS_EINVAL, "plan and state have different qubit counts");
    if (p->p.dt != s->dt) return fail(QS_EINVAL, "plan was built for the other precision (options.dtype)");
    if (cap < p->p.steps.size()) return fail(QS_EINVAL, "step_ms has fewer entries than the plan has steps");
    const int bmax = max_slab_bits(s->dt);
    for (const DevPass &ps : p->p.passes)
        if (ps.b > bmax) return fail(QS_EINVAL, "plan slab too large for this dtype");
    qs_status st = canonicalize_state(s);
    if (st) return st;
    StepTimer timer;
    st = run_plan(s, const_cast<qs_plan *>(p), &timer);
    if (st) return st;
    st = cuda_status(cudaEventSynchronize(timer.ev.back()), "step timing");
    if (st) return st;
    for (size_t i = 0; i + 1 < timer.ev.size(); ++i) step_ms[i] = timer.between(i, i + 1);
    s->phys_of = p->p.final_phys_of;
    return check_device(s);
    QS_GUARD_END
}

qs_status qs_plan_features(const qs_plan *p, float *out, size_t cap_rows, size_t *nrows)
{
    QS_GUARD_BEGIN
    if (!p || !nrows || (!out && cap_rows)) return fail(QS_EINVAL, "NULL argument");
    std::vector<float> rows;
    plan_features(p->p, rows);
    const size_t r = rows.size() / QS_PLAN_FEATURES;
    *nrows = r;
    if (cap_rows < r) return fail(QS_EINVAL, "output has fewer rows than the plan has steps");
    if (r) std::memcpy(out, rows.data(), rows.size() * sizeof(float));
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_apply_circuit(qs_state *s, const qs_gate *g, size_t ng, const qs_options *o)
{
    QS_GUARD_BEGIN
    if (!s) return fail(QS_EINVAL, "state is NULL");
    qs_options opt;
    if (o) opt = *o;
    else qs_options_default(&opt);
    opt.dtype = s->dt;
    qs_plan *p = nullptr;
    qs_status st = qs_fuse(g, ng, s->n, &opt, &p);
    if (st) return st;
    st = qs_apply_plan(s, p);
    cudaStreamSynchronize(s->stream);
    delete p;
    return st;
    QS_GUARD_END
}

qs_status qs_remap(qs_state *s, int k, const int *A, const int *B)
{
    QS_GUARD_BEGIN
    if (!s || (k > 0 && (!A || !B)) || k < 0) return fail(QS_EINVAL, "bad argument");
    std::vector<int> a(A, A + k), b(B, B + k);
    std::unique_ptr<qs_plan> pl(new qs_plan());
    pl->p.n = s->n;
    pl->p.dt = s->dt;
    std::string err;
    int rc = plan_remap(s->n, s->dt, a, b, pl->p, err);
    if (rc) return fail((qs_status)rc, err);
    qs_status st = run_plan(s, pl.get());
    if (st) return st;
    cudaStreamSynchronize(s->stream);
    std::vector<int> logi(s->n);
    for (int q = 0; q < s->n; ++q) logi[s->phys_of[q]] = q;
    for (int j = 0; j < k; ++j) std::swap(logi[a[j]], logi[b[j]]);
    for (int p = 0; p < s->n; ++p) s->phys_of[logi[p]] = p;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_norm2(qs_state *s, double *host_out)
{
    QS_GUARD_BEGIN
    if (!s || !host_out) return fail(QS_EINVAL, "NULL argument");
    qs_status st = ensure_scratch(s, reduce_scratch_bytes());
    if (st) return st;
    LaunchCtx c{s->amp, s->n, s->dt, (void *)s->stream};
    char err[256] = {0};
    int rc = launch_norm2(c, s->scratch, host_out, err, sizeof err);
    return rc ? fail((qs_status)rc, err) : check_device(s);
    QS_GUARD_END
}

qs_status qs_sample(qs_state *s, const double *u, size_t shots, uint64_t *host_out)
{
    QS_GUARD_BEGIN
    if (!s || (shots && (!u || !host_out))) return fail(QS_EINVAL, "NULL argument");
    if (shots > (size_t(1) << 28)) return fail(QS_EINVAL, "at most 2^28 shots per call");
    for (size_t k = 0; k < shots; ++k)
        if (!(u[k] >= 0.0 && u[k] < 1.0)) return fail(QS_EINVAL, "uniforms must lie in [0, 1)");
    qs_status st = canonicalize_state(s);  // outcomes are logical indices
    if (st) return st;
    const size_t base = (sample_scratch_bytes(s->n) + 255) & ~size_t(255);
    st = ensure_scratch(s, base + shots * (sizeof(double) + sizeof(uint64_t)) + 256);
    if (st) return st;
    char *scr = reinterpret_cast<char *>(s->scratch);
    double *d_u = reinterpret_cast<double *>(scr + base);
    uint64_t *d_out = reinterpret_cast<uint64_t *>(scr + base + shots * sizeof(double));
    if (shots) {
        st = cuda_status(cudaMemcpyAsync(d_u, u, shots * sizeof(double), cudaMemcpyHostToDevice, s->stream),
                         "sample upload");
        if (st) return st;
    }
    LaunchCtx c{s->amp, s->n, s->dt, (void *)s->stream};
    char err[256] = {0};
    const int rc = launch_sample(c, d_u, shots, d_out, s->scratch, err, sizeof err);
    if (rc) return fail((qs_status)rc, err);
    double total = 0.0;
    st = cuda_status(cudaMemcpyAsync(&total, s->scratch + sample_total_index(s->n), sizeof(double),
                                     cudaMemcpyDeviceToHost, s->stream),
                     "sample readback");
    if (!st && shots)
        st = cuda_status(cudaMemcpyAsync(host_out, d_out, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream),
                         "sample readback");
    if (!st) st = cuda_status(cudaStreamSynchronize(s->stream), "sample");
    if (st) return st;
    if (!(total > 0.0)) return fail(QS_EINVAL, "the state has zero norm");
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_probs(qs_state *s, const int *qubits, int nq, double *host_out)
{
    QS_GUARD_BEGIN
    if (!s || !host_out || (nq > 0 && !qubits)) return fail(QS_EINVAL, "NULL argument");
    if (nq < 0 || nq > 24 || nq > s->n) return fail(QS_EINVAL, "nq must be in [0, min(24, n)]");
    uint64_t seen = 0;
    std::vector<int> phys(nq > 0 ? nq : 1);
    for (int j = 0; j < nq; ++j) {
        const int q = qubits[j];
        if (q < 0 || q >= s->n || (seen >> q & 1)) return fail(QS_EINVAL, "qubit out of range or repeated");
        seen |= 1ull << q;
        phys[j] = s->phys_of[q];
    }
    qs_status st = ensure_scratch(s, std::max(reduce_scratch_bytes(), (size_t(1) << nq) * sizeof(double)));
    if (st) return st;
    LaunchCtx c{s->amp, s->n, s->dt, (void *)s->stream};
    char err[256] = {0};
    int rc = launch_probs(c, phys.data(), nq, s->scratch, s->scratch_bytes, host_out, err, sizeof err);
    return rc ? fail((qs_status)rc, err) : QS_OK;
    QS_GUARD_END
}

// Allocation-free readout: validates on the host, then runs the probabilities kernel with the
// fixed device histogram (k_reduce.cu).  Nothing here allocates host or device memory.
qs_status qs_probs_noalloc(const void *dev_amp, int n, qs_dtype dt, const int *qubits, int nq,
                           void *stream, double *host_out)
{
    QS_GUARD_BEGIN
    if (!dev_amp || !host_out || (nq > 0 && !qubits)) return fail(QS_EINVAL, "NULL argument");
    if (reinterpret_cast<uintptr_t>(dev_amp) & 15) return fail(QS_EINVAL, "dev_amp must be 16-byte aligned");
    if (n < 1 || n > QS_MAX_QUBITS) return fail(QS_EINVAL, "n must be in [1, 36]");
    if (dt != QS_C64 && dt != QS_C128) return fail(QS_EINVAL, "bad dtype");
    if (nq < 0 || nq > n) return fail(QS_EINVAL, "nq must be in [0, n]");
    if (nq > kStaticProbsMaxQubits)
        return fail(QS_EINVAL, "qs_probs_noalloc: nq exceeds the fixed 2^14-bin histogram");
    uint64_t seen = 0;
    int phys[kStaticProbsMaxQubits + 1];
    for (int j = 0; j < nq; ++j) {
        const int q = qubits[j];
        if (q < 0 || q >= n || (seen >> q & 1)) return fail(QS_EINVAL, "qubit out of range or repeated");
        seen |= 1ull << q;
        phys[j] = q;
    }
    // The buffer must be device (or managed) memory of the current device: a host pointer or
    // another GPU's memory would make the kernel fault.  Neither query allocates.
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ECUDA, "qs_probs_noalloc: no current CUDA device");
    }
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, dev_amp) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_EINVAL, "qs_probs_noalloc: dev_amp is not a CUDA device pointer");
    }
    if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != cur)
        return fail(QS_EINVAL, "qs_probs_noalloc: dev_amp must be device memory of the current device");
    // The call synchronises and copies into pageable host memory, neither of which a stream
    // capture allows.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_EINVAL, "qs_probs_noalloc: invalid stream");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return fail(QS_EINVAL, "qs_probs_noalloc: the stream is being captured");
    LaunchCtx c{const_cast<void *>(dev_amp), n, dt, stream};
    char err[256] = {0};
    const int rc = launch_probs_static(c, phys, nq, host_out, err, sizeof err);
    return rc ? fail((qs_status)rc, err) : QS_OK;
    QS_GUARD_END
}

qs_status qs_expect_pauli_sum(qs_state *s, const qs_pauli_term *terms, size_t nterms, double *host_out)
{
    QS_GUARD_BEGIN
    if (!s || !host_out || (nterms && !terms)) return fail(QS_EINVAL, "NULL argument");
    const uint64_t valid = s->n >= 64 ? ~0ull : ((1ull << s->n) - 1);
    std::vector<uint64_t> xm(nterms), zm(nterms);
    std::vector<double> cf(nterms);
    for (size_t t = 0; t < nterms; ++t) {
        if ((terms[t].xmask & ~valid) || (terms[t].zmask & ~valid))
            return fail(QS_EINVAL, "Pauli mask has bits beyond n");
        if (!std::isfinite(terms[t].coeff)) return fail(QS_EINVAL, "non-finite coefficient");
        uint64_t x = 0, z = 0;
        for (int q = 0; q < s->n; ++q) {
            if (terms[t].xmask >> q & 1) x |= 1ull << s->phys_of[q];
            if (terms[t].zmask >> q & 1) z |= 1ull << s->phys_of[q];
        }
        xm[t] = x;
        zm[t] = z;
        cf[t] = terms[t].coeff;
    }
    if (nterms == 0) {
        host_out[0] = host_out[1] = 0.0;
        return QS_OK;
    }
    qs_status st = ensure_scratch(s, reduce_scratch_bytes());
    if (st) return st;
    LaunchCtx c{s->amp, s->n, s->dt, (void *)s->stream};
    char err[256] = {0};
    int rc = launch_expect(c, xm.data(), zm.data(), cf.data(), nterms, s->scratch, s->scratch_bytes,
                           host_out, err, sizeof err);
    return rc ? fail((qs_status)rc, err) : QS_OK;
    QS_GUARD_END
}

qs_status qs_stats(qs_state *s, qs_stats_t *out)
{
    QS_GUARD_BEGIN
    if (!s || !out) return fail(QS_EINVAL, "NULL argument");
    s->fold_timings();
    *out = s->stats;
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_stats_reset(qs_state *s)
{
    QS_GUARD_BEGIN
    if (!s) return fail(QS_EINVAL, "NULL argument");
    s->fold_timings();
    std::memset(&s->stats, 0, sizeof s->stats);
    return QS_OK;
    QS_GUARD_END
}

qs_status qs_set_profiling(qs_state *s, int on)
{
    QS_GUARD_BEGIN
    if (!s) return fail(QS_EINVAL, "NULL argument");
    s->profiling = on != 0;
    return QS_OK;
    QS_GUARD_END
}

}  // extern "C"
