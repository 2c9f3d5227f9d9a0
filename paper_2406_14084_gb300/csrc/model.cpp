// model.cpp -- the cost-model network object: parameters and Adam moments in device memory,
// training and inference through the kernels of k_mlp.cu, and the extern "C" model API.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "model.h"
#include "qs_internal.h"

namespace qs {
qs_status set_error(qs_status st, const std::string &msg);
}

using namespace qs;

struct qs_model {
    int F = 0, P = 0, pstride = 0;
    cudaStream_t stream = nullptr;
    // one allocation: params | m | v | grad | mu | inv_sd | loss[1] | step (int)
    void *base = nullptr;
    float *params = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
    float *mu = nullptr, *inv_sd = nullptr, *loss = nullptr;
    int *step = nullptr;
    // growable scratch
    float *X = nullptr, *T = nullptr, *y = nullptr, *losses = nullptr, *partial = nullptr;
    size_t cap_rows = 0, cap_losses = 0, cap_tiles = 0;
    std::vector<float> h_mu, h_sd;
    float ym = 0.f, ys = 1.f;
    int steps = 0;
    float last_loss = 0.f;
    std::mutex lock;

    ~qs_model()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (void *p : {(void *)X, (void *)T, (void *)y, (void *)losses, (void *)partial, base})
            if (p) cudaFree(p);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

std::atomic<qs_model *> g_default{nullptr};

qs_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return QS_OK;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return set_error(QS_ENOMEM, std::string(what) + ": out of device memory");
    return set_error(QS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return double(next() >> 11) * 0x1.0p-53; }
};

qs_status grow(float *&p, size_t &cap, size_t need, const char *what)
{
    if (need <= cap) return QS_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    qs_status st = cuda_fail(cudaMalloc(&p, need * sizeof(float)), what);
    if (st) return st;
    cap = need;
    return QS_OK;
}

qs_status ensure_rows(qs_model *m, size_t rows)
{
    if (rows <= m->cap_rows) return QS_OK;
    for (float **p : {&m->X, &m->T, &m->y})
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    m->cap_rows = 0;
    qs_status st = cuda_fail(cudaMalloc(&m->X, rows * m->F * sizeof(float)), "model input buffer");
    if (!st) st = cuda_fail(cudaMalloc(&m->T, rows * sizeof(float)), "model target buffer");
    if (!st) st = cuda_fail(cudaMalloc(&m->y, rows * sizeof(float)), "model output buffer");
    if (st) return st;
    m->cap_rows = rows;
    return QS_OK;
}

qs_status ensure_tiles(qs_model *m, size_t tiles)
{
    size_t cap = m->cap_tiles * m->pstride;
    qs_status st = grow(m->partial, cap, tiles * m->pstride, "model gradient buffer");
    if (st) return st;
    m->cap_tiles = cap / m->pstride;
    return QS_OK;
}

MlpArgs base_args(qs_model *m)
{
    MlpArgs a{};
    a.F = m->F;
    a.params = m->params;
    a.mu = m->mu;
    a.inv_sd = m->inv_sd;
    a.ym = m->ym;
    a.ys = m->ys;
    a.inv_ys = 1.f / m->ys;
    a.partial = m->partial;
    a.pstride = m->pstride;
    a.nparams = m->P;
    a.adam_m = m->adam_m;
    a.adam_v = m->adam_v;
    return a;
}

qs_status upload_norm(qs_model *m)
{
    std::vector<float> inv(m->F);
    for (int f = 0; f < m->F; ++f) inv[f] = 1.f / m->h_sd[f];
    qs_status st = cuda_fail(cudaMemcpy(m->mu, m->h_mu.data(), m->F * sizeof(float), cudaMemcpyHostToDevice),
                             "model standardisation upload");
    if (st) return st;
    return cuda_fail(cudaMemcpy(m->inv_sd, inv.data(), m->F * sizeof(float), cudaMemcpyHostToDevice),
                     "model standardisation upload");
}

qs_status reset_adam(qs_model *m)
{
    cudaMemsetAsync(m->adam_m, 0, size_t(m->P) * sizeof(float), m->stream);
    cudaMemsetAsync(m->adam_v, 0, size_t(m->P) * sizeof(float), m->stream);
    cudaMemsetAsync(m->step, 0, sizeof(int), m->stream);
    m->steps = 0;
    return cuda_fail(cudaStreamSynchronize(m->stream), "model reset");
}

qs_status forward(qs_model *m, const float *X, size_t rows, float *y)
{
    if (rows == 0) return QS_OK;
    qs_status st = ensure_rows(m, rows);
    if (st) return st;
    st = cuda_fail(cudaMemcpyAsync(m->X, X, rows * m->F * sizeof(float), cudaMemcpyHostToDevice, m->stream),
                   "model input upload");
    if (st) return st;
    MlpArgs a = base_args(m);
    a.X = m->X;
    a.B = (int)rows;
    a.y_out = m->y;
    char err[256] = {0};
    int rc = launch_mlp_forward(a, (void *)m->stream, err, sizeof err);
    if (rc) return set_error((qs_status)rc, err);
    st = cuda_fail(cudaMemcpyAsync(y, m->y, rows * sizeof(float), cudaMemcpyDeviceToHost, m->stream),
                   "model output download");
    if (st) return st;
    return cuda_fail(cudaStreamSynchronize(m->stream), "model forward");
}

#define MODEL_GUARD_BEGIN try {
#define MODEL_GUARD_END                                                                   \
    }                                                                                     \
    catch (const std::bad_alloc &) { return set_error(QS_ENOMEM, "host allocation failed"); } \
    catch (const std::exception &e) { return set_error(QS_EINVAL, e.what()); }           \
    catch (...) { return set_error(QS_EINVAL, "unknown error"); }

}  // namespace

namespace qs {

int model_predict(qs_model *m, const float *X, size_t rows, float *y, std::string &err)
{
    std::lock_guard<std::mutex> g(m->lock);
    qs_status st = forward(m, X, rows, y);
    if (st) err = "cost-model forward failed";
    return st;
}

int model_nfeat(const qs_model *m) { return m->F; }

qs_model *default_cost_model() { return g_default.load(); }

}  // namespace qs

extern "C" {

void qs_train_options_default(qs_train_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->epochs = 40;
    o->batch = 256;
    o->lr = 1e-3f;
    o->fit_norm = 1;
    o->seed = 1;
    o->graph = 1;
}

qs_status qs_model_create(int nfeat, uint64_t seed, qs_model **out)
{
    MODEL_GUARD_BEGIN
    if (!out) return set_error(QS_EINVAL, "out is NULL");
    if (nfeat < 1 || nfeat > kMlpMaxFeatures) return set_error(QS_EINVAL, "nfeat must be in [1, 32]");
    std::unique_ptr<qs_model> m(new qs_model());
    m->F = nfeat;
    m->P = mlp_param_count(nfeat);
    m->pstride = (m->P + 1 + 3) & ~3;
    qs_status st = cuda_fail(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking), "model stream");
    if (st) return st;
    const size_t P = m->P, F = nfeat;
    const size_t floats = 4 * P + 2 * F + 1 + 1;
    st = cuda_fail(cudaMalloc(&m->base, floats * sizeof(float) + 64), "model allocation");
    if (st) return st;
    float *f = static_cast<float *>(m->base);
    m->params = f;
    m->adam_m = f + P;
    m->adam_v = f + 2 * P;
    m->grad = f + 3 * P;
    m->mu = f + 4 * P;
    m->inv_sd = m->mu + F;
    m->loss = m->inv_sd + F;
    m->step = reinterpret_cast<int *>(m->loss + 1);
    // He-uniform weights (bound sqrt(6 / fan_in)), zero biases
    std::vector<float> h(P, 0.f);
    SplitMix rng{seed};
    const int H = kMlpHidden;
    auto fill = [&](size_t off, size_t count, int fan_in) {
        const double bound = std::sqrt(6.0 / fan_in);
        for (size_t i = 0; i < count; ++i) h[off + i] = float((2.0 * rng.uniform() - 1.0) * bound);
    };
    fill(0, F * H, nfeat);
    fill(F * H + H, size_t(H) * H, H);
    fill(F * H + H + size_t(H) * H + H, H, H);
    st = cuda_fail(cudaMemcpy(m->params, h.data(), P * sizeof(float), cudaMemcpyHostToDevice), "model upload");
    if (st) return st;
    m->h_mu.assign(F, 0.f);
    m->h_sd.assign(F, 1.f);
    st = upload_norm(m.get());
    if (st) return st;
    st = reset_adam(m.get());
    if (st) return st;
    *out = m.release();
    return QS_OK;
    MODEL_GUARD_END
}

qs_status qs_model_destroy(qs_model *m)
{
    if (!m) return QS_OK;
    qs_model *expected = m;
    g_default.compare_exchange_strong(expected, nullptr);
    delete m;
    return QS_OK;
}

qs_status qs_model_info_get(const qs_model *m, qs_model_info *out)
{
    if (!m || !out) return set_error(QS_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->nfeat = m->F;
    out->hidden = kMlpHidden;
    out->nparams = m->P;
    out->steps = m->steps;
    out->ym = m->ym;
    out->ys = m->ys;
    out->last_loss = m->last_loss;
    return QS_OK;
}

qs_status qs_model_get_params(const qs_model *m, float *host, size_t count)
{
    if (!m || !host) return set_error(QS_EINVAL, "NULL argument");
    if (count != (size_t)m->P) return set_error(QS_EINVAL, "count must equal the parameter count");
    qs_model *mm = const_cast<qs_model *>(m);
    std::lock_guard<std::mutex> g(mm->lock);
    cudaStreamSynchronize(mm->stream);
    return cuda_fail(cudaMemcpy(host, m->params, count * sizeof(float), cudaMemcpyDeviceToHost), "parameter download");
}

qs_status qs_model_get_moments(const qs_model *m, float *mom, float *vel, size_t count)
{
    if (!m || !mom || !vel) return set_error(QS_EINVAL, "NULL argument");
    if (count != (size_t)m->P) return set_error(QS_EINVAL, "count must equal the parameter count");
    qs_model *mm = const_cast<qs_model *>(m);
    std::lock_guard<std::mutex> g(mm->lock);
    cudaStreamSynchronize(mm->stream);
    qs_status st = cuda_fail(cudaMemcpy(mom, m->adam_m, count * sizeof(float), cudaMemcpyDeviceToHost),
                             "first-moment download");
    if (st) return st;
    return cuda_fail(cudaMemcpy(vel, m->adam_v, count * sizeof(float), cudaMemcpyDeviceToHost),
                     "second-moment download");
}

qs_status qs_model_set_params(qs_model *m, const float *host, size_t count)
{
    if (!m || !host) return set_error(QS_EINVAL, "NULL argument");
    if (count != (size_t)m->P) return set_error(QS_EINVAL, "count must equal the parameter count");
    std::lock_guard<std::mutex> g(m->lock);
    cudaStreamSynchronize(m->stream);
    qs_status st = cuda_fail(cudaMemcpy(m->params, host, count * sizeof(float), cudaMemcpyHostToDevice),
                             "parameter upload");
    if (st) return st;
    return reset_adam(m);
}

qs_status qs_model_get_norm(const qs_model *m, float *mu, float *sd, float *ym, float *ys)
{
    if (!m) return set_error(QS_EINVAL, "NULL argument");
    if (mu) std::copy(m->h_mu.begin(), m->h_mu.end(), mu);
    if (sd) std::copy(m->h_sd.begin(), m->h_sd.end(), sd);
    if (ym) *ym = m->ym;
    if (ys) *ys = m->ys;
    return QS_OK;
}

qs_status qs_model_set_norm(qs_model *m, const float *mu, const float *sd, float ym, float ys)
{
    if (!m || !mu || !sd) return set_error(QS_EINVAL, "NULL argument");
    for (int f = 0; f < m->F; ++f)
        if (!(sd[f] > 0.f) || !std::isfinite(mu[f])) return set_error(QS_EINVAL, "sd must be positive, mu finite");
    if (!(ys > 0.f) || !std::isfinite(ym)) return set_error(QS_EINVAL, "ys must be positive, ym finite");
    std::lock_guard<std::mutex> g(m->lock);
    cudaStreamSynchronize(m->stream);
    m->h_mu.assign(mu, mu + m->F);
    m->h_sd.assign(sd, sd + m->F);
    m->ym = ym;
    m->ys = ys;
    return upload_norm(m);
}

qs_status qs_model_predict(qs_model *m, const float *X, size_t rows, float *y)
{
    MODEL_GUARD_BEGIN
    if (!m || (rows && (!X || !y))) return set_error(QS_EINVAL, "NULL argument");
    if (rows > (size_t(1) << 31) / kMlpMaxFeatures) return set_error(QS_EINVAL, "too many rows");
    std::lock_guard<std::mutex> g(m->lock);
    return forward(m, X, rows, y);
    MODEL_GUARD_END
}

qs_status qs_model_loss_grad(qs_model *m, const float *X, const float *T, size_t rows, float *grad, float *loss)
{
    MODEL_GUARD_BEGIN
    if (!m || !X || !T || !grad) return set_error(QS_EINVAL, "NULL argument");
    if (rows == 0 || rows > (size_t(1) << 24)) return set_error(QS_EINVAL, "rows must be in [1, 2^24]");
    std::lock_guard<std::mutex> g(m->lock);
    qs_status st = ensure_rows(m, rows);
    if (!st) st = ensure_tiles(m, mlp_tiles((int)rows));
    if (st) return st;
    cudaMemcpyAsync(m->X, X, rows * m->F * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->T, T, rows * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    MlpArgs a = base_args(m);
    a.X = m->X;
    a.T = m->T;
    a.B = (int)rows;
    a.scale = 2.f / float(rows);
    a.step_counter = nullptr;
    a.grad_out = m->grad;
    a.loss_out = m->loss;
    char err[256] = {0};
    int rc = launch_mlp_train_step(a, 0, 0.f, (void *)m->stream, err, sizeof err);
    if (rc) return set_error((qs_status)rc, err);
    cudaMemcpyAsync(grad, m->grad, size_t(m->P) * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    float l = 0.f;
    cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    st = cuda_fail(cudaStreamSynchronize(m->stream), "model gradient");
    if (st) return st;
    if (loss) *loss = l;
    return QS_OK;
    MODEL_GUARD_END
}

qs_status qs_model_train(qs_model *m, const float *X, const float *T, size_t rows, const qs_train_options *o,
                         float *final_loss)
{
    MODEL_GUARD_BEGIN
    if (!m || !X || !T) return set_error(QS_EINVAL, "NULL argument");
    qs_train_options opt;
    if (o) opt = *o;
    else qs_train_options_default(&opt);
    if (rows == 0 || rows > (size_t(1) << 24)) return set_error(QS_EINVAL, "rows must be in [1, 2^24]");
    if (opt.epochs < 1 || opt.batch < 1 || !(opt.lr > 0.f)) return set_error(QS_EINVAL, "bad training options");
    std::lock_guard<std::mutex> g(m->lock);
    const int F = m->F;
    for (size_t i = 0; i < rows * F; ++i)
        if (!std::isfinite(X[i])) return set_error(QS_EINVAL, "non-finite feature");
    for (size_t i = 0; i < rows; ++i)
        if (!std::isfinite(T[i])) return set_error(QS_EINVAL, "non-finite target");
    if (opt.fit_norm) {
        // standardisation statistics in FP64 (data preparation)
        std::vector<double> s(F, 0.0), s2(F, 0.0);
        double t1 = 0, t2 = 0;
        for (size_t r = 0; r < rows; ++r) {
            for (int f = 0; f < F; ++f) {
                s[f] += X[r * F + f];
                s2[f] += double(X[r * F + f]) * X[r * F + f];
            }
            t1 += T[r];
            t2 += double(T[r]) * T[r];
        }
        for (int f = 0; f < F; ++f) {
            const double mean = s[f] / rows, var = std::max(0.0, s2[f] / rows - mean * mean);
            m->h_mu[f] = (float)mean;
            m->h_sd[f] = var > 1e-12 ? (float)std::sqrt(var) : 1.f;
        }
        const double tm = t1 / rows, tv = std::max(0.0, t2 / rows - tm * tm);
        m->ym = (float)tm;
        m->ys = tv > 1e-12 ? (float)std::sqrt(tv) : 1.f;
        qs_status st = upload_norm(m);
        if (st) return st;
    }
    // shuffle once (Fisher-Yates over a SplitMix64 stream)
    std::vector<size_t> perm(rows);
    for (size_t i = 0; i < rows; ++i) perm[i] = i;
    SplitMix rng{opt.seed};
    for (size_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[rng.next() % (i + 1)]);
    std::vector<float> hx(rows * F), ht(rows);
    for (size_t r = 0; r < rows; ++r) {
        std::memcpy(&hx[r * F], &X[perm[r] * F], F * sizeof(float));
        ht[r] = T[perm[r]];
    }
    const size_t bs = rows > (size_t)opt.batch ? (size_t)opt.batch : rows;
    const size_t nb = rows / bs;
    qs_status st = ensure_rows(m, rows);
    if (!st) st = ensure_tiles(m, mlp_tiles((int)bs));
    if (!st) st = grow(m->losses, m->cap_losses, nb, "model loss buffer");
    if (st) return st;
    cudaMemcpyAsync(m->X, hx.data(), rows * F * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->T, ht.data(), rows * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    st = cuda_fail(cudaStreamSynchronize(m->stream), "training data upload");
    if (st) return st;

    char err[256] = {0};
    auto epoch = [&]() -> int {
        for (size_t b = 0; b < nb; ++b) {
            MlpArgs a = base_args(m);
            a.X = m->X + b * bs * F;
            a.T = m->T + b * bs;
            a.B = (int)bs;
            a.scale = 2.f / float(bs);
            a.step_counter = m->step;
            a.loss_out = m->losses + b;
            int rc = launch_mlp_train_step(a, 1, opt.lr, (void *)m->stream, err, sizeof err);
            if (rc) return rc;
        }
        return QS_OK;
    };
    // first epoch eagerly (also sets the kernels' shared-memory attributes)
    int rc = epoch();
    if (rc) return set_error((qs_status)rc, err);
    int done = 1;
    if (opt.epochs > 1 && opt.graph) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        st = cuda_fail(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal), "training capture");
        if (st) return st;
        rc = epoch();
        cudaError_t ce = cudaStreamEndCapture(m->stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return set_error((qs_status)rc, err);
        }
        st = cuda_fail(ce, "training capture");
        if (!st) st = cuda_fail(cudaGraphInstantiate(&exec, graph, 0), "training graph instantiation");
        if (graph) cudaGraphDestroy(graph);
        if (st) return st;
        for (; done < opt.epochs && !st; ++done) st = cuda_fail(cudaGraphLaunch(exec, m->stream), "training graph launch");
        cudaStreamSynchronize(m->stream);
        cudaGraphExecDestroy(exec);
        if (st) return st;
    }
    for (; done < opt.epochs; ++done) {
        rc = epoch();
        if (rc) return set_error((qs_status)rc, err);
    }
    std::vector<float> hl(nb);
    cudaMemcpyAsync(hl.data(), m->losses, nb * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    st = cuda_fail(cudaStreamSynchronize(m->stream), "training");
    if (st) return st;
    double acc = 0;
    for (float v : hl) acc += v;
    m->last_loss = float(acc / nb);
    m->steps += int(nb) * opt.epochs;
    if (final_loss) *final_loss = m->last_loss;
    return QS_OK;
    MODEL_GUARD_END
}

qs_status qs_set_cost_model(qs_model *m)
{
    g_default.store(m);
    return QS_OK;
}

}  // extern "C"
