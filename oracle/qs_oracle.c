/*
 * qs_oracle.c -- plain FP64 CPU state-vector simulator used as the test oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
 * Python binding) may include, link, load or call this file.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg use it.  It shares no code,
 * header, table or constant with the GPU path.
 *
 * What it computes, and where the definition comes from (arXiv 2406.14084):
 *   - state: 2^n complex amplitudes a_i, qubit q = bit q of the index i
 *     (Eq. 1, Sec. II-A; low qubits are the least significant index bits, Sec. II-B);
 *   - gate application, one gate at a time, no fusion, no blocking: for every index whose
 *     target bits are 0 and control bits are 1, the 2^k amplitudes that differ only in the
 *     target bits are multiplied by the gate's 2^k x 2^k matrix (Eq. 2 for one qubit,
 *     Eq. 3 for the multi-qubit case, e.g. CNOT);
 *   - qubit swap / remap: exchanging index bits pairwise, a'[sigma(i)] = a[i]
 *     (Eq. 4, Sec. II-B; the in-memory swap of Sec. V-B computes this permutation);
 *   - readouts: probabilities |a_x|^2 (marginals by summing), Pauli-string expectations
 *     from the definition P|x> = i^{#Y} (-1)^{popcount(x&z)} |x xor xmask>;
 *   - the unitary of a gate sequence on k qubits, column j = the sequence applied to |j>
 *     (the definition of a fused gate, Sec. II-C "gate fusion", Alg. 1 doFusion);
 *   - a 3-layer ReLU MLP (forward, MSE loss, gradients, Adam step) in FP64 for the
 *     learned cost model, which the paper does not have (parity unpinned by the paper;
 *     pinned by finite differences in the tests).
 *
 * Gate matrices follow the conventions listed in the header comment of qs_oracle.h.
 * Sums in readouts use Neumaier-compensated FP64 accumulation over a fixed chunking,
 * so results do not depend on the thread count.
 */
#define _GNU_SOURCE
#include "qs_oracle.h"

#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

#define OR_MAXQ 40
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- gate matrices */

/* Fill U (dim x dim, row-major, dim = 2^nt) for the gate's target qubits only;
 * controls are handled by the caller.  Returns 0 or a negative error. */
int or_gate_matrix(const or_gate *g, double *Uout)
{
    cplx *U = (cplx *)Uout;
    const double th = g->p[0], ph = g->p[1], la = g->p[2];
    const double c = cos(th / 2.0), s = sin(th / 2.0);
    const double r = 1.0 / sqrt(2.0);
    int nt = g->nt;
    if (nt < 1 || nt > OR_MAX_DENSE)
        return -1;
    int dim = 1 << nt;
    for (int i = 0; i < dim * dim; ++i)
        U[i] = 0.0;
#define SET(row, col, v) U[(row) * dim + (col)] = (v)
    switch (g->kind) {
    case OR_H:
        if (nt != 1) return -2;
        SET(0, 0, r); SET(0, 1, r); SET(1, 0, r); SET(1, 1, -r);
        break;
    case OR_X:
    case OR_CX:
        if (nt != 1) return -2;
        SET(0, 1, 1.0); SET(1, 0, 1.0);
        break;
    case OR_Y:
        if (nt != 1) return -2;
        SET(0, 1, -I); SET(1, 0, I);
        break;
    case OR_Z:
        if (nt != 1) return -2;
        SET(0, 0, 1.0); SET(1, 1, -1.0);
        break;
    case OR_S:
        if (nt != 1) return -2;
        SET(0, 0, 1.0); SET(1, 1, I);
        break;
    case OR_SDG:
        if (nt != 1) return -2;
        SET(0, 0, 1.0); SET(1, 1, -I);
        break;
    case OR_T:
        if (nt != 1) return -2;
        SET(0, 0, 1.0); SET(1, 1, cexp(I * M_PI / 4.0));
        break;
    case OR_TDG:
        if (nt != 1) return -2;
        SET(0, 0, 1.0); SET(1, 1, cexp(-I * M_PI / 4.0));
        break;
    case OR_RX:
        if (nt != 1) return -2;
        SET(0, 0, c); SET(0, 1, -I * s); SET(1, 0, -I * s); SET(1, 1, c);
        break;
    case OR_RY:
        if (nt != 1) return -2;
        SET(0, 0, c); SET(0, 1, -s); SET(1, 0, s); SET(1, 1, c);
        break;
    case OR_RZ:
        if (nt != 1) return -2;
        SET(0, 0, cexp(-I * th / 2.0)); SET(1, 1, cexp(I * th / 2.0));
        break;
    case OR_P:
        if (nt != 1) return -2;
        SET(0, 0, 1.0); SET(1, 1, cexp(I * th));
        break;
    case OR_U3:
        if (nt != 1) return -2;
        SET(0, 0, c);
        SET(0, 1, -cexp(I * la) * s);
        SET(1, 0, cexp(I * ph) * s);
        SET(1, 1, cexp(I * (ph + la)) * c);
        break;
    case OR_CZ:
        if (nt != 2) return -2;
        SET(0, 0, 1.0); SET(1, 1, 1.0); SET(2, 2, 1.0); SET(3, 3, -1.0);
        break;
    case OR_CP:
        if (nt != 2) return -2;
        SET(0, 0, 1.0); SET(1, 1, 1.0); SET(2, 2, 1.0); SET(3, 3, cexp(I * th));
        break;
    case OR_SWAP:
        if (nt != 2) return -2;
        /* local index = b0 + 2*b1; |b1 b0> = |01> <-> |10> */
        SET(0, 0, 1.0); SET(1, 2, 1.0); SET(2, 1, 1.0); SET(3, 3, 1.0);
        break;
    case OR_RZZ:
        if (nt != 2) return -2;
        /* exp(-i th/2 Z(x)Z): even parity -> e^{-i th/2}, odd parity -> e^{+i th/2} */
        SET(0, 0, cexp(-I * th / 2.0));
        SET(1, 1, cexp(I * th / 2.0));
        SET(2, 2, cexp(I * th / 2.0));
        SET(3, 3, cexp(-I * th / 2.0));
        break;
    case OR_UNITARY:
        if (!g->m) return -3;
        for (int i = 0; i < dim * dim; ++i)
            U[i] = g->m[2 * i] + I * g->m[2 * i + 1];
        break;
    case OR_DIAG:
        if (!g->m) return -3;
        for (int i = 0; i < dim; ++i)
            U[i * dim + i] = g->m[2 * i] + I * g->m[2 * i + 1];
        break;
    default:
        return -4;
    }
#undef SET
    return 0;
}

/* ---------------------------------------------------------------- gate application */

static int check_qubits(const or_gate *g, int n)
{
    if (n < 1 || n > OR_MAXQ) return -1;
    if (g->nt < 1 || g->nt > OR_MAX_TARGETS || g->nc < 0 || g->nc > OR_MAX_CONTROLS) return -1;
    uint64_t seen = 0;
    for (int j = 0; j < g->nt; ++j) {
        int q = g->t[j];
        if (q < 0 || q >= n || (seen >> q & 1)) return -1;
        seen |= 1ull << q;
    }
    for (int j = 0; j < g->nc; ++j) {
        int q = g->c[j];
        if (q < 0 || q >= n || (seen >> q & 1)) return -1;
        seen |= 1ull << q;
    }
    return 0;
}

/* Diagonal gate (the D<k> gates of the artifact appendix): the same groups as Eq. 3, but the
 * matrix is diagonal, so amplitude a[i + off(l)] is multiplied by entry l. */
static int apply_diag(cplx *a, int n, const or_gate *g)
{
    if (!g->m) return -3;
    const int k = g->nt, dim = 1 << k;
    uint64_t tmask = 0, cmask = 0;
    for (int j = 0; j < k; ++j) tmask |= 1ull << g->t[j];
    for (int j = 0; j < g->nc; ++j) cmask |= 1ull << g->c[j];
    uint64_t *off = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)dim);
    if (!off) return -2;
    for (int l = 0; l < dim; ++l) {
        uint64_t o = 0;
        for (int j = 0; j < k; ++j)
            if (l >> j & 1) o |= 1ull << g->t[j];
        off[l] = o;
    }
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        if ((uint64_t)i & tmask) continue;
        if (((uint64_t)i & cmask) != cmask) continue;
        for (int l = 0; l < dim; ++l) {
            const cplx d = g->m[2 * l] + I * g->m[2 * l + 1];
            a[(uint64_t)i | off[l]] *= d;
        }
    }
    free(off);
    return 0;
}

/* Eq. 2/3: for each index i with all target bits 0 and all control bits 1, the 2^k
 * amplitudes a[i + sum_j bit_j(l) 2^{t_j}] (l < 2^k) are replaced by U times them. */
int or_apply_gate(double *state, int n, const or_gate *g)
{
    cplx *a = (cplx *)state;
    if (check_qubits(g, n)) return -1;
    const int k = g->nt, dim = 1 << k;
    if (g->kind == OR_DIAG) return apply_diag(a, n, g);
    if (k > OR_MAX_DENSE) return -1;
    cplx *U = (cplx *)malloc(sizeof(cplx) * (size_t)dim * dim);
    if (!U) return -2;
    int rc = or_gate_matrix(g, (double *)U);
    if (rc) { free(U); return rc; }
    uint64_t tmask = 0, cmask = 0;
    for (int j = 0; j < k; ++j) tmask |= 1ull << g->t[j];
    for (int j = 0; j < g->nc; ++j) cmask |= 1ull << g->c[j];
    /* offset of local index l: sum over its set bits j of 2^{t_j} */
    uint64_t off[OR_MAX_DENSE_DIM];
    for (int l = 0; l < dim; ++l) {
        uint64_t o = 0;
        for (int j = 0; j < k; ++j)
            if (l >> j & 1) o |= 1ull << g->t[j];
        off[l] = o;
    }
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        if ((uint64_t)i & tmask) continue;
        if (((uint64_t)i & cmask) != cmask) continue;
        cplx v[OR_MAX_DENSE_DIM], w[OR_MAX_DENSE_DIM];
        for (int l = 0; l < dim; ++l) v[l] = a[(uint64_t)i | off[l]];
        for (int r = 0; r < dim; ++r) {
            cplx acc = 0.0;
            for (int l = 0; l < dim; ++l) acc += U[r * dim + l] * v[l];
            w[r] = acc;
        }
        for (int l = 0; l < dim; ++l) a[(uint64_t)i | off[l]] = w[l];
    }
    free(U);
    return 0;
}

int or_apply_circuit(double *state, int n, const or_gate *gates, int ng)
{
    for (int j = 0; j < ng; ++j) {
        int rc = or_apply_gate(state, n, &gates[j]);
        if (rc) return rc;
    }
    return 0;
}

/* Thread count of the OpenMP loops (1 when built without OpenMP).  Results do not depend on
 * it: every loop iteration writes its own outputs. */
void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_init_basis(double *state, int n, uint64_t x)
{
    cplx *a = (cplx *)state;
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) a[i] = 0.0;
    a[x] = 1.0;
}

/* ---------------------------------------------------------------- remap (Eq. 4) */

/* Exchange index bit A[j] with index bit B[j] for every j: a'[sigma(i)] = a[i]. */
int or_remap(double *state, int n, int k, const int *A, const int *B)
{
    cplx *a = (cplx *)state;
    uint64_t used = 0;
    for (int j = 0; j < k; ++j) {
        if (A[j] < 0 || A[j] >= n || B[j] < 0 || B[j] >= n || A[j] == B[j]) return -1;
        if ((used >> A[j] & 1) || (used >> B[j] & 1)) return -1;
        used |= (1ull << A[j]) | (1ull << B[j]);
    }
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        uint64_t s = (uint64_t)i;
        for (int j = 0; j < k; ++j) {
            uint64_t ba = (uint64_t)i >> A[j] & 1, bb = (uint64_t)i >> B[j] & 1;
            s &= ~((1ull << A[j]) | (1ull << B[j]));
            s |= (bb << A[j]) | (ba << B[j]);
        }
        if (s > (uint64_t)i) {
            cplx t = a[i];
            a[i] = a[s];
            a[s] = t;
        }
    }
    return 0;
}

/* ---------------------------------------------------------------- readouts */

typedef struct { double s, c; } nsum;
static inline void nadd(nsum *acc, double x)
{
    double t = acc->s + x;
    if (fabs(acc->s) >= fabs(x)) acc->c += (acc->s - t) + x;
    else acc->c += (x - t) + acc->s;
    acc->s = t;
}

#define OR_CHUNKS 256

double or_norm2(const double *state, int n)
{
    const cplx *a = (const cplx *)state;
    const int64_t N = (int64_t)1 << n;
    const int64_t per = (N + OR_CHUNKS - 1) / OR_CHUNKS;
    double part[OR_CHUNKS];
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < OR_CHUNKS; ++ch) {
        nsum acc = {0, 0};
        int64_t lo = ch * per, hi = lo + per < N ? lo + per : N;
        for (int64_t i = lo; i < hi; ++i) {
            double re = creal(a[i]), im = cimag(a[i]);
            nadd(&acc, re * re + im * im);
        }
        part[ch] = acc.s + acc.c;
    }
    nsum tot = {0, 0};
    for (int ch = 0; ch < OR_CHUNKS; ++ch) nadd(&tot, part[ch]);
    return tot.s + tot.c;
}

/* Marginal probabilities: out[m] = sum of |a_x|^2 over x whose qubit q[j] equals bit j of m. */
/* Measurement sampling in the computational basis (Born rule, Eq. 1: outcome x has
 * probability |a_x|^2 / sum_y |a_y|^2).  For each caller-supplied uniform u[k] in [0, 1), the
 * outcome is the smallest x with C(x) > u[k] * C(2^n - 1), where C(x) = sum_{y <= x} |a_y|^2 is
 * the running sum taken in index order (inverse transform sampling).  Plain sequential FP64. */
int or_sample(const double *state, int n, const double *u, int64_t shots, uint64_t *out)
{
    const cplx *a = (const cplx *)state;
    const int64_t N = (int64_t)1 << n;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)N);
    if (!cdf) return -2;
    double run = 0.0;
    for (int64_t x = 0; x < N; ++x) {
        const double re = creal(a[x]), im = cimag(a[x]);
        run += re * re + im * im;
        cdf[x] = run;
    }
    for (int64_t k = 0; k < shots; ++k) {
        if (!(u[k] >= 0.0 && u[k] < 1.0)) {
            free(cdf);
            return -1;
        }
        const double t = u[k] * run;
        int64_t lo = 0, hi = N - 1; /* smallest x with cdf[x] > t */
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        out[k] = (uint64_t)lo;
    }
    free(cdf);
    return 0;
}

int or_probs(const double *state, int n, const int *q, int nq, double *out)
{
    const cplx *a = (const cplx *)state;
    if (nq < 0 || nq > 24 || nq > n) return -1;
    uint64_t seen = 0;
    for (int j = 0; j < nq; ++j) {
        if (q[j] < 0 || q[j] >= n || (seen >> q[j] & 1)) return -1;
        seen |= 1ull << q[j];
    }
    const int64_t M = (int64_t)1 << nq;
    const int64_t N = (int64_t)1 << n;
    nsum *acc = (nsum *)calloc((size_t)M, sizeof(nsum));
    if (!acc) return -2;
    for (int64_t x = 0; x < N; ++x) {
        uint64_t m = 0;
        for (int j = 0; j < nq; ++j) m |= ((uint64_t)x >> q[j] & 1) << j;
        double re = creal(a[x]), im = cimag(a[x]);
        nadd(&acc[m], re * re + im * im);
    }
    for (int64_t m = 0; m < M; ++m) out[m] = acc[m].s + acc[m].c;
    free(acc);
    return 0;
}

/* <psi| sum_t coeff_t P_t |psi>; out[0] = real part, out[1] = imaginary part. */
int or_expect_pauli(const double *state, int n, const double *coeff, const uint64_t *xmask,
                    const uint64_t *zmask, int nterms, double *out)
{
    const cplx *a = (const cplx *)state;
    const int64_t N = (int64_t)1 << n;
    const uint64_t valid = n >= 64 ? ~0ull : ((1ull << n) - 1);
    nsum tr = {0, 0}, ti = {0, 0};
    for (int t = 0; t < nterms; ++t) {
        if ((xmask[t] & ~valid) || (zmask[t] & ~valid)) return -1;
        const uint64_t xm = xmask[t], zm = zmask[t];
        const int ny = __builtin_popcountll(xm & zm);
        /* i^{#Y} */
        const cplx iy[4] = {1.0, I, -1.0, -I};
        const cplx ph = iy[ny & 3];
        const int64_t per = (N + OR_CHUNKS - 1) / OR_CHUNKS;
        double pr[OR_CHUNKS], pi[OR_CHUNKS];
#pragma omp parallel for schedule(static)
        for (int ch = 0; ch < OR_CHUNKS; ++ch) {
            nsum ar = {0, 0}, ai = {0, 0};
            int64_t lo = ch * per, hi = lo + per < N ? lo + per : N;
            for (int64_t x = lo; x < hi; ++x) {
                double sg = (__builtin_popcountll((uint64_t)x & zm) & 1) ? -1.0 : 1.0;
                /* P|x> = ph * sg * |x ^ xm>, contributes conj(a[x^xm]) * ph * sg * a[x] */
                cplx v = conj(a[(uint64_t)x ^ xm]) * ph * sg * a[x];
                nadd(&ar, creal(v));
                nadd(&ai, cimag(v));
            }
            pr[ch] = ar.s + ar.c;
            pi[ch] = ai.s + ai.c;
        }
        nsum sr = {0, 0}, si = {0, 0};
        for (int ch = 0; ch < OR_CHUNKS; ++ch) {
            nadd(&sr, pr[ch]);
            nadd(&si, pi[ch]);
        }
        nadd(&tr, coeff[t] * (sr.s + sr.c));
        nadd(&ti, coeff[t] * (si.s + si.c));
    }
    out[0] = tr.s + tr.c;
    out[1] = ti.s + ti.c;
    return 0;
}

/* ---------------------------------------------------------------- fused-gate definition */

/* Unitary of a gate sequence acting on qubits 0..k-1: column j is the sequence applied to |j>.
 * U is dim x dim complex, row-major. */
int or_circuit_unitary(const or_gate *gates, int ng, int k, double *Uout)
{
    if (k < 1 || k > 12) return -1;
    const int64_t dim = (int64_t)1 << k;
    cplx *U = (cplx *)Uout;
    cplx *col = (cplx *)malloc((size_t)dim * sizeof(cplx));
    if (!col) return -2;
    for (int64_t j = 0; j < dim; ++j) {
        or_init_basis((double *)col, k, (uint64_t)j);
        int rc = or_apply_circuit((double *)col, k, gates, ng);
        if (rc) { free(col); return rc; }
        for (int64_t r = 0; r < dim; ++r) U[r * dim + j] = col[r];
    }
    free(col);
    return 0;
}

/* ---------------------------------------------------------------- MLP (FP64) */
/* y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3, with W1: F x H, W2: H x H, W3: H x 1
 * (row-major, input index first).  Loss = mean over the batch of (y - target)^2. */

static void mlp_fwd_one(const double *x, int F, int H, const double *W1, const double *b1,
                        const double *W2, const double *b2, const double *W3, const double *b3,
                        double *z1, double *h1, double *z2, double *h2, double *y)
{
    for (int o = 0; o < H; ++o) {
        double s = b1[o];
        for (int i = 0; i < F; ++i) s += x[i] * W1[i * H + o];
        z1[o] = s;
        h1[o] = s > 0 ? s : 0;
    }
    for (int o = 0; o < H; ++o) {
        double s = b2[o];
        for (int i = 0; i < H; ++i) s += h1[i] * W2[i * H + o];
        z2[o] = s;
        h2[o] = s > 0 ? s : 0;
    }
    double s = b3[0];
    for (int i = 0; i < H; ++i) s += h2[i] * W3[i];
    *y = s;
}

int or_mlp_forward(const double *X, int B, int F, int H, const double *W1, const double *b1,
                   const double *W2, const double *b2, const double *W3, const double *b3,
                   double *y)
{
    double *buf = (double *)malloc(sizeof(double) * 4 * (size_t)H);
    if (!buf) return -2;
    for (int r = 0; r < B; ++r)
        mlp_fwd_one(X + (size_t)r * F, F, H, W1, b1, W2, b2, W3, b3, buf, buf + H, buf + 2 * H,
                    buf + 3 * H, &y[r]);
    free(buf);
    return 0;
}

/* Gradients of the mean squared error with respect to every parameter (backpropagation,
 * written out per sample).  Gradient buffers are overwritten. */
int or_mlp_loss_grad(const double *X, const double *target, int B, int F, int H,
                     const double *W1, const double *b1, const double *W2, const double *b2,
                     const double *W3, const double *b3, double *gW1, double *gb1, double *gW2,
                     double *gb2, double *gW3, double *gb3, double *loss)
{
    memset(gW1, 0, sizeof(double) * (size_t)F * H);
    memset(gb1, 0, sizeof(double) * (size_t)H);
    memset(gW2, 0, sizeof(double) * (size_t)H * H);
    memset(gb2, 0, sizeof(double) * (size_t)H);
    memset(gW3, 0, sizeof(double) * (size_t)H);
    gb3[0] = 0;
    double *buf = (double *)malloc(sizeof(double) * 6 * (size_t)H);
    if (!buf) return -2;
    double *z1 = buf, *h1 = buf + H, *z2 = buf + 2 * H, *h2 = buf + 3 * H, *d2 = buf + 4 * H,
           *d1 = buf + 5 * H;
    double L = 0;
    for (int r = 0; r < B; ++r) {
        const double *x = X + (size_t)r * F;
        double y;
        mlp_fwd_one(x, F, H, W1, b1, W2, b2, W3, b3, z1, h1, z2, h2, &y);
        double e = y - target[r];
        L += e * e;
        double dy = 2.0 * e / B;
        gb3[0] += dy;
        for (int i = 0; i < H; ++i) {
            gW3[i] += h2[i] * dy;
            d2[i] = z2[i] > 0 ? W3[i] * dy : 0.0;
        }
        for (int o = 0; o < H; ++o) gb2[o] += d2[o];
        for (int i = 0; i < H; ++i)
            for (int o = 0; o < H; ++o) gW2[i * H + o] += h1[i] * d2[o];
        for (int i = 0; i < H; ++i) {
            double s = 0;
            for (int o = 0; o < H; ++o) s += W2[i * H + o] * d2[o];
            d1[i] = z1[i] > 0 ? s : 0.0;
        }
        for (int o = 0; o < H; ++o) gb1[o] += d1[o];
        for (int i = 0; i < F; ++i)
            for (int o = 0; o < H; ++o) gW1[i * H + o] += x[i] * d1[o];
    }
    *loss = L / B;
    free(buf);
    return 0;
}

/* One Adam step (Kingma & Ba 2015, Algorithm 1) on a flat parameter vector, step t >= 1. */
void or_adam_step(double *p, const double *g, double *m, double *v, int64_t count, int t,
                  double lr, double beta1, double beta2, double eps)
{
    const double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int64_t i = 0; i < count; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
