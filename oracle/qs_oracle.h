/*
 * qs_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only; the product
 * path never includes this header).
 *
 * Gate conventions (arXiv 2406.14084 names the gates in Table 1 but fixes no matrices; the
 * readings below are standard textbook definitions, and RZZ's half angle is pinned by the
 * fused-diagonal values printed in the artifact appendix, cos(7) and cos(10)):
 *   H  = 1/sqrt2 [[1,1],[1,-1]]        X = [[0,1],[1,0]]        Y = [[0,-i],[i,0]]
 *   Z  = diag(1,-1)   S = diag(1,i)   SDG = diag(1,-i)   T = diag(1,e^{i pi/4})   TDG = conj(T)
 *   RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]], c = cos t/2, s = sin t/2
 *   RZ(t) = diag(e^{-it/2}, e^{it/2})            P(l) = diag(1, e^{il})
 *   U3(t,f,l) = [[c, -e^{il} s], [e^{if} s, e^{i(f+l)} c]]
 *   CX  = X on t[0], controlled by c[0] (nt = 1, nc >= 1)
 *   CZ  = diag(1,1,1,-1), CP(l) = diag(1,1,1,e^{il}), RZZ(t) = exp(-i t/2 Z(x)Z), SWAP
 *         (nt = 2, targets t[0], t[1])
 *   UNITARY: m = 2^nt x 2^nt complex, row-major, interleaved (re, im)
 *   DIAG:    m = 2^nt complex diagonal entries
 * The local matrix index has bit j equal to qubit t[j] (t[0] is the least significant bit).
 * Any gate may carry extra controls c[0..nc-1]; it then acts only where all are 1.
 */
#ifndef QS_ORACLE_H
#define QS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    OR_H = 0, OR_X, OR_Y, OR_Z, OR_S, OR_SDG, OR_T, OR_TDG, OR_RX, OR_RY, OR_RZ, OR_P, OR_U3,
    OR_CX, OR_CZ, OR_CP, OR_SWAP, OR_RZZ, OR_UNITARY, OR_DIAG
};

#define OR_MAX_TARGETS 12   /* DIAG gates; dense kinds take at most OR_MAX_DENSE targets */
#define OR_MAX_DENSE 7
#define OR_MAX_CONTROLS 8
#define OR_MAX_DENSE_DIM (1 << OR_MAX_DENSE)

typedef struct {
    int32_t kind;
    int32_t nt, nc;
    int32_t t[OR_MAX_TARGETS];
    int32_t c[OR_MAX_CONTROLS];
    double p[3];
    const double *m;
} or_gate;

/* state = 2^n complex amplitudes as interleaved (re, im) doubles */
int or_gate_matrix(const or_gate *g, double *U);
int or_apply_gate(double *state, int n, const or_gate *g);
int or_apply_circuit(double *state, int n, const or_gate *gates, int ng);
void or_init_basis(double *state, int n, uint64_t x);
void or_set_threads(int t);
int or_get_threads(void);
int or_remap(double *state, int n, int k, const int *A, const int *B);
double or_norm2(const double *state, int n);
int or_probs(const double *state, int n, const int *q, int nq, double *out);
int or_sample(const double *state, int n, const double *u, int64_t shots, uint64_t *out);
int or_expect_pauli(const double *state, int n, const double *coeff, const uint64_t *xmask,
                    const uint64_t *zmask, int nterms, double *out);
int or_circuit_unitary(const or_gate *gates, int ng, int k, double *U);
int or_mlp_forward(const double *X, int B, int F, int H, const double *W1, const double *b1,
                   const double *W2, const double *b2, const double *W3, const double *b3,
                   double *y);
int or_mlp_loss_grad(const double *X, const double *target, int B, int F, int H,
                     const double *W1, const double *b1, const double *W2, const double *b2,
                     const double *W3, const double *b3, double *gW1, double *gb1, double *gW2,
                     double *gb2, double *gW3, double *gb3, double *loss);
void or_adam_step(double *p, const double *g, double *m, double *v, int64_t count, int t,
                  double lr, double beta1, double beta2, double eps);

#ifdef __cplusplus
}
#endif
#endif
