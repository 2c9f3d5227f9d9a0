/*
 * qs.h -- C ABI of the GB300 state-vector simulator core (libqs.so).
 *
 * The library applies quantum circuits to a full 2^n-amplitude complex state vector held in
 * GPU memory, following the cache-aware method of arXiv 2406.14084 ("Queen"): gates are
 * grouped into gate blocks whose qubits fit one on-chip slab (Sec. IV, Eq. 5-7, Alg. 1-2),
 * each block is applied to every slab in one HBM round trip (Sec. V, Alg. 3, Sec. V-A), and
 * qubit remaps move qubits between slab and memory positions (Sec. V-B, Alg. 4).
 *
 * Conventions that hold for every entry point:
 *   - Every call returns a qs_status.  No C++ exception or abort crosses this boundary.  On
 *     failure, qs_last_error() returns a message (thread-local, valid until the next call on
 *     the same thread).
 *   - Invalid input returns QS_EINVAL and leaves the state untouched.
 *   - Amplitude index bit q is qubit q (Eq. 1; qubit 0 is the least significant bit).
 *   - Device work is ordered on the state's CUDA stream.  Calls that write host memory
 *     synchronise that stream before returning; the others return once work is enqueued.
 *   - Readouts (qs_probs, qs_expect_pauli_sum, qs_copy_to_host) use logical qubit order,
 *     whatever physical layout the last plan left the state in.
 *   - Pointers named host_* are host memory owned by the caller; dev pointers are device
 *     memory.  The library never frees memory it did not allocate.
 *   - A qs_state may be used by one host thread at a time.
 */
#ifndef QS_ABI_INCLUDED_H_
#define QS_ABI_INCLUDED_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype; /* complex64 / complex128 amplitudes */

typedef enum {
    QS_OK = 0,
    QS_EINVAL = 1,        /* bad argument; nothing was changed */
    QS_ENOMEM = 2,        /* device or host allocation failed */
    QS_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
    QS_ETIMEOUT = 4,      /* a bounded device-side wait ran out; results are not valid */
    QS_EUNSUPPORTED = 5   /* valid request outside what this build implements */
} qs_status;

/* Gate kinds.  Matrices (arXiv 2406.14084 names the gates in Table 1; the matrices are the
 * standard ones, RZZ's half angle is fixed by the fused-diagonal values printed in the
 * artifact appendix):
 *   H, X, Y, Z, S = diag(1,i), SDG, T = diag(1,e^{i pi/4}), TDG,
 *   RX/RY/RZ(t) = exp(-i t/2 P), P(l) = diag(1,e^{il}),
 *   U3(t,f,l) = [[cos t/2, -e^{il} sin t/2], [e^{if} sin t/2, e^{i(f+l)} cos t/2]],
 *   CX = X on t[0] controlled by c[0] (nt = 1, nc >= 1),
 *   CZ, CP(l) = diag(1,1,1,e^{il}), SWAP, RZZ(t) = exp(-i t/2 Z(x)Z) on (t[0], t[1]),
 *   UNITARY: 2^nt x 2^nt complex matrix m, row-major, interleaved (re, im) doubles,
 *   DIAG:    2^nt complex diagonal entries m.
 * The local matrix index has bit j equal to qubit t[j].  Any gate may have extra controls
 * c[0..nc-1]: it then acts only on amplitudes whose control bits are all 1 (Eq. 3). */
typedef enum {
    QS_H = 0, QS_X, QS_Y, QS_Z, QS_S, QS_SDG, QS_T, QS_TDG, QS_RX, QS_RY, QS_RZ, QS_P, QS_U3,
    QS_CX, QS_CZ, QS_CP, QS_SWAP, QS_RZZ, QS_UNITARY, QS_DIAG, QS_NUM_KINDS
} qs_kind;

#define QS_MAX_QUBITS 36
#define QS_MAX_TARGETS 7
#define QS_MAX_CONTROLS 8

/* One gate.  Caller-owned; the library copies what it needs during the call. */
typedef struct {
    int32_t kind;                  /* qs_kind */
    int32_t nt, nc;                /* number of targets (1..7), controls (0..8) */
    int32_t t[QS_MAX_TARGETS];     /* target qubits, t[0] = LSB of the local matrix index */
    int32_t c[QS_MAX_CONTROLS];    /* control qubits */
    double p[3];                   /* angles in radians (theta, phi, lambda) */
    const double *m;               /* UNITARY / DIAG entries (host memory), else NULL */
} qs_gate;

/* Pauli string term: coeff * (prod over xmask of X) (prod over zmask of Z) with Y where both
 * bits are set, i.e. P|x> = i^{#Y} (-1)^{popcount(x & zmask)} |x ^ xmask>. */
typedef struct {
    double coeff;
    uint64_t xmask, zmask;
} qs_pauli_term;

typedef enum { QS_PLANNER_GREEDY = 0, QS_PLANNER_LEARNED = 1 } qs_planner;
typedef enum { QS_TC_OFF = 0, QS_TC_TF32X3 = 1, QS_TC_BF16X3 = 2 } qs_tc_mode;
typedef enum { QS_SLAB_GATHER = 0, QS_SLAB_REMAP = 1 } qs_slab_mode;

/* Planning options.  Fill with qs_options_default() and override fields. */
typedef struct {
    int32_t fuse_width;  /* k: widest dense fused gate (0 = no fusion: gates applied as given) */
    int32_t blocking;    /* 1 = slab-blocked passes (Alg. 3), 0 = one full pass per gate */
    int32_t slab_bits;   /* b: qubits per on-chip slab, 0 = automatic */
    int32_t seg_bits;    /* low physical bits always inside a slab (contiguous segment), 0 = auto */
    int32_t slab_mode;   /* qs_slab_mode: gather slabs at any bit positions, or the paper's
                            low-block slabs plus explicit remap passes (Alg. 4) */
    int32_t planner;     /* qs_planner */
    int32_t tc;          /* qs_tc_mode: tensor-core path for wide fused gates (complex64 only) */
    int32_t tc_width;    /* qubits per tensor-core fused gate: 6 or 7 */
    int32_t graph;       /* 1 = replay the plan's launches from a captured CUDA graph */
    int32_t diag_bits;   /* widest fused diagonal table (qubits), 0 = automatic */
    int32_t dtype;       /* qs_dtype the plan's cost model targets (qs_apply_circuit sets it
                            from the state) */
    int32_t stage_bits;  /* register-stage width: slab bits held in registers per thread
                            (complex64: 4 or 5, complex128: 3 or 4; 0 = automatic) */
    int32_t reserved[4];
} qs_options;

/* Plan summary (qs_plan_info). */
typedef struct {
    int32_t n;
    int32_t passes;        /* slab passes carrying gates */
    int32_t remaps;        /* standalone remap passes */
    int32_t unblocked;     /* full-state single-op passes */
    int32_t tc_gates;      /* tensor-core fused gates */
    int32_t ops;           /* device ops after fusion */
    int32_t input_gates;   /* gates given to qs_fuse */
    int32_t slab_bits, seg_bits;
    double flops_per_amp;  /* modelled arithmetic per amplitude, summed over the plan */
    int64_t device_bytes;  /* bytes the plan uploads to the device (descriptors + coefficients)
                              for a complex128 state; half the coefficient bytes for complex64 */
    int32_t stages;        /* register stages over all passes */
    int32_t stage_ops;     /* ops executed inside register stages */
    int32_t smem_ops;      /* ops executed directly on the shared-memory slab */
    int32_t stage_bits;    /* register-stage width */
} qs_plan_info;

/* Per-state counters, accumulated since creation or the last qs_stats_reset.  The *_ms fields
 * are device times measured with CUDA events on the state's stream around every launch while
 * profiling is on (qs_set_profiling); reading them synchronises that stream. */
typedef struct {
    int64_t passes, remaps, unblocked, tc_gates, plans_applied;
    int64_t bytes_moved;   /* algorithmic HBM bytes (read + write) of the applied passes */
    double pass_ms, remap_ms, unblocked_ms, tc_ms;
    int64_t timed_launches;
} qs_stats_t;

typedef struct qs_state qs_state; /* opaque */
typedef struct qs_plan qs_plan;   /* opaque */

/* ------------------------------------------------------------------------- state */

/* Allocate a 2^n state on the current CUDA device, initialised to |0..0>.  n in [1, 36].
 * The library owns the memory; qs_destroy frees it.  QS_ENOMEM if the device is too small. */
qs_status qs_create(int n, qs_dtype dt, qs_state **out);

/* Wrap caller-owned device memory (2^n amplitudes of dt, 256-byte aligned) without copying or
 * initialising it.  stream may be NULL (legacy default stream).  The memory must outlive the
 * state; qs_destroy does not free it. */
qs_status qs_create_from_buffer(int n, qs_dtype dt, void *dev, void *stream, qs_state **out);

qs_status qs_destroy(qs_state *s);

/* Set the CUDA stream (cudaStream_t) for all later work on this state. */
qs_status qs_set_stream(qs_state *s, void *stream);

/* Set the state to the computational basis state |x> (logical order) and reset the layout. */
qs_status qs_set_basis(qs_state *s, uint64_t x);

/* Copy amplitudes [first, first+count) in logical order to / from host memory (interleaved
 * (re, im) in the state's precision).  Restores the identity layout first if needed. */
qs_status qs_copy_to_host(qs_state *s, uint64_t first, uint64_t count, void *host);
qs_status qs_copy_from_host(qs_state *s, uint64_t first, uint64_t count, const void *host);

/* Device pointer of the amplitudes and the current physical layout: phys_of[q] is the
 * physical bit of logical qubit q (n entries). */
qs_status qs_get_buffer(qs_state *s, void **dev, int *phys_of);

/* Apply one remap pass that restores the identity layout (Sec. V-B in-memory swap). */
qs_status qs_canonicalize(qs_state *s);

/* Wait for all work queued on the state's stream. */
qs_status qs_sync(qs_state *s);

/* ------------------------------------------------------------------------- planning */

void qs_options_default(qs_options *o);

/* Build a plan for an n-qubit circuit: canonicalise the gates (FP64 matrices), fuse them
 * (FP64 products; same-qubit runs, diagonal runs, dense k-qubit blocks with k = fuse_width,
 * following the fusion level of Alg. 2), and partition the result into slab passes and
 * remaps (Alg. 1 findGBs with chunkSize = slab bits).  The plan does not depend on state
 * contents and can be applied to any state with the same n.  Caller frees it with
 * qs_plan_destroy. */
qs_status qs_fuse(const qs_gate *g, size_t ng, int n, const qs_options *o, qs_plan **out);
qs_status qs_plan_destroy(qs_plan *p);
qs_status qs_plan_info_get(const qs_plan *p, qs_plan_info *out);

/* Text listing of a plan in physical bit positions, in the spirit of the optimized-circuit
 * files of the paper's artifact appendix (gate blocks, SQS swaps, D<k> diagonal gates).
 * One item per line:
 *   N <n>
 *   PASS <b> <lo> <hi positions...>        a slab pass; the OP lines that follow belong to it
 *   UNBLOCKED                              the single OP line that follows is a full-state pass
 *   REMAP <k> <A_1..A_k> <B_1..B_k>        exchange physical positions A_j <-> B_j
 *   OP <DENSE|DIAG|PERMX|SWAP> <k> t <positions...> c <positions...> [m <re im ...>]
 *      DENSE: 2^k x 2^k row-major matrix; DIAG: 2^k entries, table bit j = position t[j]
 *   LAYOUT <physical position of logical qubit 0..n-1>
 * Writes at most cap bytes (NUL-terminated) to buf; *needed receives the full length + 1.
 * Host only: needs no GPU. */
qs_status qs_plan_dump(const qs_plan *p, char *buf, size_t cap, size_t *needed);

/* Apply a plan to a state (Alg. 3: for each gate block, remap or apply to every slab). */
qs_status qs_apply_plan(qs_state *s, const qs_plan *p);

/* qs_fuse + qs_apply_plan + qs_plan_destroy. */
qs_status qs_apply_circuit(qs_state *s, const qs_gate *g, size_t ng, const qs_options *o);

/* Swap physical bit positions A[j] <-> B[j] (j < k) in one in-place pass (Alg. 4 analogue),
 * updating the layout so that readouts stay in logical order. */
qs_status qs_remap(qs_state *s, int k, const int *A, const int *B);

/* ------------------------------------------------------------------------- readouts */

/* ||psi||^2, accumulated in FP64 (complex64 states: FP32 partial sums of <= 32 terms). */
qs_status qs_norm2(qs_state *s, double *host_out);

/* Marginal probabilities over logical qubits q[0..nq-1] (nq <= 24): host_out[m] (2^nq
 * doubles) is the probability that qubit q[j] reads bit j of m.  Synchronises. */
qs_status qs_probs(qs_state *s, const int *qubits, int nq, double *host_out);

/* Allocation-free marginal probabilities (the paper has no counterpart; this is a library
 * service).  Some callers cannot allocate device memory at the moment they need a readout: a
 * framework whose caching allocator already owns all device memory, a fixed memory arena
 * budgeted up front, or a code path that must not call cudaMalloc / cudaFree (both may
 * synchronise or fail).  This entry point uses no allocation of any kind: its histogram lives
 * in one fixed device array of 2^14 doubles (128 KiB) that every GPU loading the library holds
 * until the process exits.
 *   dev_amp:   caller-owned device buffer of 2^n amplitudes of dt, read only; indices are
 *              physical (no qubit layout is applied), 16-byte aligned.
 *   qubits:    nq distinct physical bit positions, 0 <= nq <= 14 (QS_EINVAL beyond that);
 *              host_out[m] (2^nq doubles, host) = probability that bit qubits[j] reads bit j
 *              of m.
 *   stream:    cudaStream_t to run on (NULL = legacy default stream); synchronised on return.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Every call uses
 * the same array and overwrites the previous call's histogram (the bins used are cleared
 * first), so calls that overlap on the GPU (different streams or host threads at once) race
 * and must be serialised by the caller. */
qs_status qs_probs_noalloc(const void *dev_amp, int n, qs_dtype dt, const int *qubits, int nq,
                           void *stream, double *host_out);

/* host_out[0] = Re sum_t coeff_t <psi|P_t|psi>, host_out[1] = its imaginary part (zero up to
 * rounding for Hermitian sums).  FP64 accumulation.  Synchronises. */
qs_status qs_expect_pauli_sum(qs_state *s, const qs_pauli_term *terms, size_t nterms,
                              double *host_out);

/* ------------------------------------------------------------------------- batches */

/* Many independent circuits of uneven qubit counts and depths simulated together.  Each
 * circuit's gates are planned into slab passes as in qs_fuse (gather slabs); all passes of all
 * circuits then run in ONE persistent kernel launch whose CTAs take (circuit, pass, slab)
 * work items from a queue in dependency order, waiting (bounded) for a circuit's previous pass
 * to be stored before starting its next one.  A circuit whose state fits one slab (n <= slab
 * bits) runs entirely in shared memory.  The first pass prepares |0..0> in place; the last one
 * also accumulates the circuit's expectation value.  qs_apply_batch replays the launch from a
 * captured CUDA graph when options.graph is set.  Not in the paper (a library service). */
typedef struct qs_batch qs_batch;

typedef struct {
    int32_t circuits;
    int32_t items;          /* slab work items per run */
    int32_t rounds;         /* passes of the deepest circuit */
    int32_t slab_bits;      /* slab size limit in use */
    int32_t stage_bits;     /* register-stage width in use */
    int32_t graph;          /* 1 when runs replay a captured CUDA graph */
    int64_t state_bytes;    /* device memory held for the circuits' states */
    double last_run_ms;     /* device time of the last qs_apply_batch launch sequence */
    int64_t plan_bytes;     /* host-to-device bytes of the plan upload (ops, stages, items, tables) */
} qs_batch_info;

/* Plan ncirc circuits (circuit c: n[c] qubits, gates[c][0..ngates[c]) ) and allocate their
 * states on the current device.  options: dtype, slab_bits (0 = automatic), stage_bits,
 * fuse_width and graph are honoured; blocking is always on and tc must be off.
 * QS_ENOMEM if the states do not fit. */
qs_status qs_batch_create(int ncirc, const int *n, const qs_gate *const *gates, const size_t *ngates,
                          const qs_options *o, qs_batch **out);

/* Run every circuit from |0..0> and write host_out[c] = sum_t coeff_t <psi_c|Z_t|psi_c> for the
 * Z-string terms (xmask must be 0); a term with a Z bit at or above n[c] is left out for
 * circuit c.  Synchronises.  QS_ETIMEOUT if a dependency wait ran out (results invalid). */
qs_status qs_apply_batch(qs_batch *b, const qs_pauli_term *terms, size_t nterms, double *host_out);

/* Autotuner: time the batch with each candidate (slab bits x stage width), keep the fastest.
 * *chosen_slab_bits (may be NULL) receives the chosen slab size. */
qs_status qs_batch_tune(qs_batch *b, const qs_pauli_term *terms, size_t nterms, int *chosen_slab_bits);

qs_status qs_batch_info_get(const qs_batch *b, qs_batch_info *out);
qs_status qs_batch_destroy(qs_batch *b);

/* ------------------------------------------------------------------------- misc */

qs_status qs_stats(qs_state *s, qs_stats_t *out);

/* Turn per-launch CUDA-event timing on (1) or off (0) for this state. */
qs_status qs_set_profiling(qs_state *s, int on);
qs_status qs_stats_reset(qs_state *s);

/* Message for the last failed call on this thread ("" if none). */
const char *qs_last_error(void);

/* Library version string. */
const char *qs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QS_ABI_INCLUDED_H_ */
