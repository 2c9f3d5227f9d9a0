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
/* Tensor-core modes for fused 6- and 7-qubit gates on complex64 states: split precision with three
 * products (hi*hi + hi*lo + lo*hi) and FP32 accumulation, parts in TF32 (about 22 significant
 * bits for hi + lo) or BF16 (about 16 bits).  Not in the paper: a GB300 form of its dense gates. */
typedef enum { QS_TC_OFF = 0, QS_TC_TF32X3 = 1, QS_TC_BF16X3 = 2 } qs_tc_mode;
typedef enum { QS_SLAB_GATHER = 0, QS_SLAB_REMAP = 1 } qs_slab_mode;
/* Arithmetic of complex128 register stages.  QS_ARITH_FP64 (the default): FP64 FMAs.
 * QS_ARITH_DF: each slab is converted once per pass to double-float pairs (two FP32 numbers,
 * about 48 significant bits) and the register stages run on the FP32 pipe, which GB300 executes
 * about 64x faster than FP64; the state in HBM stays complex128, and passes with shared-memory
 * ops stay FP64.  Each operation then rounds at about 2^-46 instead of 2^-53 relative. */
typedef enum { QS_ARITH_FP64 = 0, QS_ARITH_DF = 1 } qs_arith;

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
    int32_t tc_width;    /* widest tensor-core fused gate: 6 (0 = 6) or 7; blocks of 4-6 qubits
                            are padded to 6, blocks of 7 run as four 64x64 products; any other
                            value: QS_EUNSUPPORTED */
    int32_t graph;       /* 1 = replay the plan's launches from a captured CUDA graph */
    int32_t diag_bits;   /* widest fused diagonal table (qubits), 0 = automatic */
    int32_t dtype;       /* qs_dtype the plan's cost model targets (qs_apply_circuit sets it
                            from the state) */
    int32_t stage_bits;  /* register-stage width: slab bits held in registers per thread
                            (complex64: 4 or 5, complex128: 3 or 4; 0 = automatic) */
    int32_t fuse_force;  /* 1 = merge dense runs up to fuse_width even where the analytic
                            cost model says the wider gate costs more (a learned-planner
                            candidate); 0 = merge only where the model says it pays */
    int32_t euler;       /* blocked plans: write complex 1-qubit gates as phase, real rotation,
                            phase (Z-Y-Z) so that register stages merge the phases.  0 or 2 =
                            split (the default), 1 = keep complex 2x2 matrices */
    int32_t factor;      /* register stages: write each real 2x2 gate M as D N, N with two unit
                            entries (one FMA per real output instead of two) and D diagonal
                            (folded into the stage's diagonal tables).  0 = on (the default),
                            1 = off */
    int32_t merge_bits;  /* register stages: most condition bits (slab or outer qubits) one merged
                            diagonal table may read besides the register bits; 0 = automatic (10
                            for complex128 stages in FP64, else 6), at most 10 (tables of
                            2^(stage_bits + merge_bits) entries) */
    int32_t arith;       /* qs_arith: arithmetic of complex128 register stages */
    int32_t reserved[3];
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
    /* learned planner (qs_fuse_learned); zero for greedy plans */
    int32_t learned;       /* 1 when the plan came from the learned planner */
    int32_t candidates;    /* candidate plans scored by the cost model */
    int32_t chosen;        /* index of the chosen candidate, -1 = the greedy plan itself */
    int32_t judge_state;   /* 0/1: next apply times the learned/greedy plan; 2: settled */
    double predicted_ms;         /* model's device-time prediction of the chosen plan */
    double greedy_predicted_ms;  /* ... and of the greedy plan */
    double judge_ms_learned;     /* measured device time of the first learned apply (0 = none) */
    double judge_ms_greedy;      /* measured device time of the first greedy apply (0 = none) */
    int32_t using_greedy;  /* 1 once the judge found the greedy plan faster */
    int32_t pad_;
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
 *   dev_amp:   caller-owned buffer of 2^n amplitudes of dt in device (or managed) memory of
 *              the current device, read only; indices are physical (no qubit layout is
 *              applied), 16-byte aligned.  A host pointer or another device's memory gives
 *              QS_EINVAL before any launch (cudaPointerGetAttributes); the buffer's size cannot
 *              be checked and must cover 2^n amplitudes.
 *   qubits:    nq distinct physical bit positions, 0 <= nq <= 14 (QS_EINVAL beyond that);
 *              host_out[m] (2^nq doubles, host) = probability that bit qubits[j] reads bit j
 *              of m.
 *   stream:    cudaStream_t to run on (NULL = legacy default stream); synchronised on return.
 *              The call copies into pageable host memory and synchronises, so it may never run
 *              while that stream is being captured: QS_EINVAL then.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current.  Every call uses
 * the same array and overwrites the previous call's histogram (the bins used are cleared
 * first), so calls that overlap on the GPU (different streams or host threads at once) race
 * and must be serialised by the caller. */
qs_status qs_probs_noalloc(const void *dev_amp, int n, qs_dtype dt, const int *qubits, int nq,
                           void *stream, double *host_out);

/* Measurement sampling in the computational basis (Born rule: outcome x with probability
 * |a_x|^2 / ||psi||^2, Eq. 1).  For each caller-supplied uniform u[k] in [0, 1) (the caller's
 * random numbers; the library draws none), host_out[k] receives the smallest logical index x
 * whose running weight sum_{y <= x} |a_y|^2 exceeds u[k] ||psi||^2 (inverse transform sampling,
 * in logical qubit order).  shots <= 2^28.  QS_EINVAL for a u outside [0, 1) or a zero state.
 * Synchronises; one read of the state plus one 2^8-amplitude block per shot.  Scratch: 2^(n-4)
 * bytes of block prefixes, held by the state. */
qs_status qs_sample(qs_state *s, const double *u, size_t shots, uint64_t *host_out);

/* host_out[0] = Re sum_t coeff_t <psi|P_t|psi>, host_out[1] = its imaginary part (zero up to
 * rounding for Hermitian sums).  Terms are grouped by X mask (at most 256 per group) and each
 * group costs one read of the state; groups of four or more terms on 16 or more qubits go
 * through Walsh-Hadamard tiles, so that read costs the same whatever the group's size.  FP64
 * accumulation across tiles (complex64 states: FP32 within a tile).  Synchronises. */
qs_status qs_expect_pauli_sum(qs_state *s, const qs_pauli_term *terms, size_t nterms,
                              double *host_out);

/* ------------------------------------------------------------------------- batches */

/* Many independent circuits of uneven qubit counts and depths simulated together.  Each
 * circuit's gates are planned into slab passes as in qs_fuse (gather slabs); all passes of all
 * circuits then run in ONE persistent kernel launch whose CTAs take (circuit, pass, slab)
 * work items from a queue in dependency order, waiting (bounded) for a circuit's previous pass
 * to be stored before starting its next one.  A circuit whose state fits one slab (n <= slab
 * bits) runs entirely in shared memory.  The first pass prepares |0..0> in place; the last one
 * accumulates the circuit's expectation value from a Walsh-Hadamard transform of each slab's
 * probabilities and stores nothing (the final states are not kept).  qs_apply_batch replays the launch from a
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

/* ------------------------------------------------------------ learned cost model
 *
 * Not in the paper, whose planner is the greedy one (Alg. 1-2).  A 3-layer perceptron (FP32,
 * hidden width 128, ReLU) predicts the device time of one plan step from QS_PLAN_FEATURES
 * numbers that describe it; its forward, backward and Adam kernels are the library's own.
 * The learned planner builds a grid of candidate plans (Z-Y-Z split or not, fusion width, forced or cost-checked
 * fusion, slab bits, register-stage width), scores every step of every candidate in one
 * batched forward launch, and keeps the candidate with the lowest predicted total.  The greedy
 * plan (the caller's options as given) is the fallback -- it is kept when no candidate is
 * predicted faster by more than 2% -- and the judge: a learned plan carries its greedy twin,
 * the first qs_apply_plan times the learned plan, the second times the greedy plan, and every
 * later apply uses whichever was faster.  Both compute the same circuit.
 *
 * Model target: y = ln(step_ms) - (n - 20) ln 2 (log device time per 2^20 amplitudes).
 *
 * Features of one plan step (row of qs_plan_features), in order:
 *   0 n                         1 dtype (0 = complex64, 1 = complex128)
 *   2-5 step kind one-hot: slab pass, remap pass, unblocked op, tensor-core gate
 *   6 slab bits b (unblocked: op width)   7 low segment bits   8 gathered high bits
 *   9 store permutation (0/1)  10 lowest gathered position  11 highest gathered position
 *  12 register-stage width     13 ops in the pass           14 register stages
 *  15 stage sub-ops   16 1-qubit complex   17 1-qubit real   18 2-qubit   19 phases
 *  20 diagonal tables   21 X / SWAP relabels   22 shared-memory dense ops
 *  23 sum of 2^k over shared-memory dense ops   24 other shared-memory ops
 *  25 ops with controls   26 analytic real FMAs per amplitude   27 widest dense op */
#define QS_PLAN_FEATURES 28

typedef struct qs_model qs_model;

typedef struct {
    int32_t nfeat, hidden, nparams;
    int32_t steps;       /* Adam steps taken */
    float ym, ys;        /* target standardisation */
    float last_loss;     /* mean squared error (standardised) of the last training epoch */
    int32_t pad_;
} qs_model_info;

typedef struct {
    int32_t epochs;      /* passes over the data */
    int32_t batch;       /* rows per Adam step (multiple of 32 recommended) */
    float lr;            /* Adam step size */
    int32_t fit_norm;    /* 1 = set feature / target standardisation from this data first */
    uint64_t seed;       /* row shuffle (fixed for all epochs) */
    int32_t graph;       /* 1 = replay each epoch from a captured CUDA graph */
    int32_t reserved[3];
} qs_train_options;

void qs_train_options_default(qs_train_options *o);

/* New model with nfeat inputs (<= 32), He-uniform weights from a SplitMix64 stream seeded
 * with `seed`, zero biases, identity standardisation, on the current device. */
qs_status qs_model_create(int nfeat, uint64_t seed, qs_model **out);
qs_status qs_model_destroy(qs_model *m);
qs_status qs_model_info_get(const qs_model *m, qs_model_info *out);
/* Flat FP32 parameters [W1 (nfeat x 128) | b1 | W2 (128 x 128) | b2 | W3 (128) | b3], row-major,
 * input index first.  count must equal nparams.  set resets the Adam moments and step. */
qs_status qs_model_get_params(const qs_model *m, float *host, size_t count);
qs_status qs_model_set_params(qs_model *m, const float *host, size_t count);
/* Adam's moment estimates m and v (Kingma & Ba, Algorithm 1), one per parameter in the order of
 * qs_model_get_params; both are zero after create / set_params.  count must equal nparams. */
qs_status qs_model_get_moments(const qs_model *m, float *mom, float *vel, size_t count);
/* Standardisation: inputs x' = (x - mu) / sd per feature, targets t' = (t - ym) / ys. */
qs_status qs_model_get_norm(const qs_model *m, float *mu, float *sd, float *ym, float *ys);
qs_status qs_model_set_norm(qs_model *m, const float *mu, const float *sd, float ym, float ys);
/* y[r] = model(X[r]) for host row-major X (rows x nfeat); predictions de-standardised. */
qs_status qs_model_predict(qs_model *m, const float *X, size_t rows, float *y);
/* Gradient of the mean squared error (standardised space) over the rows; grad has nparams
 * entries; *loss receives the error.  No update. */
qs_status qs_model_loss_grad(qs_model *m, const float *X, const float *T, size_t rows, float *grad,
                             float *loss);
/* Adam training on the device: rows are shuffled once, split into batches of o->batch rows
 * (the remainder is dropped when rows > batch), and each epoch takes one step per batch.
 * *final_loss (may be NULL) receives the mean batch loss of the last epoch. */
qs_status qs_model_train(qs_model *m, const float *X, const float *T, size_t rows,
                         const qs_train_options *o, float *final_loss);

/* Features of every step of a plan (rows x QS_PLAN_FEATURES, host, row-major).  *nrows receives
 * the step count; QS_EINVAL if cap_rows is smaller. */
qs_status qs_plan_features(const qs_plan *p, float *out, size_t cap_rows, size_t *nrows);
/* Apply a plan like qs_apply_plan and write each step's device time (ms, CUDA events on the
 * state's stream) to step_ms[0..steps).  Synchronises. */
qs_status qs_plan_profile(qs_state *s, const qs_plan *p, float *step_ms, size_t cap);
/* Learned planner: as qs_fuse, then choose among candidate plans with the model (see above).
 * With model NULL, or options that fix the plan (blocking off, tensor cores on), it returns
 * the greedy plan. */
qs_status qs_fuse_learned(const qs_gate *gates, size_t ngates, int n, const qs_options *o,
                          qs_model *model, qs_plan **out);
/* Process-wide model used when options.planner = QS_PLANNER_LEARNED in qs_fuse and
 * qs_apply_circuit (NULL = none: those calls plan greedily).  The caller keeps ownership. */
qs_status qs_set_cost_model(qs_model *m);

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
