// qs_internal.h -- types shared by the host planner (C++) and the device kernels (CUDA).
//
// A plan is a list of steps.  Each step is one full pass over the state in HBM:
//   PASS       a slab pass (gate block, Alg. 3 of arXiv 2406.14084): every CTA loads one
//              slab of 2^b amplitudes -- the low `lo` physical bits (a contiguous segment) plus
//              b-lo further physical bit positions -- applies the block's ops in shared memory,
//              and stores the slab back, optionally relabelling bits inside the slab;
//   REMAP      a slab pass with no ops whose store permutation exchanges bit positions
//              (the in-memory swap of Sec. V-B, Alg. 4);
//   UNBLOCKED  one op applied directly to the whole state in global memory (gate-by-gate);
//   TC         a wide fused gate applied as a tensor-core GEMM (complex64 only).
#pragma once

#include <cstddef>
#include <cstdint>

#include "qs.h"

namespace qs {

enum OpType : uint8_t {
    OP_DENSE = 0,  // 2^k x 2^k complex matrix on k local target bits
    OP_DIAG = 1,   // diagonal table over local bits t[0..k) and outer bits outpos[0..nout)
    OP_PERMX = 2,  // X on one local bit (swap of amplitude pairs), no arithmetic
    OP_SWAP = 3,   // exchange of two local bits on the amplitudes where controls hold
    OP_PHASE = 4,  // multiply by one complex scalar where all cmask bits are 1
};

constexpr int kMaxSlabBits = 15;    // 2^15 complex64 = 256 KiB; the kernel limit is smem
constexpr int kMaxDense = 5;        // widest dense op on the SIMT path
constexpr int kMaxDiagBits = 12;    // widest diagonal table (local + outer qubits)
constexpr int kMaxIns = 24;         // bit positions inserted when enumerating op groups

// One operation.  In a PASS the bit indices are slab-local (0..b-1) except outpos/ocmask,
// which are physical positions outside the slab.  In an UNBLOCKED step every index is a
// physical position of the full state.
struct DevOp {
    uint8_t type;
    uint8_t k;        // DENSE: #targets; DIAG: #local table bits; PERMX: 1; SWAP: 2; PHASE: 0
    uint8_t nins;     // #positions in ins[]
    uint8_t nout;     // DIAG: #outer table bits
    uint8_t t[8];     // target bits (table bits for DIAG), t[0] = LSB of the matrix/table index
    uint8_t ins[kMaxIns];     // ascending positions forced to 0 (targets) or 1 (controls)
    uint8_t outpos[kMaxDiagBits];  // DIAG: physical positions of table bits k..k+nout-1
    uint32_t mat;     // offset of the matrix / table / scalar in the plan's coefficient pool
    uint32_t pad;
    uint64_t cmask;   // control bits (same index space as t) that must be 1
    uint64_t ocmask;  // PASS only: physical control bits outside the slab that must be 1
};

struct DevPass {
    int32_t b;         // slab bits
    int32_t lo;        // low contiguous physical bits (segment = 2^lo amplitudes)
    int32_t nhi;       // b - lo
    int32_t op_begin;  // ops [op_begin, op_end) of the plan's op array
    int32_t op_end;
    int32_t has_perm;  // store with perm[]
    uint8_t hipos[32]; // physical positions of local bits lo..b-1, ascending
    uint8_t perm[32];  // local bit j of the loaded slab is stored at local bit perm[j]
};

// Register stage: ops whose non-diagonal bits all lie in `r` slab-local bits ("register bits")
// run in registers.  Each thread loads the 2^r amplitudes of one group (all register-bit
// combinations at fixed values of the other local bits) from shared memory, applies every
// sub-op of the stage, and stores them back: one shared-memory round trip per stage instead of
// one per op.  A plan op of type OP_STAGE points at one DevStage (field mat = stage index).
constexpr int kStageBitsC64 = 5;   // 32 complex64 amplitudes per thread (64 registers)
constexpr int kStageBitsC128 = 4;  // 16 complex128 amplitudes per thread (64 registers)
constexpr uint8_t OP_STAGE = 5;

enum SubType : uint8_t {
    SB_G1 = 0,     // 2x2 matrix on register bit j0
    SB_G2 = 1,     // 4x4 matrix on register bits j0 < j1 (matrix index bit 0 <-> j0)
    SB_X = 2,      // X on register bit j0
    SB_SWAP = 3,   // exchange of register bits j0, j1
    SB_PHASE = 4,  // multiply by coef[mat] where all masked bits are 1 (controlled phase)
    SB_DIAG = 5,   // diagonal table expanded over all register bits (see DevSub)
    SB_G1R = 6,    // 2x2 matrix with real entries on register bit j0
    SB_G1N = 7,    // real [[1, x], [y, 1]] on register bit j0 (coef[mat] = x, coef[mat + 1] = y)
    SB_G1A = 8,    // real [[x, 1], [1, y]] on register bit j0 (coef[mat] = x, coef[mat + 1] = y)
    SB_G1NM = 9,   // real [[1, x], [y, -1]] on register bit j0
    SB_G1AM = 10,  // real [[x, 1], [-1, y]] on register bit j0
};

// 48 bytes, 16-byte aligned: the kernels fetch the first 24 bytes with one 16-byte and one
// 8-byte load (the byte order of the first word -- type, j0, j1, ndl -- is relied upon).
struct alignas(16) DevSub {
    uint8_t type;
    uint8_t j0, j1;
    uint8_t ndl;       // SB_DIAG: non-register table bits
    uint32_t scm;      // register bits that must be 1 (controls / phase bits)
    uint32_t lcm;      // slab-local non-register bits that must be 1
    uint32_t mat;      // coefficient offset (matrix, scalar, or expanded table)
    uint64_t ocm;      // physical bits outside the slab that must be 1
    // SB_DIAG: the table holds 2^(r + ndl) entries, index = (hi << r) | e where e is the
    // register index and bit j of hi comes from slab-local bit dl[j] (dl[j] < 0x80) or from
    // physical bit (dl[j] & 0x7f) outside the slab (dl[j] >= 0x80).
    uint8_t dl[12];
    uint8_t pad[4];
};
static_assert(sizeof(DevSub) == 48, "DevSub layout");

struct DevStage {
    uint8_t r;          // register bits
    uint8_t nrest;      // non-register slab-local bits
    uint8_t sbits[6];   // slab-local position of register bit j
    uint8_t rest[16];   // non-register slab-local bits; group index bit j -> rest[j]
    uint16_t off[32];   // slab-local offset of register index e
    int32_t sub_begin, sub_end;
};

int num_sms();

// Tensor-core wide gate (complex64 states).  A TC step is a slab pass over slabs of 2^13
// amplitudes whose local bits are 6 target bits (tpos, the K index of the GEMM) and 7 row bits
// (mpos, the M index).  The operand images are the real embedding of the 64x64 unitary split
// into hi and lo parts, pre-laid-out on the host in the 128-byte-swizzled K-major layout of the
// tensor-core shared-memory descriptors.  A 7-qubit gate (width 7) puts its 7th target on row
// bit 6 (mpos[6]) and carries four such images, one per 64x64 block U[t' 64 + j'][t 64 + j]
// (t', t = the 7th target bit of output and input), in the order (t', t) = 00, 01, 10, 11.
constexpr int kTcTargets = 6;
constexpr int kTcSlabBits = 13;
constexpr int kTcRows = 128;    // GEMM M per slab
constexpr int kTcK = 128;       // real K = N = 2 * 2^6
struct DevTc {
    DevPass slab;                // slab definition (b = 13, lo, hipos); perm/op fields unused
    uint8_t tpos[8];             // slab-local bit of target j (GEMM column bit j)
    uint8_t mpos[8];             // slab-local bit of row-index bit j
    uint32_t img;                // byte offset of this gate's operand images
    int32_t mode;                // QS_TC_BF16X3 or QS_TC_TF32X3
    int32_t width;               // 6 or 7 targets
};
size_t tc_image_bytes(int mode, int width);  // bytes of the hi+lo B images of one gate

// Launch entry points implemented in the .cu files (host side, stream-ordered).
// `coef` points to the plan's coefficient pool already converted to the state precision.
struct LaunchCtx {
    void *amp;
    int n;
    qs_dtype dt;
    void *stream;  // cudaStream_t
};

struct PassArgs {
    const DevPass *pass;      // device
    const DevOp *ops;         // device, whole plan
    const DevStage *stages;   // device, whole plan
    const DevSub *subs;       // device, whole plan
    const void *coef;         // device, whole plan, state precision
    int stage_bits;           // register-stage width the plan was built for
    const void *coef_df;      // device, whole plan, double-float quadruples (or NULL)
    bool df;                  // complex128 pass of register stages only, in double-float form
};
int launch_pass(const LaunchCtx &c, const PassArgs &a, const DevPass &h_pass, char *err,
                size_t errlen);
// Device status word written by bounded waits that ran out (0 = fine).  Reading clears it.
int read_device_status(void *stream, int *status);
int *device_status_ptr();  // its device address on the current device

int launch_tc(const LaunchCtx &c, const DevTc *d_tc, const DevTc &h_tc, const void *d_images,
              char *err, size_t errlen);

// Batched circuits (k_batch.cu).
struct BatchCirc {
    uint64_t amp_off;   // first amplitude of this circuit's state in the batch buffer
    int32_t n, npass;   // qubits, slab passes
    int32_t pass0;      // its first pass in the concatenated pass array
    int32_t nslab_log;  // log2(slabs per pass)
    int32_t term0, nterm;  // its Z terms (physical masks) in the term array
    int32_t done0;      // its first per-pass done counter
    int32_t pad;
};
struct BatchItem {
    int32_t circ, pass;
    uint32_t slab;      // first slab of the run
    int32_t count;      // consecutive slabs in the run (>= 1)
};
struct BatchTerm {
    uint64_t zm;        // physical Z mask
    double c;           // coefficient
};
struct BatchArgs {
    const BatchCirc *circs;
    const BatchItem *items;
    unsigned nitems;
    const DevPass *passes;
    const DevOp *ops;
    const DevStage *stages;
    const DevSub *subs;
    const void *coef;
    const BatchTerm *terms;
    unsigned *done;     // per circuit per pass: slabs stored (zeroed before each run)
    unsigned *head;     // work-queue head (zeroed before each run)
    double *results;    // per circuit expectation (zeroed before each run)
    int *status;        // device status word
};
int launch_batch(qs_dtype dt, int stage_bits, void *states, const BatchArgs &a, int b_max, void *stream,
                 char *err, size_t errlen);
int launch_unblocked(const LaunchCtx &c, const DevOp *d_op, const DevOp &h_op,
                     const void *d_coef, char *err, size_t errlen);
size_t pass_smem_bytes(qs_dtype dt, int b, int lo);
int max_slab_bits(qs_dtype dt);

// Reductions (k_reduce.cu).  Scratch is a device buffer of at least reduce_scratch_bytes().
size_t reduce_scratch_bytes();
int launch_norm2(const LaunchCtx &c, double *d_scratch, double *h_out, char *err, size_t errlen);
int launch_probs(const LaunchCtx &c, const int *phys_q, int nq, double *d_scratch,
                 size_t scratch_bytes, double *h_out, char *err, size_t errlen);
int launch_expect(const LaunchCtx &c, const uint64_t *xm, const uint64_t *zm,
                  const double *coeff, size_t nterms, double *d_scratch, size_t scratch_bytes,
                  double *h_out, char *err, size_t errlen);
int launch_set_basis(const LaunchCtx &c, uint64_t x, char *err, size_t errlen);

// Measurement sampling (k_sample.cu): d_out[k] = outcome of uniform d_u[k]; the scratch must
// hold sample_scratch_bytes(n); the total weight is left at double index sample_total_index(n).
size_t sample_scratch_bytes(int n);
size_t sample_total_index(int n);
int launch_sample(const LaunchCtx &c, const double *d_u, uint64_t shots, uint64_t *d_out, void *d_scratch,
                  char *err, size_t errlen);

// Marginal probabilities with a fixed file-scope device histogram instead of allocated scratch
// (qs_probs_noalloc).  nq <= kStaticProbsMaxQubits.
constexpr int kStaticProbsMaxQubits = 14;
int launch_probs_static(const LaunchCtx &c, const int *phys_q, int nq, double *h_out, char *err,
                        size_t errlen);

// Cost-model network (k_mlp.cu): 3-layer perceptron, FP32, hidden width kMlpHidden.
constexpr int kMlpHidden = 128;
constexpr int kMlpMaxFeatures = 32;
struct MlpArgs {
    const float *X;       // B x F inputs (raw; standardised on load)
    const float *T;       // B targets (raw; standardised on use), training only
    int B, F;
    float *params;        // flat [W1 | b1 | W2 | b2 | W3 | b3]
    const float *mu;      // F feature means
    const float *inv_sd;  // F reciprocal feature spreads
    float ym, ys, inv_ys; // target mean, spread, 1/spread
    float scale;          // training: 2 / B (derivative of the mean squared error)
    float *y_out;         // forward: B predictions (de-standardised)
    float *partial;       // training: tiles x pstride partial gradients
    int pstride, nparams;
    int *step_counter;    // Adam step t (advanced once per training step), or NULL
    float *grad_out;      // gradient output when not updating
    float *loss_out;      // mean squared error (standardised space) of the batch
    float *adam_m, *adam_v;
};
int mlp_param_count(int F);
int mlp_tiles(int B);
int launch_mlp_forward(const MlpArgs &a, void *stream, char *err, size_t errlen);
int launch_mlp_train_step(const MlpArgs &a, int update, float lr, void *stream, char *err, size_t errlen);

}  // namespace qs
