// planner.h -- host-side planning: gate canonicalisation, FP64 fusion, gate-block finding.
#pragma once

#include <complex>
#include <string>
#include <vector>

#include "qs_internal.h"

namespace qs {

using cd = std::complex<double>;

// Canonical gate: the gate's own qubits, its controls and an FP64 matrix.
enum CClass : int { C_DENSE = 0, C_DIAG = 1, C_PERMX = 2, C_SWAP = 3 };

struct CGate {
    CClass cls = C_DENSE;
    std::vector<int> tq;  // targets; DIAG: table qubits; tq[0] = LSB of the local index
    std::vector<int> cq;  // controls
    std::vector<cd> m;    // DENSE: D x D row-major; DIAG: D entries; PERMX/SWAP: empty
    int nsrc = 1;         // input gates merged into this one
};

// Kinds of plan steps.
enum StepKind : int { S_PASS = 0, S_REMAP = 1, S_UNBLOCKED = 2, S_TC = 3 };

struct Step {
    StepKind kind;
    int index;  // S_PASS/S_REMAP: pass index; S_UNBLOCKED: op index; S_TC: tc gate index
};

// A wide fused gate for the tensor-core path: the amplitudes are viewed as rows of 2^k
// values over the k lowest physical bits; the gate acts on those bits.
struct TcGate {
    int k;
    std::vector<cd> m;  // 2^k x 2^k row-major, acting on physical bits 0..k-1
};

struct Plan {
    int n = 0;
    qs_dtype dt = QS_C64;        // precision the plan's register stages are laid out for
    int stage_bits = 0;          // register-stage width (bits per thread group)
    qs_options opt{};
    std::vector<Step> steps;
    std::vector<DevPass> passes;
    std::vector<DevOp> ops;
    std::vector<DevStage> stages;
    std::vector<DevSub> subs;
    std::vector<DevTc> tcs;                 // tensor-core steps
    std::vector<unsigned char> tc_images;   // their E_hi / E_lo operand images
    std::vector<uint32_t> tc_coef;          // FP64 matrix of each tensor-core step (for listings)
    std::vector<std::vector<int>> tc_phys;  // physical target positions of each step
    std::vector<cd> coef;        // matrices, tables and scalars, FP64
    std::vector<TcGate> tc;
    std::vector<int> final_phys_of;  // logical -> physical after the plan
    int input_gates = 0;
    int fused_ops = 0;
    double flops_per_amp = 0.0;
    int slab_bits = 0, seg_bits = 0;
};

// Convert and validate API gates.  Returns QS_OK or QS_EINVAL with a message.
int canonicalize(const qs_gate *g, size_t ng, int n, std::vector<CGate> &out, std::string &err);

// Full planning: fusion + gate-block finding + device-op construction.
int build_plan(const std::vector<CGate> &gates, int n, qs_dtype dt, const qs_options &opt,
               Plan &plan, std::string &err);

// Remap passes that take layout `phys_of` (logical -> physical) to the identity.
void plan_canonicalize(int n, qs_dtype dt, const std::vector<int> &phys_of, Plan &plan);

// Remap pass exchanging physical positions A[j] <-> B[j].
int plan_remap(int n, qs_dtype dt, const std::vector<int> &A, const std::vector<int> &B, Plan &plan,
               std::string &err);

// Analytic per-amplitude cost of one op, in FP32-FMA-equivalents (greedy planner's model).
double op_cost(const CGate &g, qs_dtype dt);

// Append one row of QS_PLAN_FEATURES numbers per plan step (learned.cpp).
void plan_features(const Plan &p, std::vector<float> &rows);

// Default slab and segment bits for a dtype.
int default_slab_bits(qs_dtype dt);
int default_seg_bits(qs_dtype dt);

}  // namespace qs
