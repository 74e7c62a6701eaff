// Host-side plan object of the temporal-boundary sweep.
#pragma once

#include <array>
#include <complex>
#include <string>
#include <vector>

#include "tb_internal.h"
#include "tbsweep.h"

namespace tb {

struct M2 {
    std::complex<double> a[4];  // row-major 2x2
};

M2 m2_mul(const M2& A, const M2& B);
M2 clifford(int k);

struct Plan {
    uint64_t uid = 0;  // unique per plan object (keys device-resident table caches)
    int n = 0, d = 0, h = 0;
    tb_opts opts{};
    std::vector<M2> U;  // (d+1)*n folded slot gates, index t*n + q
    // entangler of pair (i, i+1) in layer l: diag(1, 1, 1, W[l*(n-1) + i])
    // (-1 for CZ); entries of pairs the layer does not couple are unused
    std::vector<std::complex<double>> W;
    std::complex<double> w(int l, int i) const { return W[(size_t)l * (n - 1) + i]; }
    // paired steps of rows 1..n-2 in execution order
    std::vector<StepG> steps;
    std::vector<StepG> pass_steps;  // per pass, its steps as the pass kernel runs them (PassDesc::pstep0)
    std::vector<std::array<std::complex<double>, 16>> steps64;  // the same in FP64
    std::vector<int8_t> step_tgt, step_ctl;
    std::vector<int16_t> step_xq;
    std::vector<int32_t> row_end;
    // pass schedule (empty when the boundary fits one CTA)
    std::vector<PassDesc> passes;
    std::vector<int> windows;
    // dense tensor-core schedule (precision TF32X3 / BF16X3)
    std::vector<TcPass> tc_passes;
    std::vector<uint8_t> tc_mats;
    int tc_wb = 0;
    // open output bits (Algorithm 2): the sweep stops after row n-k-1
    int open_k = 0;
    std::vector<float2> open_E;
    std::vector<uint8_t> open_Es;  // tensor-core join operand (see JOIN_KC)
    std::vector<OpenOp> open_ops;
    std::vector<int32_t> open_seg;
    std::vector<float2> open_w;  // entangler factor w of each late crossing (-1 for CZ)
    int last_mid_row() const { return open_k ? n - open_k - 1 : n - 2; }
    int n_pass_launches() const {
        return opts.precision != TB_PRECISION_FP32 ? (int)tc_passes.size() : (int)passes.size();
    }
    // row-0 and last-row tables
    int k = 0, m = 0, top = 0;
    std::vector<float2> init_low, init_mid, init_top, red_low, red_mid, red_top;
    // Algorithm 1 counters
    int width = 0;
    double log2cost = 0;
    // device image of the tables
    TableLayout lay{};
    std::vector<uint8_t> blob;
};

uint64_t next_plan_uid();

// Early-region matrix and late-region operations of an open plan (open_plan.cpp).
int open_tables(Plan& P, std::string& err);

// Build the dense tensor-core schedule and its split matrices (tc_plan.cpp).
int tc_schedule(Plan& P, std::string& err);

int plan_build(Plan& P, int n, int d, const uint8_t* cliff, const uint8_t* tmask,
               const tb_gate1q* extra, int n_extra, const double* cphase, const tb_opts* opts,
               std::string& err);

// TF32 rounding (nearest, ties to even) and the canonical K-major operand
// offset of the tensor-core kernels (tc_plan.cpp).
float round_tf32(double v);
int64_t canon_offset(int nn, int kk, int K, int eb);

}  // namespace tb

struct tb_plan {
    tb::Plan p;
};
