// Device kernels of an open plan (Algorithm 2): launch interface.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "tb_internal.h"

namespace tb {

constexpr int LATE_MAX_OPS = 128;  // operations of one late segment

struct JoinParams {
    float2* B;             // boundary of batch element 0 (joined in place)
    int64_t b_stride;      // entries between batch elements
    int64_t tiles_per_b;   // 2^h / JOIN_TILE
    int64_t ntiles;        // nbatch * tiles_per_b
    const float2* E;       // 2^k x 2^k early-region matrix
};

struct LateParams {
    const float2* in;      // 2 * out_entries / 2^k input rows per batch element
    int64_t in_stride;
    float2* out;           // out_entries / 2^k output rows per batch element
    int64_t out_stride;
    int64_t out_entries;
    int in_shift, out_shift;  // row r starts at entry r << (k + shift): in place, output
                              // row r' lands on input row 2r' (out_shift = in_shift + 1)
    int nbatch;
    int k;
    const OpenOp* ops;     // the segment after this crossing
    int nops;
    float2 w;              // the crossing's entangler factor (-1 for CZ)
};

struct OpenFinalParams {
    const float2* Z;       // 2^k entries per batch element
    int64_t b_stride;
    const int32_t* exps;   // rescaling exponents of the sweep
    int64_t sstride;
    int nslots;
    int k;
    double* out;           // (re, im) of 2^k amplitudes per batch element
};

// Join on the tensor cores (k >= JOIN_TC_MIN_K), out of place: Z = B.E for
// every row of every batch element (join_tc.cu).
struct JoinTcParams {
    const float* in;       // boundary of batch element 0 as (re, im) floats
    int64_t in_stride;     // complex entries between batch elements
    float* out;            // Z of batch element 0
    int64_t out_stride;
    const uint8_t* Es;     // split real embedding of E (JOIN_KC x join_nt(k) blocks)
    int KR;                // 2^(k+1): reals per row
    int64_t rows;          // rows per batch element, 2^(h-k) (a multiple of 128)
    int nbatch;
    int* fault;            // bounded waits that gave up
};

cudaError_t launch_join(int k, const JoinParams& p, int grid, cudaStream_t st);
// amap: 2-D tensor map over the rows of every batch element ([rows * nbatch]
// x [2^(k+1) floats]), box JOIN_KC floats x 128 rows, 128-byte swizzle.
cudaError_t launch_join_tc(int k, const JoinTcParams& p, const CUtensorMap& amap, int grid, cudaStream_t st);
// max_grid caps the CTAs (8 warps each, one warp per output row or per
// 2^(5-k) rows for k < 5).
cudaError_t launch_late(const LateParams& p, int max_grid, cudaStream_t st);
cudaError_t launch_open_finalize(const OpenFinalParams& p, int nbatch, cudaStream_t st);

}  // namespace tb
