// Row-0 writer, last-row reduction, amplitude finalisation and the
// whole-sweep-in-shared-memory kernel for narrow boundaries
// (arXiv 2608.13110, Sec. 3.1, Algorithm 1: B <- pi[1] is the first row's
// contraction, the loop absorbs rows 2..n, and the result is a scalar).
#pragma once

#include "tb_internal.h"

namespace tb {

struct InitParams {
    float2* B;
    int64_t b_stride;
    int h, k, m, top, n;
    int chunk_shift;   // log2(chunks per batch element) = h - k
    int64_t nchunks;   // nbatch << chunk_shift
    const uint8_t* bits;
    const float2* low;   // [2^k]
    const float2* mid;   // [2][2^m]
    const float2* topt;  // [2 (x)][2 (bit k+m-1)][2^top]
    uint32_t* maxs;      // slot 0 of each batch element
    int64_t sstride;
};

struct ReduceParams {
    const float2* B;
    int64_t b_stride;
    int h, k, m, top, n;
    int chunk_shift;     // h - k
    int blocks_per_b;
    int nbatch;
    const uint8_t* bits;
    const float2* low;   // [2^k][2] column vectors
    const float2* mid;   // [2^m][4] 2x2 matrices
    const float2* topt;  // [2 (x)][2^top][2] row vectors
    const uint32_t* maxs;
    int32_t* exps;
    int64_t sstride;
    int slot;            // slot read; slot+1 written
    double2* partials;   // [nbatch][blocks_per_b]
};

struct FinalizeParams {
    const double2* partials;
    int blocks_per_b;
    const int32_t* exps;
    int64_t sstride;
    int nslots;
    int nbatch;
    double* out;  // 2 doubles per batch element
};

struct SmallParams {
    int n, h, nb;
    const uint8_t* bits;
    const StepG* steps;
    const int8_t* tgt;
    const int8_t* ctl;
    const int16_t* xq;
    const int32_t* row_end;
    int nrows;
    const float2* init_low;  // [2^h]
    const float2* init_top;  // [2 (x)][2 (bit h-1)]
    const float2* red_low;   // [2^h][2]
    double* out;
};

// One narrow plan's share of a multi-plan launch: its blocks are
// [first_block, first_block + p.nb).
struct SmallItem {
    SmallParams p;
    int64_t first_block;
};

constexpr int REDUCE_THREADS = 256;
constexpr int MAX_RED_BLOCKS = 1024;

cudaError_t launch_init(const InitParams& p, int grid, cudaStream_t st);
cudaError_t launch_reduce(const ReduceParams& p, cudaStream_t st);
cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t st);
// log-XEB estimator of nb device amplitudes (FP64, one CTA, fixed order).
cudaError_t launch_log_xeb(const double2* amp, int64_t nb, int n, double* out, cudaStream_t st);
cudaError_t launch_small(const SmallParams& p, cudaStream_t st);
cudaError_t launch_small_multi(const SmallItem* d_items, int nitems, int64_t nblocks, int hmax, cudaStream_t st);

}  // namespace tb
