// Dense tensor-core pass of the temporal-boundary sweep (precision TF32X3 /
// BF16X3): launch interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tb_internal.h"
#include "tbsweep.h"

namespace tb {

struct TcParams {
    float2* B;              // boundary of batch element 0
    int64_t b_stride;       // complex entries between batch elements
    int h, lo, n;
    int tile_shift;         // log2(tiles per batch element) = h - WB - TC_VEC_BITS
    int64_t ntiles;         // nbatch << tile_shift
    const uint8_t* mat;     // the pass's split matrix: hi part, then lo part
    const StepG* steps;     // the plan's step array
    TcStep pre, post;       // register steps around the block (t < 0: none)
    const uint8_t* bits;    // bitstring of batch element b at bits + b*n
    uint32_t* maxs;         // rescaling state as in the FP32 passes
    int32_t* exps;
    int64_t sstride;
    int slot;               // slot read; slot+1 written
    int* fault;             // incremented when a bounded wait gives up
    int selftest;           // 1: issue no MMA and give up waiting after a few tries (tests the bounded waits)
};

// precision: TB_PRECISION_TF32X3 or TB_PRECISION_BF16X3.
cudaError_t launch_tc_pass(int precision, const TcParams& p, int grid, cudaStream_t st);

// Device word counting bounded waits that gave up (all kernels of the library).
int* device_fault_word();

// Bit of a fault word raised by a tensor-core pass CTA that exited without
// seeing its last MMAs complete and therefore kept its tensor memory.
constexpr int TC_TMEM_HELD = 1 << 30;

// Record a fault word read back by the host: returns the count of waits that
// gave up; TC_TMEM_HELD disables tensor-core passes for the rest of the process.
int note_faults(int word);
// True once a tensor-core pass has kept its tensor memory (see TC_TMEM_HELD).
bool tc_passes_disabled();

}  // namespace tb
