// Internal definitions shared by the host planner and the CUDA kernels of
// the temporal-boundary sweep (arXiv 2608.13110, Sec. 3.1, Algorithm 1).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tb {

// Boundary passes work on tiles of 2^TILE_BITS complex64 entries (64 KB):
// the window's address bits plus enough low address bits for coalescing.
constexpr int TILE_BITS = 13;
constexpr int TILE = 1 << TILE_BITS;
constexpr int PASS_CONSUMERS = 256;   // 8 consumer warps, 32 entries per thread
constexpr int PASS_THREADS = PASS_CONSUMERS + 128;  // + one producer warpgroup (tensor copies)
constexpr int PASS_PRODUCER_REGS = 40;   // setmaxnreg split of the 168 registers per thread at launch:
constexpr int PASS_CONSUMER_REGS = 224;  // 128 x 40 + 256 x 224 <= 384 x 168
constexpr int PASS_CTAS_PER_SM = 1;
constexpr int REG_BITS = 5;           // entries per thread = 2^REG_BITS
constexpr int MIN_WINDOW = 5;
constexpr int MAX_WINDOW = 10;        // window at address bit 0 (whole tile is low bits)
constexpr int MAX_WINDOW_HIGH = TILE_BITS - 3;  // other windows keep >= 8 consecutive entries (64 B)
// Boundaries of width <= SMALL_H_MAX live in one CTA's shared memory for the
// whole sweep (one CTA per bitstring).
constexpr int SMALL_H_MAX = 12;
constexpr int SMALL_THREADS = 256;
constexpr int MAX_H = 35;        // widest boundary the device path evaluates (2^35 complex64 = 256 GiB)
// Widest open plan whose join runs out of place into a second boundary-size
// buffer (tensor cores, k >= JOIN_TC_MIN_K); wider open plans, and open plans
// whose HBM budget cannot hold the second buffer, join and cross in place.
constexpr int OPEN_OUT_OF_PLACE_MAX_H = 33;
// In place, the tensor-core join runs in slices of 2^-JOIN_SLICE_SHIFT of the
// boundary's rows (at least 128) through a scratch of one slice, each slice
// copied back over its rows (a row's product depends on that row alone).
constexpr int JOIN_SLICE_SHIFT = 6;
constexpr int MAX_PLAN_H = 40;   // widest circuit the planner accepts (counters only beyond MAX_H)

// Split of the boundary address bits used by the row-0 writer and the last
// row reduction: k low bits (table), m middle bits (table), top bits.
constexpr int LOW_BITS = 12;
constexpr int MID_BITS = 10;

// Pass shapes. A pass applies the steps of one window of address bits
// [lo, lo+M-1] (window-relative bit w <-> address bit lo+w):
//   FWD       forward row, targets w = 1..M-1, control w-1
//   REV       reversed row, targets w = M-2..0, control w+1
//   TOP       row turn at the top: FWD targets, then the next (reversed)
//             row's targets w = M-1 (no control), M-2..0 (control w+1)
//   BOT       row turn at address bit 0: REV targets w = M-2..0, then the
//             next (forward) row's w = 0 (no control), 1..M-1 (control w-1)
// At a turn the last two steps of one row and the first two of the next act
// on the two outermost window bits (BOT: bits 0, 1; TOP: bits M-2, M-1), and
// only the first of the four has its control outside them (bit 2; bit M-3).
// The pass kernels apply their product as one dense 4x4 block per value of
// that control (16 instead of 32 real multiply-adds per entry): TOP and BOT
// passes run 2M-4 steps, the block at index M-3 (pass_blk). The TOP block
// depends on the output bits of both rows (four variants, pass_xm).
//   BOT_START first window of the first absorbed row: w = 0 (no control), 1..M-1
//   BOT_END   last window of a reversed last row: w = M-2..0
//   TOP_END   last window of a forward last row: w = 1..M-1
enum PassType : int {
    P_FWD = 0,
    P_REV = 1,
    P_TOP = 2,
    P_BOT = 3,
    P_BOT_START = 4,
    P_BOT_END = 5,
    P_TOP_END = 6,
    P_NTYPES = 7,
    P_TENSOR = 7   // schedule code of a dense tensor-core pass
};

// Steps of a pass as the pass kernel runs them (turn blocks composed).
__host__ __device__ constexpr int pass_nsteps(int type, int M) {
    return type == P_TOP || type == P_BOT ? 2 * M - 4 : type == P_BOT_START ? M : M - 1;
}

// Index of a pass's 4x4 turn block (-1: none).
__host__ __device__ constexpr int pass_blk(int type, int M) {
    return type == P_TOP || type == P_BOT ? M - 3 : -1;
}

// Index of the step with four bitstring variants (the top turn's block), -1
// if none. Its variant is x_a + 2 x_b: x_a the output bit of the forward row
// (bit xs_step0 of the pass's variant mask), x_b that of the reversed row
// (bit XM_HIGH_BIT).
__host__ __device__ constexpr int pass_xm(int type, int M) { return type == P_TOP ? M - 3 : -1; }
constexpr int XM_HIGH_BIT = 31;

// A turn block in the pass-step table: BLK_ENTRIES consecutive StepG read as
// float2[4 variants][2 control values][4 rows q'][4 columns q], block index
// q = (bit t) + 2 (bit t+1).
constexpr int BLK_ENTRIES = 8;

// Pass-step table entry of step i of a pass.
__host__ __device__ constexpr int pass_entry(int type, int M, int i) {
    return pass_blk(type, M) >= 0 && i > pass_blk(type, M) ? i + BLK_ENTRIES - 1 : i;
}
__host__ __device__ constexpr int pass_entries(int type, int M) {
    return pass_nsteps(type, M) + (pass_blk(type, M) >= 0 ? BLK_ENTRIES - 1 : 0);
}

// One paired step: out[.., c, a', ..] = sum_s G[c][a'][s] in[.., c, s, ..] on
// the target bit, c the control bit (ignored for uncontrolled steps). Two
// variants: the step may depend on the output bit x_q of its row.
struct StepG {
    float2 g[2][8];  // [x variant][c*4 + a'*2 + s]
};
static_assert(sizeof(StepG) == 16 * sizeof(float2), "StepG entries are read as raw float2 arrays");

// Host-side description of one pass (launch arguments).
struct PassDesc {
    int type;
    int M;
    int lo;        // address bit of window bit 0
    int step0;     // first step in the device step array (the method's steps)
    int pstep0;    // first entry of the pass in the pass-step table
    int nsteps;    // pass_nsteps(type, M)
    int xs_step[2];  // bit of the pass's variant mask set by an output bit, -1 if none
    int xs_q[2];     // the qubit whose output bit sets it
};

// ---- Tensor-core dense blocks (TB_PRECISION_TF32X3 / TB_PRECISION_BF16X3) --
// A dense pass works on WB consecutive address bits [lo, lo+WB). The steps of
// the pass whose target and control both lie in the window are composed on
// the host into one 2^WB x 2^WB complex matrix; the device applies it to all
// 2^(h-WB) "vectors" (fixed values of the other address bits) as a real GEMM
// D[vector][2*j'+part'] = sum_k A[vector][k] Bm[k][2*j'+part'], k = 2*j+part,
// on the tensor cores. A step whose control bit lies outside the window, and
// the two steps that depend on an output bit, run as FP32 register steps
// before (pre) or after (post) the block.
constexpr int TC_THREADS = 128;     // one warpgroup; thread i owns TMEM lane i
constexpr int TC_VEC_BITS = 7;      // 128 vectors per tile (one per TMEM lane)
constexpr int TC_CTAS_PER_SM = 2;
constexpr int TC_WB_TF32 = 5;       // 64 x 64 real block, FP32 operands
constexpr int TC_WB_BF16 = 6;       // 128 x 128 real block, 16-bit operands
constexpr int TC_MAX_WB = 6;

// A register step around a dense block.
struct TcStep {
    int t;      // window-relative target bit; -1: no step
    int cmode;  // 0: no control; 1: control = address bit cbit (outside the
                // window, fixed per vector); 2: control = window bit cbit
    int cbit;
    int step;   // index into the plan's step array
    int xq;     // qubit whose output bit selects the variant, -1: none
};

struct TcPass {
    int lo;        // address bit of window bit 0
    TcStep pre, post;
    int64_t mat;   // byte offset of the pass's split matrix in the tc_mats table
    int step0;     // contiguous steps covered (pre, block, post)
    int nsteps;
};

// Bytes of one split matrix (hi then lo) of a dense block over WB bits.
__host__ __device__ constexpr int64_t tc_mat_bytes(int WB, int elem_bytes) {
    return 2LL * (2LL << WB) * (2LL << WB) * elem_bytes;
}

// ---- Open output bits (Algorithm 2): a batch of 2^k amplitudes per prefix --
// One operation of the open band's late region (band qubit j = q - (n-k)).
struct OpenOp {
    int kind;     // 0: one-qubit gate m on band bit j; 1: CZ on band bits j, j+1
    int j;
    float2 m[4];  // row-major 2x2 (kind 0)
};
constexpr int OPEN_MAX_K = 10;          // 2^k x 2^k early-region matrix built on the host
constexpr int JOIN_TILE = 8192;         // join kernel: boundary entries per CTA tile
// Join on the tensor cores (3xTF32) for k >= JOIN_TC_MIN_K: Z = B.E as a real
// GEMM with K = N = 2^(k+1); the split E is stored in blocks of JOIN_KC K rows
// by join_nt(k) N columns, each block in the canonical K-major layout (hi, lo).
constexpr int JOIN_TC_MIN_K = 4;
constexpr int JOIN_KC = 32;
__host__ __device__ constexpr int join_nt(int k) { return (2 << k) < 128 ? (2 << k) : 128; }
// K chunks accumulated in one tensor-memory sum before it is added in FP32
// registers (the tensor cores' FP32 accumulation loses precision over long K).
constexpr int JOIN_SEG_CHUNKS = 4;

// Byte offsets of the device tables inside the workspace head.
struct TableLayout {
    int64_t steps;     // StepG[n_steps]
    int64_t pass_steps;  // StepG[]: the steps of every pass as its kernel runs them
    int64_t step_tgt;  // int8 target bit per step
    int64_t step_ctl;  // int8 control bit per step (-1: none)
    int64_t step_xq;   // int16 qubit of the bitstring dependence (-1: none)
    int64_t row_end;   // int32 index one past the last step of each absorbed row
    int64_t init_low;  // float2[2^k]          row 0: low-bit product
    int64_t init_mid;  // float2[2][2^m]       row 0: middle factor by bit k-1
    int64_t init_top;  // float2[2][2][2^top]  row 0: [x][bit k+m-1][top bits]
    int64_t red_low;   // float2[2^k][2]       last row: column vectors
    int64_t red_mid;   // float2[2^m][4]       last row: 2x2 matrices
    int64_t red_top;   // float2[2][2^top][2]  last row: [x] row vectors
    int64_t tc_mats;   // split dense-block matrices of the tensor-core passes
    int64_t open_E;    // float2[2^k][2^k]: early region joined with the first late ops
    int64_t open_Es;   // split real embedding of open_E for the tensor-core join (k >= JOIN_TC_MIN_K)
    int64_t open_ops;  // OpenOp[]: late-region band operations
    int64_t open_seg;  // int32[h-k+1]: ops of late crossing i are [seg[i], seg[i+1])
    int64_t total;
};

// Per-bitstring rescaling state: slot 0 is written by the row-0 writer, slot
// k+1 by pass k, slot P+1 by the last-row reduction.
//   maxs[slot]: float bits of max(|re|, |im|) over the boundary after it
//   exps[slot]: the power of two the producer multiplied its input by
struct ScaleLayout {
    int nslots;
    int64_t bytes_per_b;  // maxs (uint32) then exps (int32), padded
};

constexpr int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace tb

namespace tb {

// Window-relative target bit t and control bit c (-1: none) of step i of a
// pass of the given shape; for the turn block, t is its lower bit (it acts on
// t and t+1) and c its outside control. The planner emits steps in exactly
// this order.
struct StepSpec {
    int t;
    int c;
};

__host__ __device__ constexpr StepSpec step_spec(int type, int M, int i) {
    if (type == P_FWD || type == P_TOP_END) return StepSpec{i + 1, i};
    if (type == P_REV || type == P_BOT_END) return StepSpec{M - 2 - i, M - 1 - i};
    if (type == P_BOT_START) return StepSpec{i, i == 0 ? -1 : i - 1};
    if (type == P_TOP) {  // forward targets 1..M-3, block {M-2, M-1}, reversed targets M-3..0
        if (i < M - 3) return StepSpec{i + 1, i};
        if (i == M - 3) return StepSpec{M - 2, M - 3};
        const int j = i - (M - 3);
        return StepSpec{M - 2 - j, M - 1 - j};
    }
    // P_BOT: reversed targets M-2..2, block {0, 1}, forward targets 2..M-1
    if (i < M - 3) return StepSpec{M - 2 - i, M - 1 - i};
    if (i == M - 3) return StepSpec{0, 2};
    const int j = i - (M - 3) + 1;
    return StepSpec{j, j - 1};
}

}  // namespace tb
