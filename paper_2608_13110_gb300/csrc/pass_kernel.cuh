// Fused staircase pass over the temporal boundary (arXiv 2608.13110,
// Sec. 3.1, Algorithm 1: every paired step contracts two row tensors into the
// boundary). As in the paper's production code (Sec. 5.2), where several small
// tensors are combined first so that the big boundary is touched less often,
// every step of one window of address bits is applied in a single read + write
// of the boundary.
//
// A pass applies a compile-time sequence of controlled 2x2 steps to every
// tile of 2^13 complex64 entries: the window's M address bits plus 13-M low
// address bits (the 13 lowest bits when the window starts at bit 0). At a row
// turn the four steps on the window's two outermost bits run as one 4x4 block
// (composed on the host, see tb_internal.h).
//
// Warp-specialised, one persistent CTA per SM:
//   * one producer thread moves whole tiles between HBM and a 3-stage ring of
//     shared-memory stages with tensor copies (cp.async.bulk.tensor, 128-byte
//     swizzle; 64-byte rows and swizzle for 10-bit windows above bit 0): a
//     load completes on the stage's "full" mbarrier; once the
//     consumers have written the stage back it is stored in place with one
//     bulk tensor store, and as soon as the store has read the stage the next
//     tile's load is issued into it;
//   * 8 consumer warps never touch global memory and never wait for one
//     another: warp w owns the 1024 entries of the tile that share 3 "warp
//     bits" and holds them as 32 entries per thread: 5 address bits in
//     registers, 5 on the lanes. Every window bit is one of these 10, so a
//     step on a register bit is register arithmetic and a step on a lane bit
//     exchanges the partner lane's entries with warp shuffles. A warp reads
//     its entries from the stage once, applies every step, writes them back
//     and arrives on the stage's "done" mbarrier. HBM traffic, shared-memory
//     traffic and the arithmetic of different warps all overlap.
// The tensor map orders the tile's address bits so that every warp access to
// a stage is free of shared-memory bank conflicts, except in the 64-byte-row
// layout, where they are two-way (see slot_of).
//
// Rescaling: the producer of this pass's input left max(|re|,|im|) of its
// output in maxs[slot]; this pass multiplies its input by 2^s (exact; folded
// into the first step's coefficients) with s chosen so that the maximum lands
// in [0.5, 1), records s in exps[slot+1] and writes its own output maximum to
// maxs[slot+1].
//
// Every mbarrier wait is bounded. A wait that gives up counts once per CTA in
// the device fault word; the warp stops (all its lanes decide together), the
// others then give up too, and the producer waits (bounded) for the tile
// copies it still has in flight before the CTA exits.
#pragma once

#include <cuda.h>

#include "tb_internal.h"

namespace tb {

struct PassParams {
    int h, lo, n;
    int tile_shift;       // log2(tiles per batch element) = h - TILE_BITS
    int64_t ntiles;       // nbatch << tile_shift
    const StepG* steps;   // the pass's first step
    int xs_step0, xs_q0, xs_step1, xs_q1;
    const uint8_t* bits;  // bitstring of batch element b at bits + b*n
    uint32_t* maxs;       // maxs[b*sstride + slot]
    int32_t* exps;        // exps[b*sstride + slot]
    int64_t sstride;
    int slot;             // slot read; slot+1 written
    int* fault;           // device word: bounded waits that gave up (one per CTA)
    int selftest;         // 1: the producer issues no copies, so every wait gives up
};

__device__ __forceinline__ uint32_t pass_smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Tile bits (13) of a pass and where a consumer thread holds them.
//   LAY_BOT, windows at address bit 0 (tile = the 13 lowest address bits,
//   window bits 0..M-1, M <= 10): lanes hold tile bits 0..4, registers
//   5..9, the warp index 10..12;
//   LAY_HIGH, other windows of M <= 9 bits (tile bits 0..C-1 = the C >= 4
//   lowest address bits, tile bits C..12 = the window): lane bits 0..4 hold
//   tile bits 0, 4, 5, 6, 7, registers 8..12, the warp index 1..3;
//   LAY_LOW3, other windows of 10 bits (C = 3: tile bits 0..2 = the 3 lowest
//   address bits, rows of 64 bytes): lanes hold tile bits 3..7, registers
//   8..12, the warp index 0..2.
// Every window bit is a lane or register bit in each case.
constexpr int LAY_BOT = 0, LAY_HIGH = 1, LAY_LOW3 = 2;
template <int TYPE_, int M_>
struct Shape {
    static constexpr int TYPE = TYPE_;
    static constexpr int M = M_;
    static constexpr bool BOT = TYPE == P_BOT || TYPE == P_BOT_START || TYPE == P_BOT_END;
    static constexpr int NS = pass_nsteps(TYPE, M);
    static constexpr int XM = pass_xm(TYPE, M);           // step with four variants (-1: none)
    static constexpr int BLK = pass_blk(TYPE, M);         // the turn's 4x4 block (-1: none)
    static constexpr int NB = 2 * NS + (XM >= 0 ? 2 : 0);  // coefficient blocks
    static constexpr int C = BOT ? 0 : TILE_BITS - M;  // tile bit of window bit 0
    static constexpr int LAY = BOT ? LAY_BOT : (C == 3 ? LAY_LOW3 : LAY_HIGH);
    static constexpr int REG0 = BOT ? 5 : 8;            // tile bit of register bit 0
    static constexpr int regpos(int t) { return (t >= REG0 && t < REG0 + REG_BITS) ? t - REG0 : -1; }
    static constexpr int lanepos(int t) {
        if (BOT) return t < 5 ? t : -1;
        if (LAY == LAY_LOW3) return (t >= 3 && t < 8) ? t - 3 : -1;
        return t == 0 ? 0 : (t >= 4 && t < 8) ? t - 3 : -1;
    }
    static constexpr int tgt(int i) { return C + step_spec(TYPE, M, i).t; }
    static constexpr int ctl(int i) { return step_spec(TYPE, M, i).c < 0 ? -1 : C + step_spec(TYPE, M, i).c; }
    static constexpr bool valid() {
        if (M < MIN_WINDOW || M > (BOT ? MAX_WINDOW : MAX_WINDOW_HIGH)) return false;
        for (int j = 0; j < NS; ++j) {
            if (j == BLK) {  // bottom: lanes 0, 1 with control lane 2; top: registers 3, 4 with control register 2
                if (BOT ? (lanepos(tgt(j)) != 0 || lanepos(tgt(j) + 1) != 1 || lanepos(ctl(j)) != 2)
                        : (regpos(tgt(j)) != 3 || regpos(tgt(j) + 1) != 4 || regpos(ctl(j)) != 2))
                    return false;
                continue;
            }
            if (regpos(tgt(j)) < 0 && lanepos(tgt(j)) < 0) return false;
            if (ctl(j) >= 0 && regpos(ctl(j)) < 0 && lanepos(ctl(j)) < 0) return false;
        }
        return true;
    }
};

// Tile coordinate of a consumer thread's register entry 0.
template <int LAY>
__device__ __forceinline__ uint32_t thread_base(uint32_t tid) {
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    if (LAY == LAY_BOT) return lane | (warp << 10);
    if (LAY == LAY_LOW3) return (lane << 3) | warp;
    return (lane & 1u) | ((lane >> 1) << 4) | (warp << 1);
}

// ---------------------------------------------------------------------------
// Shared-memory layout of a stage (8-byte slots). The tensor copy writes the
// box in the order of its dimensions, so the stage position of a tile
// coordinate is a permutation of its bits, and the 128-byte swizzle then XORs
// slot bits 1..3 with slot bits 4..6 (16-byte chunk index with the 128-byte
// row index, stage 1024-byte aligned). A half warp's 8-byte accesses are free
// of bank conflicts when its 16 slots differ in bits 0..3 after the swizzle.
//   * windows above bit 0: identity order. Lanes 0..3 hold tile bits 0, 4,
//     5, 6 and the warp index bits 1..3, so the swizzled bits 0..3 are
//     t0, t1^t4, t2^t5, t3^t6: a bijection of the lane bits.
//   * windows at bit 0: tile bits 0..3, then 5..12, then 4. Lanes 0..3 hold
//     tile bits 0..3 and registers bits 5..7, so the swizzled bits are
//     t0, t1^t5, t2^t6, t3^t7: again a bijection of the lane bits.
//   * 10-bit windows above bit 0 (LAY_LOW3): identity order in rows of 64
//     bytes with the 64-byte swizzle (slot bits 1..2 ^= 4..5). Slot bit 0 is
//     the warp's tile bit 0, so a half warp's 16 slots cover 8 bank pairs:
//     two-way conflicts on these passes' stage reads and writes.
// The map is linear over GF(2): for disjoint bit sets slot_of(a | b) =
// slot_of(a) ^ slot_of(b), so a thread's 32 slots are its base slot XOR
// compile-time constants.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr uint32_t swz128(uint32_t s) { return s ^ (((s >> 4) & 7u) << 1); }

// 64-byte swizzle (rows of 64 bytes, LAY_LOW3): slot bits 1..2 ^= 4..5.
__host__ __device__ constexpr uint32_t swz64(uint32_t s) { return s ^ (((s >> 4) & 3u) << 1); }

template <int LAY>
__host__ __device__ constexpr uint32_t slot_of(uint32_t idx) {
    if (LAY == LAY_LOW3) return swz64(idx);
    constexpr bool BOT = LAY == LAY_BOT;
    return swz128(BOT ? ((idx & 15u) | (((idx >> 5) & 255u) << 4) | (((idx >> 4) & 1u) << 12)) : idx);
}

template <int LAY, uint32_t J>
struct SlotC {
    static constexpr uint32_t v = slot_of<LAY>(J);
};

// ---------------------------------------------------------------------------
// Packed complex arithmetic. A thread's 32 entries are j = k + 16 v (k:
// register bits 0..3, v: register bit 4). They are held "planar" in packed
// pairs P[k] = (re_k, re_(k+16)), Q[k] = (im_k, im_(k+16)), so that one
// __ffma2_rn (sm_100+ paired FP32 FMA) advances two entries that share their
// coefficient. A register step on bit K < 4 with coefficients shared by both
// halves needs 8 paired FMAs per pair of packed registers; a step whose
// control is register bit 4 uses lane-split coefficients; a step whose target
// is register bit 4 mixes the two halves of one packed register. A step on a
// lane bit takes the partner lane's packed registers by shuffles and applies
// the row of G that belongs to this lane's own value of the target bit.
//
// Coefficients are staged in shared memory already packed, 48 float2 per
// (step, bitstring variant):
//   register target, control none / not register bit 4 (KIND_F): for c in
//     0,1: [g00r g00i -g00i g01r g01i -g01i g10r g10i -g10i g11r g11i -g11i],
//     each broadcast to both halves
//   KIND_VC (control = register bit 4): the same 12 values with half c = control
//   KIND_VT (target = register bit 4): for c in 0,1: [Ar Ai -Ai Br Bi -Bi],
//     A = (g00, g11) (own half), B = (g01, g10) (other half)
//   KIND_L (target on a lane): for a (this lane's target value) in 0,1, at
//     24 a: for c in 0,1: [sr si -si or oi -oi] broadcast, s = G[c][a][a],
//     o = G[c][a][1-a]; then at 24 a + 12 the same 6 values with half c =
//     control (control = register bit 4)
// ---------------------------------------------------------------------------
constexpr int VBIT = 4;
constexpr int KIND_F = 0, KIND_VC = 1, KIND_VT = 2, KIND_L = 3, KIND_BL = 4, KIND_BV = 5;
constexpr int CO = 48;  // packed coefficients per (step, variant)

__device__ __forceinline__ float2 f2x(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

// out = g0 * a + g1 * b (complex) on planar pairs; cf = 6 packed coefficients
// [g0r g0i -g0i g1r g1i -g1i].
__device__ __forceinline__ void cmac_planar(const float2* cf, float2 aP, float2 aQ, float2 bP, float2 bQ,
                                            float2& oP, float2& oQ) {
    oP = fma2(cf[0], aP, fma2(cf[2], aQ, fma2(cf[3], bP, mul2(cf[5], bQ))));
    oQ = fma2(cf[0], aQ, fma2(cf[1], aP, fma2(cf[3], bQ, mul2(cf[4], bP))));
}

template <int N>
__device__ __forceinline__ void load_cf(float2 (&c)[N], const float2* src, float s) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const float4 q = s4[i];
        c[2 * i] = make_float2(q.x * s, q.y * s);
        c[2 * i + 1] = make_float2(q.z * s, q.w * s);
    }
}

// Register target bit K < 4 (pairs of packed registers). CK: -1 none (block
// 0), 0..3 control register bit (block per pair), 4 control = register bit 4
// (lane-split block), 5 control on a lane (block chosen by the caller).
template <int K, int CK>
__device__ __forceinline__ void step_pairs(float2 (&P)[16], float2 (&Q)[16], const float2 (&c0)[12],
                                           const float2 (&c1)[12]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k & (1 << K)) continue;
        const int k1 = k | (1 << K);
        const bool hi = (CK >= 0 && CK < 4) ? (((k >> CK) & 1) != 0) : false;
        float2 p0, q0, p1, q1;
        if (hi) {
            cmac_planar(c1, P[k], Q[k], P[k1], Q[k1], p0, q0);
            cmac_planar(c1 + 6, P[k], Q[k], P[k1], Q[k1], p1, q1);
        } else {
            cmac_planar(c0, P[k], Q[k], P[k1], Q[k1], p0, q0);
            cmac_planar(c0 + 6, P[k], Q[k], P[k1], Q[k1], p1, q1);
        }
        P[k] = p0; Q[k] = q0; P[k1] = p1; Q[k1] = q1;
    }
}

// Register target bit 4: the pair is the two halves of one packed register.
template <int CK>
__device__ __forceinline__ void step_halves(float2 (&P)[16], float2 (&Q)[16], const float2 (&c0)[12],
                                            const float2 (&c1)[12]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const bool hi = (CK >= 0 && CK < 4) ? (((k >> CK) & 1) != 0) : false;
        const float2 p = P[k], q = Q[k];
        float2 op, oq;
        if (hi) cmac_planar(c1, p, q, swap2(p), swap2(q), op, oq);  // [Ar Ai -Ai Br Bi -Bi]
        else    cmac_planar(c0, p, q, swap2(p), swap2(q), op, oq);
        P[k] = op; Q[k] = oq;
    }
}

// Lane target (partner lane = lane ^ LM): out = s * own + o * partner. CK as
// for step_pairs; c0 / c1 hold [sr si -si or oi -oi] for control 0 / 1.
template <int CK>
__device__ __forceinline__ void step_lane(float2 (&P)[16], float2 (&Q)[16], const float2 (&c0)[6],
                                          const float2 (&c1)[6], int LM) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const bool hi = (CK >= 0 && CK < 4) ? (((k >> CK) & 1) != 0) : false;
        float2 pp, qp;
        pp.x = __shfl_xor_sync(0xffffffffu, P[k].x, LM);
        pp.y = __shfl_xor_sync(0xffffffffu, P[k].y, LM);
        qp.x = __shfl_xor_sync(0xffffffffu, Q[k].x, LM);
        qp.y = __shfl_xor_sync(0xffffffffu, Q[k].y, LM);
        float2 op, oq;
        if (hi) cmac_planar(c1, P[k], Q[k], pp, qp, op, oq);
        else    cmac_planar(c0, P[k], Q[k], pp, qp, op, oq);
        P[k] = op; Q[k] = oq;
    }
}

// out = sum of four complex products on planar pairs; cf = 12 packed
// coefficients, [re im -im] per input.
__device__ __forceinline__ void cmac4_planar(const float2* cf, float2 aP, float2 aQ, float2 bP, float2 bQ,
                                             float2 cP, float2 cQ, float2 dP, float2 dQ, float2& oP,
                                             float2& oQ) {
    oP = fma2(cf[0], aP, fma2(cf[2], aQ, fma2(cf[3], bP, fma2(cf[5], bQ,
         fma2(cf[6], cP, fma2(cf[8], cQ, fma2(cf[9], dP, mul2(cf[11], dQ))))))));
    oQ = fma2(cf[0], aQ, fma2(cf[1], aP, fma2(cf[3], bQ, fma2(cf[4], bP,
         fma2(cf[6], cQ, fma2(cf[7], cP, fma2(cf[9], dQ, mul2(cf[10], dP))))))));
}

// Turn block on lanes 0, 1 (this lane's block index r = lane & 3): out =
// sum_d B[r][r ^ d] in(lane ^ d); c = [re im -im] of B[r][r ^ d], d = 0..3.
__device__ __forceinline__ void step_block_lanes(float2 (&P)[16], float2 (&Q)[16], const float2 (&c)[12]) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float2 pp[4], qp[4];
        pp[0] = P[k]; qp[0] = Q[k];
#pragma unroll
        for (int d = 1; d < 4; ++d) {
            pp[d].x = __shfl_xor_sync(0xffffffffu, P[k].x, d);
            pp[d].y = __shfl_xor_sync(0xffffffffu, P[k].y, d);
            qp[d].x = __shfl_xor_sync(0xffffffffu, Q[k].x, d);
            qp[d].y = __shfl_xor_sync(0xffffffffu, Q[k].y, d);
        }
        cmac4_planar(c, pp[0], qp[0], pp[1], qp[1], pp[2], qp[2], pp[3], qp[3], P[k], Q[k]);
    }
}

// Turn block on registers 3 and 4 (register 4 = the packed pair's halves),
// control register 2: packed registers k and k | 8 (k < 8) form the block's
// four entries; cf = the variant's 48 coefficients (24 per control value).
__device__ __forceinline__ void step_block_regs(float2 (&P)[16], float2 (&Q)[16], const float2* cf) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float2 cc[24];
        load_cf(cc, cf + 24 * c, 1.0f);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int k0 = kk | (c << 2), k1 = k0 | 8;
            const float2 aP = P[k0], aQ = Q[k0], bP = P[k1], bQ = Q[k1];
            const float2 sP = swap2(aP), sQ = swap2(aQ), tP = swap2(bP), tQ = swap2(bQ);
            cmac4_planar(cc, aP, aQ, sP, sQ, bP, bQ, tP, tQ, P[k0], Q[k0]);
            cmac4_planar(cc + 12, aP, aQ, sP, sQ, bP, bQ, tP, tQ, P[k1], Q[k1]);
        }
    }
}

template <class SH>
__host__ __device__ constexpr int step_kind(int i) {
    if (i == SH::BLK) return SH::BOT ? KIND_BL : KIND_BV;
    const int K = SH::regpos(SH::tgt(i));
    if (K < 0) return KIND_L;
    if (K == VBIT) return KIND_VT;
    if (SH::ctl(i) >= 0 && SH::regpos(SH::ctl(i)) == VBIT) return KIND_VC;
    return KIND_F;
}

template <class SH>
__host__ __device__ constexpr uint64_t step_kinds() {
    uint64_t k = 0;
    static_assert(3 * SH::NS <= 64, "three kind bits per step");
    for (int i = 0; i < SH::NS; ++i) k |= (uint64_t)step_kind<SH>(i) << (3 * i);
    return k;
}

// Stage the packed coefficients of every step and variant into shared memory.
// Blocks 2 i + x: step i, variant x; blocks 2 NS + x: the four-variant
// step's (the top block's) variants 2 + x. Turn blocks (raw float2[variant][c][q'][q] over
// BLK_ENTRIES table entries):
//   KIND_BL (lanes 0, 1; control lane 2; no output-bit dependence): blocks
//     2 i and 2 i + 1 hold, at 12 (4 c + r), [re im -im] of B[c][r][r ^ d]
//     for d = 0..3, broadcast (r = the lane's block index)
//   KIND_BV (registers 3, 4; control register 2): per variant, at 24 c + 12 b
//     (output register: block bit t = b), four packed pairs for the inputs
//     [register t=0, swapped, register t=1, swapped]: (B[b][a], B[b+2][a+2])
//     and (B[b][a+2], B[b+2][a]) for a = 0, 1, each as [re im -im]
template <class SH>
__device__ __forceinline__ void stage_coefficients(const StepG* steps, float2* sc, uint32_t tid) {
    constexpr uint64_t KINDS = step_kinds<SH>();
    for (int w = tid; w < SH::NB; w += PASS_THREADS) {
        const int i = w < 2 * SH::NS ? w >> 1 : SH::XM, x = w & 1;
        float2* o = sc + w * CO;
        for (int e = 0; e < CO; ++e) o[e] = make_float2(0.f, 0.f);
        const int kind = (int)((KINDS >> (3 * i)) & 7u);
        if (kind == KIND_BL || kind == KIND_BV) {
            const float2* raw = &steps[pass_entry(SH::TYPE, SH::M, i)].g[0][0];
            auto Bq = [&](int v, int c, int r, int q) { return raw[((v * 2 + c) * 4 + r) * 4 + q]; };
            if (kind == KIND_BL) {  // block w - 2 i = control value c
                for (int r = 0; r < 4; ++r)
                    for (int d = 0; d < 4; ++d) {
                        const float2 z = Bq(0, x, r, r ^ d);
                        o[12 * r + 3 * d + 0] = f2x(z.x);
                        o[12 * r + 3 * d + 1] = f2x(z.y);
                        o[12 * r + 3 * d + 2] = f2x(-z.y);
                    }
            } else {
                const int v = x + (w < 2 * SH::NS ? 0 : 2);
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a)
                            for (int sw = 0; sw < 2; ++sw) {
                                const float2 lo = Bq(v, c, b, sw ? a + 2 : a), hi = Bq(v, c, b + 2, sw ? a : a + 2);
                                float2* t = o + 24 * c + 12 * b + 6 * a + 3 * sw;
                                t[0] = make_float2(lo.x, hi.x);
                                t[1] = make_float2(lo.y, hi.y);
                                t[2] = make_float2(-lo.y, -hi.y);
                            }
            }
            continue;
        }
        const float2* g = steps[pass_entry(SH::TYPE, SH::M, i)].g[x];  // [c*4 + a'*2 + s]
        if (kind == KIND_F) {
            for (int c = 0; c < 2; ++c)
                for (int e = 0; e < 4; ++e) {
                    const float2 z = g[c * 4 + e];
                    o[c * 12 + 3 * e + 0] = f2x(z.x);
                    o[c * 12 + 3 * e + 1] = f2x(z.y);
                    o[c * 12 + 3 * e + 2] = f2x(-z.y);
                }
        } else if (kind == KIND_VC) {
            for (int e = 0; e < 4; ++e) {
                const float2 z0 = g[e], z1 = g[4 + e];
                o[3 * e + 0] = make_float2(z0.x, z1.x);
                o[3 * e + 1] = make_float2(z0.y, z1.y);
                o[3 * e + 2] = make_float2(-z0.y, -z1.y);
            }
        } else if (kind == KIND_VT) {
            for (int c = 0; c < 2; ++c) {
                const float2 A0 = g[c * 4 + 0], A1 = g[c * 4 + 3];  // own half: g00 (lo), g11 (hi)
                const float2 B0 = g[c * 4 + 1], B1 = g[c * 4 + 2];  // other half: g01 (lo), g10 (hi)
                o[c * 12 + 0] = make_float2(A0.x, A1.x);
                o[c * 12 + 1] = make_float2(A0.y, A1.y);
                o[c * 12 + 2] = make_float2(-A0.y, -A1.y);
                o[c * 12 + 3] = make_float2(B0.x, B1.x);
                o[c * 12 + 4] = make_float2(B0.y, B1.y);
                o[c * 12 + 5] = make_float2(-B0.y, -B1.y);
            }
        } else {
            for (int a = 0; a < 2; ++a) {
                float2* oa = o + 24 * a;
                for (int c = 0; c < 2; ++c) {
                    const float2 sv = g[c * 4 + a * 2 + a], ov = g[c * 4 + a * 2 + (1 - a)];
                    const float v[6] = {sv.x, sv.y, -sv.y, ov.x, ov.y, -ov.y};
                    for (int e = 0; e < 6; ++e) {
                        oa[c * 6 + e] = f2x(v[e]);
                        if (c == 0) oa[12 + e].x = v[e];
                        else        oa[12 + e].y = v[e];
                    }
                }
            }
        }
    }
}

// Registers <-> shared stage: entry j of a thread sits at tile coordinate
// thread_base | j << REG0, i.e. slot base ^ SlotC<j << REG0>.
template <int LAY, int REG0, int J>
__device__ __forceinline__ void smem_read_j(float2 (&P)[16], float2 (&Q)[16], const float2* tile, uint32_t sb) {
    if constexpr (J < 32) {
        const float2 e = tile[sb ^ SlotC<LAY, ((uint32_t)J << REG0)>::v];
        if constexpr (J < 16) { P[J].x = e.x; Q[J].x = e.y; }
        else                  { P[J - 16].y = e.x; Q[J - 16].y = e.y; }
        smem_read_j<LAY, REG0, J + 1>(P, Q, tile, sb);
    }
}

template <int LAY, int REG0, int J>
__device__ __forceinline__ void smem_write_j(const float2 (&P)[16], const float2 (&Q)[16], float2* tile,
                                             uint32_t sb) {
    if constexpr (J < 32) {
        tile[sb ^ SlotC<LAY, ((uint32_t)J << REG0)>::v] =
            J < 16 ? make_float2(P[J & 15].x, Q[J & 15].x) : make_float2(P[J & 15].y, Q[J & 15].y);
        smem_write_j<LAY, REG0, J + 1>(P, Q, tile, sb);
    }
}

template <class SH, int I>
__device__ __forceinline__ void apply_step(float2 (&P)[16], float2 (&Q)[16], const float2* sc,
                                           uint32_t xmask, float scale, uint32_t tid) {
    constexpr int T = SH::tgt(I), CB = SH::ctl(I);
    constexpr int kind = step_kind<SH>(I);
    // control: -1 none, 0..4 register bit, 5 on a lane (the same for all of
    // this thread's entries)
    constexpr int CK = CB < 0 ? -1 : (SH::regpos(CB) >= 0 ? SH::regpos(CB) : 5);
    const uint32_t lane = tid & 31u;
    const float s = (I == 0) ? scale : 1.0f;
    asm volatile("" ::: "memory");  // load each step's coefficients just before it
    const float2* cf;
    if constexpr (I == SH::XM) {  // variant x_a + 2 x_b
        cf = sc + (((xmask >> XM_HIGH_BIT) & 1u) ? 2 * SH::NS : I * 2) * CO + (int)((xmask >> I) & 1u) * CO;
    } else {
        cf = sc + (I * 2 + (int)((xmask >> I) & 1u)) * CO;
    }
    if constexpr (kind == KIND_BL) {
        float2 c[12];
        static_assert(I > 0, "the first step carries the rescale");
        load_cf(c, sc + (I * 2 + (int)((lane >> 2) & 1u)) * CO + (lane & 3u) * 12u, 1.0f);  // control lane 2
        step_block_lanes(P, Q, c);
    } else if constexpr (kind == KIND_BV) {
        static_assert(I > 0 && I == SH::XM, "the top block has four variants and no rescale");
        step_block_regs(P, Q, cf);
    } else if constexpr (kind == KIND_L) {
        constexpr int L = SH::lanepos(T);
        static_assert(L >= 0, "lane target");
        const float2* ca = cf + 24 * ((lane >> L) & 1u);
        float2 c0[6], c1[6];
        if constexpr (CK == 5) {
            load_cf(c0, ca + 6 * ((lane >> SH::lanepos(CB)) & 1u), s);
        } else if constexpr (CK == 4) {
            load_cf(c0, ca + 12, s);
        } else {
            load_cf(c0, ca, s);
            if constexpr (CK >= 0) load_cf(c1, ca + 6, s);
        }
        step_lane<(CK == 4 || CK == 5) ? -1 : CK>(P, Q, c0, c1, 1 << L);
    } else {
        constexpr int K = SH::regpos(T);
        float2 c0[12], c1[12];
        if constexpr (CK == 5) {
            load_cf(c0, cf + 12 * ((lane >> SH::lanepos(CB)) & 1u), s);
        } else {
            load_cf(c0, cf, s);
        }
        if constexpr (CK >= 0 && CK < 4) load_cf(c1, cf + 12, s);
        if constexpr (kind == KIND_VT) {
            step_halves<(CK == 5) ? -1 : CK>(P, Q, c0, c1);
        } else {
            step_pairs<K, (CK == 5) ? -1 : CK>(P, Q, c0, c1);
        }
    }
}

template <class SH, int I>
__device__ __forceinline__ void run_steps(float2 (&P)[16], float2 (&Q)[16], const float2* sc, uint32_t xmask,
                                          float scale, uint32_t tid) {
    if constexpr (I < SH::NS) {
        apply_step<SH, I>(P, Q, sc, xmask, scale, tid);
        run_steps<SH, I + 1>(P, Q, sc, xmask, scale, tid);
    }
}

__device__ __forceinline__ void flush_max(float m, uint32_t* dst) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(dst, __float_as_uint(m));
}

// Power of two that brings a maximum m into [0.5, 1); 0 for m == 0.
__device__ __forceinline__ int rescale_exp(float m) {
    if (!(m > 0.0f) || !isfinite(m)) return 0;
    int e;
    frexpf(m, &e);
    return max(-100, min(100, -e));
}

// ---------------------------------------------------------------------------
// mbarriers and tensor copies (PTX)
// ---------------------------------------------------------------------------
constexpr uint32_t PASS_WAIT_TRIES = 1u << 24;    // far beyond any tile's copy or compute time
constexpr uint32_t PASS_SELFTEST_TRIES = 1u << 10;

__device__ __forceinline__ void pbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void pbar_arrive(uint32_t a) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a) : "memory");
}

__device__ __forceinline__ void pbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool pbar_wait(uint32_t a, uint32_t parity, uint32_t tries) {
    for (uint32_t it = 0; it < tries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap* m, int c3, int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %2, %2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(0), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_store_tile(const CUtensorMap* m, int c3, int c4, uint32_t src) {
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %1, %1, %2, %3}], [%4];\n" ::"l"(
            reinterpret_cast<uint64_t>(m)),
        "r"(0), "r"(c3), "r"(c4), "r"(src)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void tma_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Tensor-map coordinates (dimensions 3 and 4) of global tile gt. Windows at
// bit 0: dimension 3 is the global tile index. Other windows: dimension 3 =
// the address bits between the low bits and the window, dimension 4 = the
// bits above the window and the batch element.
template <class SH>
__device__ __forceinline__ void tile_coords(const PassParams& p, int64_t gt, int& c3, int& c4) {
    if constexpr (SH::BOT) {
        c3 = (int)gt;
        c4 = 0;
    } else {
        const int64_t b = gt >> p.tile_shift;
        const int64_t t = gt & (((int64_t)1 << p.tile_shift) - 1);
        const int nl = p.lo - SH::C;
        c3 = (int)(t & (((int64_t)1 << nl) - 1));
        c4 = (int)((b << (p.h - p.lo - SH::M)) + (t >> nl));
    }
}

constexpr int PASS_STAGES = 3;
constexpr uint32_t TILE_BYTES = (uint32_t)TILE * 8u;

template <int TYPE, int M>
constexpr int pass_smem_bytes() {
    return 1024 + PASS_STAGES * TILE * 8 + Shape<TYPE, M>::NB * CO * 8 + 2 * PASS_STAGES * 8 + 16;
}

template <int TYPE, int M>
__global__ void __launch_bounds__(PASS_THREADS, PASS_CTAS_PER_SM)
    pass_kernel(const PassParams p, const __grid_constant__ CUtensorMap tmap) {
    using SH = Shape<TYPE, M>;
    static_assert(SH::valid(), "invalid pass shape");
    static_assert(SH::NS <= XM_HIGH_BIT, "variant mask: one bit per step, bit XM_HIGH_BIT for the four-variant step");
    constexpr int NS = SH::NS;
    extern __shared__ __align__(16) uint8_t dsm[];
    uint8_t* base = dsm + ((1024u - (pass_smem_u32(dsm) & 1023u)) & 1023u);
    float2* stages = reinterpret_cast<float2*>(base);
    float2* sc = stages + PASS_STAGES * TILE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sc + SH::NB * CO);  // full[3], done[3]
    int* s_abort = reinterpret_cast<int*>(bars + 2 * PASS_STAGES);
    const uint32_t tid = threadIdx.x;
    const uint32_t full0 = pass_smem_u32(bars), done0 = full0 + 8 * PASS_STAGES;
    const uint32_t stage0 = pass_smem_u32(stages);

    stage_coefficients<SH>(p.steps, sc, tid);
    if (tid == 0) {
        for (int s = 0; s < PASS_STAGES; ++s) {
            pbar_init(full0 + 8 * s, 1);
            pbar_init(done0 + 8 * s, PASS_CONSUMERS / 32);
        }
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    const int64_t first = blockIdx.x;
    const int64_t ntl = first < p.ntiles ? (p.ntiles - 1 - first) / gridDim.x + 1 : 0;  // tiles of this CTA
    const uint32_t tries = p.selftest ? PASS_SELFTEST_TRIES : PASS_WAIT_TRIES;

    static_assert(PASS_THREADS - PASS_CONSUMERS == 128, "one producer warpgroup");
    static_assert((PASS_THREADS - PASS_CONSUMERS) * PASS_PRODUCER_REGS + PASS_CONSUMERS * PASS_CONSUMER_REGS <=
                      PASS_THREADS * (65536 / PASS_THREADS / 8 * 8),
                  "register split exceeds the launch's registers");
    if (tid >= PASS_CONSUMERS) {
        // ---------------- producer: one thread of the last warpgroup
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(PASS_PRODUCER_REGS));
        if (tid != PASS_CONSUMERS) return;
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
        int64_t last_load[PASS_STAGES];  // tile index k of the latest load per stage (-1: none)
        for (int st = 0; st < PASS_STAGES; ++st) last_load[st] = -1;
        if (!p.selftest) {
            for (int64_t k = 0; k < ntl && k < PASS_STAGES; ++k) {
                int c3, c4;
                tile_coords<SH>(p, first + k * gridDim.x, c3, c4);
                pbar_expect_tx(full0 + 8 * (int)k, TILE_BYTES);
                tma_load_tile(stage0 + (uint32_t)k * TILE_BYTES, &tmap, c3, c4, full0 + 8 * (int)k);
                last_load[k] = k;
            }
        }
        int s = 0;
        uint32_t ph = 0;
        for (int64_t k = 0; k < ntl; ++k) {
            if (!pbar_wait(done0 + 8 * s, ph, tries)) {
                if (atomicExch(s_abort, 1) == 0) atomicAdd(p.fault, 1);
                break;
            }
            int c3, c4;
            tile_coords<SH>(p, first + k * gridDim.x, c3, c4);
            tma_store_tile(&tmap, c3, c4, stage0 + (uint32_t)s * TILE_BYTES);
            if (k + PASS_STAGES < ntl) {
                tma_wait_read_all();  // the store has read the stage
                tile_coords<SH>(p, first + (k + PASS_STAGES) * gridDim.x, c3, c4);
                pbar_expect_tx(full0 + 8 * s, TILE_BYTES);
                tma_load_tile(stage0 + (uint32_t)s * TILE_BYTES, &tmap, c3, c4, full0 + 8 * s);
                last_load[s] = k + PASS_STAGES;
            }
            if (++s == PASS_STAGES) { s = 0; ph ^= 1u; }
        }
        tma_wait_all();
        if (*(volatile int*)s_abort) {
            // loads still in flight must land before the CTA's shared memory goes
            for (int st = 0; st < PASS_STAGES; ++st)
                if (last_load[st] >= 0)
                    (void)pbar_wait(full0 + 8 * st, (uint32_t)((last_load[st] / PASS_STAGES) & 1), PASS_WAIT_TRIES);
        }
        return;
    }

    // ---------------- consumers (tid < 256): 8 independent warps
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(PASS_CONSUMER_REGS));
    float runmax = 0.0f;
    int64_t cur_b = -1;
    int cur_s = 0;
    float scale = 1.0f;
    uint32_t xmask = 0;
    const int64_t tmask = ((int64_t)1 << p.tile_shift) - 1;
    const uint32_t sb = slot_of<SH::LAY>(thread_base<SH::LAY>(tid));
    int s = 0;
    uint32_t ph = 0;
    for (int64_t k = 0; k < ntl; ++k) {
        const bool gave_up = !pbar_wait(full0 + 8 * s, ph, tries);
        if (__any_sync(0xffffffffu, gave_up)) {  // the whole warp stops
            if ((tid & 31u) == 0 && atomicExch(s_abort, 1) == 0) atomicAdd(p.fault, 1);
            break;
        }
        const int64_t gt = first + k * gridDim.x;
        const int64_t b = gt >> p.tile_shift;
        const int64_t t = gt & tmask;
        if (b != cur_b) {  // per-bitstring state, read once per batch element
            if (cur_b >= 0) flush_max(runmax, p.maxs + cur_b * p.sstride + p.slot + 1);
            runmax = 0.0f;
            cur_b = b;
            cur_s = rescale_exp(__uint_as_float(p.maxs[b * p.sstride + p.slot]));
            scale = ldexpf(1.0f, cur_s);
            const uint8_t* xb = p.bits + b * p.n;
            xmask = 0;
            if (p.xs_step0 >= 0) xmask |= (xb[p.xs_q0] ? 1u : 0u) << p.xs_step0;
            if (p.xs_step1 >= 0) xmask |= (xb[p.xs_q1] ? 1u : 0u) << p.xs_step1;
        }
        if (t == 0 && tid == 0) p.exps[b * p.sstride + p.slot + 1] = cur_s;

        float2* tile = stages + s * TILE;
        float2 P[16], Q[16];
        smem_read_j<SH::LAY, SH::REG0, 0>(P, Q, tile, sb);
        run_steps<SH, 0>(P, Q, sc, xmask, scale, tid);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            runmax = fmaxf(runmax, fmaxf(fmaxf(fabsf(P[j].x), fabsf(P[j].y)), fmaxf(fabsf(Q[j].x), fabsf(Q[j].y))));
        smem_write_j<SH::LAY, SH::REG0, 0>(P, Q, tile, sb);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the tensor store
        __syncwarp();
        if ((tid & 31u) == 0) pbar_arrive(done0 + 8 * s);
        if (++s == PASS_STAGES) { s = 0; ph ^= 1u; }
    }
    if (cur_b >= 0) flush_max(runmax, p.maxs + cur_b * p.sstride + p.slot + 1);
}

// Launchers, one translation unit per pass type (pass_t<type>.cu).
cudaError_t launch_pass_t0(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st);
cudaError_t launch_pass_t1(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st);
cudaError_t launch_pass_t2(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st);
cudaError_t launch_pass_t3(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st);
cudaError_t launch_pass_t4(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st);
cudaError_t launch_pass_t5(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st);
cudaError_t launch_pass_t6(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st);

template <int TYPE, int M>
cudaError_t launch_one(const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st) {
    if constexpr (!Shape<TYPE, M>::valid()) {
        return cudaErrorInvalidValue;
    } else {
        constexpr int smem = pass_smem_bytes<TYPE, M>();
        static_assert(smem <= 227 * 1024, "pass kernel shared memory");
        cudaError_t e = cudaFuncSetAttribute(pass_kernel<TYPE, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        pass_kernel<TYPE, M><<<grid, PASS_THREADS, smem, st>>>(p, m);
        return cudaGetLastError();
    }
}

#define TB_DEFINE_LAUNCH_PASS(TYPE, NAME)                                                      \
    cudaError_t NAME(int M, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st) { \
        switch (M) {                                                                          \
            case 5: return launch_one<TYPE, 5>(p, m, grid, st);                               \
            case 6: return launch_one<TYPE, 6>(p, m, grid, st);                               \
            case 7: return launch_one<TYPE, 7>(p, m, grid, st);                               \
            case 8: return launch_one<TYPE, 8>(p, m, grid, st);                               \
            case 9: return launch_one<TYPE, 9>(p, m, grid, st);                               \
            case 10: return launch_one<TYPE, 10>(p, m, grid, st);                             \
            default: return cudaErrorInvalidValue;                                            \
        }                                                                                     \
    }

}  // namespace tb
