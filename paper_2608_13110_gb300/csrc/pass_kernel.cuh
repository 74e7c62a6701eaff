// Fused staircase pass over the temporal boundary (arXiv 2608.13110,
// Sec. 3.1, Algorithm 1: every paired step contracts two row tensors into the
// boundary). As in the paper's production code (Sec. 5.2), where several small
// tensors are combined first so that the big boundary is touched less often,
// every step of one window of address bits is applied in a single read + write
// of the boundary.
//
// A pass applies a compile-time sequence of controlled 2x2 steps to every
// tile of 2^13 complex64 entries: the window's M address bits plus 13-M low
// address bits (the 13 lowest bits when the window starts at bit 0). Each of
// the 256 threads holds 32 entries; one CTA per SM. A step acts on a
// 5-bit "register run" of the tile; between runs the tile is re-read from
// shared memory (XOR-swizzled, conflict-free for every run base used). Tiles
// stream in through a 3-stage cp.async ring; stores go from registers
// straight to HBM with 8 or more consecutive entries on consecutive lanes.
//
// Rescaling: the producer of this pass's input left max(|re|,|im|) of its
// output in maxs[slot]; this pass multiplies its input by 2^s (exact; folded
// into the first step's coefficients) with s chosen so that the maximum lands
// in [0.5, 1), records s in exps[slot+1] and writes its own output maximum to
// maxs[slot+1].
#pragma once

#include "tb_internal.h"

namespace tb {

struct PassParams {
    float2* B;            // boundary of batch element 0
    int64_t b_stride;     // complex entries between batch elements
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
};

__host__ __device__ constexpr bool in_run(int s, int r) { return s >= r && s < r + REG_BITS; }

template <int TYPE_, int M_>
struct Shape {
    static constexpr int TYPE = TYPE_;
    static constexpr int M = M_;
    static constexpr bool BOT = TYPE == P_BOT || TYPE == P_BOT_START || TYPE == P_BOT_END;
    static constexpr int NS = pass_nsteps(TYPE, M);
    static constexpr int C = BOT ? 0 : TILE_BITS - M;  // tile bit of window bit 0
    static constexpr int RA = BOT ? 0 : C;
    static constexpr int RB = BOT ? 5 : TILE_BITS - REG_BITS;
    // the tile arrives in shared memory, so the first run is the one holding
    // step 0's target; the last run must give coalesced stores from registers
    // (run 0 would put 32 consecutive entries in one thread)
    static constexpr int first_run() {
        return in_run(C + step_spec(TYPE, M, 0).t, RA) ? RA : RB;
    }
    // register run in which step i executes
    static constexpr int run_of(int i) {
        int cur = first_run();
        for (int j = 0; j <= i; ++j) {
            const int s = C + step_spec(TYPE, M, j).t;
            if (!in_run(s, cur)) cur = (cur == RA) ? RB : RA;
        }
        return cur;
    }
    static constexpr int last_run() { return BOT ? RB : run_of(NS - 1); }
    static constexpr bool valid() {
        if (M < MIN_WINDOW || M > (BOT ? MAX_WINDOW : MAX_WINDOW_HIGH)) return false;
        for (int j = 0; j < NS; ++j)
            if (!in_run(C + step_spec(TYPE, M, j).t, run_of(j))) return false;
        return true;
    }
};

// Tile coordinate of a thread's entries for register run r: the 8 thread-index
// bits fill the tile bits outside [r, r+5) from the bottom.
__device__ __forceinline__ uint32_t run_base(int r, uint32_t tid) {
    return (tid & ((1u << r) - 1u)) | ((tid >> r) << (r + REG_BITS));
}

// Shared-memory slot of tile coordinate idx. Bit 0 is never moved, so 16-byte
// chunks (two entries) stay intact for cp.async; bits 1..3 are XORed with
// bits 6, 7 and 5^8. For every register run used here (bases 0, 3..8) the 16
// lanes of a half warp then hit 16 different 8-byte bank pairs (runs >= 3,
// 8-byte accesses), and for run 0, read as 16-byte pairs, the 8 lanes of a
// quarter warp hit 8 different 16-byte bank groups.
__host__ __device__ __forceinline__ constexpr uint32_t swz(uint32_t idx) {
    return idx ^ (((idx >> 6) & 1u) << 1) ^ (((idx >> 7) & 1u) << 2) ^ ((((idx >> 5) ^ (idx >> 8)) & 1u) << 3);
}
// swz is linear over GF(2): for disjoint bit sets, swz(a | b) = swz(a) ^ swz(b),
// so a run's 32 slots are the thread's swizzled base XOR compile-time constants.
template <uint32_t J>
struct SwzC {
    static constexpr uint32_t v = swz(J);
};


// ---------------------------------------------------------------------------
// Packed complex arithmetic. A thread's 32 entries of register run R are
// j = k + 16 v (k: run bits 0..3, v: run bit 4). They are held "planar" in
// packed pairs P[k] = (re_k, re_(k+16)), Q[k] = (im_k, im_(k+16)), so that
// one __ffma2_rn (sm_100+ paired FP32 FMA) advances two entries that share
// their coefficient. A step on run bit K < 4 with coefficients shared by both
// lanes needs 8 paired FMAs per pair of packed registers (half the scalar
// count); a step whose control is run bit 4 uses lane-split coefficients; a
// step whose target is run bit 4 mixes the two lanes of one packed register.
//
// Coefficients are staged in shared memory already packed, 24 float2 per
// (step, bitstring variant):
//   KIND_F  (target, control < 4 or none): for c in 0,1:
//           [g00r g00i -g00i g01r g01i -g01i g10r g10i -g10i g11r g11i -g11i],
//           each broadcast to both lanes
//   KIND_VC (control = run bit 4): the same 12 values with lane c = control
//   KIND_VT (target = run bit 4): for c in 0,1: [Ar Ai -Ai Br Bi -Bi],
//           A = (g00, g11) (own lane), B = (g01, g10) (other lane)
// ---------------------------------------------------------------------------
constexpr int VBIT = 4;
constexpr int KIND_F = 0, KIND_VC = 1, KIND_VT = 2;
constexpr int CO = 24;  // packed coefficients per (step, variant)

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

__device__ __forceinline__ void load_cf(float2 (&c)[12], const float2* src, float s) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float4 q = s4[i];
        c[2 * i] = make_float2(q.x * s, q.y * s);
        c[2 * i + 1] = make_float2(q.z * s, q.w * s);
    }
}

// Target run bit K < 4 (pairs of packed registers). CK: -1 none (block 0),
// 0..3 control run bit (block per pair), 4 control = run bit 4 (lane split),
// 5 external control (block chosen by the caller).
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

// Target run bit 4: the pair is the two lanes of one packed register.
template <int CK>
__device__ __forceinline__ void step_lanes(float2 (&P)[16], float2 (&Q)[16], const float2 (&c0)[12],
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

template <class SH>
__host__ __device__ constexpr int step_kind(int i) {
    const StepSpec sp = step_spec(SH::TYPE, SH::M, i);
    const int R = SH::run_of(i);
    const int K = SH::C + sp.t - R;
    if (K == VBIT) return KIND_VT;
    if (sp.c >= 0 && in_run(SH::C + sp.c, R) && SH::C + sp.c - R == VBIT) return KIND_VC;
    return KIND_F;
}

template <class SH>
__host__ __device__ constexpr uint64_t step_kinds() {
    uint64_t k = 0;
    for (int i = 0; i < SH::NS; ++i) k |= (uint64_t)step_kind<SH>(i) << (2 * i);
    return k;
}

// Stage the packed coefficients of every step and variant into shared memory.
template <class SH>
__device__ __forceinline__ void stage_coefficients(const StepG* steps, float2* sc, uint32_t tid) {
    constexpr uint64_t KINDS = step_kinds<SH>();
    for (int w = tid; w < SH::NS * 2; w += PASS_THREADS) {
        const int i = w >> 1, x = w & 1;
        const float2* g = steps[i].g[x];  // [c*4 + a'*2 + s]
        float2* o = sc + w * CO;
        const int kind = (int)((KINDS >> (2 * i)) & 3u);
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
            for (int e = 12; e < 24; ++e) o[e] = make_float2(0.f, 0.f);
        } else {
            for (int c = 0; c < 2; ++c) {
                const float2 A0 = g[c * 4 + 0], A1 = g[c * 4 + 3];  // own lane: g00 (lo), g11 (hi)
                const float2 B0 = g[c * 4 + 1], B1 = g[c * 4 + 2];  // other lane: g01 (lo), g10 (hi)
                o[c * 12 + 0] = make_float2(A0.x, A1.x);
                o[c * 12 + 1] = make_float2(A0.y, A1.y);
                o[c * 12 + 2] = make_float2(-A0.y, -A1.y);
                o[c * 12 + 3] = make_float2(B0.x, B1.x);
                o[c * 12 + 4] = make_float2(B0.y, B1.y);
                o[c * 12 + 5] = make_float2(-B0.y, -B1.y);
                for (int e = 6; e < 12; ++e) o[c * 12 + e] = make_float2(0.f, 0.f);
            }
        }
    }
}

// Registers <-> shared tile for register run R (entry j = k + 16 v at tile
// coordinate base | j << R). Run 0 moves the two entries of a 16-byte chunk
// in one 16-byte access.
template <int R, int J>
__device__ __forceinline__ uint32_t run_slot(uint32_t sb) {
    return sb ^ SwzC<((uint32_t)J << R)>::v;
}

template <int R, int J>
__device__ __forceinline__ void smem_read_run(float2 (&P)[16], float2 (&Q)[16], const float2* tile, uint32_t sb) {
    if constexpr (J < 32) {
        const float2 e = tile[run_slot<R, J>(sb)];
        if constexpr (J < 16) { P[J].x = e.x; Q[J].x = e.y; }
        else                  { P[J - 16].y = e.x; Q[J - 16].y = e.y; }
        smem_read_run<R, J + 1>(P, Q, tile, sb);
    }
}

template <int R, int J>
__device__ __forceinline__ void smem_write_run(const float2 (&P)[16], const float2 (&Q)[16], float2* tile, uint32_t sb) {
    if constexpr (J < 32) {
        tile[run_slot<R, J>(sb)] = J < 16 ? make_float2(P[J & 15].x, Q[J & 15].x) : make_float2(P[J & 15].y, Q[J & 15].y);
        smem_write_run<R, J + 1>(P, Q, tile, sb);
    }
}

template <int R>
__device__ __forceinline__ void smem_read(float2 (&P)[16], float2 (&Q)[16], const float2* tile, uint32_t tid) {
    uint32_t sb = swz(run_base(R, tid));
    asm volatile("" : "+r"(sb));
    if constexpr (R == 0) {
#define TB_RD0(K, V)                                                                                         \
    {                                                                                                        \
        const float4 e = *reinterpret_cast<const float4*>(tile + run_slot<0, (K) + 16 * (V)>(sb));         \
        if ((V) == 0) { P[K].x = e.x; Q[K].x = e.y; P[(K) + 1].x = e.z; Q[(K) + 1].x = e.w; }              \
        else          { P[K].y = e.x; Q[K].y = e.y; P[(K) + 1].y = e.z; Q[(K) + 1].y = e.w; }              \
    }
        TB_RD0(0, 0) TB_RD0(2, 0) TB_RD0(4, 0) TB_RD0(6, 0) TB_RD0(8, 0) TB_RD0(10, 0) TB_RD0(12, 0) TB_RD0(14, 0)
        TB_RD0(0, 1) TB_RD0(2, 1) TB_RD0(4, 1) TB_RD0(6, 1) TB_RD0(8, 1) TB_RD0(10, 1) TB_RD0(12, 1) TB_RD0(14, 1)
#undef TB_RD0
    } else {
        smem_read_run<R, 0>(P, Q, tile, sb);
    }
}

template <int R>
__device__ __forceinline__ void smem_write(const float2 (&P)[16], const float2 (&Q)[16], float2* tile, uint32_t tid) {
    uint32_t sb = swz(run_base(R, tid));
    asm volatile("" : "+r"(sb));
    if constexpr (R == 0) {
#define TB_WR0(K, V)                                                                                          \
    {                                                                                                         \
        const float4 e = (V) == 0 ? make_float4(P[K].x, Q[K].x, P[(K) + 1].x, Q[(K) + 1].x)                   \
                                  : make_float4(P[K].y, Q[K].y, P[(K) + 1].y, Q[(K) + 1].y);                  \
        *reinterpret_cast<float4*>(tile + run_slot<0, (K) + 16 * (V)>(sb)) = e;                              \
    }
        TB_WR0(0, 0) TB_WR0(2, 0) TB_WR0(4, 0) TB_WR0(6, 0) TB_WR0(8, 0) TB_WR0(10, 0) TB_WR0(12, 0) TB_WR0(14, 0)
        TB_WR0(0, 1) TB_WR0(2, 1) TB_WR0(4, 1) TB_WR0(6, 1) TB_WR0(8, 1) TB_WR0(10, 1) TB_WR0(12, 1) TB_WR0(14, 1)
#undef TB_WR0
    } else {
        smem_write_run<R, 0>(P, Q, tile, sb);
    }
}

// Hand the tile from register run R1 to run R2: every thread writes its
// entries back to their own slots, then reads the slots of its new run.
template <int R1, int R2>
__device__ __forceinline__ void transpose(float2 (&P)[16], float2 (&Q)[16], float2* tile, uint32_t tid) {
    smem_write<R1>(P, Q, tile, tid);
    __syncthreads();
    smem_read<R2>(P, Q, tile, tid);
}

template <class SH, int I, int R>
__device__ __forceinline__ void apply_step(float2 (&P)[16], float2 (&Q)[16], const float2* sc,
                                           uint32_t xmask, float scale, uint32_t tid) {
    constexpr StepSpec sp = step_spec(SH::TYPE, SH::M, I);
    constexpr int K = SH::C + sp.t - R;
    static_assert(K >= 0 && K < REG_BITS, "step target outside its register run");
    constexpr int kind = step_kind<SH>(I);
    // control: -1 none, 0..4 run bit, 5 external (a thread bit)
    constexpr int u = SH::C + sp.c;
    constexpr int CK = sp.c < 0 ? -1 : (in_run(u, R) ? u - R : 5);
    const float s = (I == 0) ? scale : 1.0f;
    asm volatile("" ::: "memory");  // load each step's coefficients just before it
    const float2* cf = sc + (I * 2 + (int)((xmask >> I) & 1u)) * CO;
    float2 c0[12], c1[12];
    if constexpr (CK == 5) {
        const uint32_t c = (run_base(R, tid) >> u) & 1u;
        load_cf(c0, cf + 12 * c, s);
    } else {
        load_cf(c0, cf, s);
    }
    if constexpr (CK >= 0 && CK < 4) load_cf(c1, cf + 12, s);
    if constexpr (kind == KIND_VT) {
        step_lanes<CK>(P, Q, c0, c1);
    } else {
        step_pairs<K, (kind == KIND_VC ? 4 : CK)>(P, Q, c0, c1);
    }
}

template <class SH, int I>
__device__ __forceinline__ void run_steps(float2 (&P)[16], float2 (&Q)[16], const float2* sc, uint32_t xmask,
                                          float scale, uint32_t tid, float2* tile) {
    if constexpr (I < SH::NS) {
        constexpr int R = SH::run_of(I);
        constexpr int RP = (I == 0) ? SH::first_run() : SH::run_of(I - 1);
        if constexpr (R != RP) transpose<RP, R>(P, Q, tile, tid);
        apply_step<SH, I, R>(P, Q, sc, xmask, scale, tid);
        run_steps<SH, I + 1>(P, Q, sc, xmask, scale, tid, tile);
    }
}

template <class SH>
__device__ __forceinline__ int64_t tile_addr(uint32_t idx, int lo) {
    if constexpr (SH::BOT) return idx;
    else return (int64_t)(idx & ((1u << SH::C) - 1u)) + ((int64_t)(idx >> SH::C) << lo);
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

__device__ __forceinline__ void cp_async16(float2* sdst, const float2* gsrc) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int PASS_STAGES = 3;

// Origin (in entries) of tile t of one batch element.
template <class SH>
__device__ __forceinline__ int64_t tile_origin(int64_t t, int lo) {
    if constexpr (SH::BOT) {
        return t << TILE_BITS;
    } else {
        const int nl = lo - SH::C;
        return ((t & (((int64_t)1 << nl) - 1)) << SH::C) | ((t >> nl) << (lo + SH::M));
    }
}

// Issue the 16-byte copies of tile gt into a stage (4096 chunks, 16 per thread;
// chunk c = j*256 + tid covers tile coordinates 2c, 2c+1).
// Chunk c = j*256 + tid: tile coordinate 2*tid + 512*j. The two terms have
// disjoint bits, so the swizzled slot is swz(2*tid) + 512*j and the HBM offset
// is tile_addr(2*tid) + tile_addr(512*j) (a per-thread base plus constants).
template <class SH>
__device__ __forceinline__ void issue_tile(const PassParams& p, int64_t gt, float2* stage, uint32_t s0,
                                           int64_t a0) {
    const int64_t b = gt >> p.tile_shift;
    const int64_t t = gt & (((int64_t)1 << p.tile_shift) - 1);
    const float2* base = p.B + b * p.b_stride + tile_origin<SH>(t, p.lo) + a0;
    const int64_t st = tile_addr<SH>(2u * PASS_THREADS, p.lo);  // HBM offset of j = 1
#pragma unroll
    for (int j = 0; j < TILE / 2 / PASS_THREADS; ++j)
        cp_async16(stage + s0 + 2u * PASS_THREADS * j, base + j * st);
}


template <int TYPE, int M>
__global__ void __launch_bounds__(PASS_THREADS, PASS_CTAS_PER_SM) pass_kernel(const PassParams p) {
    using SH = Shape<TYPE, M>;
    static_assert(SH::valid(), "invalid pass shape");
    static_assert(SH::NS <= 32, "step mask holds 32 steps");
    constexpr int NS = SH::NS;
    extern __shared__ __align__(16) float2 smem[];
    float2* sc = smem + PASS_STAGES * TILE;
    const uint32_t tid = threadIdx.x;

    stage_coefficients<SH>(p.steps, sc, tid);

    // per-thread parts of the tile copy addresses (see issue_tile)
    const uint32_t cs0 = swz(2u * tid);
    const int64_t ca0 = tile_addr<SH>(2u * tid, p.lo);
    // prologue: the first PASS_STAGES-1 tiles of this CTA
#pragma unroll
    for (int s = 0; s < PASS_STAGES - 1; ++s) {
        const int64_t gt = blockIdx.x + (int64_t)s * gridDim.x;
        if (gt < p.ntiles) issue_tile<SH>(p, gt, smem + s * TILE, cs0, ca0);
        cp_async_commit();
    }

    const int64_t tmask = ((int64_t)1 << p.tile_shift) - 1;
    float runmax = 0.0f;
    int64_t cur_b = -1;
    int cur_s = 0;
    float scale = 1.0f;
    uint32_t xmask = 0;
    int stage = 0;
    for (int64_t gt = blockIdx.x; gt < p.ntiles; gt += gridDim.x) {
        {   // keep PASS_STAGES-1 tiles in flight
            const int64_t nx = gt + (int64_t)(PASS_STAGES - 1) * gridDim.x;
            const int ns = (stage + PASS_STAGES - 1) % PASS_STAGES;
            if (nx < p.ntiles) issue_tile<SH>(p, nx, smem + ns * TILE, cs0, ca0);
            cp_async_commit();
        }
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

        float2* tile = smem + stage * TILE;
        cp_async_wait<PASS_STAGES - 1>();
        __syncthreads();

        float2 P[16], Q[16];
        smem_read<SH::first_run()>(P, Q, tile, tid);
        run_steps<SH, 0>(P, Q, sc, xmask, scale, tid, tile);
        constexpr int RL = SH::run_of(NS - 1);
        constexpr int RS = SH::last_run();
        if constexpr (RL != RS) transpose<RL, RS>(P, Q, tile, tid);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            runmax = fmaxf(runmax, fmaxf(fmaxf(fabsf(P[k].x), fabsf(P[k].y)), fmaxf(fabsf(Q[k].x), fabsf(Q[k].y))));
        {
            float2* dst = p.B + b * p.b_stride + tile_origin<SH>(t, p.lo);
            const uint32_t c0 = run_base(RS, tid);
            int64_t off0 = tile_addr<SH>(c0, p.lo);
            int64_t st = tile_addr<SH>(1u << RS, p.lo);
            asm volatile("" : "+l"(off0), "+l"(st));
#pragma unroll
            for (int v = 0; v < 2; ++v) {
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    float2* q = dst + off0 + (int64_t)(16 * v + 8 * g) * st;
                    asm volatile("" : "+l"(q));
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int k = 8 * g + j;
                        q[j * st] = v == 0 ? make_float2(P[k].x, Q[k].x) : make_float2(P[k].y, Q[k].y);
                    }
                }
            }
        }
        __syncthreads();  // every thread is done with this stage before it is refilled
        stage = (stage + 1) % PASS_STAGES;
    }
    cp_async_wait<0>();
    if (cur_b >= 0) flush_max(runmax, p.maxs + cur_b * p.sstride + p.slot + 1);
}

template <int TYPE, int M>
constexpr int pass_smem_bytes() {
    return (PASS_STAGES * TILE + pass_nsteps(TYPE, M) * 2 * CO) * (int)sizeof(float2);
}

// Launchers, one translation unit per pass type (pass_t<type>.cu).
cudaError_t launch_pass_t0(int M, const PassParams& p, int grid, cudaStream_t st);
cudaError_t launch_pass_t1(int M, const PassParams& p, int grid, cudaStream_t st);
cudaError_t launch_pass_t2(int M, const PassParams& p, int grid, cudaStream_t st);
cudaError_t launch_pass_t3(int M, const PassParams& p, int grid, cudaStream_t st);
cudaError_t launch_pass_t4(int M, const PassParams& p, int grid, cudaStream_t st);
cudaError_t launch_pass_t5(int M, const PassParams& p, int grid, cudaStream_t st);
cudaError_t launch_pass_t6(int M, const PassParams& p, int grid, cudaStream_t st);

template <int TYPE, int M>
cudaError_t launch_one(const PassParams& p, int grid, cudaStream_t st) {
    if constexpr (!Shape<TYPE, M>::valid()) {
        return cudaErrorInvalidValue;
    } else {
    constexpr int smem = pass_smem_bytes<TYPE, M>();
    cudaError_t e = cudaFuncSetAttribute(pass_kernel<TYPE, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    pass_kernel<TYPE, M><<<grid, PASS_THREADS, smem, st>>>(p);
    return cudaGetLastError();
    }
}

#define TB_DEFINE_LAUNCH_PASS(TYPE, NAME)                                         \
    cudaError_t NAME(int M, const PassParams& p, int grid, cudaStream_t st) {    \
        switch (M) {                                                             \
            case 5: return launch_one<TYPE, 5>(p, grid, st);                     \
            case 6: return launch_one<TYPE, 6>(p, grid, st);                     \
            case 7: return launch_one<TYPE, 7>(p, grid, st);                     \
            case 8: return launch_one<TYPE, 8>(p, grid, st);                     \
            case 9: return launch_one<TYPE, 9>(p, grid, st);                     \
            case 10: return launch_one<TYPE, 10>(p, grid, st);                   \
            default: return cudaErrorInvalidValue;                               \
        }                                                                        \
    }

}  // namespace tb
