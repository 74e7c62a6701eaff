// Fused staircase pass over the temporal boundary (arXiv 2608.13110,
// Sec. 3.1, Algorithm 1: every paired step contracts two row tensors into the
// boundary; Sec. 5.2 merges small branch tensors before they touch the large
// boundary, which here becomes: apply every step of one window of address
// bits in a single read + write of the boundary).
//
// A pass applies a compile-time sequence of controlled 2x2 steps to every
// tile of 2^13 complex64 entries: the window's M address bits plus 13-M low
// address bits (the 13 lowest bits when the window starts at bit 0). Each of
// the 256 threads holds 32 entries in registers. A step acts on a 5-bit
// "register run" of the tile; between runs the tile is transposed through
// shared memory (XOR-swizzled, conflict-free for every run base 0..8). The
// first and last run keep 8 or more consecutive entries on consecutive lanes,
// so loads and stores go straight between HBM and registers.
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
        if (M < MIN_WINDOW || M > MAX_WINDOW) return false;
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
__device__ __forceinline__ uint32_t swz(uint32_t idx) {
    return idx ^ (((idx >> 6) & 1u) << 1) ^ (((idx >> 7) & 1u) << 2) ^ ((((idx >> 5) ^ (idx >> 8)) & 1u) << 3);
}

// a*g0 + b*g1 in complex arithmetic.
__device__ __forceinline__ float2 cmac2(float2 g0, float2 a, float2 g1, float2 b) {
    float2 r;
    r.x = fmaf(g0.x, a.x, fmaf(-g0.y, a.y, fmaf(g1.x, b.x, -g1.y * b.y)));
    r.y = fmaf(g0.x, a.y, fmaf(g0.y, a.x, fmaf(g1.x, b.y, g1.y * b.x)));
    return r;
}

// G = (G[a'][s]) on register bit K, same matrix for every pair.
template <int K>
__device__ __forceinline__ void step_plain(float2 (&v)[32], const float2 (&g)[4]) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j & (1 << K)) continue;
        const int j1 = j | (1 << K);
        const float2 a = v[j], b = v[j1];
        v[j] = cmac2(g[0], a, g[1], b);
        v[j1] = cmac2(g[2], a, g[3], b);
    }
}

// G[c] on register bit K, control c on register bit KC.
template <int K, int KC>
__device__ __forceinline__ void step_ctrl(float2 (&v)[32], const float2 (&g0)[4], const float2 (&g1)[4]) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j & (1 << K)) continue;
        const int j1 = j | (1 << K);
        const float2 a = v[j], b = v[j1];
        if ((j >> KC) & 1) {
            v[j] = cmac2(g1[0], a, g1[1], b);
            v[j1] = cmac2(g1[2], a, g1[3], b);
        } else {
            v[j] = cmac2(g0[0], a, g0[1], b);
            v[j1] = cmac2(g0[2], a, g0[3], b);
        }
    }
}

__device__ __forceinline__ void load4(float2 (&g)[4], const float2* src, float s) {
#pragma unroll
    for (int i = 0; i < 4; ++i) g[i] = make_float2(src[i].x * s, src[i].y * s);
}

// Registers <-> shared tile for register run R. Run 0 holds the two entries
// of each 16-byte chunk in one thread and moves them as one 16-byte access.
template <int R>
__device__ __forceinline__ void smem_read(float2 (&v)[32], const float2* tile, uint32_t tid) {
    uint32_t b = run_base(R, tid);
    asm volatile("" : "+r"(b));
    if constexpr (R == 0) {
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
            const float4 q = *reinterpret_cast<const float4*>(tile + swz(b | (uint32_t)j));
            v[j] = make_float2(q.x, q.y);
            v[j + 1] = make_float2(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = tile[swz(b | ((uint32_t)j << R))];
    }
}

template <int R>
__device__ __forceinline__ void smem_write(const float2 (&v)[32], float2* tile, uint32_t tid) {
    uint32_t b = run_base(R, tid);
    asm volatile("" : "+r"(b));
    if constexpr (R == 0) {
#pragma unroll
        for (int j = 0; j < 32; j += 2)
            *reinterpret_cast<float4*>(tile + swz(b | (uint32_t)j)) = make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y);
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[swz(b | ((uint32_t)j << R))] = v[j];
    }
}

// Hand the tile from register run R1 to run R2: every thread writes its
// entries back to their own slots, then reads the slots of its new run.
template <int R1, int R2>
__device__ __forceinline__ void transpose(float2 (&v)[32], float2* tile, uint32_t tid) {
    smem_write<R1>(v, tile, tid);
    __syncthreads();
    smem_read<R2>(v, tile, tid);
}

template <class SH, int I, int R>
__device__ __forceinline__ void apply_step(float2 (&v)[32], const float2* sg, uint32_t xmask,
                                           float scale, uint32_t tid) {
    constexpr StepSpec sp = step_spec(SH::TYPE, SH::M, I);
    constexpr int s = SH::C + sp.t;
    constexpr int K = s - R;
    static_assert(K >= 0 && K < REG_BITS, "step target outside its register run");
    const float sc = (I == 0) ? scale : 1.0f;
    asm volatile("" ::: "memory");  // load each step's coefficients just before it
    const float2* g = sg + I * 16 + (((xmask >> I) & 1u) ? 8 : 0);
    if constexpr (sp.c < 0) {
        float2 gg[4];
        load4(gg, g, sc);
        step_plain<K>(v, gg);
    } else {
        constexpr int u = SH::C + sp.c;
        if constexpr (in_run(u, R)) {
            float2 g0[4], g1[4];
            load4(g0, g, sc);
            load4(g1, g + 4, sc);
            step_ctrl<K, u - R>(v, g0, g1);
        } else {
            const uint32_t c = (run_base(R, tid) >> u) & 1u;
            float2 gg[4];
            load4(gg, g + 4 * c, sc);
            step_plain<K>(v, gg);
        }
    }
}

template <class SH, int I>
__device__ __forceinline__ void run_steps(float2 (&v)[32], const float2* sg, uint32_t xmask,
                                          float scale, uint32_t tid, float2* tile) {
    if constexpr (I < SH::NS) {
        constexpr int R = SH::run_of(I);
        constexpr int RP = (I == 0) ? SH::first_run() : SH::run_of(I - 1);
        if constexpr (R != RP) transpose<RP, R>(v, tile, tid);
        apply_step<SH, I, R>(v, sg, xmask, scale, tid);
        run_steps<SH, I + 1>(v, sg, xmask, scale, tid, tile);
    }
}

// Global offset (entries, from the tile origin) of tile coordinate idx.
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
template <class SH>
__device__ __forceinline__ void issue_tile(const PassParams& p, int64_t gt, float2* stage, uint32_t tid) {
    const int64_t b = gt >> p.tile_shift;
    const int64_t t = gt & (((int64_t)1 << p.tile_shift) - 1);
    const float2* base = p.B + b * p.b_stride + tile_origin<SH>(t, p.lo);
#pragma unroll
    for (int j = 0; j < TILE / 2 / PASS_THREADS; ++j) {
        const uint32_t idx = 2u * ((uint32_t)j * PASS_THREADS + tid);
        cp_async16(stage + swz(idx), base + tile_addr<SH>(idx, p.lo));
    }
}

template <int TYPE, int M>
__global__ void __launch_bounds__(PASS_THREADS, 1) pass_kernel(const PassParams p) {
    using SH = Shape<TYPE, M>;
    static_assert(SH::valid(), "invalid pass shape");
    constexpr int NS = SH::NS;
    extern __shared__ __align__(16) float2 smem[];
    float2* sg = smem + PASS_STAGES * TILE;
    const uint32_t tid = threadIdx.x;

    for (int i = tid; i < NS * 16; i += PASS_THREADS) sg[i] = reinterpret_cast<const float2*>(p.steps)[i];

    // prologue: the first PASS_STAGES-1 tiles of this CTA
#pragma unroll
    for (int s = 0; s < PASS_STAGES - 1; ++s) {
        const int64_t gt = blockIdx.x + (int64_t)s * gridDim.x;
        if (gt < p.ntiles) issue_tile<SH>(p, gt, smem + s * TILE, tid);
        cp_async_commit();
    }

    const int64_t tmask = ((int64_t)1 << p.tile_shift) - 1;
    float runmax = 0.0f;
    int64_t cur_b = -1;
    int stage = 0;
    for (int64_t gt = blockIdx.x; gt < p.ntiles; gt += gridDim.x) {
        {   // keep PASS_STAGES-1 tiles in flight
            const int64_t nx = gt + (int64_t)(PASS_STAGES - 1) * gridDim.x;
            const int ns = (stage + PASS_STAGES - 1) % PASS_STAGES;
            if (nx < p.ntiles) issue_tile<SH>(p, nx, smem + ns * TILE, tid);
            cp_async_commit();
        }
        const int64_t b = gt >> p.tile_shift;
        const int64_t t = gt & tmask;
        if (b != cur_b) {
            if (cur_b >= 0) flush_max(runmax, p.maxs + cur_b * p.sstride + p.slot + 1);
            runmax = 0.0f;
            cur_b = b;
        }
        const int s = rescale_exp(__uint_as_float(p.maxs[b * p.sstride + p.slot]));
        if (t == 0 && tid == 0) p.exps[b * p.sstride + p.slot + 1] = s;
        const float scale = ldexpf(1.0f, s);
        const uint8_t* xb = p.bits + b * p.n;
        uint32_t xmask = 0;
        if (p.xs_step0 >= 0) xmask |= (xb[p.xs_q0] ? 1u : 0u) << p.xs_step0;
        if (p.xs_step1 >= 0) xmask |= (xb[p.xs_q1] ? 1u : 0u) << p.xs_step1;

        float2* tile = smem + stage * TILE;
        cp_async_wait<PASS_STAGES - 1>();
        __syncthreads();

        float2 v[32];
        smem_read<SH::first_run()>(v, tile, tid);
        run_steps<SH, 0>(v, sg, xmask, scale, tid, tile);
        constexpr int RL = SH::run_of(NS - 1);
        constexpr int RS = SH::last_run();
        if constexpr (RL != RS) transpose<RL, RS>(v, tile, tid);
#pragma unroll
        for (int j = 0; j < 32; ++j) runmax = fmaxf(runmax, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
        {
            float2* dst = p.B + b * p.b_stride + tile_origin<SH>(t, p.lo);
            const uint32_t c0 = run_base(RS, tid);
            int64_t off0 = tile_addr<SH>(c0, p.lo);
            int64_t st = tile_addr<SH>(1u << RS, p.lo);
            asm volatile("" : "+l"(off0), "+l"(st));
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float2* q = dst + off0 + (int64_t)(8 * g) * st;
                asm volatile("" : "+l"(q));
#pragma unroll
                for (int j = 0; j < 8; ++j) q[j * st] = v[8 * g + j];
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
    return (PASS_STAGES * TILE + pass_nsteps(TYPE, M) * 16) * (int)sizeof(float2);
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
    constexpr int smem = pass_smem_bytes<TYPE, M>();
    cudaError_t e = cudaFuncSetAttribute(pass_kernel<TYPE, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    pass_kernel<TYPE, M><<<grid, PASS_THREADS, smem, st>>>(p);
    return cudaGetLastError();
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
