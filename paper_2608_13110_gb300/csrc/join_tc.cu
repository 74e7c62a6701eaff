// Join of Algorithm 2 on the tensor cores (sm_103a, tcgen05, 3xTF32).
//
// After the sweep of the fixed region the boundary is a matrix B[r][s]: row r
// = the late crossing bits, column s = the k crossing bits of the early region
// (address bits 0..k-1, so a row is 2^k consecutive entries). The early
// region, contracted on the host, is the dense 2^k x 2^k complex matrix E
// (Sec. 4.3, Algorithm 2), and the join is the complex matrix product
//     Z[r][y] = sum_s B[r][s] E[s][y].
// As a real GEMM over the boundary's (re, im) floats, D[r][n] = sum_kk
// A[r][kk] Bm[kk][n] with kk = 2s + part, n = 2y + part and K = N = 2^(k+1);
// the host stores Bm = Bm_hi + Bm_lo (TF32) in blocks of JOIN_KC K rows by NT
// N columns (canonical K-major layout). Here A = A_hi + A_lo is split per
// element and D = A_lo.Bm_hi + A_hi.Bm_lo + A_hi.Bm_hi accumulates in FP32 in
// tensor memory (the lo.lo term is dropped), correction products first.
// The tensor cores' FP32 accumulation drifts over long K (measured: the
// join's error grew in proportion to K, 1.6e-5 at K = 2048), so each segment
// of JOIN_SEG_CHUNKS K chunks accumulates in its own tensor-memory sum (two,
// alternating) and the segments are added in FP32 registers, round to nearest.
//
// One CTA per SM (persistent): 4 row warps, an MMA warp and a copy warp. A
// work item is 128 rows x NT output columns: row thread i owns row i
// (tensor-memory lane i). Per K chunk of JOIN_KC reals, in one of four
// stages: the copy thread brings the chunk's Bm block (hi, lo; one bulk copy)
// and the item's 128 x JOIN_KC A tile (one tensor copy) into shared memory as
// soon as the stage's previous MMAs have finished; every row thread splits
// its row's JOIN_KC floats and writes A_hi / A_lo into the stage's tensor
// memory; the MMA thread, once both are in place, issues 3 x 4 MMAs (M = 128,
// N = NT, K = 8) into the segment's sum and commits them to the stage's
// mbarrier. The three roles meet only at mbarriers, so copies, splits and
// MMAs of different chunks overlap. When a segment's first chunk has been
// split, the rows add the previous segment's sum (their row) into their
// registers. The epilogue writes the row sums to Z out of place (the input
// rows are needed by the item's other N tiles).
//
// Every wait is bounded; a give-up is counted in the fault word, the CTA
// stops together (__syncthreads_or), waits (bounded) for its last bulk copy
// and its last MMAs, and frees tensor memory only when no MMA can still write
// it (otherwise it raises TC_TMEM_HELD; see tc_pass.cuh).

#include <cuda.h>

#include "open_kernels.cuh"
#include "tc_pass.cuh"
#include "tc_ptx.cuh"

namespace tb {

namespace {

using namespace tcx;

constexpr int JT_ROWS = 128;      // row warps 0..3: thread i owns row i (tensor-memory lane i)
constexpr int JT_THREADS = JT_ROWS + 64;  // + the MMA warp + the copy warp
constexpr uint32_t JT_WAIT_TRIES = 1u << 22;
constexpr uint32_t JT_TMEM_COLS = 512;
constexpr int JT_STAGES = 4;         // B blocks in shared memory, A splits in tensor memory
constexpr uint32_t JT_A_COL = 256;  // A stage s: hi at 256 + 64 s, lo at 256 + 64 s + 32
// segment sums: columns [0, NT) and [NT, 2 NT), NT <= 128
constexpr int JT_MIN_SMEM = 120 * 1024;  // more than half the SM: one CTA per SM (it holds 512 columns)

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* m, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

template <int NT>
__global__ void __launch_bounds__(JT_THREADS, 1)
    join_tc_kernel(const JoinTcParams p, const __grid_constant__ CUtensorMap amap) {
    constexpr uint32_t PART = (uint32_t)NT * JOIN_KC * 4;  // one of hi / lo
    constexpr uint32_t BLK = 2 * PART;
    constexpr uint32_t ABYTES = 128 * JOIN_KC * 4;          // 128 rows x JOIN_KC floats
    constexpr uint32_t STG = BLK + ABYTES;                   // one stage: B block, then A rows
    constexpr uint32_t LBO = 128, SBO = (JOIN_KC / 4) * 128;
    // D = F32, A and B TF32, both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
    constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    static_assert(2 * NT <= (int)JT_A_COL && JT_A_COL + 64 * JT_STAGES <= JT_TMEM_COLS, "tensor memory plan");
    extern __shared__ __align__(16) uint8_t dsm[];
    uint8_t* base = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
    // mbarriers: b_full[S] (bulk copy landed), a_full[S] (128 rows split into
    // the stage), mma_done[S] (the stage's MMAs finished), d_free[2] (a segment
    // sum has been read by every row)
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + JT_STAGES * STG);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3 * JT_STAGES + 2);
    int* s_stop = reinterpret_cast<int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sB0 = smem_u32(base);
    const uint32_t bfull0 = smem_u32(bars), afull0 = bfull0 + 8 * JT_STAGES, mdone0 = afull0 + 8 * JT_STAGES,
                   dfree0 = mdone0 + 8 * JT_STAGES;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(JT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < JT_STAGES; ++s) {
            mbar_init(bfull0 + 8 * s, 1);
            mbar_init(afull0 + 8 * s, JT_ROWS);
            mbar_init(mdone0 + 8 * s, 1);
        }
        mbar_init(dfree0, JT_ROWS);
        mbar_init(dfree0 + 8, JT_ROWS);
        *s_stop = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const int KR = p.KR;
    const int nkc = KR / JOIN_KC, ntn = KR / NT;
    const int nseg = (nkc + JOIN_SEG_CHUNKS - 1) / JOIN_SEG_CHUNKS;
    const int64_t nrb = p.rows / 128;  // row blocks per batch element
    const int64_t items = (int64_t)p.nbatch * nrb * ntn;
    // Chunk c of this CTA (counted over all its items) uses stage c % S for its
    // B block (shared memory) and A split (tensor memory); segment g (counted
    // over all items) accumulates in D[g % 2].
    auto stage_of = [](uint32_t c) { return c % JT_STAGES; };
    auto par_of = [](uint32_t c) { return (c / JT_STAGES) & 1u; };
    auto stopped = [&]() { return *(volatile int*)s_stop != 0; };
    auto give_up = [&]() {
        if (atomicExch(s_stop, 1) == 0) atomicAdd(p.fault, 1);
    };

    __shared__ int s_held;
    if (warp == JT_ROWS / 32 + 1) {
        // ------------------------------------------------ copy warp (lane 0)
        // Chunk cc's B block and A tile go to stage cc % S once the MMAs of
        // chunk cc - S (the stage's previous reader, with the rows' A split in
        // tensor memory) have finished; copies run ahead as far as that allows.
        if ((tid & 31) == 0) {
        uint32_t c = 0;
        bool loaded[JT_STAGES];  // a copy was issued into the stage
        uint32_t load_par[JT_STAGES];
        for (int s = 0; s < JT_STAGES; ++s) { loaded[s] = false; load_par[s] = 0; }
        bool ok = true;
        for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const int nt = (int)(it % ntn);
            const int arow0 = (int)((it / ntn) * 128);  // first row of the item (batch elements are contiguous)
            for (int kc = 0; kc < nkc && ok; ++kc) {
                const uint32_t cc = c + kc, s = stage_of(cc);
                if (cc >= JT_STAGES) ok = mbar_wait(mdone0 + 8 * s, par_of(cc - JT_STAGES), JT_WAIT_TRIES);
                if (ok && stopped()) ok = false;
                if (!ok) break;
                expect_tx(bfull0 + 8 * s, STG);
                bulk_load(sB0 + s * STG, p.Es + ((int64_t)nt * nkc + kc) * BLK, BLK, bfull0 + 8 * s);
                tma_load_2d(sB0 + s * STG + BLK, &amap, kc * JOIN_KC, arow0, bfull0 + 8 * s);
                loaded[s] = true;
                load_par[s] = par_of(cc);
            }
            c += nkc;
        }
        if (!ok) give_up();
        // the copies issued must land before the CTA's shared memory goes (only
        // this thread arms b_full, so each stage's latest phase is its last copy)
        for (int s = 0; s < JT_STAGES; ++s)
            if (loaded[s]) (void)mbar_wait(bfull0 + 8 * s, load_par[s], JT_WAIT_TRIES);
        }
        __syncwarp();
    } else if (warp == JT_ROWS / 32) {
        // ------------------------------------------------ MMA warp (lane 0)
        if ((tid & 31) == 0) {
        uint32_t c = 0, g = 0;
        int64_t last_commit = -1;
        bool ok = true;
        for (int64_t it = blockIdx.x; it < items && ok && !stopped(); it += gridDim.x) {
            for (int kc = 0; kc < nkc; ++kc) {
                const uint32_t cc = c + kc, s = stage_of(cc);
                const int sg = kc / JOIN_SEG_CHUNKS;
                const uint32_t gg = g + sg;
                const bool first = kc % JOIN_SEG_CHUNKS == 0;
                // a segment's first MMA overwrites D[gg % 2], last read for segment gg - 2
                if (first && gg >= 2) ok = mbar_wait(dfree0 + 8 * (gg & 1u), ((gg - 2) >> 1) & 1u, JT_WAIT_TRIES);
                if (ok) ok = mbar_wait(bfull0 + 8 * s, par_of(cc), JT_WAIT_TRIES);
                if (ok) ok = mbar_wait(afull0 + 8 * s, par_of(cc), JT_WAIT_TRIES);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(NT * (gg & 1u));
                const uint32_t bh = sB0 + s * STG, bl = bh + PART;
                const uint32_t a_hi = tmem + JT_A_COL + 64 * s, a_lo = a_hi + 32;
#pragma unroll
                for (int prod = 0; prod < 3; ++prod) {
                    const uint32_t a = prod == 0 ? a_lo : a_hi;
                    const uint32_t bb = prod == 1 ? bl : bh;
#pragma unroll
                    for (int ks = 0; ks < JOIN_KC / 8; ++ks)
                        mma_tf32(d, a + 8 * ks, smem_desc(bb + 256 * ks, LBO, SBO), IDESC,
                                 (!first || prod > 0 || ks > 0) ? 1u : 0u);
                }
                mma_commit(mdone0 + 8 * s);
                last_commit = cc;
            }
            c += nkc;
            g += nseg;
        }
        if (!ok) give_up();
        // the MMAs must finish before the tensor memory can be freed
        bool held = false;
        if (last_commit >= 0 &&
            !mbar_wait(mdone0 + 8 * stage_of((uint32_t)last_commit), par_of((uint32_t)last_commit), JT_WAIT_TRIES))
            held = true;
        if (held) atomicOr(p.fault, TC_TMEM_HELD);
        s_held = held ? 1 : 0;
        }
        __syncwarp();
    } else {
    // ---------------------------------------------------- row warps (0..3)
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t c = 0, g = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int nt = (int)(it % ntn);
        const int64_t rbg = it / ntn;
        const int64_t b = rbg / nrb, rb = rbg - b * nrb;
        const int64_t row = rb * 128 + tid;
        float acc[NT];
#pragma unroll
        for (int e = 0; e < NT; ++e) acc[e] = 0.0f;
        // add segment gg (its last chunk is cl) to acc, then free its sum
        // (the decisions below are warp-uniform: tcgen05.ld / st are warp-collective)
        auto add_segment = [&](uint32_t gg, uint32_t cl) -> bool {
            const bool w = mbar_wait(mdone0 + 8 * stage_of(cl), par_of(cl), JT_WAIT_TRIES);
            if (__any_sync(0xffffffffu, !w)) return false;
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < NT / 16; ++q) {
                uint32_t r[16];
                tmem_ld16(lane + NT * (gg & 1u) + 16 * q, r);
                tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[16 * q + e] += __uint_as_float(r[e]);
            }
            tc_fence_before();
            mbar_arrive(dfree0 + 8 * (gg & 1u));
            return true;
        };
        for (int kc = 0; kc < nkc; ++kc) {
            const uint32_t cc = c + kc, s = stage_of(cc);
            // the stage's A tile (and B block) landed; its tensor memory was
            // freed by the MMAs of chunk cc - S before the copies were issued
            const bool w = mbar_wait(bfull0 + 8 * s, par_of(cc), JT_WAIT_TRIES);
            if (__any_sync(0xffffffffu, !w || stopped())) {
                ok = false;
                break;
            }
            // row tid of the A tile: 128 bytes, 16-byte chunks XOR-swizzled by row % 8
            const uint8_t* arow_s = base + s * STG + BLK + tid * (JOIN_KC * 4);
            float4 ac[JOIN_KC / 4];
#pragma unroll
            for (int q = 0; q < JOIN_KC / 4; ++q)
                ac[q] = *reinterpret_cast<const float4*>(arow_s + 16 * (q ^ (tid & 7)));
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 v = ac[4 * half + q];
                    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t h = to_tf32(x[e]);
                        hi[4 * q + e] = h;
                        lo[4 * q + e] = to_tf32(x[e] - __uint_as_float(h));
                    }
                }
                tmem_st16(lane + JT_A_COL + 64 * s + 16 * half, hi);
                tmem_st16(lane + JT_A_COL + 64 * s + 32 + 16 * half, lo);
            }
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(afull0 + 8 * s);
            // the previous segment's sum is complete once its last chunk's MMAs are
            if (kc % JOIN_SEG_CHUNKS == 0 && kc > 0 && !add_segment(g + kc / JOIN_SEG_CHUNKS - 1, cc - 1)) {
                ok = false;
                break;
            }
        }
        if (!ok) break;
        c += nkc;
        g += nseg;
        if (!add_segment(g - 1, c - 1)) {
            ok = false;
            break;
        }
        float4* zrow = reinterpret_cast<float4*>(p.out + 2 * (b * p.out_stride + row * (KR / 2)) + nt * NT);
#pragma unroll
        for (int q = 0; q < NT / 4; ++q) zrow[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    if (!ok) give_up();
    }  // row warps

    // exit: the MMA thread has seen its copies land and its MMAs finish (or
    // raised TC_TMEM_HELD); only then is the tensor memory freed
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && !s_held) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(JT_TMEM_COLS)
                     : "memory");
    }
}

template <int NT>
cudaError_t launch_nt(const JoinTcParams& p, const CUtensorMap& m, int grid, cudaStream_t st) {
    constexpr int need = 1024 + JT_STAGES * (2 * NT * JOIN_KC * 4 + 128 * JOIN_KC * 4) + 8 * (3 * JT_STAGES + 2) + 16;
    constexpr int smem = need > JT_MIN_SMEM ? need : JT_MIN_SMEM;
    static_assert(smem <= 227 * 1024, "join smem");
    const cudaError_t e = cudaFuncSetAttribute(join_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    join_tc_kernel<NT><<<grid, JT_THREADS, smem, st>>>(p, m);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_join_tc(int k, const JoinTcParams& p, const CUtensorMap& amap, int grid, cudaStream_t st) {
    switch (join_nt(k)) {
        case 32: return launch_nt<32>(p, amap, grid, st);
        case 64: return launch_nt<64>(p, amap, grid, st);
        case 128: return launch_nt<128>(p, amap, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tb
