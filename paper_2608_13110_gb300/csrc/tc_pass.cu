// Dense tensor-core pass of the temporal-boundary sweep (precision TF32X3 /
// BF16X3), sm_103a.
//
// One pass applies a dense 2^WB x 2^WB complex block (composed on the host
// from the paired steps of Algorithm 1 whose target and control lie in the
// window of address bits [lo, lo+WB)) to every vector of the boundary, a
// vector being the 2^WB entries that share all other address bits. As a real
// GEMM over the interleaved (re, im) components:
//     D[v][n] = sum_k A[v][k] Bm[k][n],   k = 2*j + part,  n = 2*j' + part'.
// Precision: A = A_hi + A_lo and Bm = B_hi + B_lo are split into two operands
// of the tensor-core input type (TF32 or BF16) and
//     D = A_lo.B_hi + A_hi.B_lo + A_hi.B_hi
// is accumulated in FP32 in tensor memory (the lo.lo term is dropped).
//
// Kernel layout (one warpgroup per CTA, two CTAs per SM):
//   * thread i owns TMEM lane i and vector i of the current tile (a tile is
//     128 vectors: the 7 lowest address bits outside the window);
//   * the split block Bm (hi, lo) sits in shared memory for the whole launch
//     as the K-major B operand (canonical layout, no swizzle);
//   * per tile: each thread loads its vector from HBM, applies the register
//     pre-step, splits, and writes A_hi / A_lo into its TMEM lane; one thread
//     issues 3 x 8 MMAs (M = 128 vectors, N = 2^(WB+1), A from TMEM) and
//     commits them to an mbarrier; the next tile's loads are issued while the
//     MMAs run; then each thread reads its lane of D, applies the register
//     post-step, tracks the rescaling maximum and stores its vector in place.
//   * every mbarrier wait is bounded; a wait that gives up is counted in a
//     device word, the CTA stops issuing work, waits (bounded) once more for
//     its MMAs and releases its tensor memory before it exits.

#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "tc_pass.cuh"
#include "tc_ptx.cuh"

namespace tb {

namespace {

using namespace tcx;

__device__ int g_fault_word;

template <int KIND>
struct TcCfg {
    static constexpr bool BF16 = KIND == TB_PRECISION_BF16X3;
    static constexpr int WB = BF16 ? TC_WB_BF16 : TC_WB_TF32;
    static constexpr int NV = 1 << WB;                // complex entries per vector
    static constexpr int K = 2 * NV;                  // real reduction length
    static constexpr int N = 2 * NV;                  // real outputs per vector
    static constexpr int EB = BF16 ? 2 : 4;           // operand bytes
    static constexpr int KSTEP = BF16 ? 16 : 8;       // K of one MMA instruction
    static constexpr int NKSTEPS = K / KSTEP;         // 8 for both kinds
    static constexpr int ACOLS = K * EB / 4;          // TMEM columns of one A part
    static constexpr int A_HI = 0, A_LO = ACOLS, D_COL = 2 * ACOLS;
    static constexpr int TMEM_COLS = 256;             // power of two >= D_COL + N
    static constexpr int MAT_BYTES = 2 * K * N * EB;  // hi + lo
    static constexpr uint32_t LBO = 128;                       // next core matrix along K
    static constexpr uint32_t SBO = (K * EB / 16) * 128;       // next 8-row group along N
    static constexpr int SMEM_BYTES = 80 * 1024;      // > 228 KB / 3: at most two CTAs per SM
    static_assert(D_COL + N <= TMEM_COLS, "tensor memory budget");
    static_assert(MAT_BYTES + 1024 + 64 <= SMEM_BYTES, "shared memory budget");
    static_assert(2 * TMEM_COLS <= 512, "two CTAs per SM must fit in tensor memory");
    // instruction descriptor: D = F32, A and B of the operand type, both
    // K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
    static constexpr uint32_t FMT = BF16 ? 1u : 2u;
    static constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) |
                                      ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
};

constexpr uint32_t WAIT_TRIES = 1u << 22;
constexpr uint32_t SELFTEST_TRIES = 1u << 11;

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_t, uint32_t a_t, uint64_t bdesc, uint32_t acc) {
    if constexpr (KIND == TB_PRECISION_BF16X3) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_t),
            "r"(a_t), "l"(bdesc), "r"(TcCfg<KIND>::IDESC), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_t),
            "r"(a_t), "l"(bdesc), "r"(TcCfg<KIND>::IDESC), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void flush_max_tc(float m, uint32_t* dst) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(dst, __float_as_uint(m));
}

__device__ __forceinline__ int rescale_exp_tc(float m) {
    if (!(m > 0.0f) || !isfinite(m)) return 0;
    int e;
    frexpf(m, &e);
    return max(-100, min(100, -e));
}

__device__ __forceinline__ float2 cmul_add(float2 a, float2 x, float2 b, float2 y) {
    // a*x + b*y
    float2 r;
    r.x = fmaf(a.x, x.x, fmaf(-a.y, x.y, fmaf(b.x, y.x, -b.y * y.y)));
    r.y = fmaf(a.x, x.y, fmaf(a.y, x.x, fmaf(b.x, y.y, b.y * y.x)));
    return r;
}

// Controlled 2x2 step on window bit T of a vector held in registers; the
// control value is c (the same for the whole vector) or, when CBIT >= 0,
// window bit CBIT of each entry. g = G[x][c*4 + a'*2 + s].
template <int NV, int T, int CBIT>
__device__ __forceinline__ void reg_step(float2 (&v)[NV], const float2* g, int c) {
    float2 g0[4], g1[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) { g0[e] = g[e]; g1[e] = g[4 + e]; }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        if (j & (1 << T)) continue;
        const int cv = CBIT >= 0 ? ((j >> (CBIT < 0 ? 0 : CBIT)) & 1) : c;
        const float2 v0 = v[j], v1 = v[j | (1 << T)];
        const float2 a00 = cv ? g1[0] : g0[0], a01 = cv ? g1[1] : g0[1];
        const float2 a10 = cv ? g1[2] : g0[2], a11 = cv ? g1[3] : g0[3];
        v[j] = cmul_add(a00, v0, a01, v1);
        v[j | (1 << T)] = cmul_add(a10, v0, a11, v1);
    }
}

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, TC_CTAS_PER_SM) tc_pass_kernel(const TcParams p) {
    using C = TcCfg<KIND>;
    constexpr int NV = C::NV;
    extern __shared__ __align__(16) uint8_t dsm[];
    uint8_t* base = dsm + ((1024 - (smem_u32(dsm) & 1023)) & 1023);
    uint8_t* smat = base;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(base + C::MAT_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(base + C::MAT_BYTES + 8);
    int* s_abort = reinterpret_cast<int*>(base + C::MAT_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5;

    // the split block, resident for the whole launch
    {
        const int4* src = reinterpret_cast<const int4*>(p.mat);
        int4* dst = reinterpret_cast<int4*>(smat);
        for (int i = tid; i < C::MAT_BYTES / 16; i += TC_THREADS) dst[i] = src[i];
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(mbar), 1);
        *s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t mb = smem_u32(mbar);
    const uint32_t tries = p.selftest ? SELFTEST_TRIES : WAIT_TRIES;
    const uint32_t b_hi = smem_u32(smat), b_lo = b_hi + C::MAT_BYTES / 2;

    const int lo = p.lo;
    const int64_t lomask = ((int64_t)1 << lo) - 1;
    const int64_t tmask = ((int64_t)1 << p.tile_shift) - 1;
    auto vec_addr = [&](int64_t gt) {  // entry 0 of this thread's vector in tile gt
        const int64_t b = gt >> p.tile_shift;
        const int64_t u = ((gt & tmask) << TC_VEC_BITS) | tid;
        return b * p.b_stride + (u & lomask) + ((u >> lo) << (lo + C::WB));
    };
    auto load_vec = [&](float2 (&v)[NV], int64_t a0) {
        const float2* src = p.B + a0;
        if (lo == 0) {
#pragma unroll
            for (int j = 0; j < NV; j += 2) {
                const float4 q = *reinterpret_cast<const float4*>(src + j);
                v[j] = make_float2(q.x, q.y);
                v[j + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < NV; ++j) v[j] = src[(int64_t)j << lo];
        }
    };

    float2 v[NV];
    int64_t gt = blockIdx.x;
    if (gt < p.ntiles) load_vec(v, vec_addr(gt));

    float runmax = 0.0f;
    int64_t cur_b = -1;
    float scale = 1.0f;
    int xpre = 0, xpost = 0;
    uint32_t phase = 0;
    bool mma_pending = false;  // thread 0: MMAs committed whose completion it has not seen

    for (; gt < p.ntiles; gt += gridDim.x) {
        const int64_t b = gt >> p.tile_shift;
        const int64_t a0 = vec_addr(gt);
        if (b != cur_b) {
            if (cur_b >= 0) flush_max_tc(runmax, p.maxs + cur_b * p.sstride + p.slot + 1);
            runmax = 0.0f;
            cur_b = b;
            const int s = rescale_exp_tc(__uint_as_float(p.maxs[b * p.sstride + p.slot]));
            scale = ldexpf(1.0f, s);
            if ((gt & tmask) == 0 && tid == 0) p.exps[b * p.sstride + p.slot + 1] = s;
            const uint8_t* xb = p.bits + b * p.n;
            xpre = p.pre.xq >= 0 ? (xb[p.pre.xq] ? 1 : 0) : 0;
            xpost = p.post.xq >= 0 ? (xb[p.post.xq] ? 1 : 0) : 0;
        } else if ((gt & tmask) == 0 && tid == 0) {
            p.exps[b * p.sstride + p.slot + 1] = rescale_exp_tc(__uint_as_float(p.maxs[b * p.sstride + p.slot]));
        }

        // ---- input: rescale, pre-step, split into TMEM
#pragma unroll
        for (int j = 0; j < NV; ++j) { v[j].x *= scale; v[j].y *= scale; }
        if (p.pre.t >= 0) {
            const float2* g = p.steps[p.pre.step].g[xpre];
            const int c = p.pre.cmode == 1 ? (int)(((a0 - b * p.b_stride) >> p.pre.cbit) & 1) : 0;
            if (p.pre.t == 0) reg_step<NV, 0, -1>(v, g, c);
            else reg_step<NV, C::WB - 1, -1>(v, g, c);
        }
        if constexpr (C::BF16) {
#pragma unroll
            for (int c16 = 0; c16 < NV / 16; ++c16) {
                uint32_t rh[16], rl[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const float2 z = v[16 * c16 + e];
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(z.x, z.y);
                    const float2 hf = __bfloat1622float2(h2);
                    const __nv_bfloat162 l2 = __floats2bfloat162_rn(z.x - hf.x, z.y - hf.y);
                    rh[e] = *reinterpret_cast<const uint32_t*>(&h2);
                    rl[e] = *reinterpret_cast<const uint32_t*>(&l2);
                }
                tmem_st16(lane + C::A_HI + 16 * c16, rh);
                tmem_st16(lane + C::A_LO + 16 * c16, rl);
            }
        } else {
#pragma unroll
            for (int c8 = 0; c8 < NV / 8; ++c8) {
                uint32_t rh[16], rl[16];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float2 z = v[8 * c8 + e];
                    const uint32_t hx = to_tf32(z.x), hy = to_tf32(z.y);
                    rh[2 * e] = hx;
                    rh[2 * e + 1] = hy;
                    rl[2 * e] = to_tf32(z.x - __uint_as_float(hx));
                    rl[2 * e + 1] = to_tf32(z.y - __uint_as_float(hy));
                }
                tmem_st16(lane + C::A_HI + 16 * c8, rh);
                tmem_st16(lane + C::A_LO + 16 * c8, rl);
            }
        }
        tmem_wait_st();
        tc_fence_before();
        __syncthreads();
        if (*s_abort) break;  // a wait gave up: issue nothing more
        tc_fence_after();

        // ---- the block: D = A_lo.B_hi + A_hi.B_lo + A_hi.B_hi. The FP32
        // accumulator is rounded after every MMA; adding the two small
        // correction products first keeps their rounding at their own scale,
        // so only the 8 MMAs of the leading product round at full magnitude.
        if (tid == 0 && !p.selftest) {
            const uint32_t d_t = tmem + C::D_COL;
#pragma unroll
            for (int prod = 0; prod < 3; ++prod) {
                const uint32_t a_col = prod == 0 ? C::A_LO : C::A_HI;
                const uint32_t b_addr = prod == 1 ? b_lo : b_hi;
#pragma unroll
                for (int ks = 0; ks < C::NKSTEPS; ++ks)
                    mma<KIND>(d_t, tmem + a_col + 8 * ks, smem_desc(b_addr + 256 * ks, C::LBO, C::SBO),
                              (prod > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(mb);
            mma_pending = true;
        }

        // ---- next tile's loads overlap the MMAs
        const int64_t nx = gt + gridDim.x;
        if (nx < p.ntiles) load_vec(v, vec_addr(nx));

        const bool ok = mbar_wait(mb, phase, tries);
        if (!ok) {
            atomicAdd(p.fault, 1);
            *s_abort = 1;
        } else if (tid == 0) {
            mma_pending = false;
        }
        phase ^= 1u;
        tc_fence_after();
        // a warp with a lane whose wait gave up neither reads the accumulator
        // nor stores: the tile is left as it was (and the call reports the fault)
        if (__any_sync(0xffffffffu, !ok)) continue;

        // ---- output: read D, post-step, maximum, store in place
        float2* dst = p.B + a0;
        constexpr int HALF = NV / 2;
        constexpr int NCH = NV / 8;  // chunks of 8 entries (16 columns)
#pragma unroll
        for (int c8 = 0; c8 < NCH / 2; ++c8) {
            uint32_t r0[16], r1[16];
            tmem_ld16(lane + C::D_COL + 16 * c8, r0);
            tmem_ld16(lane + C::D_COL + 16 * (c8 + NCH / 2), r1);
            tmem_wait_ld();
            float2 w0[8], w1[8];  // entries 8*c8 + e and HALF + 8*c8 + e
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                w0[e] = make_float2(__uint_as_float(r0[2 * e]), __uint_as_float(r0[2 * e + 1]));
                w1[e] = make_float2(__uint_as_float(r1[2 * e]), __uint_as_float(r1[2 * e + 1]));
            }
            if (p.post.t >= 0) {
                // target window bit WB-1, control window bit WB-2
                const float2* g = p.steps[p.post.step].g[xpost];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int cv = ((8 * c8 + e) >> (C::WB - 2)) & 1;
                    const float2 v0 = w0[e], v1 = w1[e];
                    w0[e] = cmul_add(g[cv * 4 + 0], v0, g[cv * 4 + 1], v1);
                    w1[e] = cmul_add(g[cv * 4 + 2], v0, g[cv * 4 + 3], v1);
                }
            }
#pragma unroll
            for (int e = 0; e < 8; ++e)
                runmax = fmaxf(runmax, fmaxf(fmaxf(fabsf(w0[e].x), fabsf(w0[e].y)),
                                             fmaxf(fabsf(w1[e].x), fabsf(w1[e].y))));
            if (lo == 0) {
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    *reinterpret_cast<float4*>(dst + 8 * c8 + e) = make_float4(w0[e].x, w0[e].y, w0[e + 1].x, w0[e + 1].y);
                    *reinterpret_cast<float4*>(dst + HALF + 8 * c8 + e) =
                        make_float4(w1[e].x, w1[e].y, w1[e + 1].x, w1[e + 1].y);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    dst[(int64_t)(8 * c8 + e) << lo] = w0[e];
                    dst[(int64_t)(HALF + 8 * c8 + e) << lo] = w1[e];
                }
            }
        }
    }
    if (cur_b >= 0) flush_max_tc(runmax, p.maxs + cur_b * p.sstride + p.slot + 1);
    // Tensor memory may be freed only once no MMA can still write it. Thread 0
    // issued every MMA; if it has not seen its last commit complete, it waits
    // once more (bounded). If that wait gives up too, the CTA keeps its tensor
    // memory (freeing it under a running MMA could corrupt another CTA's
    // accumulator) and raises TC_TMEM_HELD in the fault word; the host then
    // refuses further tensor-core passes in this process.
    if (tid == 0) {
        bool held = false;
        if (mma_pending && !mbar_wait(mb, phase ^ 1u, WAIT_TRIES)) held = true;
        *s_abort = held ? 2 : 0;
        if (held) atomicOr(p.fault, TC_TMEM_HELD);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && *s_abort != 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
}

template <int KIND>
cudaError_t launch_kind(const TcParams& p, int grid, cudaStream_t st) {
    using C = TcCfg<KIND>;
    static bool attr = false;  // per process; the attribute is per function
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(tc_pass_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    tc_pass_kernel<KIND><<<grid, TC_THREADS, C::SMEM_BYTES, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_pass(int precision, const TcParams& p, int grid, cudaStream_t st) {
    if (precision == TB_PRECISION_BF16X3) return launch_kind<TB_PRECISION_BF16X3>(p, grid, st);
    if (precision == TB_PRECISION_TF32X3) return launch_kind<TB_PRECISION_TF32X3>(p, grid, st);
    return cudaErrorInvalidValue;
}

namespace {
std::atomic<bool> g_tc_disabled{false};
}

int note_faults(int word) {
    if (word & TC_TMEM_HELD) g_tc_disabled = true;
    return word & ~TC_TMEM_HELD;
}

bool tc_passes_disabled() { return g_tc_disabled.load(); }

int* device_fault_word() {
    // looked up once per device (the symbol's address does not change)
    static std::mutex mu;
    static void* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev] && cudaGetSymbolAddress(&addr[dev], g_fault_word) != cudaSuccess) addr[dev] = nullptr;
    return static_cast<int*>(addr[dev]);
}

}  // namespace tb
