// Row-0 writer, last-row reduction, finalisation and the narrow-boundary
// kernel (arXiv 2608.13110, Sec. 3.1, Algorithm 1).
#include "misc_kernels.cuh"

namespace tb {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

__device__ __forceinline__ float2 cmac2m(float2 g0, float2 a, float2 g1, float2 b) {
    float2 r;
    r.x = fmaf(g0.x, a.x, fmaf(-g0.y, a.y, fmaf(g1.x, b.x, -g1.y * b.y)));
    r.y = fmaf(g0.x, a.y, fmaf(g0.y, a.x, fmaf(g1.x, b.y, g1.y * b.x)));
    return r;
}

__device__ __forceinline__ int rescale_exp_m(float m) {
    if (!(m > 0.0f) || !isfinite(m)) return 0;
    int e;
    frexpf(m, &e);
    return max(-100, min(100, -e));
}

__device__ __forceinline__ void flush_max_m(float m, uint32_t* dst) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(dst, __float_as_uint(m));
}

// ---------------------------------------------------------------------------
// Row 0 (B <- pi[1]): B_0[s] = a0[s_0] prod_(p>=1) M_p[s_p, s_(p-1)] E_x[s_(h-1)],
// factored as low[s_low] * mid[s_(k-1)][s_mid] * top[x][s_(k+m-1)][s_top].
// One chunk = the 2^k entries sharing their high bits.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) init_kernel(const InitParams p) {
    const int64_t cmask = ((int64_t)1 << p.chunk_shift) - 1;
    const int nk = 1 << p.k;
    float runmax = 0.0f;
    int64_t cur_b = -1;
    for (int64_t g = blockIdx.x; g < p.nchunks; g += gridDim.x) {
        const int64_t b = g >> p.chunk_shift;
        const int64_t c = g & cmask;
        if (b != cur_b) {
            if (cur_b >= 0) flush_max_m(runmax, p.maxs + cur_b * p.sstride);
            runmax = 0.0f;
            cur_b = b;
        }
        const int x = p.bits[b * p.n] ? 1 : 0;
        const int64_t sm = c & (((int64_t)1 << p.m) - 1);
        const int64_t st = c >> p.m;
        const int bm = (int)((sm >> (p.m - 1)) & 1);
        const float2 tv = p.topt[(((int64_t)(x * 2 + bm)) << p.top) + st];
        const float2 g0 = cmul(p.mid[sm], tv);
        const float2 g1 = cmul(p.mid[((int64_t)1 << p.m) + sm], tv);
        float2* dst = p.B + b * p.b_stride + (c << p.k);
        for (int e = threadIdx.x; e < nk; e += blockDim.x) {
            const float2 v = cmul(p.low[e], ((e >> (p.k - 1)) & 1) ? g1 : g0);
            dst[e] = v;
            runmax = fmaxf(runmax, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
    }
    if (cur_b >= 0) flush_max_m(runmax, p.maxs + cur_b * p.sstride);
}

cudaError_t launch_init(const InitParams& p, int grid, cudaStream_t st) {
    init_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Last row: psi = sum_s B[s] V[s], V[s] = top[x][s_top] . mid[s_mid] . low[s_low]
// (row vector . 2x2 . column vector). FP32 within a chunk, FP64 across chunks
// and blocks; partial sums in a fixed order (deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 block_sum_d2(double2 v, double2* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { s.x += red[i].x; s.y += red[i].y; }
    return s;  // valid in thread 0
}

__global__ void __launch_bounds__(REDUCE_THREADS) reduce_kernel(const ReduceParams p) {
    extern __shared__ float2 slow[];  // [2^k][2]
    __shared__ double2 red[REDUCE_THREADS / 32];
    const int nk = 1 << p.k;
    for (int i = threadIdx.x; i < 2 * nk; i += blockDim.x) slow[i] = p.low[i];
    __syncthreads();
    const int b = blockIdx.x / p.blocks_per_b;
    const int j = blockIdx.x - b * p.blocks_per_b;
    const int x = p.bits[(int64_t)b * p.n + p.n - 1] ? 1 : 0;
    const int s = rescale_exp_m(__uint_as_float(p.maxs[b * p.sstride + p.slot]));
    if (j == 0 && threadIdx.x == 0) p.exps[b * p.sstride + p.slot + 1] = s;
    const double sc = ldexp(1.0, s);
    const int64_t nchunks = (int64_t)1 << p.chunk_shift;
    const int64_t mmask = ((int64_t)1 << p.m) - 1;
    double ar = 0.0, ai = 0.0;
    for (int64_t c = j; c < nchunks; c += p.blocks_per_b) {
        const int64_t sm = c & mmask, stp = c >> p.m;
        const float2* tv = p.topt + ((((int64_t)x << p.top) + stp) << 1);
        const float2* md = p.mid + (sm << 2);
        const float2 r0 = cfma(tv[1], md[2], cmul(tv[0], md[0]));
        const float2 r1 = cfma(tv[1], md[3], cmul(tv[0], md[1]));
        const float2* src = p.B + (int64_t)b * p.b_stride + (c << p.k);
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        // 16 independent loads in flight per thread, then the products
        for (int e0 = threadIdx.x; e0 < nk; e0 += 16 * REDUCE_THREADS) {
            float2 v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = e0 + i * REDUCE_THREADS;
                v[i] = e < nk ? __ldcs(src + e) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = e0 + i * REDUCE_THREADS;
                if (e < nk) {
                    a0 = cfma(v[i], slow[2 * e], a0);
                    a1 = cfma(v[i], slow[2 * e + 1], a1);
                }
            }
        }
        const float2 cv = cfma(r1, a1, cmul(r0, a0));
        ar += (double)cv.x;
        ai += (double)cv.y;
    }
    const double2 tot = block_sum_d2(make_double2(ar * sc, ai * sc), red);
    if (threadIdx.x == 0) p.partials[blockIdx.x] = tot;
}

cudaError_t launch_reduce(const ReduceParams& p, cudaStream_t st) {
    const int smem = (2 << p.k) * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    reduce_kernel<<<p.nbatch * p.blocks_per_b, REDUCE_THREADS, smem, st>>>(p);
    return cudaGetLastError();
}

// psi_b = (sum of its partials) * 2^-(sum of its rescaling exponents).
__global__ void finalize_kernel(const FinalizeParams p) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int l = threadIdx.x & 31;
    if (b >= p.nbatch) return;
    double sr = 0.0, si = 0.0;
    for (int i = l; i < p.blocks_per_b; i += 32) {
        const double2 v = p.partials[(int64_t)b * p.blocks_per_b + i];
        sr += v.x;
        si += v.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (l == 0) {
        long long S = 0;
        for (int i = 0; i < p.nslots; ++i) S += p.exps[b * p.sstride + i];
        const int Si = (int)max(-1000000LL, min(1000000LL, S));
        p.out[2 * b] = scalbn(sr, -Si);
        p.out[2 * b + 1] = scalbn(si, -Si);
    }
}

// ---- log-XEB (Sec. 5.2, normalized log-XEB estimator) -----------------------
// F = gamma + n ln 2 + (1/N) sum_i ln |amp_i|^2, entirely in FP64 on the
// device. One CTA: thread t sums the terms i = t, t + 1024, ... in index
// order, then a fixed binary tree adds the 1024 partial sums, so the result
// does not depend on scheduling. A zero amplitude contributes -inf.
constexpr int XEB_THREADS = 1024;

__global__ void __launch_bounds__(XEB_THREADS) log_xeb_kernel(const double2* amp, int64_t nb, int n, double* out) {
    __shared__ double part[XEB_THREADS];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < nb; i += XEB_THREADS) {
        const double2 a = amp[i];
        s += log(fma(a.x, a.x, a.y * a.y));
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = XEB_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double gamma = 0.57721566490153286060651209;  // Euler's constant
        out[0] = gamma + (double)n * 0.69314718055994530941723212 + part[0] / (double)nb;
    }
}

cudaError_t launch_log_xeb(const double2* amp, int64_t nb, int n, double* out, cudaStream_t st) {
    log_xeb_kernel<<<1, XEB_THREADS, 0, st>>>(amp, nb, n, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t st) {
    const int warps = 4;
    finalize_kernel<<<(p.nbatch + warps - 1) / warps, 32 * warps, 0, st>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Narrow boundaries (h <= 12): one CTA per bitstring keeps B in shared memory
// for the whole sweep: row 0, every paired step of rows 1..n-2 in order, the
// last-row contraction; power-of-two rescaling after every row.
// ---------------------------------------------------------------------------
__device__ float block_max_f(float v, float* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float m = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
    return m;
}

__device__ int small_rescale(float2* Bs, int N, float* red) {
    float m = 0.0f;
    for (int e = threadIdx.x; e < N; e += blockDim.x) m = fmaxf(m, fmaxf(fabsf(Bs[e].x), fabsf(Bs[e].y)));
    m = block_max_f(m, red);
    const int s = rescale_exp_m(m);
    const float sc = ldexpf(1.0f, s);
    for (int e = threadIdx.x; e < N; e += blockDim.x) Bs[e] = make_float2(Bs[e].x * sc, Bs[e].y * sc);
    __syncthreads();
    return s;
}

// Bitstring b of one narrow plan, the whole sweep in shared memory (Bs holds
// 2^h entries).
__device__ void small_sweep(const SmallParams& p, int b, float2* Bs, float* redf, double2* redd) {
    const uint8_t* xb = p.bits + (int64_t)b * p.n;
    const int h = p.h, N = 1 << h;
    const int x0 = xb[0] ? 1 : 0;
    for (int e = threadIdx.x; e < N; e += blockDim.x)
        Bs[e] = cmul(p.init_low[e], p.init_top[x0 * 2 + ((e >> (h - 1)) & 1)]);
    __syncthreads();
    long long S = small_rescale(Bs, N, redf);
    int step = 0;
    for (int row = 0; row < p.nrows; ++row) {
        for (; step < p.row_end[row]; ++step) {
            const int t = p.tgt[step], u = p.ctl[step], q = p.xq[step];
            const int var = (q >= 0 && xb[q]) ? 1 : 0;
            const float2* g = p.steps[step].g[var];
            for (int i = threadIdx.x; i < (N >> 1); i += blockDim.x) {
                const int i0 = ((i >> t) << (t + 1)) | (i & ((1 << t) - 1));
                const int i1 = i0 | (1 << t);
                const int c = u >= 0 ? (i0 >> u) & 1 : 0;
                const float2* gg = g + 4 * c;
                const float2 a = Bs[i0], bb = Bs[i1];
                Bs[i0] = cmac2m(gg[0], a, gg[1], bb);
                Bs[i1] = cmac2m(gg[2], a, gg[3], bb);
            }
            __syncthreads();
        }
        S += small_rescale(Bs, N, redf);
    }
    const int xl = xb[p.n - 1] ? 1 : 0;
    double ar = 0.0, ai = 0.0;
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        const float2 v = cmul(Bs[e], p.red_low[2 * e + xl]);
        ar += (double)v.x;
        ai += (double)v.y;
    }
    const double2 tot = block_sum_d2(make_double2(ar, ai), redd);
    if (threadIdx.x == 0) {
        const int Si = (int)max(-1000000LL, min(1000000LL, S));
        p.out[2 * b] = scalbn(tot.x, -Si);
        p.out[2 * b + 1] = scalbn(tot.y, -Si);
    }
}

__global__ void __launch_bounds__(SMALL_THREADS) small_kernel(const SmallParams p) {
    extern __shared__ float2 Bs[];
    __shared__ float redf[SMALL_THREADS / 32];
    __shared__ double2 redd[SMALL_THREADS / 32];
    small_sweep(p, blockIdx.x, Bs, redf, redd);
}

// Several narrow plans in one launch: block i evaluates bitstring
// i - first_block of the item whose block range holds i.
__global__ void __launch_bounds__(SMALL_THREADS) small_multi_kernel(const SmallItem* items, int nitems) {
    extern __shared__ float2 Bs[];
    __shared__ float redf[SMALL_THREADS / 32];
    __shared__ double2 redd[SMALL_THREADS / 32];
    int lo = 0, hi = nitems - 1;
    const int64_t blk = blockIdx.x;
    while (lo < hi) {  // last item with first_block <= blk
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first_block <= blk) lo = mid;
        else hi = mid - 1;
    }
    const SmallParams p = items[lo].p;
    small_sweep(p, (int)(blk - items[lo].first_block), Bs, redf, redd);
}

cudaError_t launch_small_multi(const SmallItem* d_items, int nitems, int64_t nblocks, int hmax, cudaStream_t st) {
    const int smem = (1 << hmax) * (int)sizeof(float2);
    small_multi_kernel<<<(unsigned)nblocks, SMALL_THREADS, smem, st>>>(d_items, nitems);
    return cudaGetLastError();
}

cudaError_t launch_small(const SmallParams& p, cudaStream_t st) {
    const int smem = (1 << p.h) * (int)sizeof(float2);
    small_kernel<<<p.nb, SMALL_THREADS, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace tb
