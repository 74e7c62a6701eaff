// Device kernels of an open plan (Algorithm 2): join of the early region with
// the boundary, late-region crossings, and the final FP64 scaling.
//
// Boundary layout after the sweep of rows 0..n-k-1: entry (r << k) | s holds
// B[sigma], s = the k crossing bits of the early region (address bits
// 0..k-1), r = the late crossing bits (address bits k..h-1, the next one to
// be contracted lowest).

#include "open_kernels.cuh"

namespace tb {

namespace {

__device__ __forceinline__ float2 cmac(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}

// Join: Z[r][y] = sum_s B[r][s] E[s][y], in place. A CTA owns JOIN_TILE
// consecutive entries (R = JOIN_TILE / 2^k whole rows) and copies them to
// shared memory; E is staged through shared memory in chunks of SC rows
// (32 KB) and used by every row of the tile. Each thread accumulates a TR x TC
// register tile (columns cg, cg + NCG, ..., so that consecutive lanes read
// consecutive E entries and write consecutive outputs; TR rows) over all s
// and finally writes it back over the rows the CTA read.
template <int K>
__global__ void __launch_bounds__(256, 2) join_kernel(const JoinParams p) {
    constexpr int NY = 1 << K;
    constexpr int R = JOIN_TILE / NY;
    constexpr int TC = NY < 8 ? NY : 8;
    constexpr int NCG = NY / TC;       // column groups
    constexpr int TR = 32 / TC;        // rows per thread
    constexpr int SC = NY >= 64 ? 4096 / NY : NY;  // E rows per chunk (32 KB)
    static_assert((256 / NCG) * TR == R, "join tiling");
    static_assert(NY % SC == 0, "E chunks");
    extern __shared__ __align__(16) float2 smem[];
    float2* sB = smem;                 // JOIN_TILE entries
    float2* sE = smem + JOIN_TILE;     // SC x NY entries
    const int tid = threadIdx.x;
    const int cg = tid % NCG, rg = tid / NCG;
    for (int64_t tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
        const int64_t b = tile / p.tiles_per_b;
        const int64_t t = tile - b * p.tiles_per_b;
        float2* Z = p.B + b * p.b_stride + t * JOIN_TILE;
        __syncthreads();  // the previous tile is done with sB and sE
        for (int i = tid; i < JOIN_TILE / 2; i += 256)
            reinterpret_cast<float4*>(sB)[i] = reinterpret_cast<const float4*>(Z)[i];
        float2 acc[TR][TC];
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[a][c] = make_float2(0.f, 0.f);
        for (int s0 = 0; s0 < NY; s0 += SC) {
            __syncthreads();  // sE free (and sB loaded on the first chunk)
            for (int i = tid; i < SC * NY / 2; i += 256)
                reinterpret_cast<float4*>(sE)[i] = __ldg(reinterpret_cast<const float4*>(p.E + (int64_t)s0 * NY) + i);
            __syncthreads();
#pragma unroll 4
            for (int ss = 0; ss < SC; ++ss) {
                float2 e[TC];
#pragma unroll
                for (int c = 0; c < TC; ++c) e[c] = sE[ss * NY + cg + NCG * c];
#pragma unroll
                for (int a = 0; a < TR; ++a) {
                    const float2 bv = sB[(rg * TR + a) * NY + s0 + ss];
#pragma unroll
                    for (int c = 0; c < TC; ++c) acc[a][c] = cmac(acc[a][c], bv, e[c]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < TR; ++a)
#pragma unroll
            for (int c = 0; c < TC; ++c) Z[(rg * TR + a) * NY + cg + NCG * c] = acc[a][c];
    }
}

// One late crossing: out[r'][y] = seg( in[2r'][y] + w^(y_0) in[2r'+1][y] ),
// w = -1 for CZ (diag(1, 1, 1, w) in general). Rows are 2^k entries at a
// stride of 2^(k + shift) entries; in place (out == in, out_shift = in_shift
// + 1) output row r' overwrites input row 2r', which only the CTA that reads
// rows 2r' and 2r'+1 touches, after it has read them (a chunk is read whole
// into shared memory before it is written back).
// A CTA works on chunks of 2^OPEN_CHUNK_BITS output entries (or one row when
// 2^k is larger) in shared memory; the segment's operations act on chunk
// index bits 0..k-1.
__global__ void __launch_bounds__(256) late_kernel(const LateParams p) {
    __shared__ float2 v[1 << OPEN_CHUNK_BITS];
    __shared__ OpenOp ops[LATE_MAX_OPS];
    const int tid = threadIdx.x;
    for (int i = tid; i < p.nops; i += 256) ops[i] = p.ops[i];
    const int NY = 1 << p.k;
    const int chunk = NY > (1 << OPEN_CHUNK_BITS) ? NY : (1 << OPEN_CHUNK_BITS);  // k <= 10: 1024
    const int64_t per_b = p.out_entries;  // output entries per batch element
    const int64_t chunks_per_b = (per_b + chunk - 1) / chunk;
    const int64_t nchunks = chunks_per_b * p.nbatch;
    __syncthreads();
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t b = ch / chunks_per_b;
        const int64_t o0 = (ch - b * chunks_per_b) * chunk;  // first output entry
        const int len = (int)((per_b - o0) < chunk ? (per_b - o0) : chunk);
        const float2* in = p.in + b * p.in_stride;
        float2* out = p.out + b * p.out_stride;
        __syncthreads();
        for (int e = tid; e < len; e += 256) {
            const int64_t o = o0 + e;
            const int64_t rp = o >> p.k;
            const int y = (int)(o & (NY - 1));
            const float2 a = in[((2 * rp) << (p.k + p.in_shift)) + y];
            const float2 c = in[((2 * rp + 1) << (p.k + p.in_shift)) + y];
            const float2 wc = (y & 1) ? make_float2(c.x * p.w.x - c.y * p.w.y, c.x * p.w.y + c.y * p.w.x) : c;
            v[e] = make_float2(a.x + wc.x, a.y + wc.y);
        }
        __syncthreads();
        for (int q = 0; q < p.nops; ++q) {
            const OpenOp& op = ops[q];
            if (op.kind == 0) {
                const int half = len >> 1;
                for (int e = tid; e < half; e += 256) {
                    const int lo = ((e >> op.j) << (op.j + 1)) | (e & ((1 << op.j) - 1));
                    const int hi = lo | (1 << op.j);
                    const float2 x0 = v[lo], x1 = v[hi];
                    float2 r0 = make_float2(0.f, 0.f), r1 = make_float2(0.f, 0.f);
                    r0 = cmac(cmac(r0, op.m[0], x0), op.m[1], x1);
                    r1 = cmac(cmac(r1, op.m[2], x0), op.m[3], x1);
                    v[lo] = r0;
                    v[hi] = r1;
                }
            } else {  // entangler diag(1, 1, 1, m[0]) on bits j, j+1
                const float2 w = op.m[0];
                for (int e = tid; e < len; e += 256)
                    if (((e >> op.j) & 1) && ((e >> (op.j + 1)) & 1))
                        v[e] = make_float2(v[e].x * w.x - v[e].y * w.y, v[e].x * w.y + v[e].y * w.x);
            }
            __syncthreads();
        }
        for (int e = tid; e < len; e += 256) {
            const int64_t o = o0 + e;
            out[((o >> p.k) << (p.k + p.out_shift)) + (o & (NY - 1))] = v[e];
        }
    }
}

// out[b][y] (FP64) = Z[b][y] * 2^(-sum of the sweep's rescaling exponents).
__global__ void open_finalize_kernel(const OpenFinalParams p) {
    const int64_t b = blockIdx.y;
    double sc = 0.0;
    for (int s = 0; s < p.nslots; ++s) sc += (double)p.exps[b * p.sstride + s];
    const double f = exp2(-sc);
    const int NY = 1 << p.k;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < NY; y += gridDim.x * blockDim.x) {
        const float2 z = p.Z[b * p.b_stride + y];
        p.out[(b * NY + y) * 2] = (double)z.x * f;
        p.out[(b * NY + y) * 2 + 1] = (double)z.y * f;
    }
}

constexpr int JOIN_SMEM = JOIN_TILE * 8 + 32 * 1024;  // boundary rows + one E chunk

template <int K>
cudaError_t launch_join_k(const JoinParams& p, int grid, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(join_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   JOIN_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    join_kernel<K><<<grid, 256, JOIN_SMEM, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_join(int k, const JoinParams& p, int grid, cudaStream_t st) {
    switch (k) {
        case 1: return launch_join_k<1>(p, grid, st);
        case 2: return launch_join_k<2>(p, grid, st);
        case 3: return launch_join_k<3>(p, grid, st);
        case 4: return launch_join_k<4>(p, grid, st);
        case 5: return launch_join_k<5>(p, grid, st);
        case 6: return launch_join_k<6>(p, grid, st);
        case 7: return launch_join_k<7>(p, grid, st);
        case 8: return launch_join_k<8>(p, grid, st);
        case 9: return launch_join_k<9>(p, grid, st);
        case 10: return launch_join_k<10>(p, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_late(const LateParams& p, int grid, cudaStream_t st) {
    if (p.nops > LATE_MAX_OPS || p.k > OPEN_CHUNK_BITS) return cudaErrorInvalidValue;
    late_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_open_finalize(const OpenFinalParams& p, int nbatch, cudaStream_t st) {
    const int NY = 1 << p.k;
    dim3 grid((unsigned)((NY + 255) / 256), (unsigned)nbatch);
    open_finalize_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace tb
