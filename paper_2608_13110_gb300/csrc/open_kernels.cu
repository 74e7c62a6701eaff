// Device kernels of an open plan (Algorithm 2): join of the early region with
// the boundary, late-region crossings, and the final FP64 scaling.
//
// Boundary layout after the sweep of rows 0..n-k-1: entry (r << k) | s holds
// B[sigma], s = the k crossing bits of the early region (address bits
// 0..k-1), r = the late crossing bits (address bits k..h-1, the next one to
// be contracted lowest).

#include <algorithm>

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
// + 1) output row r' overwrites input row 2r', which only the warp that reads
// rows 2r' and 2r'+1 touches, after it has read them.
// One warp per output row (k >= 5: lanes hold y bits 0..4, R = 2^(k-5)
// registers the rest) or per 2^(5-k) rows (k < 5: the lanes' high bits pick
// the row): the segment's operations act on y, so a gate on a lane bit is a
// shuffle and a gate on a register bit is register arithmetic; no block
// barrier after the operations are staged.
template <int K>
struct LateShape {
    static constexpr int LB = K >= 5 ? 5 : K;              // y bits on lanes
    static constexpr int R = K >= 5 ? 1 << (K - 5) : 1;    // registers per lane
    static constexpr int ROWS = K >= 5 ? 1 : 1 << (5 - K);  // rows per warp
};

template <int K, int JR>
__device__ __forceinline__ void late_reg_gate(float2 (&v)[LateShape<K>::R], const float2* m) {
    constexpr int R = LateShape<K>::R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r & (1 << JR)) continue;
        const int r1 = r | (1 << JR);
        const float2 x0 = v[r], x1 = v[r1];
        v[r] = cmac(cmac(make_float2(0.f, 0.f), m[0], x0), m[1], x1);
        v[r1] = cmac(cmac(make_float2(0.f, 0.f), m[2], x0), m[3], x1);
    }
}

template <int K>
__global__ void __launch_bounds__(256) late_kernel(const LateParams p) {
    using S = LateShape<K>;
    constexpr int R = S::R, LB = S::LB, ROWS = S::ROWS, NRB = K - LB;  // NRB: y bits in registers
    __shared__ OpenOp ops[LATE_MAX_OPS];
    for (int i = threadIdx.x; i < p.nops; i += blockDim.x) ops[i] = p.ops[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int yl = lane & ((1 << LB) - 1);  // this lane's y bits 0..LB-1
    const int rsub = lane >> LB;            // row within the warp's group (k < 5)
    const int64_t rows_out = p.out_entries >> K;
    const int64_t groups_per_b = (rows_out + ROWS - 1) / ROWS;
    const int64_t ngroups = groups_per_b * p.nbatch;
    const int64_t wstep = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t gi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < ngroups; gi += wstep) {
        const int64_t b = gi / groups_per_b;
        const int64_t rp = (gi - b * groups_per_b) * ROWS + rsub;
        const bool valid = rp < rows_out;
        const float2* in = p.in + b * p.in_stride;
        float2* out = p.out + b * p.out_stride;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = yl | (r << LB);
            v[r] = make_float2(0.f, 0.f);
            if (valid) {
                const float2 a = in[((2 * rp) << (K + p.in_shift)) + y];
                const float2 c = in[((2 * rp + 1) << (K + p.in_shift)) + y];
                const float2 wc = (y & 1) ? make_float2(c.x * p.w.x - c.y * p.w.y, c.x * p.w.y + c.y * p.w.x) : c;
                v[r] = make_float2(a.x + wc.x, a.y + wc.y);
            }
        }
        for (int q = 0; q < p.nops; ++q) {  // warp-uniform
            const OpenOp& op = ops[q];
            const int j = op.j;
            if (op.kind == 0) {
                if (j < LB) {  // partner lane = lane ^ 2^j
                    const int a = (yl >> j) & 1;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        float2 t;
                        t.x = __shfl_xor_sync(0xffffffffu, v[r].x, 1 << j);
                        t.y = __shfl_xor_sync(0xffffffffu, v[r].y, 1 << j);
                        // lo lane: m0 own + m1 partner; hi lane: m2 partner + m3 own
                        v[r] = a ? cmac(cmac(make_float2(0.f, 0.f), op.m[2], t), op.m[3], v[r])
                                 : cmac(cmac(make_float2(0.f, 0.f), op.m[0], v[r]), op.m[1], t);
                    }
                } else if constexpr (NRB > 0) {
                    switch (j - LB) {
                        case 0: late_reg_gate<K, 0>(v, op.m); break;
                        case 1: if constexpr (NRB > 1) late_reg_gate<K, 1>(v, op.m); break;
                        case 2: if constexpr (NRB > 2) late_reg_gate<K, 2>(v, op.m); break;
                        case 3: if constexpr (NRB > 3) late_reg_gate<K, 3>(v, op.m); break;
                        case 4: if constexpr (NRB > 4) late_reg_gate<K, 4>(v, op.m); break;
                        default: break;
                    }
                }
            } else {  // entangler diag(1, 1, 1, m[0]) on bits j, j+1
                const float2 w = op.m[0];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int y = yl | (r << LB);
                    if (((y >> j) & 1) && ((y >> (j + 1)) & 1))
                        v[r] = make_float2(v[r].x * w.x - v[r].y * w.y, v[r].x * w.y + v[r].y * w.x);
                }
            }
        }
        if (valid) {
#pragma unroll
            for (int r = 0; r < R; ++r) out[(rp << (K + p.out_shift)) + (yl | (r << LB))] = v[r];
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

template <int K>
cudaError_t launch_late_k(const LateParams& p, int max_grid, cudaStream_t st) {
    constexpr int ROWS = LateShape<K>::ROWS;
    const int64_t groups = ((p.out_entries >> K) + ROWS - 1) / ROWS * p.nbatch;  // one warp each
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((groups + 7) / 8, max_grid));
    late_kernel<K><<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_late(const LateParams& p, int max_grid, cudaStream_t st) {
    if (p.nops > LATE_MAX_OPS || p.k < 1 || p.k > OPEN_MAX_K) return cudaErrorInvalidValue;
    switch (p.k) {
        case 1: return launch_late_k<1>(p, max_grid, st);
        case 2: return launch_late_k<2>(p, max_grid, st);
        case 3: return launch_late_k<3>(p, max_grid, st);
        case 4: return launch_late_k<4>(p, max_grid, st);
        case 5: return launch_late_k<5>(p, max_grid, st);
        case 6: return launch_late_k<6>(p, max_grid, st);
        case 7: return launch_late_k<7>(p, max_grid, st);
        case 8: return launch_late_k<8>(p, max_grid, st);
        case 9: return launch_late_k<9>(p, max_grid, st);
        default: return launch_late_k<10>(p, max_grid, st);
    }
}

cudaError_t launch_open_finalize(const OpenFinalParams& p, int nbatch, cudaStream_t st) {
    const int NY = 1 << p.k;
    dim3 grid((unsigned)((NY + 255) / 256), (unsigned)nbatch);
    open_finalize_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace tb
