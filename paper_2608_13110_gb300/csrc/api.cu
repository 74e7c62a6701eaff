// C-ABI of the temporal-boundary sweep (declared in include/tbsweep.h).
//
// Workspace layout of one call (all offsets 256-byte aligned):
//   [tables of the plan][host staging: bits, amplitudes (tb_amplitudes only)]
//   [per batch element: rescaling slots | reduction partials | boundary]
// The boundary of one bitstring is 2^h complex64 entries; several bitstrings
// are evaluated side by side when the workspace holds several boundaries.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "misc_kernels.cuh"
#include "pass_kernel.cuh"
#include "tc_pass.cuh"
#include "open_kernels.cuh"
#include "tb_plan.h"
#include "tb_run.h"
#include "tbsweep.h"

namespace tb {
namespace rt {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

// ---- optional per-launch timing -------------------------------------------
enum { PC_PASS = 0, PC_INIT = 1, PC_REDUCE = 2, PC_FINAL = 3, PC_SMALL = 4, PC_JOIN = 5, PC_LATE = 6, PC_N = 7 };
static_assert(PC_N == TB_PROFILE_CLASSES, "profile classes");

struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    struct Rec { int cls; double bytes; size_t e0, e1; };
    std::vector<Rec> recs;
    size_t used = 0;

    cudaEvent_t take(size_t& idx) {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        idx = used;
        return pool[used++];
    }
};
Profiler g_prof;

// Bracket one launch with events when profiling is on.
struct ProfScope {
    bool active = false;
    size_t i0 = 0, i1 = 0;
    int cls;
    double bytes;
    cudaStream_t st;
    ProfScope(int c, double b, cudaStream_t s) : cls(c), bytes(b), st(s) {
        std::lock_guard<std::mutex> lk(g_prof.mu);
        if (!g_prof.on) return;
        cudaEvent_t e = g_prof.take(i0);
        if (e && cudaEventRecord(e, st) == cudaSuccess) active = true;
    }
    ~ProfScope() {
        if (!active) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        cudaEvent_t e = g_prof.take(i1);
        if (e && cudaEventRecord(e, st) == cudaSuccess) g_prof.recs.push_back({cls, bytes, i0, i1});
    }
};

bool small_path(const Plan& P) { return P.h <= SMALL_H_MAX; }

// Set by tb_selftest_bounded_wait for the evaluation it runs on this thread.
thread_local bool t_tc_selftest = false;
thread_local bool t_pass_selftest = false;
// Waits that gave up in this thread's last tb_amplitudes call.
thread_local int t_last_faults = 0;

CallLayout call_layout(const Plan& P) {
    CallLayout c;
    if (small_path(P)) return c;
    c.nslots = P.n_pass_launches() + 2;
    c.scale_bytes = align_up((int64_t)c.nslots * 8, 256);
    const int64_t nchunks = (int64_t)1 << (P.h - P.k);
    c.red_blocks = (int)std::min<int64_t>(nchunks, MAX_RED_BLOCKS);
    c.partial_bytes = P.open_k ? 0 : align_up((int64_t)c.red_blocks * 16, 256);
    c.boundary_bytes = (int64_t)8 << P.h;
    if (P.open_k) {
        const int64_t two = c.scale_bytes + 2 * c.boundary_bytes;
        const int64_t budget = P.opts.hbm_budget_bytes;
        c.open_in_place = P.h > OPEN_OUT_OF_PLACE_MAX_H || (budget > 0 && budget < two);
        c.second_bytes = c.open_in_place ? 0 : c.boundary_bytes;
        if (c.open_in_place && P.open_k >= JOIN_TC_MIN_K) {
            // tensor-core join in slices of rows (a multiple of its 128-row blocks)
            const int64_t rows = (int64_t)1 << (P.h - P.open_k);
            const int64_t slice = std::max<int64_t>(128, rows >> JOIN_SLICE_SHIFT);
            const int64_t scratch = slice << (P.open_k + 3);
            if (budget <= 0 || c.scale_bytes + c.boundary_bytes + scratch <= budget) {
                c.join_slice_rows = slice;
                c.second_bytes = scratch;
            }
        }
    }
    c.per_b = c.scale_bytes + c.partial_bytes + c.boundary_bytes + c.second_bytes;
    return c;
}

int64_t staging_bytes(const Plan& P, int64_t nb) {
    return align_up(nb * in_row(P), 256) + align_up(nb * 16 * amps_per_row(P), 256) + 256;  // + fault word
}

int64_t max_batch(const Plan& P, const CallLayout& c) {
    if (c.per_b == 0) return INT64_MAX;
    int64_t mb = std::max<int64_t>(1, DEFAULT_BATCH_ENTRIES >> P.h);
    if (P.opts.hbm_budget_bytes > 0) mb = std::min(mb, std::max<int64_t>(1, P.opts.hbm_budget_bytes / c.per_b));
    return mb;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        cached[dev] = v;
    }
    return cached[dev];
}

// ---- tensor maps of the boundary passes -------------------------------------
// The pass kernel moves whole tiles with tensor copies. Its map views nbatch
// consecutive boundaries of 2^h complex64 entries as FP32 elements in five
// dimensions whose box is one tile (see the slot layout in pass_kernel.cuh):
//   window at bit 0: [address bits 0..3 (32 floats)][bits 5..12][bit 4]
//                    [tile index with batch][1];
//   other windows, C = 13 - M >= 4 low bits, window at bits lo..lo+M-1:
//     C = 4: [bits 0..3][window bits 0..7][window bit 8][bits 4..lo-1][rest];
//     C > 4: [bits 0..3][bits 4..C-1][window][bits C..lo-1][rest],
//   rest = the bits above the window and the batch element.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

bool is_bottom_pass(int type) { return type == P_BOT || type == P_BOT_START || type == P_BOT_END; }

int encode_pass_map(CUtensorMap* m, const PassDesc& d, const float2* B, int h, int64_t nbatch) {
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return fail(TB_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dim[5];
    cuuint64_t stride[4];  // bytes, dimensions 1..4
    cuuint32_t box[5];
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const cuuint64_t E = 8;  // bytes per entry
    if (is_bottom_pass(d.type)) {
        const cuuint64_t tiles = (cuuint64_t)nbatch << (h - TILE_BITS);
        dim[0] = 32; dim[1] = 256; dim[2] = 2; dim[3] = tiles; dim[4] = 1;
        stride[0] = 32 * E; stride[1] = 16 * E; stride[2] = (cuuint64_t)TILE * E; stride[3] = (cuuint64_t)TILE * E;
        box[0] = 32; box[1] = 256; box[2] = 2; box[3] = 1; box[4] = 1;
    } else {
        const int M = d.M, lo = d.lo, C = TILE_BITS - M;
        if (C < 3 || lo < C || lo + M > h) return fail(TB_EINVAL, "pass window outside the tensor-copy layout");
        const cuuint64_t rest = (cuuint64_t)nbatch << (h - lo - M);
        dim[0] = 32;
        stride[2] = (E << C);  // bits C..lo-1
        stride[3] = (E << (lo + M));
        dim[3] = (cuuint64_t)1 << (lo - C);
        dim[4] = rest;
        box[0] = 32; box[3] = 1; box[4] = 1;
        if (C <= 4) {  // 2^C entries per row (64 or 128 bytes), the window as 256 x 2^(M-8)
            dim[0] = (cuuint64_t)2 << C; box[0] = (cuuint32_t)2 << C;
            dim[1] = 256; dim[2] = (cuuint64_t)1 << (M - 8);
            stride[0] = E << lo; stride[1] = E << (lo + 8);
            box[1] = 256; box[2] = (cuuint32_t)1 << (M - 8);
        } else {
            dim[1] = (cuuint64_t)1 << (C - 4); dim[2] = (cuuint64_t)1 << M;
            stride[0] = 16 * E; stride[1] = E << lo;
            box[1] = (cuuint32_t)1 << (C - 4); box[2] = (cuuint32_t)1 << M;
        }
    }
    // rows of 64 bytes (a 10-bit window above bit 0) take the 64-byte swizzle
    const bool row64 = !is_bottom_pass(d.type) && TILE_BITS - d.M == 3;
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float2*>(B), dim, stride, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, row64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(TB_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ") for a pass of type " +
                                  std::to_string(d.type) + ", M=" + std::to_string(d.M) + ", lo=" + std::to_string(d.lo));
    return TB_OK;
}

// 2-D tensor map over the rows of the join's input ([rows] x [2^(k+1) floats],
// rows of consecutive batch elements back to back), box JOIN_KC floats x 128
// rows, 128-byte swizzle (the tensor-core join's A tiles).
int encode_join_map(CUtensorMap* m, const float2* base, int k, int64_t rows) {
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return fail(TB_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dim[2] = {(cuuint64_t)(2 << k), (cuuint64_t)rows};
    const cuuint64_t stride[1] = {(cuuint64_t)(2 << k) * 4};
    const cuuint32_t box[2] = {(cuuint32_t)JOIN_KC, 128}, estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(base), dim, stride, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(TB_ECUDA, "cuTensorMapEncodeTiled failed for the join (" + std::to_string((int)r) + ")");
    return TB_OK;
}

cudaError_t launch_pass(const PassDesc& d, const PassParams& p, const CUtensorMap& m, int grid, cudaStream_t st) {
    switch (d.type) {
        case P_FWD: return launch_pass_t0(d.M, p, m, grid, st);
        case P_REV: return launch_pass_t1(d.M, p, m, grid, st);
        case P_TOP: return launch_pass_t2(d.M, p, m, grid, st);
        case P_BOT: return launch_pass_t3(d.M, p, m, grid, st);
        case P_BOT_START: return launch_pass_t4(d.M, p, m, grid, st);
        case P_BOT_END: return launch_pass_t5(d.M, p, m, grid, st);
        case P_TOP_END: return launch_pass_t6(d.M, p, m, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

template <class T>
const T* tab(const void* ws, int64_t off) {
    return reinterpret_cast<const T*>(static_cast<const uint8_t*>(ws) + off);
}

// Enqueue the sweep for nb bitstrings already on the device.
int run_device(const Plan& P, const uint8_t* d_bits, int64_t nb, void* d_ws, int64_t ws_bytes,
               int64_t region_off, double* d_out, cudaStream_t st, int* fault) {
    const TableLayout& L = P.lay;
    if (!fault && !small_path(P)) {
        fault = device_fault_word();
        if (!fault) return fail(TB_ECUDA, "device fault word not found");
    }
    if (small_path(P)) {
        SmallParams sp;
        sp.n = P.n;
        sp.h = P.h;
        sp.bits = d_bits;
        sp.steps = tab<StepG>(d_ws, L.steps);
        sp.tgt = tab<int8_t>(d_ws, L.step_tgt);
        sp.ctl = tab<int8_t>(d_ws, L.step_ctl);
        sp.xq = tab<int16_t>(d_ws, L.step_xq);
        sp.row_end = tab<int32_t>(d_ws, L.row_end);
        sp.nrows = (int)P.row_end.size();
        sp.init_low = tab<float2>(d_ws, L.init_low);
        sp.init_top = tab<float2>(d_ws, L.init_top);
        sp.red_low = tab<float2>(d_ws, L.red_low);
        const int64_t chunk = 1 << 30;
        for (int64_t b0 = 0; b0 < nb; b0 += chunk) {
            sp.nb = (int)std::min(chunk, nb - b0);
            sp.bits = d_bits + b0 * P.n;
            sp.out = d_out + 2 * b0;
            ProfScope ps(PC_SMALL, 0.0, st);
            TB_CUDA(launch_small(sp, st));
        }
        return TB_OK;
    }
    const CallLayout c = call_layout(P);
    const int64_t avail = ws_bytes - region_off;
    int64_t batch = std::min<int64_t>(nb, avail / c.per_b);
    batch = std::min(batch, max_batch(P, c));
    if (batch < 1)
        return fail(TB_ENOMEM, "workspace too small: need at least " +
                                   std::to_string(region_off + c.per_b) + " bytes");
    uint8_t* region = static_cast<uint8_t*>(d_ws) + region_off;
    uint8_t* scales = region;
    double2* partials = reinterpret_cast<double2*>(region + batch * c.scale_bytes);
    float2* boundary = reinterpret_cast<float2*>(region + batch * (c.scale_bytes + c.partial_bytes));
    uint32_t* maxs = reinterpret_cast<uint32_t*>(scales);
    int32_t* exps = reinterpret_cast<int32_t*>(scales) + c.nslots;
    const int64_t sstride = c.scale_bytes / 4;
    const int64_t b_stride = (int64_t)1 << P.h;
    const int nsm = num_sms();
    const StepG* steps = tab<StepG>(d_ws, L.steps);
    const StepG* pass_steps = tab<StepG>(d_ws, L.pass_steps);
    const int xstride = (int)in_row(P);  // bytes between the input rows of two batch elements

    for (int64_t b0 = 0; b0 < nb; b0 += batch) {
        const int nbat = (int)std::min<int64_t>(batch, nb - b0);
        const uint8_t* bits = d_bits + b0 * xstride;
        TB_CUDA(cudaMemsetAsync(scales, 0, (size_t)(nbat * c.scale_bytes), st));

        InitParams ip;
        ip.B = boundary;
        ip.b_stride = b_stride;
        ip.h = P.h; ip.k = P.k; ip.m = P.m; ip.top = P.top; ip.n = xstride;
        ip.chunk_shift = P.h - P.k;
        ip.nchunks = (int64_t)nbat << ip.chunk_shift;
        ip.bits = bits;
        ip.low = tab<float2>(d_ws, L.init_low);
        ip.mid = tab<float2>(d_ws, L.init_mid);
        ip.topt = tab<float2>(d_ws, L.init_top);
        ip.maxs = maxs;
        ip.sstride = sstride;
        {
            ProfScope ps(PC_INIT, 8.0 * (double)nbat * (double)b_stride, st);
            TB_CUDA(launch_init(ip, (int)std::min<int64_t>(ip.nchunks, 8LL * nsm), st));
        }

        if (P.opts.precision != TB_PRECISION_FP32) {
            if (tc_passes_disabled())
                return fail(TB_ECUDA, "tensor-core passes are disabled in this process: a pass could not confirm "
                                      "that its MMAs completed and kept its tensor memory");
            const uint8_t* mats = static_cast<const uint8_t*>(d_ws) + L.tc_mats;
            for (size_t k = 0; k < P.tc_passes.size(); ++k) {
                const TcPass& d = P.tc_passes[k];
                TcParams tp;
                tp.B = boundary;
                tp.b_stride = b_stride;
                tp.h = P.h; tp.lo = d.lo; tp.n = xstride;
                tp.tile_shift = P.h - P.tc_wb - TC_VEC_BITS;
                tp.ntiles = (int64_t)nbat << tp.tile_shift;
                tp.mat = mats + d.mat;
                tp.steps = steps;
                tp.pre = d.pre;
                tp.post = d.post;
                tp.bits = bits;
                tp.maxs = maxs;
                tp.exps = exps;
                tp.sstride = sstride;
                tp.slot = (int)k;
                tp.fault = fault;
                tp.selftest = t_tc_selftest ? 1 : 0;
                const int grid = (int)std::min<int64_t>(tp.ntiles, (int64_t)TC_CTAS_PER_SM * nsm);
                ProfScope ps(PC_PASS, 16.0 * (double)nbat * (double)b_stride, st);
                TB_CUDA(launch_tc_pass(P.opts.precision, tp, grid, st));
            }
        }
        for (size_t k = 0; k < P.passes.size(); ++k) {
            const PassDesc& d = P.passes[k];
            PassParams pp;
            pp.h = P.h; pp.lo = d.lo; pp.n = xstride;
            pp.tile_shift = P.h - TILE_BITS;
            pp.ntiles = (int64_t)nbat << pp.tile_shift;
            pp.steps = pass_steps + d.pstep0;
            pp.xs_step0 = d.xs_step[0]; pp.xs_q0 = d.xs_q[0];
            pp.xs_step1 = d.xs_step[1]; pp.xs_q1 = d.xs_q[1];
            pp.bits = bits;
            pp.maxs = maxs;
            pp.exps = exps;
            pp.sstride = sstride;
            pp.slot = (int)k;
            pp.fault = fault;
            pp.selftest = t_pass_selftest ? 1 : 0;
            CUtensorMap tmap;
            const int rc = encode_pass_map(&tmap, d, boundary, P.h, nbat);
            if (rc != TB_OK) return rc;
            const int grid = (int)std::min<int64_t>(pp.ntiles, (int64_t)PASS_CTAS_PER_SM * nsm);  // persistent CTAs
            ProfScope ps(PC_PASS, 16.0 * (double)nbat * (double)b_stride, st);
            TB_CUDA(launch_pass(d, pp, tmap, grid, st));
        }

        if (P.open_k) {  // Algorithm 2: join, late crossings, FP64 output
            const int k = P.open_k;
            // out of place: one second 2^h buffer per element after the boundaries;
            // in place: the join's result replaces the boundary and late
            // crossing i writes output row r' over its input row 2r' (rows at
            // stride 2^(i+1)); a tensor-core join then goes through a scratch of
            // join_slice_rows rows after the boundaries, one slice at a time
            float2* second = c.open_in_place ? boundary : boundary + (int64_t)batch * b_stride;
            float2* cur = boundary;
            if (c.open_in_place && c.join_slice_rows > 0) {
                float2* scratch = boundary + (int64_t)batch * b_stride;
                const int64_t rows = b_stride >> k;
                for (int bb = 0; bb < nbat; ++bb)
                    for (int64_t r0 = 0; r0 < rows; r0 += c.join_slice_rows) {
                        float2* slice = boundary + (int64_t)bb * b_stride + (r0 << k);
                        JoinTcParams jp;
                        jp.in = reinterpret_cast<const float*>(slice);
                        jp.in_stride = 0;
                        jp.out = reinterpret_cast<float*>(scratch);
                        jp.out_stride = 0;
                        jp.Es = tab<uint8_t>(d_ws, L.open_Es);
                        jp.KR = 2 << k;
                        jp.rows = c.join_slice_rows;
                        jp.nbatch = 1;
                        jp.fault = fault;
                        const int64_t items = (jp.rows / 128) * (jp.KR / join_nt(k));
                        CUtensorMap amap;
                        const int rc = encode_join_map(&amap, slice, k, jp.rows);
                        if (rc != TB_OK) return rc;
                        {
                            ProfScope ps(PC_JOIN, 16.0 * (double)(jp.rows << k), st);
                            TB_CUDA(launch_join_tc(k, jp, amap, (int)std::min<int64_t>(items, nsm), st));
                        }
                        ProfScope ps(PC_JOIN, 16.0 * (double)(jp.rows << k), st);
                        TB_CUDA(cudaMemcpyAsync(slice, scratch, (size_t)(jp.rows << k) * sizeof(float2),
                                                cudaMemcpyDeviceToDevice, st));
                    }
            } else if (k >= JOIN_TC_MIN_K && !c.open_in_place) {  // tensor cores, out of place into the second buffer
                JoinTcParams jp;
                jp.in = reinterpret_cast<const float*>(boundary);
                jp.in_stride = b_stride;
                jp.out = reinterpret_cast<float*>(second);
                jp.out_stride = b_stride;
                jp.Es = tab<uint8_t>(d_ws, L.open_Es);
                jp.KR = 2 << k;
                jp.rows = b_stride >> k;
                jp.nbatch = nbat;
                jp.fault = fault;
                const int64_t items = (int64_t)nbat * (jp.rows / 128) * (jp.KR / join_nt(k));
                CUtensorMap amap;
                const int rc = encode_join_map(&amap, boundary, k, jp.rows * nbat);
                if (rc != TB_OK) return rc;
                ProfScope ps(PC_JOIN, 16.0 * (double)nbat * (double)b_stride, st);
                TB_CUDA(launch_join_tc(k, jp, amap, (int)std::min<int64_t>(items, nsm), st));
                cur = second;
            } else {  // FP32, in place
                JoinParams jp;
                jp.B = boundary;
                jp.b_stride = b_stride;
                jp.tiles_per_b = b_stride / JOIN_TILE;
                jp.ntiles = (int64_t)nbat * jp.tiles_per_b;
                jp.E = tab<float2>(d_ws, L.open_E);
                ProfScope ps(PC_JOIN, 16.0 * (double)nbat * (double)b_stride, st);
                TB_CUDA(launch_join(k, jp, (int)std::min<int64_t>(jp.ntiles, 2LL * nsm), st));
            }
            const OpenOp* ops = tab<OpenOp>(d_ws, L.open_ops);
            for (int i = 0; i + 1 < (int)P.open_seg.size(); ++i) {
                float2* nxt = c.open_in_place ? boundary : (cur == boundary ? second : boundary);
                LateParams lp;
                lp.in = cur;
                lp.in_stride = b_stride;
                lp.out = nxt;
                lp.out_stride = b_stride;
                lp.in_shift = c.open_in_place ? i : 0;
                lp.out_shift = c.open_in_place ? i + 1 : 0;
                lp.out_entries = (int64_t)1 << (P.h - 1 - i);
                lp.nbatch = nbat;
                lp.k = k;
                lp.ops = ops + P.open_seg[i];
                lp.nops = P.open_seg[i + 1] - P.open_seg[i];
                lp.w = P.open_w[i];
                ProfScope ps(PC_LATE, 24.0 * (double)nbat * (double)lp.out_entries, st);
                TB_CUDA(launch_late(lp, 16 * nsm, st));
                cur = nxt;
            }
            OpenFinalParams op;
            op.Z = cur;
            op.b_stride = b_stride;
            op.exps = exps;
            op.sstride = sstride;
            op.nslots = c.nslots;
            op.k = k;
            op.out = d_out + 2 * b0 * amps_per_row(P);
            ProfScope ps(PC_FINAL, 0.0, st);
            TB_CUDA(launch_open_finalize(op, nbat, st));
            continue;
        }

        ReduceParams rp;
        rp.B = boundary;
        rp.b_stride = b_stride;
        rp.h = P.h; rp.k = P.k; rp.m = P.m; rp.top = P.top; rp.n = P.n;
        rp.chunk_shift = P.h - P.k;
        rp.blocks_per_b = c.red_blocks;
        rp.nbatch = nbat;
        rp.bits = bits;
        rp.low = tab<float2>(d_ws, L.red_low);
        rp.mid = tab<float2>(d_ws, L.red_mid);
        rp.topt = tab<float2>(d_ws, L.red_top);
        rp.maxs = maxs;
        rp.exps = exps;
        rp.sstride = sstride;
        rp.slot = P.n_pass_launches();
        rp.partials = partials;
        {
            ProfScope ps(PC_REDUCE, 8.0 * (double)nbat * (double)b_stride, st);
            TB_CUDA(launch_reduce(rp, st));
        }

        FinalizeParams fp;
        fp.partials = partials;
        fp.blocks_per_b = c.red_blocks;
        fp.exps = exps;
        fp.sstride = sstride;
        fp.nslots = c.nslots;
        fp.nbatch = nbat;
        fp.out = d_out + 2 * b0;
        {
            ProfScope ps(PC_FINAL, 0.0, st);
            TB_CUDA(launch_finalize(fp, st));
        }
    }
    return TB_OK;
}

}  // namespace rt
}  // namespace tb

using namespace tb;
using namespace tb::rt;

// ---- evaluation without device allocation ----------------------------------
// Some callers cannot call cudaMalloc when they need amplitudes: a process
// whose device memory is capped by a quota someone else owns, or a plugin
// inside a host application that tracks every device allocation. For them the
// library carries one fixed scratch area in device memory, a file-scope array
// that every GPU loading the library holds until exit.
namespace {
constexpr int64_t NOALLOC_SCRATCH_BYTES = (int64_t)64 << 20;  // 64 MiB per device
static __device__ __align__(256) uint8_t g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};  // device address of the array, per device
}  // namespace

extern "C" {

int tb_plan_create(int n, int d, const uint8_t* cliff, const uint8_t* tmask, const tb_gate1q* extra,
                   int n_extra, const tb_opts* opts, tb_plan** out) {
    return tb_plan_create_cphase(n, d, cliff, tmask, extra, n_extra, nullptr, opts, 0, out);
}

int tb_plan_create_open(int n, int d, const uint8_t* cliff, const uint8_t* tmask, const tb_gate1q* extra,
                        int n_extra, const tb_opts* opts, int k, tb_plan** out) {
    if (k < 1) return fail(TB_EDOMAIN, "open bits k must satisfy 1 <= k <= min(floor(d/4), 10, n-1)");
    return tb_plan_create_cphase(n, d, cliff, tmask, extra, n_extra, nullptr, opts, k, out);
}

int tb_plan_create_cphase(int n, int d, const uint8_t* cliff, const uint8_t* tmask, const tb_gate1q* extra,
                          int n_extra, const double* cphase, const tb_opts* opts, int open_k, tb_plan** out) {
    if (!out) return fail(TB_EINVAL, "out is NULL");
    *out = nullptr;
    if (open_k != 0) {
        const int h = (d + 1) / 2;
        if (open_k < 1 || open_k > d / 4 || open_k > OPEN_MAX_K || open_k > n - 1)
            return fail(TB_EDOMAIN, "open bits k must satisfy 1 <= k <= min(floor(d/4), 10, n-1)");
        if (h <= SMALL_H_MAX) return fail(TB_EDOMAIN, "open plans need ceil(d/2) >= 13");
    }
    try {
        tb_plan* p = new tb_plan;
        p->p.open_k = open_k;
        std::string err;
        const int rc = plan_build(p->p, n, d, cliff, tmask, extra, n_extra, cphase, opts, err);
        if (rc != TB_OK) {
            delete p;
            return fail(rc, err);
        }
        p->p.uid = next_plan_uid();
        *out = p;
        return TB_OK;
    } catch (const std::bad_alloc&) {
        return fail(TB_ENOMEM, "host allocation failed");
    } catch (...) {
        return fail(TB_EINVAL, "plan construction failed");
    }
}

int tb_batched_sample(const double* amps, int k, int64_t na, const double* u, int32_t* b, double* q) {
    if (!amps || !u || !b || k < 0 || k > 30 || na < 0) return fail(TB_EINVAL, "NULL or out-of-range argument");
    const int64_t B = (int64_t)1 << k;
    for (int64_t a = 0; a < na; ++a) {
        const double* z = amps + 2 * a * B;
        double Q = 0.0;
        for (int64_t y = 0; y < B; ++y) Q += z[2 * y] * z[2 * y] + z[2 * y + 1] * z[2 * y + 1];
        if (q) q[a] = Q;
        if (!(u[a] >= 0.0 && u[a] < 1.0)) return fail(TB_EINVAL, "uniform variates must lie in [0, 1)");
        // inverse of the conditional distribution function p(b | a) = p(a, b) / Q_a
        const double target = u[a] * Q;
        double acc = 0.0;
        int64_t pick = B - 1;
        for (int64_t y = 0; y < B; ++y) {
            acc += z[2 * y] * z[2 * y] + z[2 * y + 1] * z[2 * y + 1];
            if (acc > target) { pick = y; break; }
        }
        b[a] = (int32_t)pick;
    }
    return TB_OK;
}

int tb_plan_info(const tb_plan* plan, tb_plan_info_t* info) {
    if (!plan || !info) return fail(TB_EINVAL, "NULL argument");
    const Plan& P = plan->p;
    std::memset(info, 0, sizeof(*info));
    info->n = P.n;
    info->d = P.d;
    info->width = P.width;
    info->boundary_bits = P.h;
    info->log2_cost = P.log2cost;
    info->boundary_bytes = (int64_t)8 << P.h;
    info->n_steps = (int)P.steps.size();
    info->n_passes = P.n_pass_launches();
    for (const PassDesc& d : P.passes) info->pass_madds += 8 * d.nsteps + (pass_blk(d.type, d.M) >= 0 ? 8 : 0);
    info->table_bytes = P.lay.total;
    info->open_k = P.open_k;
    info->open_width = P.open_k ? std::max(P.h, 2 * P.open_k) : 0;
    return TB_OK;
}

int tb_plan_schedule(const tb_plan* plan, int32_t* sched, int cap) {
    if (!plan) return -1;
    const Plan& P = plan->p;
    if (P.opts.precision != TB_PRECISION_FP32) {
        const int np = (int)P.tc_passes.size();
        for (int i = 0; i < np && i < cap && sched; ++i) {
            sched[3 * i] = P_TENSOR;
            sched[3 * i + 1] = P.tc_wb;
            sched[3 * i + 2] = P.tc_passes[i].lo;
        }
        return np;
    }
    const int np = (int)P.passes.size();
    for (int i = 0; i < np && i < cap && sched; ++i) {
        sched[3 * i] = P.passes[i].type;
        sched[3 * i + 1] = P.passes[i].M;
        sched[3 * i + 2] = P.passes[i].lo;
    }
    return np;
}

int64_t tb_workspace_bytes(const tb_plan* plan, int64_t nb) {
    if (!plan || nb < 0) return -1;
    const Plan& P = plan->p;
    if (P.h > MAX_H) return -1;
    const CallLayout c = call_layout(P);
    const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(nb, max_batch(P, c)));
    return P.lay.total + staging_bytes(P, nb) + (c.per_b ? batch * c.per_b : 0);
}

int64_t tb_workspace_min_bytes(const tb_plan* plan) {
    if (!plan) return -1;
    const Plan& P = plan->p;
    if (P.h > MAX_H) return -1;
    return P.lay.total + call_layout(P).per_b;
}

int tb_plan_upload(const tb_plan* plan, void* d_ws, int64_t ws_bytes, void* stream) {
    if (!plan || !d_ws) return fail(TB_EINVAL, "NULL argument");
    const Plan& P = plan->p;
    if (P.h > MAX_H) return fail(TB_EDOMAIN, "boundary wider than 2^35 entries");
    if (ws_bytes < P.lay.total) return fail(TB_ENOMEM, "workspace smaller than the plan's tables");
    TB_CUDA(cudaMemcpyAsync(d_ws, P.blob.data(), (size_t)P.lay.total, cudaMemcpyHostToDevice,
                            static_cast<cudaStream_t>(stream)));
    return TB_OK;
}

int tb_amplitudes_device(const tb_plan* plan, const uint8_t* d_bits, int64_t nb, void* d_ws,
                         int64_t ws_bytes, double* d_out, void* stream) {
    if (!plan || !d_ws || (nb > 0 && (!d_bits || !d_out)) || nb < 0)
        return fail(TB_EINVAL, "NULL or negative argument");
    const Plan& P = plan->p;
    if (P.h > MAX_H) return fail(TB_EDOMAIN, "boundary wider than 2^35 entries");
    if (nb == 0) return TB_OK;
    if (ws_bytes < P.lay.total) return fail(TB_ENOMEM, "workspace smaller than the plan's tables");
    return run_device(P, d_bits, nb, d_ws, ws_bytes, P.lay.total, d_out, static_cast<cudaStream_t>(stream));
}

int tb_amplitudes(const tb_plan* plan, const uint8_t* bits, int64_t nb, void* d_ws, int64_t ws_bytes,
                  double* out, void* stream) {
    if (!plan || !d_ws || nb < 0 || (nb > 0 && (!bits || !out)))
        return fail(TB_EINVAL, "NULL or negative argument");
    const Plan& P = plan->p;
    if (P.h > MAX_H) return fail(TB_EDOMAIN, "boundary wider than 2^35 entries");
    if (nb == 0) return TB_OK;
    for (int64_t i = 0; i < nb * in_row(P); ++i)
        if (bits[i] > 1) return fail(TB_EINVAL, "bitstring entries must be 0 or 1");
    const int64_t stage = staging_bytes(P, nb);
    if (ws_bytes < P.lay.total + stage) return fail(TB_ENOMEM, "workspace too small for the staged inputs");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    uint8_t* d_bits = ws + P.lay.total;
    double* d_out = reinterpret_cast<double*>(ws + P.lay.total + align_up(nb * in_row(P), 256));
    int* d_fault = reinterpret_cast<int*>(ws + P.lay.total + stage - 256);
    TB_CUDA(cudaMemcpyAsync(d_ws, P.blob.data(), (size_t)P.lay.total, cudaMemcpyHostToDevice, st));
    TB_CUDA(cudaMemcpyAsync(d_bits, bits, (size_t)(nb * in_row(P)), cudaMemcpyHostToDevice, st));
    TB_CUDA(cudaMemsetAsync(d_fault, 0, sizeof(int), st));
    const int rc = run_device(P, d_bits, nb, d_ws, ws_bytes, P.lay.total + stage, d_out, st, d_fault);
    if (rc != TB_OK) return rc;
    TB_CUDA(cudaMemcpyAsync(out, d_out, (size_t)(16 * nb * amps_per_row(P)), cudaMemcpyDeviceToHost, st));
    int faults = 0;
    TB_CUDA(cudaMemcpyAsync(&faults, d_fault, sizeof(int), cudaMemcpyDeviceToHost, st));
    TB_CUDA(cudaStreamSynchronize(st));
    faults = note_faults(faults);
    t_last_faults = faults;
    if (faults != 0)
        return fail(TB_ETIMEOUT, "a bounded device wait gave up in " + std::to_string(faults) +
                                     " CTA(s); the amplitudes are not valid");
    return TB_OK;
}

int tb_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = true;
    g_prof.recs.clear();
    g_prof.used = 0;
    return TB_OK;
}

int tb_profile_end(tb_profile_t* out) {
    if (!out) return fail(TB_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = false;
    std::memset(out, 0, sizeof(*out));
    for (const auto& r : g_prof.recs) {
        TB_CUDA(cudaEventSynchronize(g_prof.pool[r.e1]));
        float ms = 0.0f;
        TB_CUDA(cudaEventElapsedTime(&ms, g_prof.pool[r.e0], g_prof.pool[r.e1]));
        out->launches[r.cls] += 1;
        out->ms[r.cls] += ms;
        out->bytes[r.cls] += r.bytes;
    }
    g_prof.recs.clear();
    g_prof.used = 0;
    return TB_OK;
}

int tb_selftest_bounded_wait(int32_t* faults) {
    if (!faults) return fail(TB_EINVAL, "faults is NULL");
    *faults = 0;
    tb_opts o;
    std::memset(&o, 0, sizeof(o));
    o.precision = TB_PRECISION_BF16X3;
    tb_plan* plan = nullptr;
    int rc = tb_plan_create(3, 26, nullptr, nullptr, nullptr, 0, &o, &plan);
    if (rc != TB_OK) return rc;
    int32_t before = 0;
    rc = tb_device_faults(&before);  // clears the word
    void* ws = nullptr;
    double* out = nullptr;
    uint8_t* bits = nullptr;
    const int64_t wsb = tb_workspace_bytes(plan, 1);
    if (rc == TB_OK && (cudaMalloc(&ws, (size_t)wsb) != cudaSuccess || cudaMalloc(&out, 16) != cudaSuccess ||
                        cudaMalloc(&bits, 3) != cudaSuccess || cudaMemset(bits, 0, 3) != cudaSuccess))
        rc = fail(TB_ECUDA, "self-test allocation failed");
    if (rc == TB_OK) rc = tb_plan_upload(plan, ws, wsb, nullptr);
    if (rc == TB_OK) {
        t_tc_selftest = true;
        rc = run_device(plan->p, bits, 1, ws, wsb, plan->p.lay.total, out, nullptr);
        t_tc_selftest = false;
    }
    if (rc == TB_OK) rc = tb_device_faults(faults);
    cudaFree(bits);
    cudaFree(out);
    cudaFree(ws);
    tb_plan_destroy(plan);
    if (rc != TB_OK) return rc;
    // the FP32 pass kernels through the synchronous entry: their producer
    // issues no tile copies, every wait gives up, and tb_amplitudes must say so
    plan = nullptr;
    rc = tb_plan_create(3, 26, nullptr, nullptr, nullptr, 0, nullptr, &plan);
    if (rc != TB_OK) return rc;
    const int64_t wsb2 = tb_workspace_bytes(plan, 1);
    void* ws2 = nullptr;
    if (cudaMalloc(&ws2, (size_t)wsb2) != cudaSuccess) rc = fail(TB_ECUDA, "self-test allocation failed");
    if (rc == TB_OK) {
        const uint8_t hbits[3] = {0, 0, 0};
        double hout[2] = {0.0, 0.0};
        t_pass_selftest = true;
        const int r2 = tb_amplitudes(plan, hbits, 1, ws2, wsb2, hout, nullptr);
        t_pass_selftest = false;
        if (r2 != TB_ETIMEOUT)
            rc = fail(TB_ECUDA, "self-test: the pass kernels' bounded waits were not reported (status " +
                                    std::to_string(r2) + ")");
        else
            *faults += t_last_faults;
    }
    cudaFree(ws2);
    tb_plan_destroy(plan);
    return rc;
}

int tb_device_faults(int32_t* count) {
    if (!count) return fail(TB_EINVAL, "count is NULL");
    int* w = device_fault_word();
    if (!w) return fail(TB_ECUDA, "device fault word not found");
    TB_CUDA(cudaDeviceSynchronize());
    int v = 0;
    TB_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    TB_CUDA(cudaMemset(w, 0, sizeof(int)));
    *count = note_faults(v);
    return TB_OK;
}

int tb_amplitudes_noalloc(const tb_plan* plan, const uint8_t* d_bits, int64_t nb, double* d_out,
                          void* stream) {
    if (!plan || nb < 0 || (nb > 0 && (!d_bits || !d_out))) return fail(TB_EINVAL, "NULL or negative argument");
    const Plan& P = plan->p;
    if (P.h > MAX_H) return fail(TB_EDOMAIN, "boundary wider than 2^35 entries");
    if (P.open_k) return fail(TB_EINVAL, "open plans are evaluated by tb_amplitudes / tb_amplitudes_device");
    const int64_t need = P.lay.total + call_layout(P).per_b;
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(TB_ENOMEM, "this circuit needs " + std::to_string(need) +
                                   " bytes of scratch; the fixed scratch holds " +
                                   std::to_string(NOALLOC_SCRATCH_BYTES));
    if (nb == 0) return TB_OK;
    int dev = 0;
    TB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TB_EINVAL, "device index out of range");
    void* base = nullptr;
    {
        // set-up, once per device, with that device current: the host-side
        // name of the array is not a device address, so ask for the address
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* a = nullptr;
            TB_CUDA(cudaGetSymbolAddress(&a, g_noalloc_scratch));
            g_noalloc_addr[dev] = a;
        }
        base = g_noalloc_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TB_CUDA(cudaMemcpyAsync(base, P.blob.data(), (size_t)P.lay.total, cudaMemcpyHostToDevice, st));
    // run_device clears the rescaling slots of every batch before use; the
    // boundary and the partial sums are fully written before they are read
    return run_device(P, d_bits, nb, base, NOALLOC_SCRATCH_BYTES, P.lay.total, d_out, st);
}

int tb_log_xeb(const double* amp, int64_t nb, int n, double* out) {
    if (!amp || !out || nb <= 0 || n < 1) return fail(TB_EINVAL, "bad argument");
    const double gamma = 0.57721566490153286060651209;
    double s = 0.0;
    for (int64_t i = 0; i < nb; ++i) s += std::log(amp[2 * i] * amp[2 * i] + amp[2 * i + 1] * amp[2 * i + 1]);
    *out = gamma + n * std::log(2.0) + s / (double)nb;
    return TB_OK;
}

int tb_log_xeb_device(const double* d_amp, int64_t nb, int n, double* d_out, void* stream) {
    if (!d_amp || !d_out || nb <= 0 || n < 1) return fail(TB_EINVAL, "bad argument");
    TB_CUDA(launch_log_xeb(reinterpret_cast<const double2*>(d_amp), nb, n, d_out,
                           static_cast<cudaStream_t>(stream)));
    return TB_OK;
}

int tb_clifford_matrix(int k, double m[8]) {
    if (k < 0 || k > 23 || !m) return fail(TB_EINVAL, "index must be 0..23");
    const M2 c = clifford(k);
    for (int i = 0; i < 4; ++i) {
        m[2 * i] = c.a[i].real();
        m[2 * i + 1] = c.a[i].imag();
    }
    return TB_OK;
}

void tb_plan_destroy(tb_plan* plan) { delete plan; }

const char* tb_status_str(int status) {
    switch (status) {
        case TB_OK: return "ok";
        case TB_EINVAL: return "invalid argument";
        case TB_EDOMAIN: return "circuit outside the supported domain";
        case TB_ENOMEM: return "insufficient memory";
        case TB_ECUDA: return "CUDA error";
        case TB_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char* tb_last_error(void) { return g_err.c_str(); }

}  // extern "C"
