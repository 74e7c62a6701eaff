// Dense tensor-core schedule of the temporal-boundary sweep (precision
// TF32X3 / BF16X3).
//
// The paired steps of one absorbed row form a staircase of controlled 2x2
// gates on consecutive address bits (Algorithm 1, paired contraction). A run
// of steps whose targets and controls stay inside WB consecutive address bits
// composes into one 2^WB x 2^WB complex matrix (in the paper's production
// code, Sec. 5.2, small tensors are likewise combined ahead of the boundary
// contraction; here the combined tensor is a dense block applied by tensor
// cores). This file cuts
// every row into such runs, composes each run in FP64, embeds it as a real
// 2^(WB+1) x 2^(WB+1) matrix, splits it into a high and a low part in the
// tensor-core operand format, and lays both out as the K-major shared-memory
// operand of the MMA.
//
// Cutting rule, WB bits per window:
//   forward row (targets 0..h-1, control p-1): targets 0..WB-1 in the window
//   at bit 0 (shared with the previous reversed row's last targets), then
//   chunks of WB targets [a, a+WB-1] (window = the chunk; the first step's
//   control a-1 lies below the window and runs as a register pre-step), the
//   last chunk ending at h-1 (window [h-WB, h-1]; its last step depends on the
//   row's output bit and runs as a register post-step);
//   reversed row (targets h-1..0, control p+1): the window [h-WB, h-1] first
//   (its first step depends on the output bit: pre-step), then chunks of WB
//   targets going down, the last one ending at bit 0 in the window [0, WB-1].

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "tb_plan.h"

namespace tb {

using cd = std::complex<double>;

// Round to the nearest TF32 value (10 explicit mantissa bits, ties to even).
float round_tf32(double v) {
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return f;
    u = (u + 0xfffu + ((u >> 13) & 1u)) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Byte offset of element (row nn, column kk) of an N x K operand stored
// K-major in the tensor cores' canonical layout without swizzling: 8 rows x
// 16 bytes form one 128-byte core matrix; core matrices are consecutive along
// K (leading byte offset 128) and then along N (stride byte offset
// (K / T) * 128), T = 16 / element bytes.
int64_t canon_offset(int nn, int kk, int K, int eb) {
    const int T = 16 / eb;
    return ((int64_t)(nn / 8) * (K / T) + kk / T) * 128 + (nn % 8) * 16 + (kk % T) * eb;
}


namespace {

struct Chunk {
    int lo = 0;
    std::vector<int> steps;  // plan step indices in execution order
};

// Round to the nearest bfloat16 (ties to even), returned as a float value.
float round_bf16(double v) {
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return f;  // inf / nan unchanged
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Compose the steps (plan indices, in order) acting on address bits
// [base, base + WB) into one dense complex block in FP64, embed it as the real
// (2^(WB+1))^2 operand (k = 2*j + part_in, nn = 2*j' + part_out), split it into
// hi + lo parts of the operand type and store both at dst (hi, then lo) in the
// K-major canonical layout.
bool compose_block(const Plan& P, const std::vector<int>& steps, int base, int WB, bool tf32, uint8_t* dst,
                   std::string& err) {
    const int NV = 1 << WB, K = 2 * NV, eb = tf32 ? 4 : 2;
    std::vector<cd> Mt((size_t)NV * NV), v(NV), w(NV);
    for (int ji = 0; ji < NV; ++ji) {
        std::fill(v.begin(), v.end(), cd(0.0));
        v[ji] = 1.0;
        for (const int s : steps) {
            const int t = P.step_tgt[s] - base;
            const int ctl = P.step_ctl[s];
            const int cb = ctl < 0 ? -1 : ctl - base;
            if (t < 0 || t >= WB || (ctl >= 0 && (cb < 0 || cb >= WB)) || P.step_xq[s] >= 0) {
                err = "internal: dense block step leaves its window";
                return false;
            }
            const auto& g = P.steps64[s];  // variant x = 0 (the step does not depend on x)
            for (int j = 0; j < NV; ++j) {
                if ((j >> t) & 1) continue;
                const int cv = cb < 0 ? 0 : (j >> cb) & 1;
                const cd v0 = v[j], v1 = v[j | (1 << t)];
                w[j] = g[cv * 4 + 0] * v0 + g[cv * 4 + 1] * v1;
                w[j | (1 << t)] = g[cv * 4 + 2] * v0 + g[cv * 4 + 3] * v1;
            }
            v.swap(w);
        }
        for (int jo = 0; jo < NV; ++jo) Mt[(size_t)jo * NV + ji] = v[jo];
    }
    uint8_t* hi = dst;
    uint8_t* lo = dst + tc_mat_bytes(WB, eb) / 2;
    for (int nn = 0; nn < K; ++nn)
        for (int k = 0; k < K; ++k) {
            const cd z = Mt[(size_t)(nn >> 1) * NV + (k >> 1)];
            const int po = nn & 1, pi = k & 1;
            const double val = po == 0 ? (pi == 0 ? z.real() : -z.imag()) : (pi == 0 ? z.imag() : z.real());
            const int64_t off = canon_offset(nn, k, K, eb);
            if (tf32) {
                const float vh = round_tf32(val);
                const float vl = round_tf32(val - (double)vh);
                std::memcpy(hi + off, &vh, 4);
                std::memcpy(lo + off, &vl, 4);
            } else {
                const float vh = round_bf16(val);
                const float vl = round_bf16(val - (double)vh);
                uint32_t uh, ul;
                std::memcpy(&uh, &vh, 4);
                std::memcpy(&ul, &vl, 4);
                const uint16_t bh = (uint16_t)(uh >> 16), bl = (uint16_t)(ul >> 16);
                std::memcpy(hi + off, &bh, 2);
                std::memcpy(lo + off, &bl, 2);
            }
        }
    return true;
}

}  // namespace

int tc_schedule(Plan& P, std::string& err) {
    const int h = P.h, n = P.n;
    const bool tf32 = P.opts.precision == TB_PRECISION_TF32X3;
    const int WB = tf32 ? TC_WB_TF32 : TC_WB_BF16;
    const int eb = tf32 ? 4 : 2;
    if (h - WB < TC_VEC_BITS) {
        err = "dense tensor-core blocks need h >= WB + 7";
        return TB_EDOMAIN;
    }
    P.tc_wb = WB;

    // ---- cut every row into chunks; merge the turn at address bit 0
    std::vector<Chunk> chunks;
    int s0 = 0;
    for (int r = 1; r <= P.last_mid_row(); ++r) {
        const bool fwd = (r % 2) == 1;
        auto step_of_target = [&](int p) { return s0 + (fwd ? p : h - 1 - p); };
        if (fwd) {
            Chunk c0;
            c0.lo = 0;
            for (int p = 0; p < WB; ++p) c0.steps.push_back(step_of_target(p));
            if (r >= 3) {  // same window as the reversed row's last chunk
                Chunk& prev = chunks.back();
                prev.steps.insert(prev.steps.end(), c0.steps.begin(), c0.steps.end());
            } else {
                chunks.push_back(c0);
            }
            const int R = h - WB;
            const int C = (R + WB - 1) / WB;
            std::vector<int> sizes(C, WB);
            sizes[C - 1] = R - (C - 1) * WB;
            if (sizes[C - 1] == 1) { sizes[C - 2] -= 1; sizes[C - 1] = 2; }
            int a = WB;
            for (int j = 0; j < C; ++j) {
                Chunk c;
                const int b = a + sizes[j] - 1;
                if (j == C - 1) c.lo = h - WB;
                else c.lo = sizes[j] == WB ? a : b - WB + 1;
                for (int p = a; p <= b; ++p) c.steps.push_back(step_of_target(p));
                chunks.push_back(c);
                a = b + 1;
            }
        } else {
            Chunk top;
            top.lo = h - WB;
            for (int p = h - 1; p >= h - WB; --p) top.steps.push_back(step_of_target(p));
            chunks.push_back(top);
            int a = h - WB - 1;
            while (a >= 0) {
                const int b = std::max(0, a - WB + 1);
                Chunk c;
                c.lo = b;
                for (int p = a; p >= b; --p) c.steps.push_back(step_of_target(p));
                chunks.push_back(c);
                a = b - 1;
            }
        }
        s0 += h;
    }

    // ---- classify the steps of each chunk, compose the dense block
    const int64_t mat_bytes = tc_mat_bytes(WB, eb);
    P.tc_passes.clear();
    P.tc_mats.assign((size_t)(mat_bytes * (int64_t)chunks.size()), 0);
    int expect = 0;
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const Chunk& c = chunks[ci];
        TcPass tp;
        std::memset(&tp, 0, sizeof(tp));
        tp.lo = c.lo;
        tp.pre.t = tp.post.t = -1;
        tp.step0 = c.steps.front();
        tp.nsteps = (int)c.steps.size();
        tp.mat = (int64_t)ci * mat_bytes;
        for (int i = 0; i < tp.nsteps; ++i)
            if (c.steps[i] != tp.step0 + i || c.steps[i] != expect + i) {
                err = "internal: dense schedule out of step order";
                return TB_EINVAL;
            }
        expect += tp.nsteps;
        auto in_win = [&](int bit) { return bit >= c.lo && bit < c.lo + WB; };
        auto make_reg = [&](int s, TcStep& rs) {
            rs.t = P.step_tgt[s] - c.lo;
            rs.step = s;
            rs.xq = P.step_xq[s];
            const int ctl = P.step_ctl[s];
            if (ctl < 0) { rs.cmode = 0; rs.cbit = 0; }
            else if (in_win(ctl)) { rs.cmode = 2; rs.cbit = ctl - c.lo; }
            else { rs.cmode = 1; rs.cbit = ctl; }
        };
        int first = 0, last = tp.nsteps;
        {
            const int s = c.steps.front();
            const int ctl = P.step_ctl[s];
            if (P.step_xq[s] >= 0 || (ctl >= 0 && !in_win(ctl))) { make_reg(s, tp.pre); first = 1; }
        }
        if (last - first > 0) {
            const int s = c.steps.back();
            if (P.step_xq[s] >= 0) { make_reg(s, tp.post); last -= 1; }
        }
        // the kernel implements exactly these register steps: a pre-step on
        // window bit 0 or WB-1 controlled by an address bit outside the window
        // or by nothing, a post-step on bit WB-1 controlled by bit WB-2
        if (tp.pre.t >= 0 && ((tp.pre.t != 0 && tp.pre.t != WB - 1) || tp.pre.cmode == 2)) {
            err = "internal: unsupported pre-step";
            return TB_EINVAL;
        }
        if (tp.post.t >= 0 && (tp.post.t != WB - 1 || tp.post.cmode != 2 || tp.post.cbit != WB - 2)) {
            err = "internal: unsupported post-step";
            return TB_EINVAL;
        }
        const std::vector<int> blk(c.steps.begin() + first, c.steps.begin() + last);
        if (!compose_block(P, blk, c.lo, WB, tf32, P.tc_mats.data() + tp.mat, err)) return TB_EINVAL;
        P.tc_passes.push_back(tp);
    }
    if (expect != (int)P.steps.size()) {
        err = "internal: dense schedule does not cover every step";
        return TB_EINVAL;
    }
    return TB_OK;
}

}  // namespace tb
