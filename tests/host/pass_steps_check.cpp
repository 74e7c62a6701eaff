// Host check of the planner (no GPU): on a random boundary, applying every
// pass's steps as the pass kernels read them from the pass-step table (each
// row turn's four steps composed into one 4x4 block, the top turn's block in
// four bitstring variants) gives the same boundary as applying the method's
// paired steps one by one (Algorithm 1's sweep order, Sec. 3.1). Usage:
// pass_steps_check n d [window bottom top]; exit 0 when the relative L2
// difference is below 1e-5.
#include <cstdio>
#include <cstdlib>
#include <complex>
#include <random>
#include <vector>
#include "tb_plan.h"
using namespace tb;
using cd = std::complex<double>;
static cd C(float2 z) { return cd(z.x, z.y); }
static void step2(std::vector<cd>& B, int t, int c, const float2* g) {  // g[c*4 + a'*2 + s]
    const size_t N = B.size();
    for (size_t i = 0; i < N; ++i) {
        if (i >> t & 1) continue;
        const size_t j = i | ((size_t)1 << t);
        const int cv = c < 0 ? 0 : (int)((i >> c) & 1);
        const cd a = B[i], b = B[j];
        B[i] = C(g[cv * 4 + 0]) * a + C(g[cv * 4 + 1]) * b;
        B[j] = C(g[cv * 4 + 2]) * a + C(g[cv * 4 + 3]) * b;
    }
}
int main(int argc, char** argv) {
    const int n = argc > 1 ? atoi(argv[1]) : 8, d = argc > 2 ? atoi(argv[2]) : 30;
    const int wb = argc > 3 ? atoi(argv[3]) : 0, bb = argc > 4 ? atoi(argv[4]) : 0, tbits = argc > 5 ? atoi(argv[5]) : 0;
    std::mt19937 rng(1234 + n * 100 + d);
    std::vector<uint8_t> cliff((d + 1) * n), tm(d * n);
    for (auto& v : cliff) v = rng() % 24;
    for (auto& v : tm) v = (rng() % 10) == 0;
    tb_opts o{};
    o.window_bits = wb; o.bottom_bits = bb; o.top_bits = tbits; o.precision = TB_PRECISION_FP32;
    Plan P;
    std::string err;
    if (plan_build(P, n, d, cliff.data(), tm.data(), nullptr, 0, nullptr, &o, err) != TB_OK) { printf("plan: %s\n", err.c_str()); return 1; }
    const int h = P.h;
    std::vector<uint8_t> x(n);
    for (auto& v : x) v = rng() & 1;
    std::vector<cd> B0((size_t)1 << h);
    std::normal_distribution<double> nd;
    for (auto& v : B0) v = cd(nd(rng), nd(rng));
    std::vector<cd> A = B0, Bp = B0;
    for (size_t s = 0; s < P.steps.size(); ++s) {
        const int xv = P.step_xq[s] >= 0 ? x[P.step_xq[s]] : 0;
        step2(A, P.step_tgt[s], P.step_ctl[s], P.steps[s].g[xv]);
    }
    int nblk = 0;
    for (const PassDesc& dd : P.passes) {
        uint32_t xmask = 0;
        for (int j = 0; j < 2; ++j) if (dd.xs_step[j] >= 0) xmask |= (uint32_t)x[dd.xs_q[j]] << dd.xs_step[j];
        for (int i = 0; i < dd.nsteps; ++i) {
            const StepSpec sp = step_spec(dd.type, dd.M, i);
            const StepG* e = &P.pass_steps[dd.pstep0 + pass_entry(dd.type, dd.M, i)];
            if (i == pass_blk(dd.type, dd.M)) {
                ++nblk;
                const float2* raw = &e->g[0][0];
                const int v = (int)((xmask >> i) & 1) + 2 * (int)((xmask >> XM_HIGH_BIT) & 1);
                const int t0 = dd.lo + sp.t, cb = dd.lo + sp.c;
                for (size_t idx = 0; idx < Bp.size(); ++idx) {
                    if ((idx >> t0) & 3) continue;
                    const int cv = (int)((idx >> cb) & 1);
                    cd in[4], out[4];
                    for (int q = 0; q < 4; ++q) in[q] = Bp[idx | ((size_t)q << t0)];
                    for (int r = 0; r < 4; ++r) {
                        out[r] = 0;
                        for (int q = 0; q < 4; ++q) out[r] += C(raw[((v * 2 + cv) * 4 + r) * 4 + q]) * in[q];
                    }
                    for (int q = 0; q < 4; ++q) Bp[idx | ((size_t)q << t0)] = out[q];
                }
            } else {
                const int xv = (int)((xmask >> i) & 1);
                step2(Bp, dd.lo + sp.t, sp.c < 0 ? -1 : dd.lo + sp.c, e->g[xv]);
            }
        }
    }
    double num = 0, den = 0;
    for (size_t i = 0; i < A.size(); ++i) { num += std::norm(A[i] - Bp[i]); den += std::norm(A[i]); }
    printf("n=%d d=%d h=%d passes=%zu blocks=%d relL2=%.3e\n", n, d, h, P.passes.size(), nblk, std::sqrt(num / den));
    return std::sqrt(num / den) < 1e-5 ? 0 : 2;
}
