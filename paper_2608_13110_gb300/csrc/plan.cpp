// Host planner of the temporal-boundary sweep (arXiv 2608.13110, Sec. 3.1).
//
// Builds, in FP64, everything the device needs for one circuit:
//   * the folded one-qubit gates U_(q,t) = E . T^tau . C (Sec. 2.1 / 2.2:
//     every one-qubit gate folds into a neighbouring tensor);
//   * the paired steps of every absorbed row 1..n-2 (Algorithm 1's paired
//     contraction of two row tensors with the boundary, Proposition 1 case (a))
//     as controlled 2x2 gates on the boundary's address bits;
//   * the pass schedule that groups consecutive steps into windows of address
//     bits, one HBM pass each, sharing the window at every row turn;
//   * the row-0 product tables (B <- pi[1] in Algorithm 1) and the last-row
//     tables (the final absorption that returns the scalar);
//   * W and C of Algorithm 1's path by a symbolic run of the algorithm over
//     the tensor network's legs (Sec. 2.2 cost metrics, Proposition 1).
//
// Derivation of the step (used below). Let s_(q,l) be qubit q's value during
// CZ layer l. Because CZ is diagonal, psi(x) is a sum over all s of
//   prod_q U_(q,0)[s_(q,0),0] prod_(l>=1) U_(q,l)[s_(q,l), s_(q,l-1)] U_(q,d)[x_q, s_(q,d-1)]
//   * prod over coupled pairs of (-1)^(s_(i,l) s_(i+1,l)).
// Any diagonal entangler of operator Schmidt rank 2 works the same way
// (Sec. 2.1 allows them): a controlled phase diag(1, 1, 1, w) replaces the
// factor (-1)^(s s') by w^(s s'), so every -1 below may be a per-gate w.
// Qubit q waits for its partner q+1 in the layers L_q = {l : l = q mod 2}.
// The boundary after row q is indexed by (s_(q,l)), l in L_q, stored at
// address bit floor(l/2), h = ceil(d/2) bits. For even d every row has h such
// layers; for odd d the odd rows have h - 1 and their top bit stays 0.
// Absorbing row r walks its layers in time order (forward for odd r,
// backward for even r, the snake of Algorithm 1); each step consumes the
// stored bit of one layer (CZ sign with the row's value, summed) and creates
// the row's value of the adjacent layer at the same address bit:
//   forward,  slot p: G[c][a'][s] = sum_a U_(r,2p+1)[a',a] (-1)^(s a) U_(r,2p)[a,c]
//   backward, slot p: G[c][a'][s] = sum_a U_(r,2p+2)[c,a] (-1)^(s a) U_(r,2p+1)[a,a']
// where c is the value created by the previous step (address bit p-1 forward,
// p+1 backward). The end steps replace the missing neighbour by the input
// column U_(r,0)[.,0] or the output row U_(r,d)[x_r,.].
// Odd d (Proposition 1's turn case): a forward row's last stored layer d-1
// has no later layer of its own in L_r, so its last step sums the row out,
//   G[c][0][s] = sum_a U_(r,d)[x_r,a] (-1)^(s a) U_(r,d-1)[a,c], G[c][1][s] = 0,
// and a backward row starts with nothing to consume: its first step creates
// the value of layer d-1 from the empty top bit, G[c][a'][0] = U_(r,d)[x_r,a'],
// G[c][a'][1] = 0. Both keep the form of a controlled 2x2 step, so every
// kernel runs them unchanged.

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tb_plan.h"

namespace tb {

using cd = std::complex<double>;

M2 m2_mul(const M2& A, const M2& B) {
    M2 C;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) C.a[r * 2 + c] = A.a[r * 2] * B.a[c] + A.a[r * 2 + 1] * B.a[2 + c];
    return C;
}

static M2 m2(cd a, cd b, cd c, cd d) {
    M2 m;
    m.a[0] = a; m.a[1] = b; m.a[2] = c; m.a[3] = d;
    return m;
}

// The 24 single-qubit Cliffords C_k = P_(k mod 4) . R_(k div 4).
M2 clifford(int k) {
    const double s = std::sqrt(0.5);
    const cd i(0.0, 1.0);
    const M2 I2 = m2(1, 0, 0, 1), X = m2(0, 1, 1, 0), Y = m2(0, -i, i, 0), Z = m2(1, 0, 0, -1);
    const M2 H = m2(s, s, s, -s), S = m2(1, 0, 0, i);
    const M2 P[4] = {I2, X, Y, Z};
    const M2 R[6] = {I2, H, S, m2_mul(S, H), m2_mul(H, S), m2_mul(m2_mul(H, S), H)};
    return m2_mul(P[k % 4], R[k / 4]);
}

static float2 f2(cd z) { return make_float2((float)z.real(), (float)z.imag()); }

// ---------------------------------------------------------------------------
// Window partition and pass schedule
// ---------------------------------------------------------------------------

// Windows W_0 = [0, b-1], ..., W_K = [h-t, h-1]; consecutive windows share
// one bit, so sum(M_j) - K = h.
static std::vector<int> partition(int h, int mmax, int b, int t) {
    std::vector<int> sizes;
    sizes.push_back(b);
    const int need = (h - t) - (b - 1);  // address bits the middle windows add
    if (need < 0) return {};
    if (need > 0) {
        // as few middle windows as the limit allows, sizes as even as
        // possible, the larger ones first (they sit right above bit 0's window)
        const int mm = std::min(mmax, MAX_WINDOW_HIGH);
        const int cnt = (need + (mm - 1) - 1) / (mm - 1);
        for (int j = 0; j < cnt; ++j) {
            const int add = need / cnt + (j < need % cnt ? 1 : 0);
            sizes.push_back(add + 1);
        }
    }
    sizes.push_back(t);
    for (size_t j = 0; j < sizes.size(); ++j)
        if (sizes[j] < MIN_WINDOW || sizes[j] > (j == 0 ? MAX_WINDOW : MAX_WINDOW_HIGH)) return {};
    return sizes;
}

struct Group {
    int row;
    bool fwd;
    int win;
    std::vector<int> steps;
};

static bool build_passes(Plan& P, const std::vector<int>& sizes, std::vector<PassDesc>& out) {
    const int h = P.h, K = (int)sizes.size() - 1;
    if (K < 1) return false;
    std::vector<int> lo(K + 1), hi(K + 1);
    lo[0] = 0;
    for (int j = 0; j <= K; ++j) {
        if (j > 0) lo[j] = hi[j - 1];
        hi[j] = lo[j] + sizes[j] - 1;
    }
    if (hi[K] != h - 1) return false;
    // a window above address bit 0 shares its tile with the TILE_BITS-M
    // lowest address bits, so it must lie entirely above them
    for (int j = 1; j <= K; ++j)
        if (lo[j] + sizes[j] < TILE_BITS) return false;
    // window of each step
    std::vector<Group> groups;
    int s = 0;
    for (int r = 1; r <= P.last_mid_row(); ++r) {
        const bool fwd = (r % 2) == 1;
        for (int i = 0; i < h; ++i, ++s) {
            const int p = P.step_tgt[s];
            int w;
            if (fwd) {
                w = 0;
                while (p > hi[w]) ++w;
            } else {
                w = K;
                while (p < lo[w]) --w;
            }
            if (groups.empty() || groups.back().row != r || groups.back().win != w)
                groups.push_back(Group{r, fwd, w, {}});
            groups.back().steps.push_back(s);
        }
    }
    out.clear();
    for (size_t g = 0; g < groups.size(); ++g) {
        PassDesc d;
        std::memset(&d, 0, sizeof(d));
        d.xs_step[0] = d.xs_step[1] = -1;
        d.xs_q[0] = d.xs_q[1] = 0;
        const Group& a = groups[g];
        std::vector<int> st = a.steps;
        int type;
        const bool merge = g + 1 < groups.size() && groups[g + 1].win == a.win;
        if (merge) {
            const Group& b = groups[g + 1];
            st.insert(st.end(), b.steps.begin(), b.steps.end());
            if (a.win == K && a.fwd && !b.fwd) type = P_TOP;
            else if (a.win == 0 && !a.fwd && b.fwd) type = P_BOT;
            else return false;
            ++g;
        } else if (a.fwd) {
            type = a.win == 0 ? P_BOT_START : (a.win == K ? P_TOP_END : P_FWD);
        } else {
            if (a.win == K) return false;  // a reversed row never starts a sweep
            type = a.win == 0 ? P_BOT_END : P_REV;
        }
        const int M = sizes[a.win];
        const int B = pass_blk(type, M);  // the turn block gathers method steps B..B+3
        d.type = type;
        d.M = M;
        d.lo = lo[a.win];
        d.step0 = st.front();
        d.pstep0 = -1;  // set once the schedule is chosen (build_pass_steps)
        d.nsteps = pass_nsteps(type, M);
        // the method's steps must be contiguous and match the compile-time shape
        if ((int)st.size() != d.nsteps + (B >= 0 ? 3 : 0)) return false;
        for (size_t m = 0; m < st.size(); ++m)
            if (st[m] != d.step0 + (int)m) return false;
        auto rel = [&](int bit) { return bit < 0 ? -1 : bit - d.lo; };
        for (int i = 0; i < d.nsteps; ++i) {
            const StepSpec sp = step_spec(type, M, i);
            if (i != B) {
                const int m = (B >= 0 && i > B) ? i + 3 : i;
                if (rel(P.step_tgt[st[m]]) != sp.t || rel(P.step_ctl[st[m]]) != sp.c) return false;
                continue;
            }
            // block: targets in {t, t+1}; controls inside it, or sp.c for the first
            for (int m = B; m < B + 4; ++m) {
                const int t = rel(P.step_tgt[st[m]]), c = rel(P.step_ctl[st[m]]);
                if (t != sp.t && t != sp.t + 1) return false;
                const bool inside = c == sp.t || c == sp.t + 1;
                if (m == B ? c != sp.c : !(c < 0 || inside)) return false;
            }
        }
        int nx = 0;
        for (size_t m = 0; m < st.size(); ++m) {
            if (P.step_xq[st[m]] < 0) continue;
            const bool in_blk = B >= 0 && (int)m >= B && (int)m < B + 4;
            int bit = (B >= 0 && (int)m > B) ? (int)m - 3 : (int)m;
            if (in_blk) {  // the block's variant: first output bit low, second high
                if (pass_xm(type, M) != B) return false;
                bit = (nx > 0 && d.xs_step[nx - 1] == B) ? XM_HIGH_BIT : B;
            }
            if (nx >= 2) return false;
            d.xs_step[nx] = bit;
            d.xs_q[nx] = P.step_xq[st[m]];
            ++nx;
        }
        out.push_back(d);
    }
    return true;
}

// The steps of every pass as its kernel runs them. A turn's two steps on
// one target (A with control c, then B without control) become one step
// C[c] = B.A[c], composed in FP64; at the top both depend on an output bit,
// and the pass's entries are followed by one more holding C for x_b = 1
// (variant x_a in g[x_a]).
static void build_pass_steps(Plan& P) {
    P.pass_steps.clear();
    for (PassDesc& d : P.passes) {
        d.pstep0 = (int)P.pass_steps.size();
        const int B = pass_blk(d.type, d.M);
        for (int i = 0; i < d.nsteps; ++i) {
            if (i != B) {
                P.pass_steps.push_back(P.steps[d.step0 + ((B >= 0 && i > B) ? i + 3 : i)]);
                continue;
            }
            // the block: product of method steps B..B+3 on window bits t, t+1
            // (q = bit t + 2 bit t+1), per control value c of the first and
            // variant v = x_a + 2 x_b (x_a: bit xs_step == B, x_b: XM_HIGH_BIT)
            const int t = step_spec(d.type, d.M, B).t;
            StepG blk[BLK_ENTRIES];
            float2* out = &blk[0].g[0][0];
            for (int v = 0; v < 4; ++v)
                for (int c = 0; c < 2; ++c) {
                    cd Mx[4][4];
                    for (int r = 0; r < 4; ++r)
                        for (int q = 0; q < 4; ++q) Mx[r][q] = r == q ? 1.0 : 0.0;
                    for (int m = B; m < B + 4; ++m) {
                        const int gs = d.step0 + m;
                        const auto& G = P.steps64[gs];
                        int x = 0;
                        if (P.step_xq[gs] >= 0)
                            for (int j = 0; j < 2; ++j)
                                if (d.xs_q[j] == P.step_xq[gs] && (d.xs_step[j] == B || d.xs_step[j] == XM_HIGH_BIT))
                                    x = d.xs_step[j] == B ? (v & 1) : (v >> 1);
                        const int tb = P.step_tgt[gs] - d.lo - t;  // 0 or 1
                        // control: none (-1), block bit 0 or 1, or outside the block (2)
                        const int cw = P.step_ctl[gs] < 0 ? -1 : P.step_ctl[gs] - d.lo - t;
                        const int cb = P.step_ctl[gs] < 0 ? -1 : (cw == 0 || cw == 1) ? cw : 2;
                        cd S[4][4];
                        for (int r = 0; r < 4; ++r)
                            for (int q = 0; q < 4; ++q) {
                                S[r][q] = 0.0;
                                if (((r ^ q) & ~(1 << tb) & 3) != 0) continue;  // other bit unchanged
                                const int cv = cb < 0 ? 0 : cb < 2 ? ((q >> cb) & 1) : c;
                                S[r][q] = G[x * 8 + cv * 4 + ((r >> tb) & 1) * 2 + ((q >> tb) & 1)];
                            }
                        cd N[4][4];
                        for (int r = 0; r < 4; ++r)
                            for (int q = 0; q < 4; ++q) {
                                N[r][q] = 0.0;
                                for (int u = 0; u < 4; ++u) N[r][q] += S[r][u] * Mx[u][q];
                            }
                        std::memcpy(Mx, N, sizeof(N));
                    }
                    for (int r = 0; r < 4; ++r)
                        for (int q = 0; q < 4; ++q) out[((v * 2 + c) * 4 + r) * 4 + q] = f2(Mx[r][q]);
                }
            for (int e = 0; e < BLK_ENTRIES; ++e) P.pass_steps.push_back(blk[e]);
        }
    }
}

// Modelled time of a schedule in units of one HBM pass, a heuristic for the
// planner's default (the autotuner times candidates on the device): a pass
// costs the larger of its memory time and its arithmetic time (alpha per
// step; a turn block counts as two steps). A 10-bit window above address bit
// 0 (tiles in rows of 64 bytes) is charged row64 more, which keeps the default
// at width 32 on the schedule measured fastest there (windows 9 / 10 / 7); a
// 10-bit window of a forward or reversed row whose address span reaches 2^27
// entries (1 GiB: its tile touches about 512 pages of 2 MB) costs gamma more.
static double schedule_cost(const std::vector<PassDesc>& ps) {
    const double alpha = 0.105, gamma = 0.25, row64 = 0.35;
    double c = 0;
    for (const auto& p : ps) {
        const int steps = p.nsteps + (pass_blk(p.type, p.M) >= 0 ? 1 : 0);
        c += std::max(1.0, alpha * steps);
        const bool high = p.type != P_BOT && p.type != P_BOT_START && p.type != P_BOT_END;
        if (high && p.M == MAX_WINDOW_HIGH && TILE_BITS - p.M == 3) c += row64;
        if ((p.type == P_FWD || p.type == P_REV) && p.M >= 10 && p.lo + p.M >= 27) c += gamma;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Algorithm 1, symbolically: which tensors are contracted when, with what
// rank and cost. Tensors of the network (Sec. 2.2): each CZ half is a node
// (q, l) with a bond leg to its partner and time legs to the previous and
// next node of the same qubit; input states, output projectors and one-qubit
// gates are absorbed, so a qubit's first and last node have one time leg.
// ---------------------------------------------------------------------------
static void sym_alg1(int n, int d, int* width, double* log2cost) {
    const int h = (d + 1) / 2;
    auto coupled = [&](int q, int l) {
        return (q + 1 < n && q % 2 == l % 2) || (q >= 1 && (q - 1) % 2 == l % 2);
    };
    std::vector<std::vector<int>> pi;
    const int nbond = n * d;
    for (int q = 0; q < n; ++q) {
        std::vector<int> ls;
        for (int l = 0; l < d; ++l)
            if (coupled(q, l)) ls.push_back(l);
        std::vector<std::vector<int>> row;
        for (size_t k = 0; k < ls.size(); ++k) {
            const int l = ls[k];
            const int partner = (q + 1 < n && q % 2 == l % 2) ? q + 1 : q - 1;
            std::vector<int> legs;
            legs.push_back(std::min(q, partner) * d + l);
            if (k > 0) legs.push_back(nbond + q * d + ls[k - 1]);
            if (k + 1 < ls.size()) legs.push_back(nbond + q * d + l);
            std::sort(legs.begin(), legs.end());
            row.push_back(legs);
        }
        // FixedSweepOrder: reverse time on rows q >= 2 with q even
        if (q >= 2 && q % 2 == 0) std::reverse(row.begin(), row.end());
        for (auto& t : row) pi.push_back(t);
    }
    auto sym_diff = [](const std::vector<int>& A, const std::vector<int>& B) {
        std::vector<int> C;
        std::set_symmetric_difference(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(C));
        return C;
    };
    auto uni = [](const std::vector<int>& A, const std::vector<int>& B) {
        std::vector<int> C;
        std::set_union(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(C));
        return (int)C.size();
    };
    if (pi.empty()) { *width = 0; *log2cost = 0; return; }
    std::vector<int> B = pi[0];
    int W = (int)B.size();
    double C = 0;
    size_t i = 1;
    while (i < pi.size()) {
        const auto& X = pi[i];
        auto BX = sym_diff(B, X);
        if ((int)BX.size() <= h || i + 1 >= pi.size()) {
            C += std::ldexp(1.0, uni(B, X));
            B = BX;
            i += 1;
        } else {
            const auto& Y = pi[i + 1];
            auto XY = sym_diff(X, Y);
            C += std::ldexp(1.0, uni(X, Y));
            W = std::max(W, (int)XY.size());
            C += std::ldexp(1.0, uni(B, XY));
            B = sym_diff(B, XY);
            i += 2;
        }
        W = std::max(W, (int)B.size());
    }
    *width = W;
    *log2cost = std::log2(C);
}

// ---------------------------------------------------------------------------

int plan_build(Plan& P, int n, int d, const uint8_t* cliff, const uint8_t* tmask,
               const tb_gate1q* extra, int n_extra, const double* cphase, const tb_opts* opts,
               std::string& err) {
    if (n < 2 || d < 2 || (d + 1) / 2 > MAX_PLAN_H) {
        err = "the planner needs n >= 2, d >= 2 and ceil(d/2) <= 40";
        return TB_EDOMAIN;
    }
    if (n_extra < 0 || (n_extra > 0 && !extra)) { err = "bad extra gate list"; return TB_EINVAL; }
    P.n = n;
    P.d = d;
    P.h = (d + 1) / 2;
    const bool odd_d = (d % 2) != 0;
    if (opts) P.opts = *opts;
    else std::memset(&P.opts, 0, sizeof(P.opts));
    const int h = P.h;

    // ---- folded slot gates U_(q,t) = E . T^tau . C
    const cd w8 = std::polar(1.0, M_PI / 4);
    const M2 T = m2(1, 0, 0, w8);
    P.U.assign((size_t)(d + 1) * n, clifford(0));
    for (int t = 0; t <= d; ++t)
        for (int q = 0; q < n; ++q) {
            const int k = cliff ? cliff[(size_t)t * n + q] : 0;
            if (k > 23) { err = "Clifford index out of range"; return TB_EINVAL; }
            M2 u = clifford(k);
            if (t < d && tmask) {
                const uint8_t tv = tmask[(size_t)t * n + q];
                if (tv > 1) { err = "tmask entries must be 0 or 1"; return TB_EINVAL; }
                if (tv) u = m2_mul(T, u);
            }
            P.U[(size_t)t * n + q] = u;
        }
    for (int e = 0; e < n_extra; ++e) {
        const tb_gate1q& g = extra[e];
        if (g.qubit < 0 || g.qubit >= n || g.slot < 0 || g.slot > d) {
            err = "extra gate outside the circuit";
            return TB_EINVAL;
        }
        const M2 E = m2(cd(g.m[0], g.m[1]), cd(g.m[2], g.m[3]), cd(g.m[4], g.m[5]), cd(g.m[6], g.m[7]));
        M2& u = P.U[(size_t)g.slot * n + g.qubit];
        u = m2_mul(E, u);
    }
    auto U = [&](int q, int t) -> const M2& { return P.U[(size_t)t * n + q]; };

    // ---- entanglers: CZ, or diag(1, 1, 1, e^(i phi)) per gate (phi = pi is CZ exactly)
    P.W.assign((size_t)d * (n - 1), cd(-1.0, 0.0));
    if (cphase)
        for (int l = 0; l < d; ++l)
            for (int i = l % 2; i + 1 < n; i += 2) {
                const double phi = cphase[(size_t)l * (n - 1) + i];
                if (!std::isfinite(phi)) { err = "controlled-phase angles must be finite"; return TB_EINVAL; }
                P.W[(size_t)l * (n - 1) + i] = phi == M_PI ? cd(-1.0, 0.0) : std::polar(1.0, phi);
            }

    // ---- paired steps of rows 1..n-2
    P.steps.clear(); P.steps64.clear(); P.step_tgt.clear(); P.step_ctl.clear(); P.step_xq.clear();
    P.row_end.clear();
    for (int r = 1; r <= P.last_mid_row(); ++r) {
        const bool fwd = (r % 2) == 1;
        for (int i = 0; i < h; ++i) {
            const int p = fwd ? i : h - 1 - i;
            const bool xdep = (p == h - 1);
            StepG sg;
            std::array<cd, 16> sg64;
            for (int x = 0; x < 2; ++x)
                for (int c = 0; c < 2; ++c)
                    for (int ap = 0; ap < 2; ++ap)
                        for (int s = 0; s < 2; ++s) {
                            cd acc = 0;
                            // the consumed layer's entangler with row r-1: 1, or w when s = a = 1
                            const int lw = fwd ? 2 * p : 2 * p + 1;  // (d itself for the create step)
                            const cd wl = lw < d ? P.w(lw, r - 1) : cd(1.0);
                            if (odd_d && p == h - 1) {  // sum-out (forward) / create (backward)
                                if (fwd && ap == 0)
                                    for (int a = 0; a < 2; ++a)
                                        acc += U(r, d).a[x * 2 + a] * ((s & a) ? wl : cd(1.0)) *
                                               ((p == 0) ? U(r, 0).a[a * 2 + 0] : U(r, 2 * p).a[a * 2 + c]);
                                if (!fwd && s == 0)
                                    acc = U(r, d).a[x * 2 + ap] * ((p == 0) ? U(r, 0).a[ap * 2 + 0] : cd(1.0));
                                sg.g[x][c * 4 + ap * 2 + s] = f2(acc);
                                sg64[x * 8 + c * 4 + ap * 2 + s] = acc;
                                continue;
                            }
                            for (int a = 0; a < 2; ++a) {
                                const cd sg_ = (s & a) ? wl : cd(1.0);
                                cd left, right;
                                if (fwd) {
                                    left = U(r, 2 * p + 1).a[ap * 2 + a];
                                    right = (p == 0) ? U(r, 0).a[a * 2 + 0] : U(r, 2 * p).a[a * 2 + c];
                                } else {
                                    left = (p == h - 1) ? U(r, d).a[x * 2 + a] : U(r, 2 * p + 2).a[c * 2 + a];
                                    right = U(r, 2 * p + 1).a[a * 2 + ap];
                                }
                                acc += left * sg_ * right;
                            }
                            if (fwd && p == h - 1) acc *= U(r, d).a[x * 2 + ap];
                            if (!fwd && p == 0) acc *= U(r, 0).a[ap * 2 + 0];
                            sg.g[x][c * 4 + ap * 2 + s] = f2(acc);
                            sg64[x * 8 + c * 4 + ap * 2 + s] = acc;
                        }
            P.steps.push_back(sg);
            P.steps64.push_back(sg64);
            P.step_tgt.push_back((int8_t)p);
            int ctl = -1;
            if (fwd && p > 0) ctl = p - 1;
            if (!fwd && p < h - 1) ctl = p + 1;
            P.step_ctl.push_back((int8_t)ctl);
            P.step_xq.push_back((int16_t)(xdep ? r : -1));
        }
        P.row_end.push_back((int32_t)P.steps.size());
    }

    // ---- row-0 tables: B_0[s] = a0[s_0] prod_(p>=1) M_p[s_p, s_(p-1)] E_x[s_(h-1)]
    P.k = std::min(h, LOW_BITS);
    P.m = std::min(h - P.k, MID_BITS);
    P.top = h - P.k - P.m;
    const int k = P.k, m = P.m, top = P.top;
    std::vector<M2> Mp(h);
    for (int p = 1; p < h; ++p) Mp[p] = m2_mul(U(0, 2 * p), U(0, 2 * p - 1));
    // qubit 0 idles in odd layers: after its last stored layer come slots
    // d-1 and d (even d) or slot d alone (odd d)
    const M2 Eend = odd_d ? U(0, d) : m2_mul(U(0, d), U(0, d - 1));
    P.init_low.assign((size_t)1 << k, make_float2(0, 0));
    for (int64_t s = 0; s < ((int64_t)1 << k); ++s) {
        cd v = U(0, 0).a[(s & 1) * 2 + 0];
        for (int p = 1; p < k; ++p) v *= Mp[p].a[((s >> p) & 1) * 2 + ((s >> (p - 1)) & 1)];
        P.init_low[s] = f2(v);
    }
    P.init_mid.assign((size_t)2 << m, make_float2(0, 0));
    for (int b = 0; b < 2; ++b)
        for (int64_t s = 0; s < ((int64_t)1 << m); ++s) {
            cd v = 1.0;
            int prev = b;
            for (int j = 0; j < m; ++j) {
                const int cur = (int)((s >> j) & 1);
                v *= Mp[k + j].a[cur * 2 + prev];
                prev = cur;
            }
            P.init_mid[((size_t)b << m) + s] = f2(v);
        }
    P.init_top.assign((size_t)4 << top, make_float2(0, 0));
    for (int x = 0; x < 2; ++x)
        for (int b = 0; b < 2; ++b)
            for (int64_t s = 0; s < ((int64_t)1 << top); ++s) {
                cd v = 1.0;
                int prev = b;
                for (int j = 0; j < top; ++j) {
                    const int cur = (int)((s >> j) & 1);
                    v *= Mp[k + m + j].a[cur * 2 + prev];
                    prev = cur;
                }
                v *= Eend.a[x * 2 + prev];
                P.init_top[(((size_t)x * 2 + b) << top) + s] = f2(v);
            }

    // ---- last-row tables: V[s] = e_x^T A_(h-1)(s_(h-1)) ... A_0(s_0) U_(r,0) e_0,
    //      A_p(s) = U_(r,2p+2) D_(2p+1) U_(r,2p+1) D_(2p), D_l = diag(1, (-1)^s)
    //      on the layers where row r = n-1 meets row n-2. For odd d the last
    //      factor has no layer d and no slot d+1: A_(h-1)(s) = U_(r,d) D_(d-1)
    //      (and 0 for s = 1 when layer d-1 is not in L_(n-2): that bit is 0).
    {
        const int r = n - 1;
        auto A = [&](int p, int sbit) {
            const bool even_coupled = ((n - 2) % 2) == 0;  // L_(n-2) holds even layers
            const int lc = even_coupled ? 2 * p : 2 * p + 1;  // the coupled layer of this factor
            const M2 D = m2(1, 0, 0, (sbit && lc < d) ? P.w(lc, n - 2) : cd(1.0));
            const M2 I2 = m2(1, 0, 0, 1);
            const M2 D0 = even_coupled ? D : I2;             // layer 2p
            const M2 D1 = even_coupled ? I2 : D;             // layer 2p+1
            if (odd_d && p == h - 1) {
                if (!even_coupled && sbit) return m2(0, 0, 0, 0);
                return m2_mul(U(r, d), D0);
            }
            return m2_mul(U(r, 2 * p + 2), m2_mul(D1, m2_mul(U(r, 2 * p + 1), D0)));
        };
        std::vector<std::array<M2, 2>> Acache(h);
        for (int p = 0; p < h; ++p)
            for (int sb = 0; sb < 2; ++sb) Acache[p][sb] = A(p, sb);
        P.red_low.assign((size_t)2 << k, make_float2(0, 0));
        for (int64_t s = 0; s < ((int64_t)1 << k); ++s) {
            cd v0 = U(r, 0).a[0], v1 = U(r, 0).a[2];
            for (int p = 0; p < k; ++p) {
                const M2& a = Acache[p][(s >> p) & 1];
                const cd w0 = a.a[0] * v0 + a.a[1] * v1, w1 = a.a[2] * v0 + a.a[3] * v1;
                v0 = w0; v1 = w1;
            }
            P.red_low[2 * s] = f2(v0);
            P.red_low[2 * s + 1] = f2(v1);
        }
        P.red_mid.assign((size_t)4 << m, make_float2(0, 0));
        for (int64_t s = 0; s < ((int64_t)1 << m); ++s) {
            M2 acc = m2(1, 0, 0, 1);
            for (int j = 0; j < m; ++j) acc = m2_mul(Acache[k + j][(s >> j) & 1], acc);
            for (int e = 0; e < 4; ++e) P.red_mid[4 * s + e] = f2(acc.a[e]);
        }
        P.red_top.assign((size_t)4 << top, make_float2(0, 0));
        for (int x = 0; x < 2; ++x)
            for (int64_t s = 0; s < ((int64_t)1 << top); ++s) {
                cd v0 = x == 0 ? 1.0 : 0.0, v1 = x == 0 ? 0.0 : 1.0;  // row vector e_x^T
                for (int j = top - 1; j >= 0; --j) {
                    const M2& a = Acache[k + m + j][(s >> j) & 1];
                    const cd w0 = v0 * a.a[0] + v1 * a.a[2], w1 = v0 * a.a[1] + v1 * a.a[3];
                    v0 = w0; v1 = w1;
                }
                P.red_top[(((size_t)x << top) + s) * 2] = f2(v0);
                P.red_top[(((size_t)x << top) + s) * 2 + 1] = f2(v1);
            }
    }

    // ---- pass schedule (boundaries wider than one CTA's shared memory)
    P.passes.clear();
    P.tc_passes.clear();
    P.tc_mats.clear();
    P.tc_wb = 0;
    if (P.opts.precision != TB_PRECISION_FP32 && P.opts.precision != TB_PRECISION_TF32X3 &&
        P.opts.precision != TB_PRECISION_BF16X3) {
        err = "precision must be TB_PRECISION_FP32, _TF32X3 or _BF16X3";
        return TB_EINVAL;
    }
    if (P.opts.precision != TB_PRECISION_FP32) {
        if (h > SMALL_H_MAX && P.last_mid_row() >= 1) {
            const int rc = tc_schedule(P, err);
            if (rc != TB_OK) return rc;
        }
    } else if (h > SMALL_H_MAX && P.last_mid_row() >= 1) {
        int mmax = P.opts.window_bits ? P.opts.window_bits : MAX_WINDOW;
        if (mmax < MIN_WINDOW || mmax > MAX_WINDOW) { err = "window_bits must be in 5..10"; return TB_EINVAL; }
        const int b_lo = P.opts.bottom_bits ? P.opts.bottom_bits : MIN_WINDOW;
        const int b_hi = P.opts.bottom_bits ? P.opts.bottom_bits : MAX_WINDOW;
        const int t_lo = P.opts.top_bits ? P.opts.top_bits : MIN_WINDOW;
        const int t_hi = P.opts.top_bits ? P.opts.top_bits : MAX_WINDOW_HIGH;
        if (b_lo < MIN_WINDOW || b_hi > MAX_WINDOW) {
            err = "bottom_bits must be in 5..10";
            return TB_EINVAL;
        }
        if (t_lo < MIN_WINDOW || t_hi > MAX_WINDOW_HIGH) {
            err = "top_bits must be in 5..10";
            return TB_EINVAL;
        }
        double best = 1e300;
        for (int b = b_lo; b <= b_hi; ++b)
            for (int t = t_lo; t <= t_hi; ++t) {
                const auto sizes = partition(h, mmax, b, t);
                if (sizes.size() < 2) continue;
                std::vector<PassDesc> ps;
                if (!build_passes(P, sizes, ps)) continue;
                const double c = schedule_cost(ps);
                if (c < best - 1e-9) {
                    best = c;
                    P.passes = ps;
                    P.windows = sizes;
                }
            }
        if (P.passes.empty()) { err = "no pass schedule fits these window limits"; return TB_EINVAL; }
        build_pass_steps(P);
    }

    sym_alg1(n, d, &P.width, &P.log2cost);
    if (P.open_k > 0) {
        const int rc = open_tables(P, err);
        if (rc != TB_OK) return rc;
    }

    // ---- device table image
    TableLayout& L = P.lay;
    int64_t off = 0;
    auto put = [&](int64_t bytes) { const int64_t o = off; off = align_up(off + bytes, 256); return o; };
    const int64_t ns = (int64_t)P.steps.size();
    L.steps = put(ns * (int64_t)sizeof(StepG));
    L.pass_steps = put((int64_t)P.pass_steps.size() * (int64_t)sizeof(StepG));
    L.step_tgt = put(ns);
    L.step_ctl = put(ns);
    L.step_xq = put(ns * 2);
    L.row_end = put((int64_t)P.row_end.size() * 4);
    L.init_low = put((int64_t)P.init_low.size() * 8);
    L.init_mid = put((int64_t)P.init_mid.size() * 8);
    L.init_top = put((int64_t)P.init_top.size() * 8);
    L.red_low = put((int64_t)P.red_low.size() * 8);
    L.red_mid = put((int64_t)P.red_mid.size() * 8);
    L.red_top = put((int64_t)P.red_top.size() * 8);
    L.tc_mats = put((int64_t)P.tc_mats.size());
    L.open_E = put((int64_t)P.open_E.size() * 8);
    L.open_Es = put((int64_t)P.open_Es.size());
    L.open_ops = put((int64_t)P.open_ops.size() * (int64_t)sizeof(OpenOp));
    L.open_seg = put((int64_t)P.open_seg.size() * 4);
    L.total = off;
    P.blob.assign((size_t)L.total, 0);
    auto cp = [&](int64_t o, const void* src, size_t bytes) {
        if (bytes) std::memcpy(P.blob.data() + o, src, bytes);
    };
    cp(L.steps, P.steps.data(), P.steps.size() * sizeof(StepG));
    cp(L.pass_steps, P.pass_steps.data(), P.pass_steps.size() * sizeof(StepG));
    cp(L.step_tgt, P.step_tgt.data(), P.step_tgt.size());
    cp(L.step_ctl, P.step_ctl.data(), P.step_ctl.size());
    cp(L.step_xq, P.step_xq.data(), P.step_xq.size() * 2);
    cp(L.row_end, P.row_end.data(), P.row_end.size() * 4);
    cp(L.init_low, P.init_low.data(), P.init_low.size() * 8);
    cp(L.init_mid, P.init_mid.data(), P.init_mid.size() * 8);
    cp(L.init_top, P.init_top.data(), P.init_top.size() * 8);
    cp(L.red_low, P.red_low.data(), P.red_low.size() * 8);
    cp(L.red_mid, P.red_mid.data(), P.red_mid.size() * 8);
    cp(L.red_top, P.red_top.data(), P.red_top.size() * 8);
    cp(L.tc_mats, P.tc_mats.data(), P.tc_mats.size());
    cp(L.open_E, P.open_E.data(), P.open_E.size() * 8);
    cp(L.open_Es, P.open_Es.data(), P.open_Es.size());
    cp(L.open_ops, P.open_ops.data(), P.open_ops.size() * sizeof(OpenOp));
    cp(L.open_seg, P.open_seg.data(), P.open_seg.size() * 4);
    return TB_OK;
}

}  // namespace tb
