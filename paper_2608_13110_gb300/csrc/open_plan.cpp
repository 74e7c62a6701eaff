// Host tables of an open plan: k output bits left open (Algorithm 2).
//
// The output bits of the last k qubits (the open band, band bit j = qubit
// n-k+j) stay open; the sweep of Algorithm 1 absorbs the fixed region (rows
// 0..n-k-1) into the boundary B[sigma], sigma_l the value of qubit n-k-1 in
// the CZ layers l that couple it to qubit n-k (l = n-k-1 mod 2; sigma_l at
// address bit floor(l/2)). The band's own network splits into
//   early region: band tensors of the first c = 2k CZ layers. It meets the
//     fixed region in the k crossing layers l < c (address bits 0..k-1) and
//     leaves k open legs y (the band's values after layer c-1);
//   late region: the band tensors of layers c..d-1 and the output slot.
// Algorithm 2 contracts the early region on its own, joins it with the
// boundary over the k shared bits, and absorbs the late region layer by layer.
// Here the early region is the matrix
//   E[s][y] = <y| prod_(t < c) CZ'_t(s) U_t |0^k>,
// (U_t the band's slot-t gates, CZ'_t the band's CZs of layer t times
// Z^(s_i) on band bit 0 when t is the crossing layer with address bit i),
// multiplied on the left by the late operations that precede the first late
// crossing (they act on y only, so they commute with the join). Every later
// crossing l_i contracts sigma_(l_i) (address bit k+i-1):
//   Z'[y] = sum_s (-1)^(s y_0) Z[s][y]   (w^(s y_0) for an entangler diag(1,1,1,w)),
// followed by segment i: the band operations after layer l_i up to the band
// CZs of the next crossing layer (the output slot d after the last one).
// All of it is computed in FP64 and stored in FP32 for the device.

#include <cmath>
#include <complex>
#include <string>
#include <cstring>
#include <vector>

#include "tb_plan.h"

namespace tb {

using cd = std::complex<double>;

namespace {

struct Band {
    const Plan& P;
    int k, q0;
    std::vector<cd> psi;
    void gate(int j, const M2& u) {
        for (size_t y = 0; y < psi.size(); ++y) {
            if ((y >> j) & 1) continue;
            const size_t y1 = y | ((size_t)1 << j);
            const cd a = psi[y], b = psi[y1];
            psi[y] = u.a[0] * a + u.a[1] * b;
            psi[y1] = u.a[2] * a + u.a[3] * b;
        }
    }
    // entangler diag(1, 1, 1, w) on band bits j, j+1 (w = -1: CZ)
    void cz(int j, cd w) {
        for (size_t y = 0; y < psi.size(); ++y)
            if (((y >> j) & 1) && ((y >> (j + 1)) & 1)) psi[y] *= w;
    }
    // the crossing entangler with its fixed-region bit equal to 1: w on band bit 0
    void z0(cd w) {
        for (size_t y = 0; y < psi.size(); ++y)
            if (y & 1) psi[y] *= w;
    }
};

}  // namespace

int open_tables(Plan& P, std::string& err) {
    const int n = P.n, d = P.d, h = P.h, k = P.open_k;
    const int q0 = n - k;               // band bit 0
    const int par = (n - k - 1) % 2;    // parity of the crossing layers
    const int c = 2 * k;
    auto U = [&](int q, int t) -> const M2& { return P.U[(size_t)t * n + q]; };
    // band CZs of layer t: pairs (q, q+1), q = t mod 2, both in the band
    auto band_cz = [&](int t, std::vector<int>& js) {
        js.clear();
        for (int q = q0; q + 1 < n; ++q)
            if (q % 2 == t % 2) js.push_back(q - q0);
    };
    const int l1 = c + ((c % 2) == par ? 0 : 1);  // first late crossing layer
    // late crossings l1, l1+2, ..., d-1 or d-2: h - k of them, h - k - 1 when
    // d is odd and the crossing layers are odd (the boundary's top bit is 0
    // there and stays as the high half of the last buffer, never read)
    const int nlate = (d - 1 - l1) / 2 + 1;
    if (nlate < 1 || nlate > h - k || l1 + 2 * (nlate - 1) > d - 1) {
        err = "internal: late crossings beyond the last layer";
        return TB_EINVAL;
    }
    const size_t B = (size_t)1 << k;
    P.open_E.assign(B * B, make_float2(0, 0));
    std::vector<cd> E64(B * B);
    std::vector<int> js;
    for (size_t s = 0; s < B; ++s) {
        Band band{P, k, q0, std::vector<cd>(B, cd(0.0))};
        band.psi[0] = 1.0;
        for (int t = 0; t < c; ++t) {
            for (int j = 0; j < k; ++j) band.gate(j, U(q0 + j, t));
            band_cz(t, js);
            for (int j : js) band.cz(j, P.w(t, q0 + j));
            if (t % 2 == par && ((s >> (t / 2)) & 1)) band.z0(P.w(t, q0 - 1));
        }
        // late operations before the first late crossing's contraction
        for (int t = c; t <= l1; ++t) {
            for (int j = 0; j < k; ++j) band.gate(j, U(q0 + j, t));
            band_cz(t, js);
            for (int j : js) band.cz(j, P.w(t, q0 + j));
        }
        for (size_t y = 0; y < B; ++y) {
            P.open_E[s * B + y] = make_float2((float)band.psi[y].real(), (float)band.psi[y].imag());
            E64[s * B + y] = band.psi[y];
        }
    }
    // The tensor-core join applies Z[r][y] = sum_s B[r][s] E[s][y] as the real
    // GEMM D[r][n] = sum_kk A[r][kk] Bm[kk][n], kk = 2s + pi, n = 2y + po
    // (A = the boundary's (re, im) floats): Bm[2s][2y] = Re E, Bm[2s+1][2y] =
    // -Im E, Bm[2s][2y+1] = Im E, Bm[2s+1][2y+1] = Re E. Bm = hi + lo (TF32,
    // from the FP64 E), stored per (N tile, K chunk) block: hi then lo, each
    // NT x JOIN_KC in the canonical K-major layout.
    P.open_Es.clear();
    if (k >= JOIN_TC_MIN_K) {
        const int KR = 2 << k, NT = join_nt(k), nkc = KR / JOIN_KC;
        const int64_t part = (int64_t)NT * JOIN_KC * 4;
        P.open_Es.assign((size_t)(KR / NT) * nkc * 2 * part, 0);
        for (int n = 0; n < KR; ++n)
            for (int kk = 0; kk < KR; ++kk) {
                const cd z = E64[(size_t)(kk >> 1) * B + (n >> 1)];
                const int po = n & 1, pi = kk & 1;
                const double val = po == 0 ? (pi == 0 ? z.real() : -z.imag()) : (pi == 0 ? z.imag() : z.real());
                const int nt = n / NT, kc = kk / JOIN_KC;
                uint8_t* blk = P.open_Es.data() + ((int64_t)nt * nkc + kc) * 2 * part;
                const int64_t off = canon_offset(n % NT, kk % JOIN_KC, JOIN_KC, 4);
                const float vh = round_tf32(val);
                const float vl = round_tf32(val - (double)vh);
                std::memcpy(blk + off, &vh, 4);
                std::memcpy(blk + part + off, &vl, 4);
            }
    }
    // segments after each late crossing
    P.open_ops.clear();
    P.open_seg.assign(1, 0);
    auto push_gate = [&](int j, const M2& u) {
        OpenOp o;
        o.kind = 0;
        o.j = j;
        for (int e = 0; e < 4; ++e) o.m[e] = make_float2((float)u.a[e].real(), (float)u.a[e].imag());
        P.open_ops.push_back(o);
    };
    auto push_cz = [&](int j, cd w) {  // m[0] = w of diag(1, 1, 1, w)
        OpenOp o;
        o.kind = 1;
        o.j = j;
        for (int e = 0; e < 4; ++e) o.m[e] = make_float2(0, 0);
        o.m[0] = make_float2((float)w.real(), (float)w.imag());
        P.open_ops.push_back(o);
    };
    P.open_w.clear();
    for (int i = 0; i < nlate; ++i) {
        const int li = l1 + 2 * i;
        const cd wc = P.w(li, q0 - 1);  // crossing entangler: sum_s w^(s y0) Z[s][y]
        P.open_w.push_back(make_float2((float)wc.real(), (float)wc.imag()));
        const bool last = i + 1 == nlate;
        const int stop = last ? d : li + 2;  // next crossing layer (its band CZs included)
        for (int t = li + 1; t <= stop; ++t) {
            for (int j = 0; j < k; ++j) push_gate(j, U(q0 + j, t));
            if (t < d) {
                band_cz(t, js);
                for (int j : js) push_cz(j, P.w(t, q0 + j));
            }
        }
        P.open_seg.push_back((int32_t)P.open_ops.size());
    }
    return TB_OK;
}

}  // namespace tb
