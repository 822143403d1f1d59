// Kaiser-Bessel gridding weights and the separable gather list of one channel (host code only: the plan
// builder calls it, and a CPU test compiles it without CUDA).
//
// Separable Kaiser-Bessel kernel of W cells on a grid twice the image side (oversampling 2):
// C(t) = I0(beta sqrt(1 - (2t/W)^2)) beta / (W sinh beta) for |t| < W/2 (unit integral), with
// beta = pi sqrt((W/2)^2 (3/2)^2 - 0.8) (Beatty, Nishimura and Pauly, IEEE TMI 2005, for oversampling 2).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace blink {

constexpr int kSepRowW = 8;                  // row weights stored per record (kernels up to W = 8)

inline double kb_beta(int W) { return 3.14159265358979323846 * std::sqrt(0.5625 * W * W - 0.8); }

inline double kb_weight(double t, int W, double beta) {
    const double h = 0.5 * W;
    if (!(std::fabs(t) < h)) return 0.0;
    const double r = t / h;
    return std::cyl_bessel_i(0.0, beta * std::sqrt(1.0 - r * r)) * beta / (W * std::sinh(beta));
}

// The cells within W/2 of x (at most W, consecutive and increasing) and, when `ws` is given, their weights
// C(c - x).  Returns their number.
inline int kb_support_cells(double x, int W, double beta, int* cs, double* ws) {
    const double h = 0.5 * W;
    int n = 0;
    for (int c = (int)std::floor(x - h); c <= (int)std::ceil(x + h); c++)
        if (std::fabs((double)c - x) < h) {
            if (ws) ws[n] = kb_weight((double)c - x, W, beta);
            cs[n++] = c;
        }
    return n;
}

// One column entry of the separable list: the record's baseline b | conj << 31, its first row v0 (signed; rows
// are taken mod N), the column weight C(u - gu) and the record's number in the channel.
struct SepEntry {
    uint32_t bc;
    int32_t v0;
    float wu;
    uint32_t rec;
};

// The separable list of one channel on a grid of side N with a kernel of W <= kSepRowW cells.  A record is a
// kept cross visibility at g = uvw[b] / du (its support inside the grid: |gu|, |gv| <= N/2 - W/2), its mirror
// (the conjugate at -g), or an autocorrelation (at g = 0, no mirror), in baseline order, the visibility
// before its mirror; records whose support misses the half plane u >= 0 are left out.  Each record has a row
// of kSepRowW weights C(v0 + k - gv) (-1)^k (zero past its support) in `wrow`; each (record, column u >= 0 of
// its support) pair is an entry, sorted by (u, v0, record), and `off[u]` is column u's first entry
// (u = 0 .. N/2; entries of column u end at off[u + 1], those of column N/2 at the list's end).
// skip(b): the baseline is flagged; is_auto(b): it is an autocorrelation; uvw: [B][3] in wavelengths.
template <typename Skip, typename IsAuto>
void kb_sep_channel(int N, int W, int64_t B, bool autos, double du, const double* uvw, Skip skip, IsAuto is_auto,
                    std::vector<SepEntry>& ent, std::vector<float>& wrow, std::vector<int>& off) {
    const double beta = kb_beta(W), lim = 0.5 * N - 0.5 * W;
    const int half = N / 2;
    ent.clear();
    wrow.clear();
    struct Col {
        int u;
        SepEntry e;
    };
    std::vector<Col> cols;
    int cu[20], cv[20], us[20];
    double wu[20], wv[20], wus[20], wm[20];
    // a record of nv rows from v0 (weights ws in increasing v) meeting the columns us[0 .. n_us)
    auto record = [&](uint32_t bc, int v0, const double* ws, int nv, int n_us) {
        const uint32_t r = (uint32_t)(wrow.size() / kSepRowW);
        for (int k = 0; k < kSepRowW; k++) wrow.push_back(k < nv ? (float)((k & 1) ? -ws[k] : ws[k]) : 0.f);
        for (int q = 0; q < n_us; q++) cols.push_back({us[q], SepEntry{bc, v0, (float)wus[q], r}});
    };
    for (int64_t b = 0; b < B; b++) {
        if (skip(b)) continue;
        int n_us = 0;
        if (is_auto(b)) {
            if (!autos) continue;
            const int n = kb_support_cells(0.0, W, beta, cu, wu);
            for (int r = 0; r < n; r++)
                if (cu[r] >= 0) {
                    us[n_us] = cu[r];
                    wus[n_us++] = wu[r];
                }
            record((uint32_t)b, cu[0], wu, n, n_us);
            continue;
        }
        const double gu = uvw[b * 3 + 0] / du, gv = uvw[b * 3 + 1] / du;
        if (!(std::fabs(gu) <= lim && std::fabs(gv) <= lim)) continue;
        const int nu = kb_support_cells(gu, W, beta, cu, wu), nv = kb_support_cells(gv, W, beta, cv, wv);
        for (int r = 0; r < nu; r++)
            if (cu[r] >= 0) {
                us[n_us] = cu[r];
                wus[n_us++] = wu[r];
            }
        if (n_us) record((uint32_t)b, cv[0], wv, nv, n_us);
        // the mirror: rows -cv[nv - 1] .. -cv[0], columns -cu[r] for cu[r] <= 0
        for (int k = 0; k < nv; k++) wm[k] = wv[nv - 1 - k];
        n_us = 0;
        for (int r = 0; r < nu; r++)
            if (cu[r] <= 0) {
                us[n_us] = -cu[r];
                wus[n_us++] = wu[r];
            }
        if (n_us) record((uint32_t)b | 0x80000000u, -cv[nv - 1], wm, nv, n_us);
    }
    std::sort(cols.begin(), cols.end(), [](const Col& x, const Col& y) {
        return x.u != y.u ? x.u < y.u : (x.e.v0 != y.e.v0 ? x.e.v0 < y.e.v0 : x.e.rec < y.e.rec);
    });
    off.assign(half + 1, 0);
    size_t e = 0;
    for (int u = 0; u <= half; u++) {
        while (e < cols.size() && cols[e].u < u) e++;
        off[u] = (int)e;
    }
    ent.resize(cols.size());
    for (size_t q = 0; q < cols.size(); q++) ent[q] = cols[q].e;
}

}  // namespace blink
