"""The separable gather list of Kaiser-Bessel gridding (kb_lists.h), built on the CPU and expanded back into
half-plane cells, against the oracle's direct FP64 gridding (oracle_grid_kb).

The persistent imaging kernel grids with this list at every side it serves (W <= 8): one entry per
(visibility or its mirror, column of its support) with the column weight C(u - gu), the record's first row v0
and a row of W weights C(v - gv) (-1)^k.  A small host program compiles the library's own list builder,
expands every entry over its W rows (mod N) in FP64 and prints the half plane u in [0, N/2); the test feeds it
random baselines (some beyond the keep limit, some flagged, autocorrelations on and off) and compares with the
oracle's grid, which spreads each visibility and its mirror over the full plane.  No GPU is needed, only g++.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CXX = shutil.which("g++")

DRIVER = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include "kb_lists.h"
using namespace blink;

// stdin: N W du autos n_tiles, flags[n_tiles], then per baseline (i >= j order) u v w re im.
// stdout: the half plane [N][N/2] (row v, column u) as re im lines, and the entry and record counts.
int main() {
    int N, W, autos, nt;
    double du;
    if (std::scanf("%d %d %lf %d %d", &N, &W, &du, &autos, &nt) != 5) return 1;
    std::vector<int> fl(nt);
    for (int t = 0; t < nt; t++) std::scanf("%d", &fl[t]);
    const int64_t B = (int64_t)nt * (nt + 1) / 2;
    std::vector<double> uvw(B * 3), re(B), im(B);
    std::vector<int> bi(B), bj(B);
    for (int i = 0, b = 0; i < nt; i++)
        for (int j = 0; j <= i; j++, b++) {
            bi[b] = i;
            bj[b] = j;
            std::scanf("%lf %lf %lf %lf %lf", &uvw[b * 3], &uvw[b * 3 + 1], &uvw[b * 3 + 2], &re[b], &im[b]);
        }
    std::vector<SepEntry> ent;
    std::vector<float> wrow;
    std::vector<int> off;
    kb_sep_channel(N, W, B, autos != 0, du, uvw.data(), [&](int64_t b) { return fl[bi[b]] || fl[bj[b]]; },
                   [&](int64_t b) { return bi[b] == bj[b]; }, ent, wrow, off);
    const int half = N / 2;
    std::vector<double> H((size_t)N * half * 2, 0.0);
    for (int u = 0; u < half; u++) {
        const int end = u + 1 <= half ? off[u + 1] : (int)ent.size();
        for (int e = off[u]; e < end; e++) {
            const SepEntry& x = ent[e];
            const uint32_t b = x.bc & 0x7FFFFFFFu;
            const double xr = re[b], xi = (x.bc >> 31) ? -im[b] : im[b];
            for (int k = 0; k < W; k++) {
                const double w = (double)x.wu * (double)wrow[(size_t)x.rec * kSepRowW + k] * ((k & 1) ? -1.0 : 1.0);
                const int v = ((x.v0 + k) % N + N) % N;
                H[((size_t)v * half + u) * 2 + 0] += w * xr;
                H[((size_t)v * half + u) * 2 + 1] += w * xi;
            }
            for (int k = W; k < kSepRowW; k++)
                if (wrow[(size_t)x.rec * kSepRowW + k] != 0.f) return 2;        // rows past W must be zero
        }
    }
    for (size_t q = 0; q < H.size(); q += 2) std::printf("%.17g %.17g\n", H[q], H[q + 1]);
    std::printf("%zu %zu\n", ent.size(), wrow.size() / kSepRowW);
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if not CXX:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("kb_lists")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    cmd = [CXX, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2505_15204_gb300", "csrc"), "-o", str(exe),
           str(src)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return str(exe)


def _case(seed, N, W, nt, autos, n_flag):
    rng = np.random.default_rng(seed)
    du = 1.7
    B = nt * (nt + 1) // 2
    lim = N / 2 - W / 2
    # cell positions spread over the whole grid, a few beyond the keep limit, some on the column u = 0 and
    # on whole cells (supports of W - 1 cells)
    g = rng.uniform(-1.05 * lim, 1.05 * lim, size=(B, 2))
    g[::7, 0] = rng.uniform(-W / 2, W / 2, size=g[::7, 0].shape)
    g[::11] = np.round(g[::11])
    uvw = np.zeros((B, 3))
    uvw[:, :2] = g * du
    V = rng.normal(size=B) + 1j * rng.normal(size=B)
    flags = np.zeros(nt, np.uint8)
    flags[rng.choice(nt, size=n_flag, replace=False)] = 1
    return du, uvw, V, flags


def _run(exe, N, W, du, autos, flags, uvw, V):
    nt = len(flags)
    lines = [f"{N} {W} {float(du):.17g} {int(autos)} {nt}", " ".join(str(int(x)) for x in flags)]
    lines += [" ".join(f"{float(x):.17g}" for x in (u, v, w, z.real, z.imag)) for (u, v, w), z in zip(uvw, V)]
    r = subprocess.run([exe], input="\n".join(lines), capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    out = r.stdout.strip().splitlines()
    n_ent, n_rec = (int(t) for t in out[-1].split())
    vals = np.array([[float(t) for t in line.split()] for line in out[:-1]])
    H = (vals[:, 0] + 1j * vals[:, 1]).reshape(N, N // 2)
    return H, n_ent, n_rec


def _oracle_half(N, W, du, autos, flags, uvw, V):
    nt = len(flags)
    S = np.zeros((len(V), 4), np.complex128)
    S[:, 0] = V                          # XX with K = 1: the gridded value is V itself
    G, _ = oracle.grid_kb(S, nt, 1, uvw, du, W, N, pol=oracle.POL_XX, autos=autos, flags=flags)
    return G[:, : N // 2]                # G[v][u], the half plane u in [0, N/2)


@pytest.mark.parametrize("N,W,autos,n_flag", [(256, 6, True, 2), (256, 4, False, 0), (512, 8, True, 1),
                                              (256, 2, True, 0)])
def test_separable_list_expands_to_the_oracle_grid(driver, N, W, autos, n_flag):
    du, uvw, V, flags = _case(N + W, N, W, 24, autos, n_flag)
    H, n_ent, n_rec = _run(driver, N, W, du, autos, flags, uvw, V)
    G = _oracle_half(N, W, du, autos, flags, uvw, V)
    # FP32 weights (C(u - gu) and C(v - gv) each rounded once, 2^-24 relative) against the FP64 products:
    # measured 3e-8 to 7e-8 of the grid's peak
    assert np.abs(H - G).max() <= 3e-7 * np.abs(G).max()
    assert n_ent > 0 and n_rec > 0


def test_separable_list_counts_and_order(driver):
    # every kept cross visibility gives one record, plus one for its mirror when its support reaches u <= 0;
    # each record's entries are the columns u >= 0 of its support; nothing of a flagged tile appears
    N, W = 256, 6
    du, uvw, V, flags = _case(3, N, W, 16, True, 3)
    H, n_ent, n_rec = _run(driver, N, W, du, True, flags, uvw, V)
    nt = len(flags)
    lim, h = N / 2 - W / 2, W / 2
    want_rec = want_ent = 0
    b = 0
    for i in range(nt):
        for j in range(i + 1):
            if not (flags[i] or flags[j]):
                if i == j:
                    cells = [c for c in range(-W, W + 1) if abs(c) < h]
                    want_rec += 1
                    want_ent += sum(1 for c in cells if c >= 0)
                else:
                    gu, gv = uvw[b, 0] / du, uvw[b, 1] / du
                    if abs(gu) <= lim and abs(gv) <= lim:
                        cols = [c for c in range(int(np.floor(gu - h)), int(np.ceil(gu + h)) + 1) if abs(c - gu) < h]
                        pos, neg = [c for c in cols if c >= 0], [c for c in cols if c <= 0]
                        want_rec += bool(pos) + bool(neg)
                        want_ent += len(pos) + len(neg)
            b += 1
    assert (n_rec, n_ent) == (want_rec, want_ent)
    # a flagged tile's baselines leave their cells empty: zero V on them changes nothing
    V2 = V.copy()
    b = 0
    for i in range(nt):
        for j in range(i + 1):
            if flags[i] or flags[j]:
                V2[b] = 0
            b += 1
    H2, _, _ = _run(driver, N, W, du, True, flags, uvw, V2)
    assert np.array_equal(H, H2)
