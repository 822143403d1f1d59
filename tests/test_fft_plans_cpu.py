"""The compile-time transform plans of the mixed-radix passes (side 1200: columns 1200 = 16 x 15 x 5, rows
600 = 8 x 15 x 5) and the 15-point prime-factor DFT, run on the CPU.

The library's own stage code (fft_ct.cuh, host-callable) is compiled into a small host program in which one
host thread stands for each GPU thread of a transform and a barrier for each __syncthreads; its outputs are
compared here with a direct DFT in FP64.  No GPU is needed, only nvcc.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else shutil.which("nvcc")

DRIVER = r"""
#include <barrier>
#include <cmath>
#include <cstdio>
#include <thread>
#include <vector>
#include "fft_ct.cuh"
using namespace blink;

// argv: which (1200 | 600 | 15), then the input as re im pairs on stdin; prints the output pairs
int main(int argc, char** argv) {
    const int which = std::atoi(argv[1]);
    const int n = which;
    std::vector<float2> in(n);
    for (int i = 0; i < n; i++) std::scanf("%f %f", &in[i].x, &in[i].y);
    std::vector<float2> out(n);
    if (which == 15) {
        float2 v[15];
        for (int i = 0; i < 15; i++) v[i] = in[i];
        idft<15>(v);
        for (int i = 0; i < 15; i++) out[i] = v[i];
    } else {
        const int nt = which == 1200 ? kCol1200Threads : kRow600Threads;
        const int slots = which == 1200 ? kCol1200Slots : kRow600Slots;
        std::vector<float2> a(slots, make_float2(NAN, NAN)), b(slots, make_float2(NAN, NAN)), roots(n);
        for (int k = 0; k < n; k++) roots[k] = make_float2((float)std::cos(2 * M_PI * k / n), (float)std::sin(2 * M_PI * k / n));
        for (int i = 0; i < n; i++) a[i] = in[i];
        std::barrier bar(nt);
        std::vector<std::thread> th;
        for (int t = 0; t < nt; t++)
            th.emplace_back([&, t] {
                auto sync = [&] { bar.arrive_and_wait(); };
                if (which == 1200) fft1200_cols(a.data(), b.data(), roots.data(), t, sync);
                else fft600_rows(a.data(), b.data(), roots.data(), t, sync);
            });
        for (auto& h : th) h.join();
        for (int i = 0; i < n; i++) out[i] = b[i];
    }
    for (int i = 0; i < n; i++) std::printf("%.9g %.9g\n", out[i].x, out[i].y);
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if not NVCC:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("fft_plans")
    src = d / "driver.cu"
    src.write_text(DRIVER)
    exe = d / "driver"
    cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++20", "-O2", "-Xcompiler", "-pthread",
           "-I", os.path.join(ROOT, "paper_2505_15204_gb300", "csrc"), "-o", str(exe), str(src)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return str(exe)


def _run(exe, n, x):
    inp = "\n".join(f"{v.real:.9g} {v.imag:.9g}" for v in x.astype(np.complex64))
    r = subprocess.run([exe, str(n)], input=inp, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    vals = np.array([[float(t) for t in line.split()] for line in r.stdout.strip().splitlines()])
    return vals[:, 0] + 1j * vals[:, 1]


def _idft(x):
    n = len(x)
    k = np.arange(n)
    return np.exp(2j * np.pi * np.outer(k, k) / n) @ x.astype(np.complex128)


@pytest.mark.parametrize("n", [15, 600, 1200])
def test_fixed_plan_equals_direct_dft(driver, n):
    rng = np.random.default_rng(n)
    x = (rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64)
    got = _run(driver, n, x)
    ref = _idft(x)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


def test_fixed_plan_single_points(driver):
    # a unit impulse at point p transforms to exp(2 pi i p k / n): every twiddle of every stage is exercised
    n = 1200
    for p in (0, 1, 75, 599, 1199):
        x = np.zeros(n, np.complex64)
        x[p] = 1.0
        got = _run(driver, n, x)
        ref = np.exp(2j * np.pi * p * np.arange(n) / n)
        assert np.abs(got - ref).max() <= 2e-6, p
