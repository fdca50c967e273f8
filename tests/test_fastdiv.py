"""The stencils' point coordinates use division by invariant integers: FastDiv::of (host,
csrc/tg_common.cuh) builds the multiplier and shifts, the device computes
q = (t + ((n - t) >> s1)) >> s2 with t = mulhi(m, n).  This compiles a host program
against the library header, applies the same formula to the constants FastDiv::of produces
and compares with plain integer division: every divisor N and N^2 of the grids the
library accepts (N = 3 .. 2047 and the lattice sizes), dividends at the edges of each
quotient, and random dividends below 2^31."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cstdint>
#include <random>
#include "tg_common.cuh"
static unsigned q_of(const tg::FastDiv &f, unsigned n) {
    const unsigned t = (unsigned)(((uint64_t)f.m * n) >> 32);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}
int main() {
    std::mt19937 rng(7);
    long bad = 0, checked = 0;
    for (unsigned N = 1; N <= 2048; ++N) {
        const unsigned ds[2] = {N, N * N};
        for (unsigned d : ds) {
            const tg::FastDiv f = tg::FastDiv::of(d);
            const uint64_t top = (1ull << 31) - 1;
            const uint64_t ns[6] = {0, d - 1, d, d + 1, top, top / d * d - 1};
            for (uint64_t n : ns) {
                if (n > top) continue;
                ++checked;
                bad += q_of(f, (unsigned)n) != (unsigned)(n / d);
            }
            for (int r = 0; r < 200; ++r) {
                const unsigned n = rng() & 0x7fffffffu;
                ++checked;
                bad += q_of(f, n) != n / d;
            }
        }
    }
    std::printf("%ld %ld\n", checked, bad);
    return bad != 0;
}
'''


def test_fastdiv_constants_give_exact_quotients(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "fastdiv_check.cu"
    src.write_text(SRC)
    exe = tmp_path / "fastdiv_check"
    inc = os.path.join(ROOT, "paper_2005_03070_gb300", "csrc")
    p = subprocess.run([nvcc, "-std=c++17", "-O2", "-I" + inc, "-I" + os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe)], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    checked, bad = (int(v) for v in r.stdout.split())
    assert r.returncode == 0 and bad == 0 and checked > 800000, r.stdout
