"""The regular tile grid's divisions (lbm_step.cuh: div_magic_of on the host,
div_magic on the device): floor(n / d) = (n m) >> (32 + s) with the host's
m and s, for every list index 0 <= n < 2^31 that a launch can have.

A host program built from the library's header prints (m, s) for a set of
divisors; the check restates the device formula, (n * m) >> (32 + s), and
compares it with Python's exact integer division on the boundary cases
(multiples of d and their neighbours, the largest n) and on seeded random
indices. No GPU is needed: the constants are host code."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1605_01800_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "lbm_step.cuh"
int main(int argc, char** argv) {
    for (int i = 1; i < argc; ++i) {
        const int d = atoi(argv[i]);
        unsigned long long m = 0;
        int s = 0;
        lbm::div_magic_of(d, &m, &s);
        printf("%d %llu %d\n", d, m, s);
    }
    return 0;
}
"""


def divisors():
    rng = random.Random(20240601)
    ds = list(range(1, 130)) + [2 ** k for k in range(1, 31)] + [2 ** k - 1 for k in range(2, 32)]
    ds += [2 ** k + 1 for k in range(1, 30)] + [rng.randrange(1, 2 ** 31) for _ in range(60)]
    ds += [128 * 64, 4096 // 32, 4096 * 4096 // (32 * 16)]   # tile grids of the workloads
    return sorted(set(ds))


@pytest.fixture(scope="module")
def constants(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("divmagic")
    src, exe = d / "divmagic.cu", d / "divmagic"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-gencode", "arch=compute_103a,code=sm_103a", str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)] + [str(x) for x in divisors()], check=True, capture_output=True, text=True)
    rows = [tuple(int(v) for v in line.split()) for line in out.stdout.split("\n") if line.strip()]
    return {d: (m, s) for d, m, s in rows}


def test_constants_fit(constants):
    for d, (m, s) in constants.items():
        assert (1 << s) >= d and (s == 0 or (1 << (s - 1)) < d), d
        assert m < (1 << 34), d
        assert (2 ** 31 - 1) * m < 2 ** 64, d   # the product never leaves 64 bits


def test_division_is_exact(constants):
    rng = random.Random(7)
    for d, (m, s) in constants.items():
        ns = [0, 1, d - 1, d, d + 1, 2 ** 31 - 1, 2 ** 31 - 2]
        ns += [k * d + e for k in (1, 2, 3, (2 ** 31 - 1) // d) for e in (-1, 0, 1)]
        ns += [rng.randrange(0, 2 ** 31) for _ in range(200)]
        for n in ns:
            if 0 <= n < 2 ** 31:
                assert (n * m) >> (32 + s) == n // d, (n, d)
