"""Host checks of the CUDA path's field helpers (no GPU).

gl.cuh's host-callable helpers are compiled into a small host program with
nvcc and compared against Python integers:
- gl::mul_pow2(x, e) = x 2^e mod p for every 0 <= e < 96, canonical, and its
  negation equal to x 2^(e+96) (2^96 = -1 mod p); the in-register DFTs of the
  NTT passes multiply by roots of unity only through this helper;
- gl::reduce128(lo, hi) congruent to lo + 2^64 hi and below 2^64.
The NTT kernels also rely on w_32 = 7^((p-1)/32) being a power of 2; that
fact is pinned here from the definition of the roots.
"""
from __future__ import annotations

import os
import random
import shutil
import subprocess

import pytest

P = 2**64 - 2**32 + 1
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_03065_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "gl.cuh"
int main(int argc, char** argv)
{
    FILE* f = fopen(argv[1], "r");
    unsigned long long a, b;
    unsigned e;
    char op;
    while (fscanf(f, " %c %llu %llu %u", &op, &a, &b, &e) == 4) {
        if (op == 'p') printf("%llu\n", (unsigned long long)gl::mul_pow2(a, e));
        else printf("%llu\n", (unsigned long long)gl::reduce128(a, b));
    }
    fclose(f);
    return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("glhost")
    src = d / "t.cu"
    src.write_text(PROGRAM)
    exe = d / "t"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, "-o", str(exe), str(src)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr

    def run(ops):
        inp = d / "in.txt"
        inp.write_text("".join(f"{o} {a} {b} {e}\n" for o, a, b, e in ops))
        out = subprocess.run([str(exe), str(inp)], capture_output=True, text=True, check=True).stdout.split()
        return [int(v) for v in out]

    return run


def _samples(rng, n):
    edge = [0, 1, 2, P - 1, P - 2, 2**32 - 1, 2**32, 2**63 - 1, 2**63, P - 2**32, 2**64 - 2**33 + 1 - 2]
    return [x for x in edge if x < P] + [rng.randrange(P) for _ in range(n)]


def test_mul_pow2_all_exponents(helper):
    rng = random.Random(7)
    xs = _samples(rng, 120)
    ops = [("p", x, 0, e) for e in range(96) for x in xs]
    got = helper(ops)
    for (_, x, _, e), g in zip(ops, got):
        assert g == x * pow(2, e, P) % P, (x, e)
        assert (P - g) % P == x * pow(2, e + 96, P) % P  # the sign fold for exponents 96..191


def test_reduce128_congruent(helper):
    rng = random.Random(8)
    pairs = [(0, 0), (2**64 - 1, 2**64 - 1), (0, 2**64 - 1), (2**64 - 1, 0), (P, 0), (0, 1), (1, 2**32)]
    pairs += [(rng.getrandbits(64), rng.getrandbits(64)) for _ in range(3000)]
    got = helper([("r", lo, hi, 0) for lo, hi in pairs])
    for (lo, hi), g in zip(pairs, got):
        assert 0 <= g < 2**64
        assert g % P == (lo + (hi << 64)) % P, (lo, hi)


def test_dft_roots_are_powers_of_two():
    # 2 has order 192 mod p (2^96 = -1), so every 2^k-th root of unity with
    # 2^k | 64 is a power of 2; the generator 7's 32nd root is 2^78.
    assert pow(2, 96, P) == P - 1 and pow(2, 192, P) == 1
    w32 = pow(7, (P - 1) // 32, P)
    assert pow(2, 78, P) == w32
    assert pow(w32, 16, P) == P - 1
