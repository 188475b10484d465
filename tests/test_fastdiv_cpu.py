"""Division by invariant integers (csrc/ur_fastdiv.h, used by the denoiser's elementwise
kernels) against plain integer division: every divisor up to 4096, the image and channel
sizes the network uses, powers of two and their neighbours, random 32-bit divisors, each
with the extreme, boundary (multiples of d, +-1) and random dividends.  CPU only: the header
compiles as plain C++."""
import os
import subprocess
import textwrap

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2501_05828_gb300", "csrc")


def test_div32_matches_integer_division(tmp_path):
    src = textwrap.dedent(r'''
        #include "ur_fastdiv.h"
        #include <cstdio>
        #include <cstdlib>
        #include <random>
        #include <vector>
        using namespace ur;
        static long long bad = 0, n_checked = 0;
        static void check(uint32_t n, const Div32 &q) {
            uint32_t r;
            const uint32_t v = divmod32(n, q, r);
            if (v != n / q.d || r != n % q.d) { if (bad < 5) printf("n=%u d=%u got %u %u\n", n, q.d, v, r); ++bad; }
            ++n_checked;
        }
        int main() {
            std::mt19937_64 g(7);
            std::vector<uint32_t> ds;
            for (uint32_t d = 1; d <= 4096; ++d) ds.push_back(d);
            for (uint32_t d : {3200u, 1600u, 800u, 400u, 200u, 128u, 64u, 409600u, 102400u, 25600u, 6400u})
                ds.push_back(d);
            for (int k = 0; k < 32; ++k) for (int e = -1; e <= 1; ++e) {
                const long long d = (1ll << k) + e;
                if (d >= 1 && d <= 0xffffffffll) ds.push_back((uint32_t)d);
            }
            ds.push_back(0xffffffffu);
            for (int k = 0; k < 2000; ++k) ds.push_back((uint32_t)(g() | 1u) >> (g() % 32));
            for (uint32_t d : ds) {
                if (d == 0) continue;
                const Div32 q = make_div32(d);
                for (uint32_t n : {0u, 1u, d - 1u, d, d + 1u, 0xffffffffu, 0xfffffffeu, 0x80000000u, 0x7fffffffu}) check(n, q);
                for (uint64_t k = 1; k < 64; ++k) {
                    const uint64_t n = k * (uint64_t)d;
                    if (n <= 0xffffffffull) { check((uint32_t)n, q); check((uint32_t)(n - 1), q); if (n < 0xffffffffull) check((uint32_t)(n + 1), q); }
                }
                const uint64_t top = (0xffffffffull / d) * d;
                check((uint32_t)top, q); if (top) check((uint32_t)(top - 1), q);
                for (int k = 0; k < 200; ++k) check((uint32_t)g(), q);
            }
            printf("%lld %lld\n", n_checked, bad);
            return bad != 0;
        }
    ''')
    (tmp_path / "t.cpp").write_text(src)
    exe = tmp_path / "t"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, str(tmp_path / "t.cpp"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-500:]
    checked, bad = map(int, r.stdout.split()[-2:])
    assert bad == 0 and checked > 1_000_000
