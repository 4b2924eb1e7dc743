"""Host check of the integer-arithmetic conversions in csrc/f64bits.cuh (used
by the binning kernels and the force epilogue in place of the FP64-pipe
conversions): compiled as
plain C++ and compared bit for bit with the compiler's correctly rounded
conversions on random inputs over the whole exponent range, on exact ties and
on the edges of the binary32 range."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1903_10134_gb300", "csrc")

PROGRAM = r'''
#include "f64bits.cuh"
#include <cstdio>
#include <cmath>
#include <cfloat>
#include <random>
using namespace mdpd;

static int check(double x, long* conv) {
    bool ok;
    const float f = f64_to_f32_rn(x, &ok);
    if (!ok) return 0;
    ++*conv;
    const float want = (float)x;
    uint32_t a, b;
    std::memcpy(&a, &f, 4);
    std::memcpy(&b, &want, 4);
    if (a != b) { std::printf("MISMATCH %.17g %08x %08x\n", x, a, b); return 1; }
    return 0;
}

int main() {
    std::mt19937_64 rng(12345);
    long conv = 0;
    int bad = 0;
    // random bit patterns: every exponent, both signs
    for (int i = 0; i < 2000000; ++i) bad += check(bits_f64(rng()), &conv);
    // random values of moderate size (positions, velocities)
    std::uniform_real_distribution<double> u(-300.0, 300.0);
    for (int i = 0; i < 2000000; ++i) bad += check(u(rng), &conv);
    // exact ties between two binary32 neighbours, both parities, and +-1 ulp
    for (int i = 0; i < 200000; ++i) {
        uint64_t b = rng() & ~0x1FFFFFFFull;
        const uint64_t e = 897 + rng() % 254;
        b = (b & 0x800FFFFFE0000000ull) | (e << 52) | 0x10000000ull;
        bad += check(bits_f64(b), &conv);
        bad += check(bits_f64(b + 1), &conv);
        bad += check(bits_f64(b - 1), &conv);
    }
    // edges: zeros, the smallest normal binary32, rounding up to the next
    // binade and to infinity, the largest finite binary32
    const double edge[] = {0.0, -0.0, (double)FLT_MIN, -(double)FLT_MIN,
                           std::nextafter((double)FLT_MIN, 1.0), (double)FLT_MAX,
                           -(double)FLT_MAX, std::nextafter((double)FLT_MAX, 1e300),
                           std::ldexp(1.0, 128) * (1.0 - std::ldexp(1.0, -25)),
                           std::ldexp(1.0, 128) * (1.0 - std::ldexp(1.0, -26)),
                           1.0 - std::ldexp(1.0, -25), 2.0 - std::ldexp(1.0, -24),
                           0.5, 1.0, 127.99999999999, 1e-30, -1e-30};
    for (double x : edge) bad += check(x, &conv);
    // not converted: subnormal results, 2^128 and beyond, inf, NaN
    bool ok;
    const double rej[] = {1e-40, -1e-45, std::ldexp(1.0, 128), 1e300, INFINITY, -INFINITY, NAN};
    for (double x : rej) { f64_to_f32_rn(x, &ok); if (ok) { std::printf("ACCEPTED %g\n", x); ++bad; } }
    // binary32 to binary64 (exact): random bit patterns and the specials
    for (int i = 0; i < 2000000; ++i) {
        const uint32_t fb = (uint32_t)rng();
        float x;
        std::memcpy(&x, &fb, 4);
        const double d = f32_to_f64(x, &ok);
        if (!ok) continue;
        ++conv;
        if (f64_bits(d) != f64_bits((double)x)) { std::printf("F32 %08x\n", fb); ++bad; }
    }
    const float fr[] = {1e-40f, -1e-42f, INFINITY, NAN};
    for (float x : fr) { f32_to_f64(x, &ok); if (ok) { std::printf("ACCEPTED32 %g\n", x); ++bad; } }
    for (float x : {0.0f, -0.0f}) {
        const double d = f32_to_f64(x, &ok);
        if (!ok || f64_bits(d) != f64_bits((double)x)) { std::printf("ZERO\n"); ++bad; }
    }
    // order keys against the comparison operators (random values, both zeros,
    // infinities, neighbours of each other)
    for (int i = 0; i < 2000000; ++i) {
        double a = bits_f64(rng()), b2 = (i & 1) ? std::nextafter(a, (i & 2) ? 1e308 : -1e308)
                                                 : bits_f64(rng());
        if (std::isnan(a) || std::isnan(b2)) continue;
        if ((f64_key(a) < f64_key(b2)) != (a < b2) || (f64_key(a) >= f64_key(b2)) != (a >= b2)) {
            std::printf("KEY %.17g %.17g\n", a, b2); ++bad;
        }
    }
    const double kz[] = {0.0, -0.0, 1e-310, -1e-310, INFINITY, -INFINITY, 1.0, -1.0};
    for (double a : kz) for (double b2 : kz)
        if ((f64_key(a) < f64_key(b2)) != (a < b2)) { std::printf("KEYZ %g %g\n", a, b2); ++bad; }
    // integers to binary64
    for (int i = 0; i < 2000000; ++i) {
        const uint32_t q = (uint32_t)(rng() >> (rng() % 64));
        if (u32_to_f64(q) != (double)q) { std::printf("U32 %u\n", q); ++bad; }
    }
    const uint32_t qe[] = {0u, 1u, 2u, 3u, 0x7FFFFFFFu, 0x80000000u, 0xFFFFFFFFu, 16777217u};
    for (uint32_t q : qe) if (u32_to_f64(q) != (double)q) { std::printf("U32 %u\n", q); ++bad; }
    // cell offsets in binary32 arithmetic against the exact offset
    std::uniform_real_distribution<double> uh(0.7, 1.6), ulo(-150.0, 150.0), uu(-0.5, 0.5);
    double worst = 0.0;
    for (int i = 0; i < 1000000; ++i) {
        const double h = uh(rng), lo = ulo(rng);
        const int q = (int)(rng() % 300);
        const double c0 = lo + 0.5 * h;
        const double x = std::fma((double)q, h, c0) + uu(rng) * h;
        const float h_hi = (float)h, h_lo = (float)(h - (double)h_hi);
        const float c_hi = (float)c0, c_lo = (float)(c0 - (double)c_hi);
        float off;
        if (!cell_offset_f32(x, q, h_hi, h_lo, c_hi, c_lo, &off)) { ++bad; continue; }
        const long double exact = (long double)x - ((long double)c0 + (long double)q * (long double)h);
        const double ulp = std::ldexp(1.0, std::ilogb((double)std::fabs(exact) + 1e-30) - 23);
        const double errn = (double)std::fabs((long double)off - exact) / (ulp + 1e-9);
        if (errn > worst) worst = errn;
    }
    std::printf("offset worst %.3f\n", worst);
    if (worst > 1.5) ++bad;
    std::printf("converted %ld bad %d\n", conv, bad);
    return bad != 0;
}
'''


def test_integer_conversions_match_the_compiler(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "t.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "t"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC, str(src),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-2000:]
    conv = int(out.stdout.split()[-3])
    assert conv > 4_000_000          # most random binary64 patterns lie outside binary32
