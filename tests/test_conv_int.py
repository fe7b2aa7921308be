"""The integer-pipe FP64 <-> FP32 conversions (esmm_conv.h) against the
compiler's own casts on the host (IEEE 754: narrowing rounds to nearest,
ties to even; widening is exact), bit for bit:

  * narrowing: random bit patterns over every exponent, random doubles in
    the float range, exact halfway cases between neighbouring floats (ties
    to even both ways) and their neighbours one double ulp away, the ends
    of the normal range (rounding up into FLT_MIN, up to infinity past
    FLT_MAX), zeros, infinities and NaNs;
  * widening: every float of a stride through all 2^32 patterns, plus the
    special values.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR_DIR = os.path.join(ROOT, "paper_2107_12027_gb300", "csrc")

SRC = r"""
#include <stdio.h>
#include <math.h>
#include <float.h>
#include "esmm_conv.h"
using namespace esmm;

static uint64_t s = 0x9e3779b97f4a7c15ull;
static uint64_t next() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }

static long bad = 0, n = 0;
static void check_d(double x) {
    float a = d2f_int(x), b = (float)x;
    ++n;
    if (conv_bits32(a) != conv_bits32(b) && !(isnan(a) && isnan(b))) {
        if (bad < 5) printf("narrow %.17g: %a vs %a\n", x, a, b);
        ++bad;
    }
}
static void check_f(float x) {
    double a = f2d_int(x), b = (double)x;
    ++n;
    if (conv_bits64(a) != conv_bits64(b) && !(isnan(a) && isnan(b))) {
        if (bad < 5) printf("widen %a\n", x);
        ++bad;
    }
}
int main() {
    for (long k = 0; k < 20000000; ++k) check_d(conv_double(next()));
    for (long k = 0; k < 20000000; ++k) {
        // a random float-range double: exponent within the float range +- 2
        uint64_t b = next();
        uint64_t e = 895 + (b >> 52) % 260;
        check_d(conv_double((b & 0x800fffffffffffffull) | (e << 52)));
    }
    for (long k = 0; k < 5000000; ++k) {
        // halfway between a float f and its successor, and one double ulp either side
        uint32_t u = (uint32_t)next() & 0x7f7fffffu;
        float f = conv_float(u), g = nextafterf(f, INFINITY);
        if (!isfinite(g)) continue;
        double mid = 0.5 * ((double)f + (double)g);
        check_d(mid); check_d(-mid);
        check_d(nextafter(mid, INFINITY)); check_d(nextafter(mid, -INFINITY));
    }
    const double edge[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, FLT_MAX, -FLT_MAX, FLT_MIN, -FLT_MIN,
                           (double)FLT_MAX * (1.0 + 0x1p-24), (double)FLT_MAX * (1.0 + 0x1p-25),
                           nextafter((double)FLT_MAX * (1.0 + 0x1p-24), 0.0), (double)FLT_MIN * (1.0 - 0x1p-25),
                           (double)FLT_MIN * (1.0 - 0x1p-24), 0x1p-149, 0x1p-150, 0x1.8p-150, 1e-300, 1e300,
                           DBL_MIN, DBL_MAX, 1.0, -1.0, 0.1, 1.0 / 3.0};
    for (double x : edge) { check_d(x); check_d(-x); }
    for (uint64_t u = 0; u < 0x100000000ull; u += 97) check_f(conv_float((uint32_t)u));
    const float fedge[] = {0.0f, -0.0f, INFINITY, -INFINITY, NAN, FLT_MAX, FLT_MIN, 0x1p-149f, 1.0f};
    for (float x : fedge) { check_f(x); check_f(-x); }
    printf("%ld checked, %ld wrong\n", n, bad);
    return bad != 0;
}
"""


def test_integer_conversions_equal_the_ieee_casts(tmp_path):
    src = tmp_path / "conv.cpp"
    exe = tmp_path / "conv"
    src.write_text(SRC)
    # -ffloat-store style issues do not arise on these targets; -O2 keeps the run short
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", HDR_DIR, "-o", str(exe), str(src), "-lm"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 wrong" in r.stdout
