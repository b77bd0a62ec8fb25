"""The double <-> double-float conversions of the refinement residual
(csrc/dfloat.h), which use integer and FP32 operations only, checked on the
host: df_to_double equals one correctly rounded FP64 add of the widened
parts (ties included, normalised or not), df_from_double keeps 48
significant bits, special values map as documented.  Compiles a host
program with nvcc (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_09277_gb300", "csrc")

SRC = r'''
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "dfloat.h"
static unsigned long long bits(double x) { unsigned long long u; memcpy(&u, &x, 8); return u; }
int main() {
    std::mt19937_64 rng(7);
    long bad_to = 0, bad_from = 0, n_to = 0, n_from = 0;
    for (int it = 0; it < 1000000; ++it) {
        const int eh = 1 + (int)(rng() % 254);
        const unsigned uh = ((unsigned)(rng() % 2) << 31) | ((unsigned)eh << 23) | (unsigned)(rng() & 0x7fffff);
        float hi; memcpy(&hi, &uh, 4);
        const int mode = (int)(rng() % 4);  // normalised, a tie, or any pair
        int el = mode == 0 ? eh - 24 - (int)(rng() % 40) : (mode == 1 ? eh - 24 : 1 + (int)(rng() % 254));
        if (el < 1) el = 1;
        unsigned ul = ((unsigned)(rng() % 2) << 31) | ((unsigned)el << 23) | (unsigned)(rng() & 0x7fffff);
        if (mode == 1) ul = (ul & 0x80000000u) | ((unsigned)el << 23);
        float lo; memcpy(&lo, &ul, 4);
        const double want = (double)hi + (double)lo;
        if (std::isfinite(want)) {
            ++n_to;
            if (bits(want) != bits(df_to_double(dfloat(hi, lo)))) ++bad_to;
        }
        double x; unsigned long long xb = rng(); memcpy(&x, &xb, 8);
        const double ax = std::fabs(x);
        if (!std::isfinite(x) || ax < 0x1p-100 || ax >= 0x1p127) continue;
        ++n_from;
        const dfloat p = df_from_double(x);
        if (std::fabs(((double)p.hi + (double)p.lo) - x) > ax * 0x1p-47 ||
            std::fabs((double)p.lo) > std::fabs((double)p.hi) * 0x1p-23) ++bad_from;
    }
    const dfloat z = df_from_double(-0.0), inf = df_from_double(INFINITY), big = df_from_double(1e300),
                 tiny = df_from_double(1e-320), nan = df_from_double(NAN);
    const bool special = std::signbit(z.hi) && z.hi == 0.f && z.lo == 0.f && std::isinf(inf.hi) &&
                         std::isinf(big.hi) && tiny.hi == 0.f && std::isnan(nan.hi) &&
                         df_widen(1e-40f) == (double)1e-40f && df_widen(-3e-45f) == (double)-3e-45f &&
                         std::isinf(df_widen(INFINITY)) && df_to_double(dfloat(0.f, 0.f)) == 0.0;
    printf("%ld %ld %ld %ld %d\n", n_to, bad_to, n_from, bad_from, special ? 1 : 0);
    return 0;
}
'''


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_dfloat_conversions_match_fp64(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "dfcheck.cu"
    src.write_text(SRC)
    exe = tmp_path / "dfcheck"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    n_to, bad_to, n_from, bad_from, special = map(
        int, subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split())
    assert n_to > 500000 and bad_to == 0
    assert n_from > 50000 and bad_from == 0
    assert special == 1
