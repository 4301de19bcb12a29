"""The integer float -> double widening used by the FP64 slice sum equals the C cast for
every one of the 2^32 float bit patterns it handles (normal numbers and signed zeros),
and declines exactly the subnormal, infinite and NaN patterns."""
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_15083_gb300", "csrc")

CHECK = r"""
#include <stdio.h>
#include <string.h>
#include "widen.h"
int main(void) {
    unsigned long long bad = 0, declined = 0;
    for (unsigned long long i = 0; i < (1ull << 32); i++) {
        const uint32_t u = (uint32_t)i;
        const uint32_t e = (u >> 23) & 0xFFu;
        uint64_t d;
        const int ok = tn_widen_bits(u, &d);
        const int special = e == 0xFFu || (e == 0u && (u & 0x7FFFFFu));
        if (ok == special) { bad++; continue; }
        if (!ok) { declined++; continue; }
        float f;
        memcpy(&f, &u, 4);
        const double ref = (double)f;
        uint64_t rb;
        memcpy(&rb, &ref, 8);
        if (rb != d) bad++;
    }
    printf("%llu %llu\n", bad, declined);
    return bad != 0;
}
"""


def test_widen_matches_cast_for_every_float():
    gcc = subprocess.run(["which", "gcc"], capture_output=True, text=True).stdout.strip()
    if not gcc:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "w.c"), os.path.join(d, "w")
        open(src, "w").write(CHECK)
        subprocess.run([gcc, "-O2", "-I", CSRC, src, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
        bad, declined = map(int, r.stdout.split())
        assert r.returncode == 0 and bad == 0
        # subnormals (2 x (2^23 - 1)) plus infinities and NaNs (2 x 2^23)
        assert declined == 2 * ((1 << 23) - 1) + 2 * (1 << 23)
