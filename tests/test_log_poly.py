"""Accuracy of the polynomial logarithm used by the likelihood epilogues (csrc/log_poly.h).

The header is plain C as well as CUDA; compiled here with gcc it must stay within 1 ulp of
the correctly rounded log (FP64 reference) on a sweep over e^-20 .. e^10 and around 1, and
within 3e-8 absolute for |x - 1| < 0.3, where the deviance terms c log(p / f) live.  Its
coefficients must be the ones the committed fit script produces.
"""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_17334_gb300", "csrc")

HARNESS = r"""
#include <stdio.h>
#include <stdlib.h>
#include "log_poly.h"
static double ulp_of(double ref) {
    float r = (float)fabs(ref); int i = qst_lp_bits(r);
    return (double)qst_lp_float(i + 1) - (double)r;
}
int main(int argc, char **argv) {
    long n = atol(argv[1]);
    double max_ulp = 0, max_abs_near1 = 0;
    unsigned long long s = 88172645463325252ULL;
    for (long it = 0; it < n; ++it) {
        s ^= s << 13; s ^= s >> 7; s ^= s << 17;
        float x;
        if (it & 1) x = 1.0f + ((int)(s % 2000001) - 1000000) * 3e-7f;
        else x = (float)exp(((double)(s >> 11) / 9007199254740992.0) * 30.0 - 20.0);
        double ref = log((double)x);
        float y = qst_log_poly(x);
        double u = fabs((double)y - ref) / ulp_of(ref);
        if (u > max_ulp) max_ulp = u;
        if (fabsf(x - 1.0f) < 0.3f && fabs((double)y - ref) > max_abs_near1) max_abs_near1 = fabs((double)y - ref);
    }
    printf("%.6f %.6e\n", max_ulp, max_abs_near1);
    return 0;
}
"""


def test_log_poly_within_one_ulp(tmp_path):
    src = tmp_path / "h.c"
    src.write_text(HARNESS)
    exe = tmp_path / "h"
    subprocess.run(["gcc", "-std=c99", "-O2", "-I", CSRC, str(src), "-o", str(exe), "-lm"], check=True)
    out = subprocess.run([str(exe), "4000000"], capture_output=True, text=True, check=True).stdout.split()
    max_ulp, max_abs = float(out[0]), float(out[1])
    assert max_ulp <= 1.0, max_ulp
    assert max_abs < 3e-8, max_abs


def test_log_poly_coefficients_come_from_the_fit():
    sys.path.insert(0, CSRC)
    try:
        import log_poly_fit
    finally:
        sys.path.remove(CSRC)
    c, err = log_poly_fit.fit()
    assert err < 3e-8
    text = open(os.path.join(CSRC, "log_poly.h")).read()
    body = text[text.index("float q = "):text.index("const float f2")]
    header = [float(v) for v in re.findall(r"(-?\d\.\d+)f", body)]
    assert len(header) == 9
    want = np.float32(c[::-1])                          # Horner order: highest degree first
    assert np.array_equal(np.float32(header), want)
