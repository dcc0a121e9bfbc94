"""The decision filter's host-side constants (fastk_make in
csrc/teno_fast.cuh), checked against exact rational arithmetic: every bound
rounds the right way, the exponents are the floors the exact path computes,
and the premises of the filter's outright answers (C_r <= 1, C_T <= 0.1 at
m = 0, epsilons of at least 2^-136) are set exactly when they hold.  A small
host program built with nvcc prints the constants; no GPU is needed."""
import json
import math
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2109_14340_gb300", "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

# (cr, alpha1, alpha2, eps_beta, eps_eta)
PARAMS = [
    (0.265, 14.0, 6.4, 1e-40, 1e-40),       # the paper's values
    (2.0, 14.0, 6.4, 1e-40, 1e-40),         # C_r > 1
    (0.265, 0.5, 0.2, 1e-40, 1e-40),        # C_T = 1 at m = 0
    (0.265, 14.0, 6.4, 1e-45, 1e-40),       # eps_beta below 2^-136
    (0.265, 14.0, 6.4, 1e-40, 1e-45),       # eps_eta below 2^-136
    (0.265, 10.5, 3.5, 0.0, 1e-40),         # eps_beta = 0
    (1.0, 1.0, 0.5, 2.0 ** -136, 2.0 ** -136),   # every premise at its edge
]

HARNESS = r'''
#include <cstdio>
#include "teno_fast.cuh"
int main(int argc, char **argv)
{
    (void)argc;
    double v[5];
    for (int i = 0; i < 5; i++) sscanf(argv[1 + i], "%la", &v[i]);
    const teno::FastK F = teno::fastk_make(v[0], v[1], v[2], v[3], v[4]);
    printf("{\"eb_lo\": \"%a\", \"eb_hi\": \"%a\", \"ee_hi\": \"%a\", ", (double)F.eb_lo,
           (double)F.eb_hi, (double)F.ee_hi);
    printf("\"cr_inv_lo\": \"%a\", \"cr_inv_hi\": \"%a\", ", (double)F.cr_inv_lo,
           (double)F.cr_inv_hi);
    printf("\"nexp_smooth\": %d, \"nexp_min\": %d, \"flat_ok\": %d, \"tiny_ok\": %d, ",
           F.nexp_smooth, F.nexp_min, F.flat_ok, F.tiny_ok);
    printf("\"thr\": [");
    for (int n = 0; n < 23; n++) printf("%s\"%a\"", n ? ", " : "", (double)F.thr[n]);
    printf("], \"thr_rej\": [");
    for (int n = 0; n < 23; n++) printf("%s\"%a\"", n ? ", " : "", (double)F.thr_rej[n]);
    printf("]}\n");
    return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("fastk")
    src = d / "fastk_harness.cu"
    src.write_text(HARNESS)
    exe = d / "fastk_harness"
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I" + CSRC, "-I" + INCLUDE, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("harness build failed:\n" + r.stderr)
    return str(exe)


def constants(exe, cr, a1, a2, eb, ee):
    args = [float(x).hex() for x in (cr, a1, a2, eb, ee)]
    out = subprocess.run([exe] + args, capture_output=True, text=True, check=True).stdout
    d = json.loads(out)
    for k in ("eb_lo", "eb_hi", "ee_hi", "cr_inv_lo", "cr_inv_hi"):
        d[k] = float.fromhex(d[k])
    d["thr"] = [float.fromhex(x) for x in d["thr"]]
    d["thr_rej"] = [float.fromhex(x) for x in d["thr_rej"]]
    return d


def clamp22(x):
    return 0 if x < 0 else (22 if x > 22 else x)


@pytest.mark.parametrize("prm", PARAMS, ids=[str(p) for p in PARAMS])
def test_fastk_constants(harness, prm):
    cr, a1, a2, eb, ee = prm
    F = constants(harness, *prm)
    s100 = Fr(2) ** 100
    lo_t = Fr(eb) * s100 * (1 - Fr(1, 10 ** 6))
    hi_t = Fr(eb) * s100 * (1 + Fr(1, 10 ** 6))
    # outward rounding, and tight: within a few float ulps
    assert Fr(F["eb_lo"]) <= lo_t
    assert Fr(F["eb_hi"]) >= hi_t
    assert Fr(F["ee_hi"]) >= Fr(ee) * s100
    if eb > 0:
        assert Fr(F["eb_lo"]) >= lo_t * (1 - Fr(1, 2 ** 21))
        assert Fr(F["eb_hi"]) <= hi_t * (1 + Fr(1, 2 ** 21))
    else:
        assert F["eb_lo"] == 0.0 and F["eb_hi"] == 0.0
    assert Fr(F["cr_inv_lo"]) < 1 / Fr(cr) < Fr(F["cr_inv_hi"])
    # the exponents the exact path computes at m = 0 and at g = 0
    ns = clamp22(math.floor(a1 - a2 * (1.0 - 1.0)))
    nm = clamp22(math.floor(a1 - a2 * (1.0 - 0.0)))
    assert F["nexp_smooth"] == ns and F["nexp_min"] == nm
    # premises of the outright answers
    flat = cr <= 1.0 and ns >= 1
    tiny = flat and eb >= 2.0 ** -136 and ee >= 2.0 ** -136
    assert F["flat_ok"] == int(flat) and F["tiny_ok"] == int(tiny)
    # thresholds: thr[n] <= 1/(10^-n (1 + 2^-16)) - 1 <= thr_rej-side bound
    for n in range(23):
        acc = 1 / (Fr(1, 10 ** n) * (1 + Fr(1, 2 ** 16))) - 1
        rej = 1 / (Fr(1, 10 ** n) * (1 - Fr(1, 2 ** 16))) - 1
        assert Fr(F["thr"][n]) <= acc
        assert Fr(F["thr_rej"][n]) >= rej
