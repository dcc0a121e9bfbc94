"""The certified single-precision filter's bounds on the large smoothness
indicators, emulated on the CPU (no GPU needed).

The face kernel takes the large-stencil decisions from FP32 bounds [lo, hi]
on beta_L, computed from the exact L D L^T sum-of-squares tables in the
generated coefficient header (see csrc/teno_fast.cuh, beta_large_bounds).  A
decision is certified only if the FP64 value the exact path would compute,
and the exact value, lie inside [lo, hi].  This test emulates the kernel's
FP32 arithmetic in the same operation order (fmaf as an exact product and
sum rounded once to float32; truncating conversion of the scaled shifted
values) on random smooth, rough, step and near-constant stencils of every
width 6, 8, 10, 12, and checks both values against the bounds:
* the FP64 value from the oracle's own evaluation of the printed (or, for
  S6, derived) quadratic form;
* the exact rational value of that form on the same double inputs.
"""
from fractions import Fraction as Fr
import os
import re

import numpy as np
import pytest

import oracle

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2109_14340_gb300", "csrc",
                   "teno_coeffs.cuh")


def _f(x):
    x = x.strip().rstrip("f")
    return 0.0 if x in ("0.0", "0") else float.fromhex(x)


def _sos(L):
    text = open(HDR).read()
    w = 2 * L
    n = w - 1
    name = "TENO_SOS%d" % w
    m = re.search(r"%s_L\[%d\]\[%d\] = \{(.*?)\n\};" % (name, n, n), text, re.S)
    Lm = [[_f(x) for x in r.split(",")] for r in re.findall(r"\{([^}]*)\}", m.group(1))]
    D = [_f(x) for x in re.search(r"%s_D\[%d\] = \{(.*?)\};" % (name, n), text).group(1).split(",")]
    DC = [_f(x) for x in re.search(r"%s_DC\[%d\] = \{(.*?)\};" % (name, n), text).group(1).split(",")]
    tau2 = _f(re.search(r"#define %s_TAU2 (\S+)" % name, text).group(1))
    k0 = _f(re.search(r"#define %s_K0 (\S+)" % name, text).group(1))
    return Lm, D, DC, tau2, k0


f32 = np.float32


def fmaf(a, b, c):
    return f32(float(a) * float(b) + float(c))


def trunc_scaled(x, emax):
    """d2f_scaled: x * 2^-emax with the mantissa truncated to 24 bits; scaled
    magnitudes below 2^-100 flush to zero."""
    if x == 0.0:
        return f32(0.0)
    y = np.ldexp(x, -emax)
    if abs(y) < 2.0 ** -100:
        return f32(0.0)
    bits = np.array([y], np.float64).view(np.int64)[0]
    bits &= ~((1 << 29) - 1)
    return f32(np.array([bits], np.int64).view(np.float64)[0])


def bounds(fs, H, L, tab):
    """beta_large_bounds<H, L> on the scaled FP32 values fs (index m + H - 1)."""
    Lm, D, DC, tau2, k0 = tab
    n = 2 * L - 1
    bt, eb = f32(0.0), f32(0.0)
    for i in range(n):
        oi = L - i if i < L else L - 1 - i
        y = fs[oi + H - 1]
        for m in range(i + 1, n):
            om = L - m if m < L else L - 1 - m
            y = fmaf(Lm[m][i], fs[om + H - 1], y)
        bt = fmaf(D[i], f32(y * y), bt)
        eb = fmaf(DC[i], abs(y), eb)
    E = fmaf(tau2, eb, fmaf(bt, f32((n + 3) * f32(5.9604645e-8)), k0))
    hi = f32(f32(bt + E) * f32(1.0 + 4.0e-6))
    lo = f32(fmaf(-E, f32(1.00001), bt) * f32(1.0 - 1.0e-6))
    return float(lo), float(hi)


def stencils(W, count, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    offs = np.arange(W, dtype=float)
    out = []
    for i in range(count):
        kind = i % 5
        scale = 10.0 ** g.uniform(-6, 6)
        shift = g.uniform(-1, 1) * 10.0 ** g.uniform(-2, 4)
        if kind == 0:
            v = np.sin(g.uniform(0.01, 1.2) * offs + g.uniform(0, 6)) * scale + shift
        elif kind == 1:
            v = g.standard_normal(W) * scale + shift
        elif kind == 2:
            v = (offs >= g.integers(0, W)).astype(float) * scale + shift + 1e-3 * scale * np.sin(offs)
        elif kind == 3:
            v = shift + 1.0 + abs(shift + 1.0) * 1e-12 * g.standard_normal(W)
        else:
            v = (g.uniform(-1, 1) + g.uniform(-1, 1) * offs + 0.01 * offs ** 2) * scale + shift
        out.append(v)
    return out


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_sos_bounds_contain_fp64_and_exact_indicator(scheme):
    H = scheme // 2
    W = 2 * H
    p = oracle.params(1, [16], [1.0], scheme=scheme)
    tabs = {L: _sos(L) for L in range(3, H + 1)}
    forms = {}
    for L in range(3, H + 1):
        forms[L] = [(a, b, c) for a, b, c in oracle.beta_fractions(2 * L)]
    checked = 0
    for v in stencils(W, 600, 700 + scheme):
        s = v - v[H - 1]                              # the exact path's shifted values
        nz = [abs(x) for j, x in enumerate(s) if j != H - 1 and x != 0.0]
        if not nz:
            continue
        emax = max(int(np.frexp(x)[1]) - 1 for x in nz)
        if emax < -100 or emax > 50:
            continue
        fs = [f32(0.0) if j == H - 1 else trunc_scaled(s[j], emax) for j in range(W)]
        beta64, _ = oracle.betas(p, v)
        sc = Fr(2) ** (-2 * emax)
        for L in range(3, H + 1):
            lo, hi = bounds(fs, H, L, tabs[L])
            b64 = Fr(float(beta64[L])) * sc
            ex = sum(c * Fr(float(s[a + H - 1])) * Fr(float(s[b + H - 1]))
                     for a, b, c in forms[L]) * sc
            assert Fr(lo) <= b64 <= Fr(hi), (scheme, L, lo, float(b64), hi)
            assert Fr(lo) <= ex <= Fr(hi), (scheme, L, lo, float(ex), hi)
            checked += 1
    assert checked > 500
