"""The CUDA library's generated coefficient header against the oracle (CPU).

The twelve-point candidate S6 is derived twice, independently: by the oracle
(oracle/teno12_derive.py: primitive-function interpolation for beta_{6,12},
numerical quadrature for the optimisation of Sec. 4.1) and by the CUDA
side's generator (csrc/gen_coeffs.py: moment-matrix inversion, closed-form
integrals).  Both must round to the same doubles.  The printed tables must
match too, and the committed header must be what the generator writes."""
import os
import re

import pytest

import oracle

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2109_14340_gb300", "csrc",
                   "teno_coeffs.cuh")


def _num(x):
    x = x.strip().rstrip("f")
    return 0.0 if x in ("0.0", "0") else float.fromhex(x)


def _table(text, name, w):
    m = re.search(r"%s\[%d\]\[%d\] = \{(.*?)\n\};" % (name, w, w), text, re.S)
    rows = re.findall(r"\{([^}]*)\}", m.group(1))
    return [[_num(x) for x in r.split(",")] for r in rows]


@pytest.mark.parametrize("w", [6, 8, 10, 12])
def test_indicator_tables_equal_oracle(w):
    text = open(HDR).read()
    Q = _table(text, "TENO_Q%d" % w, w)
    lo = -w // 2 + 1
    for r in range(w):
        for c in range(w):
            want = oracle.beta_coef(w, r + lo, c + lo) if c >= r else 0.0
            assert Q[r][c] == want, (w, r, c)


def test_s6_linear_scheme_equals_oracle():
    text = open(HDR).read()
    m = re.search(r"TENO_LIN6\[12\] = \{\s*(.*?)\};", text, re.S)
    lin = [_num(x) for x in m.group(1).split(",") if x.strip()]
    assert lin == [oracle.lin_coef(6, k) for k in range(-5, 7)]


def test_header_is_generated():
    pytest.importorskip("mpmath")
    pytest.importorskip("numpy")
    import importlib.util
    path = os.path.join(os.path.dirname(HDR), "gen_coeffs.py")
    spec = importlib.util.spec_from_file_location("gen_coeffs", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert open(HDR).read() == gen.emit() + "\n"
