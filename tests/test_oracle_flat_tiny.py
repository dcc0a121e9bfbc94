"""Two facts about the method that the decision filter answers without
evaluating it, checked on the oracle (the plain FP64 evaluation of Sec.
3.2-3.4): a stencil of bit-identical values, and one whose values all differ
from the upwind cell's by less than 2^-100 (so all lie below 2^-46 in size),
select S_p with the C_T exponent of m = 0, provided C_r <= 1, C_T <= 0.1 at
m = 0 and both epsilons are at least 2^-136 (the paper's values satisfy all
three).  Families: constants over the whole double range, tiny values with
differences of one or a few ulps, tiny values straddling zero, values just
inside the 2^-100 bound, and the same with the epsilons at 2^-136."""
import numpy as np
import pytest

import oracle


def smooth_flag(po, H):
    """Decision byte of S_p with the exponent at m = 0 (the exact path's
    [beta] at g = 1)."""
    bct = po.alpha1 - po.alpha2 * (1.0 - 1.0)
    n = min(max(int(np.floor(bct)), 0), 22)
    large = 0 if H == 6 else H - 2
    return large | (((n - 7) & 7) << 5)


def constant_stencils(W, g, count=400):
    out = [np.zeros(W), np.full(W, -0.0), np.full(W, 5e-324), np.full(W, -2.2e-308)]
    for _ in range(count):
        out.append(np.full(W, g.choice([-1.0, 1.0]) * 10.0 ** g.uniform(-300, 300)))
    return out


def tiny_stencils(W, H, g, count=1500):
    out = []
    while len(out) < count:
        kind = len(out) % 4
        if kind == 0:       # one-ulp steps at a magnitude whose ulp is below 2^-100
            v0 = g.choice([-1.0, 1.0]) * 2.0 ** g.uniform(-200, -49)
            v = v0 + g.integers(-1, 2, W) * np.spacing(v0)
        elif kind == 1:     # random tiny values
            v = g.standard_normal(W) * 2.0 ** g.uniform(-300, -104)
        elif kind == 2:     # straddling zero
            v = g.integers(-3, 4, W) * 2.0 ** g.uniform(-160, -103)
        else:               # differences just inside the bound
            v0 = 2.0 ** g.uniform(-120, -50)
            v = v0 + g.uniform(-1, 1, W) * 2.0 ** -101
        s = v - v[H - 1]
        if np.all(s == 0) or np.max(np.abs(s)) >= 2.0 ** -100:
            continue
        out.append(v)
    return out


@pytest.mark.parametrize("scheme", [8, 10, 12])
@pytest.mark.parametrize("eps", [None, 2.0 ** -136], ids=["paper", "eps_2^-136"])
def test_flat_and_tiny_stencils_select_smooth_sp(scheme, eps):
    H, W = scheme // 2, scheme
    kw = {} if eps is None else {"eps_beta": eps, "eps_eta": eps}
    po = oracle.params(1, [16], [1.0], scheme=scheme, **kw)
    want = smooth_flag(po, H)
    g = np.random.Generator(np.random.PCG64(31 + scheme))
    for name, fam in (("constant", constant_stencils(W, g)), ("tiny", tiny_stencils(W, H, g))):
        bad = []
        for v in fam:
            _, fl = oracle.recon(po, v)
            if fl != want:
                bad.append((v, fl))
        assert not bad, (name, len(bad), bad[:3], want)


def test_empty_fallback_is_nan():
    """Reading of Eq. renormalize when every small-stencil cut-off fails,
    possible only for C_T = 1 ([beta] = 0): the weights are 0/0, so the
    oracle's value is NaN exactly for the fallbacks that keep no stencil,
    and a number for every other outcome."""
    po = oracle.params(1, [16], [1.0], scheme=10, alpha1=0.5, alpha2=0.2)
    g = np.random.Generator(np.random.PCG64(41))
    empty = kept = 0
    for i in range(3000):
        v = g.standard_normal(10) * 10.0 ** g.uniform(-3, 3) + g.uniform(-5, 5)
        val, fl = oracle.recon(po, v)
        sel, mask = fl & 3, (fl >> 2) & 7
        if sel == 0 and mask == 0:
            assert np.isnan(val)
            empty += 1
        else:
            assert np.isfinite(val)
            kept += 1
    assert empty > 1000 and kept >= 10
