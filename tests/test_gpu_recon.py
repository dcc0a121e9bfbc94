"""The GPU's scalar TENO-AA reconstruction (teno_reconstruct) against the
oracle, stencil by stencil, with the certified single-precision decision
filter on and off.  Besides random smooth / rough / near-constant /
degenerate data, the stencils include adversarial families placed on the
decision thresholds by bisection with the oracle: chi_p = C_T (Eq. cutoff),
eta = C_r (Eq. m_definition) and every integer boundary of [beta] in Eq.
CT_definition, each probed at the neighbouring doubles.  Values must agree
bitwise and the decision bytes exactly."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_14340_gb300 as T  # noqa: E402

DEV = torch.device("cuda:0")


def oracle_batch(scheme, V, **kw):
    p = oracle.params(1, [16], [1.0], scheme=scheme, **kw)
    out = np.empty(len(V))
    fl = np.empty(len(V), np.uint8)
    for i, v in enumerate(V):
        out[i], fl[i] = oracle.recon(p, v)
    return out, fl


def gpu_batch(scheme, V, fast, with_flags=True, **kw):
    """Values and decision bytes (None without a record: the filter may then
    accept S_p for every C_T the parameters allow without the eta measure).
    kw: teno_params fields."""
    p = T.teno_params_init(scheme=scheme, **kw)
    T.teno_set_decision_filter(fast)
    try:
        v = torch.from_numpy(np.ascontiguousarray(V)).to(DEV)
        out = torch.empty(len(V), dtype=torch.float64, device=DEV)
        fl = torch.empty(len(V), dtype=torch.uint8, device=DEV) if with_flags else None
        T.teno_reconstruct(p, v, out, fl)
        return out.cpu().numpy(), (fl.cpu().numpy() if with_flags else None)
    finally:
        T.teno_set_decision_filter(True)


def differ(a, b):
    """Mask of values that differ bit for bit, two NaNs counting as equal
    (their payloads are the host's and the device's; the empty fallback of
    C_T = 1 is 0/0)."""
    return (a.view(np.int64) != b.view(np.int64)) & ~(np.isnan(a) & np.isnan(b))


def neighbours(x, k=3):
    out = [x]
    lo = hi = x
    for _ in range(k):
        lo = np.nextafter(lo, -np.inf)
        hi = np.nextafter(hi, np.inf)
        out += [lo, hi]
    return out


def bisect(make, a, b, key, iters=200):
    """Boundary of key(oracle(make(x))) between a and b (key differs there)."""
    p = None
    ka = key(make(a))
    kb = key(make(b))
    if ka == kb:
        return None
    for _ in range(iters):
        m = 0.5 * (a + b)
        if m == a or m == b:
            break
        if key(make(m)) == ka:
            a = m
        else:
            b = m
    return a, b


def adversarial(scheme):
    H = scheme // 2
    offs = np.arange(-H + 1, H + 1, dtype=float)
    po = oracle.params(1, [16], [1.0], scheme=scheme)
    key_sel = lambda v: oracle.decode_flag(oracle.recon(po, v)[1])[0]
    key_ct = lambda v: (oracle.recon(po, v)[1] >> 5) & 7
    out = []
    # chi_p = C_T: a step at the largest stencil's edge, C_T = 1e-14 region
    for base_scale in (1.0, 1e-3, 1e4):
        def make(lam, bs=base_scale):
            return bs * (np.sin(0.3 * offs) + 2.0 + lam * (offs >= H))
        r = bisect(make, 0.0, 10.0, key_sel)
        if r:
            for x in neighbours(r[0]) + neighbours(r[1]):
                out.append(make(x))
    # eta = C_r and every [beta] boundary: slope change at the upwind cell
    def make_t(t):
        d = np.where(offs < 0, 1.0, t)
        return np.concatenate([[0.0], np.cumsum(d[1:])]) + 5.0
    ts = np.linspace(1e-4, 1.0, 400)
    cts = [key_ct(make_t(t)) for t in ts]
    for i in range(1, len(ts)):
        if cts[i] != cts[i - 1]:
            r = bisect(make_t, ts[i - 1], ts[i], key_ct)
            if r:
                for x in neighbours(r[0]) + neighbours(r[1]):
                    out.append(make_t(x))
    # chi_p = C_T with C_T in the adaptive (non-smooth) range
    for t0 in (0.05, 0.1, 0.2):
        def make2(lam, t0=t0):
            return make_t(t0) + lam * (offs >= H)
        r = bisect(make2, 0.0, 50.0, key_sel)
        if r:
            for x in neighbours(r[0]) + neighbours(r[1]):
                out.append(make2(x))
    # every decision bit (which large stencil, the small-stencil cut-offs of
    # the fallback, the exponent): steps and kinks at each stencil position
    # scanned in amplitude, each change of the decision byte bisected
    key_all = lambda v: oracle.recon(po, v)[1]
    base = np.sin(0.4 * offs) + 3.0
    for q in offs[1:]:
        fams = (lambda t, q=q: base + t * (offs >= q),
                lambda t, q=q: base + t * np.maximum(offs - q + 1, 0.0))
        for make3 in fams:
            ts = np.concatenate([[0.0], np.geomspace(1e-4, 50.0, 48)])
            ks = [key_all(make3(t)) for t in ts]
            for i in range(1, len(ts)):
                if ks[i] != ks[i - 1]:
                    r = bisect(make3, ts[i - 1], ts[i], key_all)
                    if r:
                        for x in neighbours(r[0], 2) + neighbours(r[1], 2):
                            out.append(make3(x))
    return np.array(out)


def random_stencils(scheme, n=20000, seed=7):
    g = np.random.Generator(np.random.PCG64(seed))
    W = scheme
    offs = np.arange(W, dtype=float)
    V = []
    for i in range(n):
        kind = i % 8
        scale = 10.0 ** g.uniform(-8, 8)
        shift = g.uniform(-1, 1) * 10.0 ** g.uniform(-2, 6)
        if kind == 0:      # smooth
            v = np.sin(g.uniform(0.01, 1.2) * offs + g.uniform(0, 6)) * scale + shift
        elif kind == 1:    # rough
            v = g.standard_normal(W) * scale + shift
        elif kind == 2:    # step somewhere
            v = (offs >= g.integers(0, W)).astype(float) * scale + shift + 1e-3 * scale * np.sin(offs)
        elif kind == 3:    # near-constant: rounding-level variation
            v = shift + 1.0 + np.abs(shift) * 1e-15 * g.standard_normal(W)
        elif kind == 6:    # magnitudes where 1/(beta+eps)^7 leaves the double range
            v = g.standard_normal(W) * 10.0 ** g.uniform(20, 80) + shift
        elif kind == 7:    # tiny values: indicators near eps
            v = g.standard_normal(W) * 10.0 ** g.uniform(-80, -15)
        elif kind == 4:    # ghost-like: constant run then smooth
            k = g.integers(1, W)
            v = np.sin(0.2 * offs) * scale + shift
            v[:k] = v[k]
        else:              # polynomial (smooth, exact linear recovery)
            v = (g.uniform(-1, 1) + g.uniform(-1, 1) * offs + g.uniform(-0.1, 0.1) * offs ** 2) * scale
        V.append(v)
    V.append(np.zeros(W))
    V.append(np.full(W, 3.5))
    return np.array(V)


def noise_stencils(scheme, n=6000, seed=11):
    """Values that agree to within rounding, as in a plateau that rounding
    noise has reached: O(1) values a few ulps apart (around powers of two
    too, where the exact path's own rounding changes binade), the LLF
    split's near-cancelling side (tiny values of either sign), and plateaus
    exactly constant on part of the stencil (small indicators exactly 0)."""
    g = np.random.Generator(np.random.PCG64(seed))
    W = scheme
    V = []
    for i in range(n):
        kind = i % 6
        if kind in (0, 1):     # O(1) values, offsets of a few ulps
            v0 = g.choice([-1.0, 1.0]) * 10.0 ** g.uniform(-6, 6)
            if kind == 1:      # just below / above a power of two
                v0 = np.ldexp(1.0, int(g.integers(-20, 20))) * (1.0 + g.choice([-1, 1]) * 2.0 ** -50)
            k = g.integers(-3, 4, W).astype(float)
            v = v0 + k * np.spacing(v0)
        elif kind == 2:        # tiny values of either sign
            v = g.standard_normal(W) * 10.0 ** g.uniform(-30, -8)
        elif kind == 3:        # tiny multiples of one ulp-sized unit
            v = g.integers(-4, 5, W).astype(float) * 10.0 ** g.uniform(-24, -12)
        elif kind == 4:        # exactly constant run, then a few ulps of noise
            v0 = 10.0 ** g.uniform(-3, 3)
            v = np.full(W, v0)
            j = g.integers(1, W)
            v[j:] += g.integers(-2, 3, W - j) * np.spacing(v0)
        else:                  # noise about a value with a large-ish exponent spread
            v0 = 10.0 ** g.uniform(-2, 2)
            v = v0 * (1.0 + g.standard_normal(W) * 10.0 ** g.uniform(-15, -9))
        V.append(v)
    return np.array(V)


def tiny_stencils(scheme, n=3000, seed=13):
    """Stencils whose differences all lie below 2^-100 (values below 2^-46),
    bit-identical stencils of every size, and differences in the subnormal
    range."""
    g = np.random.Generator(np.random.PCG64(seed))
    W = scheme
    V = []
    for i in range(n):
        kind = i % 4
        if kind == 0:
            v = g.standard_normal(W) * 10.0 ** g.uniform(-60, -31)
        elif kind == 1:
            v0 = g.choice([-1.0, 1.0]) * 10.0 ** g.uniform(-45, -20)
            v = v0 + g.integers(-3, 4, W) * np.spacing(v0)
        elif kind == 2:
            v = np.full(W, g.uniform(-1, 1) * 10.0 ** g.uniform(-300, 300))
        else:
            v = g.integers(-3, 4, W) * 5e-324 * float(g.integers(1, 1000))
        V.append(v)
    return np.array(V)


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_reconstruction_matches_oracle(scheme):
    V = np.concatenate([random_stencils(scheme), adversarial(scheme), noise_stencils(scheme),
                        tiny_stencils(scheme)])
    ref, rfl = oracle_batch(scheme, V)
    for fast in (True, False):
        out, fl = gpu_batch(scheme, V, fast)
        bad = np.nonzero((fl != rfl) | (differ(out, ref)))[0]
        assert bad.size == 0, (fast, bad[:10], fl[bad[:5]], rfl[bad[:5]])
        out, _ = gpu_batch(scheme, V, fast, with_flags=False)
        bad = np.nonzero(differ(out, ref))[0]
        assert bad.size == 0, (fast, "no record", bad[:10])


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_adversarial_families_reach_both_sides(scheme):
    """The bisected families really straddle thresholds (both outcomes)."""
    V = adversarial(scheme)
    _, rfl = oracle_batch(scheme, V)
    assert len(V) > 50
    dec = [oracle.decode_flag(int(f)) for f in rfl]
    sels = {d[0] for d in dec}
    assert len(sels) >= 2
    assert len(set(((rfl >> 5) & 7).tolist())) >= 5
    # every large stencil S3 .. S_H, and fallbacks with different cut-offs
    assert set(range(3, scheme // 2 + 1)) <= sels
    assert len({d[1] for d in dec if d[0] == 0}) >= 3


# (GPU field names, oracle names): C_r > 1 (eta = 1 no longer gives m = 0),
# C_T = 1 at m = 0 (chi_p = 1/4 rejects S_p), and epsilons below 2^-136
# (the tiny-difference answer no longer certain).
PARAM_SETS = [
    (dict(ct_cr=2.0), dict(cr=2.0)),
    (dict(ct_alpha1=0.5, ct_alpha2=0.2), dict(alpha1=0.5, alpha2=0.2)),
    (dict(eps_beta=1e-45, eps_eta=1e-45), dict(eps_beta=1e-45, eps_eta=1e-45)),
]


@pytest.mark.parametrize("scheme", [8, 10])
@pytest.mark.parametrize("ps", range(len(PARAM_SETS)))
def test_flat_and_tiny_cases_other_parameters(scheme, ps):
    """The filter's answers for bit-identical and tiny-difference stencils
    (S_p with the smooth exponent) rest on C_r <= 1, C_T <= 0.1 at m = 0 and
    epsilons of at least 2^-136; with parameters that break one of them the
    results must still be the oracle's, bitwise."""
    gk, ok = PARAM_SETS[ps]
    V = np.concatenate([tiny_stencils(scheme, 1200, seed=17), noise_stencils(scheme, 1200, seed=19),
                        random_stencils(scheme, 1200, seed=23)])
    ref, rfl = oracle_batch(scheme, V, **ok)
    for fast in (True, False):
        out, fl = gpu_batch(scheme, V, fast, **gk)
        bad = np.nonzero((fl != rfl) | (differ(out, ref)))[0]
        assert bad.size == 0, (fast, bad[:10], fl[bad[:5]], rfl[bad[:5]])
        out, _ = gpu_batch(scheme, V, fast, with_flags=False, **gk)
        bad = np.nonzero(differ(out, ref))[0]
        assert bad.size == 0, (fast, "no record", bad[:10])
