"""Epsilons other than the paper's 1e-40 (Eq. scale_separation; the eta
measure of Sec. 3.4).  The certified single-precision decision filter's
error bounds carry both epsilons explicitly and are used up to 1e-40; with
larger ones the library takes every decision in FP64.  With
each epsilon pair the right-hand side and its decision record must be the
same bit for bit with the filter switch on and off, and equal to the oracle
run with the same epsilons.  The data are chosen so that 1e-6 changes many
decisions against 1e-40 (the test has teeth: a filter that ignored the
epsilons would disagree)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_14340_gb300 as T  # noqa: E402

DEV = torch.device("cuda:0")

EPS = [(1e-6, 1e-6), (1e-6, 1e-40), (1e-40, 1e-6), (1e-20, 1e-30), (0.0, 1e-40)]


def _cases():
    out = []
    for scheme in (8, 10, 12):
        out.append(("1d-riemann-s%d" % scheme, workloads.riemann_1d(137, scheme=scheme)))
        out.append(("1d-smooth-s%d" % scheme, workloads.smooth_wave_1d(96, scheme, amp=1e-3)))
    out.append(("2d-quadrants-s10", workloads.quadrants_2d(37, 29, scheme=10)))
    c = workloads.tgv_3d(12, scheme=8)
    out.append(("3d-tgv-s8", c))
    return out


CASES = _cases()


def gpu_rhs(case, eb, ee, fast):
    p = T.teno_params_init(ndim=case["ndim"], n=case["n"], dx=case["dx"], scheme=case["scheme"],
                           gamma=case["gamma"], bc_lo=case["bc_lo"], bc_hi=case["bc_hi"],
                           eps_beta=eb, eps_eta=ee)
    s = T.Solver(p)
    Ud = torch.from_numpy(np.ascontiguousarray(case["U"])).to(DEV)
    T.teno_set_decision_filter(fast)
    try:
        r, fl = s.rhs(Ud, flags=True)
    finally:
        T.teno_set_decision_filter(True)
    s.status()
    return r.cpu().numpy(), fl.cpu().numpy()


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("eps", EPS, ids=["%g-%g" % e for e in EPS])
def test_rhs_with_epsilons(name, case, eps):
    eb, ee = eps
    r_on, f_on = gpu_rhs(case, eb, ee, True)
    r_off, f_off = gpu_rhs(case, eb, ee, False)
    assert np.array_equal(f_on, f_off)
    assert np.array_equal(r_on, r_off)
    po = oracle_params(case, eps_beta=eb, eps_eta=ee)
    r_o, f_o, _, _ = oracle.rhs(po, case["U"], want_flags=True, threads=4)
    assert np.count_nonzero(f_on[:f_o.size] != f_o) == 0
    assert np.array_equal(r_on, r_o)


def test_large_epsilon_changes_decisions():
    """The smooth low-amplitude wave: eps = 1e-6 against 1e-40 changes the
    decision bytes (the C_T exponent and the selections), so the test above
    compares genuinely different outcomes."""
    case = workloads.smooth_wave_1d(96, 10, amp=1e-3)
    _, f_paper = gpu_rhs(case, 1e-40, 1e-40, True)
    _, f_big = gpu_rhs(case, 1e-6, 1e-6, True)
    n = oracle.flags_size(oracle_params(case))
    assert np.count_nonzero(f_paper[:n] != f_big[:n]) > n // 10


@pytest.mark.parametrize("scheme", [8, 10, 12])
@pytest.mark.parametrize("eps", [(1e-6, 1e-6), (1e-12, 1e-40), (0.0, 1e-40)],
                         ids=["1e-6", "1e-12", "0"])
def test_reconstruct_with_epsilons(scheme, eps):
    """teno_reconstruct on smooth, small-amplitude and near-constant stencils:
    filter on and off equal, and equal to the oracle stencil by stencil."""
    eb, ee = eps
    H = scheme // 2
    g = np.random.Generator(np.random.PCG64(911 + scheme))
    x = np.arange(-H + 1, H + 1, dtype=float)
    V = []
    for k in range(600):
        a = 10.0 ** g.uniform(-8, 1)
        V.append(1.0 + a * np.sin(g.uniform(0.1, 1.5) * x + g.uniform(0, 6.3)))
    for k in range(200):
        V.append(g.uniform(-1, 1) + 10.0 ** g.uniform(-12, -4) * g.standard_normal(2 * H))
    V.append(np.full(2 * H, 0.7))
    V = np.array(V)
    p = T.teno_params_init(scheme=scheme, eps_beta=eb, eps_eta=ee)
    v = torch.from_numpy(V).to(DEV)
    res = []
    for fast in (True, False):
        T.teno_set_decision_filter(fast)
        try:
            out = torch.empty(len(V), dtype=torch.float64, device=DEV)
            fl = torch.empty(len(V), dtype=torch.uint8, device=DEV)
            T.teno_reconstruct(p, v, out, fl)
            res.append((out.cpu().numpy(), fl.cpu().numpy()))
        finally:
            T.teno_set_decision_filter(True)
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    po = oracle.params(1, [16], [1.0], scheme=scheme, eps_beta=eb, eps_eta=ee)
    for i, vv in enumerate(V):
        val, fo = oracle.recon(po, vv)
        assert res[0][1][i] == fo, i
        assert res[0][0][i] == val or (np.isnan(val) and np.isnan(res[0][0][i])), i
