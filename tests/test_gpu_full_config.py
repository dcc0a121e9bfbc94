"""GPU vs CPU-oracle parity at the full sizes the benchmark and the workload
definitions use, through the C ABI, in the launch configuration the
benchmark times:

  * 3D 256^3 periodic Taylor-Green + k^-5/3 field, TENO8-AA and TENO10-AA:
    the CFL time step and one whole SSP-RK3 step (every cell, every
    variable), and one right-hand side with its complete decision record;
  * 2D 1024^2 four-quadrant problem, TENO10-AA: 20 CFL steps, the state
    compared after every step;
  * the batched workload at its full size: 4096 problems, N ~ U{64..4096},
    TENO8|10 50/50, 10 % near vacuum with the limiter, one autotuned
    graph-mode step, every problem against the oracle's own step;
  * the same 3D field at 64^3 for its 100 steps and the 2D problem at
    256^2 for its 200 steps, compared at the final time.

Tolerances (the method's accuracy contract, Sec. 5 Eq. Runge-kutta): 1e-12
relative per variable for one RK3 step or one right-hand side, 1e-10
relative L-infinity at the final time (asserted over every cell, smooth
regions included), decision bytes identical.  Both sides evaluate every
expression in the same order with the same fused operations, so every case
is also asserted bit for bit and the number of differing values or bytes is
reported."""
import os
from concurrent.futures import ThreadPoolExecutor

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
THREADS = max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
              else (os.cpu_count() or 1))


def gpu_params(case, **over):
    kw = dict(ndim=case["ndim"], n=case["n"], dx=case["dx"], scheme=case["scheme"],
              gamma=case["gamma"], bc_lo=case["bc_lo"], bc_hi=case["bc_hi"],
              limiter=case.get("limiter", 0))
    kw.update(over)
    return T.teno_params_init(**kw)


def rel_err(a, b):
    """Largest |a - b| per conserved variable over that variable's max |b|."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return float((np.abs(a - b).max(axis=1) / scale).max())


def differing(a, b):
    """Number of values that differ (equal values and NaN pairs agree)."""
    a, b = np.asarray(a), np.asarray(b)
    return int(np.count_nonzero(~((a == b) | (np.isnan(a) & np.isnan(b)))))


@pytest.mark.parametrize("scheme", [8, 10])
def test_full_3d_cfl_and_rk3_step(scheme):
    """256^3: dt from teno_cfl_dt (kept on the device, as the benchmark step
    uses it) and one teno_rk3_step, against oracle.cfl_dt + oracle.rk3_step."""
    c = workloads.tgv_3d(256, scheme=scheme)
    pg, po = gpu_params(c), oracle_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(c["U"]).to(DEV)
    dt_d = s.cfl_dt(Ud, 0.4)
    s.step(Ud)                                       # dt read from the device scalar
    assert s.status() == 0
    dt_o, _, nb_dt = oracle.cfl_dt(po, c["U"], 0.4)
    assert nb_dt == 0
    assert float(dt_d.item()) == dt_o
    U1_o, nb = oracle.rk3_step(po, c["U"], dt_o, threads=THREADS)
    assert nb == 0
    U1_g = Ud.cpu().numpy()
    del Ud, s
    err = rel_err(U1_g, U1_o)
    nd = differing(U1_g, U1_o)
    assert err <= 1e-12, "relative error %.3g" % err
    assert nd == 0, "%d of %d values differ (max rel %.3g)" % (nd, U1_o.size, err)


@pytest.mark.parametrize("scheme", [8, 10])
def test_full_3d_rhs_decision_record(scheme):
    """256^3: one right-hand side with the whole decision record (16.8 M faces
    per direction x 5 fields x 2 signs) against the oracle's record."""
    c = workloads.tgv_3d(256, scheme=scheme)
    pg, po = gpu_params(c), oracle_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(c["U"]).to(DEV)
    r, fl = s.rhs(Ud, flags=True)
    assert s.status() == 0
    r_g = r.cpu().numpy()
    f_g = fl.cpu().numpy()
    del r, fl, Ud, s
    r_o, f_o, _, nb = oracle.rhs(po, c["U"], want_flags=True, threads=THREADS)
    assert nb == 0
    mism = int(np.count_nonzero(f_g[:f_o.size] != f_o))
    assert mism == 0, "decision bytes differ at %d of %d" % (mism, f_o.size)
    err = rel_err(r_g, r_o)
    assert err <= 1e-12
    assert differing(r_g, r_o) == 0, "max rel %.3g" % err


def test_full_2d_twenty_steps():
    """1024^2 four quadrants + entropy wave, TENO10-AA, transmissive: 20 steps
    of CFL dt + SSP-RK3, the dt and the state compared after every step."""
    c = workloads.quadrants_2d(1024, scheme=10)
    pg, po = gpu_params(c), oracle_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(c["U"]).to(DEV)
    Uo = c["U"].copy()
    worst = 0.0
    for k in range(20):
        dt_g = float(s.cfl_dt(Ud, 0.4).item())
        s.step(Ud)
        dt_o, _, _ = oracle.cfl_dt(po, Uo, 0.4)
        assert dt_g == dt_o, "step %d: dt %r vs %r" % (k, dt_g, dt_o)
        Uo, nb = oracle.rk3_step(po, Uo, dt_o, threads=THREADS)
        assert nb == 0
        Ug = Ud.cpu().numpy()
        err = rel_err(Ug, Uo)
        worst = max(worst, err)
        assert err <= 1e-12, "step %d: relative error %.3g" % (k, err)
        nd = differing(Ug, Uo)
        assert nd == 0, "step %d: %d values differ (max rel %.3g)" % (k, nd, err)
    assert s.status() == 0
    assert worst <= 1e-10


def _pack(cases):
    sizes = [c["n"][0] for c in cases]
    offs, total = T.pack_offsets(sizes)
    U = np.zeros(total)
    probs = []
    for c, o in zip(cases, offs):
        n = c["n"][0]
        U[o:o + 3 * n] = c["U"].ravel()
        probs.append(dict(n=n, offset=o, dx=c["dx"][0], scheme=c["scheme"],
                          limiter=c.get("limiter", 0), bc_lo=c["bc_lo"][0], bc_hi=c["bc_hi"][0]))
    return probs, U, offs


def _oracle_step(c):
    po = oracle_params(c)
    dt, _, _ = oracle.cfl_dt(po, c["U"], 0.4)
    U1, nb = oracle.rk3_step(po, c["U"], dt, threads=1)
    return U1, dt, nb


def test_full_batched_step():
    """The batched workload at full size (4096 problems, 8.6 M cells), one
    graph-mode step with the autotuned configuration the benchmark uses;
    every problem against the oracle's CFL dt and RK3 step on that problem
    alone.  The oracle runs one problem per host thread (the C calls release
    the interpreter lock)."""
    cases = workloads.batched_1d()
    assert len(cases) == 4096 and max(c["n"][0] for c in cases) > 4000
    assert sum(c.get("limiter", 0) for c in cases) > 300
    probs, U, offs = _pack(cases)
    B = T.Batch(T.teno_params_init(gamma=1.4), probs)
    scratch = torch.from_numpy(U.copy()).to(DEV)
    B.autotune(scratch)
    del scratch
    Ud = torch.from_numpy(U.copy()).to(DEV)
    B.steps(Ud, 1, 0.4, T.TENO_BATCH_GRAPH)
    Ug = Ud.cpu().numpy()
    with ThreadPoolExecutor(THREADS) as ex:
        res = list(ex.map(_oracle_step, cases))
    bad = []
    for k, (c, o, (Uo, dt_o, nb)) in enumerate(zip(cases, offs, res)):
        n = c["n"][0]
        Ugk = Ug[o:o + 3 * n].reshape(3, n)
        if differing(Ugk, Uo) or rel_err(Ugk, Uo) > 1e-12:
            bad.append(k)
    assert not bad, "%d of %d problems differ (first %s)" % (len(bad), len(cases), bad[:8])


def test_final_time_3d_100_steps():
    """The 3D field at 64^3 (same generator and spectrum cut-off), TENO10-AA,
    its 100 CFL steps, compared at the final time."""
    c = workloads.tgv_3d(64, scheme=10)
    pg, po = gpu_params(c), oracle_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(c["U"]).to(DEV)
    Uo = c["U"].copy()
    for k in range(100):
        dt_g = float(s.cfl_dt(Ud, 0.4).item())
        s.step(Ud)
        dt_o, _, _ = oracle.cfl_dt(po, Uo, 0.4)
        assert dt_g == dt_o, k
        Uo, _ = oracle.rk3_step(po, Uo, dt_o, threads=THREADS)
    assert s.status() == 0
    Ug = Ud.cpu().numpy()
    err = rel_err(Ug, Uo)
    assert err <= 1e-10, "final-time relative L-inf %.3g" % err
    assert differing(Ug, Uo) == 0


def test_final_time_2d_200_steps():
    """The four-quadrant problem at 256^2, TENO10-AA, its 200 CFL steps,
    compared at the final time."""
    c = workloads.quadrants_2d(256, scheme=10)
    pg, po = gpu_params(c), oracle_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(c["U"]).to(DEV)
    Uo = c["U"].copy()
    for k in range(200):
        dt_g = float(s.cfl_dt(Ud, 0.4).item())
        s.step(Ud)
        dt_o, _, _ = oracle.cfl_dt(po, Uo, 0.4)
        assert dt_g == dt_o, k
        Uo, _ = oracle.rk3_step(po, Uo, dt_o, threads=THREADS)
    assert s.status() == 0
    Ug = Ud.cpu().numpy()
    err = rel_err(Ug, Uo)
    assert err <= 1e-10, "final-time relative L-inf %.3g" % err
    assert differing(Ug, Uo) == 0


# --------------------------------------------------------------------------
# the certified single-precision decision filter at full size
# --------------------------------------------------------------------------

def _rhs_both_ways(s, Ud):
    """RHS and record with the filter on and off; the RHS without a record
    (where the filter may accept S_p without the C_T exponent) must equal
    them both ways too."""
    r_on, f_on = s.rhs(Ud, flags=True)
    assert torch.equal(s.rhs(Ud), r_on)
    T.teno_set_decision_filter(False)
    try:
        r_off, f_off = s.rhs(Ud, flags=True)
        assert torch.equal(s.rhs(Ud), r_off)
    finally:
        T.teno_set_decision_filter(True)
    return r_on, f_on, r_off, f_off


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_filter_whole_record_3d_256(scheme):
    """256^3, on the initial state and after three steps: the right-hand side
    and the whole decision record (decision bytes and splitting-speed argmax
    words of every face) with the filter on equal those with every decision
    taken in FP64."""
    c = workloads.tgv_3d(256, scheme=scheme)
    s = T.Solver(gpu_params(c))
    Ud = torch.from_numpy(c["U"]).to(DEV)
    for k in range(2):
        r_on, f_on, r_off, f_off = _rhs_both_ways(s, Ud)
        assert f_on.numel() == T.teno_flags_bytes(s.p)
        nmis = int((f_on != f_off).sum().item())
        assert nmis == 0, "record differs at %d of %d bytes" % (nmis, f_on.numel())
        assert torch.equal(r_on, r_off)
        del r_on, f_on, r_off, f_off
        for _ in range(3):
            s.cfl_dt(Ud, 0.4)
            s.step(Ud)
    assert s.status() == 0


def test_filter_whole_record_2d_1024():
    """1024^2 four quadrants (shocks, contacts, fallbacks) after 20 steps."""
    c = workloads.quadrants_2d(1024, scheme=10)
    s = T.Solver(gpu_params(c))
    Ud = torch.from_numpy(c["U"]).to(DEV)
    for _ in range(20):
        s.cfl_dt(Ud, 0.4)
        s.step(Ud)
    r_on, f_on, r_off, f_off = _rhs_both_ways(s, Ud)
    assert torch.equal(f_on, f_off)
    assert torch.equal(r_on, r_off)


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_filter_decides_noise_plateaus_2d(scheme):
    """1024^2 four quadrants after 45 steps: rounding noise has then spread
    over the constant states (the numerical domain of dependence grows by up
    to 3H cells a step), and their decisions follow the noise.  The filter
    must still decide all but a small share of the reconstructions (before
    it handled such values it sent 95 % of them to the FP64 path), with the
    decision record and the RHS identical to the FP64 path's."""
    c = workloads.quadrants_2d(1024, scheme=scheme)
    s = T.Solver(gpu_params(c))
    Ud = torch.from_numpy(c["U"]).to(DEV)
    for _ in range(45):
        s.cfl_dt(Ud, 0.4)
        s.step(Ud)
    T.teno_profile_enable(True)
    try:
        s.rhs(Ud)
        torch.cuda.synchronize()
        _, _, faces, exact = T.teno_profile_read()
    finally:
        T.teno_profile_enable(False)
    share = exact / (faces * 2 * 4)
    assert share < 0.02, "exact-path share %.4f" % share
    r_on, f_on, r_off, f_off = _rhs_both_ways(s, Ud)
    assert torch.equal(f_on, f_off)
    assert torch.equal(r_on, r_off)
