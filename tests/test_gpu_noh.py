"""3D Noh implosion (Sec. 5.5): symmetry walls at x_i = 0 (App. A.1) and
supersonic inflow through the far faces as Dirichlet states (App. A.3) with
the analytic density of Eq. density_noh, Rusanov splitting, limiter on.

* Parity: a few steps on a small grid, the inflow states updated every step,
  bitwise against the oracle.
* The analytic solution at 64^3, t = 0.6: the shock at r = t/3, the density
  (1 + t/r)^2 ahead of it and 64 behind it.  The cold inflow (p = 1e-6) makes
  the cell-level pre-shock density scatter (the indicators see amplified
  pressure noise and select low-order stencils), so the density is compared
  as shell averages; the scatter is bounded separately.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_14340_gb300 as T  # noqa: E402

DEV = torch.device("cuda:0")


def setup(n, scheme):
    c = workloads.noh_3d(n, scheme=scheme)
    st = [torch.from_numpy(a).to(DEV) for a in workloads.noh_inflow_states(c, 0.0)]
    p = T.teno_params_init(ndim=3, n=c["n"], dx=c["dx"], scheme=scheme, gamma=c["gamma"],
                           bc_lo=c["bc_lo"], bc_hi=c["bc_hi"], flux_split=c["split"],
                           limiter=c["limiter"], bc_state_hi=st)
    return c, st, p


def set_states(c, st, t):
    for d, a in enumerate(workloads.noh_inflow_states(c, t)):
        st[d].copy_(torch.from_numpy(a))


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_noh_parity_steps(scheme):
    c, st, p = setup(20, scheme)
    S = T.Solver(p)
    U = torch.from_numpy(c["U"]).to(DEV)
    Uo = c["U"].copy()
    t = 0.0
    for _ in range(4):
        states = workloads.noh_inflow_states(c, t)
        set_states(c, st, t)
        po = oracle.params(3, c["n"], c["dx"], scheme=scheme, gamma=c["gamma"], bc_lo=c["bc_lo"],
                           bc_hi=c["bc_hi"], split=c["split"], limiter=c["limiter"],
                           bc_state_hi=states)
        dt_o, _, _ = oracle.cfl_dt(po, Uo, 0.4)
        dt_g = float(S.cfl_dt(U, 0.4).item())
        assert dt_g == dt_o
        S.step(U)
        Uo, nb = oracle.rk3_step(po, Uo, dt_o, threads=4)
        assert nb == 0 and S.status() == 0
        assert np.array_equal(U.cpu().numpy(), Uo)
        t += dt_o


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_noh_analytic_solution(scheme):
    n, t_end = 64, 0.6
    c, st, p = setup(n, scheme)
    S = T.Solver(p)
    U = torch.from_numpy(c["U"]).to(DEV)
    t = 0.0
    while t < t_end - 1e-12:
        set_states(c, st, t)
        dt = min(float(S.cfl_dt(U, 0.4).item()), t_end - t)
        S.step(U, dt=dt)
        t += dt
    assert S.status() == 0                       # positive density and pressure throughout
    L = c["L"]
    dx = L / n
    cc = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(cc, cc, cc, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z).ravel()
    Uh = U.cpu().numpy()
    rho = Uh[0]
    pres = (c["gamma"] - 1.0) * (Uh[4] - 0.5 * (Uh[1:4] ** 2).sum(axis=0) / rho)
    R = t / 3.0
    # shell averages, one cell wide, inside the inscribed sphere r < L
    shell = np.floor(r / dx).astype(int)
    k = np.arange(int(L / dx))
    prof = np.array([rho[shell == i].mean() for i in k])
    pprof = np.array([pres[shell == i].mean() for i in k])
    rc = np.array([r[shell == i].mean() for i in k])
    ex = workloads.noh_density(rc, t)
    # the shock: the shell profile crosses 40 (between 16 ahead, 64 behind) at t/3
    first_below = int(np.argmax((prof < 40.0) & (rc > 0.5 * R)))
    r40 = rc[first_below]
    pre = rc > R + 6 * dx
    post = (rc > 0.4 * R) & (rc < R - 4 * dx)
    pre_err = np.abs(prof[pre] - ex[pre]) / ex[pre]
    post_mean = prof[post].mean()
    post_p = pprof[post].mean()                  # exact: 64/3 behind the shock
    cell_pre = r > R + 6 * dx
    scatter = np.percentile(np.abs(rho[cell_pre] - workloads.noh_density(r[cell_pre], t))
                            / workloads.noh_density(r[cell_pre], t), 99)
    print("noh scheme %d: r40 %.4f (t/3 %.4f), pre-shock shell error max %.4f mean %.4f, "
          "post-shock density %.2f pressure %.3f, cell scatter p99 %.3f"
          % (scheme, r40, R, pre_err.max(), pre_err.mean(), post_mean, post_p, scatter))
    assert abs(r40 - R) <= 2.5 * dx
    assert pre_err.max() <= 0.05
    # the plateau and the pressure converge slowly with the cell size (the
    # start-up error of the singular initial state moves the shock ahead);
    # at 64^3 both sit 4-6 % low
    assert abs(post_mean - 64.0) <= 0.07 * 64.0
    assert abs(post_p - 64.0 / 3.0) <= 0.07 * 64.0 / 3.0
    assert scatter <= 0.30
