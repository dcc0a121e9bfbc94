"""Domain decomposition on one GPU: a grid split into slabs along its
slowest axis, every slab a sub-problem with TENO_BC_HALO on its inner sides,
halo planes copied between slabs before every RK stage and the CFL step
taken over all slabs (teno_wave_speeds + teno_dt_from_speeds).  Each slab
computes its boundary faces from the same stencil cells as the undivided
grid, so after several steps the slabs must equal the undivided grid bit
for bit (which the parity tests pin to the oracle; one case is checked
against the oracle directly here too)."""
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


def params_of(c, **over):
    kw = dict(ndim=c["ndim"], n=c["n"], dx=c["dx"], scheme=c["scheme"], gamma=c["gamma"],
              bc_lo=c["bc_lo"], bc_hi=c["bc_hi"], limiter=c.get("limiter", 0))
    kw.update(over)
    return T.teno_params_init(**kw)


def _cases():
    out = []
    for scheme in (8, 10, 12):
        c = workloads.tgv_3d(24, scheme=scheme)
        out.append(("3d-periodic-s%d" % scheme, c, (2, 3)))
    c = workloads.boundary_walls(3, [14, 11, 20], [1, 2, 1], [2, 1, 3], seed=6003, scheme=10)
    c.pop("bc_state_lo", None)
    c.pop("bc_state_hi", None)
    out.append(("3d-walls-s10", c, (2, 4)))
    for scheme in (8, 10):
        c = workloads.quadrants_2d(40, 36, scheme=scheme)
        out.append(("2d-transmissive-s%d" % scheme, c, (2, 3)))
    c = workloads.riemann_1d(137, scheme=10)
    out.append(("1d-transmissive-s10", c, (3,)))
    c = workloads.batched_1d(count=200, nmin=120, nmax=200)[10]     # near vacuum, limiter on
    c["limiter"] = 1
    out.append(("1d-limiter-s%d" % c["scheme"], c, (2,)))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,case,splits", CASES, ids=[c[0] for c in CASES])
def test_slabs_equal_undivided_grid(name, case, splits):
    p = params_of(case)
    s = T.Solver(p)
    Ud = torch.from_numpy(np.ascontiguousarray(case["U"])).to(DEV)
    U0 = Ud.clone()
    for _ in range(3):
        s.cfl_dt(Ud)
        s.step(Ud)
    assert s.status() == 0
    for parts in splits:
        D = T.SlabDecomposition(p, parts)
        states = D.split(U0)
        for _ in range(3):
            D.cfl_dt(states)
            D.step(states)
        assert torch.equal(D.join(states), Ud), "%d slabs differ from the undivided grid" % parts


def test_slabs_against_oracle():
    c = workloads.tgv_3d(20, scheme=10)
    p = params_of(c)
    D = T.SlabDecomposition(p, 2)
    states = D.split(torch.from_numpy(c["U"]).to(DEV))
    po = oracle_params(c)
    Uo = c["U"].copy()
    for _ in range(2):
        dt_g = float(D.cfl_dt(states).item())
        D.step(states)
        dt_o, _, _ = oracle.cfl_dt(po, Uo, 0.4)
        assert dt_g == dt_o
        Uo, _ = oracle.rk3_step(po, Uo, dt_o)
    assert np.array_equal(D.join(states).cpu().numpy(), Uo)


def test_stages_equal_step():
    """teno_rk3_stage 1, 2, 3 on a grid without halos is teno_rk3_step."""
    c = workloads.quadrants_2d(33, 29, scheme=12)
    p = params_of(c)
    s = T.Solver(p)
    U = torch.from_numpy(c["U"]).to(DEV)
    U2 = U.clone()
    Us = torch.empty_like(U)
    dt = float(s.cfl_dt(U).item())
    s.step(U, dt)
    for k in (1, 2, 3):
        T.teno_rk3_stage(p, k, U2, Us, dt, None, s.ws)
    assert torch.equal(U, U2)


def test_halo_validation():
    halo = torch.zeros(4 * 5 * 16, dtype=torch.float64, device=DEV)
    p = T.teno_params_init(ndim=2, n=[16, 16], dx=[0.1, 0.1], scheme=10, bc_lo=[1, 5],
                           bc_hi=[1, 1], bc_state_lo=[None, halo])
    T.teno_workspace_bytes(p)                                   # valid
    bad = T.teno_params_init(ndim=2, n=[16, 16], dx=[0.1, 0.1], scheme=10, bc_lo=[1, 5],
                             bc_hi=[1, 1])                      # no halo array
    with pytest.raises(T.TenoError):
        T.teno_workspace_bytes(bad)
    bad = T.teno_params_init(ndim=2, n=[16, 16], dx=[0.1, 0.1], scheme=10, bc_lo=[1, 5],
                             bc_hi=[1, 1], bc_state_lo=[None, halo], limiter=1)
    with pytest.raises(T.TenoError):                            # limiter needs the whole grid
        T.teno_workspace_bytes(bad)
