"""Shared helpers for the test-suite (no scheme arithmetic)."""
import numpy as np


def oracle_params(case, **over):
    import oracle
    kw = dict(ndim=case["ndim"], n=case["n"], dx=case["dx"], scheme=case["scheme"],
              gamma=case["gamma"], bc_lo=case["bc_lo"], bc_hi=case["bc_hi"],
              limiter=case.get("limiter", 0), bc_state_lo=case.get("bc_state_lo"),
              bc_state_hi=case.get("bc_state_hi"))
    kw.update(over)
    return oracle.params(**kw)


def primitive(U, gamma):
    """(rho, velocity list, p) of conserved variables (ncons, cells)."""
    nd = U.shape[0] - 2
    rho = U[0]
    vel = [U[1 + a] / rho for a in range(nd)]
    ke = 0.5 * rho * sum(v * v for v in vel)
    p = (gamma - 1.0) * (U[-1] - ke)
    return rho, vel, p


def advance_oracle(p, U, t_end, cfl=0.4, threads=1, stage_hook=None, max_steps=100000):
    """Advance to t_end with dt from the CFL rule, the last step clipped."""
    import oracle
    t = 0.0
    steps = 0
    while t < t_end - 1e-14 and steps < max_steps:
        dt, _, _ = oracle.cfl_dt(p, U, cfl)
        dt = min(dt, t_end - t)
        if stage_hook is None:
            U, _ = oracle.rk3_step(p, U, dt, threads=threads)
        else:
            Un = U
            Uk = U
            for s in range(3):
                L, _, _, _ = oracle.rhs(p, Uk, dt, threads=threads)
                Uk = oracle.rk3_combine(s, Un, Uk, L, dt)
                stage_hook(Uk)
            U = Uk
        t += dt
        steps += 1
    return U, steps
