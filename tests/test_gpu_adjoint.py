"""Adjoint of the TENO-AA right-hand side and of the SSP-RK3 step on the GPU
(decisions frozen), checked three ways:
  * dot-product tests <J v, lam> = <v, J^T lam> with J v from central finite
    differences of the GPU forward along seeded smooth directions whose
    perturbed runs keep every decision byte identical;
  * an oracle-side reference: J^T lam of a small 1D problem assembled column
    by column from central differences of the CPU oracle (decisions checked);
  * the checkpointed rollout gradient against finite differences of the loss
    along seeded directions, decision records compared at every stage.
Tolerance: 1e-6 relative."""
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


def smooth_state(nd, n, seed, gamma=1.4):
    shape = tuple(reversed(n[:nd]))
    rho = 1.0 + 0.3 * workloads.smooth_field(shape, seed)
    vel = [0.4 * workloads.smooth_field(shape, seed + 1 + a) for a in range(nd)]
    p = 1.0 + 0.3 * workloads.smooth_field(shape, seed + 7)
    return workloads.prim_to_cons(rho.ravel(), [v.ravel() for v in vel], p.ravel(), gamma)


def direction(nd, n, seed):
    shape = (nd + 2,) + tuple(reversed(n[:nd]))
    return workloads.smooth_field(shape, seed).reshape(nd + 2, -1)


def gpu_rhs_flags(p, U):
    """RHS and the decision bits the frozen linear map depends on (stencil
    selection and cut-offs; the C_T exponent bits only feed the decision)."""
    s = T.Solver(p)
    out, fl = s.rhs(U, 0.0, flags=True)
    return out, fl & 0x1F


CASES = [
    ("1d-periodic-s8-llf", 1, [48], 8, [0], [0], 0),
    ("1d-transmissive-s10-rus", 1, [40], 10, [1], [1], 1),
    ("1d-slip-s8-llf", 1, [36], 8, [2], [2], 0),
    ("2d-mixed-s8-llf", 2, [24, 20], 8, [1, 0], [1, 0], 0),
    ("2d-slip-s10-llf", 2, [20, 22], 10, [2, 1], [2, 1], 0),
    ("3d-periodic-s10-llf", 3, [12, 11, 10], 10, [0, 0, 0], [0, 0, 0], 0),
    ("2d-noslip-s8-llf", 2, [22, 20], 8, [3, 0], [2, 0], 0),
    ("3d-noslip-s10-rus", 3, [12, 11, 10], 10, [3, 1, 0], [1, 3, 0], 1),
    ("1d-periodic-s12-llf", 1, [48], 12, [0], [0], 0),
    ("2d-slip-s12-rus", 2, [24, 22], 12, [2, 1], [2, 1], 1),
    ("3d-noslip-s12-rus", 3, [12, 11, 10], 12, [3, 1, 0], [1, 3, 0], 1),
]


def test_adjoint_rejects_dirichlet():
    """The adjoint calls do not differentiate Dirichlet ghosts (App. A.3)."""
    st = torch.ones(4, 20, dtype=torch.float64, device=DEV)
    p = T.teno_params_init(ndim=2, n=[20, 18], dx=[0.05, 0.05], scheme=8, bc_lo=[0, 4],
                           bc_hi=[0, 1], bc_state_lo=[None, st])
    aws = T.aligned_workspace(T.teno_adjoint_workspace_bytes(p), DEV)
    U = torch.ones(4, 360, dtype=torch.float64, device=DEV)
    with pytest.raises(T.TenoError) as e:
        T.teno_rhs_vjp(p, U, U.clone(), torch.empty_like(U), None, aws)
    assert e.value.code == T.TENO_EINVAL


@pytest.mark.parametrize("name,nd,n,scheme,lo,hi,split", CASES, ids=[c[0] for c in CASES])
def test_rhs_vjp_dot_product(name, nd, n, scheme, lo, hi, split):
    p = T.teno_params_init(ndim=nd, n=n, dx=[1.0 / k for k in n], scheme=scheme, bc_lo=lo,
                           bc_hi=hi, flux_split=split)
    U = torch.from_numpy(smooth_state(nd, n, 11)).to(DEV)
    lam = torch.from_numpy(direction(nd, n, 21)).to(DEV)
    mu = torch.empty_like(U)
    aws = T.aligned_workspace(T.teno_adjoint_workspace_bytes(p), DEV)
    T.teno_rhs_vjp(p, U, lam, mu, None, aws)
    _, fl0 = gpu_rhs_flags(p, U)
    checked = 0
    for seed in (31, 32, 33, 34, 35, 36, 37, 38):
        v = torch.from_numpy(direction(nd, n, seed)).to(DEV)
        for h in (1e-6, 1e-7):
            Lp, flp = gpu_rhs_flags(p, U + h * v)
            Lm, flm = gpu_rhs_flags(p, U - h * v)
            if torch.equal(flp, fl0) and torch.equal(flm, fl0):
                break
        else:
            continue                      # this direction flips a decision: not usable
        checked += 1
        jvp = (Lp - Lm) / (2 * h)
        lhs = float((jvp * lam).sum())
        rhs = float((v * mu).sum())
        assert abs(lhs - rhs) <= 1e-6 * max(abs(rhs), 1e-300), (lhs, rhs)
    assert checked >= 2


@pytest.mark.parametrize("scheme,split", [(8, 0), (10, 1), (12, 0)])
def test_rhs_vjp_matches_oracle_reference(scheme, split):
    """Full J^T lam of a 1D periodic problem, assembled from central
    differences of the CPU oracle, one conserved variable of one cell at a
    time (each perturbation keeps the oracle's decision bytes)."""
    N = 24
    U0 = smooth_state(1, [N], 41)
    lam = direction(1, [N], 42)
    po = oracle.params(1, [N], [1.0 / N], scheme=scheme, split=split)
    _, fl0, _, _ = oracle.rhs(po, U0, want_flags=True)
    fl0 = fl0 & 0x1F
    ref = np.full_like(U0, np.nan)
    for c in range(3):
        for i in range(N):
            for h in (1e-6, 1e-7, 1e-8):
                Up = U0.copy()
                Um = U0.copy()
                Up[c, i] += h
                Um[c, i] -= h
                Lp, flp, _, _ = oracle.rhs(po, Up, want_flags=True)
                Lm, flm, _, _ = oracle.rhs(po, Um, want_flags=True)
                if np.array_equal(flp & 0x1F, fl0) and np.array_equal(flm & 0x1F, fl0):
                    ref[c, i] = np.sum((Lp - Lm) / (2 * h) * lam)
                    break
    ok = np.isfinite(ref)
    assert ok.mean() >= 0.9          # columns whose perturbation keeps every decision
    p = T.teno_params_init(ndim=1, n=[N], dx=[1.0 / N], scheme=scheme, flux_split=split)
    aws = T.aligned_workspace(T.teno_adjoint_workspace_bytes(p), DEV)
    U = torch.from_numpy(U0).to(DEV)
    mu = torch.empty_like(U)
    T.teno_rhs_vjp(p, U, torch.from_numpy(lam).to(DEV), mu, None, aws)
    mu = mu.cpu().numpy()
    assert np.abs(mu[ok] - ref[ok]).max() <= 1e-6 * np.abs(ref[ok]).max()


def test_rhs_vjp_with_recorded_flags_equals_recomputed():
    nd, n = 2, [24, 20]
    p = T.teno_params_init(ndim=nd, n=n, dx=[1.0 / k for k in n], scheme=10, bc_lo=[1, 0],
                           bc_hi=[1, 0])
    U = torch.from_numpy(smooth_state(nd, n, 51)).to(DEV)
    lam = torch.from_numpy(direction(nd, n, 52)).to(DEV)
    _, fl = gpu_rhs_flags(p, U)
    aws = T.aligned_workspace(T.teno_adjoint_workspace_bytes(p), DEV)
    a, b = torch.empty_like(U), torch.empty_like(U)
    T.teno_rhs_vjp(p, U, lam, a, fl, aws)
    T.teno_rhs_vjp(p, U, lam, b, None, aws)
    assert torch.equal(a, b)


def test_rk3_record_matches_step_and_vjp_dot():
    c = workloads.adjoint_2d(40, 32)
    p = T.teno_params_init(ndim=2, n=c["n"], dx=c["dx"], scheme=8, bc_lo=c["bc_lo"],
                           bc_hi=c["bc_hi"])
    dt, _, _ = oracle.cfl_dt(oracle_params(c), c["U"], 0.4)
    U = torch.from_numpy(c["U"]).to(DEV)
    fws = T.aligned_workspace(T.teno_workspace_bytes(p), DEV)
    Ua = U.clone()
    T.teno_rk3_step(p, Ua, dt, None, fws)
    Ub = U.clone()
    U1, U2 = torch.empty_like(U), torch.empty_like(U)
    fl = torch.empty(3 * T.teno_flags_bytes(p), dtype=torch.uint8, device=DEV)
    T.teno_rk3_step_record(p, Ub, dt, U1, U2, fl, fws)
    assert torch.equal(Ua, Ub)
    aws = T.aligned_workspace(T.teno_adjoint_workspace_bytes(p), DEV)
    w = torch.from_numpy(direction(2, c["n"], 61)).to(DEV)
    abar = w.clone()
    T.teno_rk3_step_vjp(p, U, U1, U2, fl, dt, abar, aws)
    checked = 0
    for seed in (62, 63, 64, 65, 66, 67, 68, 69):
        v = torch.from_numpy(direction(2, c["n"], seed)).to(DEV) * U.abs().amax(dim=1, keepdim=True)
        for h in (1e-7, 1e-8, 1e-9):
            res, same = [], True
            for sgn in (1, -1):
                Us = U + sgn * h * v
                V1, V2 = torch.empty_like(U), torch.empty_like(U)
                fls = torch.empty_like(fl)
                T.teno_rk3_step_record(p, Us, dt, V1, V2, fls, fws)
                same = same and same_linearisation(p, fls, fl, 3)[0]
                res.append(Us)
            if same:
                break
        if not same:
            continue
        checked += 1
        jvp = (res[0] - res[1]) / (2 * h)
        lhs = float((jvp * w).sum())
        rhs = float((v * abar).sum())
        assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)
    assert checked >= 1


@pytest.mark.parametrize("nd", [2, 3])
def test_selection_only_record(nd):
    """teno_rk3_step_record_sel: the same step, stage states, argmax words and
    limiter bytes as teno_rk3_step_record, and decision bytes whose low five
    bits (all the adjoint reads) are the full record's; the C_T exponent bits
    are the full record's or zero."""
    if nd == 2:
        c = workloads.adjoint_2d(40, 32)
        scheme = 8
    else:
        c = workloads.tgv_3d(16, scheme=10)
        scheme = 10
    p = T.teno_params_init(ndim=nd, n=c["n"], dx=c["dx"], scheme=scheme, bc_lo=c["bc_lo"],
                           bc_hi=c["bc_hi"])
    dt, _, _ = oracle.cfl_dt(oracle_params(c), c["U"], 0.4)
    fws = T.aligned_workspace(T.teno_workspace_bytes(p), DEV)
    flb = T.teno_flags_bytes(p)
    ndec, tot = _decision_parts(p)
    outs = []
    for rec in (T.teno_rk3_step_record, T.teno_rk3_step_record_sel):
        U = torch.from_numpy(c["U"]).to(DEV)
        U1, U2 = torch.empty_like(U), torch.empty_like(U)
        fl = torch.empty(3 * flb, dtype=torch.uint8, device=DEV)
        rec(p, U, dt, U1, U2, fl, fws)
        outs.append((U, U1, U2, fl.cpu().numpy()))
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert torch.equal(a, b)
    fa, fb = outs[0][3], outs[1][3]
    zero_ct = 0
    for s in range(3):
        x, y = fa[s * tot:(s + 1) * tot], fb[s * tot:(s + 1) * tot]
        assert np.array_equal(x[ndec:], y[ndec:])
        assert np.array_equal(x[:ndec] & 0x1F, y[:ndec] & 0x1F)
        ct_x, ct_y = x[:ndec] >> 5, y[:ndec] >> 5
        assert np.all((ct_y == ct_x) | (ct_y == 0))
        zero_ct += int(np.count_nonzero(ct_y != ct_x))
    assert zero_ct > 0          # the quick acceptance did skip exponents


def _decision_parts(p):
    """(bytes of the per-face decision bytes, total bytes) of one record."""
    nc = p.ndim + 2
    faces = 0
    for d in range(p.ndim):
        fn = [p.n[0], p.n[1], p.n[2]]
        fn[d] += 1
        faces += fn[0] * fn[1] * fn[2]
    return faces * nc * 2, T.teno_flags_bytes(p)


def same_linearisation(p, a, b, stages=1):
    """True if two records agree on everything the linearised map depends on:
    stencil selection and cut-offs (low 5 bits of each decision byte) and the
    maximising cells of the splitting speeds.  Returns (same, n_decision
    flips, n_argmax flips)."""
    ndec, tot = _decision_parts(p)
    nd_f = na_f = 0
    for s in range(stages):
        x, y = a[s * tot:(s + 1) * tot], b[s * tot:(s + 1) * tot]
        nd_f += int(((x[:ndec] & 0x1F) != (y[:ndec] & 0x1F)).sum())
        na_f += int((x[ndec:] != y[ndec:]).sum())
    return nd_f == 0 and na_f == 0, nd_f, na_f


def _record(p, U0, dt, nsteps):
    """Run nsteps recorded steps; returns U(T) and the decision records."""
    fws = T.aligned_workspace(T.teno_workspace_bytes(p), DEV)
    U = U0.clone()
    flb = T.teno_flags_bytes(p)
    fls = []
    for _ in range(nsteps):
        U1, U2 = torch.empty_like(U), torch.empty_like(U)
        fl = torch.empty(3 * flb, dtype=torch.uint8, device=DEV)
        T.teno_rk3_step_record(p, U, dt, U1, U2, fl, fws)
        fls.append(fl)
    return U, fls


def _frozen_run(p, U0, dt, fls):
    fws = T.aligned_workspace(T.teno_workspace_bytes(p), DEV)
    U = U0.clone()
    for fl in fls:
        T.teno_rk3_step_frozen(p, U, dt, fl, fws)
    return U


def _setup(nx, ny, nsteps, every):
    c = workloads.adjoint_2d(nx, ny)
    p = T.teno_params_init(ndim=2, n=c["n"], dx=c["dx"], scheme=8, bc_lo=c["bc_lo"],
                           bc_hi=c["bc_hi"])
    dt, _, _ = oracle.cfl_dt(oracle_params(c), c["U"], 0.4)
    U0 = torch.from_numpy(c["U"]).to(DEV)
    Ut = torch.from_numpy(c["U_target_ic"]).to(DEV)
    rho_t = T.rollout(p, Ut, dt, nsteps, every)[0].detach()
    U0g = U0.clone().requires_grad_(True)
    UT = T.rollout(p, U0g, dt, nsteps, every)
    loss = 0.5 * ((UT[0] - rho_t) ** 2).sum()
    loss.backward()
    return c, p, dt, U0, rho_t, U0g.grad


@pytest.mark.parametrize("scheme", [10, 12])
def test_frozen_rhs_equals_deciding_rhs(scheme):
    nd, n = 2, [30, 26]
    p = T.teno_params_init(ndim=nd, n=n, dx=[1.0 / k for k in n], scheme=scheme, bc_lo=[1, 0],
                           bc_hi=[1, 0])
    U = torch.from_numpy(smooth_state(nd, n, 71)).to(DEV)
    s = T.Solver(p)
    r, fl = s.rhs(U, flags=True)
    rf = torch.empty_like(U)
    T.teno_rhs_frozen(p, U, rf, fl, s.ws)
    scale = r.abs().amax(dim=1, keepdim=True)
    assert float(((rf - r).abs() / scale).max()) <= 1e-13


def test_rollout_gradient_vs_frozen_decision_differences():
    """Central differences of the frozen-decision map (the base trajectory's
    recorded decisions applied along U0 +- h v) against the adjoint gradient:
    any direction, no decision can flip by construction."""
    nsteps, every = 20, 5
    c, p, dt, U0, rho_t, grad = _setup(48, 32, nsteps, every)
    _, fls = _record(p, U0, dt, nsteps)
    scale = U0.abs().amax(dim=1, keepdim=True)
    for seed in (5003, 5004, 5005, 5006):
        v = torch.from_numpy(workloads.smooth_field((4, 32, 48), seed).reshape(4, -1)).to(DEV) * scale
        h = 1e-6
        jp = 0.5 * float(((_frozen_run(p, U0 + h * v, dt, fls)[0] - rho_t) ** 2).sum())
        jm = 0.5 * float(((_frozen_run(p, U0 - h * v, dt, fls)[0] - rho_t) ** 2).sum())
        fd = (jp - jm) / (2 * h)
        ad = float((grad * v).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_rollout_gradient_vs_selection_preserving_differences():
    """Central differences of the real (deciding) forward along directions
    whose perturbed runs keep every decision of every stage (selection,
    cut-offs and maximising cells), on a smooth flow (transmissive in x,
    periodic in y), the step shrunk until that holds.  The horizon is short:
    over many stages some decision always lies within rounding of its
    threshold, so no finite step keeps them all (the frozen-decision test
    above covers long horizons)."""
    nd, n, nsteps, every = 2, [48, 32], 3, 1
    p = T.teno_params_init(ndim=nd, n=n, dx=[1.0 / k for k in n], scheme=8, bc_lo=[1, 0],
                           bc_hi=[1, 0])
    U0 = torch.from_numpy(smooth_state(nd, n, 81)).to(DEV)
    po = oracle.params(nd, n, [1.0 / k for k in n], scheme=8, bc_lo=[1, 0], bc_hi=[1, 0])
    dt, _, _ = oracle.cfl_dt(po, U0.cpu().numpy(), 0.4)
    rho_t = (U0[0] * 1.001).clone()
    U0g = U0.clone().requires_grad_(True)
    UT = T.rollout(p, U0g, dt, nsteps, every)
    (0.5 * ((UT[0] - rho_t) ** 2).sum()).backward()
    grad = U0g.grad
    _, fl0 = _record(p, U0, dt, nsteps)
    scale = U0.abs().amax(dim=1, keepdim=True)
    checked = 0
    flips = []
    for seed in range(5003, 5015):
        v = torch.from_numpy(workloads.smooth_field((4, 32, 48), seed).reshape(4, -1)).to(DEV) * scale
        ok = False
        for h in (1e-6, 1e-7, 1e-8, 1e-9):
            Up, flp = _record(p, U0 + h * v, dt, nsteps)
            Um, flm = _record(p, U0 - h * v, dt, nsteps)
            res = [(same_linearisation(p, a, d, 3), same_linearisation(p, b, d, 3))
                   for a, b, d in zip(flp, flm, fl0)]
            if all(x[0] and y[0] for x, y in res):
                ok = True
                break
            flips.append((seed, h, sum(x[1] + y[1] for x, y in res), sum(x[2] + y[2] for x, y in res)))
        if not ok:
            continue                      # a decision flips along this direction
        checked += 1
        jp = 0.5 * float(((Up[0] - rho_t) ** 2).sum())
        jm = 0.5 * float(((Um[0] - rho_t) ** 2).sum())
        fd = (jp - jm) / (2 * h)
        ad = float((grad * v).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad, h)
    assert checked >= 2, flips


def test_checkpoint_interval_does_not_change_gradient():
    """Bitwise the same gradient for checkpoints every 3, 5 (a partial last
    segment) and 12 steps (one segment, recorded by the forward itself: no
    recompute at all)."""
    c = workloads.adjoint_2d(32, 24)
    p = T.teno_params_init(ndim=2, n=c["n"], dx=c["dx"], scheme=8, bc_lo=c["bc_lo"],
                           bc_hi=c["bc_hi"])
    dt, _, _ = oracle.cfl_dt(oracle_params(c), c["U"], 0.4)
    grads = []
    for every in (3, 5, 12):
        U0 = torch.from_numpy(c["U"]).to(DEV).requires_grad_(True)
        UT = T.rollout(p, U0, dt, 12, every)
        (0.5 * (UT[0] ** 2).sum()).backward()
        grads.append(U0.grad.clone())
    assert torch.equal(grads[0], grads[1]) and torch.equal(grads[0], grads[2])
