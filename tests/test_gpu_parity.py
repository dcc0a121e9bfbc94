"""GPU (sm_103a) vs CPU-oracle parity through the C ABI.

Tolerances (stated by the method's accuracy contract): RHS and one RK3 step
within 1e-12 relative (per conserved variable, relative to its max |value|),
the 1D shock-tube run to t = 0.2 within 1e-10 relative L-infinity, and the
per-face decision bytes (stencil selection, cut-offs, C_T exponent) identical.
Both sides evaluate every expression in the same order with the same fused
operations, so the kernels are in fact expected to agree bit for bit; the
bitwise checks are separate assertions.
"""
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


def gpu_params(case, **over):
    kw = dict(ndim=case["ndim"], n=case["n"], dx=case["dx"], scheme=case["scheme"],
              gamma=case["gamma"], bc_lo=case["bc_lo"], bc_hi=case["bc_hi"],
              limiter=case.get("limiter", 0))
    keep = []
    for side in ("bc_state_lo", "bc_state_hi"):
        st = case.get(side)
        if st is not None:
            t = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in st]
            keep += t
            kw[side] = t
    kw.update(over)
    p = T.teno_params_init(**kw)
    p._keep = keep                        # the device states live as long as p
    return p


def both_params(case, split=0, limiter=None):
    lim = case.get("limiter", 0) if limiter is None else limiter
    return (gpu_params(case, flux_split=split, limiter=lim),
            oracle_params(case, split=split, limiter=lim))


def rel_err(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    scale = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return float((np.abs(a - b).max(axis=1) / scale).max())


def gpu_rhs(p, U, dt_lim=0.0):
    s = T.Solver(p)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).to(DEV)
    out, fl = s.rhs(Ud, dt_lim, flags=True)
    nb = s.status()
    return out.cpu().numpy(), fl.cpu().numpy(), nb


def _cases():
    g = np.random.Generator(np.random.PCG64(77))
    out = []
    for scheme in (8, 10, 12):
        for bc in (0, 1, 2):
            c = workloads.riemann_1d(137, seed=1001 + bc, scheme=scheme)
            c["bc_lo"] = [bc, 0, 0]
            c["bc_hi"] = [bc, 0, 0]
            out.append(("1d-riemann-s%d-bc%d" % (scheme, bc), c))
        c = workloads.smooth_wave_1d(131, scheme)
        out.append(("1d-smooth-s%d" % scheme, c))
        c = workloads.quadrants_2d(37, 29, scheme=scheme)
        out.append(("2d-quadrants-s%d" % scheme, c))
        c = workloads.tgv_3d(12, scheme=scheme)
        c["n"] = [12, 12, 12]
        out.append(("3d-tgv-s%d" % scheme, c))
    # 3D with uneven extents and mixed walls
    n = [19, 13, 11]
    cells = int(np.prod(n))
    U = workloads.prim_to_cons(g.uniform(0.3, 1.5, cells),
                               [g.uniform(-0.6, 0.6, cells) for _ in range(3)],
                               g.uniform(0.2, 1.5, cells), 1.4)
    out.append(("3d-random-walls", dict(U=U, ndim=3, n=n, dx=[0.1, 0.07, 0.05],
                                        bc_lo=[1, 2, 0], bc_hi=[2, 1, 0], scheme=10,
                                        gamma=1.4)))
    # no-slip (App. A.2) and Dirichlet (App. A.3) sides
    for scheme in (8, 10, 12):
        out.append(("1d-dirichlet-noslip-s%d" % scheme,
                    workloads.boundary_walls(1, [97], [4], [3], seed=6001, scheme=scheme)))
        out.append(("2d-dirichlet-noslip-s%d" % scheme,
                    workloads.boundary_walls(2, [33, 27], [1, 4], [3, 4], seed=6002, scheme=scheme)))
        out.append(("3d-dirichlet-noslip-s%d" % scheme,
                    workloads.boundary_walls(3, [14, 11, 9], [4, 3, 0], [2, 4, 0], seed=6003,
                                             scheme=scheme)))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("split", [0, 1])
def test_rhs_parity(name, case, split):
    pg, po = both_params(case, split=split, limiter=0)
    r_g, f_g, nb_g = gpu_rhs(pg, case["U"])
    r_o, f_o, _, nb_o = oracle.rhs(po, case["U"], want_flags=True, threads=4)
    f_g = f_g[:f_o.size]                  # the decision bytes (then the argmax words)
    assert nb_g == nb_o == 0
    mism = int(np.count_nonzero(f_g != f_o))
    assert mism == 0, "decision bytes differ at %d of %d" % (mism, f_o.size)
    assert rel_err(r_g, r_o) <= 1e-12
    assert np.array_equal(r_g, r_o), "not bitwise (max rel %.3g)" % rel_err(r_g, r_o)


@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_rhs_parity_without_record(name, case):
    """Without a decision record the sweeps leave out face n of periodic
    lines and the flux difference takes face 0 in its place (the same
    stencil cells, so the same flux): the RHS must still be the oracle's,
    which computes face n."""
    pg, po = both_params(case, split=0, limiter=0)
    s = T.Solver(pg)
    Ud = torch.from_numpy(np.ascontiguousarray(case["U"])).to(DEV)
    r_g = s.rhs(Ud, 0.0).cpu().numpy()
    r_o, _, _, _ = oracle.rhs(po, case["U"], threads=4)
    assert s.status() == 0
    assert np.array_equal(r_g, r_o), "not bitwise (max rel %.3g)" % rel_err(r_g, r_o)


@pytest.mark.parametrize("which", [10, 117, 3])
def test_rhs_parity_limiter(which):
    c = workloads.batched_1d(count=200, nmin=64, nmax=200)[which]
    pg, po = both_params(c, limiter=1)
    dt, _, _ = oracle.cfl_dt(po, c["U"], 0.4)
    r_g, f_g, nb_g = gpu_rhs(pg, c["U"], dt)
    r_o, f_o, lf_o, nb_o = oracle.rhs(po, c["U"], dt, want_flags=True)
    _, _, lim0, tot = T.record_layout(pg)
    assert f_g.size == tot
    lf_g = f_g[lim0:]                     # part 3: where the limiter bound
    f_g = f_g[:f_o.size]
    assert nb_g == nb_o
    assert np.count_nonzero(f_g != f_o) == 0
    assert np.array_equal(lf_g, lf_o)
    assert rel_err(r_g, r_o) <= 1e-12
    assert np.array_equal(r_g, r_o)


@pytest.mark.parametrize("scheme", [8, 10])
def test_limiter_record_parity(scheme):
    """The double rarefaction (near vacuum at the centre, Sec. 5.3) after four
    oracle steps, where the limiter binds on some faces: the limiter part of
    the decision record names the same faces as the oracle's, and the RHS
    and decision bytes are bitwise the oracle's."""
    c = workloads.double_rarefaction_1d(200, scheme=scheme)
    pg, po = both_params(c, limiter=1)
    U = c["U"].copy()
    for _ in range(4):
        dt, _, _ = oracle.cfl_dt(po, U, 0.4)
        U, _ = oracle.rk3_step(po, U, dt)
    dt, _, _ = oracle.cfl_dt(po, U, 0.4)
    r_g, f_g, nb_g = gpu_rhs(pg, U, dt)
    r_o, f_o, lf_o, nb_o = oracle.rhs(po, U, dt, want_flags=True)
    assert lf_o.sum() > 0
    assert np.array_equal(f_g[T.record_layout(pg)[2]:], lf_o)
    assert np.array_equal(f_g[:f_o.size], f_o)
    assert nb_g == nb_o
    assert np.array_equal(r_g, r_o)


def test_rhs_parity_limiter_2d():
    c = workloads.quadrants_2d(24, 20, scheme=8)
    pg, po = both_params(c, limiter=1)
    dt, _, _ = oracle.cfl_dt(po, c["U"], 0.4)
    r_g, f_g, _ = gpu_rhs(pg, c["U"], dt)
    r_o, f_o, lf_o, _ = oracle.rhs(po, c["U"], dt, want_flags=True)
    assert np.array_equal(f_g[:f_o.size], f_o)
    assert np.array_equal(f_g[T.record_layout(pg)[2]:], lf_o)
    assert rel_err(r_g, r_o) <= 1e-12
    assert np.array_equal(r_g, r_o)


@pytest.mark.parametrize("name,case", CASES[::3], ids=[c[0] for c in CASES[::3]])
def test_rk3_step_and_cfl_parity(name, case):
    pg, po = both_params(case)
    s = T.Solver(pg)
    Ud = torch.from_numpy(np.ascontiguousarray(case["U"])).to(DEV)
    dt_d = s.cfl_dt(Ud, 0.4)
    dt_o, _, _ = oracle.cfl_dt(po, case["U"], 0.4)
    assert float(dt_d.item()) == dt_o
    s.step(Ud)                                   # dt from the device scalar
    U1_o, _ = oracle.rk3_step(po, case["U"], dt_o, threads=4)
    assert s.status() == 0
    U1_g = Ud.cpu().numpy()
    assert rel_err(U1_g, U1_o) <= 1e-12
    assert np.array_equal(U1_g, U1_o)


def test_shock_tube_run_parity():
    """Seeded 1D two-state problem, TENO8-AA, N = 400, CFL 0.4, t = 0.2."""
    c = workloads.riemann_1d(400, scheme=8)
    pg, po = both_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(np.ascontiguousarray(c["U"])).to(DEV)
    Uo = c["U"].copy()
    t, steps = 0.0, 0
    while t < c["t_end"] - 1e-14:
        dt_g = float(s.cfl_dt(Ud).item())
        dt_o, _, _ = oracle.cfl_dt(po, Uo, 0.4)
        assert dt_g == dt_o
        dt = min(dt_o, c["t_end"] - t)
        s.step(Ud, dt)
        Uo, _ = oracle.rk3_step(po, Uo, dt)
        t += dt
        steps += 1
    assert s.status() == 0
    Ug = Ud.cpu().numpy()
    assert steps > 100
    assert rel_err(Ug, Uo) <= 1e-10
    assert np.array_equal(Ug, Uo)


def test_advance_host_matches_device_path():
    c = workloads.quadrants_2d(40, 33, scheme=10)
    pg, _ = both_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(np.ascontiguousarray(c["U"])).to(DEV)
    for _ in range(3):
        s.cfl_dt(Ud)
        s.step(Ud)
    Uh = torch.from_numpy(np.ascontiguousarray(c["U"])).pin_memory()
    Ud2 = torch.empty_like(Ud)
    ws2 = torch.zeros_like(s.ws)
    t = T.teno_advance_host(pg, Uh, Ud2, 3, 0.4, ws2)
    assert t > 0
    assert torch.equal(Uh, Ud.cpu())


@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_full_size_3d_sampled(scheme):
    """256^3 periodic Taylor-Green + k^-5/3 field, the launch configuration
    of the benchmark: the RHS at sampled cells (corners, faces, interior)
    against the oracle evaluated cell by cell."""
    c = workloads.tgv_3d(256, scheme=scheme)
    pg, po = both_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(c["U"]).to(DEV)
    r = s.rhs(Ud)
    assert s.status() == 0
    g = np.random.Generator(np.random.PCG64(31))
    n = 256
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n - 1, 0, 200), (127, 128, 0)]
    pts += [tuple(int(v) for v in g.integers(0, n, 3)) for _ in range(40)]
    cells = np.array([x + n * (y + n * z) for x, y, z in pts], np.int64)
    ro = oracle.rhs_at(po, c["U"], cells, threads=8)
    rg = r[:, torch.from_numpy(cells).to(DEV)].cpu().numpy()
    scale = r.abs().amax(dim=1).cpu().numpy()[:, None]
    assert np.abs(rg - ro).max(axis=1).max() <= 1e-12 * scale.max()
    assert np.array_equal(rg, ro)


def test_full_size_2d_sampled():
    c = workloads.quadrants_2d(1024, scheme=10)
    pg, po = both_params(c)
    s = T.Solver(pg)
    Ud = torch.from_numpy(c["U"]).to(DEV)
    r = s.rhs(Ud)
    g = np.random.Generator(np.random.PCG64(33))
    pts = [(0, 0), (1023, 1023), (511, 512), (512, 511), (0, 700)]
    pts += [tuple(int(v) for v in g.integers(0, 1024, 2)) for _ in range(60)]
    cells = np.array([x + 1024 * y for x, y in pts], np.int64)
    ro = oracle.rhs_at(po, c["U"], cells, threads=8)
    rg = r[:, torch.from_numpy(cells).to(DEV)].cpu().numpy()
    assert np.array_equal(rg, ro)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [8, 10, 12])
def test_minimum_grid(scheme):
    """n = H cells per axis (the smallest valid grid) in 2D, periodic and
    slip walls."""
    H = scheme // 2
    g = np.random.Generator(np.random.PCG64(41))
    n = [H, H + 1]
    cells = n[0] * n[1]
    U = workloads.prim_to_cons(g.uniform(0.5, 1.5, cells), [g.uniform(-0.5, 0.5, cells)] * 2,
                               g.uniform(0.5, 1.5, cells), 1.4)
    for bc in (0, 2):
        case = dict(U=U, ndim=2, n=n, dx=[0.1, 0.1], bc_lo=[bc] * 2, bc_hi=[bc] * 2,
                    scheme=scheme, gamma=1.4)
        pg, po = both_params(case)
        r_g, f_g, _ = gpu_rhs(pg, U)
        r_o, f_o, _, _ = oracle.rhs(po, U, want_flags=True)
        assert np.array_equal(f_g[:f_o.size], f_o)
        assert np.array_equal(r_g, r_o)


def test_nonphysical_counted_not_trapped():
    """Negative pressure and a NaN cell are counted on the device; the call
    returns normally and the context stays usable."""
    c = workloads.riemann_1d(64, scheme=8)
    U = c["U"].copy()
    U[2, 10] = -1.0                     # E < 0: negative pressure
    U[0, 40] = np.nan
    pg, po = both_params(c)
    _, _, nb_g = gpu_rhs(pg, U)
    _, _, _, nb_o = oracle.rhs(po, U)
    assert nb_g > 0 and nb_g == nb_o    # the same cells and faces counted
    # still usable
    r_g, _, nb = gpu_rhs(pg, c["U"])
    assert nb == 0 and np.isfinite(r_g).all()


def test_invalid_parameters_rejected():
    p = T.teno_params_init(ndim=1, n=[3], dx=[0.1], scheme=8)       # n < H
    with pytest.raises(T.TenoError) as e:
        T.teno_workspace_bytes(p)
    assert e.value.code == T.TENO_EINVAL
    p = T.teno_params_init(ndim=1, n=[64], dx=[0.1], scheme=8)
    s = T.Solver(p)
    U = torch.ones(3, 64, dtype=torch.float64, device=DEV)
    small = torch.zeros(4, dtype=torch.float64, device=DEV)
    with pytest.raises(T.TenoError):
        T.teno_rhs(p, U, torch.empty_like(U), 0.0, None, small)      # workspace too small
    with pytest.raises(T.TenoError):
        T.teno_rhs(p, U, U, 0.0, None, s.ws)                         # aliasing
    big = torch.ones(3 * 64 + 1, dtype=torch.float64, device=DEV)
    with pytest.raises(T.TenoError):
        T.teno_rhs(p, big[1:], torch.empty_like(U), 0.0, None, s.ws)  # 8-byte offset
