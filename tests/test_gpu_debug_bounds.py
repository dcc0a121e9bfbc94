"""The bounds-checked build (libteno_gb300_debug.so, -DTENO_DEBUG_BOUNDS) on
small grids (16-64 cells per axis): every global-memory index of the face
sweeps, the combine and the primitives kernel, and the sweeps' shared-memory
queue indices, range-checked on the device, must stay in range -- the
status block's out-of-range counter stays zero -- while the results stay
bitwise the oracle's.  Cases: 1D/2D/3D grids with every boundary rule
(periodic, transmissive, slip and no-slip walls, Dirichlet, halo sides of a
slab decomposition), the three schemes, both splittings, the limiter near
vacuum, decision records, RK3 steps and the batched face kernel.

The checked library is built and run in a child process (TENO_GB300_DEBUG=1
selects it in the binding; a process loads one build)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_bounds_checked_build():
    env = dict(os.environ, TENO_GB300_DEBUG="1", PYTHONPATH=ROOT + os.pathsep + os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, capture_output=True,
                       text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    res = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert res["build_flags"] == 1
    assert res["cases"] >= 20
    assert res["out_of_range"] == [], res["out_of_range"]
    assert res["not_bitwise"] == [], res["not_bitwise"]
    n, line, idx, ext = res["planted"]
    assert n > 0 and idx == 15 and ext == 8 and line > 0     # a 2H = 8 stencil


# --------------------------------------------------------------------------
# child: runs with the bounds-checked library
# --------------------------------------------------------------------------

def _child():
    from paper_2109_14340_gb300 import _build
    _build.build(debug=True)
    import oracle
    import workloads
    from helpers import oracle_params
    import paper_2109_14340_gb300 as T
    assert os.path.basename(T.lib_path()) == "libteno_gb300_debug.so"
    dev = torch.device("cuda:0")
    out = {"build_flags": T.teno_build_flags(), "cases": 0, "out_of_range": [], "not_bitwise": []}

    def gparams(c, **over):
        kw = dict(ndim=c["ndim"], n=c["n"], dx=c["dx"], scheme=c["scheme"], gamma=c["gamma"],
                  bc_lo=c["bc_lo"], bc_hi=c["bc_hi"], limiter=c.get("limiter", 0))
        keep = []
        for side in ("bc_state_lo", "bc_state_hi"):
            st = c.get(side)
            if st is not None:
                t = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                     for a in st]
                keep += t
                kw[side] = t
        kw.update(over)
        p = T.teno_params_init(**kw)
        p._keep = keep
        return p

    def check(name, ws):
        n, line, idx, ext = T.teno_debug_bounds(ws)
        if n:
            out["out_of_range"].append((name, n, line, idx, ext))

    def rhs_case(name, c, split=0, steps=1, dt_lim=0.0):
        pg = gparams(c, flux_split=split)
        po = oracle_params(c, split=split)
        s = T.Solver(pg, dev)
        U = torch.from_numpy(np.ascontiguousarray(c["U"])).to(dev)
        r, fl = s.rhs(U, dt_lim, flags=True)
        ro, fo, lo, _ = oracle.rhs(po, c["U"], dt_lim, want_flags=True)
        ok = np.array_equal(r.cpu().numpy(), ro) and \
            np.array_equal(fl.cpu().numpy()[:fo.size], fo)
        Uo = c["U"].copy()
        for _ in range(steps):
            dt = float(s.cfl_dt(U).item())
            s.step(U)
            dto, _, _ = oracle.cfl_dt(po, Uo, 0.4)
            Uo, _ = oracle.rk3_step(po, Uo, dto)
            ok = ok and dt == dto
        ok = ok and np.array_equal(U.cpu().numpy(), Uo)
        s.status()
        check(name, s.ws)
        out["cases"] += 1
        if not ok:
            out["not_bitwise"].append(name)

    for scheme in (8, 10, 12):
        for bc in (0, 1, 2, 3):
            c = workloads.riemann_1d(40, seed=1001 + bc, scheme=scheme)
            c["bc_lo"], c["bc_hi"] = [bc, 0, 0], [bc, 0, 0]
            rhs_case("1d-s%d-bc%d" % (scheme, bc), c, split=bc % 2, steps=2)
        rhs_case("2d-s%d" % scheme, workloads.quadrants_2d(24, 20, scheme=scheme), steps=2)
        c = workloads.tgv_3d(16, scheme=scheme)
        rhs_case("3d-s%d" % scheme, c, split=1)
    rhs_case("2d-dirichlet", workloads.boundary_walls(2, [33, 27], [1, 4], [3, 4], seed=6002,
                                                       scheme=10), steps=2)
    rhs_case("3d-dirichlet", workloads.boundary_walls(3, [16, 17, 18], [4, 3, 0], [2, 4, 0],
                                                       seed=6003, scheme=8))
    # limiter near vacuum, where it binds
    c = workloads.double_rarefaction_1d(64, scheme=10)
    c["limiter"] = 1
    po = oracle_params(c)
    U = c["U"].copy()
    for _ in range(4):
        dt, _, _ = oracle.cfl_dt(po, U, 0.4)
        U, _ = oracle.rk3_step(po, U, dt)
    c["U"] = U
    dt, _, _ = oracle.cfl_dt(po, U, 0.4)
    rhs_case("1d-limiter", c, dt_lim=dt)
    # halo sides of a slab decomposition
    c = workloads.tgv_3d(16, scheme=10)
    c["n"] = [16, 16, 16]
    p = gparams(c)
    s = T.Solver(p, dev)
    Ud = torch.from_numpy(c["U"]).to(dev)
    U0 = Ud.clone()
    s.cfl_dt(Ud)
    s.step(Ud)
    D = T.SlabDecomposition(p, 2, dev)
    parts = D.split(U0)
    D.cfl_dt(parts)
    D.step(parts)
    for k, sv in enumerate(D.solvers):
        sv.status()
        check("slab-%d" % k, sv.ws)
    out["cases"] += 1
    if not torch.equal(D.join(parts), Ud):
        out["not_bitwise"].append("slabs")
    # the batched face kernel (the same face code)
    cases = workloads.batched_1d(count=12, nmin=16, nmax=64)
    sizes = [cc["n"][0] for cc in cases]
    offs, total = T.pack_offsets(sizes)
    Uh = np.zeros(total)
    probs = []
    for cc, o in zip(cases, offs):
        Uh[o:o + 3 * cc["n"][0]] = cc["U"].ravel()
        probs.append(dict(n=cc["n"][0], offset=o, dx=cc["dx"][0], scheme=cc["scheme"],
                          limiter=cc.get("limiter", 0), bc_lo=1, bc_hi=1))
    B = T.Batch(T.teno_params_init(gamma=1.4), probs, dev)
    Ub = torch.from_numpy(Uh).to(dev)
    B.steps(Ub, 2, 0.4, T.TENO_BATCH_STREAM)
    torch.cuda.synchronize()
    check("batched", B.ws)
    out["cases"] += 1
    for cc, o in zip(cases, offs):
        pco = oracle_params(cc)
        Uo = cc["U"].copy()
        for _ in range(2):
            dt, _, _ = oracle.cfl_dt(pco, Uo, 0.4)
            Uo, _ = oracle.rk3_step(pco, Uo, dt)
        if not np.array_equal(Ub[o:o + 3 * cc["n"][0]].cpu().numpy().reshape(3, -1), Uo):
            out["not_bitwise"].append("batched-%d" % o)
    # the checks catch what they are for: a decision record whose splitting-
    # speed words name stencil cells beyond the stencil (15 >= 2H) makes
    # the frozen evaluation index outside the staged cells; the checked build
    # counts it and uses cell 0 instead (the release build never gets such a
    # record from its own calls)
    c = workloads.riemann_1d(40, scheme=8)
    p = gparams(c)
    s = T.Solver(p, dev)
    U = torch.from_numpy(np.ascontiguousarray(c["U"])).to(dev)
    _, rec = s.rhs(U, flags=True)
    d0, a0, l0, tot = T.record_layout(p)
    rec[a0:l0] = 0xFF
    T.teno_rhs_frozen(p, U, torch.empty_like(U), rec, s.ws)
    out["planted"] = T.teno_debug_bounds(s.ws)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    _child()
