"""teno_rhs_static -- the right-hand side for callers that cannot allocate
device memory (plugins in applications that own the memory pool, fixed
memory budgets, code running under CUDA graph capture).  Its scratch is one
fixed device array inside the library.

The test calls it through the C ABI twice in a row (different inputs, so the
second call must not see the first call's leftovers) and compares each result
with teno_rhs on a workspace, with the same tolerance and bitwise expectation
as the rest of the GPU suite.  It also checks that an oversized grid is
rejected before any work is enqueued.  This file is collected last."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2109_14340_gb300 as T  # noqa: E402

DEV = torch.device("cuda:0")


def _params(case, limiter=0):
    return T.teno_params_init(ndim=case["ndim"], n=case["n"], dx=case["dx"],
                              scheme=case["scheme"], gamma=case["gamma"], bc_lo=case["bc_lo"],
                              bc_hi=case["bc_hi"], limiter=limiter)


def _rel(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return float((np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)).max())


@pytest.mark.parametrize("cases", [
    ("1d", lambda: workloads.riemann_1d(400, scheme=8), lambda: workloads.riemann_1d(400, seed=1007, scheme=8)),
    ("2d", lambda: workloads.quadrants_2d(64, 48, scheme=10), lambda: workloads.quadrants_2d(64, 48, seed=2002, scheme=10)),
    ("3d", lambda: workloads.tgv_3d(24, scheme=10), lambda: workloads.tgv_3d(24, seed=3002, scheme=10)),
], ids=lambda c: c[0])
def test_static_matches_workspace_twice(cases):
    _, first, second = cases
    for make in (first, second):
        case = make()
        p = _params(case)
        U = torch.from_numpy(np.ascontiguousarray(case["U"])).to(DEV)
        ws = torch.zeros((T.teno_workspace_bytes(p) + 7) // 8, dtype=torch.float64, device=DEV)
        ref = torch.empty_like(U)
        fl_ref = torch.zeros(T.teno_flags_bytes(p), dtype=torch.uint8, device=DEV)
        T.teno_rhs(p, U, ref, 0.0, fl_ref, ws)
        out = torch.full_like(U, float("nan"))
        fl = torch.zeros_like(fl_ref)
        T.teno_rhs_static(p, U, out, 0.0, fl)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert _rel(a, b) <= 1e-12
        assert np.array_equal(a, b)
        assert torch.equal(fl, fl_ref)


def test_static_with_limiter_twice():
    cases = workloads.batched_1d(count=200, nmin=64, nmax=200)
    for which in (10, 117):
        case = cases[which]
        p = _params(case, limiter=1)
        U = torch.from_numpy(np.ascontiguousarray(case["U"])).to(DEV)
        ws = torch.zeros((T.teno_workspace_bytes(p) + 7) // 8, dtype=torch.float64, device=DEV)
        ref = torch.empty_like(U)
        T.teno_rhs(p, U, ref, 1e-4, None, ws)
        out = torch.empty_like(U)
        T.teno_rhs_static(p, U, out, 1e-4, None)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_static_rejects_oversized_grid():
    p = T.teno_params_init(ndim=3, n=[128, 128, 128], dx=[0.1] * 3, scheme=10)
    U = torch.ones(5, 128 ** 3, dtype=torch.float64, device=DEV)
    out = torch.empty_like(U)
    with pytest.raises(ValueError):
        T.teno_rhs_static(p, U, out)
    code = T.load().teno_rhs_static(T.ctypes.byref(p), T._ptr(U), T._ptr(out), 0.0, None,
                                    T._stream(None))
    assert code == T.TENO_EINVAL
