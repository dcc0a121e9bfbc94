"""Batched mode on the GPU: many 1D problems of uneven size (schemes 8|10
mixed, some near vacuum with the limiter on) advanced in one persistent launch
per stage with per-problem CFL steps.  The CUDA-graph, direct-launch and
per-problem-launch modes must give bitwise identical states, equal to the
oracle advancing every problem on its own (same per-problem dt rule)."""
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


def pack(cases):
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


@pytest.fixture(scope="module")
def batch_case():
    cases = workloads.batched_1d(count=48, nmin=16, nmax=300)
    probs, U, offs = pack(cases)
    return cases, probs, U, offs


def test_modes_bitwise_equal_and_match_oracle(batch_case):
    cases, probs, U, offs = batch_case
    common = T.teno_params_init(gamma=1.4)
    results = {}
    for mode in (T.TENO_BATCH_GRAPH, T.TENO_BATCH_STREAM, T.TENO_BATCH_PER_PROBLEM):
        B = T.Batch(common, probs)
        Ud = torch.from_numpy(U.copy()).to(DEV)
        B.steps(Ud, 3, 0.4, mode)
        torch.cuda.synchronize()
        results[mode] = (Ud.cpu().numpy(), B.times() if mode != T.TENO_BATCH_PER_PROBLEM else None)
    g, s, p = (results[m][0] for m in (0, 1, 2))
    assert np.array_equal(g, s)
    assert np.array_equal(g, p)
    # oracle, problem by problem, same dt rule
    for k, (c, o) in enumerate(zip(cases, offs)):
        po = oracle_params(c)
        Uo = c["U"].copy()
        t = 0.0
        for _ in range(3):
            dt, _, _ = oracle.cfl_dt(po, Uo, 0.4)
            Uo, _ = oracle.rk3_step(po, Uo, dt)
            t = t + dt
        n = c["n"][0]
        assert np.array_equal(g[o:o + 3 * n].reshape(3, n), Uo), k
        assert results[0][1][k] == t


def test_autotune_keeps_results(batch_case):
    cases, probs, U, offs = batch_case
    common = T.teno_params_init(gamma=1.4)
    B = T.Batch(common, probs)
    scratch = torch.from_numpy(U.copy()).to(DEV)
    tile, bps = B.autotune(scratch)
    assert tile in (64, 128, 256) and bps in (1, 2, 4)
    Ud = torch.from_numpy(U.copy()).to(DEV)
    B.steps(Ud, 2, 0.4, T.TENO_BATCH_GRAPH)
    B2 = T.Batch(common, probs)
    Ud2 = torch.from_numpy(U.copy()).to(DEV)
    B2.steps(Ud2, 2, 0.4, T.TENO_BATCH_PER_PROBLEM)
    assert torch.equal(Ud, Ud2)


def test_graph_replay_after_new_state(batch_case):
    """The captured step follows the data (same buffers, new contents)."""
    cases, probs, U, offs = batch_case
    common = T.teno_params_init(gamma=1.4)
    B = T.Batch(common, probs)
    Ud = torch.from_numpy(U.copy()).to(DEV)
    B.steps(Ud, 1, 0.4, T.TENO_BATCH_GRAPH)
    Ud.copy_(torch.from_numpy(U))
    B.steps(Ud, 2, 0.4, T.TENO_BATCH_GRAPH)
    B2 = T.Batch(common, probs)
    Ud2 = torch.from_numpy(U.copy()).to(DEV)
    B2.steps(Ud2, 2, 0.4, T.TENO_BATCH_STREAM)
    assert torch.equal(Ud, Ud2)
