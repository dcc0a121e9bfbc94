"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point declared in include/teno.h; parameter validation and
workspace sizing (pure host logic) behave as documented."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "teno.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(teno_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_2109_14340_gb300 as T
    from paper_2109_14340_gb300 import _build
    _build.build()
    T.load()
    return T


def test_header_declares_expected_calls():
    syms = declared_symbols()
    for s in ("teno_rhs", "teno_rk3_step", "teno_cfl_dt", "teno_status", "teno_workspace_bytes",
              "teno_strerror"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(teno_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib.load(), s)


def test_defaults_are_the_papers(lib):
    p = lib.teno_params_init()
    assert (p.ct_alpha1, p.ct_alpha2, p.ct_cr) == (14.0, 6.4, 0.265)
    assert (p.eps_beta, p.eps_eta, p.q) == (1e-40, 1e-40, 7)
    assert p.scheme == 8 and p.gamma == 1.4


def test_workspace_sizing(lib):
    p = lib.teno_params_init(ndim=3, n=[16, 12, 10], dx=[0.1] * 3, scheme=10)
    nb = lib.teno_workspace_bytes(p)
    nc, cells = 5, 16 * 12 * 10
    faces = 17 * 12 * 10 + 16 * 13 * 10 + 16 * 12 * 11
    assert nb >= 8 * nc * (cells + faces) + 256
    assert lib.teno_flags_bytes(p) == faces * (nc * 2 + 2 + 1)


@pytest.mark.parametrize("bad", [
    dict(scheme=9), dict(scheme=11), dict(scheme=14), dict(scheme=12, n=[5]),
    dict(ndim=4), dict(q=2), dict(gamma=1.0), dict(n=[3]),
    dict(bc_lo=[0], bc_hi=[1]), dict(bc_lo=[5], bc_hi=[5]), dict(dx=[0.0]),
    dict(flux_split=2), dict(limiter=2), dict(ct_cr=0.0), dict(n=[64, 2]),
    dict(ndim=3, n=[8, 8, 65536], dx=[0.1] * 3), dict(ndim=2, n=[8, 65536], dx=[0.1] * 2),
])
def test_invalid_parameters(lib, bad):
    kw = dict(ndim=1, n=[64], dx=[0.1], scheme=8)
    kw.update(bad)
    p = lib.teno_params_init(**kw)
    with pytest.raises(lib.TenoError) as e:
        lib.teno_workspace_bytes(p)
    assert e.value.code == lib.TENO_EINVAL


def test_strerror(lib):
    assert "invalid" in lib.teno_strerror(lib.TENO_EINVAL)
    assert lib.teno_strerror(99) == "unknown error code"


def _probs(lib, sizes, schemes, offsets=None):
    offs, _ = lib.pack_offsets(sizes)
    offs = offsets or offs
    return [dict(n=n, offset=o, dx=1.0 / n, scheme=s, limiter=0, bc_lo=1, bc_hi=1)
            for n, s, o in zip(sizes, schemes, offs)]


def test_batch_plan_host_logic(lib):
    common = lib.teno_params_init()
    h = lib.teno_batch_create(common, _probs(lib, [64, 100, 7], [8, 10, 8]))
    try:
        nb = lib.teno_batch_workspace_bytes(h)
        faces = 65 + 101 + 8
        assert nb > 8 * 3 * (faces + 64 + 100 + 7)
    finally:
        lib.teno_batch_destroy(h)


def test_twelve_point_scheme_accepted(lib):
    """scheme 12 (TENO12-AA) is valid with n >= 6 on every used axis."""
    for kw in (dict(ndim=1, n=[6], dx=[0.1]), dict(ndim=3, n=[6, 7, 8], dx=[0.1] * 3)):
        p = lib.teno_params_init(scheme=12, **kw)
        assert lib.teno_workspace_bytes(p) > 0


@pytest.mark.parametrize("bad", ["overlap", "odd_offset", "too_small", "scheme", "scheme12"])
def test_batch_plan_rejects(lib, bad):
    common = lib.teno_params_init()
    sizes, schemes, offs = [64, 64], [8, 10], None
    if bad == "overlap":
        offs = [0, 100]
    elif bad == "odd_offset":
        offs = [0, 193]
    elif bad == "too_small":
        sizes = [64, 4]
    elif bad == "scheme":
        schemes = [8, 9]
    elif bad == "scheme12":            # batched mode runs the 8/10-point schemes only
        schemes = [8, 12]
    with pytest.raises(lib.TenoError) as e:
        lib.teno_batch_create(common, _probs(lib, sizes, schemes, offs))
    assert e.value.code == lib.TENO_EINVAL
