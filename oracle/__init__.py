"""TENO-AA CPU oracle -- test infrastructure only.

A plain FP64 C restatement of the TENO-AA method (arXiv 2109.14340, Secs. 2-5
and App. A) and this thin ctypes wrapper around it.  Only the tests, the smoke
check (``__graft_entry__.smoke``) and the benchmark's CPU-baseline / reference
leg may import this package; the CUDA library never does, and the two share no
code.

Parity pins live in ``tests/test_oracle_*.py``.  Parity unpinned: the exact
formula of the positivity-preserving limiter (Sec. 5.3 cites it without stating
it); only its invariants (positivity, theta = 1 on smooth data) are pinned.
The twelve-point candidate S6 (``teno12_derive.py``) is not printed; its
recipe is pinned on the printed S3-S5 and its result on order, optimality and
the exact indicator derivation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "teno_oracle.c")
_TABLES = os.path.join(_HERE, "teno12_tables.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libteno_oracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_TRANSMISSIVE, BC_SLIPWALL, BC_NOSLIP, BC_DIRICHLET = 0, 1, 2, 3, 4
SPLIT_LLF, SPLIT_RUSANOV = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE division/sqrt)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_TABLES))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Oracle-private parameter block (mirrors ``or_params`` in teno_oracle.c)."""
    _fields_ = [
        ("ndim", ctypes.c_int32), ("scheme", ctypes.c_int32),
        ("split", ctypes.c_int32), ("limiter", ctypes.c_int32),
        ("n", ctypes.c_int64 * 3), ("dx", ctypes.c_double * 3),
        ("gamma", ctypes.c_double), ("alpha1", ctypes.c_double),
        ("alpha2", ctypes.c_double), ("cr", ctypes.c_double),
        ("eps_beta", ctypes.c_double), ("eps_eta", ctypes.c_double),
        ("lim_eps", ctypes.c_double),
        ("bc_lo", ctypes.c_int32 * 3), ("bc_hi", ctypes.c_int32 * 3),
        ("bc_state_lo", ctypes.c_void_p * 3), ("bc_state_hi", ctypes.c_void_p * 3),
    ]


def params(ndim, n, dx, scheme=8, gamma=1.4, bc=BC_PERIODIC, bc_lo=None, bc_hi=None,
           split=SPLIT_LLF, limiter=0, alpha1=14.0, alpha2=6.4, cr=0.265,
           eps_beta=1e-40, eps_eta=1e-40, lim_eps=1e-13, bc_state_lo=None,
           bc_state_hi=None) -> Params:
    """Parameter block with the paper's built-in values as defaults (Sec. 3.2,
    Sec. 3.4: eps = 1e-40, q = 7, C_r = 0.265, alpha1 = 14, alpha2 = 6.4).
    bc_state_lo / bc_state_hi: per axis None or the BC_DIRICHLET boundary-face
    primitives (rho, u..., p) as an array [ndim + 2][faces of the side, other
    axes x fastest] (App. A.3); the block keeps them alive."""
    p = Params()
    p._keep = []
    for name, states in (("bc_state_lo", bc_state_lo), ("bc_state_hi", bc_state_hi)):
        states = list(states or []) + [None] * 3
        for a in range(3):
            if states[a] is not None:
                arr = np.ascontiguousarray(states[a], np.float64)
                p._keep.append(arr)
                getattr(p, name)[a] = arr.ctypes.data
    p.ndim, p.scheme, p.split, p.limiter = ndim, scheme, split, limiter
    n = list(n) + [1] * (3 - len(n))
    dx = list(dx) + [1.0] * (3 - len(dx))
    for a in range(3):
        p.n[a] = int(n[a])
        p.dx[a] = float(dx[a])
    lo = list(bc_lo) if bc_lo is not None else [bc] * 3
    hi = list(bc_hi) if bc_hi is not None else [bc] * 3
    lo, hi = lo + [bc] * (3 - len(lo)), hi + [bc] * (3 - len(hi))
    for a in range(3):
        p.bc_lo[a], p.bc_hi[a] = int(lo[a]), int(hi[a])
    p.gamma, p.alpha1, p.alpha2, p.cr = gamma, alpha1, alpha2, cr
    p.eps_beta, p.eps_eta, p.lim_eps = eps_beta, eps_eta, lim_eps
    return p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(Params)
            dp = ctypes.POINTER(ctypes.c_double)
            u8 = ctypes.POINTER(ctypes.c_uint8)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_rhs.argtypes = [P, dp, dp, ctypes.c_double, u8, u8, ctypes.c_int]
            lib.oracle_rhs.restype = ctypes.c_int64
            lib.oracle_rk3_step.argtypes = [P, dp, ctypes.c_double, ctypes.c_int]
            lib.oracle_rk3_step.restype = ctypes.c_int64
            lib.oracle_cfl_dt.argtypes = [P, dp, ctypes.c_double, dp, i64p]
            lib.oracle_cfl_dt.restype = ctypes.c_double
            lib.oracle_rk3_combine.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, dp,
                                               ctypes.c_double, dp]
            lib.oracle_rhs_at.argtypes = [P, dp, i64p, ctypes.c_int64, ctypes.c_double, dp,
                                          ctypes.c_int]
            lib.oracle_teno_recon.argtypes = [P, dp, u8]
            lib.oracle_teno_recon.restype = ctypes.c_double
            lib.oracle_eigensystem.argtypes = [P, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_eigensystem.restype = ctypes.c_double
            lib.oracle_round_ratio.argtypes = [ctypes.c_char_p, ctypes.c_char_p]
            lib.oracle_round_ratio.restype = ctypes.c_double
            lib.oracle_beta_coef.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_beta_coef.restype = ctypes.c_double
            lib.oracle_lin_coef.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_lin_coef.restype = ctypes.c_double
            ci = ctypes.POINTER(ctypes.c_int)
            cs = ctypes.POINTER(ctypes.c_char_p)
            lib.oracle_beta_terms.argtypes = [ctypes.c_int, ctypes.c_int, ci, ci, cs, cs]
            lib.oracle_beta_terms.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_betas.argtypes = [P, dp, dp, dp]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def ncons(p: Params) -> int:
    return p.ndim + 2


def ncells(p: Params) -> int:
    return p.n[0] * p.n[1] * p.n[2]


def flags_size(p: Params) -> int:
    """Bytes of the per-face decision record: per direction, per face of the
    face grid, per characteristic field, per sign."""
    tot = 0
    for d in range(p.ndim):
        fn = [p.n[0], p.n[1], p.n[2]]
        fn[d] += 1
        tot += fn[0] * fn[1] * fn[2] * ncons(p) * 2
    return tot


def lim_flags_size(p: Params) -> int:
    tot = 0
    for d in range(p.ndim):
        fn = [p.n[0], p.n[1], p.n[2]]
        fn[d] += 1
        tot += fn[0] * fn[1] * fn[2]
    return tot


def _state(p, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.size == ncons(p) * ncells(p), (U.shape, ncons(p), ncells(p))
    return U


def max_threads() -> int:
    return _load().oracle_max_threads()


def rhs(p: Params, U, dt_lim: float = 0.0, want_flags: bool = False, threads: int = 1):
    """Semi-discrete right-hand side L(U) (Eq. approximateEq, dimension by
    dimension).  Returns (rhs, flags or None, lim_flags or None, nonphysical)."""
    lib = _load()
    U = _state(p, U)
    out = np.empty_like(U)
    fl = np.zeros(flags_size(p), np.uint8) if want_flags else None
    lf = np.zeros(lim_flags_size(p), np.uint8) if want_flags else None
    nb = lib.oracle_rhs(ctypes.byref(p), _dp(U), _dp(out), float(dt_lim),
                        _u8(fl) if fl is not None else None,
                        _u8(lf) if lf is not None else None, int(threads))
    return out, fl, lf, int(nb)


def rk3_step(p: Params, U, dt: float, threads: int = 1):
    """One SSP-RK3 step (Eq. Runge-kutta).  Returns (U_new, nonphysical)."""
    lib = _load()
    U = _state(p, U).copy()
    nb = lib.oracle_rk3_step(ctypes.byref(p), _dp(U), float(dt), int(threads))
    return U, int(nb)


def cfl_dt(p: Params, U, cfl: float = 0.4):
    """dt = cfl / sum_d max(|u_d| + c) / dx_d.  Returns (dt, A[3], nonphysical)."""
    lib = _load()
    U = _state(p, U)
    A = np.zeros(3)
    nb = ctypes.c_int64(0)
    dt = lib.oracle_cfl_dt(ctypes.byref(p), _dp(U), float(cfl), _dp(A), ctypes.byref(nb))
    return dt, A, int(nb.value)


def rk3_combine(stage: int, Un, Uk, L, dt: float):
    lib = _load()
    Un = np.ascontiguousarray(Un, np.float64)
    Uk = np.ascontiguousarray(Uk, np.float64)
    L = np.ascontiguousarray(L, np.float64)
    out = np.empty_like(Un)
    lib.oracle_rk3_combine(int(stage), Un.size, _dp(Un), _dp(Uk), _dp(L), float(dt), _dp(out))
    return out


def rhs_at(p: Params, U, cells, dt_lim: float = 0.0, threads: int = 1):
    """L(U) at the listed linear cell indices only; returns (ncons, len(cells))."""
    lib = _load()
    U = _state(p, U)
    cells = np.ascontiguousarray(cells, np.int64)
    out = np.empty((ncons(p), cells.size))
    lib.oracle_rhs_at(ctypes.byref(p), _dp(U),
                      cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cells.size,
                      float(dt_lim), _dp(out), int(threads))
    return out


def half_width(p: Params) -> int:
    """H = 4, 5, 6 for TENO8, TENO10, TENO12-AA."""
    return {8: 4, 10: 5, 12: 6}[p.scheme]


def recon(p: Params, v):
    """Scalar TENO-AA reconstruction at face i+1/2 from v at offsets -H+1..H.
    Returns (value, flag byte)."""
    lib = _load()
    H = half_width(p)
    v = np.ascontiguousarray(v, np.float64)
    assert v.size == 2 * H
    fl = np.zeros(1, np.uint8)
    val = lib.oracle_teno_recon(ctypes.byref(p), _dp(v), _u8(fl))
    return float(val), int(fl[0])


def eigensystem(p: Params, d: int, UL, UR):
    lib = _load()
    nc = ncons(p)
    UL = np.ascontiguousarray(UL, np.float64)
    UR = np.ascontiguousarray(UR, np.float64)
    Lm = np.zeros((nc, nc))
    Rm = np.zeros((nc, nc))
    c2 = lib.oracle_eigensystem(ctypes.byref(p), int(d), _dp(UL), _dp(UR), _dp(Lm), _dp(Rm))
    return Lm, Rm, c2


def round_ratio(num: int, den: int) -> float:
    return _load().oracle_round_ratio(str(num).encode(), str(den).encode())


def beta_terms(width: int):
    """The printed integer terms (a, b, coefficient) and denominator of the
    width-point smoothness indicator (6, 8, 10), as the oracle transcribed
    them."""
    assert width in (6, 8, 10)
    lib = _load()
    a, b = ctypes.c_int(), ctypes.c_int()
    c, den = ctypes.c_char_p(), ctypes.c_char_p()
    nt = lib.oracle_beta_terms(width, -1, ctypes.byref(a), ctypes.byref(b),
                               ctypes.byref(c), ctypes.byref(den))
    terms = []
    for i in range(nt):
        lib.oracle_beta_terms(width, i, ctypes.byref(a), ctypes.byref(b),
                              ctypes.byref(c), ctypes.byref(den))
        terms.append((a.value, b.value, int(c.value.decode())))
    return terms, int(den.value.decode())


def beta_fractions(width: int):
    """Terms (a, b, Fraction) of the width-point indicator as the oracle
    holds them: the printed ones (6, 8, 10) or the derived beta_{6,12}."""
    from fractions import Fraction
    if width != 12:
        terms, den = beta_terms(width)
        return [(a, b, Fraction(c, den)) for a, b, c in terms]
    lib = _load()
    a, b = ctypes.c_int(), ctypes.c_int()
    c, den = ctypes.c_char_p(), ctypes.c_char_p()
    nt = lib.oracle_beta_terms(12, -1, ctypes.byref(a), ctypes.byref(b),
                               ctypes.byref(c), ctypes.byref(den))
    out = []
    for i in range(nt):
        lib.oracle_beta_terms(12, i, ctypes.byref(a), ctypes.byref(b),
                              ctypes.byref(c), ctypes.byref(den))
        out.append((a.value, b.value, Fraction(int(c.value.decode()), int(den.value.decode()))))
    return out


def lin_coef(L: int, off: int) -> float:
    """Coefficient of the large stencil S_L's linear scheme at offset off."""
    return _load().oracle_lin_coef(L, off)


def betas(p: Params, v):
    """(beta_0..beta_6, fhat_0..fhat_6) of one stencil v at offsets -H+1..H
    (entries above L = H are zero)."""
    lib = _load()
    H = half_width(p)
    v = np.ascontiguousarray(v, np.float64)
    assert v.size == 2 * H
    b = np.zeros(7)
    f = np.zeros(7)
    lib.oracle_betas(ctypes.byref(p), _dp(v), _dp(b), _dp(f))
    return b, f


def beta_coef(width: int, r: int, s: int) -> float:
    return _load().oracle_beta_coef(width, r, s)


def decode_flag(fl: int):
    """(selected large stencil 3|4|5|6 or 0 for the small-stencil fallback,
    (delta0, delta1, delta2), C_T exponent).  Bits 0-4 all zero mean S6."""
    sel = fl & 3
    ct = ((fl >> 5) & 7) + 7
    if (fl & 31) == 0:
        return 6, (0, 0, 0), ct
    return (sel + 2 if sel else 0, ((fl >> 2) & 1, (fl >> 3) & 1, (fl >> 4) & 1), ct)
