"""Python binding of the GB300 TENO-AA library (C ABI in include/teno.h).

Argument marshalling only: every step of the right-hand side, the RK3 step and
the CFL reduction runs in the sm_103a kernels of libteno_gb300.so.  PyTorch
supplies device memory (CUDA tensors) and streams.  There is no CPU fallback:
if the shared library is missing the calls raise.

The function names mirror the C entry points:
  teno_params_init, teno_workspace_bytes, teno_flags_bytes, teno_rhs,
  teno_rk3_step, teno_cfl_dt, teno_status, teno_advance_host, teno_strerror.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

TENO_OK, TENO_EINVAL, TENO_ECUDA, TENO_ENONPHYSICAL, TENO_ETIMEOUT, TENO_EBOUNDS = 0, 1, 2, 3, 4, 5
TENO_BC_PERIODIC, TENO_BC_TRANSMISSIVE, TENO_BC_SLIPWALL = 0, 1, 2
TENO_BC_NOSLIP, TENO_BC_DIRICHLET, TENO_BC_HALO = 3, 4, 5
TENO_SPLIT_LLF, TENO_SPLIT_RUSANOV = 0, 1

_lock = threading.Lock()
_lib = None


class TenoError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (code %d)" % (what, teno_strerror(code), code))
        self.code = code


TENO_BATCH_GRAPH, TENO_BATCH_STREAM, TENO_BATCH_PER_PROBLEM = 0, 1, 2


class teno_batch_problem(ctypes.Structure):
    """Mirror of struct teno_batch_problem (include/teno.h)."""
    _fields_ = [("n", ctypes.c_int64), ("offset", ctypes.c_int64), ("dx", ctypes.c_double),
                ("scheme", ctypes.c_int32), ("limiter", ctypes.c_int32),
                ("bc_lo", ctypes.c_int32), ("bc_hi", ctypes.c_int32)]


class teno_params(ctypes.Structure):
    """Mirror of struct teno_params (include/teno.h)."""
    _fields_ = [
        ("ndim", ctypes.c_int32), ("scheme", ctypes.c_int32),
        ("flux_split", ctypes.c_int32), ("limiter", ctypes.c_int32),
        ("n", ctypes.c_int64 * 3), ("dx", ctypes.c_double * 3),
        ("gamma", ctypes.c_double), ("ct_alpha1", ctypes.c_double),
        ("ct_alpha2", ctypes.c_double), ("ct_cr", ctypes.c_double),
        ("eps_beta", ctypes.c_double), ("eps_eta", ctypes.c_double),
        ("limiter_eps", ctypes.c_double), ("q", ctypes.c_int32),
        ("bc_lo", ctypes.c_int32 * 3), ("bc_hi", ctypes.c_int32 * 3),
        ("reserved", ctypes.c_int32),
        ("bc_state_lo", ctypes.c_void_p * 3), ("bc_state_hi", ctypes.c_void_p * 3),
    ]


def lib_path() -> str:
    """The library load() opens: the bounds-checked build when the
    environment sets TENO_GB300_DEBUG=1 (built by _build.build(debug=True)),
    else the release build."""
    return _build.DEBUG_LIB if os.environ.get("TENO_GB300_DEBUG") == "1" else _build.LIB


def load():
    """Load libteno_gb300.so (build it first with build()); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("%s is not built (run __graft_entry__.build() or "
                               "paper_2109_14340_gb300._build.build()); there is no fallback"
                               % os.path.basename(path))
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER(teno_params)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        lib.teno_params_init.argtypes = [P]
        lib.teno_params_init.restype = None
        lib.teno_workspace_bytes.argtypes = [P, ctypes.POINTER(sz)]
        lib.teno_flags_bytes.argtypes = [P, ctypes.POINTER(sz)]
        lib.teno_rhs.argtypes = [P, vp, vp, ctypes.c_double, vp, vp, sz, vp]
        lib.teno_rk3_step.argtypes = [P, vp, ctypes.c_double, vp, vp, sz, vp]
        lib.teno_cfl_dt.argtypes = [P, vp, ctypes.c_double, vp, vp, sz, vp]
        lib.teno_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int64)]
        lib.teno_advance_host.argtypes = [P, vp, vp, ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double), vp, sz, vp]
        lib.teno_rhs_static.argtypes = [P, vp, vp, ctypes.c_double, vp, vp]
        lib.teno_rk3_stage.argtypes = [P, ctypes.c_int, vp, vp, ctypes.c_double, vp, vp, sz, vp]
        lib.teno_wave_speeds.argtypes = [P, vp, vp, vp, sz, vp]
        lib.teno_dt_from_speeds.argtypes = [P, vp, ctypes.c_int32, ctypes.c_double, vp, vp]
        u8p = ctypes.c_void_p
        lib.teno_adjoint_workspace_bytes.argtypes = [P, ctypes.POINTER(sz)]
        lib.teno_rhs_vjp.argtypes = [P, vp, vp, vp, vp, vp, sz, vp]
        lib.teno_rk3_step_record.argtypes = [P, vp, ctypes.c_double, vp, vp, u8p, vp, sz, vp]
        lib.teno_rk3_step_record_sel.argtypes = [P, vp, ctypes.c_double, vp, vp, u8p, vp, sz, vp]
        lib.teno_rk3_step_vjp.argtypes = [P, vp, vp, vp, u8p, ctypes.c_double, vp, vp, sz, vp]
        lib.teno_rhs_frozen.argtypes = [P, vp, vp, ctypes.c_double, u8p, vp, sz, vp]
        lib.teno_rk3_step_frozen.argtypes = [P, vp, ctypes.c_double, u8p, vp, sz, vp]
        BP = ctypes.POINTER(teno_batch_problem)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.teno_batch_create.argtypes = [P, BP, ctypes.c_int32, ctypes.POINTER(vp)]
        lib.teno_batch_workspace_bytes.argtypes = [vp, ctypes.POINTER(sz)]
        lib.teno_batch_autotune.argtypes = [vp, vp, vp, sz, vp, i32p, i32p]
        lib.teno_batch_rk3_steps.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_int32, vp, sz, vp]
        lib.teno_batch_times.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
        lib.teno_batch_destroy.argtypes = [vp]
        lib.teno_batch_destroy.restype = None
        lib.teno_profile_enable.argtypes = [ctypes.c_int]
        lib.teno_set_decision_filter.argtypes = [ctypes.c_int]
        lib.teno_reconstruct.argtypes = [P, vp, ctypes.c_int64, vp, vp, vp]
        lib.teno_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.teno_debug_bounds.argtypes = [vp, vp, i64p, i64p, i64p, i64p]
        lib.teno_build_flags.argtypes = []
        lib.teno_strerror.argtypes = [ctypes.c_int]
        lib.teno_strerror.restype = ctypes.c_char_p
        for name in ("teno_workspace_bytes", "teno_flags_bytes", "teno_rhs", "teno_rk3_step",
                     "teno_cfl_dt", "teno_status", "teno_advance_host", "teno_profile_enable",
                     "teno_profile_read", "teno_set_decision_filter", "teno_reconstruct", "teno_rhs_static", "teno_batch_create",
                     "teno_batch_workspace_bytes", "teno_batch_autotune", "teno_batch_rk3_steps",
                     "teno_batch_times", "teno_adjoint_workspace_bytes", "teno_rhs_vjp",
                     "teno_rk3_step_record", "teno_rk3_step_record_sel", "teno_rk3_step_vjp",
                     "teno_rhs_frozen", "teno_rk3_step_frozen", "teno_rk3_stage", "teno_wave_speeds",
                     "teno_dt_from_speeds", "teno_debug_bounds", "teno_build_flags"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


EXPORTS = ("teno_params_init", "teno_workspace_bytes", "teno_flags_bytes", "teno_rhs",
           "teno_rk3_step", "teno_cfl_dt", "teno_status", "teno_advance_host",
           "teno_profile_enable", "teno_profile_read", "teno_strerror", "teno_rhs_static",
           "teno_set_decision_filter", "teno_reconstruct",
           "teno_batch_create", "teno_batch_workspace_bytes", "teno_batch_autotune",
           "teno_batch_rk3_steps", "teno_batch_times", "teno_batch_destroy",
           "teno_adjoint_workspace_bytes", "teno_rhs_vjp", "teno_rk3_step_record",
           "teno_rk3_step_record_sel", "teno_rk3_step_vjp", "teno_rhs_frozen", "teno_rk3_step_frozen",
           "teno_rk3_stage", "teno_wave_speeds", "teno_dt_from_speeds", "teno_debug_bounds",
           "teno_build_flags")

TENO_RHS_STATIC_SCRATCH_BYTES = 16 << 20


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


def _check(code, what):
    if code != TENO_OK:
        raise TenoError(code, what)


def teno_strerror(code: int) -> str:
    return load().teno_strerror(int(code)).decode()


def teno_params_init(**kw) -> teno_params:
    """Paper defaults (Sec. 3.2, 3.4), then keyword overrides.  Sequences for
    n, dx, bc_lo, bc_hi are padded to three axes (n: 1, dx: 1.0, bc: 0).
    bc_state_lo / bc_state_hi: per axis a device tensor (or None) holding the
    TENO_BC_DIRICHLET boundary-face primitives, [ndim + 2][faces of the side]
    (include/teno.h); the caller keeps the tensors alive while p is used."""
    p = teno_params()
    load().teno_params_init(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("bc_state_lo", "bc_state_hi"):
            v = list(v) + [None] * (3 - len(v))
            arr = getattr(p, k)
            for i in range(3):
                if v[i] is None or isinstance(v[i], int):
                    arr[i] = v[i]
                else:
                    arr[i] = _ptr(v[i]).value
        elif k in ("n", "dx", "bc_lo", "bc_hi"):
            v = list(v)
            pad = {"n": 1, "dx": 1.0, "bc_lo": 0, "bc_hi": 0}[k]
            v = v + [pad] * (3 - len(v))
            arr = getattr(p, k)
            for i in range(3):
                arr[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def teno_workspace_bytes(p: teno_params) -> int:
    n = ctypes.c_size_t()
    _check(load().teno_workspace_bytes(ctypes.byref(p), ctypes.byref(n)), "teno_workspace_bytes")
    return n.value


def teno_flags_bytes(p: teno_params) -> int:
    n = ctypes.c_size_t()
    _check(load().teno_flags_bytes(ctypes.byref(p), ctypes.byref(n)), "teno_flags_bytes")
    return n.value


def record_layout(p: teno_params):
    """Byte offsets of the three parts of a decision record (include/teno.h,
    teno_flags_bytes): (decision bytes, argmax words, limiter bytes, total)."""
    nc = p.ndim + 2
    faces = 0
    for d in range(p.ndim):
        m = 1
        for a in range(3):
            m *= p.n[a] + (1 if a == d else 0)
        faces += m
    return 0, faces * nc * 2, faces * nc * 2 + 2 * faces, faces * (nc * 2 + 3)


def teno_rhs(p, U, rhs, dt_limiter=0.0, flags=None, ws=None, stream=None):
    _check(load().teno_rhs(ctypes.byref(p), _ptr(U), _ptr(rhs), float(dt_limiter), _ptr(flags),
                           _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "teno_rhs")


def teno_rhs_static(p, U, rhs, dt_limiter=0.0, flags=None, stream=None):
    """teno_rhs for callers that cannot allocate: scratch comes from the
    library's fixed device array (TENO_RHS_STATIC_SCRATCH_BYTES).  Calls that
    overlap on the GPU race on that array; serialise them."""
    teno_workspace_bytes(p)                   # validates p
    a256 = lambda x: (x + 255) // 256 * 256
    need = 256 + sum(a256(8 * (p.ndim + 2) * (p.n[0] + (d == 0)) * (p.n[1] + (d == 1)) *
                          (p.n[2] + (d == 2))) for d in range(p.ndim))
    if need > TENO_RHS_STATIC_SCRATCH_BYTES:
        raise ValueError("teno_rhs_static: this grid needs about %d bytes of scratch but the "
                         "static array holds %d; use teno_rhs with a workspace"
                         % (need, TENO_RHS_STATIC_SCRATCH_BYTES))
    _check(load().teno_rhs_static(ctypes.byref(p), _ptr(U), _ptr(rhs), float(dt_limiter),
                                  _ptr(flags), _stream(stream)), "teno_rhs_static")


def teno_rk3_step(p, U, dt=0.0, dt_device=None, ws=None, stream=None):
    _check(load().teno_rk3_step(ctypes.byref(p), _ptr(U), float(dt), _ptr(dt_device), _ptr(ws),
                                ws.numel() * ws.element_size(), _stream(stream)), "teno_rk3_step")


def teno_rk3_stage(p, stage, U, Us, dt=0.0, dt_device=None, ws=None, stream=None):
    _check(load().teno_rk3_stage(ctypes.byref(p), int(stage), _ptr(U), _ptr(Us), float(dt),
                                 _ptr(dt_device), _ptr(ws), ws.numel() * ws.element_size(),
                                 _stream(stream)), "teno_rk3_stage")


def teno_wave_speeds(p, U, amax_device, ws, stream=None):
    _check(load().teno_wave_speeds(ctypes.byref(p), _ptr(U), _ptr(amax_device), _ptr(ws),
                                   ws.numel() * ws.element_size(), _stream(stream)),
           "teno_wave_speeds")


def teno_dt_from_speeds(p, amax_device, ncopies, cfl, dt_device, stream=None):
    _check(load().teno_dt_from_speeds(ctypes.byref(p), _ptr(amax_device), int(ncopies),
                                      float(cfl), _ptr(dt_device), _stream(stream)),
           "teno_dt_from_speeds")


def teno_cfl_dt(p, U, cfl, dt_device, ws=None, stream=None):
    _check(load().teno_cfl_dt(ctypes.byref(p), _ptr(U), float(cfl), _ptr(dt_device), _ptr(ws),
                              ws.numel() * ws.element_size(), _stream(stream)), "teno_cfl_dt")


def teno_debug_bounds(ws, stream=None):
    """(count, source line, index, extent) of the out-of-range accesses the
    bounds-checked build recorded in this workspace (cleared by the call)."""
    c, l, i, e = (ctypes.c_int64() for _ in range(4))
    code = load().teno_debug_bounds(_ptr(ws), _stream(stream), ctypes.byref(c), ctypes.byref(l),
                                    ctypes.byref(i), ctypes.byref(e))
    if code not in (TENO_OK, TENO_EBOUNDS):
        raise TenoError(code, "teno_debug_bounds")
    return c.value, l.value, i.value, e.value


def teno_build_flags() -> int:
    return int(load().teno_build_flags())


def teno_status(ws, stream=None):
    """Synchronise; return the non-physical count (and clear it)."""
    n = ctypes.c_int64()
    code = load().teno_status(_ptr(ws), _stream(stream), ctypes.byref(n))
    if code not in (TENO_OK, TENO_ENONPHYSICAL):
        raise TenoError(code, "teno_status")
    return int(n.value)


def teno_advance_host(p, U_host, U_dev, nsteps, cfl, ws, stream=None):
    """U_host: contiguous CPU float64 tensor (pinned for full copy speed)."""
    t = ctypes.c_double()
    if U_host.is_cuda or not U_host.is_contiguous():
        raise ValueError("U_host must be a contiguous CPU tensor")
    _check(load().teno_advance_host(ctypes.byref(p), ctypes.c_void_p(U_host.data_ptr()),
                                    _ptr(U_dev), int(nsteps), float(cfl), ctypes.byref(t),
                                    _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "teno_advance_host")
    return t.value


def teno_reconstruct(p, v, out, flags=None, stream=None):
    """v: CUDA float64 [count, scheme]; out: [count]; flags: uint8 [count]."""
    _check(load().teno_reconstruct(ctypes.byref(p), _ptr(v), v.shape[0], _ptr(out), _ptr(flags),
                                   _stream(stream)), "teno_reconstruct")


def teno_set_decision_filter(on: bool = True):
    _check(load().teno_set_decision_filter(1 if on else 0), "teno_set_decision_filter")


def teno_profile_enable(on: bool = True):
    _check(load().teno_profile_enable(1 if on else 0), "teno_profile_enable")


def teno_profile_read():
    """(milliseconds, launches, faces, exact-path reconstructions) of the
    recorded face-sweep launches."""
    ms = ctypes.c_double()
    nl = ctypes.c_int64()
    nf = ctypes.c_int64()
    ne = ctypes.c_int64()
    _check(load().teno_profile_read(ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(nf),
                                    ctypes.byref(ne)), "teno_profile_read")
    return ms.value, nl.value, nf.value, ne.value


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Solver:
    """Owns a workspace (and a device dt scalar) for one parameter set."""

    def __init__(self, p: teno_params, device="cuda"):
        import torch
        self.p = p
        self.device = torch.device(device)
        nb = teno_workspace_bytes(p)
        self.ws = torch.zeros((nb + 7) // 8, dtype=torch.float64, device=self.device)
        self.dt = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.ncons = p.ndim + 2
        self.ncells = p.n[0] * p.n[1] * p.n[2]

    def rhs(self, U, dt_limiter=0.0, flags=False, stream=None):
        import torch
        out = torch.empty_like(U)
        fl = None
        if flags:
            fl = torch.zeros(teno_flags_bytes(self.p), dtype=torch.uint8, device=self.device)
        teno_rhs(self.p, U, out, dt_limiter, fl, self.ws, stream)
        return (out, fl) if flags else out

    def cfl_dt(self, U, cfl=0.4, stream=None):
        teno_cfl_dt(self.p, U, cfl, self.dt, self.ws, stream)
        return self.dt

    def step(self, U, dt=None, stream=None):
        """One RK3 step in place; dt=None uses the device scalar self.dt."""
        if dt is None:
            teno_rk3_step(self.p, U, 0.0, self.dt, self.ws, stream)
        else:
            teno_rk3_step(self.p, U, float(dt), None, self.ws, stream)

    def status(self, stream=None):
        return teno_status(self.ws, stream)


# ---------------------------------------------------------------------------
# domain decomposition: slabs along the slowest axis exchanging halo planes
# ---------------------------------------------------------------------------

def slab_plan(n_axis, parts, H, periodic):
    """Split n_axis cells into `parts` slabs (sizes differ by at most one).
    Returns per slab (start, stop, lo, hi): lo / hi the neighbouring slab
    whose cells fill the halo on that side, or None at a physical end.
    Every slab needs at least H cells, so its halo comes from one neighbour."""
    if parts < 1 or n_axis < parts * H:
        raise ValueError("cannot split %d cells into %d slabs of at least %d" % (n_axis, parts, H))
    base, extra = divmod(n_axis, parts)
    plan, start = [], 0
    for k in range(parts):
        size = base + (1 if k < extra else 0)
        lo = k - 1 if k > 0 else (parts - 1 if periodic else None)
        hi = k + 1 if k < parts - 1 else (0 if periodic else None)
        plan.append((start, start + size, lo, hi))
        start += size
    return plan


def halo_planes(U, n_slab, m, H, side):
    """The H boundary planes of a slab state U ([nc][n_slab * m], the slab
    axis slowest) that a neighbour needs: its first H planes ('lo') or its
    last H planes ('hi'), as a [nc][H * m] view."""
    V = U.view(U.shape[0], n_slab * m)
    return V[:, :H * m] if side == "lo" else V[:, (n_slab - H) * m:]


def exchange_halos_dist(U, n_slab, m, H, halo_lo, halo_hi, lo, hi, group=None):
    """Halo exchange of one slab with its neighbouring ranks through
    torch.distributed (any backend; the tests run gloo with host tensors):
    send the first / last H planes to the lo / hi neighbour, receive the
    neighbours' planes into halo_lo / halo_hi ([nc][H * m], contiguous).
    lo / hi: neighbour ranks or None at a physical end."""
    import torch.distributed as dist
    reqs = []
    if lo is not None:
        reqs.append(dist.isend(halo_planes(U, n_slab, m, H, "lo").contiguous(), lo, group, tag=1))
        reqs.append(dist.irecv(halo_lo, lo, group, tag=2))
    if hi is not None:
        reqs.append(dist.isend(halo_planes(U, n_slab, m, H, "hi").contiguous(), hi, group, tag=2))
        reqs.append(dist.irecv(halo_hi, hi, group, tag=1))
    for r in reqs:
        r.wait()


class SlabDecomposition:
    """A grid split into slabs along its slowest axis, every slab a
    sub-problem on this device with TENO_BC_HALO on its inner sides; the
    halo planes are copied between slabs on the device before every stage
    and the CFL time step is taken over all slabs, so the slabs advance
    exactly like the undivided grid (bitwise).  The halo copies are where a
    multi-GPU run would exchange planes between ranks (exchange_halos_dist)."""

    def __init__(self, p: teno_params, parts: int, device="cuda"):
        import torch
        self.device = torch.device(device)
        nd = p.ndim
        ax = nd - 1
        self.ax, self.nc, self.H = ax, nd + 2, p.scheme // 2
        self.m = 1
        for a in range(ax):
            self.m *= p.n[a]
        periodic = p.bc_lo[ax] == TENO_BC_PERIODIC
        self.plan = slab_plan(p.n[ax], parts, self.H, periodic)
        self.params, self.halos, self.solvers, self.Us = [], [], [], []
        for (a0, a1, lo, hi) in self.plan:
            hl = torch.zeros(self.nc, self.H * self.m, dtype=torch.float64, device=self.device)
            hh = torch.zeros_like(hl)
            q = teno_params()
            ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(p))
            q.n[ax] = a1 - a0
            if lo is not None:
                q.bc_lo[ax] = TENO_BC_HALO
                q.bc_state_lo[ax] = hl.data_ptr()
            if hi is not None:
                q.bc_hi[ax] = TENO_BC_HALO
                q.bc_state_hi[ax] = hh.data_ptr()
            self.params.append(q)
            self.halos.append((hl, hh))
            self.solvers.append(Solver(q, self.device))
            self.Us.append(None)
        self.amax = torch.zeros(len(self.plan) * 3, dtype=torch.float64, device=self.device)
        self.dt = torch.zeros(1, dtype=torch.float64, device=self.device)

    def split(self, U):
        """Slab states (copies) of a whole-grid state [nc][cells]."""
        V = U.view(self.nc, -1)
        return [V[:, a0 * self.m:a1 * self.m].contiguous() for (a0, a1, _, _) in self.plan]

    def join(self, parts):
        import torch
        return torch.cat(parts, dim=1)

    def exchange(self, states):
        """Fill every slab's halo arrays from its neighbours' current states."""
        for k, (a0, a1, lo, hi) in enumerate(self.plan):
            hl, hh = self.halos[k]
            if lo is not None:
                n_lo = self.plan[lo][1] - self.plan[lo][0]
                hl.copy_(halo_planes(states[lo], n_lo, self.m, self.H, "hi"))
            if hi is not None:
                n_hi = self.plan[hi][1] - self.plan[hi][0]
                hh.copy_(halo_planes(states[hi], n_hi, self.m, self.H, "lo"))

    def cfl_dt(self, parts, cfl=0.4):
        """The whole grid's CFL time step from every slab's wave speeds."""
        for k, U in enumerate(parts):
            teno_wave_speeds(self.params[k], U, self.amax[3 * k:3 * k + 3], self.solvers[k].ws)
        teno_dt_from_speeds(self.params[0], self.amax, len(parts), cfl, self.dt)
        return self.dt

    def step(self, parts, dt=None):
        """One SSP-RK3 step of every slab, halos exchanged before each stage;
        dt=None uses the device scalar of cfl_dt."""
        import torch
        for k, U in enumerate(parts):
            if self.Us[k] is None or self.Us[k].shape != U.shape:
                self.Us[k] = torch.empty_like(U)
        for stage in (1, 2, 3):
            self.exchange(parts if stage == 1 else self.Us)
            for k, U in enumerate(parts):
                s = self.solvers[k]
                teno_rk3_stage(self.params[k], stage, U, self.Us[k],
                               0.0 if dt is None else float(dt),
                               self.dt if dt is None else None, s.ws)

    def status(self):
        return sum(s.status() for s in self.solvers)


# ---------------------------------------------------------------------------
# batched mode
# ---------------------------------------------------------------------------

def pack_offsets(sizes):
    """Offsets (in doubles, 16-byte aligned) of [3][n] state blocks packed
    back to back, and the total length."""
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += 3 * int(n)
        o += o & 1
    return offs, o


def teno_batch_create(common: teno_params, problems):
    """problems: sequence of dicts with n, offset, dx, scheme, limiter,
    bc_lo, bc_hi.  Returns an opaque handle (free with teno_batch_destroy)."""
    arr = (teno_batch_problem * len(problems))()
    for i, q in enumerate(problems):
        arr[i].n, arr[i].offset, arr[i].dx = int(q["n"]), int(q["offset"]), float(q["dx"])
        arr[i].scheme, arr[i].limiter = int(q["scheme"]), int(q.get("limiter", 0))
        arr[i].bc_lo, arr[i].bc_hi = int(q.get("bc_lo", 1)), int(q.get("bc_hi", 1))
    h = ctypes.c_void_p()
    _check(load().teno_batch_create(ctypes.byref(common), arr, len(problems), ctypes.byref(h)),
           "teno_batch_create")
    return h


def teno_batch_workspace_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(load().teno_batch_workspace_bytes(h, ctypes.byref(n)), "teno_batch_workspace_bytes")
    return n.value


def teno_batch_autotune(h, U_scratch, ws, stream=None):
    t, bps = ctypes.c_int32(), ctypes.c_int32()
    _check(load().teno_batch_autotune(h, _ptr(U_scratch), _ptr(ws), ws.numel() * ws.element_size(),
                                      _stream(stream), ctypes.byref(t), ctypes.byref(bps)),
           "teno_batch_autotune")
    return t.value, bps.value


def teno_batch_rk3_steps(h, U, nsteps, cfl, mode, ws, stream=None):
    _check(load().teno_batch_rk3_steps(h, _ptr(U), int(nsteps), float(cfl), int(mode), _ptr(ws),
                                       ws.numel() * ws.element_size(), _stream(stream)),
           "teno_batch_rk3_steps")


def teno_batch_times(h, ws, nprob, stream=None):
    out = (ctypes.c_double * nprob)()
    _check(load().teno_batch_times(h, _ptr(ws), _stream(stream), out), "teno_batch_times")
    return list(out)


def teno_batch_destroy(h):
    if h:
        load().teno_batch_destroy(h)


class Batch:
    """Owns a batch plan and its workspace."""

    def __init__(self, common: teno_params, problems, device="cuda"):
        import torch
        self.problems = problems
        self.h = teno_batch_create(common, problems)
        nb = teno_batch_workspace_bytes(self.h)
        # 256-byte aligned workspace
        self._ws = torch.zeros((nb + 512) // 8, dtype=torch.float64, device=device)
        shift = (-self._ws.data_ptr() % 256) // 8
        self.ws = self._ws[shift:shift + (nb + 7) // 8]

    def autotune(self, U_scratch, stream=None):
        return teno_batch_autotune(self.h, U_scratch, self.ws, stream)

    def steps(self, U, nsteps, cfl=0.4, mode=TENO_BATCH_GRAPH, stream=None):
        teno_batch_rk3_steps(self.h, U, nsteps, cfl, mode, self.ws, stream)

    def times(self, stream=None):
        return teno_batch_times(self.h, self.ws, len(self.problems), stream)

    def __del__(self):
        try:
            teno_batch_destroy(self.h)
        except Exception:
            pass
        self.h = None


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

def teno_adjoint_workspace_bytes(p) -> int:
    n = ctypes.c_size_t()
    _check(load().teno_adjoint_workspace_bytes(ctypes.byref(p), ctypes.byref(n)),
           "teno_adjoint_workspace_bytes")
    return n.value


def aligned_workspace(nbytes, device):
    """A zeroed float64 tensor view whose data pointer is 256-byte aligned."""
    import torch
    raw = torch.zeros((nbytes + 512) // 8, dtype=torch.float64, device=device)
    shift = (-raw.data_ptr() % 256) // 8
    return raw[shift:shift + (nbytes + 7) // 8]


def teno_rhs_vjp(p, U, lam, mu, flags=None, ws=None, stream=None):
    _check(load().teno_rhs_vjp(ctypes.byref(p), _ptr(U), _ptr(lam), _ptr(flags), _ptr(mu),
                               _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "teno_rhs_vjp")


def teno_rk3_step_record(p, U, dt, U1, U2, flags, ws, stream=None):
    _check(load().teno_rk3_step_record(ctypes.byref(p), _ptr(U), float(dt), _ptr(U1), _ptr(U2),
                                       _ptr(flags), _ptr(ws), ws.numel() * ws.element_size(),
                                       _stream(stream)), "teno_rk3_step_record")


def teno_rk3_step_record_sel(p, U, dt, U1, U2, flags, ws, stream=None):
    """teno_rk3_step_record whose decision bytes carry the C_T exponent only
    where it was needed (the selection bits, argmax words and states are
    the full record's)."""
    _check(load().teno_rk3_step_record_sel(ctypes.byref(p), _ptr(U), float(dt), _ptr(U1),
                                           _ptr(U2), _ptr(flags), _ptr(ws),
                                           ws.numel() * ws.element_size(), _stream(stream)),
           "teno_rk3_step_record_sel")


def teno_rhs_frozen(p, U, rhs, decisions, ws, dt_limiter=0.0, stream=None):
    _check(load().teno_rhs_frozen(ctypes.byref(p), _ptr(U), _ptr(rhs), float(dt_limiter),
                                  _ptr(decisions), _ptr(ws), ws.numel() * ws.element_size(),
                                  _stream(stream)), "teno_rhs_frozen")


def teno_rk3_step_frozen(p, U, dt, decisions, ws, stream=None):
    _check(load().teno_rk3_step_frozen(ctypes.byref(p), _ptr(U), float(dt), _ptr(decisions),
                                       _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
           "teno_rk3_step_frozen")


def teno_rk3_step_vjp(p, Un, U1, U2, flags, dt, abar, ws, stream=None):
    _check(load().teno_rk3_step_vjp(ctypes.byref(p), _ptr(Un), _ptr(U1), _ptr(U2), _ptr(flags),
                                    float(dt), _ptr(abar), _ptr(ws),
                                    ws.numel() * ws.element_size(), _stream(stream)),
           "teno_rk3_step_vjp")


def _rollout_class():
    import torch

    class TenoRollout(torch.autograd.Function):
        """nsteps SSP-RK3 steps at a fixed dt; the backward walks checkpoint
        segments in reverse: recompute the segment's steps keeping stage
        states and selection-only decision records (the last segment's are
        kept from the forward), then apply teno_rk3_step_vjp step by step
        (decisions frozen as in the forward)."""

        @staticmethod
        def forward(ctx, U0, p, dt, nsteps, every):
            dev = U0.device
            ws = aligned_workspace(teno_workspace_bytes(p), dev)
            U = U0.detach().contiguous().clone()
            ckpts = []
            # the last segment is recorded as it is computed (stage states and
            # decision records, bitwise the same steps): the backward starts
            # with it and need not recompute it
            last = ((nsteps - 1) // every) * every if nsteps > 0 else 0
            flb = teno_flags_bytes(p)
            rec = []
            for k in range(nsteps):
                if k % every == 0:
                    ckpts.append(U.clone())
                if k >= last:
                    Un, U1, U2 = U.clone(), torch.empty_like(U), torch.empty_like(U)
                    fl = torch.empty(3 * flb, dtype=torch.uint8, device=dev)
                    teno_rk3_step_record_sel(p, U, float(dt), U1, U2, fl, ws)
                    rec.append((Un, U1, U2, fl))
                else:
                    teno_rk3_step(p, U, float(dt), None, ws)
            ctx.p, ctx.dt, ctx.nsteps, ctx.every = p, float(dt), nsteps, every
            ctx.ckpts = ckpts
            ctx.last_rec = rec
            return U

        @staticmethod
        def backward(ctx, gU):
            p, dt, nsteps, every = ctx.p, ctx.dt, ctx.nsteps, ctx.every
            dev = gU.device
            abar = gU.detach().contiguous().clone()
            fws = aligned_workspace(teno_workspace_bytes(p), dev)
            aws = aligned_workspace(teno_adjoint_workspace_bytes(p), dev)
            flb = teno_flags_bytes(p)
            nseg = len(ctx.ckpts)
            for s in reversed(range(nseg)):
                start = s * every
                stop = min(start + every, nsteps)
                if s == nseg - 1 and ctx.last_rec:
                    rec, ctx.last_rec = ctx.last_rec, None
                else:
                    U = ctx.ckpts[s].clone()
                    rec = []
                    for _ in range(start, stop):
                        Un = U.clone()
                        U1 = torch.empty_like(U)
                        U2 = torch.empty_like(U)
                        fl = torch.empty(3 * flb, dtype=torch.uint8, device=dev)
                        teno_rk3_step_record_sel(p, U, dt, U1, U2, fl, fws)
                        rec.append((Un, U1, U2, fl))
                for Un, U1, U2, fl in reversed(rec):
                    teno_rk3_step_vjp(p, Un, U1, U2, fl, dt, abar, aws)
                del rec
            ctx.ckpts = None
            ctx.last_rec = None
            return abar, None, None, None, None

    return TenoRollout


_ROLLOUT = None


def rollout(p, U0, dt, nsteps, checkpoint_every=20):
    """Differentiable: U(T) after nsteps SSP-RK3 steps of fixed dt from U0
    (a CUDA float64 tensor [ncons, ncells]); gradients flow to U0 through
    the frozen-decision adjoint with checkpoint-every-m recomputation."""
    global _ROLLOUT
    if _ROLLOUT is None:
        _ROLLOUT = _rollout_class()
    return _ROLLOUT.apply(U0, p, float(dt), int(nsteps), int(checkpoint_every))
