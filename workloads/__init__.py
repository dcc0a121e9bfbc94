"""Seeded synthetic inputs for the TENO-AA Euler solver.

Shared by the CPU oracle tests, the GPU parity tests and the benchmark as
*inputs only*: this module holds initial conditions and nothing of the scheme's
arithmetic.  Every generator uses numpy's PCG64 with a fixed seed and returns
conserved variables U with shape (ncons, nz, ny, nx) flattened to
(ncons, cells) in x-fastest order, ncons = ndim + 2: (rho, rho*u_x, ..., E).

Workloads, shaped like the paper's 1D/2D/3D shock and turbulence problems
(arXiv 2109.14340, Sec. 5):
  * riemann_1d        seeded two-state shock tube on [0,1] (Sec. 5.2 style)
  * smooth_wave_1d    periodic density sine wave (order study, Sec. 5.1 style)
  * quadrants_2d      four-quadrant Riemann problem + entropy wave
  * tgv_3d            Mach-0.5 Taylor-Green field + k^-5/3 solenoidal noise
  * batched_1d        thousands of independent Riemann problems, uneven sizes
  * sod_1d, double_rarefaction_1d   textbook problems of Sec. 5.2 / 5.3
  * boundary_walls    random flow with no-slip / Dirichlet sides (App. A.2, A.3)
"""
from __future__ import annotations

import math

import numpy as np

PERIODIC, TRANSMISSIVE, SLIPWALL = 0, 1, 2


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def prim_to_cons(rho, vel, p, gamma):
    """Initial-condition helper: primitive (rho, velocity list, p) to conserved."""
    rho = np.asarray(rho, np.float64)
    vel = [np.broadcast_to(np.asarray(v, np.float64), rho.shape) for v in vel]
    p = np.broadcast_to(np.asarray(p, np.float64), rho.shape)
    ke = 0.5 * rho * sum(v * v for v in vel)
    E = p / (gamma - 1.0) + ke
    return np.stack([rho] + [rho * v for v in vel] + [E]).reshape(len(vel) + 2, -1)


def _case(U, ndim, n, dx, bc_lo, bc_hi, scheme, gamma=1.4, **extra):
    d = dict(U=np.ascontiguousarray(U, np.float64), ndim=ndim, n=list(n) + [1] * (3 - len(n)),
             dx=list(dx) + [1.0] * (3 - len(dx)), bc_lo=list(bc_lo) + [0] * (3 - len(bc_lo)),
             bc_hi=list(bc_hi) + [0] * (3 - len(bc_hi)), scheme=scheme, gamma=gamma)
    d.update(extra)
    return d


def smooth_wave_1d(N: int, scheme: int = 8, gamma: float = 1.4, amp: float = 0.2):
    """rho = 1 + amp sin(2 pi x), u = 1, p = 1 on periodic [0,1]: the exact
    solution is a translation; the exact RHS is -(rho', rho', rho'/2)."""
    x = (np.arange(N) + 0.5) / N
    rho = 1.0 + amp * np.sin(2 * np.pi * x)
    U = prim_to_cons(rho, [np.ones(N)], np.ones(N), gamma)
    d = 2 * np.pi * amp * np.cos(2 * np.pi * x)
    exact = -np.stack([d, d, 0.5 * d])
    return _case(U, 1, [N], [1.0 / N], [PERIODIC], [PERIODIC], scheme, gamma, x=x,
                 exact_rhs=exact)


def riemann_1d(N: int = 400, seed: int = 1001, scheme: int = 8, gamma: float = 1.4):
    """Seeded piecewise-constant two-state IC split at x = 0.5 on [0,1],
    rho in [0.1,1], u in [-0.5,0.5], p in [0.1,1]; transmissive ends."""
    g = rng(seed)
    rl, rr = g.uniform(0.1, 1.0, 2)
    ul, ur = g.uniform(-0.5, 0.5, 2)
    pl, pr = g.uniform(0.1, 1.0, 2)
    x = (np.arange(N) + 0.5) / N
    left = x < 0.5
    rho = np.where(left, rl, rr)
    u = np.where(left, ul, ur)
    p = np.where(left, pl, pr)
    U = prim_to_cons(rho, [u], p, gamma)
    return _case(U, 1, [N], [1.0 / N], [TRANSMISSIVE], [TRANSMISSIVE], scheme, gamma, x=x,
                 states=((rl, ul, pl), (rr, ur, pr)), t_end=0.2)


def sod_1d(N: int, scheme: int = 8, gamma: float = 1.4):
    """Sod's shock tube (Sec. 5.2): (1,0,1) | (0.125,0,0.1) at x = 0.5, t = 0.2."""
    x = (np.arange(N) + 0.5) / N
    left = x < 0.5
    U = prim_to_cons(np.where(left, 1.0, 0.125), [np.zeros(N)], np.where(left, 1.0, 0.1), gamma)
    return _case(U, 1, [N], [1.0 / N], [TRANSMISSIVE], [TRANSMISSIVE], scheme, gamma, x=x,
                 states=((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)), t_end=0.2)


def double_rarefaction_1d(N: int = 400, scheme: int = 8, gamma: float = 1.4):
    """Double rarefaction toward vacuum (Sec. 5.3): (1,-2,0.1) | (1,2,0.1), t = 0.1."""
    x = (np.arange(N) + 0.5) / N
    left = x < 0.5
    U = prim_to_cons(np.ones(N), [np.where(left, -2.0, 2.0)], np.full(N, 0.1), gamma)
    return _case(U, 1, [N], [1.0 / N], [TRANSMISSIVE], [TRANSMISSIVE], scheme, gamma, x=x,
                 states=((1.0, -2.0, 0.1), (1.0, 2.0, 0.1)), t_end=0.1)


def quadrants_2d(nx: int = 1024, ny: int | None = None, seed: int = 2001, scheme: int = 10,
                 gamma: float = 1.4):
    """Four-quadrant Riemann IC on the unit square (per quadrant rho in
    [0.1,1.5], u,v in [-1,1], p in [0.03,1.5]) plus rho' = 0.2 sin(5x) in the
    lower-left quadrant; transmissive boundaries."""
    ny = nx if ny is None else ny
    g = rng(seed)
    rho_q = g.uniform(0.1, 1.5, 4)
    u_q = g.uniform(-1.0, 1.0, 4)
    v_q = g.uniform(-1.0, 1.0, 4)
    p_q = g.uniform(0.03, 1.5, 4)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")          # shape (ny, nx), x fastest
    q = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    rho = rho_q[q] + np.where(q == 0, 0.2 * np.sin(5 * X), 0.0)
    U = prim_to_cons(rho, [u_q[q], v_q[q]], p_q[q], gamma)
    return _case(U, 2, [nx, ny], [1.0 / nx, 1.0 / ny], [TRANSMISSIVE] * 2, [TRANSMISSIVE] * 2,
                 scheme, gamma, steps=200)


def tgv_3d(n: int = 256, seed: int = 3001, scheme: int = 10, gamma: float = 1.4,
           mach: float = 0.5, kmax: int = 16, rms_frac: float = 0.1):
    """Periodic [0,2pi]^3: rho = 1, u = sin x cos y cos z, v = -cos x sin y cos z,
    w = 0, p = (1/M)^2/gamma, plus a seeded solenoidal field with E(k) ~ k^-5/3
    for 1 <= |k| <= kmax, scaled to rms_frac of the Taylor-Green rms speed."""
    L = 2 * np.pi
    x = (np.arange(n) + 0.5) * (L / n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")     # (nz, ny, nx)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    del X, Y, Z
    g = rng(seed)
    k1 = np.fft.fftfreq(n, 1.0 / n)
    kh = np.fft.rfftfreq(n, 1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, kh, indexing="ij")
    K2 = KX * KX + KY * KY + KZ * KZ
    K = np.sqrt(K2)
    band = (K >= 1.0) & (K <= kmax)
    amp = np.where(band, np.power(np.where(band, K, 1.0), -11.0 / 6.0), 0.0)
    comps = []
    for _ in range(3):
        ph = g.uniform(0.0, 2 * np.pi, K.shape)
        mag = g.standard_normal(K.shape)
        comps.append(amp * mag * np.exp(1j * ph))
    Ksafe = np.where(K2 > 0, K2, 1.0)
    div = (KX * comps[0] + KY * comps[1] + KZ * comps[2]) / Ksafe
    comps = [comps[0] - KX * div, comps[1] - KY * div, comps[2] - KZ * div]
    pert = [np.fft.irfftn(c, s=(n, n, n), axes=(0, 1, 2)) for c in comps]
    del comps, KX, KY, KZ, K, K2, Ksafe, div
    rms_tgv = math.sqrt(np.mean(u * u + v * v + w * w))
    rms_p = math.sqrt(np.mean(pert[0] ** 2 + pert[1] ** 2 + pert[2] ** 2))
    s = rms_frac * rms_tgv / rms_p if rms_p > 0 else 0.0
    u += s * pert[0]
    v += s * pert[1]
    w += s * pert[2]
    rho = np.ones_like(u)
    p = np.full_like(u, (1.0 / mach) ** 2 / gamma)
    U = prim_to_cons(rho, [u, v, w], p, gamma)
    dx = L / n
    return _case(U, 3, [n, n, n], [dx, dx, dx], [PERIODIC] * 3, [PERIODIC] * 3, scheme, gamma,
                 steps=100)


def batched_1d(count: int = 4096, seed: int = 4001, nmin: int = 64, nmax: int = 4096,
               gamma: float = 1.4, vacuum_frac: float = 0.1):
    """Independent 1D Riemann problems on [0,1] with N ~ U{nmin..nmax}, schemes
    8|10 mixed 50/50, rho in [0.1,1] per side, pressure ratio log-uniform in
    [1,1e5] with a random high side; a vacuum_frac share gets one side at
    rho = 1e-6 with the same temperature (positivity limiter on)."""
    g = rng(seed)
    probs = []
    for _ in range(count):
        N = int(g.integers(nmin, nmax + 1))
        scheme = 8 if g.random() < 0.5 else 10
        rl, rr = g.uniform(0.1, 1.0, 2)
        plow = g.uniform(0.1, 1.0)
        ratio = math.exp(g.uniform(0.0, math.log(1e5)))
        high_left = g.random() < 0.5
        pl, pr = (plow * ratio, plow) if high_left else (plow, plow * ratio)
        vac = g.random() < vacuum_frac
        if vac:
            if g.random() < 0.5:
                pl, rl = pl * (1e-6 / rl), 1e-6
            else:
                pr, rr = pr * (1e-6 / rr), 1e-6
        x = (np.arange(N) + 0.5) / N
        left = x < 0.5
        U = prim_to_cons(np.where(left, rl, rr), [np.zeros(N)], np.where(left, pl, pr), gamma)
        probs.append(_case(U, 1, [N], [1.0 / N], [TRANSMISSIVE], [TRANSMISSIVE], scheme, gamma,
                           limiter=1 if vac else 0))
    return probs


def smooth_field(shape, seed, modes=4, amp=1.0, periodic_axes=None):
    """Seeded smooth field on the unit box (sum of a few low Fourier modes),
    shape (nz, ny, nx) or shorter; used for perturbations and directions."""
    g = rng(seed)
    grids = np.meshgrid(*[(np.arange(s) + 0.5) / s for s in shape], indexing="ij")
    out = np.zeros(shape)
    for _ in range(modes):
        k = g.integers(1, 4, len(shape))
        ph = g.uniform(0, 2 * np.pi)
        a = g.uniform(-1, 1)
        arg = sum(2 * np.pi * k[i] * grids[i] for i in range(len(shape))) + ph
        out += a * np.sin(arg)
    return amp * out / max(1e-300, np.abs(out).max())


def adjoint_2d(n: int = 512, ny: int | None = None, seed: int = 5001, scheme: int = 8,
               gamma: float = 1.4, target_seed: int = 5002, target_amp: float = 1e-3):
    """Stationary Mach-2 normal shock at x = 0.5 on the unit square with a
    uniform tangential velocity v = u1/2 (an oblique-shock flow that stays
    y-periodic), upstream rho = 1, p = 1/gamma (c = 1), Rankine-Hugoniot
    downstream; seeded smooth entropy wave + isentropic vortex upstream and a
    1e-3 generic smooth field everywhere.
    Transmissive in x, periodic in y.  Also returns the initial state of the
    target run: the same IC plus a seeded smooth perturbation of relative
    size target_amp."""
    ny = n if ny is None else ny
    g = rng(seed)
    M = 2.0
    r1, p1, u1 = 1.0, 1.0 / gamma, 2.0
    r2 = r1 * (gamma + 1) * M * M / ((gamma - 1) * M * M + 2)
    p2 = p1 * (1 + 2 * gamma / (gamma + 1) * (M * M - 1))
    u2 = u1 * r1 / r2
    vt = 0.5 * u1
    x = (np.arange(n) + 0.5) / n
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    up = X < 0.5
    rho = np.where(up, r1, r2)
    u = np.where(up, u1, u2)
    p = np.where(up, p1, p2)
    win = 0.5 * (1 - np.tanh((X - 0.38) / 0.02))
    ky = int(g.integers(1, 4))
    kx = g.uniform(2, 6)
    ph = g.uniform(0, 2 * np.pi)
    rho = rho * (1 + 0.05 * win * np.sin(2 * np.pi * (kx * X + ky * Y) + ph))
    x0, y0 = g.uniform(0.15, 0.3), g.uniform(0.3, 0.7)
    eps, R = 0.3, 0.05
    r2v = ((X - x0) ** 2 + (Y - y0) ** 2) / (R * R)
    e = np.exp(0.5 * (1 - r2v))
    u = u + eps / (2 * np.pi) * (-(Y - y0) / R) * e * win
    v = vt + eps / (2 * np.pi) * ((X - x0) / R) * e * win
    T1 = p1 / r1
    dT = -(gamma - 1) * eps * eps / (8 * gamma * np.pi ** 2) * e * e * win
    T = np.where(up, T1 + dT, p / rho)
    rho = np.where(up, rho * ((T1 + dT) / T1) ** (1 / (gamma - 1)), rho)
    p = np.where(up, rho * T, p)
    # a small generic smooth field in every primitive variable, so that no
    # characteristic field is constant only up to rounding (there TENO's
    # decisions follow rounding noise and the map is not differentiable)
    gen = smooth_field((4, ny, n), seed + 100, modes=6)
    rho = rho * (1 + 1e-3 * gen[0])
    u = u + 1e-3 * gen[1]
    v = v + 1e-3 * gen[2]
    p = p * (1 + 1e-3 * gen[3])
    U = prim_to_cons(rho, [u, v], p, gamma)
    pert = smooth_field((4, ny, n), target_seed)
    Ut = U * (1 + target_amp * pert.reshape(4, -1))
    return _case(U, 2, [n, ny], [1.0 / n, 1.0 / ny], [TRANSMISSIVE, PERIODIC],
                 [TRANSMISSIVE, PERIODIC], scheme, gamma, U_target_ic=Ut, steps=200,
                 checkpoint_every=20)


def boundary_walls(ndim: int, n, bc_lo, bc_hi, seed: int = 6001, scheme: int = 10,
                   gamma: float = 1.4):
    """Random smooth-plus-noise flow with no-slip and Dirichlet sides (App.
    A.2, A.3).  The Dirichlet sides get seeded boundary-face primitives
    (rho, u..., p) as arrays [ndim + 2][faces of the side, other axes x
    fastest] under "bc_state_lo" / "bc_state_hi" (None for other sides)."""
    g = np.random.Generator(np.random.PCG64(seed))
    n = list(n) + [1] * (3 - len(n))
    cells = n[0] * n[1] * n[2]
    rho = g.uniform(0.4, 1.4, cells)
    vel = [g.uniform(-0.6, 0.6, cells) for _ in range(ndim)]
    pr = g.uniform(0.3, 1.5, cells)
    U = prim_to_cons(rho, vel, pr, gamma)
    lo = list(bc_lo) + [0] * (3 - len(bc_lo))
    hi = list(bc_hi) + [0] * (3 - len(bc_hi))
    st_lo, st_hi = [None] * 3, [None] * 3
    for d in range(ndim):
        m = cells // n[d]
        for side, bcs, st in ((0, lo, st_lo), (1, hi, st_hi)):
            if bcs[d] == 4:
                # 2 phi' - phi stays positive: rho' >= 0.8 > 1.4 / 2, p' >= 0.9 > 1.5 / 2
                st[d] = np.stack([g.uniform(0.8, 1.2, m)] +
                                 [g.uniform(-0.4, 0.4, m) for _ in range(ndim)] +
                                 [g.uniform(0.9, 1.3, m)])
    dx = [0.1, 0.08, 0.06][:ndim]
    return _case(U, ndim, n[:ndim], dx, lo[:ndim], hi[:ndim], scheme, gamma,
                 bc_state_lo=st_lo, bc_state_hi=st_hi)


def noh_3d(n: int = 64, scheme: int = 10, L: float = 0.256, gamma: float = 5.0 / 3.0,
           p0: float = 1e-6):
    """3D Noh implosion (Sec. 5.5): cube [0, L]^3, rho = 1, velocity -x_i / r
    toward the origin, p = p0; symmetry (slip) walls at x_i = 0 and
    supersonic inflow through the far faces, given there as Dirichlet states
    (noh_inflow_states) with the initial velocity and pressure and the
    analytic density.  Rusanov splitting, limiter on, t_end = 0.6."""
    dx = L / n
    c = (np.arange(n) + 0.5) * dx
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    U = prim_to_cons(np.ones_like(r).ravel(), [(-X / r).ravel(), (-Y / r).ravel(), (-Z / r).ravel()],
                     np.full(r.size, p0), gamma)
    return _case(U, 3, [n, n, n], [dx, dx, dx], [SLIPWALL] * 3, [4] * 3, scheme, gamma,
                 L=L, p0=p0, t_end=0.6, split=1, limiter=1)


def noh_density(r, t):
    """Analytic density of the 3D Noh problem (Eq. density_noh): 64 behind the
    shock r < t/3, (1 + t/r)^2 ahead of it."""
    r = np.asarray(r, np.float64)
    return np.where(r < t / 3.0, 64.0, (1.0 + t / np.maximum(r, 1e-300)) ** 2)


def noh_inflow_states(case, t: float):
    """Boundary-face primitives (rho, u, v, w, p) of the far faces x_d = L at
    time t, [5][n*n] per axis, the other two axes x fastest: the analytic
    density and the initial velocity -x_i / r and pressure."""
    n, L, p0 = case["n"][0], case["L"], case["p0"]
    dx = L / n
    c = (np.arange(n) + 0.5) * dx
    out = []
    for d in range(3):
        B, A = np.meshgrid(c, c, indexing="ij")       # (slow, fast) of the other two axes
        coords = [None] * 3
        others = [a for a in range(3) if a != d]
        coords[d] = np.full_like(A, L)
        coords[others[0]] = A
        coords[others[1]] = B
        r = np.sqrt(coords[0] ** 2 + coords[1] ** 2 + coords[2] ** 2)
        st = np.stack([noh_density(r, t), -coords[0] / r, -coords[1] / r, -coords[2] / r,
                       np.full_like(r, p0)])
        out.append(st.reshape(5, -1))
    return out
