"""Direct pin of the oracle's characteristic-wise local Lax-Friedrichs
splitting (Sec. 5): for each characteristic field k of the Roe-averaged flux
Jacobian, f+-_k = (g_k +- alpha_k w_k) / 2 with alpha_k the largest |lambda_k|
over the stencil's cells, lambda_k(U_j) being cell j's own u_d - c, u_d or
u_d + c for the field of the Roe eigenvalue u~_d - c~, u~_d or u~_d + c~.

The restatement here shares nothing with the oracle's eigensystem: the flux
Jacobian at the Roe state is taken by complex-step differentiation of a
numpy Euler flux, its eigenvalues by LAPACK and its eigenvectors as null
spaces (any scaling and any basis of the repeated eigenvalue's space give
the same face flux).  The C_T parameters are set so that the largest
stencil S_p is accepted almost everywhere (alpha_2 = 0, alpha_1 = 22: C_T =
1e-22; only the nearly flat minus-split fluxes of the waves moving the other
way can still reject it).  The comparison runs over the cells whose two
faces in every direction took S_p for every field and sign, as the oracle's
decision record says; there every reconstruction is the printed linear
scheme of S_p, and the face flux R (f^+_hat + f^-_hat) is a plain sum.

The data are periodic and smooth but only 8-10 cells per wavelength, so that
the splitting's dissipative part (the printed scheme's odd part times
alpha_k) is some 1e-6 of the flux: exchanging the u - c and u + c speeds,
taking the speeds from cells i and i+1 only, or using one speed for all
fields moves the right-hand side by orders of magnitude more than the
1e-12 tolerance (checked in the test itself)."""
import numpy as np
import pytest
from scipy.linalg import null_space

import oracle

GAMMA = 1.4


def euler_flux(U, d):
    nd = U.shape[0] - 2
    rho, m, E = U[0], U[1:1 + nd], U[-1]
    u = m / rho
    p = (GAMMA - 1.0) * (E - 0.5 * rho * (u * u).sum(axis=0))
    F = np.empty_like(U)
    F[0] = m[d]
    F[1:1 + nd] = m[d] * u
    F[1 + d] = F[1 + d] + p
    F[-1] = u[d] * (E + p)
    return F


def primitives(U):
    nd = U.shape[0] - 2
    rho = U[0]
    u = U[1:1 + nd] / rho
    p = (GAMMA - 1.0) * (U[-1] - 0.5 * rho * (u * u).sum(axis=0))
    return rho, u, p


def roe_jacobian(UL, UR, d):
    """dF_d/dU at the Roe average of two cells, by complex-step
    differentiation at a state with the Roe velocity and enthalpy (the
    Jacobian depends on U only through u and H)."""
    nd = UL.shape[0] - 2
    rl, ul, pl = primitives(UL[:, None])
    rr, ur, pr = primitives(UR[:, None])
    Hl = (UL[-1] + pl[0]) / rl[0]
    Hr = (UR[-1] + pr[0]) / rr[0]
    sl, sr = np.sqrt(rl[0]), np.sqrt(rr[0])
    ut = (sl * ul[:, 0] + sr * ur[:, 0]) / (sl + sr)
    Ht = (sl * Hl + sr * Hr) / (sl + sr)
    q2 = float((ut * ut).sum())
    p = (GAMMA - 1.0) / GAMMA * (Ht - 0.5 * q2)          # rho = 1: c^2 = gamma p
    U0 = np.concatenate([[1.0], ut, [p / (GAMMA - 1.0) + 0.5 * q2]]).astype(complex)
    nc = nd + 2
    A = np.empty((nc, nc))
    h = 1e-30
    for j in range(nc):
        Uc = U0.copy()
        Uc[j] += 1j * h
        A[:, j] = euler_flux(Uc[:, None], d)[:, 0].imag / h
    return A


def eigensystem(A, nd):
    """R (columns: u~-c~, the nd-fold u~, u~+c~) and L = R^-1, with the
    field order the speeds below use."""
    lam = np.sort(np.linalg.eigvals(A).real)
    nc = nd + 2
    cols = [null_space(A - lam[0] * np.eye(nc), rcond=1e-9)]
    mid = lam[1:1 + nd].mean()
    cols.append(null_space(A - mid * np.eye(nc), rcond=1e-7))
    cols.append(null_space(A - lam[-1] * np.eye(nc), rcond=1e-9))
    assert [c.shape[1] for c in cols] == [1, nd, 1]
    R = np.hstack(cols)
    return R, np.linalg.inv(R)


def cell_speeds(U, d):
    """|u_d - c|, |u_d|, |u_d + c| per cell."""
    rho, u, p = primitives(U)
    c = np.sqrt(GAMMA * p / rho)
    return np.abs(u[d] - c), np.abs(u[d]), np.abs(u[d] + c)


def face_fluxes_line(Uline, d, H, coef, variant="llf"):
    """Face fluxes F_{i+1/2}, i = 0..n-1, of one periodic line (nc, n) along
    direction d, every reconstruction the S_p linear scheme."""
    nc, n = Uline.shape
    nd = nc - 2
    F = euler_flux(Uline, d)
    sp = cell_speeds(Uline, d)
    out = np.empty((nc, n))
    offs = np.arange(-H + 1, H + 1)
    for i in range(n):
        idx = (i + offs) % n                    # stencil cells i-H+1 .. i+H
        A = roe_jacobian(Uline[:, i], Uline[:, (i + 1) % n], d)
        R, L = eigensystem(A, nd)
        speed_of_field = [sp[0]] + [sp[1]] * nd + [sp[2]]
        if variant == "swapped":                # u-c and u+c speeds exchanged
            speed_of_field = [sp[2]] + [sp[1]] * nd + [sp[0]]
        w = L @ Uline[:, idx]
        g = L @ F[:, idx]
        h = np.empty(nc)
        for k in range(nc):
            s = speed_of_field[k]
            if variant == "local":              # cells i and i+1 only
                alpha = max(s[i], s[(i + 1) % n])
            elif variant == "single":           # one speed for every field
                alpha = max(np.max(sp[0][idx]), np.max(sp[2][idx]))
            else:
                alpha = np.max(s[idx])
            fp = 0.5 * (g[k] + alpha * w[k])
            fm = 0.5 * (g[k] - alpha * w[k])
            # f+ at offset m is cell i+m; f- at offset m is cell i+1-m
            hp = sum(coef[m] * fp[m + H - 1] for m in coef)
            hm = sum(coef[m] * fm[(1 - m) + H - 1] for m in coef)
            h[k] = hp + hm
        out[:, i] = R @ h
    return out


def restated_rhs(U, n, dx, H, coef, variant="llf"):
    nc = U.shape[0]
    nd = nc - 2
    shape = (nc,) + tuple(reversed(n[:nd]))   # (nc, [ny,] nx)
    Ug = U.reshape(shape)
    L = np.zeros_like(Ug)
    for d in range(nd):
        ax = nd - d                           # array axis of direction d
        Um = np.moveaxis(Ug, ax, -1)
        lines = Um.reshape(nc, -1, n[d])
        Fl = np.empty_like(lines)
        for q in range(lines.shape[1]):
            Fl[:, q] = face_fluxes_line(lines[:, q], d, H, coef, variant)
        Ff = Fl.reshape(Um.shape)
        dF = (Ff - np.roll(Ff, 1, axis=-1)) / dx[d]
        L -= np.moveaxis(dF, -1, ax)
    return L.reshape(nc, -1)


def smooth_state(n, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    nd = len(n)
    axes = [(np.arange(m) + 0.5) / m for m in n]
    X = np.meshgrid(*reversed(axes), indexing="ij")[::-1]     # X[0] = x, ...

    def field(base, amp):
        f = np.full(X[0].shape, base)
        for _ in range(3):
            k = [int(g.integers(0, 4)) for _ in range(nd)]
            k[int(g.integers(0, nd))] = int(g.integers(1, 4))
            ph = sum(2 * np.pi * k[a] * X[a] for a in range(nd))
            f = f + amp * g.uniform(0.3, 1.0) * np.sin(ph + g.uniform(0, 6.3))
        return f

    rho = field(1.0, 0.12)
    u = [field(0.35 if a == 0 else -0.2, 0.12) for a in range(nd)]
    p = field(1.0, 0.15)
    E = p / (GAMMA - 1.0) + 0.5 * rho * sum(v * v for v in u)
    U = np.stack([rho] + [rho * v for v in u] + [E])
    return U.reshape(nd + 2, -1)


def clean_cells(fl, n, H):
    """Cells whose faces (both sides, every direction) took S_H for every
    field and sign, from the oracle's decision record (per direction, the
    face grid n with n_d + 1 faces along d, x fastest; face f lies between
    cells f - 1 and f)."""
    nd = len(n)
    nc = nd + 2
    sel = np.array([oracle.decode_flag(b)[0] for b in range(256)])
    ok = np.ones(tuple(reversed(n)), bool)
    off = 0
    for d in range(nd):
        fn = list(n)
        fn[d] += 1
        cnt = int(np.prod(fn))
        rec = fl[off:off + cnt * nc * 2].reshape(cnt, nc * 2)
        off += cnt * nc * 2
        face_ok = (sel[rec] == H).all(axis=1).reshape(tuple(reversed(fn)))
        ax = nd - 1 - d
        lo = np.take(face_ok, np.arange(n[d]), axis=ax)
        hi = np.take(face_ok, np.arange(1, n[d] + 1), axis=ax)
        ok &= lo & hi
    return ok.reshape(-1)


CASES = [((32,), 8, 1101), ((40,), 10, 1102), ((40,), 12, 1103), ((40, 36), 8, 1104),
         ((36, 40), 10, 1105)]


@pytest.mark.parametrize("n,scheme,seed", CASES)
def test_llf_face_flux_matches_restatement(n, scheme, seed):
    H = scheme // 2
    nd = len(n)
    dx = [1.0 / m for m in n]
    U = smooth_state(n, seed)
    po = oracle.params(nd, list(n), dx, scheme=scheme, gamma=GAMMA, bc=0, alpha1=22.0,
                       alpha2=0.0)
    r_o, fl, _, nb = oracle.rhs(po, U, want_flags=True)
    assert nb == 0
    clean = clean_cells(fl, n, H)
    assert clean.mean() > 0.4, "only %.2f of the cells have S_%d on every face" % (clean.mean(), H)
    coef = {m: oracle.lin_coef(H, m) for m in range(1 - H, H + 1)}
    scale = np.abs(r_o).max(axis=1)

    def err(r):
        return float((np.abs(r - r_o)[:, clean].max(axis=1) / scale).max())

    e = err(restated_rhs(U, n, dx, H, coef))
    assert e <= 1e-12, "characteristic LLF flux differs from the restatement by %.3g" % e
    # the pin has teeth: each plausible misreading of the speeds is far away
    for variant in ("swapped", "local", "single"):
        ev = err(restated_rhs(U, n, dx, H, coef, variant))
        assert ev > 1e-9, "%s speeds indistinguishable (%.3g)" % (variant, ev)
