"""Linear-algebra side of the oracle: the step in matrix form, its Fourier symbol, and exact
solutions of the Linearized Euler Equations used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np

from . import VelSet


def h_matrix(s: VelSet, tau: float) -> np.ndarray:
    """H(tau) of Sec. 6 (eq. "LBE linear equation"), built entry by entry from the printed
    formula, with one reading: the velocity term carries 1/rho0, b c_i.c_j / rho0, because
    u' = <v g>_S / rho0 (Sec. 4).  As printed (without 1/rho0) the matrix H(1) of the diatomic
    D2Q5 set (rho0 = 20/3) is not a projection; with 1/rho0 it is.  The rho0 = 1 sets are
    unaffected.

    H_ij = (1 - 1/tau) delta_ij + (1/tau) ( a1 + |c_i|^2 c1 / 2 + (b / rho0) c_i.c_j
           + ((gamma - 1) (|c_j|^2 + beta_j) / 2 - theta0) (a2 + |c_i|^2 c2 / 2) / rho0 ) f*_i
    """
    q = s.q
    c = s.c.astype(np.float64)
    H = np.zeros((q, q))
    for i in range(q):
        ci2 = float(c[i] @ c[i])
        for j in range(q):
            cj2 = float(c[j] @ c[j])
            k = (s.a1 + 0.5 * ci2 * s.c1 + (s.b / s.rho0) * float(c[i] @ c[j])
                 + ((s.gamma - 1.0) * 0.5 * (cj2 + s.beta[j]) - s.theta0) * (s.a2 + 0.5 * ci2 * s.c2) / s.rho0)
            H[i, j] = (1.0 - 1.0 / tau) * (i == j) + (1.0 / tau) * k * s.f[i]
    return H


def gamma_symbol(s: VelSet, tau: float, k) -> np.ndarray:
    """Gamma(k) = D(k) H(tau), D_mm = exp(-i k.c_m) (Sec. 7, von Neumann analysis; lattice units,
    epsilon = 1).  It advances the Fourier coefficient of the pre-collision populations."""
    k = np.asarray(k, dtype=np.float64)
    kk = np.zeros(3)
    kk[: k.size] = k
    phase = np.exp(-1j * (s.c.astype(np.float64) @ kk))
    return phase[:, None] * h_matrix(s, tau)


def step_matrix(s: VelSet, shape, tau: float) -> np.ndarray:
    """The whole periodic update as one explicit (q*cells) x (q*cells) matrix,
    M[(i, x + c_i), (j, x)] = H_ij(tau), i.e. M = S (I_cells (x) H) with S the periodic shift of
    each population along its velocity.  Row/column index = i * cells + cell."""
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    cells = nx * ny * nz
    H = h_matrix(s, tau)
    M = np.zeros((s.q * cells, s.q * cells))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                src = x + nx * (y + ny * z)
                for i in range(s.q):
                    tx = (x + s.c[i, 0]) % nx
                    ty = (y + s.c[i, 1]) % ny
                    tz = (z + s.c[i, 2]) % nz
                    dst = tx + nx * (ty + ny * tz)
                    for j in range(s.q):
                        M[i * cells + dst, j * cells + src] += H[i, j]
    return M


def dalembert_d1q3(G: np.ndarray, t: int) -> np.ndarray:
    """Exact LEE density for the D1Q3 background (rho0 = 1, theta0 = 1/3, gamma = 3, so the sound
    speed gamma * theta0 = 1 equals the lattice speed) with rho'(0) = G, u' = theta' = 0 on a
    periodic grid: the entropy part (1 - 1/gamma) G stays, the acoustic part G / gamma splits into
    two halves moving one cell per step left and right (Sec. 9.1)."""
    gam = 3.0
    return (1.0 - 1.0 / gam) * G + (0.5 / gam) * (np.roll(G, t) + np.roll(G, -t))


def lee_spectral(s: VelSet, shape, rho, u, theta, t: float):
    """Exact solution at time t (lattice units) of the LEE without background velocity (Sec. 2.1)
    for periodic initial fields given on the grid, mode by mode.  With p' = rho0 theta' +
    theta0 rho', the longitudinal velocity U = k^.u' and c_s^2 = gamma theta0:
        p^(t) = p^0 cos(c_s|k|t) - i rho0 c_s U^0 sin(c_s|k|t)
        U^(t) = U^0 cos(c_s|k|t) - i p^0 / (rho0 c_s) sin(c_s|k|t)
        rho^(t) = rho^0 + (p^(t) - p^0) / c_s^2,   theta^(t) = (p^(t) - theta0 rho^(t)) / rho0
    and the transverse velocity and the k = 0 mode do not change."""
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    D = s.D
    grid = (nz, ny, nx)
    R = np.fft.fftn(np.asarray(rho, dtype=np.float64).reshape(grid))
    T = np.fft.fftn(np.asarray(theta, dtype=np.float64).reshape(grid))
    Uv = [np.fft.fftn(np.asarray(u, dtype=np.float64).reshape(D, -1)[a].reshape(grid)) for a in range(D)]
    kz = 2 * np.pi * np.fft.fftfreq(nz)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    Kvec = [KX, KY, KZ][:D]
    Kmag = np.sqrt(sum(k * k for k in Kvec))
    safe = np.where(Kmag > 0, Kmag, 1.0)
    khat = [k / safe for k in Kvec]
    cs = np.sqrt(s.cs2)
    P0 = s.rho0 * T + s.theta0 * R
    U0 = sum(khat[a] * Uv[a] for a in range(D))
    w = cs * Kmag * t
    Pt = P0 * np.cos(w) - 1j * s.rho0 * cs * U0 * np.sin(w)
    Ut = U0 * np.cos(w) - 1j * P0 / (s.rho0 * cs) * np.sin(w)
    zero = Kmag == 0
    Pt = np.where(zero, P0, Pt)
    Ut = np.where(zero, U0, Ut)
    Rt = R + (Pt - P0) / s.cs2
    Tt = (Pt - s.theta0 * Rt) / s.rho0
    Uout = [Uv[a] + khat[a] * (Ut - U0) for a in range(D)]
    back = lambda A: np.real(np.fft.ifftn(A)).ravel()  # noqa: E731
    return back(Rt), np.stack([back(A) for A in Uout]), back(Tt)


def maxwellian_moments(D: int, rho0: float, theta0: float) -> dict:
    """Closed-form moments of M(v) = rho0 (2 pi theta0)^(-D/2) exp(-|v|^2 / (2 theta0)) for the
    similarity conditions of Sec. 4: <1>, <|v|^2/2>, <v_a v_b>, <|v|^2 v_a v_b / 2>, <|v|^4 / 4>
    (Gaussian integrals: <v_a^2> = rho0 theta0, <v_a^4> = 3 rho0 theta0^2,
    <v_a^2 v_b^2> = rho0 theta0^2 for a != b)."""
    v2 = rho0 * theta0
    v4_same = 3.0 * rho0 * theta0 ** 2
    v4_cross = rho0 * theta0 ** 2
    half_e_vv = 0.5 * (v4_same + (D - 1) * v4_cross)  # <|v|^2 v_a^2 / 2>
    quarter_v4 = 0.25 * (D * v4_same + D * (D - 1) * v4_cross)
    return {"one": rho0, "half_v2": 0.5 * D * v2, "vavb_diag": v2, "half_v2_vavb_diag": half_e_vv,
            "quarter_v4": quarter_v4}


def discrete_moments(s: VelSet) -> dict:
    """The same moments as maxwellian_moments, taken over the discrete set with weights f*."""
    c = s.c[:, : s.D].astype(np.float64)
    c2 = (c * c).sum(1)
    f = s.f
    out = {"one": f.sum(), "half_v2": (0.5 * c2 * f).sum(), "quarter_v4": (0.25 * c2 * c2 * f).sum()}
    vv = np.einsum("i,ia,ib->ab", f, c, c)
    evv = np.einsum("i,i,ia,ib->ab", f, 0.5 * c2, c, c)
    out["vavb"] = vv
    out["half_v2_vavb"] = evv
    return out
