"""Von Neumann stability scan of the LBE update (Sec. 7, Theorem 1) for the oracle (TEST
INFRASTRUCTURE ONLY: tests use it; the library never does).

Wave numbers: an m^D grid, k_a = 2 pi (j_a - m/2) / m, j_a = 0 .. m-1 (lattice units, k eps in
[-pi, pi)), point index j = j_x + m (j_y + m j_z).  Amplification matrix (Sec. 7):
    Gamma(k) = D(k) H(tau),  D_nn = exp(-i k.c_n),  H from the printed H_ij (analysis.h_matrix).
Theorem 1 asks for (1) Gamma regular, (2) rho(Gamma) <= 1, (3) a bounded condition number of the
eigenvector matrix, for every k.  Where eigenvalues repeat (at tau = 1/2 the non-propagating
entropy and vorticity modes give lambda = 1 at every k) the eigenvector matrix is not unique, so
condition (3) is evaluated on a fixed similar matrix and a fixed basis:
    Gamma_W(k) = W^(1/2) Gamma(k) W^(-1/2) = D(k) S,  W = diag(1 / f*_n),  S = W^(1/2) H W^(-1/2),
whose eigenvalues are those of Gamma.  H is self-adjoint in the inner product weighted by W, so S
is symmetric.  kappa_W(k) is the 2-norm condition number of the eigenvectors of Gamma_W with unit
columns, orthonormal within each cluster of eigenvalues closer than `delta` (each cluster's
basis: the right singular vectors of Gamma_W - lambda_c I for its smallest singular values).
Then kappa_2(V) <= sqrt(max f* / min f*) kappa_W for the matching eigenvectors V of Gamma.
Also reported: the normality defect nu(k) = ||G^H G - G G^H||_F / ||G||_F^2 of G = Gamma_W.
"""
from __future__ import annotations

import numpy as np

from . import velset
from .analysis import h_matrix


def k_grid(D: int, m: int) -> np.ndarray:
    """[m^D][D] wave vectors in point order (x fastest)."""
    ax = 2.0 * np.pi * (np.arange(m) - m // 2) / m
    grids = np.meshgrid(*([ax] * D), indexing="ij")  # grids[a][j_0, .., j_{D-1}]
    return np.stack([g.transpose(*reversed(range(D))).ravel() for g in grids], axis=1)


def symmetrized(name: str, tau: float) -> np.ndarray:
    """S = W^(1/2) H(tau) W^(-1/2) with W = diag(1 / f*)."""
    s = velset(name)
    w = np.sqrt(1.0 / np.asarray(s.f, dtype=np.float64))
    return w[:, None] * h_matrix(s, tau) / w[None, :]


def clusters(lam: np.ndarray, delta: float):
    """Groups of indices whose eigenvalues are chained by distances below delta."""
    n = len(lam)
    parent = list(range(n))

    def find(i):
        while parent[i] != i:
            i = parent[i]
        return i

    for i in range(n):
        for j in range(i + 1, n):
            if abs(lam[i] - lam[j]) < delta:
                parent[find(j)] = find(i)
    groups = {}
    for i in range(n):
        groups.setdefault(find(i), []).append(i)
    return list(groups.values())


def scan(name: str, tau: float, m: int, kappa: bool = True, delta: float = 1e-6):
    """Eigenvalues [m^D][q] (complex), spectral radius [m^D], kappa_W [m^D] (or None) and the
    normality defect [m^D] of Gamma_W."""
    s = velset(name)
    S = symmetrized(name, tau)
    ks = k_grid(s.D, m)
    cs = np.asarray(s.c, dtype=np.float64)[:, : s.D]
    lam = np.empty((len(ks), s.q), dtype=np.complex128)
    kap = np.empty(len(ks)) if kappa else None
    nu = np.empty(len(ks))
    for j, k in enumerate(ks):
        G = np.exp(-1j * (cs @ k))[:, None] * S
        ev = np.linalg.eigvals(G)
        lam[j] = ev
        GH = G.conj().T
        nu[j] = np.linalg.norm(GH @ G - G @ GH) / np.linalg.norm(G) ** 2
        if kappa:
            cols = []
            for grp in clusters(ev, delta):
                lc = ev[grp].mean()
                _, _, vh = np.linalg.svd(G - lc * np.eye(s.q))
                cols.append(vh[-len(grp):].conj().T)  # right singular vectors, smallest singular values
            kap[j] = np.linalg.cond(np.concatenate(cols, axis=1))
    return lam, np.abs(lam).max(axis=1), kap, nu
