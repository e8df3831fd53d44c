"""Pins of the oracle's stability scan (oracle/stability.py) against closed forms of Sec. 7-8 and
the symmetry of H in the f*-weighted inner product."""
import numpy as np
import pytest

import oracle
from oracle import stability as st

SETS = ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q9", "D3Q13", "D3Q19", "D3Q7_DI"]


def test_k_grid_order_and_range():
    ks = st.k_grid(2, 4)
    assert ks.shape == (16, 2)
    np.testing.assert_allclose(ks[1], [-np.pi / 2, -np.pi])  # x fastest
    np.testing.assert_allclose(ks[4], [-np.pi, -np.pi / 2])
    assert ks.min() == -np.pi and ks.max() == np.pi / 2


@pytest.mark.parametrize("name", SETS)
@pytest.mark.parametrize("tau", [0.5, 0.6, 1.3])
def test_spectrum_at_k_zero_is_conserved_moments_and_relaxation(name, tau):
    """Gamma(0) = H(tau) = (1 - 1/tau) I + (1/tau) E with E the projection onto the equilibria:
    eigenvalue 1 for the D + 2 conserved moments, 1 - 1/tau for the other q - D - 2 modes."""
    s = oracle.velset(name)
    m = 4
    lam, rho, _, _ = st.scan(name, tau, m, kappa=False)
    j0 = (m // 2) * sum(m ** a for a in range(s.D))  # k = 0
    want = np.sort(np.r_[np.ones(s.D + 2), np.full(s.q - s.D - 2, 1 - 1 / tau)])
    np.testing.assert_allclose(np.sort(lam[j0].real), want, atol=1e-12)
    np.testing.assert_allclose(lam[j0].imag, 0, atol=1e-12)


def test_d1q3_spectrum_is_the_pure_shift():
    """Sec. 8.1: for D1Q3, H = I and Gamma = diag(1, exp(-ik), exp(ik))."""
    m = 16
    lam, rho, kap, nu = st.scan("D1Q3", 0.8, m)
    for j, k in enumerate(st.k_grid(1, m)[:, 0]):
        want = np.sort_complex(np.array([1, np.exp(-1j * k), np.exp(1j * k)]))
        np.testing.assert_allclose(np.sort_complex(lam[j]), want, atol=1e-13)
    np.testing.assert_allclose(rho, 1, atol=1e-13)
    np.testing.assert_allclose(kap, 1, atol=1e-10)


@pytest.mark.parametrize("name", SETS)
def test_symmetrized_collision_matrix_is_symmetric(name):
    """H(tau) is self-adjoint in <x, y> = sum x_i y_i / f*_i (the equilibrium projection is
    symmetric in that inner product), so S = W^(1/2) H W^(-1/2) is symmetric, and at tau = 1/2 it
    is a reflection (S^2 = I: eigenvalues +-1)."""
    for tau in (0.5, 0.7):
        S = st.symmetrized(name, tau)
        np.testing.assert_allclose(S, S.T, atol=1e-14)
    S = st.symmetrized(name, 0.5)
    np.testing.assert_allclose(S @ S, np.eye(len(S)), atol=1e-13)


@pytest.mark.parametrize("name", SETS)
def test_gamma_is_normal_with_unit_spectrum_at_tau_half(name):
    """Secs. 8.1-8.3 show Gamma(1/2) unitary for every set but D3Q19; in the f*-weighted basis it
    is unitary for every set (D3Q19 included), so |lambda| = 1, the normality defect vanishes and
    the cluster-orthonormal eigenvectors are orthonormal: kappa_W = 1 at every k."""
    s = oracle.velset(name)
    m = {1: 16, 2: 8, 3: 4}[s.D]
    lam, rho, kap, nu = st.scan(name, 0.5, m)
    np.testing.assert_allclose(np.abs(lam), 1, atol=1e-12)
    np.testing.assert_allclose(nu, 0, atol=1e-13)
    np.testing.assert_allclose(kap, 1, atol=1e-9)


@pytest.mark.parametrize("name", ["D2Q5", "D3Q7", "D3Q19"])
def test_gamma_is_not_normal_away_from_tau_half(name):
    """For tau != 1/2, Gamma_W^H Gamma_W = S^2 differs from Gamma_W Gamma_W^H = D S^2 D^H unless D
    commutes with S^2, so the defect is positive at generic k and kappa_W > 1 there."""
    s = oracle.velset(name)
    lam, rho, kap, nu = st.scan(name, 0.7, 4)
    assert nu.max() > 1e-3
    assert kap.max() > 1.0 + 1e-3
    assert np.isfinite(kap).all()


@pytest.mark.parametrize("name", SETS)
@pytest.mark.parametrize("tau", [0.5, 0.55, 0.8, 2.0])
def test_spectral_radius_within_the_weighted_norm_bound(name, tau):
    """H(tau) is self-adjoint in <x, y> = sum x_i y_i / f*_i and D(k) is unitary and diagonal, so
    rho(Gamma) <= ||Gamma||_W = max(1, |1 - 1/tau|) = 1 for tau >= 1/2; at k = 0 the eigenvalue 1
    makes it equal."""
    s = oracle.velset(name)
    m = {1: 32, 2: 10, 3: 5}[s.D]
    lam, rho, _, _ = st.scan(name, tau, m, kappa=False)
    assert rho.max() <= 1 + 1e-12
    assert rho.max() >= 1 - 1e-12


@pytest.mark.parametrize("name", ["D2Q5", "D3Q19", "D3Q7_DI"])
def test_tau_below_half_is_unstable(name):
    """For tau < 1/2 the relaxation eigenvalue 1 - 1/tau leaves the unit disc (k = 0 already)."""
    s = oracle.velset(name)
    lam, rho, _, _ = st.scan(name, 0.45, 4, kappa=False)
    assert rho.max() == pytest.approx(1 / 0.45 - 1, rel=1e-12)
    assert rho.max() > 1
