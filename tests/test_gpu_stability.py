"""GPU stability scan (include/lee_stability.h) against the oracle's (oracle/stability.py):
eigenvalues, spectral radius, normality defect and kappa_W on grids of wave vectors, for every
set and several tau; then properties of Theorem 1 at full grid sizes."""
import numpy as np
import pytest

import oracle
from oracle import stability as st

pytestmark = pytest.mark.gpu

SETS = ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q9", "D3Q13", "D3Q19", "D3Q7_DI"]


def gpu_scan(lee, name, tau, m, delta=1e-6):
    import torch

    s = oracle.velset(name)
    n = m ** s.D
    dev = torch.device("cuda")
    rho = torch.empty(n, dtype=torch.float64, device=dev)
    lam = torch.empty((n, s.q, 2), dtype=torch.float64, device=dev)
    kap = torch.empty(n, dtype=torch.float64, device=dev)
    nu = torch.empty(n, dtype=torch.float64, device=dev)
    lee.lee_stability_scan(name, tau, m, rho, lam, kap, nu, delta=delta)
    lam = lam.cpu().numpy()
    return lam[..., 0] + 1j * lam[..., 1], rho.cpu().numpy(), kap.cpu().numpy(), nu.cpu().numpy()


def match_multisets(a, b):
    """Largest distance after greedily pairing each eigenvalue of a with the nearest unused one of b."""
    worst = 0.0
    for x, y in zip(a, b):
        used = np.zeros(len(y), bool)
        for v in x:
            d = np.abs(y - v) + used * 1e9
            i = int(np.argmin(d))
            used[i] = True
            worst = max(worst, float(d[i]))
    return worst


@pytest.mark.parametrize("name", SETS)
@pytest.mark.parametrize("tau", [0.5, 0.7, 0.45])
def test_scan_matches_oracle(gpu_lib, name, tau):
    s = oracle.velset(name)
    m = {1: 64, 2: 12, 3: 5}[s.D]
    lam_g, rho_g, kap_g, nu_g = gpu_scan(gpu_lib, name, tau, m)
    lam_o, rho_o, kap_o, nu_o = st.scan(name, tau, m)
    np.testing.assert_allclose(rho_g, rho_o, rtol=0, atol=1e-11)
    assert match_multisets(lam_g, lam_o) < 1e-9
    np.testing.assert_allclose(nu_g, nu_o, rtol=1e-10, atol=1e-13)
    # kappa where the clusters are unambiguous: every eigenvalue distance below 1e-9 or above 1e-4
    d = np.abs(lam_o[:, :, None] - lam_o[:, None, :])
    clear = np.all((d < 1e-9) | (d > 1e-4), axis=(1, 2))
    assert clear.mean() > 0.5
    np.testing.assert_allclose(kap_g[clear], kap_o[clear], rtol=1e-7)


@pytest.mark.parametrize("name,m", [("D2Q5", 256), ("D3Q19", 32), ("D3Q7_DI", 32)])
def test_theorem1_conditions_at_full_grids(gpu_lib, name, m):
    """tau = 1/2: rho = 1, kappa_W = 1 and Gamma_W normal at every k (the weighted form of the
    unitarity shown in Secs. 8.1-8.3, D3Q19 included); tau = 0.7: rho <= 1 with kappa_W bounded;
    tau = 0.45: rho = 1/tau - 1 > 1 (unstable)."""
    lam, rho, kap, nu = gpu_scan(gpu_lib, name, 0.5, m)
    assert np.isfinite(rho).all()
    np.testing.assert_allclose(np.abs(lam), 1, atol=1e-11)
    np.testing.assert_allclose(kap, 1, atol=1e-8)
    assert nu.max() < 1e-12
    lam, rho, kap, nu = gpu_scan(gpu_lib, name, 0.7, m)
    assert rho.max() <= 1 + 1e-12 and rho.max() >= 1 - 1e-12
    assert np.isfinite(kap).all() and kap.max() < 1e3
    lam, rho, kap, nu = gpu_scan(gpu_lib, name, 0.45, m)
    assert rho.max() == pytest.approx(1 / 0.45 - 1, rel=1e-12)
