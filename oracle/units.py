"""Non-dimensionalisation of Sec. 2.1, restated for the oracle (TEST INFRASTRUCTURE ONLY).

Dimensional quantities (underlined in the paper) relate to the non-dimensional ones by
    rho0_dim = rho* rho0,  rho'_dim = rho* rho',  theta0_dim = theta* theta0,
    theta'_dim = theta* theta',  u'_dim = u* u',  u* = x* / t*,  (u*)^2 = theta*,
    x_dim = x* x,  t_dim = t* t.
A velocity set fixes the non-dimensional rho0 and theta0 (Sec. 8), so a dimensional background
(rho0_dim, theta0_dim) and a length scale x* fix every scale.  A lattice of n cells on a
non-dimensional length L advances time eps = L / n per step (Sec. 6: dx = dt = eps).
"""
from __future__ import annotations

import math

from . import VelSet


def scales(set_name: str, rho0_dim: float, theta0_dim: float, x_star: float = 1.0) -> dict:
    s = VelSet(set_name)
    rho_star = rho0_dim / s.rho0
    theta_star = theta0_dim / s.theta0
    u_star = math.sqrt(theta_star)
    t_star = x_star / u_star
    return {"rho_star": rho_star, "theta_star": theta_star, "u_star": u_star, "x_star": x_star, "t_star": t_star}


def run_length(set_name: str, rho0_dim: float, theta0_dim: float, length_dim: float, n_cells: int, t_end_dim: float,
               x_star: float = 1.0) -> dict:
    """Non-dimensional end time T = t_end_dim / t*, lattice step eps = (length_dim / x*) / n,
    number of steps round(T / eps) and the end-time mismatch T - steps * eps (Table 1)."""
    sc = scales(set_name, rho0_dim, theta0_dim, x_star)
    T = t_end_dim / sc["t_star"]
    eps = (length_dim / x_star) / n_cells
    steps = int(math.floor(T / eps + 0.5))  # T, eps > 0: halves round up
    return dict(sc, T=T, eps=eps, steps=steps, mismatch=T - steps * eps)
