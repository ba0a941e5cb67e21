"""Closed-form laminar channel flows used as physical pins (test helper).

Lattice units: node i of a walled axis sits at i + 1/2 from the wall, time
step 1, kinematic viscosity nu = (tau - 1/2) cs^2 (Eq. viscosity, Sec. II),
body force G per step applied as the covariant streamwise component.
"""
import math

import numpy as np

CS2 = 1.0 - math.sqrt(2.0 / 5.0)


def nu(tau):
    return (tau - 0.5) * CS2


def plane_poiseuille(n, G, tau):
    """u(y) = G/(2 nu) (y - y0)(y1 - y) between walls at y0 = -1/2, y1 = n - 1/2."""
    y = np.arange(n) + 0.0
    return G / (2.0 * nu(tau)) * (y + 0.5) * (n - 0.5 - y)


def curved_poiseuille_coeffs(r_i, r_o, h, G, tau):
    """Azimuthal speed v(r) = A r ln r + B r + C / r between concentric
    cylinders with v(r_i) = v(r_o) = 0, for a constant covariant force G per
    step (physical force density G/(h r) along e_theta, nu_phys = nu h).

    Steady axisymmetric momentum balance nu (v'' + v'/r - v/r^2) = -G/(h^2 r)
    (in the units where lattice speeds equal physical speeds) has the
    particular solution A r ln r with A = -G / (2 nu h^2).
    """
    A = -G / (2.0 * nu(tau) * h * h)
    M = np.array([[r_i, 1.0 / r_i], [r_o, 1.0 / r_o]])
    rhs = -A * np.array([r_i * math.log(r_i), r_o * math.log(r_o)])
    B, C = np.linalg.solve(M, rhs)
    return A, B, C


def curved_poiseuille(r_i, r_o, n, G, tau):
    """(r, v(r), u^theta = v/r) at the n nodes r = r_i + (i + 1/2) h."""
    h = (r_o - r_i) / n
    r = r_i + (np.arange(n) + 0.5) * h
    A, B, C = curved_poiseuille_coeffs(r_i, r_o, h, G, tau)
    v = A * r * np.log(r) + B * r + C / r
    return r, v, v / r
