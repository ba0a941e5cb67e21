"""Macroscopic observables of a channel, computed by brute force.

Paper:
  * Dean number, Eq. (dean-number) in Sec. III and its Sec. IV form:
    De = <v_theta> d / nu * sqrt(d / R), nu = (tau - 1/2) cs^2 (lattice),
    R = r_i (cylinder) or r_i b^2 (ellipsoid).
  * mean streamwise velocity, Sec. IV: <v_theta> = (1/S) int u^theta r^2 b
    cos(phi) dr dphi with S = int r dr dphi.
  * mean absolute streamwise vorticity, Sec. III (cylinder) and Sec. IV
    (ellipsoid): <omega^theta> = (1/S) int |d_3 u^r - d_r u^3| w dr dx3.

Readings:
  * Both integrals are written with the metric: the physical streamwise speed
    is sqrt(g_theta theta) u^theta, the cross-section's area element is
    sqrt(det of its (r, x3) metric block) (1 for the cylinder, r for the
    ellipsoid), and the vorticity weight is sqrt(g_theta theta) of the
    physical metric (r, resp. r b cos phi). For the cylinder, where the paper
    writes no formula for <v_theta>, this gives the plain area mean of r u^theta.
  * Sums run over every node (all theta planes); cell sizes cancel.
  * Derivatives are lattice-unit finite differences: central inside,
    second-order one-sided at the first and last node of a walled axis using
    u = 0 on the wall half a node away; periodic axes wrap.
  * Equilibrium (Dirichlet) walls: the wall nodes' velocity is the wall
    value 0 in every observable (their streamed moments are replaced in the
    collision); derivatives at a wall node are the second-order one-sided
    differences of the node values; the channel width in lattice units is
    N_r - 1 (wall nodes at both ends) in the Dean number.
  * vortex amplitude = rms of u^r over all nodes; vortex_amp_x3 = rms of
    u^r minus its mean along x3 (the x3-periodic part that Dean vortices
    carry); max_speed = largest Euclidean norm of the coordinate velocity.
  * mass: sum of rho' over nodes, and the physical mass sum of rho sqrt(g)
    = sum of rho' g (rho = rho' sqrt(g), Sec. II; volume element sqrt(g)).

Oracle module: test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import math

import numpy as np

from . import lattice as L
from .geometry import Channel


def _d_axis(u, axis, walled, on_nodes=False):
    """Derivative of u (nr, nt, n3) along an axis, lattice units; on_nodes:
    the walls are the first and last node (equilibrium walls)."""
    n = u.shape[axis]
    u = np.moveaxis(u, axis, 0)
    d = np.empty_like(u)
    if walled and on_nodes:
        d[1:-1] = 0.5 * (u[2:] - u[:-2])
        d[0] = 0.5 * (-3.0 * u[0] + 4.0 * u[1] - u[2])
        d[-1] = 0.5 * (3.0 * u[-1] - 4.0 * u[-2] + u[-3])
    elif walled:
        if n == 1:
            d[0] = 0.0
        else:
            d[1:-1] = 0.5 * (u[2:] - u[:-2])
            # value 0 on the wall at -1/2 and at n - 1/2 (quadratic fit)
            d[0] = u[0] + u[1] / 3.0
            d[-1] = -(u[-1] + u[-2] / 3.0)
    else:
        d[:] = 0.5 * (np.roll(u, -1, axis=0) - np.roll(u, 1, axis=0))
    return np.moveaxis(d, 0, axis)


def diagnostics(ch: Channel, geo: dict, tau: float, rho, u) -> dict:
    """Observables from rho' (n,) and u (n,3) of one channel."""
    shp = ch.shape
    rho = np.asarray(rho, float).reshape(shp)
    u = np.asarray(u, float).reshape(shp + (3,))

    def cells(a):
        if ch.theta_resolved:
            return np.asarray(a).reshape(shp)
        return np.broadcast_to(np.asarray(a).reshape(ch.nr, 1, ch.n3), shp)

    sqrtg, speed = cells(geo["sqrtg"]), cells(geo["speed"])
    wA, wOm = cells(geo["wA"]), cells(geo["wOmega"])

    eqw = ch.wall == "equilibrium"
    if eqw:  # wall nodes carry the Dirichlet velocity 0
        u = u.copy()
        u[0], u[-1] = 0.0, 0.0
        if not ch.periodic3:
            u[:, :, 0], u[:, :, -1] = 0.0, 0.0
    finite = np.isfinite(rho) & np.isfinite(u).all(axis=-1)
    out = {"nonfinite": int((~finite).sum())}
    out["mass_rho_prime"] = float(rho.sum())
    out["mass_physical"] = float((sqrtg * sqrtg * rho).sum())
    vmean = float((speed * u[..., 1] * wA).sum() / wA.sum())
    out["mean_v_theta"] = vmean
    nu = (tau - 0.5) * L.CS2
    d = ch.r_outer - ch.r_inner
    R = ch.curvature_radius
    width = d / ch.h                                   # N_r, or N_r - 1 with wall nodes
    out["dean"] = 0.0 if math.isinf(R) else vmean * width / nu * math.sqrt(d / R)
    walled = ch.walled
    w = _d_axis(u[..., 0], 2, walled[2], eqw) - _d_axis(u[..., 2], 0, walled[0], eqw)
    out["mean_vorticity"] = float((np.abs(w) * wOm).sum() / wA.sum())
    out["vortex_amp"] = float(np.sqrt((u[..., 0] ** 2).mean()))
    ur_fluct = u[..., 0] - u[..., 0].mean(axis=2, keepdims=True)
    out["vortex_amp_x3"] = float(np.sqrt((ur_fluct ** 2).mean()))
    out["max_speed"] = float(np.sqrt((u ** 2).sum(axis=-1)).max())
    return out
