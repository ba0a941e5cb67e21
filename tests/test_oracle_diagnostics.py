"""Oracle pins for the observables (Dean number, Sec. III Eq. dean-number and
its Sec. IV form; mean velocity; mean vorticity; vortex amplitude; mass).

What pins it: fields whose finite differences and weighted means are known in
closed form (a sampled sine along a periodic axis, a quadratic vanishing on
both walls), and a naive per-node loop on a tiny grid.
"""
import math

import numpy as np
import pytest

from oracle import lattice as L
from oracle.diagnostics import diagnostics
from oracle.geometry import Channel, channel_geometry


def test_closed_form_fields_cylinder():
    ch = Channel("cylindrical", 1.0, 1 / 0.975, 8, 2, 12)
    geo = channel_geometry(ch)
    nr, nt, n3 = ch.shape
    ir, it, i3 = np.meshgrid(np.arange(nr), np.arange(nt), np.arange(n3), indexing="ij")
    k, A, V = 2 * math.pi * 2 / n3, 3e-3, 0.02
    r = ch.r_inner + (ir + 0.5) * ch.h
    u = np.zeros(ch.shape + (3,))
    u[..., 0] = A * np.sin(k * i3)                      # periodic x3 -> central diff exact
    u[..., 2] = 1e-4 * (ir + 0.5) * (nr - 0.5 - ir)      # quadratic, zero on walls
    u[..., 1] = V / r                                    # speed r u^theta = V
    rho = 1.0 / r
    tau = 0.8
    d = diagnostics(ch, geo, tau, rho.reshape(-1), u.reshape(-1, 3))
    assert d["mean_v_theta"] == pytest.approx(V, rel=1e-14)
    nu = (tau - 0.5) * (1 - math.sqrt(0.4))
    assert d["dean"] == pytest.approx(V * nr / nu * math.sqrt((1 / 0.975 - 1) / 1.0), rel=1e-14)
    dur = A * math.sin(k) * np.cos(k * i3)
    duz = 1e-4 * (nr - 1 - 2 * ir)
    w = np.abs(dur - duz) * r
    assert d["mean_vorticity"] == pytest.approx(w.sum() / w.size, rel=1e-13)
    assert d["vortex_amp"] == pytest.approx(A / math.sqrt(2), rel=1e-13)
    assert d["vortex_amp_x3"] == pytest.approx(A / math.sqrt(2), rel=1e-13)
    assert d["mass_rho_prime"] == pytest.approx((1 / r).sum(), rel=1e-14)
    assert d["mass_physical"] == pytest.approx(r.sum(), rel=1e-14)
    assert d["nonfinite"] == 0


def test_naive_loop_ellipsoid_walls():
    ch = Channel("ellipsoidal", 1.0, 1.1, 8, 4, 8, b=0.9, periodic3=False)
    geo = channel_geometry(ch)
    rng = np.random.default_rng(0)
    n = ch.ncells
    rho = 1 + 0.01 * rng.random(n)
    u = 0.01 * rng.standard_normal((n, 3))
    tau = 0.6
    d = diagnostics(ch, geo, tau, rho, u)
    nr, nt, n3 = ch.shape
    U = u.reshape(nr, nt, n3, 3)
    num = den = vs = m = mp = 0.0
    for i in range(nr):
        for j in range(nt):
            for k in range(n3):
                def ur(kk):
                    return 0.0 if kk < 0 or kk >= n3 else U[i, j, kk, 0]

                def uz(ii):
                    return 0.0 if ii < 0 or ii >= nr else U[ii, j, k, 2]
                # one-sided at walls: u(0) + u(1)/3 ; interior central
                if k == 0:
                    d3 = ur(0) + ur(1) / 3
                elif k == n3 - 1:
                    d3 = -(ur(n3 - 1) + ur(n3 - 2) / 3)
                else:
                    d3 = 0.5 * (ur(k + 1) - ur(k - 1))
                if i == 0:
                    dr = uz(0) + uz(1) / 3
                elif i == nr - 1:
                    dr = -(uz(nr - 1) + uz(nr - 2) / 3)
                else:
                    dr = 0.5 * (uz(i + 1) - uz(i - 1))
                rr = geo["r_phys"][i, k]
                ph = (k + 0.5 - n3 / 2) * ch.h
                wOm = rr * ch.b * math.cos(ph)
                num += abs(d3 - dr) * wOm
                den += rr
                vs += rr * ch.b * math.cos(ph) * U[i, j, k, 1] * rr
                R = rho.reshape(nr, nt, n3)[i, j, k]
                m += R
                mp += R * (ch.b * rr * rr * math.cos(ph)) ** 2
    assert d["mean_vorticity"] == pytest.approx(num / den, rel=1e-13)
    assert d["mean_v_theta"] == pytest.approx(vs / den, rel=1e-13)
    assert d["mass_rho_prime"] == pytest.approx(m, rel=1e-14)
    assert d["mass_physical"] == pytest.approx(mp, rel=1e-13)


def test_nonfinite_count():
    ch = Channel("cylindrical", 1.0, 1.1, 8, 1, 8)
    geo = channel_geometry(ch)
    rho = np.ones(ch.ncells)
    u = np.zeros((ch.ncells, 3))
    rho[3] = np.nan
    u[10, 1] = np.inf
    u[11, 0] = np.nan
    assert diagnostics(ch, geo, 0.7, rho, u)["nonfinite"] == 3
