"""Pins of the oracle's equilibrium (Dirichlet) walls, the paper's own wall
condition (Sec. III: zero wall velocity imposed through the equilibrium on
both walls at every step),
against what the mathematics fixes:

* the flat rest state is a fixed point with walls on two axes;
* streaming: the clamp onto the wall layer, by an independent per-node loop;
* wall nodes leave every step as f^eq(rho', 0): zero momentum, exactly;
* plane and curved Poiseuille flow between wall NODES (walls on the end
  nodes, d = (N_r - 1) h): the equilibrium condition is first-order
  accurate, so the error against the closed form halves with h. Walls
  misplaced by half a node, a mirrored ghost or a missing wall reset would
  converge to another profile or not at all.
"""
import math

import numpy as np
import pytest

from analytic import curved_poiseuille_coeffs, nu
from oracle import lattice as OL
from oracle.geometry import Channel, channel_geometry
from oracle.lbm import Params, Simulation, StreamMap, equilibrium, moments
from test_oracle_physics import _run_to_steady


def test_flat_rest_state_is_fixed_point_with_walls_on_two_axes():
    ch = Channel("flat", 0.0, 1.0, 9, 2, 8, periodic3=False, wall="equilibrium")
    sim = Simulation(ch, Params(0.7))
    sim.init_rest()
    f0 = sim.f.copy()
    sim.step(5)
    assert np.abs(sim.f - f0).max() < 1e-15


def test_clamped_streaming_against_a_node_loop():
    ch = Channel("flat", 0.0, 1.0, 7, 3, 8, periodic3=False, wall="equilibrium")
    smap = StreamMap(ch)
    nr, nt, n3 = ch.shape
    for l in range(OL.Q):
        c = OL.C[l]
        for ir in range(nr):
            for it in range(nt):
                for i3 in range(n3):
                    yr = min(max(ir - c[0], 0), nr - 1)        # beyond a wall: the wall node
                    yt = (it - c[1]) % nt                      # periodic theta
                    y3 = min(max(i3 - c[2], 0), n3 - 1)
                    cell = (ir * nt + it) * n3 + i3
                    assert smap.src_cell[l, cell] == (yr * nt + yt) * n3 + y3
                    assert smap.src_pop[l, cell] == l


def test_wall_nodes_leave_each_step_at_rest_equilibrium():
    ch = Channel("cylindrical", 1.0, 1.1, 9, 2, 7, wall="equilibrium")
    sim = Simulation(ch, Params(0.8, 1e-3))
    rng = np.random.default_rng(5)
    sim.init_rest(rng.uniform(-1e-2, 1e-2, size=(ch.ncells, 3)))
    fs = sim.streamed()
    sim.step(1)
    w = sim.wall_nodes
    assert w.sum() == 2 * ch.ntheta * ch.n3
    rho, u = moments(sim.f[:, w])
    assert np.abs(u).max() < 1e-15
    rho_s, _ = moments(fs[:, w])
    np.testing.assert_allclose(rho, rho_s, rtol=1e-14)
    feq = equilibrium(rho_s, np.zeros((w.sum(), 3)), sim.Delta[w])
    np.testing.assert_allclose(sim.f[:, w], feq, rtol=1e-14, atol=0)


def test_node_positions_put_the_walls_on_the_end_nodes():
    ch = Channel("cylindrical", 1.0, 1.1, 11, 1, 7, periodic3=False, wall="equilibrium")
    r = channel_geometry(ch)["r_phys"][:, 0]
    assert r[0] == pytest.approx(1.0, abs=1e-15) and r[-1] == pytest.approx(1.1, abs=1e-14)
    assert ch.h == pytest.approx(0.01)


def _plane_profile(n, G, tau):
    i = np.arange(n)
    return G / (2.0 * nu(tau)) * i * (n - 1 - i)


def test_plane_poiseuille_first_order():
    tau, G = 1.0, 1e-6
    errs = []
    for n in (9, 17, 33):
        ch = Channel("flat", 0.0, 1.0, n, 1, 1, wall="equilibrium")
        sim = Simulation(ch, Params(tau, G))
        ua = _plane_profile(n, G, tau)
        u0 = np.zeros((n, 3))
        u0[:, 1] = ua
        sim.init_fields(np.ones(n), u0)
        u = _run_to_steady(sim, ua, 20000)
        errs.append(np.abs(u[:, 1] - ua).max() / ua.max())
    assert errs[0] < 0.1
    assert errs[0] / errs[1] > 1.7 and errs[1] / errs[2] > 1.7, errs


@pytest.mark.slow
def test_curved_poiseuille_first_order():
    tau, G, ri, ro = 1.0, 1e-6, 1.0, 1.0 / 0.975
    errs = []
    for n in (9, 17, 33):
        ch = Channel("cylindrical", ri, ro, n, 1, 1, wall="equilibrium")
        sim = Simulation(ch, Params(tau, G))
        r = ri + np.arange(n) * ch.h
        A, B, C = curved_poiseuille_coeffs(ri, ro, ch.h, G, tau)
        uth = (A * r * np.log(r) + B * r + C / r) / r
        u0 = np.zeros((n, 3))
        u0[:, 1] = uth
        sim.init_rest(u0)
        u = _run_to_steady(sim, uth, 3 * n * n / 0.18)
        errs.append(np.abs(u[:, 1] - uth).max() / uth.max())
    assert errs[0] < 0.1
    assert errs[0] / errs[1] > 1.7 and errs[1] / errs[2] > 1.7, errs


def test_observables_use_the_wall_value_and_one_sided_differences():
    """u^3 = i (N_r - 1 - i) vanishes on both wall nodes; its r-derivative
    N_r - 1 - 2 i is exact for the second-order differences everywhere, so
    the mean |vorticity| of the flat channel is the node mean of |N_r - 1 -
    2 i|. Garbage velocities on the wall nodes must not change anything."""
    from oracle.diagnostics import diagnostics
    ch = Channel("flat", 0.0, 1.0, 9, 2, 8, periodic3=False, wall="equilibrium")
    geo = channel_geometry(ch)
    nr, nt, n3 = ch.shape
    i = np.arange(nr)[:, None, None] * np.ones((1, nt, n3))
    u = np.zeros(ch.shape + (3,))
    u[..., 2] = i * (nr - 1 - i)
    u[:, :, 0, 2] = 0.0
    u[:, :, -1, 2] = 0.0                      # x3 wall nodes hold the wall value too
    rho = np.ones(ch.ncells)
    d = diagnostics(ch, geo, 0.8, rho, u.reshape(-1, 3))
    expect = np.abs(nr - 1 - 2 * i)            # d_r u^3; d_3 u^r = 0 everywhere
    expect[:, :, 0] = 0.0                       # u^3 = 0 on the x3 wall columns
    expect[:, :, -1] = 0.0
    assert d["mean_vorticity"] == pytest.approx(expect.mean(), rel=1e-14)
    noisy = u.copy()
    noisy[0] = 7.0
    noisy[-1] = -3.0
    noisy[:, :, 0] = 5.0
    noisy[:, :, -1] = 2.0
    d2 = diagnostics(ch, geo, 0.8, rho, noisy.reshape(-1, 3))
    for k in ("mean_vorticity", "mean_v_theta", "vortex_amp", "vortex_amp_x3", "max_speed"):
        assert d2[k] == pytest.approx(d[k], rel=1e-14, abs=1e-300), k


def test_dean_number_uses_the_wall_node_width():
    from oracle.diagnostics import diagnostics
    ch = Channel("cylindrical", 1.0, 1.1, 11, 1, 4, wall="equilibrium")
    geo = channel_geometry(ch)
    u = np.zeros((ch.ncells, 3))
    u[:, 1] = 0.01
    d = diagnostics(ch, geo, 0.8, np.ones(ch.ncells), u)
    # <v_theta> = mean of r u^theta over the 9 fluid nodes and 2 wall nodes (value 0)
    r = 1.0 + 0.01 * np.arange(11)
    vmean = (r * 0.01)[1:-1].sum() / 11
    assert d["mean_v_theta"] == pytest.approx(vmean, rel=1e-13)
    nu_l = (0.8 - 0.5) * OL.CS2
    assert d["dean"] == pytest.approx(vmean * 10 / nu_l * math.sqrt(0.1 / 1.0), rel=1e-13)
