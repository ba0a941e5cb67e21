"""Pins of the oracle's equilibrium (Dirichlet) walls, the paper's own wall
condition (Sec. III: f^eq evaluated with u = 0 at r_i and r_o every step),
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
