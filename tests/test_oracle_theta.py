"""Oracle pins for the theta-resolved double-curved channel (the metric of
each theta node's own theta, Sec. IV; periodic theta axis).

What pins it:
  * at every node, the scaled metric equals the Sec. IV metric printed in
    tests/golden/printed_geometry.txt evaluated at the node's physical
    (r, theta, phi), transformed by the lattice map (g'_ij = g_ij s_i s_j);
  * the nodes are placed symmetrically about theta = 0: for odd N_theta the
    middle theta layer is the theta-frozen channel's geometry, and mirrored
    layers carry mirrored off-diagonal components (g_r theta, g_theta phi
    odd in theta; every other component even);
  * b = 1 (a spherical shell) has no theta dependence: the resolved channel
    equals the frozen one field by field (to rounding), and so does an LB
    run on it;
  * the Christoffel symbols are those of the frozen channel at every theta
    (Sec. IV: they depend on neither b nor theta);
  * an LB run keeps the exact mass budget of the frozen channel's pin with
    the per-node fields: sum_l f changes by sum_x -2 rho' u^i Gamma^j_ij.
"""
import numpy as np
import pytest

from oracle.geometry import Channel, channel_geometry, geometry_shape, node_coordinates
from oracle.lbm import Params, Simulation
from tests.test_oracle_geometry import _printed_arrays


def _resolved(b=0.9, nr=8, nt=5, n3=10, periodic3=False, dtheta_scale=8.0):
    return Channel("ellipsoidal", 1.0, 1.2, nr, nt, n3, b=b, periodic3=periodic3,
                   dtheta_scale=dtheta_scale, d3_scale=2.0, theta_resolved=True)


def _frozen(ch):
    return Channel(ch.metric, ch.r_inner, ch.r_outer, ch.nr, ch.ntheta, ch.n3, b=ch.b,
                   periodic3=ch.periodic3, dtheta_scale=ch.dtheta_scale, d3_scale=ch.d3_scale,
                   wall=ch.wall)


def test_theta_nodes_and_shapes():
    ch = _resolved()
    assert geometry_shape(ch) == (8, 5, 10)
    pts = node_coordinates(ch).reshape(8, 5, 10, 3)
    yt = pts[0, :, 0, 1]
    assert np.allclose(yt, (np.arange(5) - 2) * ch.h, atol=1e-15)    # centred, one h apart
    assert np.array_equal(pts[:, 2, :, :], node_coordinates(_frozen(ch)).reshape(8, 10, 3))


@pytest.mark.parametrize("b", [0.9, 1.6])
def test_resolved_metric_is_the_printed_metric_at_each_node(b):
    ch = _resolved(b=b)
    geo = channel_geometry(ch)
    s = np.array([1.0, ch.dtheta_scale, ch.d3_scale])
    phys = node_coordinates(ch) * s                       # physical (r, theta, phi)
    assert np.abs(phys[:, 1]).max() > 0.3                  # theta well away from 0
    gp, _ = _printed_arrays("ellipsoidal", phys, b)
    gp = gp * s[None, :, None] * s[None, None, :]
    g = geo["g"].reshape(-1, 3, 3)
    assert np.abs(g - gp).max() < 1e-13
    # every off-diagonal component is present off theta = 0
    off = np.abs(g[:, [0, 0, 1], [1, 2, 2]]).max(axis=0)
    assert (off > 1e-3).all()
    assert np.allclose(geo["sqrtg"].reshape(-1), np.sqrt(np.linalg.det(gp)), rtol=1e-13)


def test_middle_layer_is_the_frozen_channel_and_layers_mirror():
    ch = _resolved(nt=5)
    geo, fz = channel_geometry(ch), channel_geometry(_frozen(ch))
    for key in ("g", "ginv", "Delta", "sqrtg", "Gamma_hat", "fdir", "speed", "wA", "wOmega"):
        assert np.abs(geo[key][:, 2] - fz[key]).max() < 1e-14, key
    g = geo["g"]
    odd = {(0, 1), (1, 2)}
    for it in range(5):
        m = 4 - it
        for i in range(3):
            for j in range(3):
                sign = -1.0 if (min(i, j), max(i, j)) in odd else 1.0
                assert np.abs(g[:, it, :, i, j] - sign * g[:, m, :, i, j]).max() < 1e-14
    assert np.abs(g[:, 0, :, 0, 1]).max() > 1e-3


def test_sphere_has_no_theta_dependence():
    ch = _resolved(b=1.0, nt=4)
    geo, fz = channel_geometry(ch), channel_geometry(_frozen(ch))
    for key in ("g", "Delta", "sqrtg", "Gamma_hat", "fdir", "speed", "wA", "wOmega"):
        for it in range(4):
            assert np.abs(geo[key][:, it] - fz[key]).max() < 1e-13, key


def test_christoffel_symbols_do_not_depend_on_theta():
    ch = _resolved(b=0.7, nt=6)
    geo, fz = channel_geometry(ch), channel_geometry(_frozen(ch))
    for it in range(6):
        assert np.abs(geo["Gamma_hat"][:, it] - fz["Gamma_hat"]).max() < 1e-14


def test_lb_on_a_resolved_sphere_equals_the_frozen_run():
    ch = _resolved(b=1.0, nr=8, nt=3, n3=9, dtheta_scale=2.0)
    fz = _frozen(ch)
    rng = np.random.default_rng(4)
    u0 = 1e-3 * rng.standard_normal((ch.ncells, 3))
    out = []
    for c in (ch, fz):
        sim = Simulation(c, Params(0.7, 2e-5))
        sim.init_rest(u0)
        sim.step(6)
        out.append(sim.f)
    assert np.abs(out[0] - out[1]).max() < 1e-14 * np.abs(out[1]).max()


def test_resolved_channel_keeps_the_exact_mass_budget():
    """Every step changes sum_l f by sum_x -2 rho' u^i Gamma^j_ij (streaming
    and bounce-back permute, BGK conserves sum_l f; the velocity-dependent
    Christoffel force carries this zeroth moment) with the per-node fields of
    the resolved channel."""
    from oracle.lbm import moments
    ch = _resolved(b=0.8, nr=8, nt=4, n3=9, dtheta_scale=2.0)
    sim = Simulation(ch, Params(0.8, 1e-4))
    rng = np.random.default_rng(9)
    sim.init_rest(1e-3 * rng.standard_normal((ch.ncells, 3)))
    for _ in range(3):
        m0 = sim.f.sum()
        rho, u = moments(sim.streamed())
        src = -2.0 * np.einsum("n,ni,njij->n", rho, u, sim.Gamma_hat).sum()
        sim.step()
        assert abs(sim.f.sum() - m0 - src) <= 1e-14 * m0
        assert abs(src) > 1e-10 * m0


def test_simulation_fields_follow_the_cell_order():
    """Cell index (i_r N_theta + i_theta) N_3 + i_3 carries the metric of its
    own node: Delta = g'^-1 - 1 of the printed metric at (r, theta, phi) of
    (i_r, i_theta, i_3), and the body force direction g'^{i theta}."""
    ch = _resolved(b=0.85, nr=8, nt=4, n3=9)
    sim = Simulation(ch, Params(0.8, 1e-4))
    s = np.array([1.0, ch.dtheta_scale, ch.d3_scale])
    for ir, it, i3 in ((2, 1, 3), (6, 3, 0), (0, 0, 8)):
        cell = (ir * ch.ntheta + it) * ch.n3 + i3
        y = np.array([[ch.r_inner + (ir + 0.5) * ch.h, (it + 0.5 - ch.ntheta / 2) * ch.h,
                       (i3 + 0.5 - ch.n3 / 2) * ch.h]])
        gp, _ = _printed_arrays("ellipsoidal", y * s, ch.b)
        ginv = np.linalg.inv(gp[0] * s[:, None] * s[None, :])
        assert np.abs(sim.Delta[cell] - (ginv - np.eye(3))).max() < 1e-12
        assert np.abs(sim.fext[cell] - 1e-4 * ginv[:, 1]).max() < 1e-16


def test_observables_of_a_resolved_sphere_are_the_frozen_ones():
    from oracle.diagnostics import diagnostics
    ch = _resolved(b=1.0, nr=8, nt=3, n3=9, dtheta_scale=2.0)
    rng = np.random.default_rng(6)
    rho = 1.0 + 1e-3 * rng.standard_normal(ch.ncells)
    u = 1e-2 * rng.standard_normal((ch.ncells, 3))
    a = diagnostics(ch, channel_geometry(ch), 0.8, rho, u)
    b = diagnostics(_frozen(ch), channel_geometry(_frozen(ch)), 0.8, rho, u)
    for k in a:
        assert abs(a[k] - b[k]) <= 1e-12 * max(1.0, abs(b[k])), k
