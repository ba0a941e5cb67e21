"""Parity at the full size of the timed workload: the 64 x 4 x 256
cylindrical channel (eta = 0.975), 24 instances (12 Dean numbers in 25..60
for tau = 0.55 and 0.6), FP32, started from the laminar profile plus 1e-4
noise, in the launch configuration bench.py times.

The oracle recomputes one step at sampled nodes (walls, corners of the
periodic wrap, interior) from the library's own pre-step state, and the
whole-field mass budget is checked at every node.
"""
import numpy as np
import pytest

from gpu_helpers import lib, perm_lib_to_oracle, spec_of
from oracle.geometry import Channel, channel_geometry
from oracle.lbm import Params, Simulation, StreamMap, moments
from paper_1411_3133_gb300.workloads import cylinder_sweep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    L = lib()
    wl = cylinder_sweep()
    ch = Channel(**wl.geometry_kwargs())
    desc = spec_of(ch).desc()
    params = []
    for b in range(wl.batch):
        G = L.lb_force_for_dean("cylindrical", desc, wl.taus[b], wl.deans[b])
        params.append(L.make_params(wl.taus[b], G, False, wl.seeds[b], wl.noise_amp, True))
    ctx = L.LBContext(spec_of(ch), batch=wl.batch, precision="fp32")
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, 256)
    ctx.lb_init(params)
    ctx.lb_step(200)                        # leave the initial transient
    f0 = ctx.lb_get_populations()
    rho0, u0 = ctx.lb_macros()
    ctx.lb_step(1)
    f1 = ctx.lb_get_populations()
    ctx.close()
    return wl, ch, params, f0, f1, rho0, u0


def test_sampled_nodes_match_oracle(run):
    wl, ch, params, f0, f1, _, _ = run
    inv = perm_lib_to_oracle()
    geo, smap = channel_geometry(ch), StreamMap(ch)
    rs = [0, 1, 2, 3, 31, 60, 61, 62, 63]
    ts = [0, 3]
    zs = [0, 1, 2, 128, 253, 254, 255]
    cells = np.array([(r * ch.ntheta + t) * ch.n3 + z for r in rs for t in ts for z in zs])
    for b in (0, 13, wl.batch - 1):
        sim = Simulation(ch, Params(wl.taus[b], params[b].force_G), geo, smap)
        sim.f = f0[b][inv]
        want = sim.step_cells(cells)
        got = f1[b][inv][:, cells]
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
        rw, uw = moments(want)
        rg, ug = moments(got)
        assert np.abs(ug - uw).max() <= 1e-5 * np.abs(uw).max()
        assert np.abs(rg - rw).max() <= 1e-6 * np.abs(rw).max()


def _budget(ch, f0, f1, rho0, u0, b):
    """(change of sum f over one step, sum_x -2 rho' u^r Gamma^theta_{r theta})."""
    geo = channel_geometry(ch)
    g = np.repeat(geo["Gamma_hat"][:, 0, 1, 0, 1], ch.ntheta * ch.n3)   # h / r
    return f1[b].sum() - f0[b].sum(), (-2.0 * rho0[b] * u0[b, 0] * g).sum()


def test_mass_budget_full_field_fp32(run):
    """FP32 BGK conserves sum_l f only up to the rounding of each stored
    population (eps_32 relative per node, with a common sign); the budget
    holds to a few eps_32 of the total mass."""
    wl, ch, _, f0, f1, rho0, u0 = run
    eps32 = 2.0 ** -24
    for b in range(wl.batch):
        d, src = _budget(ch, f0, f1, rho0, u0, b)
        assert abs(d - src) <= 4 * eps32 * f0[b].sum(), (b, d, src)


def test_mass_budget_full_field_fp64():
    """The same workload in FP64: the budget holds to roundoff at every size."""
    L = lib()
    wl = cylinder_sweep(precision="fp64")
    ch = Channel(**wl.geometry_kwargs())
    desc = spec_of(ch).desc()
    params = [L.make_params(wl.taus[b], L.lb_force_for_dean("cylindrical", desc, wl.taus[b],
                                                           wl.deans[b]),
                            False, wl.seeds[b], wl.noise_amp, True) for b in range(wl.batch)]
    ctx = L.LBContext(spec_of(ch), batch=wl.batch, precision="fp64")
    ctx.lb_init(params)
    ctx.lb_step(50)
    f0 = ctx.lb_get_populations()
    rho0, u0 = ctx.lb_macros()
    ctx.lb_step(1)
    f1 = ctx.lb_get_populations()
    ctx.close()
    for b in range(wl.batch):
        d, src = _budget(ch, f0, f1, rho0, u0, b)
        assert abs(src) > 1e-4
        assert abs(d - src) <= 1e-12 * f0[b].sum(), (b, d, src)


def test_fields_finite_and_subsonic(run):
    _, _, _, _, f1, rho0, u0 = run
    assert np.isfinite(f1).all()
    assert np.abs(u0).max() < 0.5 and rho0.min() > 0.9
