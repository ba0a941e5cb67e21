"""Parity at the full size of every timed workload, in the launch
configuration bench.py times (128 threads per block, the library's automatic
step kernel, CUDA-graph replay):

* the Dean sweep: 64 x 4 x 256 cylindrical channel (eta = 0.975), 24
  instances (12 Dean numbers in 25..60 for tau = 0.55 and 0.6), started from
  the laminar profile plus 1e-4 noise, in FP32 storage (region-split step)
  and in FP16 and BF16 deviation storage;
* the four-wall double-curved channel of Sec. IV.B (R2/R1 = 1, 64 x 4 x
  256), 24 instances, FP32 and FP16 storage (tiled step; the 2-byte kernels
  stage each node's stream-table row in shared memory);
* the 128-channel mixed batch (cylinders and double-curved channels, N_r in
  {32, 48, 64}, N_3 in 128..512), FP32 and BF16 storage, one lb_batch after
  its autotuner.

The oracle recomputes one step at sampled nodes (the wall layers, the
corners of the periodic wrap and of the x3 walls, the interior) from the
library's own pre-step state; the FP32 cylinder's mass budget is checked at
every node. A 2000-step laminar FP32 run is compared with the oracle over
the whole field.
"""
import numpy as np
import pytest

from gpu_helpers import Twin, lib, max_rel, perm_lib_to_oracle, spec_of
from oracle.geometry import Channel, channel_geometry
from oracle.lbm import Params, Simulation, StreamMap, moments
from paper_1411_3133_gb300.workloads import (cylinder_sweep, ellipsoid_cross_section, force_reference_cylinder,
                                             mixed_batch, noise_field)

pytestmark = pytest.mark.gpu

BENCH_THREADS = 128          # bench.py --threads default
# per storage format: (populations, u against max |u|, rho' against max rho')
TOL = {"fp32": (1e-6, 1e-5, 1e-6), "fp16_shifted": (1e-4, 1e-4, 1e-4), "bf16_shifted": (1e-3, 1e-3, 1e-3)}
# channels started from rest keep the rest state as the 2-byte storage
# reference, so the stored deviations are O(u / cs^2) and the format's
# mantissa bounds u's error: 2^-11 (FP16) and 2^-8 (BF16) relative, i.e.
# 1e-3 and 1e-2 of u_max (the reduced-precision bound; the sweep above stores
# deviations from the laminar rows and keeps 1e-4 / 1e-3)
TOL_REST = {"fp32": TOL["fp32"], "fp16_shifted": (1e-4, 1e-3, 1e-4), "bf16_shifted": (1e-3, 1e-2, 1e-3)}


def _sample_cells(ch):
    """Wall layers and their neighbours on r (and on x3 when walled), the
    periodic wrap's corners and the middle, at the first and last theta."""
    def pick(n):
        return sorted({0, 1, 2, 3, n // 2, n - 4, n - 3, n - 2, n - 1})
    return np.array([(r * ch.ntheta + t) * ch.n3 + z
                     for r in pick(ch.nr) for t in sorted({0, ch.ntheta - 1}) for z in pick(ch.n3)])


def _check_step(ch, tau, G, f0, f1, tol, geo=None, smap=None):
    """One oracle step at the sampled cells from f0 (library order) against
    the library's f1 at those cells."""
    inv = perm_lib_to_oracle()
    cells = _sample_cells(ch)
    sim = Simulation(ch, Params(tau, G), geo if geo is not None else channel_geometry(ch),
                     smap if smap is not None else StreamMap(ch))
    sim.f = f0[inv]
    want = sim.step_cells(cells)
    got = f1[inv][:, cells]
    tf, tu, tr = tol
    assert np.abs(got - want).max() <= tf * np.abs(want).max()
    rw, uw = moments(want)
    rg, ug = moments(got)
    assert np.abs(ug - uw).max() <= tu * np.abs(uw).max()
    assert np.abs(rg - rw).max() <= tr * np.abs(rw).max()


def _sweep_run(precision):
    L = lib()
    wl = cylinder_sweep(precision=precision)
    ch = Channel(**wl.geometry_kwargs())
    desc = spec_of(ch).desc()
    params = []
    for b in range(wl.batch):
        G = L.lb_force_for_dean("cylindrical", desc, wl.taus[b], wl.deans[b])
        params.append(L.make_params(wl.taus[b], G, False, wl.seeds[b], wl.noise_amp, True))
    ctx = L.LBContext(spec_of(ch), batch=wl.batch, precision=precision)
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, BENCH_THREADS)
    ctx.lb_init(params)
    ctx.lb_step(200)                        # leave the initial transient
    f0 = ctx.lb_get_populations()
    rho0, u0 = ctx.lb_macros()
    ctx.lb_step(1)
    f1 = ctx.lb_get_populations()
    ctx.close()
    return wl, ch, params, f0, f1, rho0, u0


@pytest.fixture(scope="module")
def run():
    return _sweep_run("fp32")


def test_sampled_nodes_match_oracle(run):
    wl, ch, params, f0, f1, _, _ = run
    geo, smap = channel_geometry(ch), StreamMap(ch)
    for b in (0, 13, wl.batch - 1):
        _check_step(ch, wl.taus[b], params[b].force_G, f0[b], f1[b], TOL["fp32"], geo, smap)


@pytest.mark.parametrize("precision", ["fp16_shifted", "bf16_shifted"])
def test_sampled_nodes_match_oracle_two_byte_storage(precision):
    """The 2-byte deviation storage on the same sweep: the oracle's step from
    the decoded pre-step state against the decoded post-step state, which
    carries the rounding of one encode."""
    wl, ch, params, f0, f1, _, _ = _sweep_run(precision)
    geo, smap = channel_geometry(ch), StreamMap(ch)
    for b in (0, 11, 17, wl.batch - 1):
        _check_step(ch, wl.taus[b], params[b].force_G, f0[b], f1[b], TOL[precision], geo, smap)
    assert np.isfinite(f1).all()


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


@pytest.mark.parametrize("precision", ["fp32", "fp16_shifted"])
def test_ellipsoid_four_walls_sampled_nodes_match_oracle(precision):
    """bench.py --workload ellipsoid: 24 instances of the 64 x 4 x 256
    double-curved channel with walls on r and phi, De 20..150 through the
    force of the cylinder of the same streamwise radius, tau 0.55, from rest
    plus noise; the tiled step (interior and wall-node tiles)."""
    L = lib()
    wl = ellipsoid_cross_section(1.0, precision=precision)
    ch = Channel(**wl.geometry_kwargs())
    ref = L.make_desc(1.0, 1.0 + (wl.r_outer - wl.r_inner), wl.nr, wl.ntheta, wl.n3)
    deans = np.linspace(20, 150, 24)
    Gs = [L.lb_force_for_dean("cylindrical", ref, 0.55, float(de)) for de in deans]
    params = [L.make_params(0.55, G, False, wl.seeds[0] + b, 1e-4, False) for b, G in enumerate(Gs)]
    ctx = L.LBContext(spec_of(ch), batch=24, precision=precision)
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, BENCH_THREADS)
    ctx.lb_init(params)
    ctx.lb_step(1000)
    f0 = ctx.lb_get_populations()
    ctx.lb_step(1)
    f1 = ctx.lb_get_populations()
    ctx.close()
    assert np.isfinite(f1).all()
    geo, smap = channel_geometry(ch), StreamMap(ch)
    # the flow starts from rest: instances of De >= 85 reach u_max ~ 1e-2 by
    # now, where 1e-5 u_max lies above the FP32 resolution of populations
    # ~0.3 (the low-De instances' u_max ~ 1e-3 does not)
    for b in (12, 18, 23):
        _check_step(ch, 0.55, Gs[b], f0[b], f1[b], TOL_REST[precision], geo, smap)


@pytest.mark.parametrize("precision", ["fp32", "bf16_shifted"])
def test_mixed_batch_members_match_oracle(precision):
    """bench.py --workload mixed: the 128-channel batch after its autotuner,
    graph replay; members of both metric kinds and every N_r checked."""
    import torch
    from paper_1411_3133_gb300.sweep import mixed_contexts
    L = lib()
    insts = mixed_batch()
    ctxs, batch = mixed_contexts(insts, precision)
    batch.lb_batch_set_option(L.LB_OPT_USE_GRAPH, 1)
    batch.lb_batch_autotune(20)
    batch.lb_batch_step(1500)
    # per metric kind and N_r the member of the largest Dean number: the flow
    # starts from rest, and these reach u_max >~ 1e-2 by now, where 1e-5 u_max
    # lies above the FP32 resolution of populations ~0.3
    picks = []
    for metric in ("cylindrical", "ellipsoidal"):
        for nr in (32, 48, 64):
            group = [i for i, x in enumerate(insts) if x.metric == metric and x.nr == nr]
            picks.append(max(group, key=lambda i: insts[i].dean))
    f0 = [ctxs[i].lb_get_populations()[0] for i in picks]
    batch.lb_batch_step(1)
    f1 = [ctxs[i].lb_get_populations()[0] for i in picks]
    torch.cuda.synchronize()
    batch.close()
    for c in ctxs:
        c.close()
    for k, i in enumerate(picks):
        inst = insts[i]
        ch = Channel(**inst.geometry_kwargs())
        r = force_reference_cylinder(inst)
        G = L.lb_force_for_dean("cylindrical", L.make_desc(r["r_inner"], r["r_outer"], r["nr"], r["ntheta"],
                                                         r["n3"]), inst.tau, inst.dean)
        assert np.isfinite(f1[k]).all()
        _check_step(ch, inst.tau, G, f0[k], f1[k], TOL_REST[precision])


def test_fp32_laminar_2000_steps():
    """FP32 storage and arithmetic over 2000 steps of the laminar curved
    channel (16 x 1 x 32, eta = 0.975, tau = 0.8, u_max ~ 0.05 from the
    laminar profile plus noise), bench's block size and graph replay,
    against the FP64 oracle.

    After 100 steps u lies within 1e-5 of u_max. Later the FP32 rounding of
    the stored populations -- nearly equal at neighbouring nodes, so rounded
    alike -- accumulates coherently. A bound from the arithmetic: each step
    moves u by at most 2^-24 sum_l |c_l| f_l / rho' ~ 1.5 x 2^-24 (each
    stored population off by half an ulp, all with one sign), and the mean
    flow forgets a disturbance on the viscous time N_r^2 / (pi^2 nu) ~ 240
    steps, so the steady error stays below 240 x 1.5 x 2^-24 ~ 2e-5
    absolute, 4e-4 of u_max. Mass has no such decay: rho' may drift by n
    eps_32 after n steps."""
    from analytic import curved_poiseuille
    L = lib()
    ch = Channel("cylindrical", 1.0, 1 / 0.975, 16, 1, 32)
    G = 1.745e-4
    tw = Twin(ch, [dict(tau=0.8, G=G, seed=21, amp=1e-4, base=True)], "fp32")
    tw.ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    tw.ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, BENCH_THREADS)
    tw.ctx.lb_init(tw.lparams)
    _, _, uth = curved_poiseuille(ch.r_inner, ch.r_outer, ch.nr, G, 0.8)
    u = noise_field(21, tw.N, 1e-4)
    u[:, 1] += np.repeat(uth, ch.ntheta * ch.n3)
    tw.sims[0].init_rest(u)
    nu = (0.8 - 0.5) * (1 - np.sqrt(0.4))
    t_visc = ch.nr ** 2 / (np.pi ** 2 * nu)
    done = 0
    for n in (100, 500, 1000, 2000):
        tw.step(n - done)
        done = n
        rl, ul = tw.lib_macros()
        ro, uo = tw.oracle_macros()
        er, eu = max_rel(rl, ro, np.abs(ro).max()), max_rel(ul, uo, np.abs(uo).max())
        print("step %d: rho' rel err %.2e, u err / u_max %.2e" % (n, er, eu))
        if n == 100:
            assert eu <= 1e-5
        assert eu * np.abs(uo).max() <= t_visc * 1.5 * 2.0 ** -24
        assert er <= n * 2.0 ** -24
    tw.close()
