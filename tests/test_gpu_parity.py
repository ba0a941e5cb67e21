"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances (stated by the target, applied relative to the field's scale):
FP64 1e-12 (rho' against max rho', u against max |u|), FP32 1e-5 of u_max.
Sizes span several thread blocks, ragged tails (n3 not a multiple of 32),
walls on one and on two axes, theta extents 1, 2 and 4, all three metrics.
"""
import math

import numpy as np
import pytest

from analytic import curved_poiseuille
from gpu_helpers import Twin, lib, max_rel, spec_of
from oracle.diagnostics import diagnostics
from oracle.geometry import Channel
from paper_1411_3133_gb300.workloads import noise_field

pytestmark = pytest.mark.gpu

ETA = 0.975
CYL1 = Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 32)          # 16 x 4 x 32 cylinder
G_LAMINAR = 1.745e-4                                            # De ~ 0.8 at tau = 0.8


def _rest_fields(tw, amps_seeds):
    rho = np.stack([1.0 / s.sqrtg for s in tw.sims])
    u = np.stack([noise_field(seed, tw.N, amp) for amp, seed in amps_seeds])
    return rho, u


def _compare_macros(tw, tol_rho, tol_u):
    rl, ul = tw.lib_macros()
    ro, uo = tw.oracle_macros()
    er = max_rel(rl, ro, np.abs(ro).max())
    eu = max_rel(ul, uo, np.abs(uo).max())
    assert er <= tol_rho and eu <= tol_u, (er, eu)
    return er, eu


def test_seeded_init_matches_oracle():
    params = [dict(tau=0.8, seed=20241111, amp=1e-3), dict(tau=0.7, seed=7, amp=2e-2)]
    tw = Twin(CYL1, params)
    tw.ctx.lb_init(tw.lparams)
    for b, s in enumerate(tw.sims):
        s.init_rest(noise_field(params[b]["seed"], tw.N, params[b]["amp"]))
    fl = tw.lib_f()
    fo = np.stack([s.f for s in tw.sims])
    assert max_rel(fl, fo, np.abs(fo).max()) <= 1e-14
    tw.close()


def test_base_flow_init_matches_closed_form():
    params = [dict(tau=0.8, G=G_LAMINAR, seed=3, amp=1e-4, base=True)]
    tw = Twin(CYL1, params)
    tw.ctx.lb_init(tw.lparams)
    _, _, uth = curved_poiseuille(CYL1.r_inner, CYL1.r_outer, CYL1.nr, G_LAMINAR, 0.8)
    u = noise_field(3, tw.N, 1e-4)
    u[:, 1] += np.repeat(uth, CYL1.ntheta * CYL1.n3)
    tw.sims[0].init_rest(u)
    fo = tw.sims[0].f
    assert max_rel(tw.lib_f()[0], fo, np.abs(fo).max()) <= 1e-14
    tw.close()


CASES = {
    "cyl16x4x32": (CYL1, [dict(tau=0.8, G=G_LAMINAR, seed=11, amp=1e-3, base=True)]),
    "cyl_ragged9x3x13": (Channel("cylindrical", 1.0, 1 / 0.9, 9, 3, 13),
                         [dict(tau=0.65, G=2e-4, seed=5, amp=5e-3)]),
    "cyl_ntheta1": (Channel("cylindrical", 1.0, 1 / ETA, 12, 1, 40),
                    [dict(tau=0.9, G=1e-4, seed=6, amp=1e-3)]),
    "cyl_old_forcing": (Channel("cylindrical", 1.0, 1 / 0.8, 10, 2, 20),
                        [dict(tau=0.75, G=3e-4, seed=8, amp=1e-2, old=True)]),
    "flat_walls4": (Channel("flat", 0.0, 1.0, 8, 2, 9, periodic3=False),
                    [dict(tau=0.6, G=1e-3, seed=9, amp=1e-2)]),
    "ell_4walls": (Channel("ellipsoidal", 1.0, 1.1, 10, 4, 14, b=0.9, periodic3=False),
                   [dict(tau=0.7, G=3e-4, seed=10, amp=1e-2)]),
    "ell_rescaled": (Channel("ellipsoidal", 0.5, 0.525, 12, 2, 40, b=2 ** 0.5, periodic3=False,
                             dtheta_scale=1.0, d3_scale=2.0),
                     [dict(tau=0.55, G=5e-4, seed=12, amp=1e-2)]),
    "ell_periodic_phi": (Channel("ellipsoidal", 1.0, 1.1, 8, 3, 35, b=1.2),
                         [dict(tau=0.8, G=2e-4, seed=13, amp=1e-2)]),
    "cyl_eqwall": (Channel("cylindrical", 1.0, 1 / ETA, 17, 4, 32, wall="equilibrium"),
                   [dict(tau=0.8, G=2e-4, seed=21, amp=1e-2)]),
    "flat_eqwall_4": (Channel("flat", 0.0, 1.0, 9, 2, 9, periodic3=False, wall="equilibrium"),
                      [dict(tau=0.6, G=1e-3, seed=22, amp=1e-2)]),
    "ell_eqwall_4": (Channel("ellipsoidal", 1.0, 1.1, 10, 4, 14, b=0.9, periodic3=False,
                             wall="equilibrium"), [dict(tau=0.7, G=3e-4, seed=23, amp=1e-2)]),
    "ell_eqwall_periodic": (Channel("ellipsoidal", 1.0, 1.1, 8, 3, 35, b=1.2, wall="equilibrium"),
                            [dict(tau=0.8, G=2e-4, seed=24, amp=1e-2)]),
    "cyl_eqwall_nr3": (Channel("cylindrical", 1.0, 1.02, 3, 2, 8, wall="equilibrium"),
                       [dict(tau=0.9, G=1e-4, seed=25, amp=1e-2)]),
    # the half-force velocity variant (old_forcing 2), alone and mixed with the literal step
    "cyl_shift": (Channel("cylindrical", 1.0, 1 / 0.8, 10, 2, 20),
                  [dict(tau=0.75, G=3e-4, seed=8, amp=1e-2, shift=True)]),
    "ell_shift_mixed": (Channel("ellipsoidal", 1.0, 1.1, 10, 4, 14, b=0.9, periodic3=False),
                        [dict(tau=0.7, G=3e-4, seed=10, amp=1e-2, shift=True),
                         dict(tau=0.9, G=2e-4, seed=14, amp=1e-2)]),
    "cyl_eqwall_shift": (Channel("cylindrical", 1.0, 1 / ETA, 17, 4, 32, wall="equilibrium"),
                         [dict(tau=0.8, G=2e-4, seed=21, amp=1e-2, shift=True)]),
    "flat_shift": (Channel("flat", 0.0, 1.0, 8, 2, 9, periodic3=False),
                   [dict(tau=0.6, G=1e-3, seed=9, amp=1e-2, shift=True)]),
    # theta-resolved double-curved channel: the metric of each theta node (full Delta, body force
    # with r and phi components), walls on r and phi / equilibrium walls with a periodic phi
    "ellT_4wall": (Channel("ellipsoidal", 1.0, 1.1, 10, 8, 14, b=0.6, periodic3=False,
                           dtheta_scale=1 / 0.6, theta_resolved=True),
                   [dict(tau=0.7, G=3e-4, seed=31, amp=1e-2)]),
    "ellT_eqwall_periodic": (Channel("ellipsoidal", 1.0, 1.1, 9, 8, 16, b=1.5, dtheta_scale=1 / 1.5,
                                     wall="equilibrium", theta_resolved=True),
                             [dict(tau=0.8, G=2e-4, seed=32, amp=1e-2),
                              dict(tau=0.65, G=1e-4, seed=33, amp=1e-2, old=True)]),
    "batch3": (Channel("cylindrical", 1.0, 1 / ETA, 8, 4, 33),
               [dict(tau=0.8, G=1e-4, seed=1, amp=1e-3), dict(tau=0.6, G=3e-4, seed=2, amp=2e-3),
                dict(tau=1.1, G=0.0, seed=3, amp=5e-3, old=True)]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_step_parity(case):
    ch, params = CASES[case]
    tw = Twin(ch, params, "fp64")
    tw.ctx.lb_init(tw.lparams)
    for b, s in enumerate(tw.sims):
        p = params[b]
        u = noise_field(p["seed"], tw.N, p["amp"])
        if p.get("base"):
            _, _, uth = curved_poiseuille(ch.r_inner, ch.r_outer, ch.nr, p["G"], p["tau"])
            u[:, 1] += np.repeat(uth, ch.ntheta * ch.n3)
        s.init_rest(u)
    done = 0
    for n in (1, 10, 100):
        tw.step(n - done)
        done = n
        _compare_macros(tw, 1e-12, 1e-12)
    fl, fo = tw.lib_f(), np.stack([s.f for s in tw.sims])
    assert max_rel(fl, fo, np.abs(fo).max()) <= 1e-12
    tw.close()


def test_fp64_laminar_5000_steps():
    ch = Channel("cylindrical", 1.0, 1 / ETA, 16, 1, 32)
    params = [dict(tau=0.8, G=G_LAMINAR, seed=21, amp=1e-4, base=True)]
    tw = Twin(ch, params, "fp64")
    tw.ctx.lb_init(tw.lparams)
    _, _, uth = curved_poiseuille(ch.r_inner, ch.r_outer, ch.nr, G_LAMINAR, 0.8)
    u = noise_field(21, tw.N, 1e-4)
    u[:, 1] += np.repeat(uth, ch.ntheta * ch.n3)
    tw.sims[0].init_rest(u)
    tw.step(5000)
    _compare_macros(tw, 1e-12, 1e-12)
    tw.close()


def _smooth_flow(ch, amp=0.05):
    """Streamwise flow vanishing on the walls of r (and x3 when walled): half
    a node outside the end nodes for bounce-back walls, on the end nodes for
    equilibrium walls (whose end nodes lie on the walls)."""
    ir, it, i3 = np.meshgrid(np.arange(ch.nr), np.arange(ch.ntheta), np.arange(ch.n3), indexing="ij")
    if ch.wall == "equilibrium":
        prof = np.sin(np.pi * ir / (ch.nr - 1))
        if not ch.periodic3:
            prof = prof * np.sin(np.pi * i3 / (ch.n3 - 1))
    else:
        prof = np.sin(np.pi * (ir + 0.5) / ch.nr)
        if not ch.periodic3:
            prof = prof * np.sin(np.pi * (i3 + 0.5) / ch.n3)
    u = np.zeros(ch.shape + (3,))
    u[..., 1] = amp * prof
    return u.reshape(-1, 3)


@pytest.mark.parametrize("ch", [CYL1, Channel("ellipsoidal", 1.0, 1.1, 10, 4, 40, b=0.9,
                                              periodic3=False),
                                Channel("ellipsoidal", 1.0, 1.1, 10, 4, 40, b=0.9, periodic3=False,
                                        wall="equilibrium"),
                                Channel("ellipsoidal", 1.0, 1.1, 10, 8, 40, b=0.6, periodic3=False,
                                        dtheta_scale=1 / 0.6, theta_resolved=True)],
                         ids=["cyl", "ell", "ell_eqwall", "ell_theta"])
def test_fp32_step_parity(ch):
    """FP32 against the FP64 oracle, 1e-5 of u_max for a flow of realistic
    magnitude (u_max ~ 0.05), after 1, 10 and 100 steps."""
    params = [dict(tau=0.8, G=G_LAMINAR)]
    tw = Twin(ch, params, "fp32")
    rho = np.stack([1.0 / tw.sims[0].sqrtg])
    u = (_smooth_flow(ch) + noise_field(31, tw.N, 1e-3))[None]
    tw.init_fields(rho, u)
    done = 0
    for n in (1, 10, 100):
        tw.step(n - done)
        done = n
        _compare_macros(tw, 1e-5, 1e-5)
    tw.close()


@pytest.mark.parametrize("ch", [CYL1, Channel("ellipsoidal", 1.0, 1.1, 10, 4, 40, b=0.9,
                                              periodic3=False, wall="equilibrium")],
                         ids=["cyl", "ell_eqwall"])
def test_fp32_half_force_variant_parity(ch):
    """The half-force velocity variant in FP32 against the FP64 oracle's
    variant, 1e-5 of u_max."""
    params = [dict(tau=0.8, G=G_LAMINAR, shift=True)]
    tw = Twin(ch, params, "fp32")
    rho = np.stack([1.0 / tw.sims[0].sqrtg])
    u = (_smooth_flow(ch) + noise_field(32, tw.N, 1e-3))[None]
    tw.init_fields(rho, u)
    done = 0
    for n in (1, 10, 100):
        tw.step(n - done)
        done = n
        _compare_macros(tw, 1e-5, 1e-5)
    tw.close()


def test_half_force_variant_rules():
    """2-byte storage rejects the variant; a batch refuses a member using it;
    the autotuner keeps to the plain kernel."""
    L = lib()
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / ETA, 8, 4, 32)
    p2 = [L.make_params(0.8, 1e-4, 2, 1, 1e-3, False)]
    with L.LBContext(spec, 1, "fp16_shifted") as c:
        with pytest.raises(L.LBError) as e:
            c.lb_init(p2)
        assert "half-force" in str(e.value)
    with L.LBContext(spec, 1, "fp32") as c:
        with pytest.raises(L.LBError) as e:
            c.lb_init([L.make_params(0.8, 1e-4, 3, 1, 1e-3, False)])
        assert "0, 1 or 2" in str(e.value)
    with L.LBContext(spec, 1, "fp32") as c, L.LBContext(spec, 1, "fp32", stream=c.stream) as d:
        c.lb_init(p2)
        d.lb_init([L.make_params(0.8, 1e-4, 0, 1, 1e-3, False)])
        best, trials = c.lb_autotune(2)
        assert {t["schedule"] for t in trials} == {1}
        b = L.LBBatch([c, d])
        with pytest.raises(L.LBError) as e:
            b.lb_batch_step(1)
        assert "half-force" in str(e.value)
        b.close()


def test_init_fields_matches_oracle():
    ch = Channel("ellipsoidal", 1.0, 1.1, 9, 2, 16, b=0.8, periodic3=False)
    params = [dict(tau=0.7, G=1e-4), dict(tau=0.9, G=0.0)]
    tw = Twin(ch, params, "fp64")
    rng = np.random.default_rng(0)
    rho = 1.0 + 0.01 * rng.random((2, tw.N))
    u = 0.02 * rng.standard_normal((2, tw.N, 3))
    tw.init_fields(rho, u)
    fo = np.stack([s.f for s in tw.sims])
    assert max_rel(tw.lib_f(), fo, np.abs(fo).max()) <= 1e-14
    tw.step(7)
    _compare_macros(tw, 1e-12, 1e-12)
    tw.close()


@pytest.mark.parametrize("wall", ["bounceback", "equilibrium"])
def test_diagnostics_match_oracle(wall):
    ch = Channel("ellipsoidal", 1.0, 1.1, 10, 3, 16, b=0.9, periodic3=False, wall=wall)
    params = [dict(tau=0.7, G=3e-4, seed=4, amp=1e-2), dict(tau=0.6, G=1e-4, seed=5, amp=1e-2)]
    tw = Twin(ch, params, "fp64")
    tw.ctx.lb_init(tw.lparams)
    for b, s in enumerate(tw.sims):
        s.init_rest(noise_field(params[b]["seed"], tw.N, params[b]["amp"]))
    tw.step(20)
    dl = tw.ctx.lb_diagnostics()
    for b, s in enumerate(tw.sims):
        rho, u = s.macros()
        do = diagnostics(ch, tw.geo, params[b]["tau"], rho, u)
        for k in ("mass_rho_prime", "mass_physical", "mean_v_theta", "dean", "mean_vorticity",
                  "vortex_amp", "vortex_amp_x3", "max_speed"):
            assert dl[b][k] == pytest.approx(do[k], rel=1e-11, abs=1e-18), k
        assert dl[b]["nonfinite"] == 0 and dl[b]["step"] == 20
    tw.close()


@pytest.mark.parametrize("wall", ["bounceback", "equilibrium"])
def test_diagnostics_match_oracle_theta_resolved(wall):
    """Observables of the theta-resolved channel: per-node weights (sqrt g,
    sqrt g_thth, the area element of the (r, phi) block) from each node's own
    metric."""
    ch = Channel("ellipsoidal", 1.0, 1.1, 10, 6, 16, b=0.6, periodic3=False, dtheta_scale=1 / 0.6,
                 wall=wall, theta_resolved=True)
    params = [dict(tau=0.7, G=3e-4, seed=4, amp=1e-2)]
    tw = Twin(ch, params, "fp64")
    tw.ctx.lb_init(tw.lparams)
    tw.sims[0].init_rest(noise_field(4, tw.N, 1e-2))
    tw.step(20)
    dl = tw.ctx.lb_diagnostics()
    rho, u = tw.sims[0].macros()
    do = diagnostics(ch, tw.geo, 0.7, rho, u)
    for k in ("mass_rho_prime", "mass_physical", "mean_v_theta", "dean", "mean_vorticity",
              "vortex_amp", "vortex_amp_x3", "max_speed"):
        assert dl[0][k] == pytest.approx(do[k], rel=1e-11, abs=1e-18), k
    tw.close()


def test_theta_resolved_restrictions():
    """The theta-resolved ellipsoid runs FP64 / FP32 storage in the plain
    step kernel: 2-byte storage, the other step kernels, batches, the
    half-force variant and the no-alloc observables are refused."""
    L = lib()
    ch = Channel("ellipsoidal", 1.0, 1.1, 8, 4, 12, b=0.8, periodic3=False, theta_resolved=True)
    for prec in ("fp16_shifted", "bf16_shifted"):
        with pytest.raises(L.LBError) as e:
            L.LBContext(spec_of(ch), batch=1, precision=prec)
        assert e.value.status == L.LB_ERR_ARG
    tw = Twin(ch, [dict(tau=0.8)], "fp32")
    tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, 1)
    for bad in (2, 4, 5):
        with pytest.raises(L.LBError) as e:
            tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, bad)
        assert e.value.status == L.LB_ERR_ARG
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_init([L.make_params(0.8, 1e-5, 2, 1, 0.0, False)])
    assert e.value.status == L.LB_ERR_ARG
    tw.close()


def test_equilibrium_wall_base_flow_vanishes_on_wall_nodes():
    """lb_init's laminar profile with wall nodes: zero velocity on the end
    nodes, the closed form in between, and it stays near it (first-order
    wall condition) over 200 steps."""
    from analytic import curved_poiseuille_coeffs
    ch = Channel("cylindrical", 1.0, 1 / ETA, 17, 2, 8, wall="equilibrium")
    tau, G = 0.8, 2e-4
    tw = Twin(ch, [dict(tau=tau, G=G, base=True)], "fp64")
    tw.ctx.lb_init(tw.lparams)
    r = 1.0 + np.arange(ch.nr) * ch.h
    A, B, C = curved_poiseuille_coeffs(1.0, 1 / ETA, ch.h, G, tau)
    uth = (A * r * np.log(r) + B * r + C / r) / r
    rho, u = tw.lib_macros()
    ut = u[0, :, 1].reshape(ch.nr, -1)
    assert abs(uth[0]) < 1e-12 * abs(uth).max() and abs(uth[-1]) < 1e-12 * abs(uth).max()
    tw.ctx.lb_step(200)
    rho, u = tw.lib_macros()
    ut = u[0, :, 1].reshape(ch.nr, -1).mean(axis=1)
    assert np.abs(ut[1:-1] - uth[1:-1]).max() < 0.15 * np.abs(uth).max()
    tw.close()


def test_mass_budget_on_gpu():
    """sum f(t+1) - sum f(t) = sum_x -2 rho' u^r Gamma^theta_{r theta} (cylinder)."""
    L = lib()
    ch = Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 64)
    tw = Twin(ch, [dict(tau=0.7, G=2e-4, seed=1, amp=1e-2)], "fp64")
    tw.ctx.lb_init(tw.lparams)
    g = tw.geo["Gamma_hat"][:, 0, 1, 0, 1]             # h / r per i_r
    for _ in range(3):
        f0 = tw.ctx.lb_get_populations().sum()
        rho, u = tw.lib_macros()
        src = (-2.0 * rho[0] * u[0, :, 0] * np.repeat(g, ch.ntheta * ch.n3)).sum()
        tw.ctx.lb_step(1)
        f1 = tw.ctx.lb_get_populations().sum()
        assert abs(f1 - f0 - src) <= 1e-13 * f0
    tw.close()


def test_checkpoint_resume_bitwise():
    L = lib()
    for prec in ("fp64", "fp32"):
        tw = Twin(CYL1, [dict(tau=0.8, G=1e-4, seed=2, amp=1e-3)], prec)
        tw.ctx.lb_init(tw.lparams)
        tw.ctx.lb_step(5)
        buf = np.zeros(tw.ctx.lb_state_bytes(), dtype=np.uint8)
        tw.ctx.lb_get_state(buf)
        tw.ctx.lb_step(10)
        a = tw.ctx.lb_get_populations()
        tw.ctx.lb_set_state(buf)
        assert tw.ctx.lb_step_count() == 15        # the counter is not part of the raw state
        tw.ctx.lb_step(10)
        b = tw.ctx.lb_get_populations()
        assert np.array_equal(a, b)
        # populations round trip exactly
        tw.ctx.lb_set_populations(a)
        assert np.array_equal(tw.ctx.lb_get_populations(), a)
        tw.close()


def test_graph_replay_matches_plain_launches():
    L = lib()
    outs = []
    for graph in (0, 1):
        tw = Twin(CYL1, [dict(tau=0.8, G=1e-4, seed=2, amp=1e-3)], "fp32")
        tw.ctx.lb_set_option(L.LB_OPT_USE_GRAPH, graph)
        tw.ctx.lb_init(tw.lparams)
        tw.ctx.lb_step(1)
        tw.ctx.lb_step(37)
        outs.append(tw.ctx.lb_get_populations())
        assert tw.ctx.lb_step_count() == 38
        tw.close()
    assert np.array_equal(outs[0], outs[1])


def test_block_size_option_is_bitwise_neutral():
    L = lib()
    outs = []
    for threads in (64, 128, 256):
        tw = Twin(CYL1, [dict(tau=0.8, G=1e-4, seed=2, amp=1e-3)], "fp32")
        tw.ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, threads)
        tw.ctx.lb_init(tw.lparams)
        tw.ctx.lb_step(12)
        outs.append(tw.ctx.lb_get_populations())
        tw.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_nan_injection_is_detected_and_poisons():
    L = lib()
    tw = Twin(CYL1, [dict(tau=0.8, G=1e-4, seed=2, amp=1e-3)], "fp64")
    tw.ctx.lb_init(tw.lparams)
    f = tw.ctx.lb_get_populations()
    f[0, 5, 100] = np.nan
    tw.ctx.lb_set_populations(f)
    tw.ctx.lb_set_option(L.LB_OPT_CHECK_EVERY, 1)
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_step(3)
    assert e.value.status == L.LB_ERR_NONFINITE
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_step(1)
    assert e.value.status == L.LB_ERR_STATE
    tw.ctx.lb_init(tw.lparams)                      # a fresh start clears the poison
    tw.ctx.lb_step(2)
    assert tw.ctx.lb_diagnostics()[0]["nonfinite"] == 0
    tw.close()


def test_literal_dean30_on_16_nodes_is_reported():
    """De = 30 at N_r = 16, tau = 0.8 needs <v> ~ 1.3 (Mach > 2): the run
    either diverges, which lb_step must report as LB_ERR_NONFINITE, or stays
    finite; it must not hang or crash."""
    L = lib()
    desc = L.make_desc(1.0, 1 / ETA, 16, 4, 32)
    G = L.lb_force_for_dean("cylindrical", desc, 0.8, 30.0)
    tw = Twin(CYL1, [dict(tau=0.8, G=G, seed=20241111, amp=1e-4)], "fp64")
    tw.ctx.lb_set_option(L.LB_OPT_CHECK_EVERY, 100)
    tw.ctx.lb_init(tw.lparams)
    try:
        tw.ctx.lb_step(5000)
        d = tw.ctx.lb_diagnostics()[0]
        assert d["nonfinite"] == 0
    except L.LBError as e:
        assert e.status == L.LB_ERR_NONFINITE
    tw.close()


def test_state_and_argument_errors():
    L = lib()
    tw = Twin(CYL1, [dict(tau=0.8)], "fp32")
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_step(1)
    assert e.value.status == L.LB_ERR_STATE
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_init([L.make_params(0.5)])
    assert e.value.status == L.LB_ERR_ARG
    tw.ctx.lb_init(tw.lparams)
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_step(-1)
    assert e.value.status == L.LB_ERR_ARG
    with pytest.raises(L.LBError):
        tw.ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, 100)
    tw.close()


@pytest.mark.parametrize("ch,batch", [
    (Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 256), 2),
    (Channel("ellipsoidal", 1.0, 1.1, 12, 3, 128, b=0.9, periodic3=False), 1),
    (Channel("ellipsoidal", 1.0, 1.1, 9, 2, 128, b=1.1), 1),
    (Channel("flat", 0.0, 1.0, 10, 1, 256), 3),
], ids=["cyl256", "ell4wall128", "ellper128", "flat256"])
def test_tma_kernel_is_bitwise_equal_to_plain_kernel(ch, batch):
    """The TMA-pipelined FP32 kernel and the plain kernel share the arithmetic;
    they must give identical states."""
    L = lib()
    params = [dict(tau=0.6 + 0.1 * b, G=2e-4, seed=40 + b, amp=1e-2) for b in range(batch)]
    outs = []
    for kern in (1, 2):
        tw = Twin(ch, params, "fp32")
        tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, kern)
        tw.ctx.lb_init(tw.lparams)
        tw.ctx.lb_step(30)
        outs.append(tw.ctx.lb_get_populations())
        tw.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision", ["fp32", "fp64", "bf16_shifted"])
@pytest.mark.parametrize("ch,batch", [
    (Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 256), 2),
    (Channel("cylindrical", 1.0, 1 / 0.9, 9, 3, 13), 3),
    (Channel("cylindrical", 1.0, 1 / ETA, 7, 1, 40), 1),
    (Channel("ellipsoidal", 1.0, 1.1, 8, 3, 35, b=1.2), 1),
], ids=["cyl256", "cyl_ragged", "cyl_nr7", "ell_periodic"])
def test_region_split_kernel_is_bitwise_equal_to_plain_kernel(ch, batch, precision):
    """Wall layers and interior in two kernels give the one-kernel states."""
    L = lib()
    params = [dict(tau=0.6 + 0.1 * b, G=2e-4, seed=60 + b, amp=1e-2) for b in range(batch)]
    outs = []
    for kern, threads in ((1, 128), (4, 128), (4, 64)):
        tw = Twin(ch, params, precision)
        tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, kern)
        tw.ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, threads)
        tw.ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
        tw.ctx.lb_init(tw.lparams)
        tw.ctx.lb_step(17)
        outs.append(tw.ctx.lb_get_populations())
        tw.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)
    tw = Twin(Channel("flat", 0.0, 1.0, 8, 2, 9, periodic3=False), params[:1], precision)
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, 4)        # walls on x3: not supported
    assert e.value.status == L.LB_ERR_ARG
    tw.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16_shifted"])
@pytest.mark.parametrize("ch,batch", [
    (Channel("ellipsoidal", 1.0, 1.1, 12, 3, 40, b=0.9, periodic3=False), 2),
    (Channel("flat", 0.0, 1.0, 8, 2, 9, periodic3=False), 1),
    (Channel("cylindrical", 1.0, 1 / 0.9, 9, 3, 13), 3),
    (Channel("cylindrical", 1.0, 1 / ETA, 9, 2, 16, wall="equilibrium"), 2),
    (Channel("cylindrical", 1.0, 1 / 0.9, 7, 2, 12, periodic3=False), 2),
], ids=["ell4wall", "flat4wall", "cyl_ragged", "cyl_eqwall", "cyl_nr7_walled"])
def test_tiled_step_is_bitwise_equal_to_plain_kernel(ch, batch, precision):
    """Interior runs and the three classes of wall nodes -- r-layer folds,
    x3-layer folds, the general rule (corners, equilibrium walls) -- in the
    work-list kernels (option 5) give the one-kernel states (whose x3-wall
    nodes take the general rule), with graph replay and odd step counts."""
    L = lib()
    params = [dict(tau=0.6 + 0.1 * b, G=2e-4, seed=70 + b, amp=1e-2) for b in range(batch)]
    outs = []
    for kern, threads in ((1, 128), (5, 128), (5, 64)):
        tw = Twin(ch, params, precision)
        tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, kern)
        tw.ctx.lb_set_option(L.LB_OPT_BLOCK_THREADS, threads)
        tw.ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
        tw.ctx.lb_init(tw.lparams)
        tw.ctx.lb_step(3)
        tw.ctx.lb_step(14)
        outs.append(tw.ctx.lb_get_populations())
        tw.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_step_kernel_option_validation():
    L = lib()
    tw = Twin(CYL1, [dict(tau=0.8)], "fp16_shifted")
    for bad in (3, 6, -1):                 # 3: the prefetching kernel, no longer built
        with pytest.raises(L.LBError) as e:
            tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, bad)
        assert e.value.status == L.LB_ERR_ARG
    tw.close()


def test_tma_kernel_option_validation():
    L = lib()
    tw = Twin(CYL1, [dict(tau=0.8)], "fp32")          # n3 = 32: not supported
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, 2)
    assert e.value.status == L.LB_ERR_ARG
    tw.close()
    tw = Twin(Channel("cylindrical", 1.0, 1 / ETA, 8, 2, 256), [dict(tau=0.8)], "fp64")
    with pytest.raises(L.LBError):
        tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, 2)
    tw.close()


@pytest.mark.parametrize("prec,tol", [("fp16_shifted", 1e-3), ("bf16_shifted", 1e-2)])
@pytest.mark.parametrize("ch", [Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 64),
                                Channel("ellipsoidal", 1.0, 1.1, 12, 4, 40, b=0.9, periodic3=False)],
                         ids=["cyl", "ell"])
def test_reduced_precision_storage_against_fp64_oracle(ch, prec, tol):
    """Populations stored as FP16/BF16 deviations (f - w)/w from the rest
    state (reference mode 0), FP32 arithmetic: u within tol * u_max of the
    FP64 oracle after 1, 10 and 100 steps for a flow of realistic magnitude
    (u_max ~ 0.05). FP16 meets the 1e-3 target; BF16's 8-bit mantissa gives
    about 1e-2."""
    L = lib()
    params = [dict(tau=0.8, G=G_LAMINAR)]
    tw = Twin(ch, params, prec)
    tw.ctx.lb_set_option(L.LB_OPT_STORAGE_REFERENCE, 0)
    rho = np.stack([1.0 / tw.sims[0].sqrtg])
    u = (_smooth_flow(ch) + noise_field(31, tw.N, 1e-3))[None]
    tw.init_fields(rho, u)
    done = 0
    for n in (1, 10, 100):
        tw.step(n - done)
        done = n
        _compare_macros(tw, tol, tol)
    tw.close()


@pytest.mark.parametrize("prec,tol", [("fp16_shifted", 1e-4), ("bf16_shifted", 1e-3)])
@pytest.mark.parametrize("ch", [Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 64),
                                Channel("ellipsoidal", 1.0, 1.1, 12, 4, 40, b=0.9, periodic3=False)],
                         ids=["cyl", "ell"])
def test_reduced_precision_with_row_reference(ch, prec, tol):
    """The default reference (mode 1): deviations from the equilibrium of the
    rows' mean initial state. The flow's row profile is then stored exactly
    in FP32 and only the departures from it in 2 bytes: an order of magnitude
    closer to the FP64 oracle than mode 0 for the same flow."""
    params = [dict(tau=0.8, G=G_LAMINAR)]
    tw = Twin(ch, params, prec)
    rho = np.stack([1.0 / tw.sims[0].sqrtg])
    u = (_smooth_flow(ch) + noise_field(31, tw.N, 1e-3))[None]
    tw.init_fields(rho, u)
    done = 0
    for n in (1, 10, 100):
        tw.step(n - done)
        done = n
        er, eu = _compare_macros(tw, tol, tol)
        print(ch.metric, prec, n, er, eu)
    tw.close()


def test_storage_reference_option():
    L = lib()
    tw = Twin(CYL1, [dict(tau=0.8, G=1e-4, seed=2, amp=1e-3)], "fp32")
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_set_option(L.LB_OPT_STORAGE_REFERENCE, 0)    # FP32 has no reference
    assert e.value.status == L.LB_ERR_ARG
    tw.close()
    tw = Twin(CYL1, [dict(tau=0.8, G=1e-4, seed=2, amp=1e-3)], "fp16_shifted")
    tw.ctx.lb_init(tw.lparams)
    tw.ctx.lb_set_option(L.LB_OPT_STORAGE_REFERENCE, 0)        # changes meaning: re-init needed
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_step(1)
    assert e.value.status == L.LB_ERR_STATE
    with pytest.raises(L.LBError) as e:
        tw.ctx.lb_set_option(L.LB_OPT_STORAGE_REFERENCE, 2)
    assert e.value.status == L.LB_ERR_ARG
    tw.ctx.lb_init(tw.lparams)
    tw.ctx.lb_step(2)
    tw.close()


@pytest.mark.parametrize("prec,tol", [("fp16_shifted", 1e-4), ("bf16_shifted", 1e-3)])
def test_capture_reference_keeps_the_state_and_the_parity(prec, tol):
    """lb_capture_reference moves the developed state's row means into the
    reference: the populations change by at most one rounding of the new
    encoding, the stored deviations shrink, and the run stays on the FP64
    oracle."""
    import torch
    L = lib()
    ch = Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 64)
    tw = Twin(ch, [dict(tau=0.8, G=G_LAMINAR)], prec)
    rho = np.stack([1.0 / tw.sims[0].sqrtg])
    u = (_smooth_flow(ch) + noise_field(33, tw.N, 1e-3))[None]
    tw.init_fields(rho, u)
    tw.step(40)
    before = tw.ctx.lb_get_populations()
    raw0 = torch.empty(tw.ctx.lb_state_bytes(), dtype=torch.uint8)
    tw.ctx.lb_get_state(raw0)
    tw.ctx.lb_capture_reference()
    after = tw.ctx.lb_get_populations()
    w = L.lb_velocity_set()[1]
    ulp = 2.0 ** (-11 if prec == "fp16_shifted" else -8)
    # one rounding of the new deviation, whose size is below the old one's
    old_dev = np.abs(before / w[None, :, None] - 1.0).max()
    assert (np.abs(after - before) / w[None, :, None]).max() <= ulp * old_dev
    raw1 = torch.empty_like(raw0)
    tw.ctx.lb_get_state(raw1)
    dt = torch.float16 if prec == "fp16_shifted" else torch.bfloat16
    assert raw1.view(dt).float().abs().max() < 0.5 * raw0.view(dt).float().abs().max()
    f_lib = tw.lib_f()[0]
    for s in tw.sims:
        s.f = f_lib.copy()                      # continue the oracle from the captured state
    tw.step(60)
    _compare_macros(tw, tol, tol)
    tw.close()
    tw2 = Twin(CYL1, [dict(tau=0.8)], "fp32")   # FP32 has no reference
    tw2.ctx.lb_init(tw2.lparams)
    with pytest.raises(L.LBError) as e:
        tw2.ctx.lb_capture_reference()
    assert e.value.status == L.LB_ERR_ARG
    tw2.close()


@pytest.mark.parametrize("prec", ["fp16_shifted", "bf16_shifted"])
def test_reduced_precision_state_round_trips(prec):
    L = lib()
    tw = Twin(CYL1, [dict(tau=0.8, G=1e-4, seed=2, amp=1e-3, base=True)], prec)
    tw.ctx.lb_init(tw.lparams)
    tw.ctx.lb_step(5)
    assert tw.ctx.lb_state_bytes() == 41 * tw.N * 2
    a = tw.ctx.lb_get_populations()
    tw.ctx.lb_set_populations(a)
    assert np.array_equal(tw.ctx.lb_get_populations(), a)
    buf = np.zeros(tw.ctx.lb_state_bytes(), dtype=np.uint8)
    tw.ctx.lb_get_state(buf)
    tw.ctx.lb_step(7)
    b = tw.ctx.lb_get_populations()
    tw.ctx.lb_set_state(buf)
    tw.ctx.lb_step(7)
    assert np.array_equal(tw.ctx.lb_get_populations(), b)
    tw.close()


@pytest.mark.parametrize("prec,tol", [("fp16_shifted", 1e-4), ("bf16_shifted", 1e-3)])
@pytest.mark.parametrize("ch,kern", [
    (Channel("flat", 0.0, 1.0, 8, 2, 9, periodic3=False), 0),                        # walls on x3: 7 row classes
    (Channel("cylindrical", 1.0, 1 / ETA, 9, 3, 13, periodic3=False), 0),
    (Channel("cylindrical", 1.0, 1 / ETA, 16, 2, 16, wall="equilibrium"), 0),        # wall nodes store f^eq
    (Channel("ellipsoidal", 1.0, 1.1, 10, 3, 20, b=0.9, periodic3=False, wall="equilibrium"), 0),
    (Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 64), 4),                            # region split
    (Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 64), 5),                            # tiled
    (Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 64), 1),                            # one kernel
], ids=["flat4wall", "cyl_walled_x3", "cyl_eqwall", "ell_eqwall", "cyl_split", "cyl_tiled", "cyl_plain"])
def test_deviation_collision_every_stream_row_kind(ch, kern, prec, tol):
    """The 2-byte collision runs on the stored deviations through a table per
    stream row (i_r; (i_r, i_3) for the ellipsoid; (i_r, distance class to an
    x3 wall) when x3 has walls), including equilibrium-wall nodes, which store
    f^eq against the reference table: every kind against the FP64 oracle
    after 1, 10 and 60 steps, in each step kernel that runs it. Where x3 has
    walls but the geometry rows (and so the reference) are per i_r only, the
    flow's x3 profile is not in the reference and is stored in 2 bytes: the
    tolerance there is the reduced-precision bound of the target, 1e-3 u_max
    (FP16), and 1e-2 u_max for BF16's 8-bit mantissa (as with the rest-state
    reference). The channels are sized so that the laminar flow of the first
    instance's force is about the initial one: the stored deviations then
    stay small (a flow far from its reference, e.g. a 9-node channel whose
    laminar speed is a quarter of the initial one, stores O(u_max)
    deviations and needs the reference recaptured, lb_capture_reference)."""
    L = lib()
    if not ch.periodic3 and ch.metric != "ellipsoidal" and ch.wall == "bounceback":
        tol *= 10
    tw = Twin(ch, [dict(tau=0.8, G=G_LAMINAR), dict(tau=0.65, G=2 * G_LAMINAR)], prec)
    if kern:
        tw.ctx.lb_set_option(L.LB_OPT_STEP_KERNEL, kern)
    rho = np.stack([1.0 / s.sqrtg for s in tw.sims])
    u = np.stack([_smooth_flow(ch) + noise_field(41 + b, tw.N, 1e-3) for b in range(2)])
    tw.init_fields(rho, u)
    done = 0
    for n in (1, 10, 60):
        tw.step(n - done)
        done = n
        _compare_macros(tw, tol, tol)
    tw.close()
