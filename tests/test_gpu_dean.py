"""Physics gate on the GPU: the critical Dean number of a narrow curved
channel (eta = r_i/r_o = 0.975, 64 x 4 x 256, L_z = 4 d) from the saturated
Dean-vortex amplitude (A^2 ~ De - De_c), against Dean's narrow-gap value ~36
printed in the paper's introduction (+-10%: the finite gap raises it, the
periodic box quantises the vortex wavelength, and the lattice has a finite
Mach number). The two relaxation times describe the same physics and must
agree to 5%."""
import numpy as np
import pytest

from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def test_critical_dean_narrow_gap():
    lib()
    from paper_1411_3133_gb300 import lbgm as L
    from paper_1411_3133_gb300.sweep import run_sweep, summarize
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / 0.975, 64, 4, 256)
    deans = list(np.linspace(25.0, 60.0, 12))
    taus = [0.55] * 12 + [0.6] * 12
    res = run_sweep(spec, taus, deans + deans, steps=300_000, sample_every=2000)
    summ = summarize(res)
    dec = {tau: summ[tau]["De_c"] for tau in summ}
    print("De_c", dec, "growth-rate De_c", {t: summ[t]["De_c_growth"] for t in summ},
          "seconds", res.seconds)
    assert 36 * 0.9 <= dec[0.55] <= 36 * 1.1, dec
    assert 36 * 0.9 <= dec[0.6] <= 36 * 1.1, dec
    assert abs(dec[0.55] / dec[0.6] - 1) < 0.05, dec


def test_continuation_sweep_starts_every_instance_from_the_donor():
    """Mechanics of the continuation: every instance starts from the donor's
    populations (same state, so the same vortex amplitude at the first
    sample up to one sample interval of evolution), each keeps its own force
    (the measured Dean number follows the target), and the estimators return
    numbers or NaN, never raise."""
    lib()
    from paper_1411_3133_gb300 import lbgm as L
    from paper_1411_3133_gb300.sweep import continuation_sweep
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / 0.9, 17, 1, 32, wall="equilibrium")
    deans = [2.0, 4.0, 6.0]                 # laminar mean speed <= 0.13 at this size
    r = continuation_sweep(spec, 0.8, deans, donor_dean=8.0, donor_steps=3000, steps=2000,
                           sample_every=500, noise_amp=1e-3)
    assert r["donor_amp"] > 0
    assert len(r["dean"]) == 3 and all(np.isfinite(r["dean"]))
    assert r["dean"][0] < r["dean"][1] < r["dean"][2]
    for k in ("De_c_saturation", "De_c_decay"):
        assert isinstance(r[k], float)


def test_double_curved_study_runs_both_curvature_families():
    lib()
    from paper_1411_3133_gb300.sweep import double_curved_study
    cases = [("b=0.9", 1.0, 0.9), ("r_i=1.2", 1.2, 1.0 / np.sqrt(1.2))]
    # 17 radial nodes: De <= 12 keeps the laminar mean speed below 0.4
    r = double_curved_study(cases, deans=[2.0, 4.0, 6.0, 8.0, 10.0], steps=2000, sample_every=500,
                            nr=17, ntheta=4, n3=32)
    assert r["steps"] == 2000 and len(r["cases"]) == 2
    for c in r["cases"]:
        assert len(c["dean"]) == len(c["vorticity"]) == len(c["dean_target"]) == 5
        assert np.all(np.isfinite(c["vorticity"]))
        assert np.all(np.diff(c["dean"]) > 0)           # measured De follows the force
        assert isinstance(c["De_c"], float)
    assert r["cases"][1]["R_theta"] == pytest.approx(1.0)


def test_developed_vortex_has_two_dean_cells():
    """A supercritical narrow channel with the paper's cross-section shape
    (L_z = 2 L_r, Sec. III: "perfectly adapted to the 2-cell vortex
    solution") develops one pair of counter-rotating cells: u^r at mid-gap
    changes sign twice along the periodic z (sweep.vortex_cells)."""
    lib()
    from paper_1411_3133_gb300 import lbgm as L
    from paper_1411_3133_gb300.sweep import vortex_cells
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / 0.975, 32, 1, 64)
    G = L.lb_force_for_dean("cylindrical", spec.desc(), 0.6, 44.0)
    ctx = L.LBContext(spec, batch=1, precision="fp32")
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    ctx.lb_init([L.make_params(0.6, G, False, 20241111, 1e-3, True)])
    ctx.lb_step(400_000)
    d = ctx.lb_diagnostics()[0]
    _, u = ctx.lb_macros()
    ctx.close()
    assert d["vortex_amp_x3"] > 1e-3 * d["max_speed"], d       # developed, not noise
    assert vortex_cells(u[0, 0], 32, 1, 64, periodic=True) == 2
