"""Host logic of the critical-Dean finder (no GPU): growth-rate fit and the
sign-change interpolation on synthetic amplitude series with known answers."""
import numpy as np
import pytest

from paper_1411_3133_gb300.sweep import critical_dean, growth_rate


def test_growth_rate_recovers_exponent_after_transient():
    t = np.arange(0, 200001, 2000, dtype=float)
    for sigma in (-3e-5, -1e-6, 2e-6, 4e-5):
        # a fast-decaying transient on top of the leading mode
        A = 1e-6 * np.exp(sigma * t) + 1e-4 * np.exp(-2e-4 * t)
        assert growth_rate(t, A) == pytest.approx(sigma, rel=0.05, abs=2e-8)


def test_growth_rate_stops_before_saturation():
    t = np.arange(0, 200001, 1000, dtype=float)
    sigma = 1e-4
    A = 1e-7 * np.exp(sigma * t)
    A = A / (1 + A / 1e-2)            # saturates at 1e-2
    assert growth_rate(t, A) == pytest.approx(sigma, rel=0.05)


def test_critical_dean_interpolates_first_sign_change():
    de = [25, 30, 35, 40, 45]
    s = [-3.0, -2.0, -1.0, 1.0, 3.0]
    assert critical_dean(de, s) == pytest.approx(37.5)
    assert np.isnan(critical_dean(de, [-1, -1, -1, -1, -1]))
    # unsorted input
    assert critical_dean(de[::-1], s[::-1]) == pytest.approx(37.5)


def test_critical_dean_from_saturated_amplitude():
    from paper_1411_3133_gb300.sweep import critical_dean_saturation
    de = np.array([30.0, 34.0, 38.0, 42.0, 46.0, 50.0])
    dec = 37.0
    a = np.where(de > dec, np.sqrt(np.clip(2e-7 * (de - dec), 0, None)), 3e-7)
    assert critical_dean_saturation(de, a) == pytest.approx(dec, rel=1e-9)
    assert np.isnan(critical_dean_saturation(de, np.full(6, 3e-7)))


def test_saturation_test_excludes_slowly_growing_instances():
    from paper_1411_3133_gb300.sweep import critical_dean_saturation, is_saturated
    t = np.arange(0, 300001, 2000, dtype=float)
    floor = 1e-8
    de = np.array([30.0, 34.0, 38.0, 39.0, 42.0, 46.0, 50.0, 54.0])
    dec = 37.5
    series = []
    for x in de:
        if x < dec:                                  # decays to the floor
            A = floor * (1 + 1e-2 * np.sin(t / 7e3))
        elif x < 40.0:                               # just above threshold: still growing
            A = 1e-6 * np.exp(2e-5 * t)
        else:                                        # logistic growth to sqrt(a (De - De_c))
            Asat = np.sqrt(2e-7 * (x - dec))
            A0 = 1e-6
            A = Asat / np.sqrt(1 + (Asat ** 2 / A0 ** 2 - 1) * np.exp(-2 * 1e-4 * t))
        series.append(A)
    sat = np.array([is_saturated(A, floor) for A in series])
    assert sat.tolist() == [False, False, False, False, True, True, True, True]
    a_fin = np.array([A[-1] for A in series])
    assert critical_dean_saturation(de, a_fin, floor, saturated=sat) == pytest.approx(dec, rel=1e-3)
    # a floor-only test would take the growing instance at De = 39 as saturated and be biased
    assert abs(critical_dean_saturation(de, a_fin, floor) - dec) > 0.1


def test_mixed_batch_recipe_is_seeded_and_in_range():
    from paper_1411_3133_gb300.workloads import BASE_SEED, force_reference_cylinder, mixed_batch
    a, b = mixed_batch(), mixed_batch()
    assert a == b                                          # seeded
    assert len(a) == 128
    assert sum(i.metric == "cylindrical" for i in a) == 64
    for k, inst in enumerate(a):
        assert inst.nr in (32, 48, 64) and 128 <= inst.n3 <= 512 and inst.ntheta == 4
        assert 20.0 <= inst.dean <= 150.0 and inst.tau == 0.55 and inst.seed == BASE_SEED + k
        ref = force_reference_cylinder(inst)
        assert ref["metric"] == "cylindrical" and ref["nr"] == inst.nr
        if inst.metric == "ellipsoidal":
            assert 0.25 <= inst.R2_over_R1 <= 4.0 and not inst.periodic3
            # Sec. IV.B recipe: R_theta = r_i b^2 = 1, d = R1/40
            assert inst.r_inner * inst.b ** 2 == pytest.approx(1.0)
            assert inst.r_outer - inst.r_inner == pytest.approx(1 / 40)
            assert ref["r_outer"] - ref["r_inner"] == pytest.approx(1 / 40)
    total = sum(i.ncells for i in a)
    assert 7.0e6 < total < 9.5e6                           # about 7.9 M nodes expected
    ratios = np.log([i.R2_over_R1 for i in a if i.metric == "ellipsoidal"])
    assert ratios.min() < np.log(0.5) and ratios.max() > np.log(2.0)   # spans the range


def test_knee_of_imperfect_bifurcation_curve():
    """A base flow ~ De^2 plus a smooth onset (softplus) at De_c: the largest
    curvature of <omega>(De) sits at De_c; a pure power law has no knee."""
    from paper_1411_3133_gb300.sweep import critical_dean_knee
    for dec, s in ((30.0, 1.5), (24.3, 1.0), (35.7, 2.0)):
        de = np.linspace(14.0, 44.0, 16)
        w = 1e-7 * de ** 2 + 1e-4 * s * np.log1p(np.exp((de - dec) / s))
        got = critical_dean_knee(de, w)
        assert abs(got - dec) < 0.35 * (de[1] - de[0]), (dec, got)
        # uneven, unsorted samples
        rng = np.random.default_rng(3)
        de2 = np.sort(14.0 + 30.0 * rng.random(24))
        w2 = 1e-7 * de2 ** 2 + 1e-4 * s * np.log1p(np.exp((de2 - dec) / s))
        perm = rng.permutation(24)
        assert abs(critical_dean_knee(de2[perm], w2[perm]) - dec) < 1.0
    de = np.linspace(14.0, 44.0, 16)
    assert np.isnan(critical_dean_knee(de, 1e-7 * de ** 3))
    assert np.isnan(critical_dean_knee(de[:4], de[:4]))
    # NaN samples (diverged instances) are dropped
    w = 1e-7 * de ** 2 + 1e-4 * np.log1p(np.exp(de - 30.0))
    w[-2:] = np.nan
    assert abs(critical_dean_knee(de, w) - 30.0) < 0.7


def test_decay_rate_and_its_zero_crossing():
    from paper_1411_3133_gb300.sweep import critical_dean_decay, decay_rate
    t = np.arange(2000, 400001, 2000, dtype=float)
    dec, slope = 47.3, 4e-7
    de = np.array([40.0, 42.0, 44.0, 46.0, 48.0, 50.0])
    sig_true = slope * (de - dec)
    sig = []
    for s in sig_true:
        # mean-flow transient early on, then the slow mode; a floor at 1e-9
        A = np.maximum(3e-3 * np.exp(s * t) + 1e-3 * np.exp(-1e-4 * t), 1e-9)
        sig.append(decay_rate(t, A, 1e-9) if s < 0 else float("nan"))
    sig = np.array(sig)
    assert np.allclose(sig[:4], sig_true[:4], rtol=0.02)
    assert critical_dean_decay(de, sig) == pytest.approx(dec, abs=0.05)
    # a fast decay that hits the floor early keeps only the samples above it
    A = np.maximum(1e-3 * np.exp(-5e-5 * t), 1e-9)
    assert decay_rate(t, A, 1e-9) == pytest.approx(-5e-5, rel=1e-6)
    assert np.isnan(decay_rate(t, np.full_like(t, 1e-9), 1e-9))
    assert np.isnan(critical_dean_decay(de, [np.nan, -1e-6, np.nan, 1e-6, 1e-6, 1e-6]))


def test_double_curved_case_lists_follow_the_paper():
    """Sec. IV.A varies R_theta = r_i b^2 at r_i = 1; Sec. IV.B varies
    R_phi = r_i at R_theta = 1."""
    from paper_1411_3133_gb300.sweep import cross_section_curvature_cases, streamwise_curvature_cases
    for label, ri, b in streamwise_curvature_cases():
        assert ri == 1.0 and 0.6 <= b * b * ri <= 1.5
    for label, ri, b in cross_section_curvature_cases():
        assert ri * b * b == pytest.approx(1.0)


def test_dean_bracket_between_last_decaying_and_first_saturated():
    from paper_1411_3133_gb300.sweep import dean_bracket
    assert dean_bracket([43.0, 40.0, 42.0, 41.0], [True, False, True, False]) == [41.0, 42.0]
    lo, hi = dean_bracket([40.0, 41.0], [False, False])
    assert lo == 41.0 and np.isnan(hi)
    lo, hi = dean_bracket([40.0, 41.0], [True, True])
    assert np.isnan(lo) and hi == 40.0


def test_vortex_cells_counts_sign_bands_along_x3():
    from paper_1411_3133_gb300.sweep import vortex_cells
    nr, nt, n3 = 9, 4, 128
    rng = np.random.default_rng(5)
    z = np.arange(n3)
    r = np.sin(np.pi * (np.arange(nr) + 0.5) / nr)[:, None, None]
    for k, cells in ((1, 2), (2, 4), (3, 6)):
        ur = r * np.sin(2 * np.pi * k * (z + 0.3) / n3)[None, None, :] * np.ones((nr, nt, 1))
        ur = ur * 1e-3 + 1e-6 * rng.standard_normal(ur.shape)
        assert vortex_cells(ur.ravel(), nr, nt, n3) == cells
        # an x3-uniform radial drift is not a vortex
        assert vortex_cells((ur + 5e-3).ravel(), nr, nt, n3) == cells
    assert vortex_cells(np.zeros(nr * nt * n3), nr, nt, n3) == 0
    # the 6-cell state of Sec. IV.B: one of the three wavelengths weaker
    ur = (np.sin(2 * np.pi * 3 * z / n3) * (1 + 0.4 * np.cos(2 * np.pi * z / n3)))[None, None, :]
    assert vortex_cells((r * ur * np.ones((nr, nt, 1))).ravel(), nr, nt, n3) == 6


def test_vortex_cells_walled_x3():
    """Four-wall channel (walls on x3): the return flow runs along the x3
    walls, so the mid-gap u^r reads -, +, - for 2 cells and -, +, -, +, -
    for 4; no wrap-around comparison (with it, the equal end signs would be
    ignored and an odd band count would gain a change)."""
    from paper_1411_3133_gb300.sweep import vortex_cells
    nr, nt, n3 = 9, 2, 96
    x = (np.arange(n3) + 0.5) / n3                      # 0..1 between the walls
    r = np.sin(np.pi * (np.arange(nr) + 0.5) / nr)[:, None, None]
    env = 1.0 - (2.0 * x - 1.0) ** 8                     # u = 0 on the walls, flat inside
    for k, cells in ((1, 2), (2, 4), (3, 6)):
        prof = -np.cos(2 * np.pi * k * x) * env          # negative at both walls
        ur = (r * prof[None, None, :] * np.ones((nr, nt, 1))).ravel() * 1e-3
        assert vortex_cells(ur, nr, nt, n3, periodic=False) == cells
        # with an area weight along x3 the count is unchanged
        assert vortex_cells(ur, nr, nt, n3, periodic=False, weights=1.0 + 0.2 * x) == cells
    # two bands (+, -) between walls: one change; the periodic count would
    # add a second at the wrap
    prof = np.cos(np.pi * x) * env
    ur = (r * prof[None, None, :] * np.ones((nr, nt, 1))).ravel()
    assert vortex_cells(ur, nr, nt, n3, periodic=False) == 1
    assert vortex_cells(ur, nr, nt, n3, periodic=True) == 2
