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
