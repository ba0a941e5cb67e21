"""Host-side array logic of the surrogate pipeline (no GPU): phase
alignment of periodic vortex fields, and the input / target layouts."""
import numpy as np

from paper_1411_3133_gb300 import surrogate as S


def test_phase_alignment_maps_shifted_vortices_onto_one_phase():
    spec = S.channel()
    k = np.arange(spec.n3)
    B, N = 4, spec.ncells
    u = np.zeros((B, 3, N))
    rho = np.ones((B, N))
    shifts = [0, 5, 17, 40]
    for b, sh in enumerate(shifts):
        prof = np.sin(np.pi * (np.arange(spec.nr) + 0.5) / spec.nr)[:, None, None]
        f = np.cos(2 * np.pi * (k - sh) / spec.n3) + 0.3 * np.cos(4 * np.pi * (k - sh) / spec.n3)
        u[b, 0] = (prof * f[None, None, :] * np.ones((1, spec.ntheta, 1))).ravel()
        u[b, 2] = (prof * np.sin(2 * np.pi * (k - sh) / spec.n3)[None, None, :]
                   * np.ones((1, spec.ntheta, 1))).ravel()
        rho[b] = 1.0 + 1e-3 * u[b, 0]
    r, a = S.align_phase(S.theta_mean(spec, rho), S.theta_mean(spec, u))
    for b in range(1, B):
        assert np.abs(a[b] - a[0]).max() < 1e-12
        assert np.abs(r[b] - r[0]).max() < 1e-12
    # a laminar field (no x3 dependence) is left alone
    lam = np.zeros((1, 3, spec.nr, spec.n3))
    lam[0, 1] = 0.1
    _, b2 = S.align_phase(np.ones((1, spec.nr, spec.n3)), lam)
    assert np.array_equal(b2, lam)


def test_inputs_and_targets_layout():
    spec = S.channel()
    x = S.inputs(spec, [30.0, 45.0])
    assert x.shape == (2 * spec.nr * spec.n3, 3)
    assert np.allclose(x[0], [0.30, 0.5 / spec.nr, 0.5 / spec.n3])
    assert np.allclose(x[spec.n3], [0.30, 1.5 / spec.nr, 0.5 / spec.n3])     # next i_r
    assert np.allclose(x[spec.nr * spec.n3], [0.45, 0.5 / spec.nr, 0.5 / spec.n3])
    rho = np.arange(2 * spec.nr * spec.n3, dtype=float).reshape(2, spec.nr, spec.n3)
    u = np.stack([rho + 1, rho + 2, rho + 3], axis=1)
    y = S.targets(rho, u)
    assert y.shape == (2 * spec.nr * spec.n3, 4)
    assert np.allclose(y[7], [7, 8, 9, 10])


def test_steps_to_developed():
    t = np.arange(1, 11) * 2000
    grow = np.array([1e-6, 1e-5, 1e-4, 6e-4, 1.1e-3, 1.19e-3, 1.2e-3, 1.2e-3, 1.21e-3, 1.2e-3])
    warm = np.full(10, 1.2e-3)
    late = grow.copy()
    late[-1] = 2e-3                                   # leaves the band at the end: never developed
    a = np.stack([grow, warm, late], axis=1)
    s = S.steps_to_developed(t, a, np.array([1.2e-3, 1.2e-3, 1.2e-3]))
    assert s[0] == 12000 and s[1] == 2000 and np.isinf(s[2])      # 1.19e-3 is within 2 %


def test_mixed_draws_respect_the_speed_cap_and_the_distribution():
    insts = S.draw_mixed(300, 5, speed_cap=0.25)
    assert len(insts) == 300
    assert all(S.laminar_speed(i) <= 0.25 for i in insts)
    kinds = {i.metric for i in insts}
    assert kinds == {"cylindrical", "ellipsoidal"}
    assert {i.nr for i in insts} == {32, 48, 64}
    assert all(128 <= i.n3 <= 512 and 20 <= i.dean <= 150 and i.tau == 0.55 for i in insts)
    ell = [i for i in insts if i.metric == "ellipsoidal"]
    assert all(0.25 <= i.R2_over_R1 <= 4.0 for i in ell)
    # the cap removes high Dean numbers on coarse grids only
    assert max(i.dean for i in insts if i.nr == 32) < 70 < max(i.dean for i in insts if i.nr == 64)


def test_laminar_speed_matches_the_dean_number_definition():
    from paper_1411_3133_gb300.workloads import Instance
    inst = Instance("cylindrical", 1.0, 1 / 0.975, 64, 4, 256, 0.55, 40.0, 1)
    nu = 0.05 * (1 - np.sqrt(0.4))
    d = 1 / 0.975 - 1
    U = S.laminar_speed(inst)
    assert abs(U * 64 / nu * np.sqrt(d) - 40.0) < 1e-12


def test_mixed_inputs_fields_and_alignment(monkeypatch):
    from paper_1411_3133_gb300.workloads import Instance
    cyl = Instance("cylindrical", 1.0, 1 / 0.975, 8, 4, 24, 0.55, 40.0, 1)
    ell = Instance("ellipsoidal", 2.0, 2.025, 8, 4, 24, 0.55, 60.0, 2, b=2 ** -0.5, periodic3=False,
                   dtheta_scale=0.5 ** 0.5 / 2, d3_scale=0.5, R2_over_R1=2.0)
    x = S.mixed_inputs(ell, 8, 24)
    assert x.shape == (8 * 24, S.N_PLAIN_MIXED + 1)
    assert np.allclose(x[0], [60 / 150, 1, 0.5, 24 / 8 / 16, 0.5 / 8, 0.5, 0.5 / 24])
    assert np.allclose(x[24, 4], 1.5 / 8)                  # next i_r
    assert S.mixed_inputs(cyl, 8, 24)[0, 2] == 0.0        # no cross-sectional curvature
    # targets -> fields round trip (sqrt g from the library's host geometry)
    monkeypatch.setattr(S, "_sqrtg", lambda inst: np.linspace(0.9, 1.1, inst.nr * inst.n3).reshape(inst.nr, inst.n3))
    rng = np.random.default_rng(1)
    rho = 1 + 0.01 * rng.standard_normal((8, 24))
    u = 0.05 * rng.standard_normal((3, 8, 24))
    y = S.mixed_targets(ell, rho, u)
    r2, u2 = S.mixed_fields(ell, y, 4)
    assert np.allclose(r2.reshape(8, 4, 24)[:, 2], rho, rtol=1e-6)
    assert np.allclose(u2.reshape(3, 8, 4, 24)[:, :, 1], u, rtol=1e-5, atol=1e-9)
    # a periodic 4-cell field shifted along z aligns onto the unshifted one;
    # a walled channel's field is left in place
    z = np.arange(24)
    prof = np.sin(np.pi * (np.arange(8) + 0.5) / 8)[:, None]
    base = np.stack([prof * np.cos(4 * np.pi * z / 24)[None, :], np.full((8, 24), 0.1),
                     prof * np.sin(4 * np.pi * z / 24)[None, :]])
    _, a0 = S.align_mixed(cyl, np.ones((8, 24)), base)
    _, a1 = S.align_mixed(cyl, np.ones((8, 24)), np.roll(base, 5, axis=-1))
    assert np.abs(a0 - a1).max() < 1e-12
    _, w = S.align_mixed(ell, np.ones((8, 24)), np.roll(base, 5, axis=-1))
    assert np.array_equal(w, np.roll(base, 5, axis=-1))
