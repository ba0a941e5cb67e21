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
