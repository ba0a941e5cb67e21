"""Oracle pins for the equilibrium, the forcing term and the BGK collision.

What pins them (all derived from Hermite orthogonality and the D3Q41 moment
identities up to 6th order, not from the oracle's code):
  * f^eq moments 0..3: rho', rho' u, rho' cs^2 g^ij + rho' u u, and
    rho' cs^2 (g^ij u^k + g^jk u^i + g^ki u^j) + rho' u u u. The 2nd moment is
    how the metric enters the pressure tensor of Sec. II's momentum equation.
  * forcing moments:
      sum_l F_l          = -2 a1^i Gamma^j_ij   (the covariant continuity
                           equation's source for rho' = rho/sqrt g)
      sum_l c^m F_l      = a0 F_ext^m - a0 cs^2 (Gamma^m_jj + 2 Gamma^j_jm)
                           - 2 A2^ml Gamma^j_jl - A2^lj Gamma^m_lj
      (Gamma = 0) sum c^m c^n F_l     = a1^m F^n + a1^n F^m
      (Gamma = 0) sum c^m c^n c^p F_l = a0 cs^2 (d^mn F^p + d^np F^m + d^pm F^n)
                                        + A2^mn F^p + A2^np F^m + A2^pm F^n
  * collision: BGK conserves mass and momentum when the forcing vanishes; the
    improved coefficient A2 = a2^eq + (1 - 1/(2 tau)) Pi^neq (Sec. II) is seen
    in the 3rd moment of the forcing for a state with a known Pi^neq.
"""
import itertools

import numpy as np
import pytest

from oracle import lattice as L
from oracle.lbm import collide, equilibrium, force_vectors, forcing

CS2 = 1.0 - np.sqrt(0.4)
C = L.C.astype(float)
D = np.eye(3)


def _random_state(rng, n=5):
    rho = rng.uniform(0.8, 1.2, n)
    u = rng.uniform(-0.1, 0.1, (n, 3))
    A = rng.normal(size=(n, 3, 3)) * 0.1
    g = D + 0.5 * (A + A.transpose(0, 2, 1))
    Delta = np.linalg.inv(g) - D
    Gam = rng.normal(size=(n, 3, 3, 3)) * 0.01
    Gam = 0.5 * (Gam + Gam.transpose(0, 1, 3, 2))       # symmetric lower indices
    return rho, u, g, Delta, Gam


def _close(got, exp, rel=1e-12):
    """Equal up to roundoff: max error <= rel * largest expected magnitude."""
    scale = max(np.abs(exp).max(), 1e-300)
    err = np.abs(got - exp).max()
    assert err <= rel * scale, (err, scale)


def _mom(f, k):
    """sum_l c^a ... c^(k) f_l, shape (n,) + (3,) * k."""
    if k == 0:
        return f.sum(0)
    ops = [C] * k
    letters = "abc"[:k]
    return np.einsum(",".join("l" + x for x in letters) + ",ln->n" + letters, *ops, f)


def test_equilibrium_moments():
    rng = np.random.default_rng(0)
    rho, u, g, Delta, _ = _random_state(rng)
    f = equilibrium(rho, u, Delta)
    gi = np.linalg.inv(g)
    assert np.allclose(_mom(f, 0), rho, rtol=1e-14)
    assert np.allclose(_mom(f, 1), rho[:, None] * u, rtol=0, atol=1e-15)
    m2 = rho[:, None, None] * (CS2 * gi + np.einsum("ni,nj->nij", u, u))
    assert np.abs(_mom(f, 2) - m2).max() < 1e-14
    m3 = (rho[:, None, None, None] * CS2
          * (np.einsum("nij,nk->nijk", gi, u) + np.einsum("njk,ni->nijk", gi, u)
             + np.einsum("nki,nj->nijk", gi, u))
          + rho[:, None, None, None] * np.einsum("ni,nj,nk->nijk", u, u, u))
    assert np.abs(_mom(f, 3) - m3).max() < 1e-14


def test_equilibrium_flat_rest_is_weights():
    f = equilibrium(np.array([1.3]), np.zeros((1, 3)), np.zeros((1, 3, 3)))
    assert np.allclose(f[:, 0], 1.3 * L.W, rtol=1e-15)


def _coeffs(rng, n):
    a0 = rng.uniform(0.8, 1.2, n)
    a1 = rng.normal(size=(n, 3)) * 0.1
    A2 = rng.normal(size=(n, 3, 3)) * 0.1
    A2 = 0.5 * (A2 + A2.transpose(0, 2, 1))
    fext = rng.normal(size=(n, 3)) * 1e-3
    return a0, a1, A2, fext


def test_forcing_zeroth_and_first_moment():
    rng = np.random.default_rng(1)
    n = 6
    a0, a1, A2, fext = _coeffs(rng, n)
    _, _, _, _, Gam = _random_state(rng, n)
    Fl = forcing(a0, a1, A2, force_vectors(Gam, fext))
    # sum_l F_l = -2 a1^i Gamma^j_ij
    exp0 = np.array([-2 * sum(a1[p, i] * Gam[p, j, i, j] for i in range(3) for j in range(3))
                     for p in range(n)])
    _close(Fl.sum(0), exp0)
    exp1 = np.zeros((n, 3))
    for p in range(n):
        for m in range(3):
            v = a0[p] * fext[p, m]
            v -= a0[p] * CS2 * sum(Gam[p, m, j, j] + 2 * Gam[p, j, j, m] for j in range(3))
            v -= 2 * sum(A2[p, m, l] * Gam[p, j, j, l] for l in range(3) for j in range(3))
            v -= sum(A2[p, l, j] * Gam[p, m, l, j] for l in range(3) for j in range(3))
            exp1[p, m] = v
    _close(_mom(Fl, 1), exp1)


def test_forcing_second_and_third_moment_external_force():
    rng = np.random.default_rng(2)
    n = 4
    a0, a1, A2, fext = _coeffs(rng, n)
    Fl = forcing(a0, a1, A2, force_vectors(np.zeros((n, 3, 3, 3)), fext))
    exp2 = np.einsum("nm,nk->nmk", a1, fext) + np.einsum("nk,nm->nmk", a1, fext)
    _close(_mom(Fl, 2), exp2)
    exp3 = np.zeros((n, 3, 3, 3))
    for p, m, q, r in itertools.product(range(n), range(3), range(3), range(3)):
        F = fext[p]
        exp3[p, m, q, r] = (a0[p] * CS2 * (D[m, q] * F[r] + D[q, r] * F[m] + D[r, m] * F[q])
                            + A2[p, m, q] * F[r] + A2[p, q, r] * F[m] + A2[p, r, m] * F[q])
    _close(_mom(Fl, 3), exp3)


def test_collision_conserves_without_force():
    rng = np.random.default_rng(3)
    rho, u, g, Delta, _ = _random_state(rng)
    f = equilibrium(rho, u, Delta) * (1 + 0.05 * rng.normal(size=(41, len(rho))))
    n = f.shape[1]
    fs = collide(f, Delta, np.zeros((n, 3, 3, 3)), np.zeros((n, 3)), tau=0.7)
    assert np.allclose(fs.sum(0), f.sum(0), rtol=1e-14)
    assert np.abs(_mom(fs, 1) - _mom(f, 1)).max() < 1e-15


def test_collision_mass_source():
    rng = np.random.default_rng(4)
    rho, u, g, Delta, Gam = _random_state(rng)
    f = equilibrium(rho, u, Delta) * (1 + 0.05 * rng.normal(size=(41, len(rho))))
    n = f.shape[1]
    fext = rng.normal(size=(n, 3)) * 1e-3
    fs = collide(f, Delta, Gam, fext, tau=0.9)
    r = f.sum(0)
    uu = _mom(f, 1) / r[:, None]
    src = -2 * np.einsum("n,ni,njij->n", r, uu, Gam)
    assert np.abs(fs.sum(0) - f.sum(0) - src).max() < 1e-15


def test_collision_tau_one_is_equilibrium_plus_forcing():
    rng = np.random.default_rng(6)
    rho, u, g, Delta, Gam = _random_state(rng)
    f = equilibrium(rho, u, Delta) * (1 + 0.05 * rng.normal(size=(41, len(rho))))
    n = f.shape[1]
    r = f.sum(0)
    uu = _mom(f, 1) / r[:, None]
    fs0 = collide(f, Delta, np.zeros((n, 3, 3, 3)), np.zeros((n, 3)), tau=1.0)
    assert np.abs(fs0 - equilibrium(r, uu, Delta)).max() < 1e-16


@pytest.mark.parametrize("old", [False, True])
def test_improved_forcing_uses_nonequilibrium_stress(old):
    """State f = f^eq + w H2:P/(2 cs^4): same rho', u, and sum c c (f - f^eq) = P.
    The forcing's 3rd moment (Gamma = 0) then shows A2 = a2^eq + (1 - 1/(2 tau)) P
    (improved, Sec. II) or A2 = a2^eq (old method)."""
    rng = np.random.default_rng(8)
    rho, u, g, Delta, _ = _random_state(rng, 3)
    n = len(rho)
    P = rng.normal(size=(n, 3, 3)) * 0.01
    P = 0.5 * (P + P.transpose(0, 2, 1))
    feq = equilibrium(rho, u, Delta)
    df = L.W[:, None] * np.einsum("lij,nij->ln", L.H2, P) / (2 * CS2 ** 2)
    f = feq + df
    assert np.abs(_mom(f - feq, 2) - P).max() < 1e-16
    tau = 0.65
    fext = rng.normal(size=(n, 3)) * 1e-3
    fs = collide(f, Delta, np.zeros((n, 3, 3, 3)), fext, tau=tau, old_forcing=old)
    Fl = fs - (f - (f - feq) / tau)
    a2eq = rho[:, None, None] * (CS2 * Delta + np.einsum("ni,nj->nij", u, u))
    A2 = a2eq if old else a2eq + (1 - 1 / (2 * tau)) * P
    exp3 = np.zeros((n, 3, 3, 3))
    for p, m, q, r in itertools.product(range(n), range(3), range(3), range(3)):
        F = fext[p]
        exp3[p, m, q, r] = (rho[p] * CS2 * (D[m, q] * F[r] + D[q, r] * F[m] + D[r, m] * F[q])
                            + A2[p, m, q] * F[r] + A2[p, q, r] * F[m] + A2[p, r, m] * F[q])
    _close(_mom(Fl, 3), exp3)
