"""Oracle pins for the D3Q41 lattice (Table I) and its Hermite tensors.

What pins it: the velocities and weights printed in Table I (golden fixture),
exact rational/irrational arithmetic of the weights, and the quadrature
identities the lattice must satisfy for Gauss-Hermite quadrature to hold
(Sec. II: moments of the equilibrium are preserved exactly).
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import lattice as L

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d3q41_table1.txt")
NS = {"sqrt": math.sqrt}


def _golden():
    rows, cs2 = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = [p.strip() for p in line.split("|")]
        if parts[0] == "cs2":
            cs2 = parts[1]
            continue
        pats = [tuple(int(v) for v in p.strip("()").split(",")) for p in parts[1].split()]
        rows.append((parts[0], pats, parts[2]))
    return cs2, rows


def test_cs2_matches_paper():
    cs2, _ = _golden()
    assert L.CS2 == pytest.approx(eval(cs2, NS), abs=1e-16)


def test_velocities_and_weights_match_table_I():
    _, rows = _golden()
    expected = {}
    for lam, pats, wexpr in rows:
        w = eval(wexpr, NS)
        lo, _, hi = lam.partition("-")
        count = int(hi or lo) - int(lo) + 1
        vecs = set()
        for p in pats:
            axes = [i for i, v in enumerate(p) if v]
            for signs in itertools.product((1, -1), repeat=len(axes)):
                v = [0, 0, 0]
                for a, s in zip(axes, signs):
                    v[a] = s * p[a]
                vecs.add(tuple(v))
        assert len(vecs) == count, lam
        for v in vecs:
            expected[v] = w
    got = {tuple(int(x) for x in c): w for c, w in zip(L.C, L.W)}
    assert len(got) == 41 == len(expected)
    assert set(got) == set(expected)
    for v in got:
        assert got[v] == pytest.approx(expected[v], rel=1e-14, abs=1e-18)


def test_weights_sum_to_one_exactly():
    sympy = pytest.importorskip("sympy")
    _, rows = _golden()
    total = 0
    for lam, _, wexpr in rows:
        lo, _, hi = lam.partition("-")
        count = int(hi or lo) - int(lo) + 1
        total += count * sympy.sympify(wexpr)
    assert sympy.simplify(total - 1) == 0


def test_opposite_map():
    assert (L.C[L.OPPOSITE] == -L.C).all()
    assert (L.OPPOSITE[L.OPPOSITE] == np.arange(41)).all()


def _moment(n):
    """sum_l w_l c^i1 ... c^in as a rank-n array."""
    c = L.C.astype(float)
    letters = "abcdefgh"[:n]
    spec = "l," + ",".join("l" + x for x in letters) + "->" + letters
    return np.einsum(spec, L.W, *([c] * n))


def _iso(n):
    """Isotropic tensor: sum over all pairings of delta products (rank n even)."""
    idx = list(range(n))
    out = np.zeros((3,) * n)

    def pairings(items):
        if not items:
            yield []
            return
        a = items[0]
        for i in range(1, len(items)):
            b = items[i]
            rest = items[1:i] + items[i + 1:]
            for p in pairings(rest):
                yield [(a, b)] + p

    for p in pairings(idx):
        for ind in itertools.product(range(3), repeat=n):
            if all(ind[a] == ind[b] for a, b in p):
                out[ind] += 1.0
    return out


@pytest.mark.parametrize("n", [1, 3, 5, 7])
def test_odd_moments_vanish(n):
    assert np.abs(_moment(n)).max() < 1e-15


@pytest.mark.parametrize("n", [2, 4, 6])
def test_even_moments_isotropic(n):
    # sum_l w_l c^i1 ... c^in = cs^n * (sum over pairings of deltas)
    expected = L.CS2 ** (n // 2) * _iso(n)
    assert np.abs(_moment(n) - expected).max() < 5e-15


def test_hermite_orthogonality():
    # sum_l w_l H_m H_n = 0 for m != n (m, n <= 3), and the norms
    # cs^2 delta, cs^4 (dd + dd), cs^6 (sum over the 6 index permutations).
    W, tol = L.W, 1e-15
    for H in (L.H1, L.H2, L.H3):
        assert np.abs(np.tensordot(W, H, axes=1)).max() < tol
    assert np.abs(np.einsum("l,li,ljk->ijk", W, L.H1, L.H2)).max() < tol
    assert np.abs(np.einsum("l,li,ljkm->ijkm", W, L.H1, L.H3)).max() < tol
    assert np.abs(np.einsum("l,lij,lkmn->ijkmn", W, L.H2, L.H3)).max() < tol
    d = np.eye(3)
    n1 = np.einsum("l,li,lj->ij", W, L.H1, L.H1)
    assert np.abs(n1 - L.CS2 * d).max() < tol
    n2 = np.einsum("l,lij,lkm->ijkm", W, L.H2, L.H2)
    exp2 = L.CS2 ** 2 * (np.einsum("ik,jm->ijkm", d, d) + np.einsum("im,jk->ijkm", d, d))
    assert np.abs(n2 - exp2).max() < tol
    n3 = np.einsum("l,lijk,labc->ijkabc", W, L.H3, L.H3)
    exp3 = L.CS2 ** 3 * sum(_perm_delta(p) for p in itertools.permutations(range(3)))
    assert np.abs(n3 - exp3).max() < 1e-14  # entries up to 0.3, sums of c^6 <= 729


def _perm_delta(perm):
    """delta^{i a_perm0} delta^{j a_perm1} delta^{k a_perm2} as a rank-6 array."""
    out = np.zeros((3,) * 6)
    for ijk in itertools.product(range(3), repeat=3):
        abc = [0, 0, 0]
        for src, dst in enumerate(perm):
            abc[dst] = ijk[src]
        out[ijk + tuple(abc)] += 1.0
    return out
