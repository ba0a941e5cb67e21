"""D3Q41 discrete velocity set (Table I) and its tensor Hermite polynomials.

Paper: Sec. II, Table I (velocities and weights), the speed of sound
cs^2 = 1 - sqrt(2/5) (Sec. II, text after the D3Q41 citation), and the
normalised Hermite polynomials that appear in the lattice equilibrium and in
the forcing term (Sec. II, lattice f^eq and forcing expressions).

Ordering (0-based index = Table I's lambda - 1): the rest velocity, then the
shells in Table I's row order. Inside a row with several sign patterns the
order is lexicographic with '+' before '-'. The table does not fix this order;
nothing in the method depends on it.

Oracle module: test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

SQRT10 = math.sqrt(10.0)

# cs^2 = 1 - sqrt(2/5)  (Sec. II)
CS2 = 1.0 - math.sqrt(2.0 / 5.0)

# Table I, one entry per row: (list of velocity patterns, weight).
# A pattern is a 3-tuple whose entries are 0 or a magnitude s; every non-zero
# entry takes both signs.
_TABLE_I = [
    ([(0, 0, 0)], 2.0 / 2025.0 * (5045.0 - 1507.0 * SQRT10)),
    ([(1, 0, 0), (0, 1, 0), (0, 0, 1)], 37.0 / (5.0 * SQRT10) - 91.0 / 40.0),
    ([(1, 1, 0), (1, 0, 1), (0, 1, 1)], (55.0 - 17.0 * SQRT10) / 50.0),
    ([(1, 1, 1)], (233.0 * SQRT10 - 730.0) / 1600.0),
    ([(3, 0, 0), (0, 3, 0), (0, 0, 3)], (295.0 - 92.0 * SQRT10) / 16200.0),
    ([(3, 3, 3)], (130.0 - 41.0 * SQRT10) / 129600.0),
]


def _expand(pattern):
    """All sign choices of a Table I pattern, '+' before '-' (lexicographic)."""
    axes = [i for i, v in enumerate(pattern) if v != 0]
    out = []
    for signs in itertools.product((1, -1), repeat=len(axes)):
        v = [0, 0, 0]
        for a, s in zip(axes, signs):
            v[a] = s * pattern[a]
        out.append(tuple(v))
    return out


def _build():
    cs, ws = [], []
    for patterns, weight in _TABLE_I:
        for p in patterns:
            for v in _expand(p):
                cs.append(v)
                ws.append(weight)
    return np.array(cs, dtype=np.int64), np.array(ws, dtype=np.float64)


C, W = _build()          # C: (41, 3) integer velocities; W: (41,) weights
Q = C.shape[0]
assert Q == 41

# index of the opposite velocity -c
OPPOSITE = np.array([int(np.flatnonzero((C == -C[l]).all(axis=1))[0]) for l in range(Q)])

DELTA = np.eye(3)


def hermite_tensors(c=C, cs2=CS2):
    """Lattice Hermite tensors used in Sec. II's f^eq and forcing sums.

    H1[l,i]     = c^i
    H2[l,i,j]   = c^i c^j - cs^2 delta^ij
    H3[l,i,j,k] = c^i c^j c^k - cs^2 (delta^ij c^k + delta^jk c^i + delta^ki c^j)
    """
    c = c.astype(np.float64)
    d = DELTA
    H1 = c.copy()
    H2 = np.einsum("li,lj->lij", c, c) - cs2 * d[None, :, :]
    H3 = (np.einsum("li,lj,lk->lijk", c, c, c)
          - cs2 * (np.einsum("ij,lk->lijk", d, c)
                   + np.einsum("jk,li->lijk", d, c)
                   + np.einsum("ki,lj->lijk", d, c)))
    return H1, H2, H3


H1, H2, H3 = hermite_tensors()
