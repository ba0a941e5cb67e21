"""Oracle pins for streaming with walls (Eq. LB left-hand side, walls).

What pins it:
  * away from walls the pull map is a plain periodic shift, f(x + c) <- f*(x),
    i.e. numpy.roll by +c: a wrong sign or axis fails;
  * the map is a permutation of (population, node) pairs, so streaming
    conserves every population sum exactly;
  * hand-worked wall cases of the full bounce-back rule, each traced by hand
    on paper (walls halfway outside the first and last node):
      |c_r| = 1 at the first node: same node, opposite population
      |c_r| = 3 at nodes 0, 1, 2: source node 2 (tangential +2 sign(c_t)),
        same node, node 0 (tangential -2 sign(c_t)); opposite population
      a 7 x 7 corner where the path meets walls three times in one step;
  * a uniform rest state f_l = w_l is unchanged by streaming with walls.
"""
import numpy as np
import pytest

from oracle import lattice as L
from oracle.geometry import Channel
from oracle.lbm import StreamMap

CHANNELS = [
    Channel("cylindrical", 1.0, 1 / 0.975, 16, 4, 32),
    Channel("cylindrical", 1.0, 1 / 0.975, 7, 1, 5),
    Channel("ellipsoidal", 1.0, 1.025, 7, 3, 7, periodic3=False),
    Channel("ellipsoidal", 1.0, 1.025, 9, 2, 8, periodic3=False),
    Channel("flat", 0.0, 1.0, 8, 2, 1),
]


def _lam(c):
    return int(np.flatnonzero((L.C == np.array(c)).all(axis=1))[0])


@pytest.mark.parametrize("ch", CHANNELS, ids=lambda c: f"{c.metric}{c.shape}{c.periodic3}")
def test_stream_map_is_a_permutation(ch):
    sm = StreamMap(ch)
    flat = sm.src_pop * ch.ncells + sm.src_cell
    assert np.unique(flat).size == flat.size == L.Q * ch.ncells
    f = np.random.default_rng(0).random((L.Q, ch.ncells))
    assert sm.apply(f).sum() == pytest.approx(f.sum(), rel=1e-15)


def test_interior_streaming_is_numpy_roll():
    ch = Channel("cylindrical", 1.0, 1 / 0.975, 12, 5, 9)
    sm = StreamMap(ch)
    f = np.random.default_rng(1).random((L.Q, ch.ncells))
    fs = sm.apply(f).reshape((L.Q,) + ch.shape)
    f3 = f.reshape((L.Q,) + ch.shape)
    for l in range(L.Q):
        rolled = np.roll(f3[l], shift=tuple(int(v) for v in L.C[l]), axis=(0, 1, 2))
        # rows 3..N-4 along r are out of reach of the walls
        assert np.array_equal(fs[l, 3:-3], rolled[3:-3]), l


def _src(sm, ch, x, c):
    l = _lam(c)
    cell = (x[0] * ch.ntheta + x[1]) * ch.n3 + x[2]
    s = int(sm.src_cell[l, cell])
    y = np.unravel_index(s, ch.shape)
    return tuple(int(v) for v in y), int(sm.src_pop[l, cell])


def test_hand_worked_wall_cases_cylinder():
    ch = Channel("cylindrical", 1.0, 1 / 0.975, 8, 6, 10)
    sm = StreamMap(ch)
    op = lambda c: _lam(tuple(-v for v in c))
    # |c_r| = 1, first node: halfway bounce-back
    assert _src(sm, ch, (0, 2, 4), (1, 1, 0)) == ((0, 2, 4), op((1, 1, 0)))
    # |c_r| = 3 at node 0: source node 2, theta + 2
    assert _src(sm, ch, (0, 2, 4), (3, 3, 3)) == ((2, 4, 6), op((3, 3, 3)))
    assert _src(sm, ch, (0, 2, 4), (3, -3, 3)) == ((2, 0, 6), op((3, -3, 3)))
    assert _src(sm, ch, (0, 2, 4), (3, 0, 0)) == ((2, 2, 4), op((3, 0, 0)))
    # node 1: same node
    assert _src(sm, ch, (1, 2, 4), (3, 0, 0)) == ((1, 2, 4), op((3, 0, 0)))
    assert _src(sm, ch, (1, 2, 4), (3, 3, 3)) == ((1, 2, 4), op((3, 3, 3)))
    # node 2: source node 0, tangential -2 sign(c_t)
    assert _src(sm, ch, (2, 2, 4), (3, 3, -3)) == ((0, 0, 6), op((3, 3, -3)))
    # node 3: no wall within reach
    assert _src(sm, ch, (3, 2, 4), (3, 0, 0)) == ((0, 2, 4), _lam((3, 0, 0)))
    # outer wall (mirror image): last node N-1 = 7, c_r = -3 -> source node 5
    assert _src(sm, ch, (7, 2, 4), (-3, 0, 0)) == ((5, 2, 4), op((-3, 0, 0)))
    assert _src(sm, ch, (7, 2, 4), (-1, 0, 1)) == ((7, 2, 4), op((-1, 0, 1)))
    # periodic wrap in theta and z
    assert _src(sm, ch, (4, 0, 9), (3, 3, -3)) == ((1, 3, 2), _lam((3, 3, -3)))


def test_hand_worked_corner_three_reflections():
    """7 x 7 walled cross-section, node (0, th, 6), c = (3, 3, 3). Backwards the
    path meets r = -1/2 at t = 1/6, then x3 = 6.5 at t = 1/2, then r = -1/2 at
    t = 5/6, and ends at t = 1 on its starting node: odd count, opposite."""
    ch = Channel("ellipsoidal", 1.0, 1.025, 7, 2, 7, periodic3=False)
    sm = StreamMap(ch)
    assert _src(sm, ch, (0, 1, 6), (3, 3, 3)) == ((0, 1, 6), _lam((-3, -3, -3)))
    # one reflection off the x3 wall only: node (3, ., 0), c = (0, 0, 3)
    assert _src(sm, ch, (3, 1, 0), (0, 0, 3)) == ((3, 1, 2), _lam((0, 0, -3)))


def test_uniform_rest_state_is_invariant():
    for ch in CHANNELS:
        sm = StreamMap(ch)
        f = np.repeat(L.W[:, None], ch.ncells, axis=1)
        assert np.array_equal(sm.apply(f), f)
