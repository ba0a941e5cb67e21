"""The lattice Boltzmann update in generalized metrics, plain and slow.

Paper: Sec. II.
  * moments  rho' = sum_l f_l,  rho' u^i = sum_l c^i_l f_l  (rho' = rho/sqrt g)
  * equilibrium Hermite coefficients a0..a3 with Delta^ij = g^ij - delta^ij,
    and the lattice f^eq (Gauss-Hermite quadrature with the Table I weights)
  * improved forcing coefficients: a0, a1 from f^eq, a2 = a2^eq - sigma with
    sigma^ij = -(1 - 1/(2 tau)) sum_l c^i c^j (f_l - f^eq_l)
  * forcing term F_l truncated at third order, F^i_l = -Gamma^i_jk c^j c^k,
    plus an external force F^i_l -> F^i_l + F^i_ext
  * LB equation (Eq. LB): f_l(x + c_l, t + 1) - f_l(x, t)
        = -(f_l - f^eq_l)/tau + F_l        (lattice units, Delta t = 1)
  * time stepping: initial f = f^eq(rho, u); each step is a free-streaming
    step followed by a collision step (end of Sec. II).

Readings:
  * State. The stored state is the post-collision population f* of the last
    step (at t = 0, f^eq of the initial fields). One step streams it (pull)
    and collides. ``macros`` reports the moments of the streamed populations,
    i.e. the rho' and u entering the next collision.
  * The velocity in f^eq and in the forcing is u = (sum c f)/rho' with no
    half-force shift (literal Sec. II).
  * tau is in units of the time step: collision factor 1/tau per step.
  * Walls (instead of the paper's Dirichlet equilibrium nodes): full
    bounce-back on the walls halfway outside the first and last node of a
    walled axis, applied along the whole path of a population within one time
    step. A population travelling from its source is reflected (velocity
    reversed) each time its straight path meets a wall; it lands where that
    folded path ends after one time unit. ``_trace_source`` follows the path
    backwards from the destination with exact rational arithmetic.
  * "Old" forcing (the paper's comparison method): a2 = a2^eq.
  * Equilibrium walls (the paper's own Dirichlet condition, Sec. III: the
    wall velocity 0 enters through the equilibrium on both walls at every
    step): the end nodes of a
    walled axis lie on the walls; after streaming, a wall node's populations
    are replaced by f^eq(rho', 0) of its own density and metric (no BGK
    relaxation, no forcing). A population whose source x - c lies beyond a
    wall is taken from the wall node of the same line (the source clamped
    onto the wall layer), i.e. nodes outside hold the wall's equilibrium.

Oracle module: test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction

import numpy as np

from . import lattice as L
from .geometry import Channel, channel_geometry


def _es(*args):
    """numpy einsum with contraction-order optimisation (same sums)."""
    return np.einsum(*args, optimize=True)


# --------------------------------------------------------------------------
# streaming with walls
# --------------------------------------------------------------------------
def _trace_source(x, c, dims, walled):
    """Where the population arriving at node x with velocity c came from.

    Follows the path backwards in time for one time unit, starting at x with
    velocity -c. A wall of axis a sits at -1/2 and at dims[a] - 1/2 when
    walled[a]; meeting one reverses the whole velocity (bounce-back). Returns
    (source position as integers, number of reflections).
    """
    pos = [Fraction(v) for v in x]
    vel = [-ci for ci in c]
    t_left = Fraction(1)
    reflections = 0
    while True:
        t_hit = None
        for a in range(3):
            if not walled[a] or vel[a] == 0:
                continue
            wall = Fraction(-1, 2) if vel[a] < 0 else Fraction(2 * dims[a] - 1, 2)
            t = (wall - pos[a]) / vel[a]
            if t_hit is None or t < t_hit:
                t_hit = t
        if t_hit is None or t_hit >= t_left:
            pos = [p + v * t_left for p, v in zip(pos, vel)]
            break
        pos = [p + v * t_hit for p, v in zip(pos, vel)]
        t_left -= t_hit
        vel = [-v for v in vel]
        reflections += 1
    assert all(p.denominator == 1 for p in pos), "source must be a lattice node"
    return [int(p) for p in pos], reflections


class StreamMap:
    """Pull map of one streaming step: destination (l, cell) <- source.

    f_streamed[l, cell] = f[src_pop[l, cell], src_cell[l, cell]]
    Cells are numbered (i_r * N_theta + i_theta) * N_3 + i_3.
    """

    def __init__(self, ch: Channel):
        dims = ch.shape
        walled = ch.walled
        nr, nt, n3 = dims
        cells = np.arange(ch.ncells)
        x = np.stack(np.unravel_index(cells, dims), axis=1)       # (n, 3)
        if ch.wall == "equilibrium":
            self._init_clamped(x, dims, walled)
            return
        # The traced path depends only on the coordinates along walled axes,
        # and not even on those when the node is at least 3 nodes away from
        # both walls (|c| <= 3 cannot reach a wall 3.5 away). Trace one
        # representative node per class and apply it to the whole class.
        key = np.zeros_like(x)
        for a in range(3):
            if walled[a]:
                far = (x[:, a] >= 3) & (x[:, a] <= dims[a] - 4)
                key[:, a] = np.where(far, 3, x[:, a])
        ukeys, inverse = np.unique(key, axis=0, return_inverse=True)
        inverse = inverse.reshape(-1)
        self.src_cell = np.empty((L.Q, ch.ncells), dtype=np.int64)
        self.src_pop = np.empty((L.Q, ch.ncells), dtype=np.int64)
        for l in range(L.Q):
            c = [int(v) for v in L.C[l]]
            disp = np.zeros((len(ukeys), 3), dtype=np.int64)
            odd = np.zeros(len(ukeys), dtype=bool)
            for u_i, probe in enumerate(ukeys):
                probe = tuple(int(v) for v in probe)
                src, k = _trace_source(probe, c, dims, walled)
                disp[u_i] = [s - p for s, p in zip(src, probe)]
                odd[u_i] = (k % 2 == 1)
            y = x + disp[inverse]
            for a in range(3):
                if not walled[a]:
                    y[:, a] %= dims[a]
            self.src_cell[l] = (y[:, 0] * nt + y[:, 1]) * n3 + y[:, 2]
            self.src_pop[l] = np.where(odd[inverse], L.OPPOSITE[l], l)

    def _init_clamped(self, x, dims, walled):
        """Equilibrium walls: source x - c, periodic axes wrapped, walled axes
        clamped onto the wall layer; the population index is kept."""
        nr, nt, n3 = dims
        self.src_cell = np.empty((L.Q, len(x)), dtype=np.int64)
        self.src_pop = np.empty((L.Q, len(x)), dtype=np.int64)
        for l in range(L.Q):
            y = x - L.C[l][None, :]
            for a in range(3):
                if walled[a]:
                    y[:, a] = np.clip(y[:, a], 0, dims[a] - 1)
                else:
                    y[:, a] %= dims[a]
            self.src_cell[l] = (y[:, 0] * nt + y[:, 1]) * n3 + y[:, 2]
            self.src_pop[l] = l

    def apply(self, f):
        """f: (Q, ncells) -> streamed populations (Q, ncells)."""
        return f[self.src_pop, self.src_cell]


# --------------------------------------------------------------------------
# equilibrium and forcing
# --------------------------------------------------------------------------
def moments(f):
    """rho' = sum_l f_l and u^i = sum_l c^i_l f_l / rho'  (Sec. II)."""
    rho = f.sum(axis=0)
    j = _es("li,ln->ni", L.C.astype(np.float64), f)
    return rho, j / rho[:, None]


def equilibrium_coefficients(rho, u, Delta, cs2=L.CS2):
    """Hermite coefficients of f^eq (Sec. II, Eq. hermite-coefficients-eq).

    a0 = rho', a1^i = rho' u^i, a2^ij = rho' cs^2 Delta^ij + rho' u^i u^j,
    a3^ijk = rho' cs^2 (Delta^ij u^k + Delta^jk u^i + Delta^ki u^j)
             + rho' u^i u^j u^k.
    Shapes: rho (n,), u (n,3), Delta (n,3,3).
    """
    a0 = rho
    a1 = rho[:, None] * u
    a2 = rho[:, None, None] * (cs2 * Delta + _es("ni,nj->nij", u, u))
    a3 = (rho[:, None, None, None] * cs2
          * (_es("nij,nk->nijk", Delta, u)
             + _es("njk,ni->nijk", Delta, u)
             + _es("nki,nj->nijk", Delta, u))
          + rho[:, None, None, None] * _es("ni,nj,nk->nijk", u, u, u))
    return a0, a1, a2, a3


def equilibrium(rho, u, Delta, cs2=L.CS2):
    """Lattice equilibrium f^eq_l (Sec. II):

    f^eq_l = w_l ( a0 + a1.H1/cs^2 + a2:H2/(2 cs^4) + a3:H3/(6 cs^6) ).
    Returns (Q, n).
    """
    a0, a1, a2, a3 = equilibrium_coefficients(rho, u, Delta, cs2)
    s = (a0[None, :]
         + _es("li,ni->ln", L.H1, a1) / cs2
         + _es("lij,nij->ln", L.H2, a2) / (2.0 * cs2 ** 2)
         + _es("lijk,nijk->ln", L.H3, a3) / (6.0 * cs2 ** 3))
    return L.W[:, None] * s


def force_vectors(Gamma_hat, fext):
    """F^i_l = -Gamma^i_jk c^j_l c^k_l + F^i_ext  (Sec. II).

    Gamma_hat (n,3,3,3), fext (n,3) -> (Q, n, 3).
    """
    c = L.C.astype(np.float64)
    geo = -_es("nijk,lj,lk->lni", Gamma_hat, c, c)
    return geo + fext[None, :, :]


def forcing(a0, a1, A2, F, cs2=L.CS2):
    """Discrete forcing term, truncated at third order (Sec. II):

    F_l = w_l ( a0 F_l.H1/cs^2 + a1^i F^j_l H2^ij/cs^4
                + A2^ij F^k_l H3^ijk/(2 cs^6) ).
    a0 (n,), a1 (n,3), A2 (n,3,3), F (Q,n,3) -> (Q, n).
    """
    t0 = a0[None, :] * _es("lni,li->ln", F, L.H1) / cs2
    t1 = _es("ni,lnj,lij->ln", a1, F, L.H2) / cs2 ** 2
    t2 = _es("nij,lnk,lijk->ln", A2, F, L.H3) / (2.0 * cs2 ** 3)
    return L.W[:, None] * (t0 + t1 + t2)


def collide(f, Delta, Gamma_hat, fext, tau, old_forcing=False, cs2=L.CS2, half_force_shift=False):
    """BGK collision with the metric forcing term, one step (Eq. LB, RHS).

    f (Q, n) are the streamed (pre-collision) populations.
    Returns the post-collision populations (Q, n).

    half_force_shift selects a variant that is not the paper's printed
    scheme (Sec. II takes u = sum c f / rho'): the velocity of f^eq and of
    the forcing term is u_s with u_s = u + M(u_s) / (2 rho'), M the forcing
    term's first moment, taken by two fixed-point iterations from u
    (u_1 = u + M(u) / (2 rho'), u_s = u + M(u_1) / (2 rho')), and the
    forcing term is scaled by 1 - 1/(2 tau) -- the usual second-order
    treatment of a force in a discrete-time BGK update.
    """
    rho, u = moments(f)
    F = force_vectors(Gamma_hat, fext)
    c = L.C.astype(np.float64)

    def equilibrium_and_forcing(u):
        a0, a1, a2eq, _ = equilibrium_coefficients(rho, u, Delta, cs2)
        feq = equilibrium(rho, u, Delta, cs2)
        if old_forcing:
            A2 = a2eq
        else:
            # sigma^ij = -(1 - 1/(2 tau)) sum_l c^i c^j (f_l - f^eq_l);  a2 = a2^eq - sigma
            sigma = -(1.0 - 1.0 / (2.0 * tau)) * _es("li,lj,ln->nij", c, c, f - feq)
            A2 = a2eq - sigma
        return feq, forcing(a0, a1, A2, F, cs2)

    feq, Fl = equilibrium_and_forcing(u)
    if not half_force_shift:
        return f - (f - feq) / tau + Fl
    u0 = u
    for _ in range(2):
        u = u0 + 0.5 * _es("li,ln->ni", c, Fl) / rho[:, None]
        feq, Fl = equilibrium_and_forcing(u)
    return f - (f - feq) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fl


# --------------------------------------------------------------------------
# a channel simulation
# --------------------------------------------------------------------------
@dataclass
class Params:
    """Per-run parameters: relaxation time tau, covariant streamwise force G
    (lattice units per step), and the forcing variant."""
    tau: float
    G: float = 0.0
    old_forcing: bool = False
    half_force_shift: bool = False


class Simulation:
    """One channel, state f* (Q, N_cells) in the oracle's velocity order."""

    def __init__(self, ch: Channel, params: Params, geometry=None, stream_map=None):
        self.ch = ch
        self.p = params
        self.geo = geometry if geometry is not None else channel_geometry(ch)
        self.smap = stream_map if stream_map is not None else StreamMap(ch)
        nt = ch.ntheta
        # per-cell fields: rows (i_r, i_3) repeated over theta, or one value
        # per node for a theta-resolved channel
        def cells(a):
            a = np.asarray(a)
            if ch.theta_resolved:
                return a.reshape((ch.ncells,) + a.shape[3:])
            rows = a.reshape((ch.nr, 1, ch.n3) + a.shape[2:])
            return np.broadcast_to(rows, (ch.nr, nt, ch.n3) + a.shape[2:]).reshape(
                (ch.ncells,) + a.shape[2:])
        self.cells = cells
        self.Delta = cells(self.geo["Delta"])
        self.Gamma_hat = cells(self.geo["Gamma_hat"])
        self.fext = params.G * cells(self.geo["fdir"])
        self.sqrtg = cells(self.geo["sqrtg"])
        # wall nodes of the equilibrium-wall channel (end nodes of walled axes)
        self.wall_nodes = np.zeros(ch.ncells, dtype=bool)
        if ch.wall == "equilibrium":
            x = np.stack(np.unravel_index(np.arange(ch.ncells), ch.shape), axis=1)
            for a, w in enumerate(ch.walled):
                if w:
                    self.wall_nodes |= (x[:, a] == 0) | (x[:, a] == ch.shape[a] - 1)
        self.f = None
        self.t = 0

    # initial state -------------------------------------------------------
    def init_fields(self, rho, u):
        """f = f^eq(rho', u) at t = 0 (end of Sec. II). rho (n,), u (n,3)."""
        self.f = equilibrium(np.asarray(rho, float), np.asarray(u, float), self.Delta)
        self.t = 0

    def init_rest(self, u0=None):
        """Uniform density rho = rho' sqrt(g) = 1 (Sec. IV), optional u0."""
        rho = 1.0 / self.sqrtg
        u = np.zeros((self.ch.ncells, 3)) if u0 is None else np.asarray(u0, float)
        self.init_fields(rho, u)

    # stepping --------------------------------------------------------------
    def streamed(self):
        return self.smap.apply(self.f)

    def _collide(self, fs, cells=slice(None)):
        out = collide(fs, self.Delta[cells], self.Gamma_hat[cells], self.fext[cells],
                      self.p.tau, self.p.old_forcing, half_force_shift=self.p.half_force_shift)
        wall = self.wall_nodes[cells]
        if wall.any():  # Dirichlet walls: f^eq(rho', u = 0) of the wall node
            rho, _ = moments(fs[:, wall])
            out[:, wall] = equilibrium(rho, np.zeros((len(rho), 3)), self.Delta[cells][wall])
        return out

    def step(self, n=1):
        for _ in range(n):
            fs = self.smap.apply(self.f)
            self.f = self._collide(fs)
            self.t += 1

    def step_cells(self, cells):
        """Post-collision populations of the next step at the given cells only
        (Q, len(cells)); the state is not changed."""
        cells = np.asarray(cells)
        fs = self.f[self.smap.src_pop[:, cells], self.smap.src_cell[:, cells]]
        return self._collide(fs, cells)

    def macros(self):
        """(rho', u) of the streamed populations: shapes (n,), (n,3)."""
        return moments(self.streamed())
