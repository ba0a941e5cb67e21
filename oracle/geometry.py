"""Channel geometry: embeddings, metric tensor and Christoffel symbols.

Paper sources
  * Cylindrical coordinates (r, theta, z), Sec. III: metric diag(1, r^2, 1).
  * Ellipsoidal coordinates (r, theta, phi), Sec. IV: the embedding
    x = r a cos(theta) cos(phi), y = r b sin(theta) cos(phi), z = r c sin(phi)
    with a = c = 1.
  * Christoffel symbols of a commuting coordinate basis, Sec. III:
    Gamma^i_jk = 1/2 g^im (d_k g_mj + d_j g_mk - d_m g_jk).
  * Lattice map, Sec. III and IV: Delta r = Delta theta = Delta z = Delta t = h,
    and the rescaled spacings Delta theta = h/(b r_i), Delta phi = h/r_i of the
    cross-sectional study (Sec. IV.B).

How the oracle gets there: the metric is computed from the embedding's
Jacobian, g_ij = dX/dx^i . dX/dx^j, and the Christoffel symbols from the
formula above, with exact first and second derivatives by hyper-dual
(forward-mode) automatic differentiation. The printed closed forms are NOT
used here; the tests compare against them.

Readings (where the paper is silent or ambiguous):
  * Node positions, bounce-back walls: r = r_i + (i_r + 1/2) h, i_r =
    0..N_r-1, so that walls sit halfway between nodes exactly at r_i and r_o
    and d = r_o - r_i = N_r h. The third axis is centred: x3 = (i_3 + 1/2 -
    N_3/2) h in scaled units.
  * Node positions, equilibrium (Dirichlet) walls as in Sec. III: the first
    and last node of a walled axis lie on the walls, r = r_i + i_r h with
    d = (N_r - 1) h; a walled third axis likewise x3 = (i_3 - (N_3 - 1)/2) h.
  * Rescaled spacings: scaled coordinates y^i with x^i = s_i y^i, s = (1,
    dtheta_scale, d3_scale), so that every lattice spacing is h. The chain
    rule through the embedding gives the scaled metric and symbols.
  * Lattice Christoffel symbols: Gamma_hat = h * Gamma (lattice velocities are
    per time step and Delta t = h).
  * The metric is evaluated at theta = 0 for every theta node (quasi-2-D
    channel, periodic in theta). Gamma does not depend on theta for either
    coordinate system.
  * theta-resolved channel (Channel.theta_resolved): the metric is evaluated
    at each theta node, theta = dtheta_scale * (i_theta + 1/2 - N_theta/2) h,
    centred on theta = 0 like the third axis, and the theta axis stays
    periodic (the paper's inlet and outlet are not specified). Off theta = 0
    and with b != 1 the metric has every off-diagonal component (Sec. IV).
  * Body force: constant covariant streamwise component F_theta = G, i.e.
    F^i = g^{i theta} G (the only reading that is a pure theta pressure
    gradient).

Oracle module: test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# hyper-dual numbers: a + b e1 + c e2 + d e1 e2, e1^2 = e2^2 = 0
# --------------------------------------------------------------------------
class HyperDual:
    __slots__ = ("a", "b", "c", "d")

    def __init__(self, a, b=0.0, c=0.0, d=0.0):
        self.a, self.b, self.c, self.d = a, b, c, d

    @staticmethod
    def _lift(x):
        return x if isinstance(x, HyperDual) else HyperDual(x)

    def __add__(self, o):
        o = self._lift(o)
        return HyperDual(self.a + o.a, self.b + o.b, self.c + o.c, self.d + o.d)

    __radd__ = __add__

    def __neg__(self):
        return HyperDual(-self.a, -self.b, -self.c, -self.d)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) - self

    def __mul__(self, o):
        o = self._lift(o)
        return HyperDual(self.a * o.a,
                         self.a * o.b + self.b * o.a,
                         self.a * o.c + self.c * o.a,
                         self.a * o.d + self.b * o.c + self.c * o.b + self.d * o.a)

    __rmul__ = __mul__


def hd_sin(x: HyperDual) -> HyperDual:
    s, c = np.sin(x.a), np.cos(x.a)
    return HyperDual(s, c * x.b, c * x.c, c * x.d - s * x.b * x.c)


def hd_cos(x: HyperDual) -> HyperDual:
    s, c = np.sin(x.a), np.cos(x.a)
    return HyperDual(c, -s * x.b, -s * x.c, -s * x.d - c * x.b * x.c)


# --------------------------------------------------------------------------
# embeddings X(x^1, x^2, x^3) into Euclidean space
# --------------------------------------------------------------------------
def embed_flat(x1, x2, x3, b=1.0):
    """Cartesian channel: walls normal to x^1, flow along x^2."""
    return (x1, x2, x3)


def embed_cylindrical(r, th, z, b=1.0):
    """Cylindrical coordinates (Sec. III)."""
    return (r * hd_cos(th), r * hd_sin(th), z)


def embed_ellipsoidal(r, th, ph, b=1.0):
    """Ellipsoidal coordinates with a = c = 1 (Sec. IV)."""
    return (r * hd_cos(th) * hd_cos(ph),
            r * b * hd_sin(th) * hd_cos(ph),
            r * hd_sin(ph))


EMBEDDINGS = {"flat": embed_flat, "cylindrical": embed_cylindrical,
              "ellipsoidal": embed_ellipsoidal}


def metric_and_christoffel(metric: str, y: np.ndarray, scale=(1.0, 1.0, 1.0), b=1.0):
    """Metric g_ij and Christoffel symbols Gamma^i_jk at points y (P, 3).

    The coordinates are scaled coordinates y with physical x^i = scale_i y^i.
    Returns g (P,3,3), dg (P,3,3,3) with dg[:,k,i,j] = d_k g_ij, and
    Gamma (P,3,3,3) with Gamma[:,i,j,k] = Gamma^i_jk.
    """
    embed = EMBEDDINGS[metric]
    y = np.asarray(y, dtype=np.float64)
    P = y.shape[0]
    J = np.zeros((P, 3, 3))        # J[:, a, j] = d X^a / d y^j
    H = np.zeros((P, 3, 3, 3))     # H[:, a, j, k] = d^2 X^a / d y^j d y^k
    for j in range(3):
        for k in range(3):
            coords = []
            for m in range(3):
                coords.append(HyperDual(scale[m] * y[:, m],
                                        scale[m] * (1.0 if m == j else 0.0),
                                        scale[m] * (1.0 if m == k else 0.0),
                                        0.0))
            X = embed(*coords, b=b)
            for a in range(3):
                Xa = HyperDual._lift(X[a])
                J[:, a, j] = Xa.b * np.ones(P)
                H[:, a, j, k] = Xa.d * np.ones(P)
    # g_ij = sum_a dX^a/dy^i dX^a/dy^j
    g = np.einsum("pai,paj->pij", J, J)
    # d_k g_ij = sum_a (d_i d_k X^a d_j X^a + d_i X^a d_j d_k X^a)
    dg = np.einsum("paik,paj->pkij", H, J) + np.einsum("pai,pajk->pkij", J, H)
    ginv = np.linalg.inv(g)
    # Gamma^i_jk = 1/2 g^im (d_k g_mj + d_j g_mk - d_m g_jk)
    bracket = (np.einsum("pkmj->pmjk", dg) + np.einsum("pjmk->pmjk", dg)
               - np.einsum("pmjk->pmjk", dg))
    Gamma = 0.5 * np.einsum("pim,pmjk->pijk", ginv, bracket)
    return g, dg, Gamma


# --------------------------------------------------------------------------
# a channel on the lattice
# --------------------------------------------------------------------------
@dataclass
class Channel:
    """A channel of N_r x N_theta x N_3 fluid nodes.

    metric        'flat', 'cylindrical' or 'ellipsoidal'
    r_inner/outer wall positions r_i, r_o (x^1 for 'flat')
    b             ellipsoid semi-axis (Sec. IV); ignored otherwise
    periodic3     True: periodic third axis (z or phi); False: walls there too
    dtheta_scale  Delta theta / h   (1 except in Sec. IV.B's rescaling)
    d3_scale      Delta x3 / h
    wall          'bounceback' (walls halfway outside the end nodes) or
                  'equilibrium' (the end nodes are wall nodes held at
                  f^eq(rho', u = 0), Sec. III)
    theta_resolved  False: the metric of theta = 0 at every theta node;
                  True: the metric of each theta node's own theta
    """
    metric: str
    r_inner: float
    r_outer: float
    nr: int
    ntheta: int
    n3: int
    b: float = 1.0
    periodic3: bool = True
    dtheta_scale: float = 1.0
    d3_scale: float = 1.0
    wall: str = "bounceback"
    theta_resolved: bool = False

    @property
    def h(self) -> float:
        if self.wall == "equilibrium":
            return (self.r_outer - self.r_inner) / (self.nr - 1)
        return (self.r_outer - self.r_inner) / self.nr

    @property
    def shape(self):
        return (self.nr, self.ntheta, self.n3)

    @property
    def ncells(self) -> int:
        return self.nr * self.ntheta * self.n3

    @property
    def walled(self):
        """Per axis: True where the axis is bounded by walls."""
        return (True, False, not self.periodic3)

    @property
    def curvature_radius(self) -> float:
        """Streamwise curvature radius of the inner wall: r_i (cylinder),
        r_i b^2 (ellipsoid, Sec. IV); infinite for the flat channel."""
        if self.metric == "cylindrical":
            return self.r_inner
        if self.metric == "ellipsoidal":
            return self.r_inner * self.b ** 2
        return math.inf


def geometry_shape(ch: Channel):
    """Leading axes of the geometric fields: (N_r, N_3) rows, or every node
    (N_r, N_theta, N_3) for a theta-resolved channel."""
    return (ch.nr, ch.ntheta, ch.n3) if ch.theta_resolved else (ch.nr, ch.n3)


def node_coordinates(ch: Channel):
    """Scaled coordinates (y_r, y_theta, y_3) of the geometry's points
    (geometry_shape order, flattened): the (N_r, N_3) node rows at y_theta =
    0, or every node with y_theta = (i_theta + 1/2 - N_theta/2) h."""
    h = ch.h
    ir = np.arange(ch.nr)
    i3 = np.arange(ch.n3)
    if ch.wall == "equilibrium":
        yr = ch.r_inner + ir * h
        y3 = (i3 + 0.5 - ch.n3 / 2.0) * h if ch.periodic3 else (i3 - (ch.n3 - 1) / 2.0) * h
    else:
        yr = ch.r_inner + (ir + 0.5) * h
        y3 = (i3 + 0.5 - ch.n3 / 2.0) * h
    if ch.theta_resolved:
        yt = (np.arange(ch.ntheta) + 0.5 - ch.ntheta / 2.0) * h
        R, T, Y3 = np.meshgrid(yr, yt, y3, indexing="ij")
        return np.stack([R, T, Y3], axis=-1).reshape(-1, 3)
    R, Y3 = np.meshgrid(yr, y3, indexing="ij")
    pts = np.stack([R, np.zeros_like(R), Y3], axis=-1).reshape(-1, 3)
    return pts


def channel_geometry(ch: Channel) -> dict:
    """All per-node geometric fields on the (N_r, N_3) rows (theta-frozen),
    or on every node of a theta-resolved channel.

    Keys (leading axes geometry_shape(ch): (N_r, N_3) or (N_r, N_theta, N_3)):
      g, ginv, Delta (= g^ij - delta^ij), sqrtg     scaled metric
      Gamma_hat  (.., i, j, k) = h * Gamma^i_jk      lattice Christoffels
      fdir       (.., i)      = g^{i theta}          body force per unit G
      speed      sqrt(g_theta theta)                 lattice speed per u^theta
      wA         sqrt(det of the (r, x3) block of the physical metric)
      wOmega     sqrt(g_theta theta) of the physical metric
      r_phys     physical radius of the node
    """
    pts = node_coordinates(ch)
    scale = (1.0, ch.dtheta_scale, ch.d3_scale)
    g, _, Gam = metric_and_christoffel(ch.metric, pts, scale=scale, b=ch.b)
    gp, _, _ = metric_and_christoffel(ch.metric, pts * np.array(scale), b=ch.b)
    ginv = np.linalg.inv(g)
    shp = geometry_shape(ch)
    out = {
        "g": g.reshape(shp + (3, 3)),
        "ginv": ginv.reshape(shp + (3, 3)),
        "Delta": (ginv - np.eye(3)).reshape(shp + (3, 3)),
        "sqrtg": np.sqrt(np.linalg.det(g)).reshape(shp),
        "Gamma_hat": (ch.h * Gam).reshape(shp + (3, 3, 3)),
        "fdir": ginv[:, :, 1].reshape(shp + (3,)),
        "speed": np.sqrt(g[:, 1, 1]).reshape(shp),
        "wA": np.sqrt(gp[:, 0, 0] * gp[:, 2, 2] - gp[:, 0, 2] ** 2).reshape(shp),
        "wOmega": np.sqrt(gp[:, 1, 1]).reshape(shp),
        "r_phys": pts[:, 0].reshape(shp),
    }
    return out
