"""Helpers shared by the GPU tests: build/load the library, translate between
the library's population order and the oracle's, and run both sides on the
same seeded inputs."""
import numpy as np

from oracle import lattice as OL
from oracle.geometry import Channel, channel_geometry
from oracle.lbm import Params, Simulation, StreamMap


def lib():
    from paper_1411_3133_gb300 import build, lbgm
    build.build()
    lbgm.load_library()
    return lbgm


def perm_lib_to_oracle():
    """inv[l_oracle] = l_lib, so f_oracle_order = f_lib[inv]."""
    c, _ = lib().lb_velocity_set()
    return np.array([int(np.flatnonzero((c == OL.C[l]).all(axis=1))[0]) for l in range(41)])


def spec_of(ch: Channel):
    metric = "ellipsoidal_theta" if ch.theta_resolved else ch.metric
    return lib().ChannelSpec(metric, ch.r_inner, ch.r_outer, ch.nr, ch.ntheta, ch.n3, ch.b,
                             ch.periodic3, ch.dtheta_scale, ch.d3_scale, ch.wall)


class Twin:
    """The same channel batch on the GPU (library) and in the oracle.

    params: list of dicts with keys tau, G, old, shift, seed, amp, base
    (shift: the half-force velocity variant, old_forcing 2 of the library).
    """

    def __init__(self, ch: Channel, params, precision="fp64", stream=None):
        L = lib()
        self.ch = ch
        self.params = params
        self.B = len(params)
        self.N = ch.ncells
        self.ctx = L.LBContext(spec_of(ch), batch=self.B, precision=precision, stream=stream)
        self.geo = channel_geometry(ch)
        smap = StreamMap(ch)
        self.sims = [Simulation(ch, Params(p["tau"], p.get("G", 0.0), p.get("old", False),
                                           half_force_shift=p.get("shift", False)),
                                self.geo, smap) for p in params]
        self.lparams = [L.make_params(p["tau"], p.get("G", 0.0), 2 if p.get("shift") else p.get("old", False),
                                      p.get("seed", 0), p.get("amp", 0.0), p.get("base", False))
                        for p in params]

    def init_fields(self, rho, u):
        """rho (B, N), u (B, N, 3) -> both sides start from f^eq(rho, u)."""
        ub = np.ascontiguousarray(np.transpose(u, (0, 2, 1)))
        self.ctx.lb_init_fields(self.lparams, np.ascontiguousarray(rho, dtype=np.float64), ub)
        for b, s in enumerate(self.sims):
            s.init_fields(rho[b], u[b])

    def step(self, n):
        self.ctx.lb_step(n)
        for s in self.sims:
            s.step(n)

    def lib_f(self):
        """Library state in the oracle's population order, (B, 41, N)."""
        return self.ctx.lb_get_populations()[:, perm_lib_to_oracle(), :]

    def lib_macros(self):
        rho, u = self.ctx.lb_macros()
        return rho, np.transpose(u, (0, 2, 1))

    def oracle_macros(self):
        out = [s.macros() for s in self.sims]
        return np.stack([o[0] for o in out]), np.stack([o[1] for o in out])

    def close(self):
        self.ctx.close()


def max_rel(a, b, scale):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / scale)
