"""Seeded synthetic workloads shaped like the paper's channels.

This module holds input generators and workload recipes only, none of the
method's arithmetic; tests feed the same inputs to the CUDA library and to the
CPU oracle.

Velocity noise: u^i(cell) = amp * (2 U - 1) with U = (s >> 11) * 2^-53 and s
the output number k = 3 * cell + i (from 0) of SplitMix64 seeded with `seed`
(Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; the mixing function of Vigna's reference splitmix64.c):
    z = seed + (k + 1) * 0x9E3779B97F4A7C15
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    s = z ^ (z >> 31)            (all arithmetic mod 2^64)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 20241111


def splitmix64_at(seed: int, k: np.ndarray) -> np.ndarray:
    """Output number k (uint64 array, from 0) of SplitMix64 seeded with seed."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k + np.uint64(1)) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def noise_field(seed: int, ncells: int, amp: float) -> np.ndarray:
    """Uniform velocity noise in [-amp, amp), shape (ncells, 3)."""
    k = np.arange(3 * ncells, dtype=np.uint64)
    s = splitmix64_at(seed, k)
    U = (s >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return (amp * (2.0 * U - 1.0)).reshape(ncells, 3)


# ---------------------------------------------------------------------------
# recipes
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    """A batch of instances of one channel geometry."""
    name: str
    metric: str
    r_inner: float
    r_outer: float
    nr: int
    ntheta: int
    n3: int
    precision: str
    taus: list
    deans: list
    b: float = 1.0
    periodic3: bool = True
    dtheta_scale: float = 1.0
    d3_scale: float = 1.0
    noise_amp: float = 1e-4
    seeds: list = field(default_factory=list)
    init_base_flow: bool = False

    @property
    def batch(self):
        return len(self.taus)

    @property
    def ncells(self):
        return self.nr * self.ntheta * self.n3

    def geometry_kwargs(self):
        return dict(metric=self.metric, r_inner=self.r_inner, r_outer=self.r_outer, nr=self.nr,
                    ntheta=self.ntheta, n3=self.n3, b=self.b, periodic3=self.periodic3,
                    dtheta_scale=self.dtheta_scale, d3_scale=self.d3_scale)


def cylinder_single(nr=16, ntheta=4, n3=32, tau=0.8, precision="fp64", eta=0.975):
    """Narrow cylindrical channel, r_i = 1 (Sec. III), eta = r_i / r_o."""
    return Workload("cylinder", "cylindrical", 1.0, 1.0 / eta, nr, ntheta, n3, precision,
                    taus=[tau], deans=[0.0], seeds=[BASE_SEED])


def cylinder_sweep(nr=64, ntheta=4, n3=256, taus=(0.55, 0.6), n_dean=12, de_lo=25.0, de_hi=60.0,
                   precision="fp32", eta=0.975):
    """Dean-number sweep: every (tau, De) pair is one instance of a 64 x 4 x 256
    cylindrical channel (eta = 0.975), started from the laminar profile plus
    +-1e-4 noise; seeds BASE_SEED + instance index."""
    deans = list(np.linspace(de_lo, de_hi, n_dean))
    tt, dd = [], []
    for t in taus:
        for d in deans:
            tt.append(float(t))
            dd.append(float(d))
    return Workload(f"cylinder_sweep_{nr}x{ntheta}x{n3}_b{len(tt)}", "cylindrical", 1.0, 1.0 / eta,
                    nr, ntheta, n3, precision, taus=tt, deans=dd,
                    seeds=[BASE_SEED + i for i in range(len(tt))], init_base_flow=True)


def ellipsoid_cross_section(R2_over_R1=1.0, nr=64, ntheta=4, n3=256, tau=0.55, precision="fp32"):
    """Double-curved channel (Sec. IV.B): R_theta = R1 = r_i b^2 = 1 fixed,
    R_phi = R2 = r_i, width d = R1/40, Delta theta = h/(b r_i), Delta phi =
    h/r_i, walls on r and phi."""
    ri = float(R2_over_R1)
    b = 1.0 / math.sqrt(ri)
    d = 1.0 / 40.0
    return Workload(f"ellipsoid_R2_{R2_over_R1:g}", "ellipsoidal", ri, ri + d, nr, ntheta, n3,
                    precision, taus=[tau], deans=[0.0], b=b, periodic3=False,
                    dtheta_scale=1.0 / (b * ri), d3_scale=1.0 / ri, seeds=[BASE_SEED])


@dataclass
class Instance:
    """One channel of a mixed batch (one context of batch 1)."""
    metric: str
    r_inner: float
    r_outer: float
    nr: int
    ntheta: int
    n3: int
    tau: float
    dean: float
    seed: int
    b: float = 1.0
    periodic3: bool = True
    dtheta_scale: float = 1.0
    d3_scale: float = 1.0
    R2_over_R1: float = 0.0
    noise_amp: float = 1e-4

    @property
    def ncells(self):
        return self.nr * self.ntheta * self.n3

    def geometry_kwargs(self):
        return dict(metric=self.metric, r_inner=self.r_inner, r_outer=self.r_outer, nr=self.nr,
                    ntheta=self.ntheta, n3=self.n3, b=self.b, periodic3=self.periodic3,
                    dtheta_scale=self.dtheta_scale, d3_scale=self.d3_scale)


def mixed_batch(n=128, seed=BASE_SEED, tau=0.55, eta=0.975, ntheta=4, nr_choices=(32, 48, 64),
                n3_lo=128, n3_hi=512, de_lo=20.0, de_hi=150.0, ratio_lo=0.25, ratio_hi=4.0):
    """Mixed sweep of `n` channels: alternately a cylinder (eta = 0.975, as in
    Sec. III) and a double-curved channel (Sec. IV.B recipe of
    ellipsoid_cross_section with R2/R1 log-uniform in [ratio_lo, ratio_hi]);
    N_r uniform over nr_choices, N_3 uniform in [n3_lo, n3_hi], target De
    uniform in [de_lo, de_hi]. Draws come from numpy's PCG64 seeded with
    `seed`; instance i gets noise seed BASE_SEED + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        nr = int(rng.choice(nr_choices))
        n3 = int(rng.integers(n3_lo, n3_hi + 1))
        de = float(rng.uniform(de_lo, de_hi))
        ratio = float(math.exp(rng.uniform(math.log(ratio_lo), math.log(ratio_hi))))
        if i % 2 == 0:
            out.append(Instance("cylindrical", 1.0, 1.0 / eta, nr, ntheta, n3, tau, de, BASE_SEED + i))
        else:
            w = ellipsoid_cross_section(ratio, nr, ntheta, n3, tau)
            out.append(Instance("ellipsoidal", w.r_inner, w.r_outer, nr, ntheta, n3, tau, de,
                                BASE_SEED + i, b=w.b, periodic3=False, dtheta_scale=w.dtheta_scale,
                                d3_scale=w.d3_scale, R2_over_R1=ratio))
    return out


def force_reference_cylinder(inst: Instance):
    """Cylinder whose closed-form force-to-Dean map (lb_force_for_dean) sets
    the drive of `inst`: the instance itself, or for a double-curved channel
    the cylinder of the same streamwise radius R1 = 1, width and N_r."""
    if inst.metric == "cylindrical":
        return dict(metric="cylindrical", r_inner=inst.r_inner, r_outer=inst.r_outer, nr=inst.nr,
                    ntheta=inst.ntheta, n3=inst.n3)
    d = inst.r_outer - inst.r_inner
    return dict(metric="cylindrical", r_inner=1.0, r_outer=1.0 + d, nr=inst.nr, ntheta=inst.ntheta,
                n3=inst.n3)
