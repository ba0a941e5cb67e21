"""Dean-number sweeps and the critical Dean number.

Paper: the bifurcation from curved channel Poiseuille flow to Dean vortex
flow is located by varying the driving force (Sec. III; Sec. IV for the
double-curved channel); Dean's narrow-gap critical value is De_c ~ 36
(Introduction). The paper reads De_c off the rise of the mean vorticity.
Here:

  * every instance of a batch is one Dean number (force from
    lb_force_for_dean), started from the laminar profile plus seeded noise;
  * every `sample_every` steps the library reduces the observables on the GPU
    (lb_diagnostics) and the amplitude A(t) = rms of u^r minus its x3 mean is
    recorded (the x3-uniform part of u^r is not a vortex); the Dean number
    reported is the one measured from <v_theta> in the laminar phase;
  * primary estimate: the bifurcation is supercritical, so the saturated
    amplitude obeys A^2 ~ (De - De_c) just above threshold; a straight line
    through A_sat^2(De) of the first saturated Dean numbers crosses zero at
    De_c;
  * secondary: sigma = slope of ln A(t) over the window where the leading
    mode dominates and the amplitude is still small; the first sign change of
    sigma(De). Below threshold A sits on the FP32 round-off floor, so this
    estimate is noisy near De_c.

All stepping and reductions run in the CUDA library; this module only
orchestrates calls and fits a straight line.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import lbgm as L


@dataclass
class SweepResult:
    deans: list                      # target Dean numbers
    taus: list
    times: np.ndarray                # (S,) step counts of the samples
    amp: np.ndarray                  # (S, B) vortex amplitudes
    dean_measured: np.ndarray        # (S, B)
    vorticity: np.ndarray            # (S, B)
    sigma: np.ndarray = field(default=None)   # (B,) growth rates per step
    seconds: float = 0.0


def growth_rate(t, A, skip_frac=0.3, grow_cap=1e3, sat_frac=0.01):
    """Slope of ln A over the linear window: after the first skip_frac of the
    run, and, for a growing mode, from its minimum only up to where A has grown
    grow_cap times or reached sat_frac of its largest value (before
    saturation)."""
    t = np.asarray(t, float)
    A = np.asarray(A, float)
    ok = np.isfinite(A) & (A > 0)
    t, A = t[ok], A[ok]
    start = int(len(t) * skip_frac)
    t, A = t[start:], A[start:]
    if len(t) < 3:
        return float("nan")
    i0 = int(np.argmin(A))
    if A[-1] > A[i0] * 10:                      # growing: fit from the minimum
        t, A = t[i0:], A[i0:]
        keep = A <= min(A[0] * grow_cap, sat_frac * A.max())
        t, A = t[keep], A[keep]
    if len(t) < 3:
        return float("nan")
    return float(np.polyfit(t, np.log(A), 1)[0])


def critical_dean(deans, sigmas):
    """First De where sigma changes sign from negative to positive, by linear
    interpolation between the bracketing samples (NaN if none)."""
    d = np.asarray(deans, float)
    s = np.asarray(sigmas, float)
    order = np.argsort(d)
    d, s = d[order], s[order]
    for i in range(len(d) - 1):
        if np.isfinite(s[i]) and np.isfinite(s[i + 1]) and s[i] < 0 <= s[i + 1]:
            return float(d[i] - s[i] * (d[i + 1] - d[i]) / (s[i + 1] - s[i]))
    return float("nan")


def run_sweep(spec: L.ChannelSpec, taus, deans, steps: int, sample_every: int = 1000,
              precision: str = "fp32", seed: int = 20241111, noise_amp: float = 1e-4,
              use_graph: bool = True) -> SweepResult:
    """One batched run: instance b has tau = taus[b] and target De = deans[b]."""
    import time

    import torch

    assert len(taus) == len(deans)
    desc = spec.desc()
    params = []
    for b, (tau, de) in enumerate(zip(taus, deans)):
        G = L.lb_force_for_dean(spec.metric, desc, tau, de)
        params.append(L.make_params(tau, G, False, seed + b, noise_amp, True))
    ctx = L.LBContext(spec, batch=len(taus), precision=precision)
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, int(use_graph))
    ctx.lb_set_option(L.LB_OPT_CHECK_EVERY, 0)
    ctx.lb_init(params)
    ts, amps, des, vort = [], [], [], []
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        n = min(sample_every, steps - done)
        ctx.lb_step(n)
        done += n
        d = ctx.lb_diagnostics()
        ts.append(done)
        amps.append([x["vortex_amp_x3"] for x in d])
        des.append([x["dean"] for x in d])
        vort.append([x["mean_vorticity"] for x in d])
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ctx.close()
    res = SweepResult(list(deans), list(taus), np.array(ts), np.array(amps), np.array(des),
                      np.array(vort), seconds=sec)
    res.sigma = np.array([growth_rate(res.times, res.amp[:, b]) for b in range(len(taus))])
    return res


def mixed_contexts(instances, precision="fp32", stream=None, init=True):
    """One context (batch 1) per workloads.Instance, all on one stream, and
    the lb_batch over them. Instances start from rest (rho' = 1/sqrt(g)) plus
    their seeded noise, driven by the force of the target Dean number (the
    closed form of the cylinder named by workloads.force_reference_cylinder).
    Returns (contexts, batch)."""
    import torch

    from .workloads import force_reference_cylinder

    stream = stream if stream is not None else torch.cuda.Stream()
    ctxs = []
    for inst in instances:
        spec = L.ChannelSpec(**inst.geometry_kwargs())
        ctx = L.LBContext(spec, batch=1, precision=precision, stream=stream)
        if init:
            ref = force_reference_cylinder(inst)
            rdesc = L.make_desc(ref["r_inner"], ref["r_outer"], ref["nr"], ref["ntheta"], ref["n3"])
            G = L.lb_force_for_dean("cylindrical", rdesc, inst.tau, inst.dean)
            ctx.lb_init([L.make_params(inst.tau, G, False, inst.seed, inst.noise_amp, False)])
        ctxs.append(ctx)
    return ctxs, L.LBBatch(ctxs)


def critical_dean_saturation(deans, a_final, floor=None, npoints=4, sat_factor=100.0):
    """De_c from saturated amplitudes: least-squares line A^2 = a (De - De_c)
    through the first `npoints` Dean numbers whose final amplitude exceeds
    sat_factor x the round-off floor (the median final amplitude of the
    instances that did not grow, if not given). NaN if fewer than two."""
    d = np.asarray(deans, float)
    a = np.asarray(a_final, float)
    order = np.argsort(d)
    d, a = d[order], a[order]
    if floor is None:
        quiet = a[a < 1e-5]
        floor = float(np.median(quiet)) if len(quiet) else 1e-7
    sat = a > sat_factor * floor
    x, y = d[sat][:npoints], (a[sat] ** 2)[:npoints]
    if len(x) < 2:
        return float("nan")
    slope, icpt = np.polyfit(x, y, 1)
    return float(-icpt / slope) if slope > 0 else float("nan")


def summarize(res: SweepResult):
    """{tau: {"dean": measured De, "a_final": ..., "sigma": ..., "De_c": ...,
    "De_c_growth": ...}} from one sweep holding several tau values."""
    out = {}
    S = len(res.times)
    for tau in sorted(set(res.taus)):
        idx = [b for b, t in enumerate(res.taus) if t == tau]
        # measured (not target) Dean numbers, laminar phase (first quarter)
        de = np.array([float(np.nanmean(res.dean_measured[: max(2, S // 4), b])) for b in idx])
        a_fin = np.array([float(np.nanmean(res.amp[-max(2, S // 8):, b])) for b in idx])
        sig = res.sigma[idx]
        out[tau] = {"dean": de.tolist(), "a_final": a_fin.tolist(), "sigma": sig.tolist(),
                    "De_c": critical_dean_saturation(de, a_fin),
                    "De_c_growth": critical_dean(de, sig)}
    return out
