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
    estimate is noisy near De_c;
  * continuation (continuation_sweep, continue_from): a developed vortex
    starts every Dean number, so decay rates below threshold are measured
    far above the round-off floor and the saturated amplitudes above it
    settle quickly; the bracket and both lines are reported;
  * the double-curved channel carries a secondary flow at every De
    (imperfect bifurcation): De_c is the knee of the mean vorticity curve
    (critical_dean_knee; double_curved_study runs the Sec. IV.A and IV.B
    curvature families).

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
              use_graph: bool = True, capture_at: int = 20_000, init_fields=None) -> SweepResult:
    """One batched run: instance b has tau = taus[b] and target De = deans[b].
    With 2-byte storage the developed laminar state becomes the storage
    reference at step `capture_at` (lb_capture_reference), before the
    vortices have grown out of the noise floor. init_fields (rho (B, N), u
    (B, 3, N)): start from these fields (lb_init_fields, e.g. a surrogate's
    prediction) instead of the laminar profile plus noise."""
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
    if init_fields is None:
        ctx.lb_init(params)
    else:
        ctx.lb_init_fields(params, np.ascontiguousarray(init_fields[0], dtype=np.float64),
                           np.ascontiguousarray(init_fields[1], dtype=np.float64))
    ts, amps, des, vort = [], [], [], []
    t0 = time.perf_counter()
    done = 0
    two_byte = precision in ("fp16_shifted", "bf16_shifted")
    while done < steps:
        n = min(sample_every, steps - done)
        if two_byte and done < capture_at <= done + n:
            ctx.lb_step(capture_at - done)
            ctx.lb_capture_reference()
            ctx.lb_step(done + n - capture_at)
        else:
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


def is_saturated(A, floor, sat_factor=100.0, window=0.2, tol=0.05):
    """True when the amplitude series A (samples in time order) ends above
    sat_factor x the round-off floor and changed by less than tol (relative)
    over its last `window` fraction: the vortex has reached its nonlinear
    amplitude. An instance just above threshold grows slowly (growth rate
    ~ De - De_c) and may still be growing at the end of the run; it is not
    saturated and must not enter the A^2 line."""
    A = np.asarray(A, float)
    A = A[np.isfinite(A)]
    if len(A) < 4:
        return False
    k = max(2, int(round(len(A) * window)))
    tail = A[-k:]
    return bool(tail[-1] > sat_factor * floor and abs(tail[-1] / tail[0] - 1.0) < tol)


def critical_dean_saturation(deans, a_final, floor=None, npoints=4, sat_factor=100.0, saturated=None):
    """De_c from saturated amplitudes: least-squares line A^2 = a (De - De_c)
    through the first `npoints` Dean numbers that saturated -- `saturated` (a
    boolean per instance, e.g. from is_saturated) or, if not given, those whose
    final amplitude exceeds sat_factor x the round-off floor (the median final
    amplitude of the instances that did not grow, if not given). NaN if fewer
    than two."""
    d = np.asarray(deans, float)
    a = np.asarray(a_final, float)
    if floor is None:
        quiet = a[a < 1e-5]
        floor = float(np.median(quiet)) if len(quiet) else 1e-7
    sat = np.asarray(saturated, bool) if saturated is not None else a > sat_factor * floor
    order = np.argsort(d)
    d, a, sat = d[order], a[order], sat[order]
    x, y = d[sat][:npoints], (a[sat] ** 2)[:npoints]
    if len(x) < 2:
        return float("nan")
    slope, icpt = np.polyfit(x, y, 1)
    return float(-icpt / slope) if slope > 0 else float("nan")


def summarize(res: SweepResult):
    """{tau: {"dean": measured De, "a_final": ..., "saturated": ..., "sigma":
    ..., "De_c": ..., "De_c_growth": ...}} from one sweep holding several tau
    values."""
    out = {}
    S = len(res.times)
    for tau in sorted(set(res.taus)):
        idx = [b for b, t in enumerate(res.taus) if t == tau]
        # measured (not target) Dean numbers, laminar phase (first quarter)
        de = np.array([float(np.nanmean(res.dean_measured[: max(2, S // 4), b])) for b in idx])
        a_fin = np.array([float(np.nanmean(res.amp[-max(2, S // 8):, b])) for b in idx])
        quiet = a_fin[a_fin < 1e-5]
        floor = float(np.median(quiet)) if len(quiet) else 1e-7
        sat = np.array([is_saturated(res.amp[:, b], floor) for b in idx])
        sig = res.sigma[idx]
        out[tau] = {"dean": de.tolist(), "a_final": a_fin.tolist(), "saturated": sat.tolist(),
                    "sigma": sig.tolist(),
                    "De_c": critical_dean_saturation(de, a_fin, floor, saturated=sat),
                    "De_c_growth": critical_dean(de, sig)}
    return out


def run_sweep_sequential(spec: L.ChannelSpec, taus, deans, steps: int, sample_every: int = 1000,
                         precision: str = "fp64", seed: int = 20241111, noise_amp: float = 1e-4,
                         use_graph: bool = True) -> SweepResult:
    """The unbatched sweep: instance b runs alone in its own context, one
    after the other, with the same inputs as instance b of run_sweep."""
    import time

    import torch

    parts = []
    t0 = time.perf_counter()
    for b, (tau, de) in enumerate(zip(taus, deans)):
        parts.append(run_sweep(spec, [tau], [de], steps, sample_every, precision, seed + b, noise_amp,
                               use_graph))
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    res = SweepResult(list(deans), list(taus), parts[0].times,
                      np.concatenate([p.amp for p in parts], axis=1),
                      np.concatenate([p.dean_measured for p in parts], axis=1),
                      np.concatenate([p.vorticity for p in parts], axis=1), seconds=sec)
    res.sigma = np.concatenate([p.sigma for p in parts])
    return res


def compare_time_to_critical_dean(steps=300_000, sample_every=2000, modes=None):
    """Wall time and De_c of the 24-instance sweep (64 x 4 x 256 cylinder,
    eta = 0.975, 12 De in [25, 60] x tau in {0.55, 0.6}) run as the plain FP64
    sweep (instances one after another) and as one batched launch per step in
    each storage precision. Returns {mode: {"seconds", "De_c": {tau: ...}, ...}}
    with each mode's speed-up and De_c error against the plain FP64 sweep."""
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / 0.975, 64, 4, 256)
    deans = list(np.linspace(25.0, 60.0, 12))
    taus = [0.55] * 12 + [0.6] * 12
    deans2 = deans + deans
    modes = modes or ["fp64_sequential", "fp64", "fp32", "fp16_shifted", "bf16_shifted"]
    out = {}
    for mode in modes:
        if mode == "fp64_sequential":
            res = run_sweep_sequential(spec, taus, deans2, steps, sample_every, "fp64")
        else:
            res = run_sweep(spec, taus, deans2, steps, sample_every, mode)
        summ = summarize(res)
        out[mode] = {"seconds": res.seconds,
                     "De_c": {str(t): summ[t]["De_c"] for t in summ},
                     "De_c_growth": {str(t): summ[t]["De_c_growth"] for t in summ},
                     "dean": {str(t): summ[t]["dean"] for t in summ},
                     "a_final": {str(t): summ[t]["a_final"] for t in summ},
                     "saturated": {str(t): summ[t]["saturated"] for t in summ},
                     "times": res.times.tolist(), "amp": res.amp.tolist()}
    ref = out.get("fp64_sequential")
    if ref:
        for mode, r in out.items():
            r["speedup_vs_fp64_sequential"] = ref["seconds"] / r["seconds"]
            r["De_c_rel_err_vs_fp64_sequential"] = {
                t: abs(r["De_c"][t] / ref["De_c"][t] - 1.0) for t in r["De_c"]}
    return out


def critical_dean_fixed(res: SweepResult):
    """The estimator of the combined-sweep comparison, one rule for every
    mode: per tau, the A^2 line (critical_dean_saturation, four points)
    through the final amplitudes of the instances is_saturated marks, the
    floor taken as in summarize, against the *target* Dean numbers (the
    force of lb_force_for_dean): a warm-started run has no laminar phase in
    which to measure De, and at eta = 0.975 the laminar flow's measured De
    sits within 0.2 % of the target. {tau: De_c}."""
    out = {}
    S = len(res.times)
    for tau in sorted(set(res.taus)):
        idx = [b for b, t in enumerate(res.taus) if t == tau]
        de = np.array([res.deans[b] for b in idx], float)
        a_fin = np.array([float(np.nanmean(res.amp[-max(2, S // 8):, b])) for b in idx])
        quiet = a_fin[a_fin < 1e-5]
        floor = float(np.median(quiet)) if len(quiet) else 1e-7
        sat = np.array([is_saturated(res.amp[:, b], floor) for b in idx])
        out[tau] = critical_dean_saturation(de, a_fin, floor, saturated=sat)
    return out


def combined_sweep(net_path, steps=300_000, sample_every=2000, precision="fp16_shifted", baseline=True,
                   noise_amp=1e-4, seed=20241111, warm=True):
    """The whole pattern on the narrow-gap sweep (64 x 4 x 256 cylinder, eta
    = 0.975, 12 De in [25, 60] x tau in {0.55, 0.6}): every instance starts
    from the mixed surrogate's prediction (surrogate.predict_mixed of the
    saved network, plus the sweep's seeded noise), all 24 run in one batched
    launch per step (graph replay) in 2-byte storage with the laminar state
    captured as the storage reference at step 20 000, and De_c comes from
    critical_dean_fixed. With baseline, the plain FP64 sweep (instances one
    after another, laminar profile plus noise, the same steps) runs first
    and is estimated by the same rule. Wall times include the surrogate's
    inference, not its training. warm=False starts the batched run from the
    laminar profile plus noise instead (the same run without the surrogate)."""
    import time

    import torch

    from . import surrogate as SG
    from .workloads import Instance, noise_field
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / 0.975, 64, 4, 256)
    deans = list(np.linspace(25.0, 60.0, 12))
    taus = [0.55] * 12 + [0.6] * 12
    deans2 = deans + deans
    out = {"steps": steps, "precision": precision, "estimator": "critical_dean_fixed"}
    if baseline:
        res = run_sweep_sequential(spec, taus, deans2, steps, sample_every, "fp64", seed, noise_amp)
        out["fp64_sequential"] = {"seconds": res.seconds,
                                  "De_c": {str(t): v for t, v in critical_dean_fixed(res).items()},
                                  "De_c_measured_de": {str(t): v["De_c"] for t, v in summarize(res).items()}}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    init = None
    if warm:
        net = SG.load_mixed_net(net_path)
        N = spec.ncells
        rho = np.empty((24, N))
        u = np.empty((24, 3, N))
        for b, (tau, de) in enumerate(zip(taus, deans2)):
            inst = Instance("cylindrical", 1.0, 1 / 0.975, 64, 4, 256, tau, de, seed + b)
            rho[b], u[b] = SG.predict_mixed(net, inst, 4)
            u[b] += noise_field(seed + b, N, noise_amp).T
        net.close()
        init = (rho, u)
    t_inf = time.perf_counter() - t0
    res = run_sweep(spec, taus, deans2, steps, sample_every, precision, seed, noise_amp, init_fields=init)
    total = time.perf_counter() - t0
    out["combined"] = {"seconds": total, "inference_seconds": t_inf, "lb_seconds": res.seconds, "warm": warm,
                       "De_c": {str(t): v for t, v in critical_dean_fixed(res).items()},
                       "a_final": res.amp[-1].tolist()}
    if baseline:
        ref = out["fp64_sequential"]
        out["speedup"] = ref["seconds"] / total
        out["De_c_rel_err"] = {t: out["combined"]["De_c"][t] / ref["De_c"][t] - 1.0 for t in ref["De_c"]}
    return out


def critical_dean_knee(deans, w):
    """De_c of an imperfect bifurcation read off the mean-vorticity curve
    <omega>(De) (Sec. IV: the double-curved channel carries a secondary flow
    at every De, and the paper takes the Dean number where the vorticity
    starts to rise steeply): the De of the largest second derivative
    d^2<omega>/dDe^2 (three-point formula on the sampled, possibly uneven
    grid), refined by the vertex of the parabola through that value and its
    two neighbours. NaN when the largest value sits at either end of the
    range (no knee inside the sweep, e.g. a curve that is still convex at the
    last De) or fewer than five finite samples."""
    d = np.asarray(deans, float)
    w = np.asarray(w, float)
    ok = np.isfinite(d) & np.isfinite(w)
    d, w = d[ok], w[ok]
    order = np.argsort(d)
    d, w = d[order], w[order]
    n = len(d)
    if n < 5:
        return float("nan")
    h1 = d[1:-1] - d[:-2]
    h2 = d[2:] - d[1:-1]
    w2 = 2.0 * (h1 * w[2:] - (h1 + h2) * w[1:-1] + h2 * w[:-2]) / (h1 * h2 * (h1 + h2))
    k = int(np.argmax(w2))
    if k == 0 or k == len(w2) - 1:
        return float("nan")
    x = d[k:k + 3]                      # abscissae of w2[k-1], w2[k], w2[k+1]
    a, b, _ = np.polyfit(x, w2[k - 1:k + 2], 2)
    if a >= 0:
        return float(x[1])
    return float(np.clip(-b / (2.0 * a), x[0], x[2]))


def vortex_cells(u_r, nr, ntheta, n3, rel=0.2, periodic=True, weights=None):
    """Number of Dean cells across the x3 extent of one instance: the sign
    changes of the radial velocity at mid-gap (i_r = nr // 2, averaged over
    theta) along x3, counting only samples whose magnitude exceeds `rel` x
    the largest.

    periodic=True (the cylinder's periodic z): the count wraps around, so a
    2-cell flow (one outward and one inward band of u^r) has two sign
    changes, a 4-cell flow four. periodic=False (walls on x3, the four-wall
    channel): no wrap-around; the return flow runs along the x3 walls, so a
    2-cell flow reads -, +, - (two changes) and a 4-cell flow -, +, -, +, -
    (four). The x3 mean of u^r (the x3-uniform radial drift, not a vortex)
    is removed first, weighted by `weights` along x3 when given (the area
    element of the cross-section).
    u_r: the instance's radial velocity in the field layout of lb_macros
    ([i_r][i_theta][i_3], x3 fastest). 0 for a field without vortices."""
    u = np.asarray(u_r, float).reshape(nr, ntheta, n3)[nr // 2].mean(axis=0)
    w = np.ones(n3) if weights is None else np.asarray(weights, float)
    u = u - (w * u).sum() / w.sum()
    m = np.abs(u).max()
    if not np.isfinite(m) or m == 0.0:
        return 0
    sig = np.sign(u[np.abs(u) > rel * m])
    if len(sig) < 2:
        return 0
    if periodic:
        return int(np.count_nonzero(sig != np.roll(sig, 1)))
    return int(np.count_nonzero(sig[1:] != sig[:-1]))


def first_dean_with_cells(deans, cells, n):
    """Smallest Dean number whose final state has at least n Dean cells
    (vortex_cells), or NaN when none has: the measured onset of the 4- and
    6-cell flows of Sec. IV.B on the sampled Dean numbers."""
    d = np.asarray(deans, float)
    c = np.asarray(cells)
    hit = d[c >= n]
    return float(hit.min()) if hit.size else float("nan")


def decay_rate(t, A, floor, skip_frac=0.25, above=100.0):
    """Slope of ln A over the samples after the first skip_frac of the run that
    lie above `above` x the round-off floor: the decay rate (negative) of a
    vortex below threshold. NaN with fewer than three such samples."""
    t = np.asarray(t, float)
    A = np.asarray(A, float)
    start = int(len(t) * skip_frac)
    t, A = t[start:], A[start:]
    keep = np.isfinite(A) & (A > above * floor)
    if keep.sum() < 3:
        return float("nan")
    return float(np.polyfit(t[keep], np.log(A[keep]), 1)[0])


def critical_dean_decay(deans, sigmas, npoints=4):
    """De_c from decay rates below threshold: the linear stability rate obeys
    sigma ~ (De - De_c) near threshold, so a least-squares line through the
    `npoints` negative rates closest to threshold (largest De) crosses zero
    at De_c. NaN if fewer than two negative rates."""
    d = np.asarray(deans, float)
    s = np.asarray(sigmas, float)
    ok = np.isfinite(d) & np.isfinite(s) & (s < 0)
    d, s = d[ok], s[ok]
    if len(d) < 2:
        return float("nan")
    order = np.argsort(d)[::-1][:npoints]
    slope, icpt = np.polyfit(d[order], s[order], 1)
    return float(-icpt / slope) if slope > 0 else float("nan")


def develop_donor(spec: L.ChannelSpec, tau, donor_dean, donor_steps=400_000, precision="fp32",
                  seed=20241111, noise_amp=1e-4, forcing=0):
    """One instance at donor_dean (above threshold), started from the laminar
    profile plus seeded noise and run donor_steps: returns its populations
    (host FP64, shape (1, Q, N)) and its vortex amplitude. `forcing` is
    lb_params.old_forcing (0 the paper's improved forcing, 2 the half-force
    velocity variant)."""
    desc = spec.desc()
    donor = L.LBContext(spec, batch=1, precision=precision)
    try:
        donor.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
        donor.lb_set_option(L.LB_OPT_CHECK_EVERY, 0)
        donor.lb_init([L.make_params(tau, L.lb_force_for_dean(spec.metric, desc, tau, donor_dean), forcing,
                                     seed, noise_amp, True)])
        donor.lb_step(donor_steps)
        amp = donor.lb_diagnostics()[0]["vortex_amp_x3"]
        return donor.lb_get_populations(), amp
    finally:
        donor.close()


def donor_cells(spec: L.ChannelSpec, f_donor, tau):
    """Dean cells of a donor state (host populations (1, Q, N)): loaded into
    a scratch context, its u^r counted by vortex_cells (periodic x3)."""
    ctx = L.LBContext(spec, batch=1, precision="fp64")
    try:
        ctx.lb_init([L.make_params(tau, 0.0, False, 0, 0.0, False)])
        ctx.lb_set_populations(np.ascontiguousarray(f_donor, dtype=np.float64))
        _, u = ctx.lb_macros()
        return vortex_cells(u[0, 0], spec.nr, spec.ntheta, spec.n3, periodic=bool(spec.periodic3))
    finally:
        ctx.close()


def continue_from(spec: L.ChannelSpec, tau, deans, f_donor, steps=400_000, sample_every=2000,
                  precision="fp32", recapture_every=50_000, forcing=0):
    """Every instance of a batch (one per Dean number, each with its own
    force and, for 2-byte storage, its own laminar reference table) starts
    from the donor populations and runs `steps`. Above threshold the vortex
    settles at its saturated amplitude (A^2 ~ De - De_c); below it decays
    exponentially at a rate ~ De_c - De, far above the round-off floor.
    With 2-byte storage the row means of the state become the storage
    reference every `recapture_every` steps (lb_capture_reference), so the
    stored deviations stay the vortex alone while the mean flow adjusts and
    the slow mass drift accumulates. The round-off floor is the smallest
    final amplitude: the lowest Dean numbers must lie far enough below
    threshold to decay onto it. An instance counts as saturated when it ends
    steady above 10 x that floor.
    Returns {"dean", "a_final", "saturated", "sigma", "De_c_saturation",
    "De_c_decay", "De_c_bracket", "floor", "times", "amp", "seconds"}."""
    import time

    import torch

    desc = spec.desc()
    params = [L.make_params(tau, L.lb_force_for_dean(spec.metric, desc, tau, de), forcing, 0, 0.0, True)
              for de in deans]
    ctx = L.LBContext(spec, batch=len(deans), precision=precision)
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    ctx.lb_set_option(L.LB_OPT_CHECK_EVERY, 0)
    ctx.lb_init(params)
    ctx.lb_set_populations(np.ascontiguousarray(np.repeat(f_donor, len(deans), axis=0)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ts, amps, des = [], [], []
    done = 0
    two_byte = precision in ("fp16_shifted", "bf16_shifted")
    while done < steps:
        n = min(sample_every, steps - done)
        if two_byte and recapture_every and (done + n) // recapture_every > done // recapture_every:
            k = (done + n) // recapture_every * recapture_every - done   # steps up to the capture point
            if k:
                ctx.lb_step(k)
            ctx.lb_capture_reference()
            if n - k:
                ctx.lb_step(n - k)
        else:
            ctx.lb_step(n)
        done += n
        dg = ctx.lb_diagnostics()
        ts.append(done)
        amps.append([x["vortex_amp_x3"] for x in dg])
        des.append([x["dean"] for x in dg])
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ctx.close()
    A = np.array(amps)
    S = len(A)
    de = np.array(des)[-max(2, S // 4):].mean(axis=0)      # the developed flow's Dean number
    a_fin = A[-max(2, S // 8):].mean(axis=0)
    floor = max(1e-14 if precision == "fp64" else 1e-9, float(np.nanmin(a_fin)))
    sat = np.array([is_saturated(A[:, i], floor, sat_factor=10.0) for i in range(A.shape[1])])
    sig = np.array([decay_rate(ts, A[:, i], floor, above=10.0) if not sat[i] else float("nan")
                    for i in range(A.shape[1])])
    return {"dean": de.tolist(), "a_final": a_fin.tolist(), "saturated": sat.tolist(),
            "sigma": sig.tolist(), "times": ts, "amp": A.tolist(), "floor": floor,
            "De_c_saturation": critical_dean_saturation(de, a_fin, floor, saturated=sat),
            "De_c_decay": critical_dean_decay(de, sig),
            "De_c_bracket": dean_bracket(de, sat),
            "seconds": sec}


def dean_bracket(deans, saturated):
    """(largest De that did not saturate below the first saturated one, first
    saturated De): the interval holding De_c; NaN ends when missing."""
    d = np.asarray(deans, float)
    s = np.asarray(saturated, bool)
    order = np.argsort(d)
    d, s = d[order], s[order]
    if not s.any():
        return [float(d[-1]) if len(d) else float("nan"), float("nan")]
    k = int(np.argmax(s))
    return [float(d[k - 1]) if k > 0 else float("nan"), float(d[k])]


def continuation_sweep(spec: L.ChannelSpec, tau, deans, donor_dean, donor_steps=400_000,
                       steps=400_000, sample_every=2000, precision="fp32", seed=20241111,
                       noise_amp=1e-4, forcing=0):
    """De_c of a sharp (supercritical) Dean bifurcation by continuation from
    a developed 2-cell vortex (develop_donor, then continue_from). Adds
    "donor_amp" and the total "seconds" of both phases to continue_from's
    result."""
    import time
    t0 = time.perf_counter()
    f, amp = develop_donor(spec, tau, donor_dean, donor_steps, precision, seed, noise_amp, forcing)
    r = continue_from(spec, tau, deans, f, steps, sample_every, precision, forcing=forcing)
    r["donor_amp"] = amp
    r["seconds"] = time.perf_counter() - t0
    return r


def compare_precisions_continuation(modes=("fp64", "fp32", "fp16_shifted", "bf16_shifted"), tau=0.6,
                                    deans=None, donor_dean=44.0, donor_steps=300_000, steps=500_000,
                                    sample_every=2000):
    """The 64 x 4 x 256 narrow-gap sweep (eta = 0.975) by continuation, one
    batched run per storage precision from the same FP32 donor: De_c per
    precision, its deviation from the FP64 run, and each run's wall time."""
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / 0.975, 64, 4, 256)
    deans = list(np.linspace(35.0, 41.0, 10)) if deans is None else list(deans)
    f, amp = develop_donor(spec, tau, donor_dean, donor_steps, "fp32")
    out = {"donor_amp": amp, "tau": tau, "steps": steps}
    for m in modes:
        r = continue_from(spec, tau, deans, f, steps, sample_every, m)
        out[m] = r
    if "fp64" in out:
        ref = out["fp64"]
        for m in modes:
            for k in ("De_c_saturation", "De_c_decay"):
                out[m][k + "_rel_err"] = out[m][k] / ref[k] - 1.0 if np.isfinite(ref[k]) else float("nan")
            out[m]["speedup_vs_fp64"] = ref["seconds"] / out[m]["seconds"]
    return out


def double_curved_study(cases, deans=None, steps=300_000, sample_every=2000, tau=1.0, eta=0.9,
                        nr=65, ntheta=4, n3=128, noise_amp=1e-4, seed=20241111, precision="fp32",
                        wall="equilibrium", max_speed=0.4, theta_resolved=False):
    """The double-curved channel of Sec. IV: walls at r_i and r_o = r_i / eta
    (the paper's Dirichlet walls by default), periodic in phi over n3 nodes,
    tau = 1, for each case (label, r_i, b): streamwise curvature radius
    R_theta = r_i b^2, cross-sectional radius R_phi = r_i. One context per
    case holds the Dean numbers (force from the cylinder of radius R_theta
    and the same width and N_r, which drops targets whose laminar mean speed
    would exceed max_speed lattice units); one lb_batch steps all cases --
    or, theta_resolved, the metric of each theta node (ntheta of them, one h
    apart, centred on theta = 0) with each context stepped in the plain
    kernel. Per case: measured De, final mean vorticity <omega^theta> and
    vortex amplitude, and De_c read off the vorticity curve
    (critical_dean_knee)."""
    import time

    import torch

    deans = list(np.linspace(14.0, 44.0, 16)) if deans is None else list(deans)
    cs2 = 1.0 - np.sqrt(0.4)
    nu = (tau - 0.5) * cs2
    stream = torch.cuda.Stream()
    ctxs, kept = [], []
    for k, (label, ri, b) in enumerate(cases):
        ro = ri / eta
        spec = L.ChannelSpec("ellipsoidal_theta" if theta_resolved else "ellipsoidal", ri, ro, nr, ntheta, n3,
                             b=b, periodic3=True, wall=wall)
        R = ri * b * b
        d = ro - ri
        des_k = [de for de in deans if de * nu / ((nr - 1) * np.sqrt(d / R)) <= max_speed]
        ref = L.make_desc(R, R + d, nr, ntheta, n3, wall=wall)  # cylinder of the same R_theta
        params = [L.make_params(tau, L.lb_force_for_dean("cylindrical", ref, tau, de), False,
                                seed + 100 * k + i, noise_amp, False) for i, de in enumerate(des_k)]
        ctx = L.LBContext(spec, batch=len(des_k), precision=precision, stream=stream)
        ctx.lb_init(params)
        ctxs.append(ctx)
        kept.append(des_k)
    batch = None if theta_resolved else L.LBBatch(ctxs)
    if batch is not None:
        batch.lb_batch_set_option(L.LB_OPT_USE_GRAPH, 1)
    else:
        for ctx in ctxs:
            ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    amps = [[] for _ in cases]
    vort = [[] for _ in cases]
    des = [[] for _ in cases]
    t0 = time.perf_counter()
    for _ in range(steps // sample_every):
        if batch is not None:
            batch.lb_batch_step(sample_every)
        else:
            for ctx in ctxs:
                ctx.lb_step(sample_every)
        for k, ctx in enumerate(ctxs):
            dg = ctx.lb_diagnostics()
            amps[k].append([x["vortex_amp_x3"] for x in dg])
            vort[k].append([x["mean_vorticity"] for x in dg])
            des[k].append([x["dean"] for x in dg])
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    # Dean cells of the final state of every instance (periodic phi), and
    # its mid-gap radial velocity along phi (theta mean)
    cells, ur_mid = [], []
    for ctx in ctxs:
        _, u = ctx.lb_macros()
        cells.append([vortex_cells(u[i, 0], nr, ntheta, n3, periodic=True) for i in range(u.shape[0])])
        ur_mid.append([u[i, 0].reshape(nr, ntheta, n3)[nr // 2].mean(axis=0).tolist() for i in range(u.shape[0])])
    nodes = sum(c.batch * c.spec.ncells for c in ctxs) if batch is None else batch.lb_batch_nodes()
    out = {"seconds": sec, "steps": steps, "nodes": nodes, "ntheta": ntheta,
           "theta_resolved": theta_resolved, "cases": []}
    for k, (label, ri, b) in enumerate(cases):
        A = np.array(amps[k])
        W = np.array(vort[k])
        S = len(A)
        de = np.array(des[k])[: max(2, S // 4)].mean(axis=0)
        w_fin = W[-max(2, S // 8):].mean(axis=0)
        # still moving at the end of the run: last tenth vs the one before
        k10 = max(2, S // 10)
        drift = np.abs(W[-1] / W[-k10] - 1.0)
        out["cases"].append({"label": label, "r_i": ri, "b": b, "R_theta": ri * b * b, "R_phi": ri,
                             "dean_target": kept[k], "dean": de.tolist(),
                             "vorticity": w_fin.tolist(), "a_final": A[-max(2, S // 8):].mean(axis=0).tolist(),
                             "drift": drift.tolist(),
                             "cells": cells[k], "ur_midgap": ur_mid[k],
                             "De_4cell": first_dean_with_cells(de, cells[k], 4),
                             "De_6cell": first_dean_with_cells(de, cells[k], 6),
                             "De_c": critical_dean_knee(de, w_fin)})
    if batch is not None:
        batch.close()
    for c in ctxs:
        c.close()
    return out


def forcing_comparison(etas=(0.8, 0.9, 0.975), forcings=(0, 1), steps=400_000, sample_every=2000,
                       tau=0.9, n=16, precision="fp32", donor_factors=(1.1, 1.18, 1.26, 1.35)):
    """De_c(eta) of the cylinder (Sec. III: 129 x 1 x 256 nodes with the
    paper's equilibrium walls, L_z / L_r = 2, tau = 0.9) with the improved
    forcing (old_forcing 0: the non-equilibrium stress in the forcing term's
    second-order coefficient) and the old one of the earlier publication
    (old_forcing 1: that coefficient from the equilibrium alone), the
    comparison of Sec. III (Fig. 4). Each pair continues n Dean numbers in
    [0.8, 1.25] x a first guess 36 + 60 (1 - eta) from a donor at the first
    of donor_factors x the guess whose developed state holds exactly two
    Dean cells (donor_cells). Returns one row per (eta, forcing)."""
    import time
    rows = []
    for eta in etas:
        guess = 36.0 + 60.0 * (1.0 - eta)
        deans = list(np.linspace(0.8 * guess, 1.25 * guess, n))
        spec = L.ChannelSpec("cylindrical", 1.0, 1.0 / eta, 129, 1, 256, wall="equilibrium")
        for fo in forcings:
            # the donor must carry the 2-cell vortex: a donor above the second
            # bifurcation (4 cells) continues the 4-cell branch, whose lower
            # end lies above the first threshold
            t0 = time.perf_counter()
            tried = []
            for fac in donor_factors:
                f, amp = develop_donor(spec, tau, fac * guess, steps, precision, forcing=fo)
                cells = donor_cells(spec, f, tau) if amp > 1e-4 else 0
                tried.append({"donor_dean": fac * guess, "amp": amp, "cells": cells})
                if cells == 2:
                    break
            r = continue_from(spec, tau, deans, f, steps, sample_every, precision, forcing=fo)
            r["donor_amp"], r["donor_dean"], r["donors_tried"] = amp, fac * guess, tried
            r["seconds"] = time.perf_counter() - t0
            rows.append({"eta": eta, "old_forcing": fo, "deans_target": deans,
                         **{k: v for k, v in r.items() if k not in ("amp", "times")}})
    return rows


def streamwise_curvature_cases(bs=(0.8, 0.85, 0.9, 0.95, 1.0, 1.05, 1.1, 1.2)):
    """Sec. IV.A: r_i = R_phi = 1 fixed, R_theta = b^2 varied."""
    return [("b=%g" % b, 1.0, b) for b in bs]


def cross_section_curvature_cases(ris=(0.8, 0.9, 1.0, 1.1, 1.2, 1.4, 1.6, 1.8)):
    """Sec. IV.B: R_theta = r_i b^2 = 1 fixed, R_phi = r_i varied."""
    return [("r_i=%g" % ri, ri, 1.0 / np.sqrt(ri)) for ri in ris]


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="time-to-critical-Dean comparison of sweep modes")
    ap.add_argument("--steps", type=int, default=300_000)
    ap.add_argument("--sample-every", type=int, default=2000)
    ap.add_argument("--modes", default="fp64_sequential,fp64,fp32,fp16_shifted,bf16_shifted")
    ap.add_argument("--out", default=None)
    ap.add_argument("--double-curved", action="store_true",
                    help="the Sec. IV studies instead: R_theta = b^2 (r_i = 1) and R_phi = r_i (R_theta = 1)")
    ap.add_argument("--theta-resolved", action="store_true",
                    help="--double-curved: the metric of each theta node (with --ntheta nodes)")
    ap.add_argument("--ntheta", type=int, default=4, help="--double-curved: theta nodes")
    ap.add_argument("--bs", default=None,
                    help="--double-curved: the streamwise-curvature cases only, b values (comma list)")
    ap.add_argument("--dean-range", default=None, help="--double-curved: lo,hi,n of the target Dean numbers")
    ap.add_argument("--continuation", default=None, metavar="ETA",
                    help="De_c of the cylinder of aspect ratio ETA (128 x 1 x 256, tau 0.9, Sec. III) "
                         "by continuation from a developed vortex")
    ap.add_argument("--deans", default="38,53", help="--continuation: lowest,highest target De (16 values)")
    ap.add_argument("--donor", type=float, default=54.0, help="--continuation: the donor's target De")
    ap.add_argument("--forcing", type=int, default=0,
                    help="lb_params.old_forcing for --continuation: 0 the paper's improved forcing, "
                         "2 the half-force velocity variant")
    ap.add_argument("--combined", default=None, metavar="NET",
                    help="the combined sweep (surrogate warm start from the saved network NET, batched, "
                         "2-byte storage) against the plain FP64 sweep")
    ap.add_argument("--no-baseline", action="store_true", help="--combined: skip the FP64 sweep")
    ap.add_argument("--precision", default="fp16_shifted", help="--combined: storage of the batched run")
    ap.add_argument("--cold", action="store_true",
                    help="--combined: start the batched run from the laminar profile (no surrogate)")
    ap.add_argument("--forcing-comparison", action="store_true",
                    help="De_c(eta) at eta 0.8, 0.9, 0.975 with the improved and the old forcing (Sec. III, "
                         "129 x 1 x 256, tau 0.9), by continuation")
    ap.add_argument("--precisions", action="store_true",
                    help="De_c of the 64 x 4 x 256 narrow-gap sweep by continuation in every storage precision")
    a = ap.parse_args()
    L.load_library()
    if a.combined:
        r = combined_sweep(a.combined, steps=a.steps, sample_every=a.sample_every,
                           baseline=not a.no_baseline, precision=a.precision, warm=not a.cold)
        print(json.dumps({k: ({kk: vv for kk, vv in v.items() if kk != "a_final"} if isinstance(v, dict) else v)
                          for k, v in r.items()}, indent=1))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        raise SystemExit(0)
    if a.forcing_comparison:
        rows = forcing_comparison(steps=a.steps, sample_every=a.sample_every)
        for r in rows:
            print("eta %.3f old_forcing %d  De_c %.2f (A^2 line) %.2f (decay line)  bracket %s  donor De %.1f "
                  "(%s)  %.1f s" %
                  (r["eta"], r["old_forcing"], r["De_c_saturation"], r["De_c_decay"], r["De_c_bracket"],
                   r["donor_dean"], r["donors_tried"], r["seconds"]))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(rows, f)
        raise SystemExit(0)
    if a.precisions:
        modes = [m for m in a.modes.split(",") if m != "fp64_sequential"]
        r = compare_precisions_continuation(modes=modes, steps=a.steps,
                                            sample_every=a.sample_every)
        print(json.dumps({m: ({k: v for k, v in x.items() if k not in ("amp", "times")}
                              if isinstance(x, dict) else x) for m, x in r.items()}, indent=1))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        raise SystemExit(0)
    if a.double_curved:
        cases = (streamwise_curvature_cases([float(x) for x in a.bs.split(",")]) if a.bs
                 else streamwise_curvature_cases() + cross_section_curvature_cases())
        deans = None
        if a.dean_range:
            lo, hi, n = a.dean_range.split(",")
            deans = list(np.linspace(float(lo), float(hi), int(n)))
        r = double_curved_study(cases, deans=deans, steps=a.steps, sample_every=a.sample_every,
                                ntheta=a.ntheta, theta_resolved=a.theta_resolved)
        for c in r["cases"]:
            print("%-10s R_theta %.3f R_phi %.2f De_c %.2f  4-cell from De %.1f  6-cell from De %.1f  "
                  "cells %s  max drift %.3f" %
                  (c["label"], c["R_theta"], c["R_phi"], c["De_c"], c["De_4cell"], c["De_6cell"],
                   c["cells"], max(c["drift"])))
        print("seconds %.1f  nodes %d" % (r["seconds"], r["nodes"]))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        raise SystemExit(0)
    if a.continuation:
        eta = float(a.continuation)
        spec = L.ChannelSpec("cylindrical", 1.0, 1.0 / eta, 129, 1, 256, wall="equilibrium")
        lo, hi = (float(x) for x in a.deans.split(","))
        r = continuation_sweep(spec, 0.9, list(np.linspace(lo, hi, 16)), donor_dean=a.donor,
                               donor_steps=a.steps, steps=a.steps, sample_every=a.sample_every,
                               forcing=a.forcing)
        print(json.dumps({k: v for k, v in r.items() if k not in ("amp", "times")}, indent=1))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        raise SystemExit(0)
    r = compare_time_to_critical_dean(a.steps, a.sample_every, a.modes.split(","))
    text = json.dumps(r)
    print(json.dumps({m: {k: v for k, v in x.items() if k not in ("amp", "times")} for m, x in r.items()},
                     indent=1))
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
