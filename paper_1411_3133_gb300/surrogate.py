"""Surrogate warm start of Dean-vortex runs.

A small network (lb_mlp, include/lbgm.h) learns the developed flow of a
curved channel -- laminar below the critical Dean number, Dean vortices
above it (Sec. III) -- from converged runs of the library itself, and
initialises new runs (lb_init_fields) close to their end state. The LB
still runs every instance to convergence, so the surrogate only changes how
many steps that takes, never the answer; its error is measured against the
converged LB fields.

Pipeline (all stepping, reductions and network arithmetic in the library's
kernels; this module orchestrates and rearranges arrays):
  1. `converge`: a batch of cylinder channels (one context), each at its own
     Dean number, stepped until max |u(t) - u(t - K)| <= r K max |u| (per-step
     residual r, lb_velocity_change) or a step cap;
  2. `align_phase`: the x3 position of Dean vortices is set by the seeded
     noise, so every converged field is shifted along the periodic x3 axis to
     put the phase of the first x3 Fourier mode of u^r at zero; the network
     learns this canonical phase;
  3. `train`: inputs (De / 100, (i_r + 1/2) / N_r, (i_3 + 1/2) / N_3), outputs
     the theta-averaged (rho', u^r, u^theta, u^3), Adam on minibatches;
  4. held-out Dean numbers run twice for the same number of steps -- from
     the laminar profile plus noise (as a sweep starts) and from the network's
     prediction -- reporting the steps each needed until the vortex amplitude
     stays within 2 % of its developed value, and the prediction's error
     against the developed field. (A velocity-residual test alone is fooled
     by the slow exponential growth of a supercritical vortex from noise:
     the per-step change is tiny long before the flow has developed.)
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import lbgm as L


def channel(nr=32, ntheta=4, n3=64, eta=0.975):
    """The paper's channel shape L_z = 2 L_r (Sec. III) at N_r = 32."""
    return L.ChannelSpec("cylindrical", 1.0, 1.0 / eta, nr, ntheta, n3)


def converge(spec, deans, tau=0.6, tol=1e-8, check_every=2000, max_steps=400_000, seed=20241111,
             init_fields=None, precision="fp32", noise_amp=1e-4):
    """Run every Dean number to a per-step residual <= tol (or max_steps).

    init_fields: None (laminar profile + seeded noise) or (rho (B, N), u (B, 3, N))
    host arrays for lb_init_fields. Returns (rho (B, N), u (B, 3, N), steps (B,),
    converged (B,) bool, seconds)."""
    import torch
    B, N = len(deans), spec.ncells
    desc = spec.desc()
    params = [L.make_params(tau, L.lb_force_for_dean(spec.metric, desc, tau, float(de)), False,
                            seed + b, noise_amp, init_fields is None) for b, de in enumerate(deans)]
    ctx = L.LBContext(spec, batch=B, precision=precision)
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    if init_fields is None:
        ctx.lb_init(params)
    else:
        rho0, u0 = init_fields
        ctx.lb_init_fields(params, np.ascontiguousarray(rho0, dtype=np.float64),
                           np.ascontiguousarray(u0, dtype=np.float64))
    u_prev = torch.empty(B * 3 * N, dtype=torch.float64, device="cuda")
    ctx.lb_macros(None, u_prev, on_device=True)
    steps = np.full(B, max_steps)
    done = np.zeros(B, dtype=bool)
    t0 = time.perf_counter()
    t = 0
    while t < max_steps and not done.all():
        ctx.lb_step(check_every)
        t += check_every
        change, umax = ctx.lb_velocity_change(u_prev)
        now = (change <= tol * check_every * np.maximum(umax, 1e-300)) & ~done
        steps[now] = t
        done |= now
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    rho, u = ctx.lb_macros()
    ctx.close()
    return rho, u, steps, done, sec


def trajectory(spec, deans, steps, sample_every=2000, tau=0.55, seed=20241111, init_fields=None,
               precision="fp32", noise_amp=1e-4):
    """Run every Dean number for `steps` steps, sampling the vortex amplitude
    (lb_diagnostics' rms of u^r minus its x3 mean) every `sample_every`.
    Returns (times (S,), amplitudes (S, B), rho (B, N), u (B, 3, N), seconds)."""
    import torch
    B = len(deans)
    desc = spec.desc()
    params = [L.make_params(tau, L.lb_force_for_dean(spec.metric, desc, tau, float(de)), False,
                            seed + b, noise_amp, init_fields is None) for b, de in enumerate(deans)]
    ctx = L.LBContext(spec, batch=B, precision=precision)
    ctx.lb_set_option(L.LB_OPT_USE_GRAPH, 1)
    if init_fields is None:
        ctx.lb_init(params)
    else:
        ctx.lb_init_fields(params, np.ascontiguousarray(init_fields[0], dtype=np.float64),
                           np.ascontiguousarray(init_fields[1], dtype=np.float64))
    ts, amps = [], []
    t0 = time.perf_counter()
    for t in range(sample_every, steps + 1, sample_every):
        ctx.lb_step(sample_every)
        ts.append(t)
        amps.append([d["vortex_amp_x3"] for d in ctx.lb_diagnostics()])
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    rho, u = ctx.lb_macros()
    ctx.close()
    return np.array(ts), np.array(amps), rho, u, sec


def steps_to_developed(times, amps, a_final, rel=0.02, floor=1e-6):
    """Per instance: the first sample time from which the amplitude stays
    within rel * a_final (+ floor) of its developed value a_final."""
    out = np.empty(amps.shape[1])
    for b in range(amps.shape[1]):
        ok = np.abs(amps[:, b] - a_final[b]) <= rel * a_final[b] + floor
        bad = np.flatnonzero(~ok)
        out[b] = times[0] if len(bad) == 0 else (times[bad[-1] + 1] if bad[-1] + 1 < len(times) else np.inf)
    return out


def theta_mean(spec, a):
    """(B, N) or (B, 3, N) node arrays -> (B, [3,] N_r, N_3) theta averages."""
    a = np.asarray(a)
    shp = a.shape[:-1] + (spec.nr, spec.ntheta, spec.n3)
    return a.reshape(shp).mean(axis=-2)


def align_phase(rho, u):
    """Shift each instance's (N_r, N_3) fields along x3 so that the first x3
    Fourier mode of u^r, summed over r, has phase zero. rho (B, nr, n3),
    u (B, 3, nr, n3)."""
    n3 = rho.shape[-1]
    out_r, out_u = rho.copy(), u.copy()
    k = np.arange(n3)
    for b in range(len(rho)):
        c = (u[b, 0] * np.exp(-2j * np.pi * k / n3)[None, :]).sum()
        if not np.isfinite(c) or abs(c) < 1e-12 * max(1e-300, np.abs(u[b, 0]).max() * u[b, 0].size):
            continue                                      # no vortex: nothing to align
        # a field f(k) = F(k - s) has c ~ exp(-2 pi i s / n3); rolling by
        # angle(c) n3 / (2 pi) = -s brings it to F(k)
        shift = int(round(np.angle(c) / (2 * np.pi) * n3)) % n3
        out_r[b] = np.roll(rho[b], shift, axis=-1)
        out_u[b] = np.roll(u[b], shift, axis=-1)
    return out_r, out_u


def inputs(spec, deans):
    """Network inputs (B * nr * n3, 3) on the (r, x3) grid, rows ordered
    instance, i_r, i_3."""
    r = (np.arange(spec.nr) + 0.5) / spec.nr
    z = (np.arange(spec.n3) + 0.5) / spec.n3
    R, Z = np.meshgrid(r, z, indexing="ij")
    x = []
    for de in deans:
        x.append(np.stack([np.full(R.size, de / 100.0), R.ravel(), Z.ravel()], axis=1))
    return np.concatenate(x).astype(np.float32)


def targets(rho, u):
    """(B, nr, n3) and (B, 3, nr, n3) -> (B * nr * n3, 4)."""
    B = rho.shape[0]
    y = np.concatenate([rho[:, None], u], axis=1)          # (B, 4, nr, n3)
    return np.moveaxis(y, 1, -1).reshape(B * rho.shape[1] * rho.shape[2], 4).astype(np.float32)


def train(x, y, epochs=30, batch=16384, lr=2e-3, seed=20241111, width=256, depth=5, n_fourier=4, log=None):
    """Fit an LBMlp to (x, y); returns (net, losses per epoch)."""
    import torch
    net = L.LBMlp(n_fourier=n_fourier, width=width, depth=depth, max_batch=batch, seed=seed)
    net.set_output_scale(y.mean(axis=0), np.maximum(y.std(axis=0), 1e-12))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    n = len(x)
    g = torch.Generator(device="cuda").manual_seed(seed)
    losses = []
    for ep in range(epochs):
        step_lr = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))   # cosine schedule
        perm = torch.randperm(n, device="cuda", generator=g)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            last = s + 2 * batch > n
            loss = net.train_step(xd[idx].contiguous(), yd[idx].contiguous(), step_lr, want_loss=last)
            if last:
                tot, cnt = loss, 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep} loss {losses[-1]:.3e}")
    return net, losses


def predict_fields(net, spec, deans):
    """Network fields broadcast over theta: rho (B, N), u (B, 3, N)."""
    import torch
    x = torch.from_numpy(inputs(spec, deans)).cuda()
    y = np.concatenate([net.predict(x[s:s + net.max_batch]).cpu().numpy()
                        for s in range(0, len(x), net.max_batch)])
    B = len(deans)
    y = y.reshape(B, spec.nr, 1, spec.n3, 4)
    y = np.broadcast_to(y, (B, spec.nr, spec.ntheta, spec.n3, 4)).reshape(B, -1, 4)
    return y[..., 0].copy(), np.moveaxis(y[..., 1:], -1, 1).copy()


def field_error(spec, u_pred, u_ref):
    """Relative L2 error of the theta-averaged velocity after phase alignment."""
    rp = np.zeros((len(u_pred), spec.nr, spec.n3))
    _, a = align_phase(rp, theta_mean(spec, u_pred))
    _, b = align_phase(rp, theta_mean(spec, u_ref))
    err = np.sqrt(((a - b) ** 2).sum(axis=(1, 2, 3))) / np.sqrt((b ** 2).sum(axis=(1, 2, 3)))
    return err


def run(n_train=512, n_test=128, de_lo=20.0, de_hi=60.0, tau=0.55, chunk=512, tol=None, max_steps=400_000,
        epochs=40, batch=4096, seed=20241111, log=print):
    """The whole pipeline; returns a report dict. (At N_r = 32 the laminar
    mean speed is De nu / (N_r sqrt(d / r_i)): tau = 0.55 keeps it below
    0.22 up to De = 60.)"""
    spec = channel()
    rng = np.random.default_rng(seed)
    de_train = rng.uniform(de_lo, de_hi, n_train)
    de_test = rng.uniform(de_lo, de_hi, n_test)
    rep = {"channel": f"cylinder {spec.nr}x{spec.ntheta}x{spec.n3}, eta 0.975, tau {tau}",
           "steps_per_run": max_steps, "n_train": n_train, "n_test": n_test,
           "dean_range": [de_lo, de_hi],
           "developed": "vortex amplitude within 2 % (+1e-6) of the cold run's final value, to the end"}
    # 1. developed training states: a fixed number of steps (a residual test
    # alone would stop supercritical runs before their vortices have grown)
    t0 = time.perf_counter()
    R, U, OK = [], [], []
    for s in range(0, n_train, chunk):
        _, amps, rho, u, sec = trajectory(spec, de_train[s:s + chunk], max_steps, tau=tau, seed=seed + s)
        R.append(rho)
        U.append(u)
        OK.append(np.isfinite(rho).all(axis=1) & np.isfinite(u).all(axis=(1, 2)))
        log(f"train states {s}..{s + len(rho)}: {sec:.1f} s")
    keep = np.concatenate(OK)
    rho, u = align_phase(theta_mean(spec, np.concatenate(R)[keep]), theta_mean(spec, np.concatenate(U)[keep]))
    rep["train_generation_s"] = time.perf_counter() - t0
    rep["train_states_used"] = int(keep.sum())
    # 2. training
    t0 = time.perf_counter()
    net, losses = train(inputs(spec, de_train[keep]), targets(rho, u), epochs=epochs, batch=batch, seed=seed,
                        log=log)
    rep["train_s"] = time.perf_counter() - t0
    rep["loss_first_last"] = [losses[0], losses[-1]]
    # 3. held-out: cold (laminar + noise) and warm (network) starts, both run
    # for max_steps; the developed amplitude is the cold run's final one
    tc, ac, rho_c, u_c, sec_c = trajectory(spec, de_test, max_steps, tau=tau, seed=seed + 7)
    rho_p, u_p = predict_fields(net, spec, de_test)
    tw, aw, rho_w, u_w, sec_w = trajectory(spec, de_test, max_steps, tau=tau, seed=seed + 7,
                                           init_fields=(rho_p, u_p))
    a_fin = ac[-max(2, len(tc) // 20):].mean(axis=0)
    sc = steps_to_developed(tc, ac, a_fin)
    sw = steps_to_developed(tw, aw, a_fin)
    sup = a_fin > 1e-5
    err_pred = field_error(spec, u_p, u_c)
    err_final = field_error(spec, u_w, u_c)
    fin = np.isfinite(sc) & np.isfinite(sw)
    rep.update({
        "test_deans": de_test.tolist(), "a_final": a_fin.tolist(),
        "steps_cold": sc.tolist(), "steps_warm": sw.tolist(),
        "seconds_each_run": [sec_c, sec_w],
        "supercritical_fraction": float(sup.mean()),
        "supercritical_mean_steps_cold": float(np.mean(sc[sup & fin])) if (sup & fin).any() else None,
        "supercritical_mean_steps_warm": float(np.mean(sw[sup & fin])) if (sup & fin).any() else None,
        "subcritical_mean_steps_cold": float(np.mean(sc[~sup & fin])) if (~sup & fin).any() else None,
        "subcritical_mean_steps_warm": float(np.mean(sw[~sup & fin])) if (~sup & fin).any() else None,
        "mean_steps_saved": float(np.mean((sc - sw)[fin])),
        "surrogate_rel_l2_error_median": float(np.median(err_pred)),
        "surrogate_rel_l2_error_p90": float(np.percentile(err_pred, 90)),
        "warm_vs_cold_final_rel_l2_median": float(np.median(err_final)),
        "warm_vs_cold_final_rel_l2_max": float(np.max(err_final)),
    })
    net.close()
    return rep


# ---------------------------------------------------------------------------
# the mixed-channel surrogate: cylinders and double-curved channels
# ---------------------------------------------------------------------------
NU_055 = (0.55 - 0.5) * (1.0 - math.sqrt(0.4))     # lattice viscosity at tau = 0.55
N_PLAIN_MIXED = 6                                 # De, kind, curvature, aspect, r, theta (then z)
N_FOURIER_MIXED = 12                              # up to 12 x3 periods: 2 N_3 / N_r <= 32 cells


def laminar_speed(inst):
    """Mean streamwise speed (lattice units) of a channel of workloads.Instance
    inst at its target Dean number, from the Dean number's definition
    (Sec. III / IV: De = <v> (d / h) / nu sqrt(d / R_theta)) with R_theta = 1
    for both kinds and d / h = N_r (bounce-back walls)."""
    d = inst.r_outer - inst.r_inner
    nu = (inst.tau - 0.5) * (1.0 - math.sqrt(0.4))
    return inst.dean * nu / (inst.nr * math.sqrt(d / 1.0))


def draw_mixed(n, seed, speed_cap=0.25):
    """n instances of the mixed-batch distribution (workloads.mixed_batch:
    alternately cylinder and double-curved, N_r in {32, 48, 64}, N_3 in
    128..512, De in 20..150, R2/R1 log-uniform in 0.25..4, tau 0.55), keeping
    only draws whose laminar mean speed stays <= speed_cap (a converged state
    at De = 150 and N_r = 32 would run at Mach ~ 0.9)."""
    from .workloads import mixed_batch
    out, k = [], 0
    while len(out) < n:
        for inst in mixed_batch(n=256, seed=seed + 7919 * k):
            if laminar_speed(inst) <= speed_cap:
                out.append(inst)
        k += 1
    return out[:n]


def mixed_inputs(inst, nr, n3, ntheta=1):
    """Network inputs of every (i_r, i_3) node of inst, rows i_r-major:
    (De / 150, kind (0 cylinder, 1 double-curved), log2(R2/R1) / 2 (0 for a
    cylinder, whose R2 is infinite), aspect N_3 / N_r / 16, (i_r + 1/2) / N_r,
    theta = 1/2 (the fields are theta-uniform), then z = (i_3 + 1/2) / N_3)."""
    ell = inst.metric == "ellipsoidal"
    r = (np.arange(nr) + 0.5) / nr
    z = (np.arange(n3) + 0.5) / n3
    R, Z = np.meshgrid(r, z, indexing="ij")
    m = R.size
    cols = [np.full(m, inst.dean / 150.0), np.full(m, 1.0 if ell else 0.0),
            np.full(m, math.log2(inst.R2_over_R1) / 2.0 if ell else 0.0), np.full(m, n3 / nr / 16.0),
            R.ravel(), np.full(m, 0.5), Z.ravel()]
    return np.stack(cols, axis=1).astype(np.float32)


def _spec(inst, ntheta):
    kw = inst.geometry_kwargs()
    kw["ntheta"] = ntheta
    return L.ChannelSpec(**kw)


def _sqrtg(inst):
    desc = _spec(inst, 1).desc()
    return L.lb_geometry_eval(inst.metric, desc)[:, :, 39]      # (nr, n3): sqrt g of the lattice metric


def mixed_targets(inst, rho, u):
    """Normalised targets of one converged instance: rho' sqrt(g) (about 1)
    and u / U (U = laminar_speed), theta-averaged; rho (nr, n3), u (3, nr, n3)
    -> (nr * n3, 4)."""
    U = laminar_speed(inst)
    y = np.concatenate([(rho * _sqrtg(inst))[None], u / U], axis=0)
    return np.moveaxis(y, 0, -1).reshape(-1, 4).astype(np.float32)


def mixed_fields(inst, y, ntheta):
    """Network outputs (nr * n3, 4) of one instance back to fields broadcast
    over theta: rho (N,), u (3, N) in the field layout of lb_init_fields."""
    nr, n3 = inst.nr, inst.n3
    y = np.asarray(y, np.float64).reshape(nr, n3, 4)
    rho = y[..., 0] / _sqrtg(inst)
    u = np.moveaxis(y[..., 1:], -1, 0) * laminar_speed(inst)
    rho = np.broadcast_to(rho[:, None, :], (nr, ntheta, n3)).reshape(-1)
    u = np.broadcast_to(u[:, :, None, :], (3, nr, ntheta, n3)).reshape(3, -1)
    return np.ascontiguousarray(rho), np.ascontiguousarray(u)


def align_mixed(inst, rho, u):
    """Phase alignment of a periodic channel's fields (the cylinders': the
    vortex position along z is set by the noise) on the dominant x3 Fourier
    mode of u^r; walled channels are returned unchanged. rho (nr, n3), u (3,
    nr, n3)."""
    if inst.periodic3:
        n3 = rho.shape[-1]
        F = np.abs(np.fft.rfft(u[0].sum(axis=0)))
        k = int(np.argmax(F[1:]) + 1) if len(F) > 1 else 1
        c = (u[0] * np.exp(-2j * np.pi * k * np.arange(n3) / n3)[None, :]).sum()
        if np.isfinite(c) and abs(c) > 1e-12 * max(1e-300, np.abs(u[0]).max() * u[0].size):
            shift = int(round(np.angle(c) / (2 * np.pi * k) * n3)) % n3
            return np.roll(rho, shift, axis=-1), np.roll(u, shift, axis=-1)
    return rho, u


def converge_mixed(instances, ntheta=1, tol=1e-8, amp_tol=0.01, check_every=10_000, max_steps=600_000,
                   warm=None, stream=None, log=None):
    """Run every instance (one context each, one lb_batch over those still
    running) until it is converged: the per-step velocity residual
    max |u(t) - u(t - K)| / (K max |u|) <= tol (lb_velocity_change, K =
    check_every) and the vortex amplitude (rms u^r minus its x3 mean) within
    amp_tol of its value one and two checks earlier, or below 1e-5 max |u|
    over the last three checks (no vortex: round-off) -- the residual alone
    passes during the slow exponential growth of a vortex from noise. Cold
    start (warm None): rest plus seeded noise, as the mixed sweep starts;
    warm: per instance (rho (N,), u (3, N)) for lb_init_fields.
    Returns (theta-mean rho (list of (nr, n3)), u (list of (3, nr, n3)),
    steps (array), converged (bool array), seconds)."""
    import torch

    from .workloads import force_reference_cylinder
    stream = stream if stream is not None else torch.cuda.Stream()
    ctxs, uprev = [], []
    for k, inst in enumerate(instances):
        spec = _spec(inst, ntheta)
        ref = force_reference_cylinder(inst)
        G = L.lb_force_for_dean("cylindrical", L.make_desc(ref["r_inner"], ref["r_outer"], ref["nr"], 1, ref["n3"]),
                                inst.tau, inst.dean)
        ctx = L.LBContext(spec, batch=1, precision="fp32", stream=stream)
        p = [L.make_params(inst.tau, G, False, inst.seed, inst.noise_amp, False)]
        if warm is None:
            ctx.lb_init(p)
        else:
            ctx.lb_init_fields(p, warm[k][0][None], warm[k][1][None])
        u0 = torch.empty(3 * spec.ncells, dtype=torch.float64, device="cuda")
        ctx.lb_macros(None, u0, on_device=True)
        ctxs.append(ctx)
        uprev.append(u0)
    n = len(instances)
    steps = np.full(n, max_steps)
    done = np.zeros(n, dtype=bool)
    amps = [[] for _ in range(n)]
    t0 = time.perf_counter()
    t = 0
    while t < max_steps and not done.all():
        live = [i for i in range(n) if not done[i]]
        batch = L.LBBatch([ctxs[i] for i in live])
        batch.lb_batch_set_option(L.LB_OPT_USE_GRAPH, 1)
        batch.lb_batch_step(check_every)
        batch.close()
        t += check_every
        for i in live:
            change, umax = ctxs[i].lb_velocity_change(uprev[i])
            a = ctxs[i].lb_diagnostics()[0]["vortex_amp_x3"]
            amps[i].append(a)
            h = amps[i][-3:]
            # a vortex amplitude below 1e-5 max |u| is round-off, not a vortex
            steady = len(h) == 3 and (max(abs(x - a) for x in h) <= amp_tol * a or
                                      max(h) <= 1e-5 * umax[0])
            if change[0] <= tol * check_every * max(umax[0], 1e-300) and steady:
                steps[i] = t
                done[i] = True
        if log:
            log(f"  step {t}: {int(done.sum())}/{n} converged")
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    rho_out, u_out = [], []
    for inst, ctx in zip(instances, ctxs):
        rho, u = ctx.lb_macros()
        rho_out.append(rho[0].reshape(inst.nr, ntheta, inst.n3).mean(axis=1))
        u_out.append(u[0].reshape(3, inst.nr, ntheta, inst.n3).mean(axis=2))
        ctx.close()
    return rho_out, u_out, steps, done, sec


def save_mixed_net(net, mean, std, path):
    """The mixed surrogate's parameters and output scale as an .npz file."""
    np.savez(path, params=net.get_params(), mean=np.asarray(mean, np.float32), std=np.asarray(std, np.float32),
             shape=np.array([N_PLAIN_MIXED, N_FOURIER_MIXED, net.width, net.depth]))


def load_mixed_net(path, max_batch=16384):
    """An LBMlp holding a saved mixed surrogate (save_mixed_net)."""
    z = np.load(path)
    npl, nf, w, d = (int(v) for v in z["shape"])
    net = L.LBMlp(n_fourier=nf, width=w, depth=d, max_batch=max_batch, n_plain=npl)
    net.set_params(z["params"])
    net.set_output_scale(z["mean"], z["std"])
    return net


def predict_mixed(net, inst, ntheta):
    """The surrogate's fields for instance inst on its grid with ntheta theta
    nodes: rho (N,), u (3, N) for lb_init_fields."""
    import torch
    xi = torch.from_numpy(mixed_inputs(inst, inst.nr, inst.n3)).cuda()
    yi = np.concatenate([net.predict(xi[s:s + net.max_batch]).cpu().numpy()
                         for s in range(0, len(xi), net.max_batch)])
    return mixed_fields(inst, yi, ntheta)


def run_mixed(n_train=2000, n_test=256, chunk=500, epochs=30, batch=16384, lr=2e-3, max_steps=600_000,
              check_every=10_000, train_ntheta=1, test_ntheta=4, seed=20241111, speed_cap=0.25, log=print,
              save=None):
    """The surrogate over the mixed-channel distribution: n_train converged
    states (generated with train_ntheta theta nodes: the developed flow is
    theta-uniform), a network of (De, kind, R2/R1, aspect, r, theta, z) ->
    (rho', u), then n_test held-out instances on their own grids (test_ntheta
    theta nodes) run to convergence from rest plus noise (cold) and from the
    network's prediction (warm). Reports steps and field error per metric
    kind."""
    import torch
    rep = {"n_train": n_train, "n_test": n_test, "speed_cap": speed_cap, "tol": 1e-8,
           "check_every": check_every, "max_steps": max_steps, "train_ntheta": train_ntheta,
           "test_ntheta": test_ntheta}
    train_set = draw_mixed(n_train, seed, speed_cap)
    test_set = draw_mixed(n_test, seed + 1_000_003, speed_cap)
    # 1. converged training states
    t0 = time.perf_counter()
    X, Y, st = [], [], []
    for s in range(0, n_train, chunk):
        part = train_set[s:s + chunk]
        rho, u, steps, ok, sec = converge_mixed(part, ntheta=train_ntheta, max_steps=max_steps,
                                                check_every=check_every)
        for inst, r_, u_, good in zip(part, rho, u, ok):
            if not (good and np.isfinite(r_).all() and np.isfinite(u_).all()):
                continue
            r_, u_ = align_mixed(inst, r_, u_)
            X.append(mixed_inputs(inst, inst.nr, inst.n3))
            Y.append(mixed_targets(inst, r_, u_))
        st.append(steps)
        log(f"train states {s}..{s + len(part)}: {sec:.1f} s, {int(ok.sum())} converged")
    rep["train_generation_s"] = time.perf_counter() - t0
    rep["train_states_used"] = len(X)
    rep["train_steps_mean"] = float(np.mean(np.concatenate(st)))
    x = np.concatenate(X)
    y = np.concatenate(Y)
    # 2. training
    t0 = time.perf_counter()
    net = L.LBMlp(n_fourier=N_FOURIER_MIXED, width=256, depth=5, max_batch=batch, seed=seed,
                  n_plain=N_PLAIN_MIXED)
    y_mean, y_std = y.mean(axis=0), np.maximum(y.std(axis=0), 1e-12)
    net.set_output_scale(y_mean, y_std)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    g = torch.Generator(device="cuda").manual_seed(seed)
    nsamp = len(x)
    losses = []
    for ep in range(epochs):
        step_lr = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        perm = torch.randperm(nsamp, device="cuda", generator=g)
        last = None
        for s in range(0, nsamp - batch + 1, batch):
            idx = perm[s:s + batch]
            want = s + 2 * batch > nsamp
            l_ = net.train_step(xd[idx].contiguous(), yd[idx].contiguous(), step_lr, want_loss=want)
            if want:
                last = l_
        losses.append(last)
        log(f"epoch {ep} loss {last:.3e}")
    rep["train_s"] = time.perf_counter() - t0
    rep["train_samples"] = nsamp
    rep["loss_first_last"] = [losses[0], losses[-1]]
    del xd, yd
    if save:
        save_mixed_net(net, y_mean, y_std, save)
    # 3. held-out: cold and warm starts to convergence
    t0 = time.perf_counter()
    preds = [predict_mixed(net, inst, test_ntheta) for inst in test_set]
    rep["inference_s"] = time.perf_counter() - t0
    rho_c, u_c, sc, okc, sec_c = converge_mixed(test_set, ntheta=test_ntheta, max_steps=max_steps,
                                                check_every=check_every, log=log)
    rho_w, u_w, sw, okw, sec_w = converge_mixed(test_set, ntheta=test_ntheta, max_steps=max_steps,
                                                check_every=check_every, warm=preds, log=log)
    rep["seconds_cold_warm"] = [sec_c, sec_w]
    err_pred, err_final = [], []
    for k, inst in enumerate(test_set):
        up = preds[k][1].reshape(3, inst.nr, test_ntheta, inst.n3).mean(axis=2)
        _, a = align_mixed(inst, rho_c[k], u_c[k])
        _, bp = align_mixed(inst, rho_c[k], up)
        _, bw = align_mixed(inst, rho_w[k], u_w[k])
        nrm = np.sqrt((a ** 2).sum())
        err_pred.append(float(np.sqrt(((bp - a) ** 2).sum()) / nrm))
        err_final.append(float(np.sqrt(((bw - a) ** 2).sum()) / nrm))
    err_pred, err_final = np.array(err_pred), np.array(err_final)
    for kind in ("cylindrical", "ellipsoidal"):
        sel = np.array([i.metric == kind for i in test_set])
        both = sel & okc & okw
        fin = sel & np.isfinite(err_pred) & np.isfinite(err_final)
        rep[kind] = {
            "instances": int(sel.sum()), "converged_cold": int((sel & okc).sum()),
            "converged_warm": int((sel & okw).sum()), "converged_both": int(both.sum()),
            "steps_cold_mean": float(sc[both].mean()) if both.any() else None,
            "steps_warm_mean": float(sw[both].mean()) if both.any() else None,
            "steps_saved_fraction": float(1.0 - sw[both].sum() / sc[both].sum()) if both.any() else None,
            "steps_saved_fraction_all_capped": float(1.0 - sw[sel].sum() / sc[sel].sum()),
            "nonfinite_fields": int((sel & ~fin).sum()),
            "surrogate_rel_l2_median": float(np.median(err_pred[fin])) if fin.any() else None,
            "surrogate_rel_l2_p90": float(np.percentile(err_pred[fin], 90)) if fin.any() else None,
            "warm_vs_cold_final_rel_l2_median": float(np.median(err_final[fin])) if fin.any() else None,
        }
    rep["test"] = [{"metric": i.metric, "nr": i.nr, "n3": i.n3, "dean": i.dean, "R2_over_R1": i.R2_over_R1,
                    "steps_cold": int(sc[k]), "steps_warm": int(sw[k]), "err_pred": float(err_pred[k]),
                    "err_final": float(err_final[k])} for k, i in enumerate(test_set)]
    net.close()
    return rep


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="surrogate warm start of Dean-vortex runs")
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--max-steps", type=int, default=400_000)

    ap.add_argument("--mixed", action="store_true",
                    help="the surrogate over the mixed-channel distribution (cylinders and double-curved "
                         "channels, inputs De, kind, R2/R1, aspect, r, theta, z)")
    ap.add_argument("--chunk", type=int, default=500)
    ap.add_argument("--save", default=None, help="--mixed: write the trained network here (.npz)")
    ap.add_argument("--check-every", type=int, default=10_000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    L.load_library()
    if a.mixed:
        r = run_mixed(a.train, a.test, chunk=a.chunk, epochs=a.epochs, max_steps=a.max_steps,
                      check_every=a.check_every, save=a.save)
        print(json.dumps({k: v for k, v in r.items() if k != "test"}, indent=1))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        raise SystemExit(0)
    r = run(a.train, a.test, epochs=a.epochs, max_steps=a.max_steps)
    print(json.dumps({k: v for k, v in r.items() if not isinstance(v, list)}, indent=1))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)
