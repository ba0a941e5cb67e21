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


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="surrogate warm start of Dean-vortex runs")
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--max-steps", type=int, default=400_000)

    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    L.load_library()
    r = run(a.train, a.test, epochs=a.epochs, max_steps=a.max_steps)
    print(json.dumps({k: v for k, v in r.items() if not isinstance(v, list)}, indent=1))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)
