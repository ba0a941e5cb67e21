"""Mixed-geometry batches (lb_batch_*) and the launch autotuners.

A batch step is one work-list launch per metric kind over instances of
different size; node for node it is the update of lb_step, so the states must
be bitwise those of every member stepped alone -- whatever the block size,
schedule, graph use, or interleaving with single-member steps. The small
members are also compared with the FP64 oracle (1e-12, as the FP64 parity
tests). Full size: the 128-instance mixed sweep (cylinders and double-curved
channels, N_r in {32, 48, 64}, N_3 in 128..512), sampled members bitwise
against standalone runs.
"""
import numpy as np
import pytest

from gpu_helpers import Twin, lib, max_rel, spec_of
from oracle.geometry import Channel
from paper_1411_3133_gb300.workloads import mixed_batch, noise_field

pytestmark = pytest.mark.gpu

ETA = 0.975
# (channel, per-instance params): every metric kind, ragged sizes, walls on
# one and two axes, one member holding three instances
MEMBERS = [
    (Channel("cylindrical", 1.0, 1 / 0.9, 9, 3, 13), [dict(tau=0.65, G=2e-4, seed=5, amp=5e-3)]),
    (Channel("flat", 0.0, 1.0, 8, 2, 9, periodic3=False), [dict(tau=0.6, G=1e-3, seed=9, amp=1e-2)]),
    (Channel("ellipsoidal", 1.0, 1.1, 10, 4, 14, b=0.9, periodic3=False),
     [dict(tau=0.7, G=3e-4, seed=10, amp=1e-2)]),
    (Channel("cylindrical", 1.0, 1 / ETA, 8, 4, 33),
     [dict(tau=0.8, G=1e-4, seed=1, amp=1e-3), dict(tau=0.6, G=3e-4, seed=2, amp=2e-3),
      dict(tau=1.1, G=0.0, seed=3, amp=5e-3, old=True)]),
    (Channel("ellipsoidal", 1.0, 1.1, 8, 3, 35, b=1.2), [dict(tau=0.8, G=2e-4, seed=13, amp=1e-2)]),
    (Channel("cylindrical", 1.0, 1 / ETA, 16, 4, 200), [dict(tau=0.55, G=3e-5, seed=14, amp=1e-3)]),
    (Channel("ellipsoidal", 1.0, 1.1, 9, 3, 11, b=0.9, periodic3=False, wall="equilibrium"),
     [dict(tau=0.7, G=3e-4, seed=15, amp=1e-2)]),
]


def _contexts(precision, stream=None):
    import torch
    L = lib()
    stream = stream if stream is not None else torch.cuda.Stream()
    out = []
    for ch, params in MEMBERS:
        c = L.LBContext(spec_of(ch), batch=len(params), precision=precision, stream=stream)
        c.lb_init([L.make_params(p["tau"], p["G"], p.get("old", False), p["seed"], p["amp"], False)
                   for p in params])
        out.append(c)
    return out


def _state(ctx):
    import torch
    buf = torch.empty(ctx.lb_state_bytes(), dtype=torch.uint8, device="cuda")
    ctx.lb_get_state(buf, on_device=True)
    return buf.cpu().numpy()


def _assert_same(batched, alone):
    for i, (a, b) in enumerate(zip(batched, alone)):
        assert np.array_equal(_state(a), _state(b)), f"member {i} differs"
        assert a.lb_step_count() == b.lb_step_count()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16_shifted", "bf16_shifted"])
@pytest.mark.parametrize("threads,schedule", [(64, 0), (128, 1), (256, 0), (192, 1)])
def test_batch_is_bitwise_lb_step(precision, threads, schedule):
    L = lib()
    batched, alone = _contexts(precision), _contexts(precision)
    batch = L.LBBatch(batched)
    batch.lb_batch_set_option(L.LB_OPT_BLOCK_THREADS, threads)
    batch.lb_batch_set_option(L.LB_OPT_SCHEDULE, schedule)
    batch.lb_batch_set_option(L.LB_OPT_USE_GRAPH, 1)
    for n in (1, 4, 7):        # odd counts leave the graph pair at parity 1
        batch.lb_batch_step(n)
    for c in alone:
        c.lb_step(12)
    assert batch.lb_batch_step_count() == 12
    assert batch.lb_batch_nodes() == sum(ch.ncells * len(p) for ch, p in MEMBERS)
    _assert_same(batched, alone)
    batch.close()


def test_batch_members_interleaved_with_single_steps():
    L = lib()
    batched, alone = _contexts("fp32"), _contexts("fp32")
    batch = L.LBBatch(batched)
    batch.lb_batch_set_option(L.LB_OPT_USE_GRAPH, 1)
    batch.lb_batch_step(3)
    batched[2].lb_step(1)            # one member runs ahead: the records follow its parity
    batch.lb_batch_step(4)
    batched[0].lb_set_state(_state(alone[0]))   # checkpoint restore resets that member's parity
    batch.lb_batch_step(2)
    for i, c in enumerate(alone):
        c.lb_step(2 if i == 0 else 9 + (i == 2))
    for i in range(1, len(MEMBERS)):
        assert np.array_equal(_state(batched[i]), _state(alone[i])), i
    assert np.array_equal(_state(batched[0]), _state(alone[0]))
    batch.close()


def test_batch_members_against_oracle():
    """The batch path itself, compared with the FP64 oracle."""
    import torch
    L = lib()
    stream = torch.cuda.Stream()
    twins = [Twin(ch, params, "fp64", stream=stream) for ch, params in MEMBERS[:5] + MEMBERS[6:]]
    for tw in twins:
        tw.ctx.lb_init(tw.lparams)
        for b, s in enumerate(tw.sims):
            p = tw.params[b]
            s.init_rest(noise_field(p["seed"], tw.N, p["amp"]))
    batch = L.LBBatch([tw.ctx for tw in twins])
    batch.lb_batch_set_option(L.LB_OPT_BLOCK_THREADS, 64)
    batch.lb_batch_step(10)
    for tw in twins:
        for s in tw.sims:
            s.step(10)
        rl, ul = tw.lib_macros()
        ro, uo = tw.oracle_macros()
        assert max_rel(rl, ro, np.abs(ro).max()) <= 1e-12
        assert max_rel(ul, uo, np.abs(uo).max()) <= 1e-12
        fl, fo = tw.lib_f(), np.stack([s.f for s in tw.sims])
        assert max_rel(fl, fo, np.abs(fo).max()) <= 1e-12
    batch.close()


def test_batch_autotune_steps_are_real_steps():
    L = lib()
    batched, alone = _contexts("fp32"), _contexts("fp32")
    batch = L.LBBatch(batched)
    best, trials = batch.lb_batch_autotune(steps_per_trial=3)
    assert len(trials) == 18                              # FP32: blocks up to 128
    assert {(t["block_threads"], t["schedule"], t["tile_nodes"]) for t in trials} == \
        {(t, s, t * k) for t in (64, 96, 128) for s in (0, 1) for k in (1, 2, 4)}
    assert all(t["ms_per_step"] > 0 for t in trials)
    assert best["ms_per_step"] == min(t["ms_per_step"] for t in trials)
    steps = 18 * (3 + 1)
    assert batch.lb_batch_step_count() == steps
    batch.lb_batch_step(5)          # with the chosen configuration
    for c in alone:
        c.lb_step(steps + 5)
    _assert_same(batched, alone)
    batch.close()


def test_context_autotune_steps_are_real_steps():
    L = lib()
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / ETA, 16, 4, 128)
    a = L.LBContext(spec, batch=2, precision="fp32")
    b = L.LBContext(spec, batch=2, precision="fp32")
    params = [L.make_params(0.6, 1e-4, False, 7 + i, 1e-3, True) for i in range(2)]
    a.lb_init(params)
    b.lb_init(params)
    best, trials = a.lb_autotune(steps_per_trial=2)
    # three block sizes for the plain, region-split and tiled kernels, and
    # the TMA kernel (n3 = 128)
    assert len(trials) == 10
    assert {t["schedule"] for t in trials} == {1, 2, 4, 5}
    for k in (1, 4, 5):
        assert {t["block_threads"] for t in trials if t["schedule"] == k} == {64, 96, 128}
    assert all(t["tile_nodes"] == 0 for t in trials)
    assert best["ms_per_step"] == min(t["ms_per_step"] for t in trials)
    assert a.lb_step_count() == 10 * 3
    b.lb_step(30)
    assert np.array_equal(_state(a), _state(b))
    a.close()
    b.close()


def test_batch_errors():
    import torch
    L = lib()
    ctxs = _contexts("fp32")
    with pytest.raises(L.LBError) as e:
        L.LBBatch([ctxs[0], ctxs[1], ctxs[0]])
    assert e.value.status == L.LB_ERR_ARG and "twice" in str(e.value)
    other = L.LBContext(spec_of(MEMBERS[0][0]), batch=1, precision="fp64", stream=ctxs[0].stream)
    with pytest.raises(L.LBError) as e:
        L.LBBatch([ctxs[0], other])
    assert e.value.status == L.LB_ERR_ARG
    own = L.LBContext(spec_of(MEMBERS[0][0]), batch=1, precision="fp32", stream=torch.cuda.Stream())
    with pytest.raises(L.LBError):
        L.LBBatch([ctxs[0], own])
    fresh = L.LBContext(spec_of(MEMBERS[0][0]), batch=1, precision="fp32", stream=ctxs[0].stream)
    batch = L.LBBatch([ctxs[1], fresh])          # creating is fine; stepping needs lb_init
    with pytest.raises(L.LBError) as e:
        batch.lb_batch_step(1)
    assert e.value.status == L.LB_ERR_STATE
    for opt, val in ((L.LB_OPT_BLOCK_THREADS, 48), (L.LB_OPT_SCHEDULE, 2), (L.LB_OPT_STEP_KERNEL, 1),
                     (99, 0)):
        with pytest.raises(L.LBError) as e:
            batch.lb_batch_set_option(opt, val)
        assert e.value.status == L.LB_ERR_ARG
    with pytest.raises(L.LBError) as e:
        batch.lb_batch_step(-1)
    assert e.value.status == L.LB_ERR_STATE      # still the uninitialised member
    batch.close()


def test_batch_nan_poisons_only_that_member():
    L = lib()
    ctxs = _contexts("fp64")
    f = ctxs[3].lb_get_populations()
    f[1, 7, 50] = np.nan
    ctxs[3].lb_set_populations(f)
    batch = L.LBBatch(ctxs)
    batch.lb_batch_set_option(L.LB_OPT_CHECK_EVERY, 1)
    with pytest.raises(L.LBError) as e:
        batch.lb_batch_step(3)
    assert e.value.status == L.LB_ERR_NONFINITE and "member 3" in str(e.value)
    with pytest.raises(L.LBError) as e:
        ctxs[3].lb_step(1)
    assert e.value.status == L.LB_ERR_STATE
    ctxs[0].lb_step(1)                           # the others stay usable
    ctxs[3].lb_init([L.make_params(p["tau"], p["G"], p.get("old", False), p["seed"], p["amp"], False)
                     for p in MEMBERS[3][1]])
    batch.lb_batch_step(2)                       # after re-initialisation the batch runs again
    assert ctxs[3].lb_diagnostics()[1]["nonfinite"] == 0
    batch.close()


def test_mixed_sweep_full_size_sampled_members_bitwise():
    """128 mixed instances (8.3 M nodes) in FP32 and BF16 storage: sampled
    members bitwise equal to the same channel stepped alone."""
    import torch

    from paper_1411_3133_gb300.sweep import mixed_contexts
    L = lib()
    insts = mixed_batch()
    for precision in ("fp32", "bf16_shifted"):
        ctxs, batch = mixed_contexts(insts, precision)
        batch.lb_batch_set_option(L.LB_OPT_USE_GRAPH, 1)
        batch.lb_batch_step(9)
        for i in (0, 1, 64, 127):
            alone, _ = mixed_contexts([insts[i]], precision, stream=torch.cuda.Stream())
            alone[0].lb_step(9)
            assert np.array_equal(_state(ctxs[i]), _state(alone[0])), (precision, i)
            _.close()
            alone[0].close()
        d = [c.lb_diagnostics()[0] for c in ctxs]
        assert all(x["nonfinite"] == 0 for x in d)
        batch.close()
        for c in ctxs:
            c.close()


def test_velocity_change_monitor():
    import torch
    L = lib()
    ctxs = _contexts("fp32")
    c = ctxs[3]                                   # three instances
    N = c.spec.ncells
    u_prev = torch.empty(3 * 3 * N, dtype=torch.float64, device="cuda")
    c.lb_macros(None, u_prev, on_device=True)
    ch, um = c.lb_velocity_change(u_prev)
    assert np.all(ch == 0)
    _, u = c.lb_macros()
    assert np.allclose(um, np.abs(u).reshape(3, -1).max(axis=1), rtol=0, atol=0)
    before = u_prev.cpu().numpy().reshape(3, -1)
    c.lb_step(5)
    ch, um = c.lb_velocity_change(u_prev)
    _, u = c.lb_macros()
    assert np.allclose(ch, np.abs(u.reshape(3, -1) - before).max(axis=1), rtol=0, atol=0)
    assert np.array_equal(u_prev.cpu().numpy().reshape(3, -1), u.reshape(3, -1))
