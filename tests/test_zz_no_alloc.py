"""lb_diagnostics_noalloc: the observables for callers that cannot call
cudaMalloc (their device memory is owned by another allocator, or they must
not allocate after start-up). It must agree with the context's own
lb_diagnostics on the same state, call after call, while allocating nothing
on the device. This file is collected last on purpose."""
import numpy as np
import pytest

from gpu_helpers import lib

pytestmark = pytest.mark.gpu

FIELDS = ("mass_rho_prime", "mass_physical", "mean_v_theta", "dean", "mean_vorticity",
          "vortex_amp", "vortex_amp_x3", "max_speed")


@pytest.mark.parametrize("metric,geom", [
    ("cylindrical", dict(r_inner=1.0, r_outer=1 / 0.975, nr=16, ntheta=4, n3=32)),
    ("ellipsoidal", dict(r_inner=1.0, r_outer=1.1, nr=10, ntheta=3, n3=40, b=0.9,
                         periodic3=False)),
], ids=["cyl", "ell4wall"])
def test_noalloc_diagnostics_match_context(metric, geom):
    import torch
    L = lib()
    spec = L.ChannelSpec(metric, **geom)
    taus = [0.8, 0.6, 0.7]
    params = [L.make_params(t, 2e-4, False, 100 + i, 1e-2) for i, t in enumerate(taus)]
    ctx = L.LBContext(spec, batch=len(taus), precision="fp64")
    ctx.lb_init(params)
    ctx.lb_step(25)
    ref = ctx.lb_diagnostics()
    N = spec.ncells
    rho = torch.empty(len(taus) * N, dtype=torch.float64, device="cuda")
    u = torch.empty(len(taus) * 3 * N, dtype=torch.float64, device="cuda")
    ctx.lb_macros(rho, u, on_device=True)
    ctx.stream.synchronize()
    for _ in range(2):                       # the second call reuses the same scratch
        got = L.lb_diagnostics_noalloc(metric, spec.desc(), taus, rho, u, stream=ctx.stream)
        for b in range(len(taus)):
            for k in FIELDS:
                assert got[b][k] == pytest.approx(ref[b][k], rel=1e-12, abs=1e-300), (b, k)
            assert got[b]["nonfinite"] == ref[b]["nonfinite"] == 0
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    L = lib()
    desc = L.make_desc(1.0, 1.1, 512, 4, 512)          # geometry weights alone: 8 MiB
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError) as e:
        L.lb_diagnostics_noalloc("cylindrical", desc, [0.8], rho, rho)
    assert e.value.status == L.LB_ERR_ARG and "scratch" in str(e.value)
