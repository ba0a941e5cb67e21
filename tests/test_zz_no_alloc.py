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
    L.lb_diagnostics_noalloc(metric, spec.desc(), taus, rho, u, stream=ctx.stream)  # module loaded
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):                       # the second call reuses the same scratch
        got = L.lb_diagnostics_noalloc(metric, spec.desc(), taus, rho, u, stream=ctx.stream)
        assert torch.cuda.mem_get_info()[0] == free0     # nothing allocated on the device
        for b in range(len(taus)):
            for k in FIELDS:
                assert got[b][k] == pytest.approx(ref[b][k], rel=1e-12, abs=1e-300), (b, k)
            assert got[b]["nonfinite"] == ref[b]["nonfinite"] == 0
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Fields of the right size, a geometry whose weights alone need 8 MiB:
    the library itself refuses (the binding's own checks pass)."""
    import torch
    L = lib()
    desc = L.make_desc(1.0, 1.1, 512, 4, 512)
    n = 512 * 4 * 512
    rho = torch.ones(n, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError) as e:
        L.lb_diagnostics_noalloc("cylindrical", desc, [0.8], rho, u)
    assert e.value.status == L.LB_ERR_ARG and "scratch" in str(e.value)


def test_noalloc_binding_refuses_wrong_fields():
    """A float32 or undersized field never reaches the library."""
    import torch
    L = lib()
    desc = L.make_desc(1.0, 1.1, 8, 2, 8)
    n = 8 * 2 * 8
    rho = torch.ones(n, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBError, match="float64"):
        L.lb_diagnostics_noalloc("cylindrical", desc, [0.8], rho.float(), u)
    with pytest.raises(L.LBError, match="needs"):
        L.lb_diagnostics_noalloc("cylindrical", desc, [0.8], rho[:-1], u)
    with pytest.raises(L.LBError, match="needs"):
        L.lb_diagnostics_noalloc("cylindrical", desc, [0.8, 0.8], rho, u)
