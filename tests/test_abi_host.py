"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/lbgm.h declares, and its host-side logic (velocity table,
FP64 geometry precompute, force for a Dean number, argument validation)
agrees with the oracle and the closed forms."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from analytic import CS2, curved_poiseuille
from oracle import lattice as OL
from oracle.geometry import Channel, channel_geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1411_3133_gb300 import build, lbgm
    build.build()
    return lbgm


def _declared():
    src = open(os.path.join(ROOT, "include", "lbgm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_\w+)\s*\(", src)))


def test_exports_every_declared_function(L):
    lib = L.load_library()
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.SIGNATURES), "binding and header disagree"


def test_velocity_set_matches_table_I(L):
    c, w = L.lb_velocity_set()
    lib = {tuple(v): x for v, x in zip(c.tolist(), w)}
    ora = {tuple(v): x for v, x in zip(OL.C.tolist(), OL.W)}
    assert set(lib) == set(ora)
    for v in lib:
        assert lib[v] == pytest.approx(ora[v], rel=1e-14)
    assert c[0].tolist() == [0, 0, 0]
    for k in range(20):
        assert (c[2 * k + 1] == -c[2 * k + 2]).all()


CHANNELS = [
    Channel("cylindrical", 1.0, 1 / 0.975, 16, 4, 32),
    Channel("cylindrical", 1.0, 1 / 0.8, 9, 2, 7),
    Channel("flat", 0.0, 1.0, 8, 1, 1),
    Channel("ellipsoidal", 1.0, 1.1, 8, 4, 12, b=0.9, periodic3=False),
    Channel("ellipsoidal", 0.25, 0.275, 16, 4, 32, b=2.0, periodic3=False,
            dtheta_scale=2.0, d3_scale=4.0),
    Channel("cylindrical", 1.0, 1 / 0.975, 17, 4, 32, wall="equilibrium"),
    Channel("ellipsoidal", 1.0, 1.1, 9, 4, 13, b=0.9, periodic3=False, wall="equilibrium"),
    Channel("ellipsoidal", 1.0, 1.1, 9, 4, 13, b=0.9, wall="equilibrium"),
    Channel("ellipsoidal", 1.0, 1.2, 8, 5, 10, b=0.9, periodic3=False, dtheta_scale=8.0, d3_scale=2.0,
            theta_resolved=True),
    Channel("ellipsoidal", 0.25, 0.275, 9, 6, 12, b=1.7, dtheta_scale=3.0, wall="equilibrium",
            theta_resolved=True),
]


@pytest.mark.parametrize("ch", CHANNELS,
                         ids=lambda c: f"{c.metric}{'T' if c.theta_resolved else ''}{c.shape}{c.wall[:2]}"
                                       f"{int(c.periodic3)}")
def test_geometry_matches_oracle(L, ch):
    desc = L.make_desc(ch.r_inner, ch.r_outer, ch.nr, ch.ntheta, ch.n3, ch.b, ch.periodic3,
                       ch.dtheta_scale, ch.d3_scale, ch.wall)
    rows = L.lb_geometry_eval("ellipsoidal_theta" if ch.theta_resolved else ch.metric, desc)
    geo = channel_geometry(ch)
    assert np.allclose(rows[..., 0:9].reshape(geo["Delta"].shape), geo["Delta"], rtol=0, atol=1e-13)
    assert np.allclose(rows[..., 9:36].reshape(geo["Gamma_hat"].shape), geo["Gamma_hat"],
                       rtol=0, atol=1e-15 * max(1.0, np.abs(geo["Gamma_hat"]).max()))
    assert np.allclose(rows[..., 36:39], geo["fdir"], rtol=1e-13, atol=0)
    for k, name in [(39, "sqrtg"), (40, "speed"), (41, "wA"), (42, "wOmega"), (43, "r_phys")]:
        assert np.allclose(rows[..., k], geo[name], rtol=1e-13, atol=0), name


@pytest.mark.parametrize("nr,tau,De", [(16, 0.8, 30.0), (64, 0.55, 36.0), (64, 0.6, 60.0)])
def test_force_for_dean_matches_closed_form(L, nr, tau, De):
    ri, ro = 1.0, 1 / 0.975
    desc = L.make_desc(ri, ro, nr, 4, 32)
    G = L.lb_force_for_dean("cylindrical", desc, tau, De)
    _, v, _ = curved_poiseuille(ri, ro, nr, G, tau)
    nu = (tau - 0.5) * CS2
    assert v.mean() * nr / nu * math.sqrt((ro - ri) / ri) == pytest.approx(De, rel=1e-12)


def test_force_for_dean_with_wall_nodes(L):
    """Wall nodes: d = (N_r - 1) h, nodes r_i + i h, the laminar profile
    vanishing on the end nodes; De = <v> (N_r - 1) / nu sqrt(d / r_i)."""
    from analytic import curved_poiseuille_coeffs
    ri, ro, nr, tau, De = 1.0, 1 / 0.975, 33, 0.6, 40.0
    desc = L.make_desc(ri, ro, nr, 4, 32, wall="equilibrium")
    G = L.lb_force_for_dean("cylindrical", desc, tau, De)
    h = (ro - ri) / (nr - 1)
    r = ri + np.arange(nr) * h
    A, B, C = curved_poiseuille_coeffs(ri, ro, h, G, tau)
    v = A * r * np.log(r) + B * r + C / r
    assert abs(v[0]) < 1e-12 * abs(v).max() and abs(v[-1]) < 1e-12 * abs(v).max()
    nu = (tau - 0.5) * CS2
    assert v.mean() * (nr - 1) / nu * math.sqrt((ro - ri) / ri) == pytest.approx(De, rel=1e-12)


@pytest.mark.parametrize("kw,msg", [
    (dict(r_inner=1.0, r_outer=0.9), "r_outer"),
    (dict(nr=6), "nr >= 7"),
    (dict(nr=2, wall="equilibrium"), "nr >= 3"),
    (dict(periodic3=False, n3=2, wall="equilibrium"), "n3 >= 3"),
    (dict(ntheta=0), "ntheta"),
    (dict(periodic3=False, n3=5), "n3 >= 7"),
    (dict(dtheta_scale=0.0), "dtheta_scale"),
])
def test_invalid_geometry_rejected(L, kw, msg):
    base = dict(r_inner=1.0, r_outer=1.1, nr=16, ntheta=4, n3=32, b=1.0, periodic3=True,
                dtheta_scale=1.0, d3_scale=1.0)
    base.update(kw)
    desc = L.make_desc(**base)
    with pytest.raises(L.LBError) as e:
        L.lb_geometry_eval("cylindrical", desc)
    assert e.value.status == L.LB_ERR_ARG and msg in str(e.value)


def test_ellipsoid_pole_rejected(L):
    desc = L.make_desc(1.0, 1.1, 16, 4, 600, b=1.0, periodic3=False)  # |phi| up to 1.9
    with pytest.raises(L.LBError) as e:
        L.lb_geometry_eval("ellipsoidal", desc)
    assert "pole" in str(e.value)


def test_force_for_dean_rejects_ellipsoid(L):
    desc = L.make_desc(1.0, 1.1, 16, 4, 32)
    with pytest.raises(L.LBError):
        L.lb_force_for_dean("ellipsoidal", desc, 0.6, 30.0)


def test_splitmix64_reference_recurrence():
    """The counter form equals running the sequential generator k + 1 times."""
    from paper_1411_3133_gb300.workloads import splitmix64_at
    mask = (1 << 64) - 1
    seed = 20241111
    state, seq = seed, []
    for _ in range(6):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        seq.append(z ^ (z >> 31))
    got = splitmix64_at(seed, np.arange(6, dtype=np.uint64))
    assert [int(v) for v in got] == seq


def test_batch_entry_points_reject_bad_arguments_without_a_gpu(L):
    lib = L.load_library()
    out = ctypes.c_void_p(123)
    assert lib.lb_batch_create(None, 0, ctypes.byref(out)) == L.LB_ERR_ARG
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.lb_batch_create(arr, 0, ctypes.byref(out)) == L.LB_ERR_ARG
    assert out.value is None                      # cleared on failure
    assert lib.lb_batch_create(arr, 1, ctypes.byref(out)) == L.LB_ERR_ARG
    assert b"NULL" in lib.lb_batch_last_error(None)
    assert lib.lb_batch_step(None, 1) == L.LB_ERR_ARG
    assert lib.lb_batch_set_option(None, 0, 0) == L.LB_ERR_ARG
    assert lib.lb_batch_nodes(None) == -1 and lib.lb_batch_step_count(None) == -1
    lib.lb_batch_destroy(None)
    assert lib.lb_autotune(None, 1, None, None, 0, None) == L.LB_ERR_ARG


def test_mlp_create_rejects_bad_arguments_without_a_gpu(L):
    lib = L.load_library()
    out = ctypes.c_void_p(5)
    assert lib.lb_mlp_create(2, 2, 2, 5, 16, 1, None, ctypes.byref(out)) == L.LB_ERR_ARG
    assert out.value is None
    assert lib.lb_mlp_create(2, 2, 64, 1, 16, 1, None, ctypes.byref(out)) == L.LB_ERR_ARG
    assert b"width" in lib.lb_mlp_last_error(None)
    assert lib.lb_mlp_create(0, 2, 64, 3, 16, 1, None, ctypes.byref(out)) == L.LB_ERR_ARG
    assert b"n_plain" in lib.lb_mlp_last_error(None)
    assert lib.lb_mlp_param_count(None) == 0
    lib.lb_mlp_destroy(None)


def test_fma_peak_rejects_bad_arguments_without_a_gpu(L):
    lib = L.load_library()
    v = ctypes.c_double(-1.0)
    assert lib.lb_fma_peak(L.PRECISIONS["fp16_shifted"], None, ctypes.byref(v)) == L.LB_ERR_ARG
    assert b"precision" in lib.lb_last_error(None)
    assert lib.lb_fma_peak(L.PRECISIONS["fp64"], None, None) == L.LB_ERR_ARG
    assert v.value == -1.0                        # untouched on failure


def test_noalloc_binding_checks_fields_before_the_call(L):
    """The binding refuses host tensors, wrong dtypes and undersized fields
    itself: the C side reads B*N and 3*B*N doubles from raw pointers."""
    import torch
    desc = L.make_desc(1.0, 1.1, 8, 2, 8)
    n = 8 * 2 * 8 * 2
    good_rho = torch.zeros(n, dtype=torch.float64)
    good_u = torch.zeros(3 * n, dtype=torch.float64)
    with pytest.raises(L.LBError, match="CUDA tensor"):
        L.lb_diagnostics_noalloc("cylindrical", desc, [0.8, 0.7], good_rho, good_u)
    with pytest.raises(L.LBError, match="CUDA tensor"):
        L.lb_diagnostics_noalloc("cylindrical", desc, [0.8, 0.7], good_rho.numpy(), good_u)


def test_theta_resolved_geometry_validation(L):
    """The theta-resolved ellipsoid takes the ellipsoid's checks (b > 0, phi
    off the poles) and writes one row per node."""
    good = L.make_desc(1.0, 1.1, 8, 3, 10, 0.9, False)
    rows = L.lb_geometry_eval("ellipsoidal_theta", good)
    assert rows.shape == (8, 3, 10, 44)
    for bad in (L.make_desc(1.0, 1.1, 8, 3, 10, -1.0, False),          # b <= 0
                L.make_desc(1.0, 1.1, 8, 3, 400, 0.9, False, d3_scale=1.0)):  # phi reaches the pole
        with pytest.raises(L.LBError) as e:
            L.lb_geometry_eval("ellipsoidal_theta", bad)
        assert e.value.status == L.LB_ERR_ARG
