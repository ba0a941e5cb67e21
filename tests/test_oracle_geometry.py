"""Oracle pins for the geometry: metric and Christoffel symbols.

What pins it:
  * the metric components and the non-vanishing Christoffel symbols printed in
    Sec. III (cylinder) and Sec. IV (ellipsoid), stored verbatim in
    tests/golden/printed_geometry.txt, at random points (theta not frozen);
  * b- and theta-independence of the ellipsoidal symbols, sqrt(g) = r and
    b r^2 cos(phi) (det of the printed metrics, by hand);
  * the tensor transformation law under a linear rescaling of coordinates
    (the Sec. IV.B spacings), a property of tensors, not of the code;
  * central finite differences of the printed metric, fed to the Christoffel
    formula of Sec. III (an independent numerical route).
"""
import math
import os

import numpy as np
import pytest

from oracle.geometry import Channel, channel_geometry, metric_and_christoffel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "printed_geometry.txt")
AX = {"r": 0, "th": 1, "z": 2, "ph": 2}


def _printed(metric):
    g, G = {}, {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        coords, qty, idx, expr = [p.strip() for p in line.split("|")]
        if coords != metric:
            continue
        key = tuple(AX[t] for t in idx.split())
        (g if qty == "g" else G)[key] = expr
    return g, G


def _eval(expr, r, th, x3, b):
    ns = {"sin": np.sin, "cos": np.cos, "tan": np.tan, "r": r, "th": th,
          "ph": x3, "z": x3, "b": b}
    return eval(expr, ns) * np.ones_like(r)


def _printed_arrays(metric, pts, b):
    gexpr, Gexpr = _printed(metric)
    r, th, x3 = pts[:, 0], pts[:, 1], pts[:, 2]
    g = np.zeros((len(pts), 3, 3))
    for (i, j), e in gexpr.items():
        g[:, i, j] = g[:, j, i] = _eval(e, r, th, x3, b)
    Gam = np.zeros((len(pts), 3, 3, 3))
    for (i, j, k), e in Gexpr.items():
        Gam[:, i, j, k] = _eval(e, r, th, x3, b)
    return g, Gam


def _random_points(rng, n=16):
    return np.stack([rng.uniform(0.3, 3.0, n), rng.uniform(-1.2, 1.2, n),
                     rng.uniform(-1.2, 1.2, n)], axis=1)


@pytest.mark.parametrize("metric", ["cylindrical", "ellipsoidal"])
@pytest.mark.parametrize("b", [1.0, 0.9, 1.7])
def test_metric_and_symbols_match_printed(metric, b):
    rng = np.random.default_rng(1 + int(10 * b))
    pts = _random_points(rng)
    g, _, Gam = metric_and_christoffel(metric, pts, b=b)
    gp, Gp = _printed_arrays(metric, pts, b)
    assert np.abs(g - gp).max() < 1e-13
    assert np.abs(Gam - Gp).max() < 1e-12


def test_flat_metric_is_euclidean():
    pts = _random_points(np.random.default_rng(3))
    g, dg, Gam = metric_and_christoffel("flat", pts)
    assert np.abs(g - np.eye(3)).max() == 0.0
    assert np.abs(dg).max() == 0.0 and np.abs(Gam).max() == 0.0


def test_ellipsoidal_symbols_independent_of_b_and_theta():
    rng = np.random.default_rng(7)
    pts = _random_points(rng)
    _, _, G1 = metric_and_christoffel("ellipsoidal", pts, b=0.6)
    _, _, G2 = metric_and_christoffel("ellipsoidal", pts, b=2.3)
    pts0 = pts.copy()
    pts0[:, 1] = 0.0
    _, _, G3 = metric_and_christoffel("ellipsoidal", pts0, b=1.4)
    assert np.abs(G1 - G2).max() < 1e-12
    assert np.abs(G1 - G3).max() < 1e-12


def test_sqrt_det_g():
    rng = np.random.default_rng(11)
    pts = _random_points(rng)
    r, ph = pts[:, 0], pts[:, 2]
    g, _, _ = metric_and_christoffel("cylindrical", pts)
    assert np.allclose(np.sqrt(np.linalg.det(g)), r, rtol=1e-14)
    for b in (0.7, 1.3):
        g, _, _ = metric_and_christoffel("ellipsoidal", pts, b=b)
        assert np.allclose(np.sqrt(np.linalg.det(g)), b * r ** 2 * np.cos(ph), rtol=1e-12)


def test_christoffel_formula_by_finite_differences():
    """Gamma^i_jk = 1/2 g^im (d_k g_mj + d_j g_mk - d_m g_jk) from central
    differences of the PRINTED metric, against the oracle's symbols."""
    rng = np.random.default_rng(5)
    pts = _random_points(rng, 6)
    b, eps = 0.8, 1e-5
    _, _, Gam = metric_and_christoffel("ellipsoidal", pts, b=b)
    dg = np.zeros((len(pts), 3, 3, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        gp, _ = _printed_arrays("ellipsoidal", pts + e, b)
        gm, _ = _printed_arrays("ellipsoidal", pts - e, b)
        dg[:, k] = (gp - gm) / (2 * eps)
    g, _ = _printed_arrays("ellipsoidal", pts, b)
    gi = np.linalg.inv(g)
    fd = np.zeros_like(Gam)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for m in range(3):
                    fd[:, i, j, k] += 0.5 * gi[:, i, m] * (dg[:, k, m, j] + dg[:, j, m, k]
                                                           - dg[:, m, j, k])
    assert np.abs(fd - Gam).max() < 1e-8


def test_rescaled_coordinates_follow_tensor_law():
    """x^i = s_i y^i: g'_ij = g_ij s_i s_j and Gamma'^i_jk = Gamma^i_jk s_j s_k / s_i."""
    rng = np.random.default_rng(9)
    y = _random_points(rng)
    s = np.array([1.0, 0.37, 2.5])
    gy, _, Gy = metric_and_christoffel("ellipsoidal", y, scale=s, b=1.2)
    gx, _, Gx = metric_and_christoffel("ellipsoidal", y * s, b=1.2)
    assert np.abs(gy - gx * s[None, :, None] * s[None, None, :]).max() < 1e-13
    expect = Gx * s[None, None, :, None] * s[None, None, None, :] / s[None, :, None, None]
    assert np.abs(Gy - expect).max() < 1e-12


def test_channel_lattice_map_cylinder():
    eta = 0.975
    ch = Channel("cylindrical", 1.0, 1.0 / eta, 16, 4, 32)
    geo = channel_geometry(ch)
    h = (1.0 / eta - 1.0) / 16
    assert ch.h == pytest.approx(h, rel=1e-15)
    r = 1.0 + (np.arange(16) + 0.5) * h
    assert np.allclose(geo["r_phys"][:, 0], r, rtol=0, atol=1e-15)
    # Sec. III closed forms, scaled to the lattice by h
    G = geo["Gamma_hat"][:, 0]
    assert np.allclose(G[:, 0, 1, 1], -h * r, rtol=1e-13)
    assert np.allclose(G[:, 1, 0, 1], h / r, rtol=1e-13)
    assert np.allclose(G[:, 1, 1, 0], h / r, rtol=1e-13)
    mask = np.ones((3, 3, 3), bool)
    mask[0, 1, 1] = mask[1, 0, 1] = mask[1, 1, 0] = False
    assert np.abs(G[:, mask]).max() < 1e-17
    assert np.allclose(geo["Delta"][:, 0, 1, 1], 1 / r ** 2 - 1, rtol=1e-13)
    assert np.allclose(geo["sqrtg"][:, 0], r, rtol=1e-14)
    assert np.allclose(geo["fdir"][:, 0], np.stack([0 * r, 1 / r ** 2, 0 * r], 1), rtol=1e-14)
    assert np.allclose(geo["speed"][:, 0], r) and np.allclose(geo["wOmega"][:, 0], r)
    assert np.allclose(geo["wA"], 1.0)
    assert ch.curvature_radius == 1.0


def test_channel_lattice_map_ellipsoid_rescaled():
    """Sec. IV.B: R_theta = r_i b^2 = 1 via b = 1/sqrt(r_i); Delta theta =
    h/(b r_i), Delta phi = h/r_i; evaluated at theta = 0."""
    ri = 2.0
    b = 1.0 / math.sqrt(ri)
    ch = Channel("ellipsoidal", ri, ri + 0.025, 8, 4, 12, b=b, periodic3=False,
                 dtheta_scale=1.0 / (b * ri), d3_scale=1.0 / ri)
    geo = channel_geometry(ch)
    h = 0.025 / 8
    r = geo["r_phys"]
    ph = (np.arange(12) + 0.5 - 6.0) * h / ri
    PH = np.broadcast_to(ph, r.shape)
    st, s3 = 1.0 / (b * ri), 1.0 / ri
    G = geo["Gamma_hat"]
    assert np.allclose(G[..., 0, 1, 1], -h * r * np.cos(PH) ** 2 * st ** 2, rtol=1e-12)
    assert np.allclose(G[..., 0, 2, 2], -h * r * s3 ** 2, rtol=1e-12)
    assert np.allclose(G[..., 1, 0, 1], h / r, rtol=1e-12)
    assert np.allclose(G[..., 2, 0, 2], h / r, rtol=1e-12)
    assert np.allclose(G[..., 1, 1, 2], -h * np.tan(PH) * s3, rtol=1e-12, atol=1e-18)
    assert np.allclose(G[..., 2, 1, 1], h * np.sin(PH) * np.cos(PH) * st ** 2 / s3,
                       rtol=1e-12, atol=1e-18)
    # theta = 0: diagonal metric, g_thth = b^2 r^2 cos^2 phi, g_phph = r^2 (unscaled)
    g = geo["g"]
    assert np.abs(g[..., 0, 1]).max() < 1e-15 and np.abs(g[..., 0, 2]).max() < 1e-15
    assert np.allclose(g[..., 1, 1], (b * r * np.cos(PH) * st) ** 2, rtol=1e-13)
    assert np.allclose(g[..., 2, 2], (r * s3) ** 2, rtol=1e-13)
    assert np.allclose(geo["sqrtg"], b * r ** 2 * np.cos(PH) * st * s3, rtol=1e-13)
    assert np.allclose(geo["wA"], r, rtol=1e-13)
    assert np.allclose(geo["wOmega"], r * b * np.cos(PH), rtol=1e-13)
    assert ch.curvature_radius == pytest.approx(1.0)
