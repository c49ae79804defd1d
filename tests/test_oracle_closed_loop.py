"""Pins of the oracle's closed loop (Alg. 1): the mirrors' field at the sensor
nodes for affine mirror shapes (exact under bilinear interpolation, so it
fixes the shift theta_g h_m and the cone factor 1 - h_m/H_g), the slopes it
makes, and the identity between a closed-loop frame on residual slopes and an
open-loop frame on the full slopes."""

import copy

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth


def _affine_mirrors(fg, coef):
    """a_m(X, Y) = alpha_m X + beta_m Y + gamma_m at the actuators of mirror m."""
    out = []
    for m in range(fg.M):
        al, be, ga = coef[m]
        X = fg.A0[m] + np.arange(fg.na[m]) * fg.pitch[m]
        XX, YY = np.meshgrid(X, X, indexing="xy")
        out.append((al * XX + be * YY + ga).ravel())
    return np.concatenate(out)


@pytest.mark.parametrize("lgs", [True, False])
def test_affine_mirrors_seen_by_each_sensor(lgs):
    cfg = configs.mcao_small(lgs=lgs)
    g = fo.Geometry(cfg)
    fg = fo.FitGeometry(g)
    coef = [(0.3, -0.7, 1.5), (-1.1, 0.4, -0.2)]
    a = _affine_mirrors(fg, coef)
    for q in range(g.G):
        w = cfg["wfs"][q]
        x = g.x_nodes[q]
        XX, YY = np.meshgrid(x, x, indexing="xy")
        want = np.zeros_like(XX)
        sx_want = sy_want = 0.0
        for m, (al, be, ga) in enumerate(coef):
            h = fg.hm[m]
            sc = 1.0 - h / w["gs_height"] if w["gs_height"] > 0 else 1.0
            want += al * (sc * XX + w["theta_x"] * h) + be * (sc * YY + w["theta_y"] * h) + ga
            sx_want += al * sc * g.d[q]
            sy_want += be * sc * g.d[q]
        got = fg.dm_to_wfs(a, q)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
        sx, sy = g.split_slopes(fg.dm_slopes(a), q)
        assert np.allclose(sx, sx_want, rtol=0, atol=1e-12) and np.allclose(sy, sy_want, rtol=0, atol=1e-12)


def test_constant_mirrors_add_no_slopes():
    g = fo.Geometry(configs.mcao_small())
    fg = fo.FitGeometry(g)
    assert np.abs(fg.dm_slopes(np.full(fg.NA, 3.25))).max() < 1e-13


def test_closed_loop_on_residual_slopes_equals_open_loop():
    """With the same state, a closed-loop frame on s - Gamma P_DM a^(-1)
    reconstructs exactly what an open-loop frame on s does; only the gain law
    differs: a1 = a0 + g (a~ - a^(-1))."""
    cfg = configs.mcao_small()
    S, _ = synth.frames(cfg, 3)
    A = fo.Reconstructor(cfg)
    for k in range(2):
        A.frame(S[k], 4, warm=True, gain=0.5)
    rng = np.random.default_rng(3)
    A.state.a_prev = rng.standard_normal(A.fitgeom.NA) * 0.1
    B = copy.deepcopy(A)
    s_res = S[2] - A.fitgeom.dm_slopes(A.state.a_prev)
    a_prev, a_cur = A.state.a_prev.copy(), A.state.a_cur.copy()
    oa = A.frame(S[2], 4, warm=True, gain=0.5, loop="open")
    ob = B.frame(s_res, 4, warm=True, gain=0.5, loop="closed")
    assert np.abs(ob["c"] - oa["c"]).max() <= 1e-11 * np.abs(oa["c"]).max()
    assert np.abs(B.state.a_fit - A.state.a_fit).max() <= 1e-11 * np.abs(A.state.a_fit).max()
    want = a_cur + 0.5 * (B.state.a_fit - a_prev)
    assert np.abs(ob["a"] - want).max() <= 1e-13 * np.abs(want).max()
    assert np.array_equal(B.state.a_prev, a_cur)


def test_sensor_beyond_the_mirror_is_a_geometry_error():
    cfg = configs.mcao_small(lgs=False)
    cfg["wfs"][0]["theta_x"] = 90.0 * fo.ARCSEC     # beyond the +-30 arcsec the mirrors cover
    g = fo.Geometry(cfg)
    fg = fo.FitGeometry(g)
    with pytest.raises(fo.GeometryError):
        fg.dm_slopes(np.zeros(fg.NA))
