"""Pins of the oracle's MAORY-like setting (Sec. 4.1, Table 2): the low-order
sensors' masks (reading R14), the co-located fit for L = M (reading R16: each
mirror samples its layer, exact for affine layers), and the configuration's
mirror sizes against Table 2."""

import copy

import numpy as np

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs


def test_low_order_sensors_are_fully_active():
    for n in (1, 2):
        assert fo.subaperture_mask(n, 0.28).sum() == n * n
    m3 = fo.subaperture_mask(3, 0.28)
    assert m3[1, 1] == 0 and m3.sum() == 8          # the centre rule still applies from 3 on


def test_table2_mirror_sizes_and_colocation():
    cfg = configs.maory()
    g = fo.Geometry(cfg)
    fg = fo.FitGeometry(g)
    assert g.colocated
    assert fg.na == [81, 48, 48, 48, 48, 54]
    assert [w["n_sub"] for w in cfg["wfs"]] == [80] * 6 + [2, 1, 1]
    for m in range(fg.M):   # the layer grid covers its mirror's actuators
        assert g.E[m] >= (fg.na[m] - 1) * fg.pitch[m] - 1e-9


def test_colocated_fit_is_exact_for_affine_layers():
    cfg = configs.maory(n_layers=3)
    g = fo.Geometry(cfg)
    fg = fo.FitGeometry(g)
    coef = [(0.2, -0.5, 1.0), (-0.9, 0.3, 0.1), (0.05, 0.7, -2.0)]
    phi = []
    for l, (al, be, ga) in enumerate(coef):
        X = g.X0[l] + np.arange(g.n[l]) * g.delta[l]
        XX, YY = np.meshgrid(X, X, indexing="xy")
        phi.append(al * XX + be * YY + ga)
    a = fg.colocated_fit(phi)
    for m, (al, be, ga) in enumerate(coef):
        X = fg.A0[m] + np.arange(fg.na[m]) * fg.pitch[m]
        XX, YY = np.meshgrid(X, X, indexing="xy")
        want = al * XX + be * YY + ga
        assert np.abs(fg.dm(a, m) - want).max() <= 1e-12 * np.abs(want).max()


def test_mirror_off_its_layer_keeps_the_least_squares_fit():
    cfg = copy.deepcopy(configs.maory(n_layers=3))
    cfg["dms"][1]["height"] = 5000.0
    assert not fo.Geometry(cfg).colocated
