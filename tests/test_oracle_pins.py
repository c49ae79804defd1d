"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand, a swapped axis) fails one of them.
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------------------- db3 / DWT

def test_db3_matches_closed_form(golden):
    s = math.sqrt(5 + 2 * math.sqrt(10))
    r10 = math.sqrt(10)
    cf = np.array([1 + r10 + s, 5 + r10 + 3 * s, 10 - 2 * r10 + 2 * s, 10 - 2 * r10 - 2 * s,
                   5 + r10 - 3 * s, 1 + r10 - s]) / (16 * math.sqrt(2))
    assert np.max(np.abs(fo.DB3_H - cf)) < 1e-14
    assert np.max(np.abs(fo.DB3_H - np.array(golden["db3_closed_form"]["h_approx"]))) < 1e-13


def test_daubechies_family_special_cases():
    h1, g1 = fo.daubechies_filters(1)
    assert np.allclose(h1, [1 / math.sqrt(2)] * 2, atol=1e-15)
    assert np.allclose(g1, [1 / math.sqrt(2), -1 / math.sqrt(2)], atol=1e-15)
    h2, _ = fo.daubechies_filters(2)
    r3 = math.sqrt(3)
    assert np.allclose(h2, np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * math.sqrt(2)), atol=1e-14)


def test_db3_filter_identities():
    h, g = fo.DB3_H, fo.DB3_G
    assert abs(h.sum() - math.sqrt(2)) < 1e-14
    assert abs((h * h).sum() - 1) < 1e-14
    for m in (1, 2):
        assert abs(np.dot(h[2 * m:], h[:-2 * m])) < 1e-14
    k = np.arange(6)
    for p in range(3):
        assert abs(np.sum((-1.0) ** k * k ** p * h)) < 1e-12   # 3 vanishing moments
    assert abs(np.dot(h, g)) < 1e-15
    assert np.allclose(g, [(-1) ** i * h[5 - i] for i in range(6)])


@pytest.mark.parametrize("n", [8, 16, 32])
def test_dwt_dense_orthogonal_every_level(n):
    for J in range(1, int(math.log2(n))):
        W = np.stack([fo.fwd_dwt2(e.reshape(n, n), J).ravel() for e in np.eye(n * n)], axis=1)
        assert np.max(np.abs(W.T @ W - np.eye(n * n))) < 1e-13
        Wi = np.stack([fo.inv_dwt2(e.reshape(n, n), J).ravel() for e in np.eye(n * n)], axis=1)
        assert np.max(np.abs(Wi - W.T)) < 1e-13      # synthesis is the transpose


@pytest.mark.parametrize("n,J", [(128, 4), (256, 6), (64, 3)])
def test_dwt_perfect_reconstruction(n, J):
    x = np.random.default_rng(n).standard_normal((n, n))
    c = fo.fwd_dwt2(x, J)
    assert np.max(np.abs(fo.inv_dwt2(c, J) - x)) < 1e-13
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)


def test_dwt_smooth_field_has_small_details():
    # a quadratic (degree < 3 vanishing moments) away from the periodic seam
    n, J = 64, 3
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    f = np.sin(2 * np.pi * x / n) * np.cos(2 * np.pi * y / n)
    c = fo.fwd_dwt2(f, J)
    lev = fo.level_map(n, J)
    fine = np.abs(c[(lev == 1)]).max()
    assert fine < 1e-3 * np.abs(c).max()


def test_level_map_blocks():
    lev = fo.level_map(16, 3)
    assert lev[0, 0] == 3 and lev[1, 1] == 3 and lev[3, 3] == 3
    assert lev[4, 0] == 2 and lev[0, 7] == 2
    assert lev[8, 0] == 1 and lev[15, 15] == 1 and lev[0, 8] == 1


# --------------------------------------------------------------------------- Gamma

def test_gamma_hand_examples(golden):
    for key in ("gamma_single_subaperture", "gamma_two_by_two"):
        ex = golden[key]
        sx, sy = fo.Gamma(np.array(ex["psi"]))
        assert np.array_equal(sx, np.array(ex["sx"]))
        assert np.array_equal(sy, np.array(ex["sy"]))


def test_gamma_constant_and_plane():
    n, D = 12, 3.0
    d = D / n
    x = -D / 2 + np.arange(n + 1) * d
    X, Y = np.meshgrid(x, x, indexing="xy")
    sx, sy = fo.Gamma(np.full((n + 1, n + 1), 3.7))
    assert np.all(sx == 0) and np.all(sy == 0)
    a, b = 0.37, -1.25
    sx, sy = fo.Gamma(a * X + b * Y + 0.5)
    assert np.max(np.abs(sx - a * d)) < 1e-14
    assert np.max(np.abs(sy - b * d)) < 1e-14


def test_gamma_adjoint():
    rng = np.random.default_rng(3)
    n = 9
    psi = rng.standard_normal((n + 1, n + 1))
    sx, sy = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    gx, gy = fo.Gamma(psi)
    lhs = (gx * sx).sum() + (gy * sy).sum()
    rhs = (psi * fo.Gamma_T(sx, sy)).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# --------------------------------------------------------------------------- mask

def test_mask_hand_example(golden):
    ex = golden["mask_n4_obstruction_half"]
    assert np.array_equal(fo.subaperture_mask(ex["n"], ex["obstruction"]), np.array(ex["mask"], float))


def test_mask_elt_area_and_symmetry():
    m = fo.subaperture_mask(84, 0.28)
    assert np.array_equal(m, m[::-1]) and np.array_equal(m, m[:, ::-1]) and np.array_equal(m, m.T)
    area = math.pi / 4 * 84 ** 2 * (1 - 0.28 ** 2)
    assert abs(m.sum() - area) < 0.03 * area
    assert fo.subaperture_mask(2, 0.0).sum() == 4


# --------------------------------------------------------------------------- P

@pytest.mark.parametrize("lgs", [False, True])
def test_P_adjoint(lgs):
    g = fo.Geometry(configs.tiny(lgs=lgs, n_sub=6))
    rng = np.random.default_rng(5)
    for gg in range(g.G):
        for l in range(g.L):
            phi = rng.standard_normal((g.n[l], g.n[l]))
            y = rng.standard_normal((g.n_sub[gg] + 1,) * 2)
            lhs = (fo.P_layer(g, phi, gg, l) * y).sum()
            rhs = (phi * fo.PT_layer(g, y, gg, l)).sum()
            assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_P_adjoint_elt_geometry():
    g = fo.Geometry(configs.c2_elt())
    rng = np.random.default_rng(6)
    phi = rng.standard_normal((128, 128))
    y = rng.standard_normal((85, 85))
    for (gg, l) in [(0, 0), (3, 8), (5, 4)]:
        lhs = (fo.P_layer(g, phi, gg, l) * y).sum()
        rhs = (phi * fo.PT_layer(g, y, gg, l)).sum()
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("cfgname", ["c1_plain", "c2_elt", "c5_autograd"])
def test_P_reproduces_affine_layers_with_cone_and_shift(cfgname):
    """phi_l = a_l X + b_l Y + c_l maps to sum_l a_l (s x + th_x h) + b_l (s y + th_y h) + c_l."""
    cfg = configs.ALL[cfgname]()
    g = fo.Geometry(cfg)
    rng = np.random.default_rng(7)
    coef = rng.standard_normal((g.L, 3))
    phi = []
    for l in range(g.L):
        X = g.X0[l] + np.arange(g.n[l]) * g.delta[l]
        XX, YY = np.meshgrid(X, X, indexing="xy")
        phi.append(coef[l, 0] * XX + coef[l, 1] * YY + coef[l, 2])
    for gg in range(g.G):
        w = cfg["wfs"][gg]
        x = g.x_nodes[gg]
        XX, YY = np.meshgrid(x, x, indexing="xy")
        H = w["gs_height"]
        want = np.zeros_like(XX)
        for l in range(g.L):
            h = g.h[l]
            s = 1 - h / H if H > 0 else 1.0
            want += (coef[l, 0] * (s * XX + w["theta_x"] * h) + coef[l, 1] * (s * YY + w["theta_y"] * h)
                     + coef[l, 2])
        got = fo.P_apply(g, phi, gg)
        assert np.max(np.abs(got - want)) < 1e-11 * (1 + np.abs(want).max())


def test_P_identity_for_colocated_ground_layer():
    cfg = configs.tiny(n_sub=8, n=9)
    cfg["layers"] = [{"height": 0.0, "cn2": 1.0, "n": 9, "levels": 1}]
    g = fo.Geometry(cfg)
    phi = np.random.default_rng(8).standard_normal((9, 9))
    for gg in range(g.G):
        assert np.max(np.abs(fo.P_layer(g, phi, gg, 0) - phi)) < 1e-14


def test_layer_grid_extent_hand_examples(golden):
    """Layer extents, spacings and origins worked by hand for an NGS layer, an
    LGS cone layer, a layer set by the fitting directions, one set by the
    co-located mirror's actuator cover and one set by a tip-tilt NGS; plus the
    bilinear cell and weight of two sensor nodes, one on the last-node
    tie-break."""
    from paper_2009_00946_b300 import configs
    for case in golden["layer_grid_extents"]["cases"]:
        geo = fo.Geometry(getattr(configs, case["config"])())
        l = case["layer"]
        assert abs(geo.E[l] - case["E"]) <= 1e-9 * case["E"], case["config"]
        assert abs(geo.delta[l] - case["delta"]) <= 1e-9 * case["delta"], case["config"]
        assert abs(geo.X0[l] - case["X0"]) <= 1e-9 * abs(case["X0"]), case["config"]
        smp = case.get("sample")
        if smp:
            cy, ty, cx, tx = geo.tab[smp["wfs"]][l]
            assert cy[smp["i_last"]] == smp["cell_last"] and abs(ty[smp["i_last"]] - smp["t_last"]) < 1e-9
            assert cy[smp["i_first"]] == smp["cell_first"] and abs(ty[smp["i_first"]] - smp["t_first"]) < 1e-6


def test_geometry_error_outside_layer_grid():
    cfg = configs.tiny()
    g = fo.Geometry(cfg)
    g.X0[1] += 1.0   # shift the grid away from the footprint
    with pytest.raises(fo.GeometryError):
        g._table(0, 1)


# --------------------------------------------------------------------------- D

def test_regulariser_scaling():
    cfg = configs.tiny(n=16, levels=(3, 3))
    g = fo.Geometry(cfg)
    pr = g.default_params()
    D = g.D_diag(pr)
    l0 = g.layer(D, 0)
    lev = fo.level_map(16, 3)
    v1 = l0[lev == 1]
    v2 = l0[lev == 2]
    assert np.allclose(v1, v1[0]) and np.allclose(v2, v2[0])
    assert abs(v1[0] / v2[0] - 2.0 ** (11.0 / 3.0)) < 1e-13   # finer level, larger penalty
    pr2 = fo.Params(cn2=pr.cn2 * np.array([2.0, 1.0]), alpha=pr.alpha, w=pr.w)
    D2 = g.D_diag(pr2)
    assert np.allclose(g.layer(D2, 0), g.layer(D, 0) / 2.0, rtol=1e-15)
    assert np.allclose(g.layer(D2, 1), g.layer(D, 1), rtol=1e-15)


# --------------------------------------------------------------------------- M, b, J

def _functional(g, pr, c, s):
    """F(c) = sum_g w_g |mask (Gamma P W^T c - s)|^2 + alpha c^T D c, written through A."""
    phi = fo.layers_from_coeffs(g, c)
    As = fo.forward_slopes(g, phi)
    val = 0.0
    for gg in range(g.G):
        r = (As - s)[g.soff[gg]:g.soff[gg + 1]].reshape(2, g.n_sub[gg], g.n_sub[gg])
        val += pr.w[gg] * np.sum(g.mask[gg] * r ** 2)
    return val + pr.alpha * np.sum(g.D_diag(pr) * c * c)


@pytest.mark.parametrize("lgs,obs", [(False, 0.0), (True, 0.3)])
def test_M_and_b_against_map_functional(lgs, obs):
    cfg = configs.tiny(lgs=lgs, obstruction=obs, n_sub=6)
    g = fo.Geometry(cfg)
    pr = g.default_params()
    rng = np.random.default_rng(9)
    s = rng.standard_normal(g.S)
    z = np.zeros(g.S)
    for _ in range(3):
        v = rng.standard_normal(g.N)
        quad = _functional(g, pr, v, z)                 # = v^T M v
        assert abs(v @ fo.apply_M(g, v, pr) - quad) < 1e-11 * quad
        bv = (_functional(g, pr, -v, s) - _functional(g, pr, v, s)) / 4.0   # = b^T v
        assert abs(fo.rhs(g, s, pr) @ v - bv) < 1e-9 * (abs(bv) + 1)


def test_M_symmetric_positive_definite_dense():
    for levels in [(1, 1), (1, 2), (2, 2)]:
        g = fo.Geometry(configs.tiny(levels=levels))
        M = fo.assemble_M_dense(g)
        assert np.max(np.abs(M - M.T)) < 1e-13 * np.abs(M).max()
        assert np.linalg.eigvalsh((M + M.T) / 2).min() > 0


@pytest.mark.parametrize("kw", [dict(), dict(lgs=True, obstruction=0.3, n_sub=6, levels=(2, 2)),
                                dict(n=16, levels=(3, 2), n_sub=5)])
def test_jacobi_equals_dense_diagonal(kw):
    g = fo.Geometry(configs.tiny(**kw))
    M = fo.assemble_M_dense(g)
    Jd = fo.jacobi_diag(g)
    assert np.max(np.abs(Jd - np.diag(M))) < 1e-12 * np.diag(M).max()


# --------------------------------------------------------------------------- PCG

def test_alg2_equals_textbook_pcg():
    cfg = configs.c1_plain()
    R = fo.Reconstructor(cfg)
    g = R.geom
    s = synth.random_slopes(cfg, 12)
    b = fo.rhs(g, s, R.params)
    for k in (1, 2, 5, 20):
        c2, r2 = fo.pcg_alg2(R.Mop, R.Jinv, np.zeros(g.N), b, k)
        ct, rt = fo.pcg_textbook(R.Mop, R.Jinv, np.zeros(g.N), b, k)
        assert np.linalg.norm(c2 - ct) <= 1e-10 * np.linalg.norm(ct)
        assert np.linalg.norm(r2 - rt) <= 1e-9 * np.linalg.norm(b)


def test_pcg_converges_to_cholesky_solution():
    cfg = configs.tiny(levels=(2, 2))
    g = fo.Geometry(cfg)
    pr = g.default_params()
    M = fo.assemble_M_dense(g, pr)
    s = np.random.default_rng(10).standard_normal(g.S)
    b = fo.rhs(g, s, pr)
    L = np.linalg.cholesky(M)
    c_star = np.linalg.solve(L.T, np.linalg.solve(L, b))
    Jinv = 1.0 / fo.jacobi_diag(g, pr)
    Mop = lambda v: fo.apply_M(g, v, pr)
    ct, _ = fo.pcg_textbook(Mop, Jinv, np.zeros(g.N), b, 4 * g.N, tol=1e-14)
    assert np.linalg.norm(ct - c_star) <= 1e-10 * np.linalg.norm(c_star)
    c2, _ = fo.pcg_alg2(Mop, Jinv, np.zeros(g.N), b, 200)
    assert np.linalg.norm(c2 - c_star) <= 1e-10 * np.linalg.norm(c_star)
    # the MAP functional is stationary at the solution
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.standard_normal(g.N)
        eps = 1e-3
        dF = (_functional(g, pr, c_star + eps * v, s) - _functional(g, pr, c_star - eps * v, s)) / (2 * eps)
        dF0 = (_functional(g, pr, eps * v, s) - _functional(g, pr, -eps * v, s)) / (2 * eps)
        assert abs(dF) < 1e-8 * abs(dF0)


def test_pcg_breakdown_detected():
    N = 10
    with pytest.raises(fo.BreakdownError):
        fo.pcg_alg2(lambda v: -v, np.ones(N), np.zeros(N), np.ones(N), 2)


def test_warm_restart_recurrence_matches_replacement():
    cfg = configs.tiny(levels=(2, 2))
    cfg["alpha"] = 200.0
    S, _ = synth.frames(cfg, 3)
    Ra = fo.Reconstructor(cfg)
    Rb = fo.Reconstructor(cfg)
    for k in range(3):
        oa = Ra.frame(S[k], 6, warm=True, k_rr=0)     # recurrence only
        ob = Rb.frame(S[k], 6, warm=True, k_rr=1)     # replacement every frame (k > 0)
        assert np.linalg.norm(oa["c"] - ob["c"]) <= 1e-10 * np.linalg.norm(ob["c"])


# --------------------------------------------------------------------------- fitting

def _fit_cfg():
    cfg = configs.tiny(n_sub=6, n=16, levels=(2, 2), D=4.0)
    cfg["fit_dirs"] = [(x * fo.ARCSEC, y * fo.ARCSEC) for y in (-20.0, 20.0) for x in (-20.0, 0.0, 20.0)]
    cfg["dms"] = [{"height": 0.0, "pitch": 0.5}, {"height": 5000.0, "pitch": 0.8}]
    return cfg


def test_fitting_cg_matches_dense_normal_equations():
    cfg = _fit_cfg()
    g = fo.Geometry(cfg)
    F = fo.FitGeometry(g)
    rng = np.random.default_rng(12)
    phi = [rng.standard_normal((n, n)) for n in g.n]
    A = np.stack([F.normal_op(e) for e in np.eye(F.NA)], axis=1)
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.abs(A).max()
    x_star = np.linalg.solve(A, F.normal_rhs(phi))
    x = F.fit(phi, np.zeros(F.NA), 40 * F.NA)
    assert np.linalg.norm(x - x_star) <= 1e-8 * np.linalg.norm(x_star)


def test_fitting_reproduces_a_representable_field():
    """A ground layer equal to a bilinear DM shape is fitted exactly by that DM."""
    cfg = _fit_cfg()
    cfg["dms"] = [{"height": 0.0, "pitch": 0.5}]
    cfg["layers"] = [{"height": 0.0, "cn2": 1.0, "n": 16, "levels": 2}]
    g = fo.Geometry(cfg)
    F = fo.FitGeometry(g)
    # a field affine in x, y: both the layer and the DM represent it exactly
    X = g.X0[0] + np.arange(16) * g.delta[0]
    XX, YY = np.meshgrid(X, X, indexing="xy")
    phi = [0.3 * XX - 0.7 * YY + 0.1]
    x = F.fit(phi, np.zeros(F.NA), 400)
    for t in range(len(F.dirs)):
        assert np.max(np.abs(F.P_dm(x, t) - F.P_lay(phi, t))) < 1e-5


# --------------------------------------------------------------------------- inputs

def test_synth_plane_wave_slopes_exact():
    n, D = 10, 5.0
    x = -D / 2 + np.arange(2 * n + 1) * (D / (2 * n))
    X, Y = np.meshgrid(x, x, indexing="xy")
    s = synth.fine_grid_slopes(0.4 * X - 0.9 * Y, n)
    d = D / n
    assert np.max(np.abs(s[: n * n] - 0.4 * d)) < 1e-13
    assert np.max(np.abs(s[n * n:] + 0.9 * d)) < 1e-13


@pytest.mark.slow
def test_synth_structure_function():
    r0, L0, dx, N = 0.157, 25.0, 0.04, 1024
    rng = np.random.Generator(np.random.PCG64(123))
    acc = {5: [], 10: [], 20: []}
    for _ in range(6):
        scr = synth.von_karman_screen(N, dx, r0, L0, rng)
        for k in acc:
            acc[k].append(np.mean((scr[:, k:] - scr[:, :-k]) ** 2))
            acc[k].append(np.mean((scr[k:, :] - scr[:-k, :]) ** 2))
    for k, v in acc.items():
        want = synth.structure_function_vk(k * dx, r0, L0)
        assert abs(np.mean(v) / want - 1) < 0.10, (k, np.mean(v), want)
