"""Pins of the oracle's LTAO / MOAO fitting modes (Sec. 1 and 4.3; reading
R17): a MOAO fit is block diagonal -- mirror t's normal equations and right-hand
side are exactly those of a one-mirror fit in direction t alone, and the CG fit
reaches the dense solution of that block system; every mode reproduces a field
its mirrors can represent; MOAO is open loop only."""

import copy

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth


def _single(g, t):
    """The one-mirror, one-direction (LTAO-type) fit of MOAO object t, on the
    same layer grids (their extent depends on all fitting directions, R3)."""
    g1 = copy.copy(g)
    g1.dms = [g.dms[t]]
    g1.fit_dirs = [g.fit_dirs[t]]
    g1.moao = False
    return fo.FitGeometry(g1)


def _random_layers(g, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((n, n)) for n in g.n]


def test_moao_normal_equations_are_per_object_fits():
    cfg = configs.ao_mode_small("moao")
    g = fo.Geometry(cfg)
    F = fo.FitGeometry(g)
    assert g.moao and F.M == len(F.dirs) == 3
    rng = np.random.default_rng(3)
    a = rng.standard_normal(F.NA)
    phi = _random_layers(g, 4)
    Na = F.normal_op(a) - F.eps * a
    rhs = F.normal_rhs(phi)
    for t in range(F.M):
        S = _single(g, t)
        blk = slice(F.aoff[t], F.aoff[t + 1])
        at = a[blk]
        want = S.normal_op(at) - S.eps * at
        assert np.max(np.abs(Na[blk] - want)) <= 1e-12 * np.abs(want).max(), t
        want_rhs = S.normal_rhs(phi)
        assert np.max(np.abs(rhs[blk] - want_rhs)) <= 1e-12 * np.abs(want_rhs).max(), t
    # another object's mirror does not enter block t
    b = a.copy()
    b[F.aoff[1]:F.aoff[2]] += rng.standard_normal(F.aoff[2] - F.aoff[1])
    Nb = F.normal_op(b) - F.eps * b
    assert np.array_equal(Nb[F.aoff[0]:F.aoff[1]], Na[F.aoff[0]:F.aoff[1]])
    assert np.array_equal(Nb[F.aoff[2]:F.aoff[3]], Na[F.aoff[2]:F.aoff[3]])


def test_moao_cg_fit_reaches_dense_block_solution():
    cfg = configs.ao_mode_small("moao")
    g = fo.Geometry(cfg)
    F = fo.FitGeometry(g)
    phi = _random_layers(g, 5)
    A = np.stack([F.normal_op(e) for e in np.eye(F.NA)], axis=1)
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.abs(A).max()
    for s in range(F.M):
        for t in range(F.M):
            if s != t:
                assert not A[F.aoff[s]:F.aoff[s + 1], F.aoff[t]:F.aoff[t + 1]].any(), (s, t)
    x_star = np.linalg.solve(A, F.normal_rhs(phi))
    x = F.fit(phi, np.zeros(F.NA), 6 * F.NA)
    assert np.linalg.norm(x - x_star) <= 1e-8 * np.linalg.norm(x_star)


@pytest.mark.parametrize("mode", ["ltao", "moao"])
def test_mode_reproduces_a_representable_field(mode):
    """A single ground layer that is affine is represented exactly by a ground
    mirror: every object sees it through its own mirror without error."""
    cfg = configs.ao_mode_small(mode)
    cfg["layers"] = [{"height": 0.0, "cn2": 1.0, "n": 32, "levels": 3}]
    g = fo.Geometry(cfg)
    F = fo.FitGeometry(g)
    X = g.X0[0] + np.arange(32) * g.delta[0]
    XX, YY = np.meshgrid(X, X, indexing="xy")
    phi = [0.3 * XX - 0.7 * YY + 0.1]
    x = F.fit(phi, np.zeros(F.NA), 600)
    for t in range(len(F.dirs)):
        assert np.max(np.abs(F.P_dm(x, t) - F.P_lay(phi, t))) < 1e-5, t


def test_moao_is_open_loop_only_and_needs_a_mirror_per_object():
    cfg = configs.ao_mode_small("moao")
    R = fo.Reconstructor(cfg)
    s = synth.frames(cfg, 1)[0][0]
    out = R.frame(s, 2, warm=False, gain=0.5)
    assert out["a"].shape == (sum(n * n for n in R.fitgeom.na),) and np.isfinite(out["a"]).all()
    with pytest.raises(ValueError):
        R.frame(s, 2, warm=True, gain=0.5, loop="closed")
    bad = copy.deepcopy(cfg)
    bad["dms"] = bad["dms"][:2]
    with pytest.raises(ValueError):
        fo.Geometry(bad)
