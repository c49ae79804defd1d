"""Pins of the level-weighted ("modified") Jacobi preconditioner (reading R18):
no weights is exactly the plain Jacobi diag(M); each coefficient's diagonal is
scaled by its level's weight, the level read from the coefficient's position
in the Mallat layout; the preconditioned CG reaches the same solution as a
dense Cholesky solve (the weights change the path, not the fixed point); and
in a 4-step frame they change the result."""

import copy

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth


def _cfg(weights=None):
    cfg = configs.tiny(n_sub=4, n=8, levels=(2, 2), G=2)
    if weights is not None:
        cfg["jacobi_level_weights"] = weights
    return cfg


def test_no_weights_is_plain_jacobi():
    g = fo.Geometry(_cfg())
    assert np.array_equal(fo.preconditioner_diag(g), fo.jacobi_diag(g))
    g1 = fo.Geometry(_cfg([1.0, 1.0]))
    assert np.array_equal(fo.preconditioner_diag(g1), fo.jacobi_diag(g1))


def test_weights_follow_the_mallat_levels():
    """Level 1 (finest) is the part of the layout outside the n/2 block, level 2
    the part of the n/2 block outside the n/4 block, and with J = 2 the n/4 LL
    block is level 2 as well."""
    g = fo.Geometry(_cfg([3.0, 0.5]))
    ratio = fo.preconditioner_diag(g) / fo.jacobi_diag(g)
    for l in range(g.L):
        n = g.n[l]
        r = ratio[g.off[l]:g.off[l + 1]].reshape(n, n)
        outer = np.ones((n, n), bool)
        outer[: n // 2, : n // 2] = False
        assert np.allclose(r[outer], 3.0, rtol=0, atol=1e-15)
        assert np.allclose(r[: n // 2, : n // 2], 0.5, rtol=0, atol=1e-15)


def test_modified_jacobi_pcg_reaches_the_dense_solution():
    g = fo.Geometry(_cfg([0.25, 4.0]))
    pr = g.default_params()
    M = fo.assemble_M_dense(g, pr)
    s = np.random.default_rng(21).standard_normal(g.S)
    b = fo.rhs(g, s, pr)
    L = np.linalg.cholesky(M)
    c_star = np.linalg.solve(L.T, np.linalg.solve(L, b))
    Jinv = 1.0 / fo.preconditioner_diag(g, pr)
    c, _ = fo.pcg_textbook(lambda v: fo.apply_M(g, v, pr), Jinv, np.zeros(g.N), b, 4 * g.N, tol=1e-14)
    assert np.linalg.norm(c - c_star) <= 1e-10 * np.linalg.norm(c_star)


def test_weights_change_a_short_solve_and_are_validated():
    cfg0 = configs.mcao_small(True)
    cfg1 = copy.deepcopy(cfg0)
    cfg1["jacobi_level_weights"] = [1.0, 0.5, 0.25]
    s = synth.frames(cfg0, 1)[0][0]
    R0, R1 = fo.Reconstructor(cfg0), fo.Reconstructor(cfg1)
    R0.frame(s, 4, warm=False)
    R1.frame(s, 4, warm=False)
    assert np.linalg.norm(R0.layers() - R1.layers()) > 1e-6 * np.linalg.norm(R0.layers())
    bad = copy.deepcopy(cfg0)
    bad["jacobi_level_weights"] = [1.0, 0.0]
    with pytest.raises(ValueError):
        fo.Reconstructor(bad)
