"""Each operator of M on its own through fewha_apply_operator, against the
oracle's definition: W and W^T (periodic db3, Sec. 2.2), P and P^T (bilinear
propagation with the LGS cone, Sec. 2.1), Gamma and Gamma^T (Shack-Hartmann on
the bilinear grid, Sec. 2.1).  FP64 <= 1e-12, FP32 <= 1e-5 (relative L2)."""

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


def _oracle(op, g, x):
    lay = lambda v: [v[g.off[l]:g.off[l + 1]].reshape(g.n[l], g.n[l]) for l in range(g.L)]
    noff = np.concatenate([[0], np.cumsum([(n + 1) ** 2 for n in g.n_sub])])
    nodes = lambda v: [v[noff[q]:noff[q + 1]].reshape(g.n_sub[q] + 1, -1) for q in range(g.G)]
    if op == 0:
        return np.concatenate([fo.fwd_dwt2(p, g.J[l]).ravel() for l, p in enumerate(lay(x))])
    if op == 1:
        return np.concatenate([fo.inv_dwt2(p, g.J[l]).ravel() for l, p in enumerate(lay(x))])
    if op == 2:
        return np.concatenate([fo.P_apply(g, lay(x), q).ravel() for q in range(g.G)])
    if op == 3:
        ps = nodes(x)
        return np.concatenate([sum(fo.PT_layer(g, ps[q], q, l) for q in range(g.G)).ravel() for l in range(g.L)])
    if op == 4:
        return np.concatenate([np.concatenate([a.ravel() for a in fo.Gamma(p)]) for p in nodes(x)])
    out = []
    for q in range(g.G):
        sx, sy = g.split_slopes(x, q)
        out.append(fo.Gamma_T(sx, sy).ravel())
    return np.concatenate(out)


@pytest.mark.parametrize("name", ["c1_plain", "c2_elt"])
@pytest.mark.parametrize("op", [0, 1, 2, 3, 4, 5])
def test_operator_matches_oracle(fw, name, op):
    cfg = getattr(configs, name)()
    g = fo.Geometry(cfg)
    for prec, tol in ((fw.FP64, 1e-12), (fw.FP32, 1e-5)):
        with fw.Solver(cfg, precision=prec) as S:
            ni, no = S.operator_dims(op)
            x = np.random.default_rng(op + 10).standard_normal(ni)
            got = S.apply_operator(op, x)
            want = _oracle(op, g, x.astype(S.np_dtype).astype(np.float64))
            assert got.size == no == want.size
            assert rel(got, want) < tol, (name, op, prec, rel(got, want))
            assert S.time_operator(op, 3) > 0.0
