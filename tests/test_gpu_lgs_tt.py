"""LGS tip-tilt filter (reading R15) on the GPU against the FP64 oracle: M and
the exact Jacobi diagonal (FP64 <= 1e-12), whole frames with the mirror fit on
the plain path (FP64 <= 1e-10, FP32 <= 1e-4) and on the fused path (FP32
<= 1e-4, the level-stacked layer phase, which applies the filter's rank-2 term
to the staged sensor fields), the MAORY-like setting of Sec. 4.1 with the
filter on its laser guide stars through the fused frame graph; the row-stripe
layer phase, batches and differentiation refuse the filter instead of
ignoring it."""

import numpy as np
import pytest

from _cases import elementwise_check

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

pytestmark = pytest.mark.gpu
N_FR = 8


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


def _cfg():
    cfg = configs.mcao_small()
    cfg["lgs_tip_tilt_filter"] = True
    return cfg


@pytest.fixture(scope="module")
def tt_ref():
    cfg = _cfg()
    S_in, _ = synth.frames(cfg, N_FR)
    R = fo.Reconstructor(cfg)
    ref = []
    for k in range(N_FR):
        o = R.frame(S_in[k], 4, warm=True, k_rr=10, gain=0.5, n_fit=8)
        ref.append((o["a"].copy(), R.layers()))
    return cfg, S_in, ref


def test_filtered_M_and_jacobi_match_oracle(fw):
    cfg = _cfg()
    g = fo.Geometry(cfg)
    assert all(g.tt[:4])
    with fw.Solver(cfg, precision=fw.FP64) as S:
        x = synth.random_coeffs(cfg, 5)
        assert rel(S.apply_M(x), fo.apply_M(g, x)) < 1e-12
        assert rel(S.vector(fw.VEC_JACOBI), fo.jacobi_diag(g)) < 1e-12


@pytest.mark.parametrize("prec_tol", [("FP64", 1e-10), ("FP32", 1e-4)])
def test_filtered_frames_match_oracle(fw, tt_ref, prec_tol):
    cfg, S_in, ref = tt_ref
    prec = getattr(fw, prec_tol[0])
    with fw.Solver(cfg, precision=prec, path=fw.PATH_PLAIN, k_rr=10) as S:
        for k in range(N_FR):
            S.set_frame(np.asarray(S_in[k], dtype=S.np_dtype))
            S.solve(4, warm=True)
            a = S.fit_dm(gain=0.5, n_fit=8)
            assert rel(a, ref[k][0]) < prec_tol[1], k
            assert rel(S.layers(), ref[k][1]) < prec_tol[1], k


def test_filtered_frames_fused_match_oracle(fw, tt_ref):
    cfg, S_in, ref = tt_ref
    sides = [l["n"] for l in cfg["layers"]]
    with fw.Solver(cfg, precision=fw.FP32, k_rr=10) as S:
        S.set_path(fw.PATH_FUSED)
        assert "level-stacked" in S.describe()
        for k in range(N_FR):
            S.set_frame(np.asarray(S_in[k], dtype=np.float32))
            S.solve(4, warm=True)
            a = S.fit_dm(gain=0.5, n_fit=8)
            assert rel(a, ref[k][0]) < 1e-4, k
            assert rel(S.layers(), ref[k][1]) < 1e-4, k
            elementwise_check(S.layers(), ref[k][1], sides, 1e-3, what=k)


def test_maory_with_lgs_filter_fused_graph_matches_oracle(fw):
    """The paper's timing setting (Sec. 4.1, Table 2): 6 LGS 80x80 with the
    tip-tilt filter and 3 tip-tilt NGS, L = M = 6 co-located mirrors, 4
    iterations and the fit, as one fused frame graph, across a replacement."""
    cfg = configs.maory()
    cfg["lgs_tip_tilt_filter"] = True
    nf = 12
    S_in, _ = synth.frames(cfg, nf)
    R = fo.Reconstructor(cfg)
    assert sum(R.geom.tt) == 6
    with fw.Solver(cfg, precision=fw.FP32, k_rr=10) as S:
        S.set_path(fw.PATH_FUSED)
        dl = np.empty(S.N, np.float32)
        da = np.empty(S.NA, np.float32)
        for k in range(nf):
            o = R.frame(S_in[k], 4, warm=True, k_rr=10, gain=0.5)
            S.frame(np.ascontiguousarray(S_in[k], dtype=np.float32), 4, warm=True, gain=0.5, layers_out=dl,
                    dm_out=da)
            assert rel(dl, R.layers()) < 1e-4, k
            assert rel(da, o["a"]) < 1e-4, k


def test_filter_refused_where_not_modelled(fw):
    import torch
    cfg = _cfg()
    with fw.Solver(cfg, precision=fw.FP32) as S:
        assert "fused" in S.describe()
        with pytest.raises(fw.FewhaError) as ei:
            S.set_layer_transform(0)          # the row-stripe layer phase does not model it
        assert ei.value.name == "ARG"
        tape = torch.empty(S.tape_bytes(2), dtype=torch.uint8, device="cuda")
        with pytest.raises(fw.FewhaError) as ei:
            S.solve_taped(torch.zeros(S.S, device="cuda"), 2, tape)
        assert ei.value.name == "STATE"
    with pytest.raises(fw.FewhaError) as ei:
        fw.Batch([cfg])
    assert ei.value.name == "ARG"
