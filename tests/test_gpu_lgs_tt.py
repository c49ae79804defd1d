"""LGS tip-tilt filter (reading R15) on the GPU's plain path against the FP64
oracle: M and the exact Jacobi diagonal (FP64 <= 1e-12), whole frames with the
mirror fit (FP64 <= 1e-10, FP32 <= 1e-4); the fused path, batches and
differentiation refuse the filter instead of ignoring it."""

import numpy as np
import pytest

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


def test_filter_refused_where_not_modelled(fw):
    import torch
    cfg = _cfg()
    with fw.Solver(cfg, precision=fw.FP32) as S:
        assert "plain" in S.describe()
        with pytest.raises(fw.FewhaError) as ei:
            S.set_path(fw.PATH_FUSED)
        assert ei.value.name == "ARG"
        tape = torch.empty(S.tape_bytes(2), dtype=torch.uint8, device="cuda")
        with pytest.raises(fw.FewhaError) as ei:
            S.solve_taped(torch.zeros(S.S, device="cuda"), 2, tape)
        assert ei.value.name == "STATE"
    with pytest.raises(fw.FewhaError) as ei:
        fw.Batch([cfg])
    assert ei.value.name == "ARG"
