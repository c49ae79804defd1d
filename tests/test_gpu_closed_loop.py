"""Closed loop of Alg. 1 on the GPU (pseudo-open-loop slopes s + Gamma P_DM
a^(-1) and the closed-loop gain) against the FP64 oracle: plain FP64 path
<= 1e-10 and the FP32 fused frame graph <= 1e-4 on the mirror commands and
the layers, over frames that cross a residual replacement."""

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

pytestmark = pytest.mark.gpu
N_FR = 12


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


@pytest.fixture(scope="module")
def closed_ref():
    cfg = configs.mcao_small()
    S_in, _ = synth.frames(cfg, N_FR)
    S_in = S_in * 0.5     # residual measurements of a partly corrected wavefront
    R = fo.Reconstructor(cfg)
    ref = []
    for k in range(N_FR):
        o = R.frame(S_in[k], 4, warm=True, k_rr=10, gain=0.5, n_fit=8, loop="closed")
        ref.append((o["a"].copy(), R.layers()))
    return cfg, S_in, ref


def test_closed_loop_fp64_plain_matches_oracle(fw, closed_ref):
    cfg, S_in, ref = closed_ref
    with fw.Solver(cfg, precision=fw.FP64, path=fw.PATH_PLAIN, k_rr=10) as S:
        S.set_loop(True)
        for k in range(N_FR):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            a = S.fit_dm(gain=0.5, n_fit=8)
            assert rel(a, ref[k][0]) < 1e-10, k
            assert rel(S.layers(), ref[k][1]) < 1e-10, k


def test_closed_loop_fp32_fused_graph_matches_oracle(fw, closed_ref):
    import torch
    cfg, S_in, ref = closed_ref
    with fw.Solver(cfg, precision=fw.FP32, k_rr=10) as S:
        S.set_path(fw.PATH_FUSED)
        S.set_loop(True)
        ds = torch.empty(S.S, dtype=torch.float32, device="cuda")
        dl = torch.empty(S.N, dtype=torch.float32, device="cuda")
        da = torch.empty(S.NA, dtype=torch.float32, device="cuda")
        for k in range(N_FR):
            with torch.cuda.stream(S.stream):
                ds.copy_(torch.from_numpy(S_in[k].astype(np.float32)).cuda())
            S.stream.synchronize()
            S.frame(ds, 4, warm=True, gain=0.5, n_fit=8, layers_out=dl, dm_out=da)
            S.sync()
            assert rel(da.cpu().numpy(), ref[k][0]) < 1e-4, k
            assert rel(dl.cpu().numpy(), ref[k][1]) < 1e-4, k


def test_set_loop_errors(fw):
    with fw.Solver(configs.c5_autograd(), precision=fw.FP32) as S:
        with pytest.raises(fw.FewhaError) as ei:
            S.set_loop(True)
        assert ei.value.name == "STATE"
    cfg = configs.mcao_small(lgs=False)
    cfg["wfs"][0]["theta_x"] = 90.0 * fo.ARCSEC
    with fw.Solver(cfg, precision=fw.FP32) as S:
        with pytest.raises(fw.FewhaError) as ei:
            S.set_loop(True)
        assert ei.value.name == "GEOMETRY"
        S.set_loop(False)
