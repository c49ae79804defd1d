"""The MAORY-like setting of Sec. 4.1 / Table 2 on the GPU (6 LGS 80x80 + 3 NGS
tip-tilt sensors of 2x2 / 1x1 / 1x1 subapertures, L = M = 6 co-located
mirrors of 81^2 / 48^2 / 54^2 actuators, 4 warm-started iterations, gain 0.5)
against the FP64 oracle: plain FP64 <= 1e-10 and the FP32 fused frame graph
<= 1e-4 on the mirror commands and the layers."""

import numpy as np
import pytest

from _cases import elementwise_check

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
def maory_ref():
    cfg = configs.maory()
    S_in, _ = synth.frames(cfg, N_FR)
    R = fo.Reconstructor(cfg)
    ref = []
    for k in range(N_FR):
        o = R.frame(S_in[k], 4, warm=True, k_rr=10, gain=0.5)
        ref.append((o["a"].copy(), R.layers()))
    return cfg, S_in, ref


def test_maory_fp64_plain_matches_oracle(fw, maory_ref):
    cfg, S_in, ref = maory_ref
    with fw.Solver(cfg, precision=fw.FP64, path=fw.PATH_PLAIN, k_rr=10) as S:
        assert S.NA == 81 ** 2 + 4 * 48 ** 2 + 54 ** 2
        for k in range(6):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            a = S.fit_dm(gain=0.5)
            assert rel(a, ref[k][0]) < 1e-10, k
            assert rel(S.layers(), ref[k][1]) < 1e-10, k


def test_maory_fp32_fused_graph_matches_oracle(fw, maory_ref):
    import torch
    cfg, S_in, ref = maory_ref
    with fw.Solver(cfg, precision=fw.FP32, k_rr=10) as S:
        S.set_path(fw.PATH_FUSED)
        ds = torch.empty(S.S, dtype=torch.float32, device="cuda")
        dl = torch.empty(S.N, dtype=torch.float32, device="cuda")
        da = torch.empty(S.NA, dtype=torch.float32, device="cuda")
        for k in range(N_FR):
            with torch.cuda.stream(S.stream):
                ds.copy_(torch.from_numpy(S_in[k].astype(np.float32)).cuda())
            S.stream.synchronize()
            S.frame(ds, 4, warm=True, gain=0.5, layers_out=dl, dm_out=da)
            S.sync()
            assert rel(da.cpu().numpy(), ref[k][0]) < 1e-4, k
            assert rel(dl.cpu().numpy(), ref[k][1]) < 1e-4, k
            elementwise_check(dl.cpu().numpy(), ref[k][1], [l["n"] for l in cfg["layers"]], 1e-3, what=k)
            elementwise_check(da.cpu().numpy(), ref[k][0], [81, 48, 48, 48, 48, 54], 1e-3, what=("dm", k))
