"""Long-run parity: 200 consecutive frozen-flow frames of the ELT bulk
workload (4 warm-started iterations per frame, 19 residual replacements)
through the fused FP32 frame graph against the FP64 oracle, every frame
within 1e-4 relative L2 and within 1e-3 of the layer's largest value per
element.  FEWHA_LONG_FRAMES sets another frame count (1000 for the full
length of the workload).

What this guards: the warm restart carries c and r from frame to frame, and
the residual replacement every 10 frames recomputes r = b - M c.  In FP32,
b and M c agree to a few per cent, so forming their difference loses the
digits; the library forms it in the slope domain instead (the same vector by
linearity).  On this trajectory frame 83 amplifies any perturbation about
eightfold (the FP64 oracle with only its carried state rounded to FP32 shows
the same jump), so an accuracy loss of that kind fails this test there."""

import os

import pytest

import long_run

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_fused_long_run_matches_oracle_every_frame():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    n = int(os.environ.get("FEWHA_LONG_FRAMES", "200"))
    res = long_run.run(n)
    r = res["per_frame_rel_l2"]
    assert len(r) == n
    assert res["layers_rel_l2_max"] < 1e-4, (res["worst_frame"], res["layers_rel_l2_max"])
    assert res["elementwise_max_over_grid_max"] < 1e-3, res["elementwise_max_over_grid_max"]
    assert res["border_max_over_grid_max"] < 1e-3, res["border_max_over_grid_max"]
