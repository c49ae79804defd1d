"""Batched instances (64 uneven telescopes, 4 warm-started iterations, FP32)
advanced by one fused launch per frame (or one per group of instances),
against the FP64 oracle run instance by instance: layers <= 1e-4 relative L2
for every instance and frame."""

import numpy as np
import pytest

from _cases import elementwise_check

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

pytestmark = pytest.mark.gpu

# a mix of layer grids 32^2 .. 256^2, 2-9 layers, 3-6 sensors, 16-84 subapertures
SUBSET = [1, 6, 2, 7, 24, 56, 8, 10]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


def _oracle_frames(cfgs, n_frames, k_rr=10):
    slopes, layers = [], []
    for cfg in cfgs:
        S_in, _ = synth.frames(cfg, n_frames)
        R = fo.Reconstructor(cfg)
        out = []
        for k in range(n_frames):
            R.frame(S_in[k], cfg["n_iter"], warm=True, k_rr=k_rr)
            out.append(R.layers())
        slopes.append(S_in.astype(np.float32))
        layers.append(out)
    return slopes, layers


@pytest.fixture(scope="module")
def subset_frames():
    cfgs = [configs.c4_instance(i) for i in SUBSET]
    return (cfgs,) + _oracle_frames(cfgs, 12)


def test_batch_subset_frames_match_oracle(fw, subset_frames):
    """Eight uneven instances, 12 frames across the residual replacement of
    frame 10, host buffers through the C ABI."""
    cfgs, slopes, ref = subset_frames
    with fw.Batch(cfgs, k_rr=10) as B:
        assert B.count == len(cfgs)
        out = np.empty(B.N, np.float32)
        for k in range(12):
            B.frame(B.concat_slopes([s[k] for s in slopes]), 4, warm=True, layers_out=out)
            for i, lay in enumerate(B.split_layers(out)):
                assert rel(lay, ref[i][k]) < 1e-4, (SUBSET[i], k)
                elementwise_check(lay, ref[i][k], [l["n"] for l in cfgs[i]["layers"]], 1e-3, what=(SUBSET[i], k))
        assert B.launch_count() == 12


@pytest.mark.parametrize("C", [4, 8, 16])
def test_batch_cluster_shapes_and_tiles(fw, subset_frames, C):
    """Forced cluster shapes and unbounded sensor tiles give the same frames;
    shapes that cannot hold the largest layer stripe are refused at create."""
    cfgs, slopes, ref = subset_frames
    try:
        B = fw.Batch(cfgs, k_rr=10, cluster_size=C, max_tile_side=0 if C == 8 else 24)
    except fw.FewhaError as e:
        assert e.name == "GEOMETRY"
        pytest.skip("no plan with cluster size %d: %s" % (C, e))
    with B:
        assert (" x %d CTAs" % C) in B.describe()
        out = np.empty(B.N, np.float32)
        for k in range(3):
            B.frame(B.concat_slopes([s[k] for s in slopes]), 4, warm=True, layers_out=out)
            for i, lay in enumerate(B.split_layers(out)):
                assert rel(lay, ref[i][k]) < 1e-4, (SUBSET[i], k)


def test_batch_device_buffers_and_state(fw, subset_frames):
    """Device tensors (enqueue only) give bit-identical layers to host
    buffers; per-instance state equals the oracle's coefficients."""
    import torch
    cfgs, slopes, ref = subset_frames
    with fw.Batch(cfgs, k_rr=10) as A, fw.Batch(cfgs, k_rr=10) as B:
        dl = torch.empty(B.N, dtype=torch.float32, device="cuda")
        hl = np.empty(A.N, np.float32)
        for k in range(3):
            s = A.concat_slopes([x[k] for x in slopes])
            A.frame(s, 4, warm=True, layers_out=hl)
            ds = torch.from_numpy(s).cuda()
            torch.cuda.synchronize()
            B.frame(ds, 4, warm=True, layers_out=dl)
            B.sync()
            assert np.array_equal(hl, dl.cpu().numpy()), k
        c, bprev, r = B.get_state(3)
        assert c.size == B.coeff_off[4] - B.coeff_off[3] and np.isfinite(c).all()


def test_batch_autotune_keeps_state_and_parity(fw, subset_frames):
    """The batch autotuner times the groupings by layer size and, per group,
    the feasible cluster shapes and tile bounds on the current frame, keeps
    the fastest and restores the state: the frames that follow still match
    the oracle."""
    cfgs, slopes, ref = subset_frames
    with fw.Batch(cfgs, k_rr=10) as B:
        out = np.empty(B.N, np.float32)
        B.frame(B.concat_slopes([s[0] for s in slopes]), 4, warm=True, layers_out=out)
        report = B.autotune(4, 2)
        # four distinct sides (32 .. 256): all ten ranges of them are tuned
        assert report.startswith("current:") and report.count("; sides ") == 10, report
        assert "sides 32-256 (8 instances): C=" in report, report
        n0 = B.launch_count()
        for k in range(1, 4):
            B.frame(B.concat_slopes([s[k] for s in slopes]), 4, warm=True, layers_out=out)
            for i, lay in enumerate(B.split_layers(out)):
                assert rel(lay, ref[i][k]) < 1e-4, (SUBSET[i], k)
        n_launch = int(B.describe().split(" launch")[0].rsplit(" ", 1)[1])
        assert B.launch_count() - n0 == 3 * n_launch


def test_batch_split_into_launches_by_hand(fw, subset_frames):
    """The instances with 256^2 layers in one launch, the rest in another:
    every instance still matches the oracle over 12 frames (across the
    residual replacement), two launches per frame; bad groupings are refused
    and leave the launches as they were."""
    cfgs, slopes, ref = subset_frames
    side = [max(l["n"] for l in c["layers"]) for c in cfgs]
    group = [0 if n == 256 else 1 for n in side]
    assert 0 < sum(group) < len(group)
    with fw.Batch(cfgs, k_rr=10) as B:
        B.set_groups(group)
        d = B.describe()
        assert "2 launches per frame" in d and "launch 0 (%d instances)" % group.count(0) in d, d
        for bad in ([0] * (B.count - 1), [0] * (B.count - 1) + [2], [0] * (B.count - 1) + [-1]):
            with pytest.raises((fw.FewhaError, ValueError)):
                B.set_groups(bad)
        assert B.describe() == d
        out = np.empty(B.N, np.float32)
        for k in range(12):
            B.frame(B.concat_slopes([s[k] for s in slopes]), 4, warm=True, layers_out=out)
            for i, lay in enumerate(B.split_layers(out)):
                assert rel(lay, ref[i][k]) < 1e-4, (SUBSET[i], k)
                elementwise_check(lay, ref[i][k], [l["n"] for l in cfgs[i]["layers"]], 1e-3, what=(SUBSET[i], k))
        assert B.launch_count() == 24
        B.set_trace(True)
        B.frame(B.concat_slopes([s[0] for s in slopes]), 4, warm=True, layers_out=out)
        B.set_trace(False)
        marks = B.fine_trace()
        # the CTAs of both launches, the first launch's first
        grids = [int(x.split(",")[0]) for x in d.split("(grid ")[1:]]
        assert len(grids) == 2 and len(marks) == sum(grids), (grids, len(marks))
        assert any(len(m) > 0 for m in marks[:grids[0]]) and any(len(m) > 0 for m in marks[grids[0]:])
        t_first = max(t for m in marks[:grids[0]] for _, t in m)
        t_second = min(t for m in marks[grids[0]:] for _, t in m)
        assert t_first <= t_second, "the second launch starts after the first ends"
        # a non-finite slope of an instance that does not lead its launch
        i = next(j for j in range(len(cfgs)) if group[j] == 0 and j != group.index(0))
        g = fo.Geometry(cfgs[i])
        per = [s[1].copy() for s in slopes]
        per[i][g.soff[0] + int(np.flatnonzero(g.mask[0].ravel() == 1)[5])] = np.nan
        with pytest.raises(fw.FewhaError) as ei:
            B.frame(B.concat_slopes(per), 4, warm=False)
        assert ei.value.name == "INPUT"
        # under a bound of one launch the autotuner brings the batch back to one
        # (after a finite frame: the autotuner times the current slopes)
        B.set_max_launches(1)
        B.frame(B.concat_slopes([s[2] for s in slopes]), 4, warm=True, layers_out=out)
        report = B.autotune(4, 1)
        assert "1 launch per frame" in B.describe() and report.count("; sides ") == 1, report
        B.frame(B.concat_slopes([s[3] for s in slopes]), 4, warm=True, layers_out=out)
        assert np.isfinite(out).all()
        B.set_max_launches(0)
        with pytest.raises(fw.FewhaError):
            B.set_max_launches(-1)


def test_batch_nan_in_one_instance_reported(fw, subset_frames):
    cfgs, slopes, ref = subset_frames
    g = fo.Geometry(cfgs[2])
    with fw.Batch(cfgs) as B:
        per = [s[0].copy() for s in slopes]
        active = int(np.flatnonzero(g.mask[1].ravel() == 1)[3])
        per[2][g.soff[1] + active] = np.nan
        with pytest.raises(fw.FewhaError) as ei:
            B.frame(B.concat_slopes(per), 4, warm=False)
        assert ei.value.name == "INPUT"


@pytest.mark.slow
def test_batch_all_64_instances_match_oracle(fw):
    """The whole 64-instance batch in the launch configuration the benchmark
    times (default tiles, then the autotuner's launches): two frames, every
    instance."""
    cfgs = configs.c4_batch(64)
    slopes, ref = _oracle_frames(cfgs, 2)
    with fw.Batch(cfgs, k_rr=10) as B:
        out = np.empty(B.N, np.float32)
        for k in range(2):
            if k == 1:
                B.autotune(4, 1)
            B.frame(B.concat_slopes([s[k] for s in slopes]), 4, warm=True, layers_out=out)
            errs = [rel(lay, ref[i][k]) for i, lay in enumerate(B.split_layers(out))]
            assert max(errs) < 1e-4, (k, int(np.argmax(errs)), max(errs))
            for i, lay in enumerate(B.split_layers(out)):
                elementwise_check(lay, ref[i][k], [l["n"] for l in cfgs[i]["layers"]], 1e-3, what=(i, k))
